"""Allocation-free slice error (ttals_slice_error_noalloc) against the stream's own
per-slice statistics (ttals_stats after ttals_push_slice), two calls in a row.

Collected last on purpose: it must pass both in a fresh process and after every
other test has used the library on the same device.
"""
import numpy as np
import pytest

from oracle import ttals_oracle as O
from paper_2606_31061_b300 import synth

pytestmark = pytest.mark.gpu


def _setup(name, ingest, **kw):
    import torch
    from paper_2606_31061_b300 import build
    build.build()
    from paper_2606_31061_b300.ttals import Stream
    sp = synth.make_stream(name, **kw)
    r = O.clamp_ranks(sp.dims, sp.ranks)
    cores, g = synth.init_cores(sp.dims, r, seed=7)
    st = Stream(sp.dims, sp.ranks, ingest=ingest)
    st.set_cores(cores, g)
    torch.cuda.synchronize()
    return sp, st


def test_noalloc_matches_stats_f64():
    import torch
    from paper_2606_31061_b300 import ttals
    sp, st = _setup("plain", "f64")
    xhat = torch.empty(sp.dims, dtype=torch.float64, device="cuda")
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    for x in sp.take(2):                       # two calls in a row on the same scratch
        xd = torch.from_numpy(x).cuda()
        st.push(xd)
        st.reconstruct(xhat, "f64")
        ttals.slice_error_noalloc(xd, xhat, res)
        xx, ee = st.stats()[:2]
        got = res.cpu().numpy()
        # ||x||^2: the same FP64 data summed in another order
        assert abs(got[0] - xx) <= 1e-12 * xx, (got[0], xx)
        # ||x - x^||^2 directly vs ||x||^2 - ||P x||^2 (cancellation ~1e-16 xx / ee)
        assert abs(got[1] - ee) <= 1e-8 * ee + 1e-13 * xx, (got[1], ee)
    st.close()


def test_noalloc_matches_stats_f16_video():
    import torch
    from paper_2606_31061_b300 import ttals
    sp, st = _setup("video", "f16", dims=(96, 128, 3))
    xhat = torch.empty(sp.dims, dtype=torch.float64, device="cuda")
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    for x in sp.take(2):
        payload, exact = synth.round_to_ingest(x, "f16")
        xd = torch.from_numpy(payload).view(torch.float16).cuda()
        st.push(xd)
        st.reconstruct(xhat, "f64")
        ttals.slice_error_noalloc(xd, xhat, res)
        xx, ee = st.stats()[:2]
        got = res.cpu().numpy()
        assert abs(got[0] - xx) <= 1e-6 * xx, (got[0], xx)
        # per-slice relative error within the FP16 stream tolerance
        assert abs(np.sqrt(got[1] / got[0]) - np.sqrt(ee / xx)) <= 1e-3, (got, xx, ee)
    st.close()


def test_noalloc_deterministic_and_limit():
    import torch
    from paper_2606_31061_b300 import ttals
    torch.manual_seed(3)
    n = 3 * 16384 + 77                          # several CTAs and a ragged tail
    x = torch.randn(n, dtype=torch.float32, device="cuda")
    y = torch.randn(n, dtype=torch.float64, device="cuda")
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    b = torch.zeros(2, dtype=torch.float64, device="cuda")
    ttals.slice_error_noalloc(x, y, a)
    ttals.slice_error_noalloc(x, y, b)
    assert torch.equal(a, b)
    xd, yd = x.double().cpu().numpy(), y.cpu().numpy()
    ref = np.array([np.sum(xd * xd), np.sum((xd - yd) ** 2)])
    assert np.allclose(a.cpu().numpy(), ref, rtol=1e-12)
    with pytest.raises(ttals.TTALSError) as ei:
        ttals.slice_error_noalloc_ptr(x.data_ptr(), "f32", y.data_ptr(), "f64", (1 << 26) + 1, a.data_ptr())
    assert ei.value.code == 1 and "static scratch limit" in str(ei.value)
