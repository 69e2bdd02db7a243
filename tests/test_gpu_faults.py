"""Failure handling on the GPU, without faulting it.

* A slice with a NaN on the fused FP16 path, and a NaN in one stream of a batch: that step
  (that stream) is not committed, ENONFINITE is latched for it alone, and the other streams
  of the batch step exactly as they would without it.
* A bounded device wait made to run out (ttals_debug_stall_solve: the local solve issues no
  copy, so its first wait has nothing to wait for): ETIMEOUT surfaces at the next sync, the
  step is not committed and the stream carries on, bitwise as if the slice had been skipped.
* An allocation the device cannot hold: ttals_create returns ENOMEM and the context stays
  usable.
"""
import numpy as np
import pytest

from oracle import ttals_oracle as O
from paper_2606_31061_b300 import synth

pytestmark = pytest.mark.gpu

DIMS = (96, 128, 3)


def _torch():
    import torch
    from paper_2606_31061_b300 import build
    build.build()
    return torch


def _frames(torch, seed, T):
    sp = synth.make_stream("video", dims=DIMS, seed=seed)
    return [torch.from_numpy(synth.round_to_ingest(x, "f16")[0]).view(torch.float16).cuda() for x in sp.take(T)]


def _fresh(ranks, seed):
    from paper_2606_31061_b300.ttals import Stream
    st = Stream(DIMS, ranks, ingest="f16")
    c, g = synth.init_cores(DIMS, O.clamp_ranks(DIMS, ranks), seed=seed)
    st.set_cores(c, g)
    return st


def _snap(torch, st):
    out = torch.empty(DIMS, dtype=torch.float64, device="cuda")
    st.reconstruct(out, "f64")
    return out.cpu().numpy().copy(), np.array(st.stats()), st.step()


def test_nonfinite_slice_fused_f16_not_committed():
    torch = _torch()
    from paper_2606_31061_b300.ttals import TTALSError
    fr = _frames(torch, 41, 6)
    a, ref = _fresh((32, 9, 3), 5), _fresh((32, 9, 3), 5)
    for f in fr[:3]:
        a.push(f)
        ref.push(f)
    before = _snap(torch, a)
    bad = fr[3].clone()
    bad[7, 11, 2] = float("nan")
    a.push(bad)
    with pytest.raises(TTALSError) as ei:
        a.sync()
    assert ei.value.name == "ENONFINITE"
    after = _snap(torch, a)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert after[2] == 3
    for f in fr[4:]:                       # the stream carries on as if the slice was skipped
        a.push(f)
        ref.push(f)
    sa, sr = _snap(torch, a), _snap(torch, ref)
    assert np.array_equal(sa[0], sr[0]) and np.array_equal(sa[1], sr[1]) and sa[2] == sr[2] == 5


def test_nonfinite_in_one_stream_of_a_batch():
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream, TTALSError
    ranks = (32, 9, 3)
    seqs = [_frames(torch, 60 + b, 4) for b in range(3)]
    inits = [synth.init_cores(DIMS, O.clamp_ranks(DIMS, ranks), seed=70 + b) for b in range(3)]

    def make():
        bt = Stream(DIMS, ranks, ingest="f16", n_streams=3)
        for b in range(3):
            bt.select(b)
            bt.set_cores(*inits[b])
        return bt

    A, B = make(), make()
    for t in range(2):
        x = torch.stack([seqs[b][t] for b in range(3)])
        A.push_batch(x)
        B.push_batch(x)
    A.select(1)
    before1 = _snap(torch, A)
    x = torch.stack([seqs[b][2] for b in range(3)])
    xbad = x.clone()
    xbad[1, 50, 3, 1] = float("inf")
    A.push_batch(xbad)
    B.push_batch(x)
    A.select(1)
    with pytest.raises(TTALSError) as ei:
        A.sync()
    assert ei.value.name == "ENONFINITE"
    after1 = _snap(torch, A)
    assert np.array_equal(before1[0], after1[0]) and after1[2] == 2
    for b in (0, 2):                       # the neighbours stepped exactly as without the bad slice
        A.select(b)
        A.sync()
        B.select(b)
        sa, sb = _snap(torch, A), _snap(torch, B)
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1]) and sa[2] == sb[2] == 3
    A.push_batch(torch.stack([seqs[b][3] for b in range(3)]))
    A.select(1)
    A.sync()
    assert A.step() == 3


def test_solve_wait_timeout_surfaces_and_stream_recovers():
    torch = _torch()
    from paper_2606_31061_b300.ttals import TTALSError
    fr = _frames(torch, 43, 6)
    a, ref = _fresh((32, 9, 3), 9), _fresh((32, 9, 3), 9)
    for f in fr[:2]:
        a.push(f)
        ref.push(f)
    before = _snap(torch, a)
    a.debug_stall_solve(1)
    a.push(fr[2])                          # its local solve's first wait runs out
    with pytest.raises(TTALSError) as ei:
        a.sync()
    assert ei.value.name == "ETIMEOUT"
    after = _snap(torch, a)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1]) and after[2] == 2
    for f in fr[3:]:
        a.push(f)
        ref.push(f)
    a.sync()                               # no error latched by the later steps
    sa, sr = _snap(torch, a), _snap(torch, ref)
    assert np.array_equal(sa[0], sr[0]) and np.array_equal(sa[1], sr[1]) and sa[2] == sr[2] == 5
    assert float(torch.ones(4, device="cuda").sum()) == 4.0   # the context is still usable


def test_create_beyond_device_memory_is_enomem():
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream, TTALSError
    # a 2^36 x 2 FP64 stream: its first core alone is 1 TiB, far beyond the device
    with pytest.raises(TTALSError) as ei:
        Stream((1 << 36, 2), (2, 2), ingest="f64")
    assert ei.value.name == "ENOMEM"
    st = Stream((16, 16), (4, 4), ingest="f64")
    st.push(torch.ones((16, 16), dtype=torch.float64, device="cuda"))
    st.sync()
    assert st.step() == 1
