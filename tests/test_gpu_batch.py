"""Batches of streams (ttals_create_batch / ttals_push_batch): every stream of a batch must
give the same results as the same stream run alone, bit for bit (the same kernels and the
same reduction orders; a batch only adds a stream index to each launch's grid)."""
import numpy as np
import pytest

from oracle import ttals_oracle as O
from paper_2606_31061_b300 import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    from paper_2606_31061_b300 import build
    build.build()
    return torch


def _streams(name, nb, T, **kw):
    """nb independent streams of one shape: dims, ranks, FP16 payloads [b][t], cores[b], g[b]."""
    frames, cores, gs = [], [], []
    for b in range(nb):
        sp = synth.make_stream(name, seed=5000 + 17 * b, **kw)
        r = O.clamp_ranks(sp.dims, sp.ranks)
        c, g = synth.init_cores(sp.dims, r, seed=300 + b)
        frames.append([synth.round_to_ingest(x, "f16")[0] for x in sp.take(T)])
        cores.append(c)
        gs.append(g)
    return sp.dims, sp.ranks, frames, cores, gs


def _run_alone(torch, dims, ranks, frames, cores, g):
    from paper_2606_31061_b300.ttals import Stream
    st = Stream(dims, ranks, ingest="f16")
    st.set_cores(cores, g)
    out = torch.empty(tuple(dims), dtype=torch.float64, device="cuda")
    xs, stats = [], []
    for x in frames:
        st.push(torch.from_numpy(x).view(torch.float16).cuda())
        st.reconstruct(out, "f64")
        xs.append(out.cpu().numpy().copy())
        stats.append(np.array(st.stats()))
    st.close()
    return xs, stats


# video-shaped (env kernel: one CTA per column tile) and square r = 40 (rank padded to 48:
# the clustered env kernel)
@pytest.mark.parametrize("name,kw", [("video", {"dims": (96, 128, 3)}), ("square", {"s": 128, "r": 16}),
                                     ("square", {"s": 192, "r": 40})])
def test_batch_equals_alone_bitwise(name, kw):
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream
    nb, T = 3, 4
    dims, ranks, frames, cores, gs = _streams(name, nb, T, **kw)
    alone = [_run_alone(torch, dims, ranks, frames[b], cores[b], gs[b]) for b in range(nb)]
    bt = Stream(dims, ranks, ingest="f16", n_streams=nb)
    assert bt.n_streams == nb
    for b in range(nb):
        bt.select(b)
        bt.set_cores(cores[b], gs[b])
    out = torch.empty(tuple(dims), dtype=torch.float64, device="cuda")
    for t in range(T):
        batch = torch.from_numpy(np.stack([frames[b][t] for b in range(nb)])).view(torch.float16).cuda()
        bt.push_batch(batch)
        for b in range(nb):
            bt.select(b)
            bt.reconstruct(out, "f64")
            x = out.cpu().numpy()
            assert np.array_equal(x, alone[b][0][t]), (name, b, t, float(np.abs(x - alone[b][0][t]).max()))
            assert np.array_equal(np.array(bt.stats()), alone[b][1][t]), (name, b, t)
    bt.close()


def test_batch_argument_errors():
    torch = _torch()
    from paper_2606_31061_b300 import ttals
    from paper_2606_31061_b300.ttals import Stream
    # a shape that does not take the fused path (FP64 ingest) cannot form a batch
    with pytest.raises(ttals.TTALSError) as ei:
        Stream((32, 32), (8, 8), ingest="f64", n_streams=2)
    assert ei.value.code == 1
    bt = Stream((96, 128, 3), (32, 9, 3), ingest="f16", n_streams=2)
    x = torch.zeros((2, 96, 128, 3), dtype=torch.float16, device="cuda")
    with pytest.raises(ttals.TTALSError) as ei:
        bt.push(x[0])                               # single-slice push on a batch
    assert ei.value.code == 6
    with pytest.raises(ttals.TTALSError) as ei:
        bt.select(2)
    assert ei.value.code == 1
    bt.push_batch(x)
    bt.sync()
    bt.close()
