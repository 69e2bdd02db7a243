"""Batches of streams (ttals_create_batch / ttals_push_batch).

* Alone vs in a batch: a batch runs the kernels tuned for throughput (rows streamed through
  a pipeline in the environment kernel, fewer k-splits of the solve), a lone stream the ones
  tuned for latency, so the two agree to FP32 summation order, not bitwise.  Checked per
  stream: the first step (same state, same slice: only the order of FP32 sums differs)
  within 1e-4 relative; later steps within 1e-3 relative.  An FP32-order difference alone
  is ~1e-6 here, but the basis Q1 is rounded to the ingest type before the environment pass
  and the state operand of the next local solve is carried in it, so a difference near a
  rounding boundary flips an entry by 2^-11 relative: measured 0.2-3e-5 after one step
  (3e-5 for 16 full-size video streams), growing about 5e-5 per step.  The relative
  reconstruction error (RE, Sec. 5.1) within 1e-3 absolute (the FP16 ingest bar against
  the FP64 oracle).
* In the mix: a stream's results do not depend on its slot or on the other streams' data,
  bit for bit (same batch size, permuted slots, one stream replaced).
"""
import numpy as np
import pytest

from oracle import ttals_oracle as O
from paper_2606_31061_b300 import synth

pytestmark = pytest.mark.gpu

# small shapes (fewer row and column stages than the pipelines hold) and 384 x 384 (more row
# stages than the environment kernel's pipeline: its refill path)
SHAPES = [("video", {"dims": (96, 128, 3)}), ("square", {"s": 128, "r": 16}), ("square", {"s": 192, "r": 40}),
          ("square", {"s": 160, "r": 64}), ("square", {"s": 384, "r": 16})]


def _torch():
    import torch
    from paper_2606_31061_b300 import build
    build.build()
    return torch


def _stream(name, kw, b, T):
    """Stream number b of a shape: dims, ranks, FP16 payloads, initial cores and g."""
    sp = synth.make_stream(name, seed=5000 + 17 * b, **kw)
    r = O.clamp_ranks(sp.dims, sp.ranks)
    c, g = synth.init_cores(sp.dims, r, seed=300 + b)
    return sp.dims, sp.ranks, [synth.round_to_ingest(x, "f16")[0] for x in sp.take(T)], c, g


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


def _run_batch(torch, dims, ranks, streams):
    """streams: list of (frames, cores, g); returns per stream (x^ list, stats list)."""
    from paper_2606_31061_b300.ttals import Stream
    nb, T = len(streams), len(streams[0][0])
    bt = Stream(dims, ranks, ingest="f16", n_streams=nb)
    assert bt.n_streams == nb
    for b, (_, c, g) in enumerate(streams):
        bt.select(b)
        bt.set_cores(c, g)
    out = torch.empty(tuple(dims), dtype=torch.float64, device="cuda")
    res = [([], []) for _ in range(nb)]
    for t in range(T):
        batch = torch.from_numpy(np.stack([s[0][t] for s in streams])).view(torch.float16).cuda()
        bt.push_batch(batch)
        for b in range(nb):
            bt.select(b)
            bt.reconstruct(out, "f64")
            res[b][0].append(out.cpu().numpy().copy())
            res[b][1].append(np.array(bt.stats()))
    bt.close()
    return res


@pytest.mark.parametrize("name,kw", SHAPES)
def test_batch_matches_alone(name, kw):
    torch = _torch()
    nb, T = 3, 5
    ss = [_stream(name, kw, b, T) for b in range(nb)]
    dims, ranks = ss[0][0], ss[0][1]
    batch = _run_batch(torch, dims, ranks, [(s[2], s[3], s[4]) for s in ss])
    worst = []
    for b, s in enumerate(ss):
        xa, sa = _run_alone(torch, dims, ranks, s[2], s[3], s[4])
        xb, sb = batch[b]
        for t in range(T):
            rel = np.linalg.norm(xb[t] - xa[t]) / max(np.linalg.norm(xa[t]), 1e-300)
            worst.append((t, rel))
            assert rel <= (1e-4 if t == 0 else 1e-3), (name, b, t, rel)
        re_a = np.sqrt(sa[-1][3] / sa[-1][2])
        re_b = np.sqrt(sb[-1][3] / sb[-1][2])
        assert abs(re_a - re_b) <= 1e-3, (name, b, re_a, re_b)
    print(f"batch vs alone {name} {kw}: max rel per step", [max(r for t, r in worst if t == u) for u in range(T)])


def test_batch_full_size_video():
    """Two 1080 x 1920 x 3 video streams: both pipelines run their refill paths."""
    torch = _torch()
    nb, T = 2, 3
    ss = [_stream("video", {}, b, T) for b in range(nb)]
    dims, ranks = ss[0][0], ss[0][1]
    batch = _run_batch(torch, dims, ranks, [(s[2], s[3], s[4]) for s in ss])
    for b, s in enumerate(ss):
        xa, sa = _run_alone(torch, dims, ranks, s[2], s[3], s[4])
        for t in range(T):
            rel = np.linalg.norm(batch[b][0][t] - xa[t]) / np.linalg.norm(xa[t])
            assert rel <= (1e-4 if t == 0 else 1e-3), (b, t, rel)


@pytest.mark.parametrize("name,kw", SHAPES[:2])
def test_batch_slot_and_neighbours_bitwise(name, kw):
    torch = _torch()
    T = 4
    s0, s1, s2, s3 = (_stream(name, kw, b, T) for b in range(4))
    dims, ranks = s0[0], s0[1]
    A = _run_batch(torch, dims, ranks, [(s[2], s[3], s[4]) for s in (s0, s1, s2)])
    B = _run_batch(torch, dims, ranks, [(s[2], s[3], s[4]) for s in (s3, s0, s1)])
    for a, b in ((0, 1), (1, 2)):
        for t in range(T):
            assert np.array_equal(A[a][0][t], B[b][0][t]), (name, a, t)
            assert np.array_equal(A[a][1][t], B[b][1][t]), (name, a, t)


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


def test_batch_tcgen05_solve_matches_alone(monkeypatch):
    """The tcgen05 local solve (forced for a small batch through TTALS_SOLVE_KERNEL, read when
    a stream is created) against the same streams alone on the mma.sync kernel."""
    torch = _torch()
    monkeypatch.setenv("TTALS_SOLVE_KERNEL", "tc")
    for name, kw in (("video", {"dims": (96, 128, 3)}), ("square", {"s": 384, "r": 16}), ("square", {"s": 160, "r": 64})):
        ss = [_stream(name, kw, b, 4) for b in range(3)]
        dims, ranks = ss[0][0], ss[0][1]
        batch = _run_batch(torch, dims, ranks, [(s[2], s[3], s[4]) for s in ss])
        monkeypatch.setenv("TTALS_SOLVE_KERNEL", "mma")
        for b, s in enumerate(ss):
            xa, sa = _run_alone(torch, dims, ranks, s[2], s[3], s[4])
            for t in range(4):
                rel = np.linalg.norm(batch[b][0][t] - xa[t]) / np.linalg.norm(xa[t])
                assert rel <= (1e-4 if t == 0 else 1e-3), (name, b, t, rel)
        monkeypatch.setenv("TTALS_SOLVE_KERNEL", "tc")


def test_batch_16_video_streams_full_size():
    """16 full-size video streams: the batch takes the tcgen05 solve on its own (its row tiles
    cover the SMs).  Streams share two frame sequences but start from different cores."""
    torch = _torch()
    T = 3
    seqs = [_stream("video", {}, b, T) for b in range(2)]
    dims, ranks = seqs[0][0], seqs[0][1]
    streams = []
    for b in range(16):
        sq = seqs[b % 2]
        c, g = synth.init_cores(dims, O.clamp_ranks(dims, ranks), seed=900 + b)
        streams.append((sq[2], c, g))
    batch = _run_batch(torch, dims, ranks, streams)
    for b in (0, 1, 7, 15):
        xa, sa = _run_alone(torch, dims, ranks, *streams[b])
        for t in range(T):
            rel = np.linalg.norm(batch[b][0][t] - xa[t]) / np.linalg.norm(xa[t])
            assert rel <= (1e-4 if t == 0 else 1e-3), (b, t, rel)


@pytest.mark.parametrize("sched", [{"solve_kernel": 2, "factor_cluster": 4},
                                   {"solve_kernel": 1, "k1_split": 1, "factor_cluster": 8},
                                   {"solve_kernel": 1, "k1_split": 2, "factor_cluster": 8},
                                   {"solve_kernel": 1, "k1_split": 4, "factor_cluster": 4},
                                   {"env_kernel": 3, "solve_kernel": 2, "factor_cluster": 4},
                                   {"env_kernel": 4, "solve_kernel": 1, "k1_split": 8, "factor_cluster": 4}])
def test_batch_schedules_agree(sched):
    """Every tile-shape schedule the autotuner may pick (solve kernel and split, environment
    kernel, factor cluster) computes the same update as the library's default schedule:
    only FP32 summation orders differ (first step within 1e-4, later ones within 1e-3)."""
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream
    nb, T = 3, 4
    ss = [_stream("video", {"dims": (96, 128, 3)}, b, T) for b in range(nb)]
    dims, ranks = ss[0][0], ss[0][1]
    base = _run_batch(torch, dims, ranks, [(s[2], s[3], s[4]) for s in ss])
    bt = Stream(dims, ranks, ingest="f16", n_streams=nb, **sched)
    for b, s in enumerate(ss):
        bt.select(b)
        bt.set_cores(s[3], s[4])
    out = torch.empty(tuple(dims), dtype=torch.float64, device="cuda")
    for t in range(T):
        bt.push_batch(torch.from_numpy(np.stack([s[2][t] for s in ss])).view(torch.float16).cuda())
        for b in range(nb):
            bt.select(b)
            bt.reconstruct(out, "f64")
            x = out.cpu().numpy()
            rel = np.linalg.norm(x - base[b][0][t]) / np.linalg.norm(base[b][0][t])
            assert rel <= (1e-4 if t == 0 else 1e-3), (sched, b, t, rel)
    bt.close()
