"""Groups of streams of uneven shapes (paper_2606_31061_b300.group) and masked batch steps.

* A masked step leaves the inactive streams exactly as they were, and a stream's results
  depend only on the slices it was given (bitwise, against a batch that fed it the same
  slices at other steps).
* Every stream of a mixed-shape group, with the autotuner's schedules, agrees with the same
  stream alone within the FP16 ingest tolerance (RE within 1e-3 absolute, each reconstructed
  slice within 1e-3 relative; the first step within 1e-4, see test_gpu_batch).
* Replaying a captured CUDA graph of two steps gives bitwise the steps run eagerly.
"""
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


def _frames(name, kw, seed, T):
    sp = synth.make_stream(name, seed=seed, **kw)
    r = O.clamp_ranks(sp.dims, sp.ranks)
    c, g = synth.init_cores(sp.dims, r, seed=seed % 997)
    return sp.dims, sp.ranks, [synth.round_to_ingest(x, "f16")[0] for x in sp.take(T)], c, g


def _state(torch, st, dims):
    out = torch.empty(tuple(dims), dtype=torch.float64, device="cuda")
    st.reconstruct(out, "f64")
    return out.cpu().numpy().copy(), np.array(st.stats()), st.step()


def test_masked_push_bitwise():
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream
    kw = {"dims": (96, 128, 3)}
    ss = [_frames("video", kw, 7000 + 13 * b, 3) for b in range(3)]
    dims, ranks = ss[0][0], ss[0][1]
    f = [[torch.from_numpy(x).view(torch.float16).cuda() for x in s[2]] for s in ss]

    def make():
        bt = Stream(dims, ranks, ingest="f16", n_streams=3)
        for b in range(3):
            bt.select(b)
            bt.set_cores(ss[b][3], ss[b][4])
        return bt

    # A: step 0 all, step 1 streams {0, 2}, step 2 all (stream 1 sees f0, then f2)
    A = make()
    A.push_batch(torch.stack([f[0][0], f[1][0], f[2][0]]))
    A.select(1)
    before = _state(torch, A, dims)
    A.push_batch(torch.stack([f[0][1], f[1][1], f[2][1]]), active=0b101)
    A.select(1)
    after = _state(torch, A, dims)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert before[2] == after[2] == 1
    A.push_batch(torch.stack([f[0][2], f[1][2], f[2][2]]))
    # C: step 0 all, step 1 all with stream 1 given f2, step 2 streams {0, 2}: every stream
    # sees the same slices as in A, stream 1 at other steps
    C = make()
    C.push_batch(torch.stack([f[0][0], f[1][0], f[2][0]]))
    C.push_batch(torch.stack([f[0][1], f[1][2], f[2][1]]))
    C.push_batch(torch.stack([f[0][2], f[1][2], f[2][2]]), active=0b101)
    for b, steps in ((0, 3), (1, 2), (2, 3)):
        A.select(b)
        C.select(b)
        xa, sa, ta = _state(torch, A, dims)
        xc, sc, tc = _state(torch, C, dims)
        assert ta == tc == steps, b
        assert np.array_equal(xa, xc) and np.array_equal(sa, sc), b
    # an all-zero mask enqueues nothing
    A.push_batch(torch.stack([f[0][0], f[1][0], f[2][0]]), active=0)
    A.select(0)
    assert A.step() == 3
    for s in (A, C):
        s.close()


def _c4_specs():
    # two sides x two ranks, some shapes repeated: four batches of 1..3 streams
    return [(128, 8), (256, 16), (128, 8), (256, 8), (128, 16), (256, 16), (128, 8)]


def test_group_mixed_shapes_match_alone():
    torch = _torch()
    from paper_2606_31061_b300.group import Group
    from paper_2606_31061_b300.ttals import Stream
    T = 4
    streams = [_frames("square", {"s": s, "r": r}, 9000 + 31 * i, T) for i, (s, r) in enumerate(_c4_specs())]
    grp = Group([(st[0], st[1]) for st in streams], depth=2, tune=True, tune_steps=3)
    assert len(grp.buckets) == 4 and grp.launches_per_step == 12
    for i, st in enumerate(streams):
        grp.set_cores(i, st[3], st[4])
    xs = {i: [] for i in range(len(streams))}
    for t in range(T):
        for i, st in enumerate(streams):
            grp.slot(i, t % 2).copy_(torch.from_numpy(st[2][t]).view(torch.float16))
        grp.step(t % 2)
        for i, st in enumerate(streams):
            out = torch.empty(tuple(st[0]), dtype=torch.float64, device="cuda")
            grp.reconstruct(i, out)
            xs[i].append(out.cpu().numpy().copy())
    for i, st in enumerate(streams):
        alone = Stream(st[0], st[1], ingest="f16")
        alone.set_cores(st[3], st[4])
        out = torch.empty(tuple(st[0]), dtype=torch.float64, device="cuda")
        for t in range(T):
            alone.push(torch.from_numpy(st[2][t]).view(torch.float16).cuda())
            alone.reconstruct(out, "f64")
            xa = out.cpu().numpy()
            rel = np.linalg.norm(xs[i][t] - xa) / np.linalg.norm(xa)
            assert rel <= (1e-4 if t == 0 else 1e-3), (i, t, rel)
        sa, sg = np.array(alone.stats()), grp.stats(i)
        assert abs(np.sqrt(sa[3] / sa[2]) - np.sqrt(sg[3] / sg[2])) <= 1e-3
        assert grp.step_count(i) == T
        alone.close()
    grp.close()


def test_group_graph_replay_matches_eager():
    torch = _torch()
    from paper_2606_31061_b300.group import Group
    specs = _c4_specs()[:4]
    streams = [_frames("square", {"s": s, "r": r}, 9100 + 7 * i, 2) for i, (s, r) in enumerate(specs)]
    cs = torch.cuda.Stream()
    groups = []
    for _ in range(2):
        grp = Group([(st[0], st[1]) for st in streams], depth=2, tune=False)
        for i, st in enumerate(streams):
            grp.set_cores(i, st[3], st[4])
            for p in range(2):
                grp.slot(i, p).copy_(torch.from_numpy(st[2][p]).view(torch.float16))
        groups.append(grp)
    eager, graphed = groups
    torch.cuda.synchronize()
    for _ in range(3):                       # 6 steps: positions 0, 1, 0, 1, 0, 1
        eager.step(0, stream=cs)
        eager.step(1, stream=cs)
    graphed.step(0, stream=cs)               # the captured steps then run 3..6 ...
    graphed.step(1, stream=cs)               # ... after two eager ones
    graphed.capture([0, 1], cs)
    graphed.replay()
    graphed.replay()
    torch.cuda.synchronize()
    for i, st in enumerate(streams):
        out_e = torch.empty(tuple(st[0]), dtype=torch.float64, device="cuda")
        out_g = torch.empty_like(out_e)
        eager.reconstruct(i, out_e)
        graphed.reconstruct(i, out_g)
        torch.cuda.synchronize()
        assert torch.equal(out_e, out_g), i
        assert np.array_equal(eager.stats(i), graphed.stats(i)), i
        assert graphed.step_count(i) == 6
    for g in groups:
        g.close()
