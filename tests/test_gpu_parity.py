"""GPU path vs the FP64 oracle, element by element on the same seeded inputs.

Tolerances (per reconstructed slice x^_t, relative ||x^_gpu - x^_orc|| / ||x^_orc||):
  FP64 ingest <= 1e-10, FP32 ingest <= 1e-5; FP16 / BF16 ingest: the stream's relative
  reconstruction error (RE, Sec. 5.1) within 1e-3 absolute of the oracle's.
The oracle ingests exactly the values the GPU ingests (the rounded slice widened to FP64).

FP32 floor probe: at steps where the tracked subspace is poorly determined (the first
step from random cores, the step after an abrupt change) x^_t is sensitive to FP32-level
perturbations of the data itself.  The oracle is rerun on inputs and initial cores
perturbed by relative 2^-24 noise; the per-step FP32 tolerance is max(1e-5, 10 x the
oracle's own movement).  Steady-state steps are held to 1e-5 regardless (asserted on the
median).
"""
import math

import numpy as np
import pytest

from oracle import ttals_oracle as O
from paper_2606_31061_b300 import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-5}
TORCH_DT = {}


def _torch():
    import torch
    if not TORCH_DT:
        TORCH_DT.update(f64=torch.float64, f32=torch.float32, f16=torch.float16, bf16=torch.bfloat16)
    return torch


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2606_31061_b300 import build
    build.build()


def _upload(x64, ingest):
    torch = _torch()
    payload, exact = synth.round_to_ingest(x64, ingest)
    t = torch.from_numpy(np.ascontiguousarray(payload))
    if ingest in ("f16", "bf16"):
        t = t.view(TORCH_DT[ingest])
    return t.cuda(), exact


FLOOR = {}


def run_pair(dims, ranks, frames, ingest, init_seed=7, qr_passes=0):
    """Run the GPU stream and the oracle on the same rounded frames.  Returns
    (gpu x^ list, oracle x^ list, exact inputs, gpu stream).  For FP32 ingest the
    oracle's FP32 floor (see the module docstring) is left in FLOOR["last"]."""
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream
    r = O.clamp_ranks(dims, ranks)
    cores, g = synth.init_cores(dims, r, seed=init_seed)
    st = Stream(dims, ranks, ingest=ingest, qr_passes=qr_passes)
    assert list(st.ranks) == r
    st.set_cores(cores, g)
    orc = O.OnlineTTALS(dims, r, cores, g)
    out = torch.empty(tuple(dims), dtype=torch.float64, device="cuda")
    xg, xo, ex = [], [], []
    for x in frames:
        dx, exact = _upload(x, ingest)
        st.push(dx)
        st.reconstruct(out, "f64")
        torch.cuda.synchronize()
        xg.append(out.cpu().numpy().copy())
        xo.append(orc.step(exact))
        ex.append(exact)
    st.sync()
    if ingest == "f32":
        rng = np.random.default_rng(12345)
        pert = lambda a: a * (1.0 + rng.uniform(-1, 1, np.shape(a)) * 2.0 ** -24)
        orp = O.OnlineTTALS(dims, r, [pert(c) for c in cores], pert(g))
        FLOOR["last"] = [rel(orp.step(pert(x)), y) for x, y in zip(ex, xo)]
    return xg, xo, ex, st


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def check(xg, xo, ex, ingest):
    if ingest == "f64":
        errs = [rel(a, b) for a, b in zip(xg, xo)]
        assert max(errs) <= TOL[ingest], f"max per-slice rel err {max(errs):.3e}"
    elif ingest == "f32":
        errs = [rel(a, b) for a, b in zip(xg, xo)]
        floor = FLOOR["last"]
        for t, (e, f) in enumerate(zip(errs, floor)):
            assert e <= max(TOL["f32"], 10.0 * f), f"step {t + 1}: rel err {e:.3e}, FP32 floor {f:.3e}"
        assert float(np.median(errs)) <= TOL["f32"]
    else:
        re_g = O.stream_relative_error(ex, xg)
        re_o = O.stream_relative_error(ex, xo)
        assert abs(re_g - re_o) <= 1e-3, (re_g, re_o)


# ----------------------------------------------------------------------------- configs
def test_plain_fp64_full_stream():
    """3rd-order 32x32 stream, ranks (8,8), T = 100, FP64 ingest."""
    sp = synth.make_stream("plain")
    xg, xo, ex, st = run_pair(sp.dims, sp.ranks, sp.take(100), "f64")
    check(xg, xo, ex, "f64")
    assert st.step() == 100


@pytest.mark.parametrize("ingest", ["f32", "f16"])
def test_video_small(ingest):
    sp = synth.make_stream("video", dims=(120, 160, 3), T=24)
    xg, xo, ex, st = run_pair(sp.dims, sp.ranks, sp.take(24), ingest)
    check(xg, xo, ex, ingest)


@pytest.mark.parametrize("ingest", ["f32", "bf16"])
def test_sensor_with_abrupt_change(ingest):
    """5th-order 32^4 stream, ranks (16,32,32,16): the saturated level is k* = 3."""
    sp = synth.make_stream("sensor", change_every=15)
    xg, xo, ex, st = run_pair(sp.dims, sp.ranks, sp.take(30), ingest)
    check(xg, xo, ex, ingest)


# (192, 40): rank padded to 48, which takes the clustered environment kernel; the others take
# the single-CTA-per-tile one
@pytest.mark.parametrize("s,r", [(128, 8), (256, 16), (160, 64), (192, 40)])
def test_square_fp16(s, r):
    sp = synth.make_stream("square", s=s, r=r)
    xg, xo, ex, st = run_pair(sp.dims, sp.ranks, sp.take(12), "f16")
    check(xg, xo, ex, "f16")


@pytest.mark.parametrize("ingest", ["f64", "f32"])
@pytest.mark.parametrize("dims,ranks", [((37, 53), (5, 5)), ((129, 65), (7, 7)), ((33, 17, 5), (6, 9, 2)),
                                        ((7, 5, 4, 3), (3, 4, 3, 2))])
def test_ragged_shapes(dims, ranks, ingest):
    """Sizes that are not multiples of any tile, several orders and saturation levels."""
    rng = np.random.default_rng(sum(dims))
    u = np.linalg.qr(rng.standard_normal((dims[0], ranks[0])))[0]
    frames = []
    base = rng.standard_normal((ranks[0],) + tuple(dims[1:]))
    for t in range(10):
        base = 0.9 * base + 0.3 * rng.standard_normal(base.shape)
        frames.append(np.tensordot(u, base, axes=([1], [0])) + 0.01 * rng.standard_normal(dims))
    xg, xo, ex, st = run_pair(dims, ranks, frames, ingest)
    check(xg, xo, ex, ingest)


@pytest.mark.parametrize("ingest", ["f64", "f32"])
@pytest.mark.parametrize("dims,ranks", [((5, 5, 5, 5, 5), (4, 4, 4, 4, 4)), ((4, 4, 4, 4, 4, 4), (3, 3, 3, 3, 3, 3))])
def test_high_order_shapes(dims, ranks, ingest):
    """Orders n = 6 and 7 (the Table-1 orders) at small mode sizes: a drifting low-rank TT."""
    sp = synth.make_stream("plain", dims=dims, ranks=ranks, gen_ranks=ranks, seed=659 + len(dims))
    xg, xo, ex, st = run_pair(dims, ranks, sp.take(8), ingest)
    check(xg, xo, ex, ingest)


def test_video_full_size_prefix():
    """The 1080x1920x3 video stream at full size, FP32 and FP16 ingest, first frames."""
    sp = synth.make_stream("video")
    frames = sp.take(5)
    for ingest in ("f32", "f16"):
        xg, xo, ex, st = run_pair(sp.dims, sp.ranks, frames, ingest)
        check(xg, xo, ex, ingest)


# ----------------------------------------------------------------------------- edge cases
def test_rank_one_and_saturated_first_level():
    for dims, ranks in (((16, 12), (1, 1)), ((6, 4), (9, 9)), ((3, 2, 2), (6, 4, 2))):
        rng = np.random.default_rng(3)
        frames = [rng.standard_normal(dims) for _ in range(5)]
        xg, xo, ex, st = run_pair(dims, ranks, frames, "f64")
        check(xg, xo, ex, "f64")


def test_zero_slice_then_recovery():
    """A zero slice reconstructs to exactly zero; later slices are finite, orthonormal and
    back to the tracking error of the oracle's stream (the completion after a zero slice
    is implementation-specific, so only these properties are compared)."""
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream
    sp = synth.make_stream("plain")
    xs = sp.take(40)
    r = O.clamp_ranks(sp.dims, sp.ranks)
    cores, g = synth.init_cores(sp.dims, r, seed=7)
    st = Stream(sp.dims, sp.ranks, ingest="f64")
    st.set_cores(cores, g)
    out = torch.empty(sp.dims, dtype=torch.float64, device="cuda")
    for x in xs[:10]:
        st.push(torch.from_numpy(x).cuda())
    st.push(torch.zeros(sp.dims, dtype=torch.float64, device="cuda"))
    st.reconstruct(out, "f64")
    assert torch.count_nonzero(out).item() == 0
    errs = []
    for x in xs[10:]:
        st.push(torch.from_numpy(x).cuda())
        st.reconstruct(out, "f64")
        xh = out.cpu().numpy()
        assert np.all(np.isfinite(xh))
        errs.append(rel(xh, x))
    g1 = st.core(1).reshape(-1, r[0])
    assert np.abs(g1.T @ g1 - np.eye(r[0])).max() < 1e-12
    assert max(errs[-10:]) < 0.05


def test_nonfinite_slice_not_committed():
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream, TTALSError
    sp = synth.make_stream("plain")
    xs = sp.take(6)
    r = O.clamp_ranks(sp.dims, sp.ranks)
    cores, g = synth.init_cores(sp.dims, r, seed=7)
    for ingest in ("f64", "f32"):
        st = Stream(sp.dims, sp.ranks, ingest=ingest)
        st.set_cores(cores, g)
        dt = torch.float64 if ingest == "f64" else torch.float32
        out_a = torch.empty(sp.dims, dtype=torch.float64, device="cuda")
        out_b = torch.empty_like(out_a)
        for x in xs[:3]:
            st.push(torch.from_numpy(x).to(dt).cuda())
        st.reconstruct(out_a, "f64")
        bad = torch.from_numpy(xs[3]).to(dt).cuda()
        bad[5, 7] = float("nan")
        st.push(bad)
        with pytest.raises(TTALSError) as ei:
            st.sync()
        assert ei.value.name == "ENONFINITE"
        st.reconstruct(out_b, "f64")
        assert torch.equal(out_a, out_b)
        assert st.step() == 3
        st.push(torch.from_numpy(xs[3]).to(dt).cuda())
        st.sync()
        assert st.step() == 4


def test_stats_match_oracle():
    sp = synth.make_stream("plain")
    frames = sp.take(20)
    xg, xo, ex, st = run_pair(sp.dims, sp.ranks, frames, "f64")
    s = st.stats()
    assert abs(s[0] - np.sum(ex[-1] ** 2)) <= 1e-12 * s[0]
    assert abs(s[1] - np.sum((ex[-1] - xo[-1]) ** 2)) <= 1e-8 * s[0]
    re = math.sqrt(s[3] / s[2])
    assert abs(re - O.stream_relative_error(ex, xo)) <= 1e-9


def test_cores_are_a_left_orthogonal_tt_of_the_reconstruction():
    """ttals_cores returns left-orthogonal cores (Sec. 2.4) whose TT contraction is x^_t."""
    torch = _torch()
    for name, kw, ingest in (("sensor", dict(change_every=15), "f32"),
                             ("video", dict(dims=(60, 80, 3)), "f64"),
                             ("plain", {}, "f64")):
        sp = synth.make_stream(name, **kw)
        xg, xo, ex, st = run_pair(sp.dims, sp.ranks, sp.take(4), ingest)
        cores, g = st.cores()
        tol = 1e-12 if ingest == "f64" else 1e-5
        for c in cores:
            u = c.reshape(-1, c.shape[-1])
            assert np.abs(u.T @ u - np.eye(u.shape[1])).max() < tol
        v = g.reshape(-1, 1)
        for c in reversed(cores):
            v = np.tensordot(c, v, axes=([2], [0])).reshape(c.shape[0], -1)
        assert rel(v.reshape(sp.dims), xg[-1]) < (1e-12 if ingest == "f64" else 1e-5)


def test_resume_from_exported_cores():
    """Checkpoint / resume: cores exported at t = 15 and loaded into a new stream continue
    the run (FP64: identical to 1e-11)."""
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream
    sp = synth.make_stream("sensor", change_every=15, dims=(8, 6, 7, 5), ranks=(4, 6, 5, 3))
    xs = sp.take(25)
    r = O.clamp_ranks(sp.dims, sp.ranks)
    cores, g = synth.init_cores(sp.dims, r, seed=7)
    a = Stream(sp.dims, sp.ranks, ingest="f64")
    a.set_cores(cores, g)
    for x in xs[:15]:
        a.push(torch.from_numpy(x).cuda())
    c15, g15 = a.cores()
    b = Stream(sp.dims, sp.ranks, ingest="f64")
    b.set_cores(c15, g15, t=15)
    oa = torch.empty(sp.dims, dtype=torch.float64, device="cuda")
    ob = torch.empty_like(oa)
    for x in xs[15:]:
        dx = torch.from_numpy(x).cuda()
        a.push(dx)
        b.push(dx)
        a.reconstruct(oa, "f64")
        b.reconstruct(ob, "f64")
        assert rel(ob.cpu().numpy(), oa.cpu().numpy()) < 1e-11
    assert b.step() == 25


def test_deterministic_bitwise():
    torch = _torch()
    sp = synth.make_stream("video", dims=(120, 160, 3))
    frames = sp.take(6)
    a = run_pair(sp.dims, sp.ranks, frames, "f32")[0]
    b = run_pair(sp.dims, sp.ranks, frames, "f32")[0]
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_argument_errors():
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream, TTALSError
    from paper_2606_31061_b300 import ttals as T
    st = Stream((16, 16), (4, 4), ingest="f32")
    x = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(TTALSError):       # dtype mismatch
        T.load()
        T._check(T.load().ttals_push_slice(st._h, T.ctypes.c_void_p(x.data_ptr()), T.F64, None), "push")
    y = torch.zeros(300, dtype=torch.float32, device="cuda")
    with pytest.raises(TTALSError):       # misaligned pointer
        T._check(T.load().ttals_push_slice(st._h, T.ctypes.c_void_p(y.data_ptr() + 4), T.F32, None), "push")
    assert st.step() == 0


@pytest.mark.parametrize("factor", ["fp64", "fp32"])
def test_fused_factor_precisions(factor):
    """The fused FP16 path with its FP64 r x r factor (the default) and with the FP32 factor
    (the faster variant): both within the FP16 ingest bar of the oracle, on a video-shaped
    stream and on a rank-64 square stream (the factor's largest size)."""
    from paper_2606_31061_b300.ttals import Stream
    torch = _torch()
    for name, kw in (("video", {"dims": (120, 160, 3)}), ("square", {"s": 256, "r": 64})):
        sp = synth.make_stream(name, **kw)
        r = O.clamp_ranks(sp.dims, sp.ranks)
        cores, g = synth.init_cores(sp.dims, r, seed=7)
        st = Stream(sp.dims, sp.ranks, ingest="f16", factor=factor)
        st.set_cores(cores, g)
        orc = O.OnlineTTALS(sp.dims, r, cores, g)
        xs, xo = [], []
        for x in sp.take(10):
            dx, exact = _upload(x, "f16")
            st.push(dx)
            xs.append(exact)
            xo.append(orc.step(exact))
        s = st.stats()
        re_o = O.stream_relative_error(xs, xo)
        assert abs(np.sqrt(s[3] / s[2]) - re_o) <= 1e-3, (name, factor, np.sqrt(s[3] / s[2]), re_o)


@pytest.mark.parametrize("factor", ["fp64", "fp32"])
def test_fused_ill_conditioned_local_solves(factor):
    """Method ranks above the data's rank make the level-1 local solve nearly rank-deficient
    (scaled pivots below 1e-4): the fused path then takes its FP64-accurate Cholesky-QR
    (float-float Gram and apply, FP64 factor), and for exactly low-rank data (pivots at FP64
    rounding) the Householder QR.  Both within the FP16 ingest bar of the oracle."""
    from paper_2606_31061_b300.ttals import Stream
    torch = _torch()
    cases = (("video", {"dims": (96, 128, 3), "gen_ranks": (8, 8, 3), "ranks": (24, 9, 3)}),
             ("square", {"s": 128, "r": 32, "gen_ranks": (8, 8), "noise": 1e-4}),
             ("square", {"s": 128, "r": 32, "gen_ranks": (8, 8), "noise": 0.0}))
    for name, kw in cases:
        sp = synth.make_stream(name, **kw)
        r = O.clamp_ranks(sp.dims, sp.ranks)
        cores, g = synth.init_cores(sp.dims, r, seed=7)
        st = Stream(sp.dims, sp.ranks, ingest="f16", factor=factor)
        st.set_cores(cores, g)
        orc = O.OnlineTTALS(sp.dims, r, cores, g)
        xs, xo = [], []
        for x in sp.take(10):
            dx, exact = _upload(x, "f16")
            st.push(dx)
            xs.append(exact)
            xo.append(orc.step(exact))
        s = st.stats()
        re_o = O.stream_relative_error(xs, xo)
        assert st.step() == 10
        assert abs(np.sqrt(s[3] / s[2]) - re_o) <= 1e-3, (name, kw, factor, np.sqrt(s[3] / s[2]), re_o)


@pytest.mark.parametrize("name,kw,ingest", [("sensor", {"dims": (12, 12, 12, 16), "ranks": (6, 12, 12, 6)}, "f32"),
                                            ("video", {"dims": (96, 128, 3)}, "f16")])
def test_programmatic_launch_bitwise(monkeypatch, name, kw, ingest):
    """Steps chained by programmatic dependent launch (each kernel may start while its
    predecessor runs and waits for it at entry) give bitwise the results of plain stream
    ordering (TTALS_NO_PDL=1, read when a stream is created): on the generic path (k* = 3)
    and on the fused path, with eight steps enqueued back to back before any read."""
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream
    sp = synth.make_stream(name, seed=77, **kw)
    r = O.clamp_ranks(sp.dims, sp.ranks)
    cores, g = synth.init_cores(sp.dims, r, seed=8)
    frames = [_upload(x, ingest)[0] for x in sp.take(8)]
    res = []
    for flag in ("0", "1"):
        monkeypatch.setenv("TTALS_NO_PDL", flag)
        st = Stream(sp.dims, sp.ranks, ingest=ingest)
        st.set_cores(cores, g)
        for x in frames:
            st.push(x)
        out = torch.empty(tuple(sp.dims), dtype=torch.float64, device="cuda")
        st.reconstruct(out, "f64")
        res.append((out.cpu().numpy().copy(), np.array(st.stats())))
        st.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
