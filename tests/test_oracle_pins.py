"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties the oracle to something other than itself: a library routine
(LAPACK QR / SVD / lstsq), a closed form derived from Algorithm 1, brute force
on tiny inputs, or an inequality the paper proves (Proposition 4.1 (Monotonicity), Proposition 4.2 (Temporal Smoothness Bound)).
"""
import math

import numpy as np
import pytest

from oracle import ttals_oracle as O
from paper_2606_31061_b300 import synth


def _orth_lapack(a):
    q, r = np.linalg.qr(a)
    s = np.sign(np.diag(r))
    s[s == 0] = 1
    return q * s, r * s[:, None]


# --------------------------------------------------------------------------- QR / LQ
@pytest.mark.parametrize("shape", [(7, 3), (40, 8), (100, 32), (9, 9), (61440 // 64, 9)])
def test_householder_matches_lapack(shape):
    """Householder QR (diag R >= 0) equals LAPACK's QR with the same sign fix."""
    a = synth.seeded_gaussian(11 + shape[0], shape)
    q, r = O.householder_qr(a)
    q2, r2 = _orth_lapack(a)
    assert np.abs(q - q2).max() < 1e-12
    assert np.abs(r - r2).max() < 1e-12 * np.abs(r2).max()
    assert np.allclose(np.tril(r, -1), 0)
    assert np.all(np.diag(r) >= 0)


def test_householder_rank_deficient_and_zero():
    a = synth.seeded_gaussian(3, (12, 2)) @ synth.seeded_gaussian(4, (2, 5))   # rank 2 of 5
    q, r = O.householder_qr(a)
    assert np.abs(q.T @ q - np.eye(5)).max() < 1e-13
    assert np.abs(q @ r - a).max() < 1e-12 * np.abs(a).max()
    z = np.zeros((6, 3))
    q, r = O.householder_qr(z)
    assert np.array_equal(q, np.eye(6, 3)) and np.array_equal(r, np.zeros((3, 3)))


def test_lq():
    a = synth.seeded_gaussian(5, (6, 20))
    l, q = O.lq(a)
    assert np.allclose(np.triu(l, 1), 0) and np.all(np.diag(l) >= 0)
    assert np.abs(q @ q.T - np.eye(6)).max() < 1e-13
    assert np.abs(l @ q - a).max() < 1e-12


# --------------------------------------------------------------------------- rank clamp
def _brute_clamp(dims, ranks):
    """Largest rank vector (componentwise) that is feasible, by enumeration."""
    import itertools
    best = None
    for cand in itertools.product(*[range(1, r + 1) for r in ranks]):
        full = [1] + list(cand)
        ok = all(full[k + 1] <= full[k] * dims[k] for k in range(len(dims)))
        ok = ok and all(full[k + 1] <= dims[k + 1] * full[k + 2] for k in range(len(dims) - 1))
        if ok and (best is None or all(c >= b for c, b in zip(cand, best))):
            best = cand
    return list(best)


@pytest.mark.parametrize("dims,ranks", [((3, 2, 2), (5, 5, 2)), ((2, 3, 2, 2), (4, 6, 4, 3)),
                                        ((4, 4), (9, 9)), ((2, 2, 2), (3, 3, 3))])
def test_clamp_matches_bruteforce(dims, ranks):
    assert O.clamp_ranks(dims, ranks) == _brute_clamp(dims, ranks)


def test_clamp_paper_configs():
    assert O.clamp_ranks((1080, 1920, 3), (32, 32, 3)) == [32, 9, 3]
    assert O.clamp_ranks((32, 32), (8, 8)) == [8, 8]
    assert O.clamp_ranks((32,) * 4, (16, 32, 32, 16)) == [16, 32, 32, 16]
    with pytest.raises(ValueError):
        O.clamp_ranks((4, 0), (2, 2))


# --------------------------------------------------------------------------- whole sweep
def _stream(name, T, **kw):
    sp = synth.make_stream(name, **kw)
    xs = sp.take(T)
    r = O.clamp_ranks(sp.dims, sp.ranks)
    cores, g = synth.init_cores(sp.dims, r, seed=sp.seed + 1)
    return sp, xs, r, cores, g


def test_closed_form_subspace_iteration_n3():
    """For n = 3, Algorithm 1 reduces (x^_t is gauge invariant) to
    U_t = orth(X_t C_{t-1}^T), C_t = U_t^T X_t, x^_t = U_t C_t with C_0 = G_2 x_3 g_n.
    The closed form uses only LAPACK QR, independent of the oracle's code."""
    sp, xs, r, cores, g = _stream("plain", 100)
    xh, _ = O.run_stream(sp.dims, r, cores, g, xs)
    c = np.tensordot(cores[1], g, axes=([2], [0]))
    for x, xo in zip(xs, xh):
        u, _ = np.linalg.qr(x @ c.T)
        c = u.T @ x
        assert np.linalg.norm(u @ c - xo) <= 1e-12 * np.linalg.norm(xo)


def test_closed_form_saturated_n4():
    """For the video shape with clamped ranks (r1, 9, 3) the later cores span every
    vector of the trailing modes, so x^_t = U_t U_t^T X_t(1) with U_t = orth(X_t(1) C_{t-1}^T)."""
    sp, xs, r, cores, g = _stream("video", 8, dims=(48, 40, 3), gen_ranks=(12, 12, 3), ranks=(12, 12, 3))
    assert r == [12, 9, 3]
    xh, _ = O.run_stream(sp.dims, r, cores, g, xs)
    c = np.tensordot(cores[1], np.tensordot(cores[2], g, axes=([2], [0])), axes=([2], [0]))
    c = c.reshape(r[0], -1)
    for x, xo in zip(xs, xh):
        x1 = x.reshape(48, -1)
        u, _ = np.linalg.qr(x1 @ c.T)
        c = u.T @ x1
        assert np.linalg.norm((u @ c).reshape(x.shape) - xo) <= 1e-11 * np.linalg.norm(xo)


def test_repeated_slice_converges_to_eckart_young():
    """Feeding one slice repeatedly makes the n = 3 update a subspace iteration on X X^T,
    whose error converges to the Eckart-Young optimum sqrt(sum_{i>r} sigma_i^2)."""
    rng = np.random.default_rng(21)
    u, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    v, _ = np.linalg.qr(rng.standard_normal((24, 24)))
    s = np.array([10.0 / (1 + i) ** 1.5 for i in range(24)])
    x = (u[:, :24] * s) @ v.T
    r = [5, 5]
    cores, g = synth.init_cores((30, 24), r, seed=3)
    st = O.OnlineTTALS((30, 24), r, cores, g)
    for _ in range(60):
        xh = st.step(x)
    ey = math.sqrt(float(np.sum(s[5:] ** 2)))
    assert abs(np.linalg.norm(x - xh) - ey) <= 1e-10 * ey


@pytest.mark.parametrize("name,kw", [("plain", dict(noise=0.0)),
                                     ("sensor", dict(dims=(5, 4, 6, 3), ranks=(3, 4, 4, 2),
                                                     noise=0.0, change_every=7)),
                                     ("square", dict(s=20, r=4, noise=0.0))])
def test_exact_recovery_noiseless_tt_stream(name, kw):
    """A noiseless stream of exact TT rank r is recovered to machine precision at every
    step (including after abrupt changes), by induction on the spans."""
    sp, xs, r, cores, g = _stream(name, 20, **kw)
    xh, _ = O.run_stream(sp.dims, r, cores, g, xs)
    for x, xo in zip(xs, xh):
        assert np.linalg.norm(x - xo) <= 1e-12 * np.linalg.norm(x)


def test_temporal_row_is_bruteforce_lstsq():
    """g_n[t] = argmin ||A_n g - x_t|| computed by dense LAPACK lstsq (Sec. 3.4.2)."""
    sp, xs, r, cores, g = _stream("sensor", 4, dims=(4, 3, 5, 2), ranks=(3, 4, 4, 2))
    st = O.OnlineTTALS(sp.dims, r, cores, g, record=True)
    for x in xs:
        st.step(x)
        a_n = st.log["a_n"]
        ref, *_ = np.linalg.lstsq(a_n, x.reshape(-1), rcond=None)
        assert np.abs(ref - st.g).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def _dense_local_lsq(a_mat, b_mat, xhat3, r0, ik, r1):
    """min_G || vec X^ - M vec G || with M[(l,i,j),(a,i',b)] = A[l,a] d(i,i') B[b,j], dense."""
    left, _, rest = xhat3.shape
    m = np.zeros((left * ik * rest, r0 * ik * r1))
    for l in range(left):
        for i in range(ik):
            for j in range(rest):
                row = (l * ik + i) * rest + j
                for a in range(r0):
                    for b in range(r1):
                        m[row, (a * ik + i) * r1 + b] = a_mat[l, a] * b_mat[b, j]
    sol, *_ = np.linalg.lstsq(m, xhat3.reshape(-1), rcond=None)
    return sol.reshape(r0, ik, r1)


@pytest.mark.parametrize("mode,ranks", [("lsq", (2, 3, 2)), ("literal", (2, 3, 1))])
def test_local_solve_is_bruteforce_least_squares(mode, ranks):
    """Each local solve G~_k equals the dense least-squares minimiser of
    f(G_k) (Eq. proposed-objective-matrix); in the literal mode this needs
    B_k B_k^T = I, which holds when r_{n-1} = 1."""
    dims = (3, 4, 3)
    r = O.clamp_ranks(dims, ranks)
    cores, g = synth.init_cores(dims, r, seed=9)
    st = O.OnlineTTALS(dims, r, cores, g, mode=mode, record=True)
    xs = [synth.seeded_gaussian(40 + t, dims) for t in range(3)]
    full = [1] + r
    for x in xs:
        st.step(x)
        for k in range(len(dims)):
            left = int(np.prod(dims[:k])) if k else 1
            rest = int(np.prod(dims[k + 1:])) if k + 1 < len(dims) else 1
            ref = _dense_local_lsq(st.log["A"][k], st.log["B"][k], x.reshape(left, dims[k], rest),
                                   full[k], dims[k], full[k + 1])
            assert np.abs(ref - st.log["gt"][k]).max() <= 1e-10 * max(1.0, np.abs(ref).max())


def test_orthogonality_invariants():
    """Left-orthogonal cores after every step, right-orthogonal cores after the LQ sweep
    (Sec. 2.4 definitions), to 1e-12."""
    sp, xs, r, cores, g = _stream("sensor", 12, dims=(6, 5, 4, 6), ranks=(4, 6, 5, 3), change_every=5)
    st = O.OnlineTTALS(sp.dims, r, cores, g, record=True)
    for x in xs:
        st.step(x)
        assert st.log["left_orth_residual"] <= 1e-12
        assert st.log["right_orth_residual"] <= 1e-12


def test_monotonicity_prop41():
    """Proposition 4.1 (Monotonicity): f(G*) <= f(G_old) for every local solve.  A theorem for the lsq mode
    (exact local least squares) and for the literal mode when r_{n-1} = 1 (then
    B_k B_k^T = I); with r_{n-1} > 1 the end-to-end bound E_t <= ||x_t - M_{t-1}|| holds."""
    for mode, ranks in (("lsq", (4, 5, 4, 3)), ("literal", (4, 5, 4, 1))):
        sp, xs, r, cores, g = _stream("sensor", 15, dims=(6, 5, 4, 5), ranks=ranks, noise=0.05,
                                      change_every=6)
        st = O.OnlineTTALS(sp.dims, r, cores, g, mode=mode, record=True)
        for x in xs:
            st.step(x)
            for fo, fn in zip(st.log["f_old"], st.log["f_new"]):
                assert fn <= fo * (1 + 1e-12) + 1e-300
            # chain: f_1(G_1^old) = 1/2 ||x - M_{t-1}||^2 and f_{k+1}(R G_{k+1}) = f_k(G_k*)
            assert abs(st.log["f_old"][0] - 0.5 * np.sum((x - st.log["prev_xhat"]) ** 2)) \
                <= 1e-9 * max(1.0, st.log["f_old"][0])
            for k in range(len(st.log["f_new"]) - 1):
                assert abs(st.log["f_old"][k + 1] - st.log["f_new"][k]) <= 1e-9 * max(1.0, st.log["f_new"][k])
    # literal, r_{n-1} > 1: end-to-end only
    sp, xs, r, cores, g = _stream("plain", 30)
    st = O.OnlineTTALS(sp.dims, r, cores, g, record=True)
    for x in xs:
        xh = st.step(x)
        assert np.linalg.norm(x - xh) <= np.linalg.norm(x - st.log["prev_xhat"]) * (1 + 1e-12)


def test_prop41_identity_under_orthogonality():
    """Under A^T A = I, B B^T = I: f(G) = f(G*) + 1/2 ||G - G*||^2 (proof of Proposition 4.1 (Monotonicity))."""
    dims = (4, 5, 3)
    r = O.clamp_ranks(dims, [3, 4, 1])
    cores, g = synth.init_cores(dims, r, seed=12)
    st = O.OnlineTTALS(dims, r, cores, g, record=True)
    x = synth.seeded_gaussian(13, dims)
    st.step(x)
    k = 1
    a_mat, b_mat, gt = st.log["A"][k], st.log["B"][k], st.log["gt"][k]
    assert np.abs(b_mat @ b_mat.T - np.eye(b_mat.shape[0])).max() < 1e-12
    xhat3 = x.reshape(dims[0], dims[1], dims[2])
    other = gt + synth.seeded_gaussian(14, gt.shape)
    f = st._local_objective(a_mat, other, b_mat, xhat3)
    fs = st._local_objective(a_mat, gt, b_mat, xhat3)
    assert abs(f - fs - 0.5 * np.sum((other - gt) ** 2)) <= 1e-10 * f


def test_temporal_smoothness_prop42():
    """Proposition 4.2 (Temporal Smoothness Bound): E_t <= E_{t-1} + ||x_t - x_{t-1}||."""
    sp, xs, r, cores, g = _stream("sensor", 25, dims=(6, 5, 4, 5), ranks=(4, 5, 4, 2), noise=0.02,
                                  change_every=9)
    xh, _ = O.run_stream(sp.dims, r, cores, g, xs)
    for t in range(1, len(xs)):
        e_t = np.linalg.norm(xs[t] - xh[t])
        e_prev = np.linalg.norm(xs[t - 1] - xh[t - 1])
        assert e_t <= e_prev + np.linalg.norm(xs[t] - xs[t - 1]) + 1e-12


def test_literal_equals_lsq_on_reconstruction():
    """range(B^T (B B^T)^+) = range(B^T), so both modes give the same x^_t."""
    sp, xs, r, cores, g = _stream("sensor", 12, dims=(6, 5, 4, 5), ranks=(4, 5, 4, 3), change_every=5)
    a, _ = O.run_stream(sp.dims, r, cores, g, xs, mode="literal")
    b, _ = O.run_stream(sp.dims, r, cores, g, xs, mode="lsq")
    for u, v in zip(a, b):
        assert np.linalg.norm(u - v) <= 1e-11 * np.linalg.norm(u)


def test_eckart_young_lower_bound():
    """x^_t is a rank-r_{n-2} projection of the (1..n-2 | n-1) unfolding, so its error is
    at least the Eckart-Young bound of that unfolding (SVD)."""
    sp, xs, r, cores, g = _stream("sensor", 10, dims=(6, 5, 4, 5), ranks=(4, 5, 3, 2), noise=0.05)
    xh, _ = O.run_stream(sp.dims, r, cores, g, xs)
    for x, xo in zip(xs, xh):
        s = np.linalg.svd(x.reshape(-1, x.shape[-1]), compute_uv=False)
        ey = math.sqrt(float(np.sum(s[r[-2]:] ** 2)))
        assert np.linalg.norm(x - xo) >= ey * (1 - 1e-12)


def test_noise_floor_statistic():
    """Exact-rank signal plus i.i.d. noise sigma: once the subspace is tracked, the residual
    is noise outside span(U) (x) R^{I_2}.  Its energy lies between the Eckart-Young value
    for a subspace fitted to the noisy slice, sigma^2 (I_1 - r)(I_2 - r), and the value for
    the true subspace, sigma^2 (I_1 - r) I_2 (5% slack for the finite sample)."""
    sig = 0.05
    sp, xs, r, cores, g = _stream("plain", 100, noise=sig, theta=0.0)
    xh, _ = O.run_stream(sp.dims, r, cores, g, xs)
    tail = list(zip(xs[20:], xh[20:]))
    num = sum(np.sum((x - xo) ** 2) for x, xo in tail) / len(tail)
    lo = sig ** 2 * (32 - 8) * (32 - 8)
    hi = sig ** 2 * (32 - 8) * 32
    assert 0.95 * lo <= num <= 1.05 * hi


def test_zero_slice_and_recovery():
    """A zero slice gives x^ = 0 and g_n = 0; the next step uses g_n = e_1 and recovers."""
    sp, xs, r, cores, g = _stream("plain", 12)
    st = O.OnlineTTALS(sp.dims, r, cores, g)
    for x in xs[:5]:
        st.step(x)
    xh = st.step(np.zeros(sp.dims))
    assert np.array_equal(xh, np.zeros(sp.dims)) and np.linalg.norm(st.g) == 0
    errs = [np.linalg.norm(x - st.step(x)) / np.linalg.norm(x) for x in xs[5:]]
    assert all(np.isfinite(errs)) and errs[-1] < 0.05


def test_stream_relative_error_definition():
    xs = [np.ones((2, 2)), 2 * np.ones((2, 2))]
    xh = [np.zeros((2, 2)), 2 * np.ones((2, 2))]
    assert abs(O.stream_relative_error(xs, xh) - math.sqrt(4 / 20)) < 1e-15


def _dense_left_interface(cores):
    """A_n by brute force: column b of A_n is the full contraction G_1 x ... x G_{n-1} x e_b,
    formed element by element over every multi-index of the slice (tiny shapes only)."""
    import itertools
    dims = [c.shape[1] for c in cores]
    rn = cores[-1].shape[2]
    a = np.zeros((int(np.prod(dims)), rn))
    for row, idx in enumerate(itertools.product(*[range(d) for d in dims])):
        v = np.ones(1)
        for c, i in zip(cores, idx):
            v = v @ c[:, i, :]
        a[row] = v
    return a


@pytest.mark.parametrize("mode", ["literal", "lsq"])
def test_all_slices_batch_least_squares(mode):
    """All slices seen so far (Eq. proposed-objective-slice): with the cores frozen after
    step t, the temporal rows that minimise the objective over x_1..x_t, found by dense
    LAPACK lstsq against a brute-force A_n, equal the oracle's refit A_n^T [x_1 .. x_t]
    (<= 1e-12), its last column is the online g_n[t], and the oracle's global objective equals
    the brute-force residual and lies above the Eckart-Young bound of the stacked slices at
    rank r_{n-1}.  The global objective is reported beside the online RE (context: the
    online RE uses time-varying cores, so no inequality links the two)."""
    dims = (4, 3, 5)
    sp = synth.make_stream("sensor", dims=dims, ranks=(3, 4, 2), noise=0.05, change_every=0)
    xs = sp.take(6)
    r = O.clamp_ranks(dims, sp.ranks)
    cores, g = synth.init_cores(dims, r, seed=31)
    st = O.OnlineTTALS(dims, r, cores, g, mode=mode)
    seen, online = [], []
    for x in xs:
        online.append(st.step(x))
        seen.append(x)
        a_n = _dense_left_interface(st.G)
        assert np.abs(a_n - O.left_interface(st.G)).max() <= 1e-13
        stacked = np.stack([s.reshape(-1) for s in seen], axis=1)
        ref, *_ = np.linalg.lstsq(a_n, stacked, rcond=None)
        rows = O.refit_temporal_rows(st.G, seen)
        assert rows.shape == (r[-1], len(seen))
        assert np.abs(rows - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
        assert np.abs(rows[:, -1] - st.g).max() <= 1e-12 * max(1.0, np.abs(st.g).max())
        brute = float(np.sum((stacked - a_n @ ref) ** 2))
        obj = O.global_objective(st.G, rows, seen)
        assert abs(obj - brute) <= 1e-12 * max(1.0, brute)
        sv = np.linalg.svd(stacked, compute_uv=False)
        assert obj >= float(np.sum(sv[r[-1]:] ** 2)) * (1 - 1e-12)
    global_re = math.sqrt(obj / sum(float(np.sum(s ** 2)) for s in seen))
    online_re = O.stream_relative_error(seen, online)
    print(f"{mode}: global RE with frozen time-{len(seen)} cores {global_re:.4f}, online RE {online_re:.4f}")
    assert 0.0 < global_re < 1.0 and 0.0 < online_re < 1.0
