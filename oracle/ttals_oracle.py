"""FP64 CPU oracle for the Online TT-ALS update of arXiv 2606.31061.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this file; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use it.  It shares no code with the CUDA path.

It executes Algorithm 1 ("Online TT-ALS", Sec. 3.4) step by step, in float64,
in the paper's order and notation:

1. right-orthogonalisation (Sec. 3.4.1): normalise g_n, absorb its norm into
   G_{n-1}, then LQ-sweep k = n-1 .. 2 with G_{k-1} <- G_{k-1} x_3^1 L;
2. right interfaces B_{n-1} = g_n, B_k = G_{k+1} x_3^1 B_{k+1};
3. forward sweep k = 1 .. n-1 (Sec. 3.4.2): local solve
   G~_k = A_k^T x X^_t x B_k^T (Eq. proposed-core-update), QR, G_k <- Q,
   propagate R into G_{k+1} (or g_n), A_{k+1} = A_k x_k^1 G_k;
4. temporal row g_n = A_n^T vec(X_t).

Index conventions (a reading; the paper's matricisation is column-major,
Sec. 2.1): slices are C-order (last mode fastest); a core G_k has shape
(r_{k-1}, I_k, r_k); its left unfolding is the (r_{k-1} I_k) x r_k matrix
``G.reshape(r0*I, r1)`` and its right unfolding the r_{k-1} x (I_k r_k) matrix
``G.reshape(r0, I*r1)``.  Renaming indices does not change any result.

Readings where the paper is silent:

* QR has diag(R) >= 0 and LQ has diag(L) >= 0; a pivot column whose norm is at
  most 64 eps ||M||_F is left unreflected (R_jj = 0), so a zero matrix gives
  Q = I[:, :n], R = 0.
* Ranks are clamped to the feasible set r_k <= min(r_{k-1} I_k, I_{k+1} r_{k+1})
  (r_0 = 1, no right bound on r_{n-1}), iterated to a fixed point; the LQ of
  Sec. 3.4.1 needs r_{k-1} <= I_k r_k and the QR of Sec. 3.4.2 needs
  r_k <= r_{k-1} I_k.
* B_{n-1} = g_n is an r_{n-1} x 1 matrix: the trailing I_n[t-1] mode printed
  for B_k and X^_t is contracted with the single vector g_n[t-1].
* If ||g_n|| = 0 the normalisation is skipped and g_n is set to e_1.

Two local-solve modes:

* ``literal`` - Eq. proposed-core-update as printed (valid as the exact local
  least-squares solution when A_k^T A_k = I and B_k B_k^T = I);
* ``lsq`` - the exact local least-squares solution for any B_k:
  G~_k = A_k^T X^ B_k^T (B_k B_k^T)^+  (Sec. 3.3, the Gram-matrix form).

and the ablation of Sec. 5.4 ("w/o Ortho", Table ablation_ortho), mode ``noortho``:
Algorithm 1 with the LQ/QR orthogonalisation steps removed (the normalisation of g_n and
the LQ sweep of Sec. 3.4.1, the QR and the R propagation of Sec. 3.4.2).  Without
orthogonal cores the local problem of Eq. proposed-objective-matrix needs the Gram inverses
that Sec. 3.3 names, so each core is its exact least-squares solution
G_k = (A_k^T A_k)^+ A_k^T X^ B_k^T (B_k B_k^T)^+ and g_n = (A_n^T A_n)^+ A_n^T vec(X_t)
(a reading: the paper states only that the steps were removed; with the printed update
alone the cores would scale without bound, and Table ablation_ortho shows both variants
equal at t = 10).  In exact arithmetic it spans what ``literal`` spans.

All slices seen so far (Eq. proposed-objective-slice, the per-slice form of Eq.
proposed-objective-full): ``refit_temporal_rows`` gives the temporal rows that
minimise it with the cores frozen at their time-t values, and ``global_objective``
its value; both are pinned against dense least squares on tiny streams.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

EPS = float(np.finfo(np.float64).eps)
ZERO_PIVOT_REL = 64.0 * EPS


def clamp_ranks(dims: Sequence[int], ranks: Sequence[int]) -> List[int]:
    """Feasible TT ranks (reading of Sec. 3.4.1/3.4.2): r_k <= r_{k-1} I_k and
    r_k <= I_{k+1} r_{k+1} for k < n-1, iterated to a fixed point."""
    dims = [int(d) for d in dims]
    r = [int(x) for x in ranks]
    if len(r) != len(dims):
        raise ValueError("need one rank per slice mode")
    if any(d < 1 for d in dims) or any(x < 1 for x in r):
        raise ValueError("dims and ranks must be >= 1")
    m = len(dims)
    while True:
        old = list(r)
        prev = 1
        for k in range(m):
            r[k] = min(r[k], prev * dims[k])
            prev = r[k]
        for k in range(m - 2, -1, -1):
            r[k] = min(r[k], dims[k + 1] * r[k + 1])
        if r == old:
            return r


def householder_qr(m_in: np.ndarray):
    """Thin Householder QR (Golub & Van Loan, Matrix Computations, Alg. 5.2.1).

    Returns (Q, R), Q m x n with orthonormal columns, R n x n upper triangular
    with diag(R) >= 0, Q @ R = M.  Requires m >= n.  Columns whose remaining
    norm is at most 64 eps ||M||_F get no reflection (R_jj = 0) and Q keeps the
    corresponding (reflected) unit vector, so Q is orthonormal for any rank.
    """
    a = np.array(m_in, dtype=np.float64, copy=True)
    m, n = a.shape
    if n > m:
        raise ValueError("householder_qr needs rows >= cols")
    thresh = ZERO_PIVOT_REL * np.linalg.norm(a)
    vs: List[Optional[np.ndarray]] = []
    for j in range(n):
        x = a[j:, j]
        nx = np.linalg.norm(x)
        if nx <= thresh:
            vs.append(None)
            continue
        alpha = -math.copysign(nx, x[0])
        v = x.copy()
        v[0] -= alpha
        v /= np.linalg.norm(v)
        a[j:, j:] -= 2.0 * np.outer(v, v @ a[j:, j:])
        vs.append(v)
    r = np.triu(a[:n, :n])
    q = np.eye(m, n)
    for j in range(n - 1, -1, -1):
        v = vs[j]
        if v is None:
            continue
        q[j:, :] -= 2.0 * np.outer(v, v @ q[j:, :])
    s = np.where(np.diag(r) < 0.0, -1.0, 1.0)
    return q * s[None, :], r * s[:, None]


def lq(m_in: np.ndarray):
    """LQ decomposition as the QR of the transpose (Sec. 3.4.1): M = L Q,
    L lower triangular with diag(L) >= 0, Q Q^T = I."""
    q, r = householder_qr(np.asarray(m_in).T)
    return r.T, q.T


class OnlineTTALS:
    """Online TT-ALS state {G_k}_{k=1}^{n-1}, g_n and the per-step update of
    Algorithm 1.  ``dims`` are the slice modes I_1..I_{n-1}; ``ranks`` are
    r_1..r_{n-1} (clamped).  ``cores``/``g`` give the initial state (copied)."""

    def __init__(self, dims, ranks, cores, g, mode: str = "literal", record: bool = False):
        if mode not in ("literal", "lsq", "noortho"):
            raise ValueError(mode)
        self.dims = [int(d) for d in dims]
        self.ranks = clamp_ranks(self.dims, ranks)
        self.full = [1] + self.ranks
        self.m = len(self.dims)  # n - 1 slice modes
        if len(cores) != self.m:
            raise ValueError("need n-1 cores")
        self.G = []
        for k, c in enumerate(cores):
            c = np.array(c, dtype=np.float64, copy=True)
            want = (self.full[k], self.dims[k], self.full[k + 1])
            if c.shape != want:
                raise ValueError(f"core {k + 1} has shape {c.shape}, expected {want}")
            self.G.append(c)
        self.g = np.array(g, dtype=np.float64, copy=True).reshape(self.full[-1])
        self.mode = mode
        self.record = record
        self.t = 0
        self.log = {}

    # -- helpers -----------------------------------------------------------
    def reconstruct(self) -> np.ndarray:
        """x^_t = G_1 x G_2 x ... x G_{n-1} x g_n (the time-t TT, Sec. 3.1)."""
        v = self.g.reshape(-1, 1)
        for k in range(self.m - 1, -1, -1):
            v = np.tensordot(self.G[k], v, axes=([2], [0])).reshape(self.full[k], -1)
        return v.reshape(self.dims)

    def _local_objective(self, a_mat, gk, b_mat, xhat) -> float:
        """f(G_k) = 1/2 || X^ - A_k x G_k x B_k ||_F^2 (Eq. proposed-objective-matrix)."""
        model = np.tensordot(np.tensordot(a_mat, gk, axes=([1], [0])), b_mat, axes=([2], [0]))
        return 0.5 * float(np.sum((xhat - model) ** 2))

    # -- Algorithm 1, one time step -----------------------------------------
    def step(self, x) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        if tuple(x.shape) != tuple(self.dims):
            raise ValueError(f"slice shape {x.shape} != {self.dims}")
        m, dims, full = self.m, self.dims, self.full
        G = self.G
        rec = {} if self.record else None
        if rec is not None:
            rec["prev_xhat"] = self.reconstruct()

        ortho = self.mode != "noortho"
        # 1. Right orthogonalisation (Sec. 3.4.1)
        rho = float(np.linalg.norm(self.g))
        if not ortho:
            if rho == 0.0:                        # zero temporal row: as in the other modes
                self.g = np.zeros_like(self.g)
                self.g[0] = 1.0
        elif rho > 0.0:
            G[m - 1] = rho * G[m - 1]
            self.g = self.g / rho
        else:
            self.g = np.zeros_like(self.g)
            self.g[0] = 1.0
        for k in range(m - 1, 0, -1) if ortho else ():   # cores G_{n-1} .. G_2
            r0, ik, r1 = G[k].shape
            l_mat, q_mat = lq(G[k].reshape(r0, ik * r1))
            G[k] = q_mat.reshape(r0, ik, r1)
            G[k - 1] = np.tensordot(G[k - 1], l_mat, axes=([2], [0]))
        if rec is not None:
            rec["right_orth_residual"] = max(
                [float(np.linalg.norm(G[k].reshape(full[k], -1) @ G[k].reshape(full[k], -1).T
                                      - np.eye(full[k]))) for k in range(1, m)] + [0.0])

        # 2. Right interfaces: B_{n-1} = g_n, B_k = G_{k+1} x_3^1 B_{k+1}
        B = [None] * m
        B[m - 1] = self.g.reshape(full[m], 1)
        for k in range(m - 2, -1, -1):
            B[k] = np.tensordot(G[k + 1], B[k + 1], axes=([2], [0])).reshape(full[k + 1], -1)

        # 3. Forward update and left orthogonalisation (Sec. 3.4.2)
        a_mat = np.ones((1, 1))                  # A_1 = 1
        f_old, f_new, bbt, a_list, gt_list = [], [], [], [], []
        for k in range(m):
            r0, ik, r1 = full[k], dims[k], full[k + 1]
            left = int(np.prod(dims[:k])) if k else 1
            rest = int(np.prod(dims[k + 1:])) if k + 1 < m else 1
            xhat3 = x.reshape(left, ik, rest)
            # local solve  G~_k = A_k^T x_2^1 X^_t x_3^1 B_k^T
            t_k = np.tensordot(a_mat.T, xhat3, axes=([1], [0]))            # (r0, ik, rest)
            gt = np.tensordot(t_k, B[k].T, axes=([2], [0]))                # (r0, ik, r1)
            if self.mode in ("lsq", "noortho"):
                gt = np.tensordot(gt, np.linalg.pinv(B[k] @ B[k].T), axes=([2], [0]))
            if not ortho:                                                   # (A_k^T A_k)^+
                gt = np.tensordot(np.linalg.pinv(a_mat.T @ a_mat), gt, axes=([1], [0]))
            if rec is not None:
                f_old.append(self._local_objective(a_mat, G[k], B[k], xhat3))
                f_new.append(self._local_objective(a_mat, gt, B[k], xhat3))
                bbt.append(float(np.linalg.norm(B[k] @ B[k].T - np.eye(r1))))
                a_list.append(a_mat.copy())
                gt_list.append(gt.copy())
            if ortho:
                q_mat, r_mat = householder_qr(gt.reshape(r0 * ik, r1))
                G[k] = q_mat.reshape(r0, ik, r1)
                if k < m - 1:                                               # propagate R
                    G[k + 1] = np.tensordot(r_mat, G[k + 1], axes=([1], [0]))
                else:
                    self.g = r_mat @ self.g
            else:
                G[k] = gt
            a_mat = (a_mat @ G[k].reshape(r0, ik * r1)).reshape(left * ik, r1)  # A_{k+1}

        # 4. Temporal row g_n = A_n^T vec(X_t)
        self.g = a_mat.T @ x.reshape(-1)
        if self.mode in ("lsq", "noortho"):
            self.g = np.linalg.pinv(a_mat.T @ a_mat) @ self.g
        self.t += 1
        xh = (a_mat @ self.g).reshape(dims)
        if rec is not None:
            rec.update(f_old=f_old, f_new=f_new, bbt_residual=bbt, a_n=a_mat, xhat=xh,
                       A=a_list, B=[b.copy() for b in B], gt=gt_list,
                       left_orth_residual=max(
                           float(np.linalg.norm(G[k].reshape(-1, full[k + 1]).T
                                                @ G[k].reshape(-1, full[k + 1])
                                                - np.eye(full[k + 1]))) for k in range(m)))
            self.log = rec
        return xh


def left_interface(cores) -> np.ndarray:
    """A_n = G_1 x_2^1 G_2 x_3^1 ... x G_{n-1} as a (I_1...I_{n-1}) x r_{n-1} matrix
    (the left interface of the temporal row, Sec. 3.2), contracted from the stored cores."""
    a = np.ones((1, 1))
    for c in cores:
        r0, ik, r1 = c.shape
        a = (a @ c.reshape(r0, ik * r1)).reshape(-1, r1)
    return a


def refit_temporal_rows(cores, slices) -> np.ndarray:
    """Temporal rows g_n[1..t] that minimise Eq. proposed-objective-slice over all slices
    seen so far with G_1..G_{n-1} held at their time-t values.  Each row is its own least
    squares problem min ||x_i - A_n g||; with left-orthogonal cores (A_n^T A_n = I, Sec. 3.3)
    its solution is A_n^T vec(x_i).  Returns an r_{n-1} x t matrix (column i = g_n[i])."""
    a = left_interface(cores)
    xs = np.stack([np.asarray(x, np.float64).reshape(-1) for x in slices], axis=1)
    return a.T @ xs


def global_objective(cores, rows, slices) -> float:
    """Value of Eq. proposed-objective-slice (the all-slices form of Eq.
    proposed-objective-full): sum_i ||x_i - G_1 x ... x G_{n-1} x g_n[i]||_F^2 for the
    given cores and temporal rows (column i of ``rows`` = g_n[i])."""
    a = left_interface(cores)
    tot = 0.0
    for i, x in enumerate(slices):
        res = np.asarray(x, np.float64).reshape(-1) - a @ rows[:, i]
        tot += float(res @ res)
    return tot


def run_stream(dims, ranks, cores, g, slices, mode="literal"):
    """Run Algorithm 1 over ``slices``; returns (list of x^_t, final state)."""
    st = OnlineTTALS(dims, ranks, cores, g, mode=mode)
    out = [st.step(x) for x in slices]
    return out, st


def stream_relative_error(slices, xhats) -> float:
    """RE = sqrt(sum_t ||x_t - x^_t||^2) / sqrt(sum_t ||x_t||^2) (Sec. 5.1, RE over
    the entire tensor, each x^_t from the time-t decomposition)."""
    num = sum(float(np.sum((np.asarray(a, np.float64) - b) ** 2)) for a, b in zip(slices, xhats))
    den = sum(float(np.sum(np.asarray(a, np.float64) ** 2)) for a in slices)
    return math.sqrt(num / den) if den > 0 else 0.0
