"""Seeded synthetic tensor streams shaped like the workloads of arXiv 2606.31061 (Sec. 5).

This module only *draws inputs*: ground-truth TT fields, drift, noise and the
rounding of a slice to an ingest dtype.  It holds none of the Online TT-ALS
arithmetic (no local solves, no interfaces, no orthogonalisation of the
estimate).  Both the FP64 oracle and the CUDA path consume what it produces, so
the two sides always see bit-identical slices.

Streams (the paper's CDnet videos are not available; these stand in for the
paper's synthetic high-order tensors, Sec. 5.1, and its video workloads):

* ``plain``  - 3rd-order stream of 32x32 slices, TT ranks (8,8).  Ground-truth
  cores are Gaussian, left-orthogonalised by QR, and every step each core's
  left unfolding is rotated by 0.01 rad in a random 2-plane.  Temporal weights
  follow a stationary AR(1) process (coefficient 0.95, N(0, I) innovations) scaled
  so the element RMS is ~1, so consecutive slices are correlated as in video;
  i.i.d. N(0, 0.01^2) noise.
* ``video``  - 4th-order H x W x C stream (default 1080x1920x3) of uint8-range
  values: a smooth TT field (DCT-II bases in the two spatial modes, ranks
  (32,32,3)) with slow sinusoidal temporal weights, plus integer uniform noise
  in {-4..4}, rounded and clipped to [0, 255].  Every value is an integer, so
  it is exact in FP16.
* ``sensor`` - 5th-order stream of 32^4 slices, TT ranks (16,32,32,16), a
  random TT (QR-orthogonalised cores, AR(1) temporal weights as in ``plain``)
  with N(0, 1e-3^2) noise; every
  ``change_every`` steps each core's left unfolding is multiplied by a fresh
  Haar-random orthogonal matrix (abrupt change).
* ``square`` - 3rd-order s x s stream with ranks (r, r), same recipe as
  ``plain`` (used for the batched-stream shapes).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Iterator, List, Sequence, Tuple

import numpy as np

__all__ = [
    "StreamSpec", "make_stream", "init_cores", "round_to_ingest", "INGEST_DTYPES",
    "seeded_gaussian",
]

INGEST_DTYPES = ("f64", "f32", "f16", "bf16")


def seeded_gaussian(seed: int, shape) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


def _qr_orth(a: np.ndarray) -> np.ndarray:
    """Orthonormal columns spanning ``a`` (library QR, signs fixed so diag(R) > 0)."""
    q, r = np.linalg.qr(a)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def _haar(rng: np.random.Generator, n: int) -> np.ndarray:
    return _qr_orth(rng.standard_normal((n, n)))


def _rotate_plane(rng: np.random.Generator, u_mat: np.ndarray, theta: float) -> np.ndarray:
    """Rotate the column space of orthonormal ``u_mat`` (m x r) by ``theta`` radians
    inside the 2-plane span(u, v), u in col(u_mat), v orthogonal to col(u_mat)."""
    m, r = u_mat.shape
    if r >= m:  # nothing orthogonal to rotate into
        return u_mat
    w = rng.standard_normal(r)
    u = u_mat @ w
    u /= np.linalg.norm(u)
    v = rng.standard_normal(m)
    v -= u_mat @ (u_mat.T @ v)
    v -= u_mat @ (u_mat.T @ v)
    v /= np.linalg.norm(v)
    coeff = u @ u_mat  # (r,)
    return u_mat + np.outer((math.cos(theta) - 1.0) * u + math.sin(theta) * v, coeff)


def _dct_basis(n: int, k: int) -> np.ndarray:
    """First ``k`` orthonormal DCT-II vectors on ``n`` points (n x k)."""
    i = np.arange(n)[:, None] + 0.5
    j = np.arange(k)[None, :]
    d = np.cos(np.pi * i * j / n) * math.sqrt(2.0 / n)
    d[:, 0] = math.sqrt(1.0 / n)
    return d


def round_to_ingest(x: np.ndarray, dtype: str) -> Tuple[np.ndarray, np.ndarray]:
    """Round a float64 slice to an ingest dtype.

    Returns ``(payload, exact)``: ``payload`` is a contiguous numpy array of the
    ingest type (``uint16`` bit patterns for f16/bf16) to upload to the device,
    and ``exact`` is the same values widened back to float64, which is what the
    oracle ingests.  Rounding is round-to-nearest-even in every case.
    """
    x = np.ascontiguousarray(x, dtype=np.float64)
    if dtype == "f64":
        return x, x
    if dtype == "f32":
        p = x.astype(np.float32)
        return p, p.astype(np.float64)
    if dtype == "f16":
        p = x.astype(np.float16)
        return p.view(np.uint16), p.astype(np.float64)
    if dtype == "bf16":
        f = x.astype(np.float32)
        bits = f.view(np.uint32).astype(np.uint64)
        # round-to-nearest-even on the upper 16 bits (inputs here are finite)
        lsb = (bits >> 16) & 1
        bits = (bits + 0x7FFF + lsb) >> 16
        b16 = bits.astype(np.uint16)
        exact = (b16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return b16, exact
    raise ValueError(f"unknown ingest dtype {dtype!r}")


def init_cores(dims: Sequence[int], ranks: Sequence[int], seed: int):
    """Seeded random initial state {G_k}, g_n (Algorithm 1, initialisation).

    Cores are Gaussian and left-orthogonalised with a library QR; ``g_n`` is
    Gaussian.  ``ranks`` must already be feasible (see the rank clamp).
    Returns ``(cores, g)`` with ``cores[k]`` of shape (r_{k-1}, I_k, r_k).
    """
    rng = np.random.default_rng(seed)
    full = [1] + list(ranks)
    cores = []
    for k, ik in enumerate(dims):
        a = rng.standard_normal((full[k] * ik, full[k + 1]))
        cores.append(_qr_orth(a).reshape(full[k], ik, full[k + 1]))
    g = rng.standard_normal(full[-1])
    return cores, g


@dataclass
class StreamSpec:
    kind: str
    dims: Tuple[int, ...]
    ranks: Tuple[int, ...]          # requested TT ranks r_1..r_{n-1}
    T: int
    seed: int
    ingest: str = "f64"
    noise: float = 0.0
    theta: float = 0.0
    change_every: int = 0
    gen_ranks: Tuple[int, ...] = ()  # ground-truth ranks (default: ``ranks``)
    extra: dict = field(default_factory=dict)

    @property
    def slice_elems(self) -> int:
        return int(np.prod(self.dims))

    def frames(self, T: int | None = None) -> Iterator[np.ndarray]:
        """Yield float64 slices X_1..X_T (before ingest rounding), in order."""
        T = self.T if T is None else T
        if self.kind in ("plain", "square", "sensor"):
            yield from _tt_drift_frames(self, T)
        elif self.kind == "video":
            yield from _video_frames(self, T)
        else:
            raise ValueError(self.kind)

    def take(self, T: int | None = None) -> List[np.ndarray]:
        return list(self.frames(T))


def _tt_drift_frames(spec: StreamSpec, T: int) -> Iterator[np.ndarray]:
    rng = np.random.default_rng(spec.seed)
    dims = spec.dims
    gr = spec.gen_ranks or spec.ranks
    full = [1] + list(gr)
    if any(full[k + 1] > full[k] * dims[k] for k in range(len(dims))):
        raise ValueError(f"ground-truth ranks {gr} exceed the mode sizes {dims}")
    lefts = [_qr_orth(rng.standard_normal((full[k] * dims[k], full[k + 1])))
             for k in range(len(dims))]
    scale = math.sqrt(float(np.prod(dims)) / full[-1])
    noise_rng = np.random.default_rng(spec.seed + 7919)
    a = float(spec.extra.get("ar", 0.95))
    g = rng.standard_normal(full[-1]) * scale
    for t in range(1, T + 1):
        if spec.change_every and t > 1 and (t - 1) % spec.change_every == 0:
            lefts = [_haar(rng, u.shape[0]) @ u for u in lefts]
        elif spec.theta and t > 1:
            lefts = [_rotate_plane(rng, u, spec.theta) for u in lefts]
        if t > 1:
            g = a * g + math.sqrt(1.0 - a * a) * scale * rng.standard_normal(full[-1])
        # contract the ground-truth train with the temporal weights
        v = g
        for k in range(len(dims) - 1, -1, -1):
            u = lefts[k].reshape(full[k], dims[k], full[k + 1])
            v = np.tensordot(u, v.reshape(full[k + 1], -1), axes=([2], [0]))
            v = v.reshape(full[k], -1)
        x = v.reshape(dims)
        if spec.noise:
            x = x + spec.noise * noise_rng.standard_normal(dims)
        yield x


def _video_frames(spec: StreamSpec, T: int) -> Iterator[np.ndarray]:
    h, w, c = spec.dims
    r1, r2, r3 = spec.gen_ranks or (32, 32, 3)
    rng = np.random.default_rng(spec.seed)
    d1 = _dct_basis(h, r1) @ _haar(rng, r1)
    decay = 1.0 / (1.0 + np.arange(r1) / 8.0)          # mild spectral decay
    g1 = d1 * decay[None, :]                            # (h, r1)
    d2 = _dct_basis(w, r2)
    hmix = _qr_orth(rng.standard_normal((r1 * r2, r2))).reshape(r1, r2, r2)
    g2 = np.einsum("ic,acb->aib", d2, hmix)             # (r1, w, r2), left-orthonormal
    g3 = _qr_orth(rng.standard_normal((r2 * c, r3))).reshape(r2, c, r3)
    periods = rng.uniform(100.0, 300.0, r3)
    phases = rng.uniform(0.0, 2 * math.pi, r3)
    amps = rng.uniform(0.5, 1.5, r3)
    noise_rng = np.random.default_rng(spec.seed + 7919)

    def field_at(t: int) -> np.ndarray:
        gt = amps * (1.0 + 0.5 * np.sin(2 * math.pi * t / periods + phases))
        k3 = np.tensordot(g3, gt, axes=([2], [0]))              # (r2, c)
        m = np.tensordot(g2, k3, axes=([2], [0])).reshape(r1, w * c)
        return (g1 @ m).reshape(h, w, c)

    f0 = field_at(1)
    q = np.quantile(np.abs(f0), 0.999)
    amp = 127.0 / q if q > 0 else 1.0
    for t in range(1, T + 1):
        f = field_at(t)
        noise = noise_rng.integers(-4, 5, size=(h, w, c))
        x = np.clip(np.rint(128.0 + amp * f + noise), 0.0, 255.0)
        yield x


def make_stream(name: str, **kw) -> StreamSpec:
    """Named synthetic streams.

    * ``plain``:  32x32, ranks (8,8), T=100, theta=0.01, sigma=0.01, FP64 ingest, seed 1001
    * ``video``:  1080x1920x3, ranks (32,32,3), T=600, FP32/FP16 ingest, seed 1002
    * ``sensor``: 32^4, ranks (16,32,32,16), T=1000, sigma=1e-3, change every 200, seed 1003
    * ``square``: s x s, ranks (r,r), theta=0.01, sigma=0.01 (``s``, ``r`` keywords), FP16
    """
    if name == "plain":
        spec = StreamSpec("plain", (32, 32), (8, 8), T=100, seed=1001, ingest="f64",
                          noise=0.01, theta=0.01)
    elif name == "video":
        spec = StreamSpec("video", (1080, 1920, 3), (32, 32, 3), T=600, seed=1002,
                          ingest="f32", gen_ranks=(32, 32, 3))
    elif name == "sensor":
        spec = StreamSpec("sensor", (32, 32, 32, 32), (16, 32, 32, 16), T=1000, seed=1003,
                          ingest="f32", noise=1e-3, change_every=200)
    elif name == "square":
        s = int(kw.pop("s", 256))
        r = int(kw.pop("r", 16))
        spec = StreamSpec("square", (s, s), (r, r), T=200, seed=1004, ingest="f16",
                          noise=0.01, theta=0.01)
    else:
        raise ValueError(f"unknown stream {name!r}")
    for k, v in kw.items():
        if not hasattr(spec, k):
            raise TypeError(f"unknown StreamSpec field {k!r}")
        if k in ("dims", "ranks", "gen_ranks"):
            v = tuple(int(a) for a in v)
        setattr(spec, k, v)
    return spec
