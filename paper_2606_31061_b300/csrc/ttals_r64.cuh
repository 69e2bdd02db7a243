// ttals_r64.cuh - FP64 r x r factorisation for the per-slice update (Sec. 3.4.2: the QR of the
// local solve G~_k = Q R, computed as the Cholesky factor of its Gram matrix: G~^T G~ = R^T R).
//
// B300's FP64 unit is narrow and slow to answer (measured on this part: a dependent DFMA takes
// 64 cycles; one warp issues 0.5 DFMA per clock, a whole SM 1.7).  A textbook Cholesky puts a
// square root or a reciprocal and a block barrier on the critical path of each of the r pivot
// steps, which made a first CTA version take 20 us at r = 32.  This one keeps the chain of a
// pivot step to one multiply, one fused multiply-add and one barrier:
//
//  * Fraction-free elimination (no division): step k replaces every trailing entry by
//      A_ij <- 2^-e (d A_ij - A_ik A_jk),  d = A_kk = c 2^e,  c in [1, 2),
//    i.e. A_ij <- c A_ij - 2^-e (A_ik A_jk).  The power of two 2^-e keeps the entries bounded:
//    with S^(k) the true Schur complements, A^(k) = P_k S^(k), P_k = c_0 c_1 ... c_{k-1}, and
//    every c_j lies in [1, 2).  The scaling by 2^-e is an exact exponent change.
//  * The Cholesky factor follows without any division on the critical path:
//      D_k = A^(k)_kk / P_k,   L_ik = A^(k)_ik / sqrt(A^(k)_kk P_k).
//  * Each thread keeps its entries of the lower triangle in registers, ordered by column
//    from the last, so the entries still to be updated at step k are a prefix of the order;
//    column k+1 is published through a double-buffered shared-memory column, one barrier per
//    step.  Four warps (one per SM sub-partition: the FP64 rate is per sub-partition) do the
//    work and synchronise through a named barrier.
//
// Used by the fused path's factor kernel (every CTA of the factor cluster factors the scaled
// Gram D W1 D of the level-1 local solve) and by the batched FP64 kernel k_r64_factor.
#pragma once

#include <cuda_runtime.h>

namespace r64 {

constexpr int kMaxR = 64;

struct Smem {
  double col[2][kMaxR];   // column k (parity k) of the current elimination step
  double dk[kMaxR];       // A^(k)_kk
  double pk[kMaxR];       // P_k
  double rs[kMaxR];       // 1 / sqrt(A^(k)_kk P_k)
  int bad;
};

// d = c 2^e with c in [1, 2) (exact) for a positive normal d below 2^1022; any other d (zero,
// negative, subnormal, huge, non-finite) gives c = 1, e = 0 (a plain step, which the pivot test
// rejects).  Integer operations only: on this part every FP64-pipe instruction, a compare or a
// conversion included, costs a warp ~64 cycles of issue.
__device__ __forceinline__ void pow2_split(double d, double& c, int& e) {
  const int hi = __double2hiint(d), lo = __double2loint(d);
  const bool ok = hi >= 0x00100000 && hi < 0x7fd00000;
  e = ok ? ((hi >> 20) & 0x7ff) - 1023 : 0;
  c = ok ? __hiloint2double((hi & 0x000fffff) | (1023 << 20), lo) : 1.0;
}

// t 2^-e by an exponent change, without a branch: exact for normal t whose result stays
// normal; a zero or subnormal t, or a result below the normal range, gives 0 (its share of an
// update is below 2^-1000 relative), a non-finite t stays non-finite (the pivot test then fails)
__device__ __forceinline__ double times_pow2(double t, int e) {
  const int hi = __double2hiint(t), lo = __double2loint(t);
  const int eb = (hi >> 20) & 0x7ff;
  const int nb = eb - e;
  const double moved = __hiloint2double(hi - e * (1 << 20), lo);
  const double scaled = (eb != 0 && nb >= 1 && nb <= 2046) ? moved : 0.0;
  return eb == 0x7ff ? t : scaled;
}

__device__ __forceinline__ void bar_sync_named(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// Cholesky factor L of the r x r symmetric matrix S (r <= RMAX <= 64) by threads 0..NT-1 of a CTA
// (NT a multiple of 32; all of them must call it, the other threads must not).  They
// synchronise among themselves with named barrier 1; the caller synchronises the rest of the
// block afterwards.  load(i, j) returns S_ij for i >= j.
// Writes L (FP32) transposed, LT[k * ldt + i] = L_ik for i >= k (entries above are not
// touched), invd[k] = 1 / L_kk (FP32) and, if L64 != nullptr, L in FP64 (L64[i * ld64 + k]).
// Returns false (the same value in every calling thread) when a pivot D_k = S^(k)_kk is not
// above tol (S not numerically positive definite); the outputs are then unspecified.
template <int NT, int RMAX, typename Load>
__device__ bool ldl_factor(int r, Load load, double tol, Smem& sm, float* LT, int ldt, float* invd, double* L64,
                           int ld64) {
  static_assert(RMAX <= kMaxR, "r x r factor up to 64");
  static_assert(NT >= 32 && NT % 32 == 0, "whole warps, warp 0 among them");
  // entries per thread for the largest r of this instantiation (the loops are unrolled over
  // them: a tight bound keeps the code, and the instruction cache misses, small)
  constexpr int MAXM = (RMAX * (RMAX + 1) / 2 + NT - 1) / NT;
  const int tid = threadIdx.x;
  const int N = r * (r + 1) / 2;
  double a[MAXM];
  int ii[MAXM], jj[MAXM];
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    const int e = tid + m * NT;
    ii[m] = 0;
    jj[m] = -1;
    a[m] = 0.0;
    if (e < N) {
      // columns from the last: column j = r-1-q holds entries e in [q(q+1)/2, (q+1)(q+2)/2)
      int q = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while (q > 0 && q * (q + 1) / 2 > e) --q;
      while ((q + 1) * (q + 2) / 2 <= e) ++q;
      const int j = r - 1 - q, i = j + (e - q * (q + 1) / 2);
      ii[m] = i;
      jj[m] = j;
      a[m] = load(i, j);
      if (j == 0) sm.col[0][i] = a[m];
    }
  }
  if (tid == 0) sm.bad = 0;
  bar_sync_named(1, NT);
  for (int k = 0; k < r; ++k) {
    const double* cb = sm.col[k & 1];
    double* nb = sm.col[(k + 1) & 1];
    const double d = cb[k];
    if (tid == 0) sm.dk[k] = d;
    double c;
    int ex;
    pow2_split(d, c, ex);
    const int nact = (r - k - 1) * (r - k) / 2;         // entries of columns > k: a prefix
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      if (m * NT < nact) {
        const bool act = tid + m * NT < nact;
        const double t = cb[act ? ii[m] : 0] * cb[act ? jj[m] : 0];
        const double v = fma(c, a[m], -times_pow2(t, ex));
        a[m] = act ? v : a[m];
        if (act && jj[m] == k + 1) nb[ii[m]] = v;
      }
    }
    bar_sync_named(1, NT);
  }
  // P_k = c_0 ... c_{k-1}, once: an exclusive product scan over the pivots' c (two per lane)
  if (tid < 32) {
    double c0 = 1.0, c1 = 1.0;
    int e_;
    if (2 * tid < r) pow2_split(sm.dk[2 * tid], c0, e_);
    if (2 * tid + 1 < r) pow2_split(sm.dk[2 * tid + 1], c1, e_);
    double incl = c0 * c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double v = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl *= v;
    }
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (tid == 0) excl = 1.0;
    if (2 * tid < kMaxR) sm.pk[2 * tid] = excl;
    if (2 * tid + 1 < kMaxR) sm.pk[2 * tid + 1] = excl * c0;
  }
  bar_sync_named(1, NT);
  if (tid < r) {
    const double dd = sm.dk[tid], pp = sm.pk[tid];
    const bool ok = dd > tol * pp;                       // D_k = dd / pp > tol (pp >= 1; false for NaN)
    sm.rs[tid] = ok ? rsqrt(dd * pp) : 0.0;
    if (!ok) sm.bad = 1;
    if (invd) invd[tid] = ok ? (float)(pp * sm.rs[tid]) : 0.f;
  }
  bar_sync_named(1, NT);
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    if (jj[m] >= 0) {
      const double l = a[m] * sm.rs[jj[m]];
      if (LT) LT[jj[m] * ldt + ii[m]] = (float)l;
      if (L64) L64[ii[m] * ld64 + jj[m]] = l;
    }
  }
  const bool ok = sm.bad == 0;
  bar_sync_named(1, NT);
  return ok;
}


// ---------------------------------------------------------------------------------------
// The batched FP64 r x r factor kernel (one CTA of four warps per matrix) and the apply of
// its inverse: the normal-equation solves of the local least-squares problem in its Gram
// form (Sec. 3.3: the inverses of A_k^T A_k and B_k B_k^T), used by the `lsq` and `noortho`
// modes of the generic path.
// ---------------------------------------------------------------------------------------
constexpr int kFactorThreads = 128;

// Matrix b of the batch: S_b = S + b * s_stride (row-major r x r, symmetric, the lower
// triangle is read).  Factors D S_b D = L' L'^T in FP64 with D = diag(S_b)^{-1/2} and writes
// the Cholesky factor of S_b, L = D^{-1} L' (row-major r x r, lower; L_b = L64 + b * 64 * 64)
// and rdiag_b[k] = 1 / L_kk (rdiag + b * 64).  A pivot of the scaled matrix at or below tol
// (a direction S_b does not determine) gets rdiag 0 and a zero column: the apply then drops
// that direction, a generalised inverse in place of S_b^{-1}.  bad[b] (if not null) = 1 when
// that happened.
template <typename TS, int RMAX>
__global__ void __launch_bounds__(kFactorThreads) k_r64_factor(const TS* __restrict__ S, long long s_stride, int r,
                                                              double tol, double* __restrict__ L64,
                                                              double* __restrict__ rdiag, int* __restrict__ bad) {
  __shared__ Smem sm;
  __shared__ double dsc[kMaxR];
  const int b = blockIdx.x, tid = threadIdx.x;
  const TS* Sb = S + (long long)b * s_stride;
  double* Lb = L64 + (long long)b * kMaxR * kMaxR;
  for (int e = tid; e < r * r; e += kFactorThreads) Lb[e] = 0.0;
  if (tid < r) {
    const double d = (double)Sb[tid * r + tid];
    dsc[tid] = d > 0.0 ? rsqrt(d) : 0.0;
  }
  __syncthreads();
  const auto load = [&](int i, int j) -> double { return (double)Sb[i * r + j] * dsc[i] * dsc[j]; };
  const bool ok = ldl_factor<kFactorThreads, RMAX>(r, load, tol, sm, nullptr, 0, nullptr, Lb, r);
  __syncthreads();
  // L = D^{-1} L' (rows scaled by sqrt(S_ii)); 1 / L_kk = dsc_k / L'_kk = dsc_k P_k rs_k
  for (int e = tid; e < r * r; e += kFactorThreads) {
    const int i = e / r;
    Lb[e] = dsc[i] > 0.0 ? Lb[e] / dsc[i] : 0.0;
  }
  if (tid < r) rdiag[(long long)b * kMaxR + tid] = dsc[tid] * sm.pk[tid] * sm.rs[tid];
  if (tid == 0 && bad) bad[b] = ok ? 0 : 1;
}

// v <- S^{-1} v for n vectors of length r (element i of vector t at V[t * vstride + i * estride])
// with S = L L^T from k_r64_factor: forward then backward substitution in FP64, one thread per
// vector, L in shared memory.  Returns at once when ctl->skip is set.
template <typename TV, int RMAX>
__global__ void __launch_bounds__(128) k_r64_apply(const double* __restrict__ L64, const double* __restrict__ rdiag,
                                                   int r, TV* __restrict__ V, long long n, long long vstride,
                                                   long long estride, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double L[RMAX * RMAX];
  __shared__ double rd[RMAX];
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) L[(e / r) * RMAX + e % r] = L64[e];
  if (threadIdx.x < r) rd[threadIdx.x] = rdiag[threadIdx.x];
  __syncthreads();
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    TV* v = V + t * vstride;
    double y[RMAX];
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
      if (i < r) {
        double acc = (double)v[i * estride];
#pragma unroll
        for (int k = 0; k < i; ++k) acc = fma(-L[i * RMAX + k], y[k], acc);
        y[i] = acc * rd[i];
      } else {
        y[i] = 0.0;
      }
    }
#pragma unroll
    for (int i = RMAX - 1; i >= 0; --i) {
      if (i < r) {
        double acc = y[i];
#pragma unroll
        for (int k = i + 1; k < RMAX; ++k)
          if (k < r) acc = fma(-L[k * RMAX + i], y[k], acc);
        y[i] = acc * rd[i];
        v[i * estride] = (TV)y[i];
      }
    }
  }
}

}  // namespace r64
