// ttals_kernels.cuh - device kernels of the Online TT-ALS update (arXiv 2606.31061).
//
// The update of Algorithm 1 is carried out in its gauge-reduced form (see ttals.cu):
//   Y   = E_k  B^_k^T      local solve, Eq. proposed-core-update (E_1 = X_t)
//   Q_k = orth(Y)          left orthogonalisation, Sec. 3.4.2
//   E_{k+1} = Q_k^T E_k    left interface A_{k+1}^T X_t
// Kernels here are generic over element types; the hot level-1 contraction has
// tensor-core specialisations in ttals_tc.cuh.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ttals {

// Compile-time phase tracing: with -DTTALS_TRACE, TTRACE(i) stores %globaltimer (ns)
// from thread 0 of the calling block into g_ttals_trace[i]; otherwise it is empty.
#ifdef TTALS_TRACE
__device__ unsigned long long g_ttals_trace[128];
#define TTRACE(i)                                                                  \
  do {                                                                             \
    if (threadIdx.x == 0) {                                                        \
      unsigned long long t_;                                                       \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                       \
      ::ttals::g_ttals_trace[(i)] = t_;                                            \
    }                                                                              \
  } while (0)
// TTRACE_CTA(k) / TTRACE_CTA2(k): per-CTA timestamps (slot k < 4) of up to 512 CTAs of
// two traced kernels (first and second half of the array)
__device__ unsigned long long g_ttals_cta[1024 * 4];
#define TTRACE_CTA_AT(base, k)                                                     \
  do {                                                                             \
    const unsigned b_ = blockIdx.y * gridDim.x + blockIdx.x;                       \
    if (threadIdx.x == 0 && b_ < 512) {                                            \
      unsigned long long t_;                                                       \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                       \
      ::ttals::g_ttals_cta[((base) + b_) * 4 + (k)] = t_;                          \
    }                                                                              \
  } while (0)
#define TTRACE_CTA(k) TTRACE_CTA_AT(0, k)
#define TTRACE_CTA2(k) TTRACE_CTA_AT(512, k)
#else
#define TTRACE(i) \
  do {            \
  } while (0)
#define TTRACE_CTA(k) \
  do {                \
  } while (0)
#define TTRACE_CTA2(k) \
  do {                 \
  } while (0)
#endif

// Programmatic dependent launch on the generic path: a kernel launched with the
// programmatic-serialisation attribute may start while its predecessor runs; it waits here
// for the predecessor's completion (and memory) before touching anything the step writes,
// and lets its own successor be scheduled at once.  Without the attribute both are no-ops.
__device__ __forceinline__ void gen_pdl_start() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// --------------------------------------------------------------------------
// control block shared by the kernels of one stream (device memory)
// --------------------------------------------------------------------------
constexpr int kMaxLevels = 8;
constexpr int kMaxSlots = 2 * kMaxLevels + 2;

struct Ctl {
  int skip;                   // the step in flight must not commit (non-finite data)
  int latched;                // sticky ttals_status code reported at the next sync
  int fallback[kMaxSlots];    // Householder path taken by orth slot s in this step
  long long t;                // committed steps
  double xx;                  // ||x_t||^2 of the step in flight / last committed step
  double ee;                  // ||x_t - x^_t||^2 of the last committed step
  double sum_xx, sum_ee;      // totals over committed steps
  double cc;                  // ||C||^2 of the committed state (C = collapsed right part)
};

// --------------------------------------------------------------------------
// element conversions
// --------------------------------------------------------------------------
template <typename T> struct Cvt;
template <> struct Cvt<double> {
  __device__ static double d(double x) { return x; }
  __device__ static float f(double x) { return (float)x; }
};
template <> struct Cvt<float> {
  __device__ static double d(float x) { return (double)x; }
  __device__ static float f(float x) { return x; }
};
template <> struct Cvt<__half> {
  __device__ static double d(__half x) { return (double)__half2float(x); }
  __device__ static float f(__half x) { return __half2float(x); }
};
template <> struct Cvt<__nv_bfloat16> {
  __device__ static double d(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
  __device__ static float f(__nv_bfloat16 x) { return __bfloat162float(x); }
};

template <typename TACC, typename T> __device__ __forceinline__ TACC cvt(T x);
template <> __device__ __forceinline__ double cvt<double, double>(double x) { return x; }
template <> __device__ __forceinline__ double cvt<double, float>(float x) { return (double)x; }
template <> __device__ __forceinline__ double cvt<double, __half>(__half x) { return Cvt<__half>::d(x); }
template <> __device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 x) { return Cvt<__nv_bfloat16>::d(x); }
template <> __device__ __forceinline__ float cvt<float, double>(double x) { return (float)x; }
template <> __device__ __forceinline__ float cvt<float, float>(float x) { return x; }
template <> __device__ __forceinline__ float cvt<float, __half>(__half x) { return __half2float(x); }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename TO> __device__ __forceinline__ TO from_acc(double x);
template <typename TO> __device__ __forceinline__ TO from_acc(float x);
template <> __device__ __forceinline__ double from_acc<double>(double x) { return x; }
template <> __device__ __forceinline__ double from_acc<double>(float x) { return (double)x; }
template <> __device__ __forceinline__ float from_acc<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ float from_acc<float>(float x) { return x; }
template <> __device__ __forceinline__ __half from_acc<__half>(double x) { return __double2half(x); }
template <> __device__ __forceinline__ __half from_acc<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(double x) { return __double2bfloat16(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// --------------------------------------------------------------------------
// block reductions
// --------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// sum over the block; every thread gets the result.  `sh` holds >= 32 doubles.
// Fixed-shape tree (warp shuffles, then one warp over the warp sums): deterministic,
// and the FP64 dependency chain stays at ~10 adds.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = (lane < nw) ? sh[lane] : 0.0;
  s = warp_sum(s);
  return s;
}

// --------------------------------------------------------------------------
// generic tiled GEMM (SIMT):  D[s](m, n) = sum_{k in split s} A(m,k) * B(k,n)
//   A(m,k) = A_KMAJ ? A[m*lda + k] : A[k*lda + m]
//   B(k,n) = B_KMAJ ? B[n*ldb + k] : B[k*ldb + n]
//   D[s](m,n) at D[s*split_stride + m*sdm + n*sdn]
// Optional: per-CTA sum of squares of A (CTAs with blockIdx.y == 0 see every A
// element once), written to sumsq[blockIdx.z*gridDim.x + blockIdx.x].
// Optional: b_zero_flag -> if *b_zero_flag == 0, B is replaced by e_0 e_0^T
// (the e_1 rule for a zero temporal row, applied to the collapsed right part).
// Optional: ctl -> returns at once when ctl->skip is set.
// --------------------------------------------------------------------------
constexpr int GB_M = 64, GB_N = 32, GB_K = 32, G_THREADS = 256;

template <typename TA, typename TB, typename TACC, typename TD, bool A_KMAJ, bool B_KMAJ>
__global__ void __launch_bounds__(G_THREADS) k_gemm(
    const TA* __restrict__ A, long long lda, const TB* __restrict__ B, long long ldb,
    TD* __restrict__ D, long long sdm, long long sdn, long long split_stride,
    int M, int N, long long K, long long kchunk, double* __restrict__ sumsq,
    const double* __restrict__ b_zero_flag, const Ctl* __restrict__ ctl, Ctl* __restrict__ reset) {
  gen_pdl_start();
  if (ctl && ctl->skip) return;
  if (reset && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
    reset->skip = 0;
    for (int i = 0; i < kMaxSlots; ++i) reset->fallback[i] = 0;
  }
  __shared__ TACC As[GB_K][GB_M + 1];
  __shared__ TACC Bs[GB_K][GB_N + 1];
  __shared__ double red[32];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.x * GB_M, n0 = blockIdx.y * GB_N;
  const long long kbeg = (long long)blockIdx.z * kchunk;
  const long long kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  const int tm = tid >> 4, tn = tid & 15;
  const bool bzero = b_zero_flag && (*b_zero_flag == 0.0);
  const bool do_ss = sumsq && blockIdx.y == 0;
  // Blocked, compensated accumulation: each k-tile's partial dot products are summed
  // in a fresh register, then added to the running sum with TwoSum (Knuth) so the
  // rounding error of a long chunk grows like that of one tile, not of the chunk.
  TACC acc[4][2], cmp[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = cmp[i][0] = cmp[i][1] = TACC(0);
  TACC ss = TACC(0);
  for (long long k0 = kbeg; k0 < kend; k0 += GB_K) {
    for (int e = tid; e < GB_M * GB_K; e += G_THREADS) {
      int mm, kk;
      if (A_KMAJ) { mm = e / GB_K; kk = e % GB_K; } else { kk = e / GB_M; mm = e % GB_M; }
      const int gm = m0 + mm;
      const long long gk = k0 + kk;
      TACC v = TACC(0);
      if (gm < M && gk < kend) v = cvt<TACC>(A_KMAJ ? A[(long long)gm * lda + gk] : A[gk * lda + gm]);
      As[kk][mm] = v;
      if (do_ss) ss += v * v;
    }
    for (int e = tid; e < GB_N * GB_K; e += G_THREADS) {
      int nn, kk;
      if (B_KMAJ) { nn = e / GB_K; kk = e % GB_K; } else { kk = e / GB_N; nn = e % GB_N; }
      const int gn = n0 + nn;
      const long long gk = k0 + kk;
      TACC v = TACC(0);
      if (gn < N && gk < kend) {
        if (bzero) v = (gn == 0 && gk == 0) ? TACC(1) : TACC(0);
        else v = cvt<TACC>(B_KMAJ ? B[(long long)gn * ldb + gk] : B[gk * ldb + gn]);
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
    TACC part[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) part[i][0] = part[i][1] = TACC(0);
#pragma unroll 8
    for (int kk = 0; kk < GB_K; ++kk) {
      TACC a[4], b[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tm * 4 + i];
      b[0] = Bs[kk][tn * 2];
      b[1] = Bs[kk][tn * 2 + 1];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        part[i][0] = fma(a[i], b[0], part[i][0]);
        part[i][1] = fma(a[i], b[1], part[i][1]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const TACC sum = acc[i][j] + part[i][j];
        const TACC bv = sum - acc[i][j];
        cmp[i][j] += (acc[i][j] - (sum - bv)) + (part[i][j] - bv);
        acc[i][j] = sum;
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] += cmp[i][0], acc[i][1] += cmp[i][1];
  TD* Ds = D + (long long)blockIdx.z * split_stride;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + tm * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gn = n0 + tn * 2 + j;
      if (gn < N) Ds[(long long)gm * sdm + (long long)gn * sdn] = from_acc<TD>(acc[i][j]);
    }
  }
  if (do_ss) {
    const double tot = block_sum((double)ss, red);
    if (tid == 0) sumsq[(long long)blockIdx.z * gridDim.x + blockIdx.x] = tot;
  }
}

// --------------------------------------------------------------------------
// Gram partials of a tall matrix.  Rows [b*rpb, (b+1)*rpb) of
//   Y = sum_{s < nsplit} P[s]     (P[s] is rows x r, element (i,j) at i*r + j)
// are formed (fixed summation order), optionally written to Yout, and
//   Wpart[b] = Y_b^T Y_b  (r x r, upper triangle; accumulated and stored in TG).
// FP32 partials P are summed as float-float pairs (TwoSum on the FP32 pipe: this part's FP64
// unit issues one warp instruction per ~64 cycles, which made FP64 sums of many partials the
// kernel's cost); FP64 partials in FP64.
// --------------------------------------------------------------------------
constexpr int GRAM_THREADS = 256;
constexpr int GRAM_CHUNK = 32;   // rows staged in shared memory at a time

template <typename TP, typename TY, typename TG>
__global__ void __launch_bounds__(GRAM_THREADS) k_gram(
    const TP* __restrict__ P, int nsplit, long long sstride, long long rows, int r,
    TY* __restrict__ Yout, TG* __restrict__ Wpart, long long rpb, const Ctl* __restrict__ ctl) {
  gen_pdl_start();
  if (ctl && ctl->skip) return;
  extern __shared__ unsigned char smem_raw[];
  TG* ys = reinterpret_cast<TG*>(smem_raw);               // GRAM_CHUNK x r
  const long long rbeg = (long long)blockIdx.x * rpb;
  const long long rend = (rbeg + rpb < rows) ? rbeg + rpb : rows;
  const int npair = r * r;
  // each thread owns up to 16 (i,j) entries (r <= 64)
  TG acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = TG(0);
  for (long long c0 = rbeg; c0 < rend; c0 += GRAM_CHUNK) {
    const int nr = (int)((c0 + GRAM_CHUNK < rend) ? GRAM_CHUNK : rend - c0);
    for (int e = threadIdx.x; e < nr * r; e += blockDim.x) {
      const long long gi = (c0 + e / r) * r + e % r;
      double v = 0.0;
      if constexpr (std::is_same<TP, float>::value) {
        float h = 0.f, l = 0.f;
        for (int s = 0; s < nsplit; ++s) {
          const float p = P[(long long)s * sstride + gi];
          const float t = h + p, bb = t - h;
          l += (h - (t - bb)) + (p - bb);
          h = t;
        }
        v = (double)h + (double)l;
      } else {
        for (int s = 0; s < nsplit; ++s) v += Cvt<TP>::d(P[(long long)s * sstride + gi]);
      }
      const TY yv = from_acc<TY>(v);
      if (Yout) Yout[gi] = yv;
      ys[e] = (TG)Cvt<TY>::d(yv);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = threadIdx.x + q * GRAM_THREADS;
      if (e >= npair) break;
      const int i = e / r, j = e % r;
      if (j < i) continue;
      TG a = acc[q];
      for (int row = 0; row < nr; ++row) a = fma(ys[row * r + i], ys[row * r + j], a);
      acc[q] = a;
    }
    __syncthreads();
  }
  TG* W = Wpart + (long long)blockIdx.x * npair;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = threadIdx.x + q * GRAM_THREADS;
    if (e < npair) W[e] = acc[q];
  }
}

// --------------------------------------------------------------------------
// r x r factor step (one CTA).  Sums the Gram partials in a fixed order, then
//   mode 0 (CHOL): D = diag(W)^(-1/2); S = chol(D W D) in FP32; T = D S^{-1}
//                  (any invertible T keeps span(Y T) = span(Y); this pass only
//                  has to make Y T well conditioned).  A scaled pivot <= 1e-4 or a
//                  non-positive diagonal selects the Householder fallback.
//                  (1e-4 bounds the orthogonality error of Y T by ~1e-3, which
//                  the POLAR pass then reduces to O(1e-10).)
//   mode 1 (POLAR): D = W - I; T = I - D/2 + 3/8 D^2, the second-order Taylor
//                  factor of W^{-1/2} (FP64; D^2 in FP32, which is exact to
//                  O(|D|^2 eps32)).  Y T is orthonormal to O(|D|^3).
// Outputs T64 (r x r FP64) and T32 (FP32; for mode 1 it holds T - I).
// When `first` is set it also sums the per-CTA ||x||^2 partials into ctl->xx and
// flags non-finite data (the step is then skipped, ENONFINITE latched).
// --------------------------------------------------------------------------
constexpr int FACT_THREADS = 256;
constexpr int kMaxRank = 64;

template <typename TW>
__global__ void __launch_bounds__(FACT_THREADS) k_factor(
    const TW* __restrict__ Wpart, int nblk, int r, int mode, double* __restrict__ T64,
    float* __restrict__ T32, Ctl* __restrict__ ctl, int slot, const double* __restrict__ sumsq,
    int nsum, int first) {
  gen_pdl_start();
  extern __shared__ unsigned char smem_raw[];
  double* W = reinterpret_cast<double*>(smem_raw);                 // r*r
  double* dsc = W + r * r;                                         // r
  float* S = reinterpret_cast<float*>(dsc + r);                    // r*(r+1)
  __shared__ double red[32];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (first) {
    double v = 0.0;
    for (int i = tid; i < nsum; i += blockDim.x) v += sumsq[i];
    const double xx = block_sum(v, red);
    if (tid == 0) {
      if (!isfinite(xx)) { ctl->skip = 1; ctl->latched = 4; }   // the committed ||x||^2 stays
      else ctl->xx = xx;
    }
    __syncthreads();
  }
  if (ctl->skip) return;
  const int rr = r * r;
  if (tid == 0) bad = 0;
  __syncthreads();
  // the upper triangle (i <= j), mirrored; each thread's loads of a batch of 8 partials are
  // issued together, then summed in block order
  for (int e = tid; e < rr; e += blockDim.x) {
    const int i = e / r, j = e % r;
    if (j < i) continue;
    double s = 0.0;
    if constexpr (std::is_same<TW, float>::value) {
      // float partials: float-float sum (TwoSum), one conversion at the end
      float h = 0.f, l = 0.f;
      for (int b0 = 0; b0 < nblk; b0 += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = b0 + q < nblk ? Wpart[(long long)(b0 + q) * rr + e] : 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float t = h + v[q], bb = t - h;
          l += (h - (t - bb)) + (v[q] - bb);
          h = t;
        }
      }
      s = (double)h + (double)l;
    } else {
      for (int b0 = 0; b0 < nblk; b0 += 8) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = b0 + q < nblk ? (double)Wpart[(long long)(b0 + q) * rr + e] : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) s += v[q];
      }
    }
    W[e] = s;
    W[j * r + i] = s;
    if (!isfinite(s)) bad = 1;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) { ctl->skip = 1; ctl->latched = 4; }
    return;
  }
  if (mode == 1) {
    // T = I - D/2 + 3/8 D^2 with D = W - I
    for (int e = tid; e < rr; e += blockDim.x) {
      const int i = e / r, j = e % r;
      S[i * (r + 1) + j] = (float)(W[e] - (i == j ? 1.0 : 0.0));
    }
    __syncthreads();
    for (int e = tid; e < rr; e += blockDim.x) {
      const int i = e / r, j = e % r;
      float d2 = 0.f;
      for (int k = 0; k < r; ++k) d2 = fmaf(S[i * (r + 1) + k], S[k * (r + 1) + j], d2);
      const double dm = W[e] - (i == j ? 1.0 : 0.0);
      const double tmi = -0.5 * dm + 0.375 * (double)d2;      // T - I
      T64[e] = (i == j ? 1.0 : 0.0) + tmi;
      T32[e] = (float)tmi;
    }
    return;
  }
  // mode 0: scaled FP32 Cholesky  S = chol(D W D),  upper triangular, S^T S = D W D
  if (tid < r) {
    const double d = W[tid * r + tid];
    dsc[tid] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    if (!(d > 0.0)) bad = 1;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) ctl->fallback[slot] = 1;
    return;
  }
  const int LD = r + 1;
  for (int e = tid; e < rr; e += blockDim.x) {
    const int i = e / r, j = e % r;
    S[i * LD + j] = (float)(W[e] * dsc[i] * dsc[j]);
  }
  __syncthreads();
  // right-looking LDL^T elimination with one barrier per pivot (S's rows keep the unscaled
  // pivot rows); the pivot's reciprocal is the hardware approximation refined by one Newton
  // step (about 1e-7 relative).  The same row operations applied to the identity build the
  // unit lower factor's inverse Li = L_u^{-1} alongside, so that with S = L_u D_p L_u^T and
  // R = D_p^{1/2} L_u^T (R^T R = D W D): T = D R^{-1} = D L_u^{-T} D_p^{-1/2}.
  __shared__ float rs[kMaxRank];                // 1 / sqrt(pivot j)
  float* Li = reinterpret_cast<float*>(W);      // r x r (W is not needed any more)
  for (int e = tid; e < rr; e += blockDim.x) Li[e] = (e / r == e % r) ? 1.f : 0.f;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    const float piv = S[j * LD + j];
    if (!(piv > 1e-4f)) {            // uniform: every thread reads the same value
      if (tid == 0) ctl->fallback[slot] = 1;
      return;
    }
    float inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(piv));
    inv = inv * fmaf(-piv, inv, 2.0f);
    if (tid == 0) rs[j] = rsqrtf(piv);
    // on a 16 x 16 thread grid (no integer division in the loops): the trailing update of S
    // (rows i > j, columns k >= i) and the inverse rows i > j (columns c <= j)
    for (int i = j + 1 + (tid >> 4); i < r; i += FACT_THREADS / 16) {
      const float sji = S[j * LD + i] * inv;
      for (int k = j + 1 + (tid & 15); k < r; k += 16)
        if (k >= i) S[i * LD + k] = fmaf(-sji, S[j * LD + k], S[i * LD + k]);
      for (int c = tid & 15; c <= j; c += 16) Li[i * r + c] = fmaf(-sji, Li[j * r + c], Li[i * r + c]);
    }
    __syncthreads();
  }
  // T[k][i] = dsc_k Li[i][k] rs_i (upper triangular)
  for (int e = tid; e < rr; e += blockDim.x) {
    const int k = e / r, i = e % r;
    const double t = i >= k ? dsc[k] * (double)(Li[i * r + k] * rs[i]) : 0.0;
    T64[e] = t;
    T32[e] = (float)t;
  }
}

// --------------------------------------------------------------------------
// Householder QR with completion (one CTA, FP64; Golub & Van Loan Alg. 5.2.1).
//   M: rows x p (row-major), p <= r_out <= rows.  Output Q: rows x r_out with
//   Q[:, :p] R = M, diag(R) >= 0, and Q[:, p:] = H_1..H_p e_j (completion).
//   A pivot column whose remaining norm is <= 64 eps ||M||_F is left unreflected.
// work: 2 * rows * p doubles.
// --------------------------------------------------------------------------
constexpr int HH_THREADS = 512;

template <typename TIN, typename TOUT>
__device__ void householder_cta(const TIN* __restrict__ M, long long rows, int p, int r_out,
                                double* __restrict__ work, TOUT* __restrict__ Q, long long ldq,
                                double* red) {
  __shared__ int skipcol[kMaxRank * 4];
  __shared__ double sgn[kMaxRank * 4];
  double* A = work;                    // rows x p
  double* V = work + rows * p;         // rows x p (column j = reflector j)
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  double ss = 0.0;
  for (long long e = tid; e < rows * p; e += blockDim.x) {
    const double v = Cvt<TIN>::d(M[e]);
    A[e] = v;
    ss += v * v;
  }
  const double thresh = 64.0 * 2.220446049250313e-16 * sqrt(block_sum(ss, red));
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    double s = 0.0;
    for (long long i = j + tid; i < rows; i += blockDim.x) s += A[i * p + j] * A[i * p + j];
    const double nx = sqrt(block_sum(s, red));
    const double x0 = A[(long long)j * p + j];
    if (nx <= thresh) {
      if (tid == 0) skipcol[j] = 1;
      __syncthreads();
      continue;
    }
    if (tid == 0) skipcol[j] = 0;
    const double alpha = -copysign(nx, x0);
    const double vn = sqrt(2.0 * nx * (nx + fabs(x0)));
    for (long long i = j + tid; i < rows; i += blockDim.x)
      V[i * p + j] = (i == j ? x0 - alpha : A[i * p + j]) / vn;
    __syncthreads();
    for (int c = j + wid; c < p; c += nw) {
      double d = 0.0;
      for (long long i = j + lane; i < rows; i += 32) d += V[i * p + j] * A[i * p + c];
      d = warp_sum(d);
      for (long long i = j + lane; i < rows; i += 32) A[i * p + c] -= 2.0 * V[i * p + j] * d;
    }
    __syncthreads();
  }
  for (int j = tid; j < p; j += blockDim.x) sgn[j] = A[(long long)j * p + j] < 0.0 ? -1.0 : 1.0;
  __syncthreads();
  // Q = H_1 ... H_p I[:, :r_out], formed in batches of p columns in the FP64 buffer A
  for (int c0 = 0; c0 < r_out; c0 += p) {
    const int nb = (r_out - c0 < p) ? r_out - c0 : p;
    for (long long e = tid; e < rows * p; e += blockDim.x) {
      const long long i = e / p;
      const int cc = (int)(e % p);
      A[e] = (cc < nb && i == c0 + cc) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = p - 1; j >= 0; --j) {
      if (skipcol[j]) continue;
      for (int cc = wid; cc < nb; cc += nw) {
        double d = 0.0;
        for (long long i = j + lane; i < rows; i += 32) d += V[i * p + j] * A[i * p + cc];
        d = warp_sum(d);
        for (long long i = j + lane; i < rows; i += 32) A[i * p + cc] -= 2.0 * V[i * p + j] * d;
      }
      __syncthreads();
    }
    for (long long e = tid; e < rows * nb; e += blockDim.x) {
      const long long i = e / nb;
      const int cc = (int)(e % nb);
      const int c = c0 + cc;
      const double s = c < p ? sgn[c] : 1.0;
      Q[i * ldq + c] = from_acc<TOUT>(s * A[i * p + cc]);
    }
    __syncthreads();
  }
}

template <typename TIN, typename TOUT>
__global__ void __launch_bounds__(HH_THREADS) k_householder(
    const TIN* __restrict__ M, long long rows, int p, int r_out, double* __restrict__ work,
    TOUT* __restrict__ Q, long long ldq) {
  __shared__ double red[32];
  householder_cta<TIN, TOUT>(M, rows, p, r_out, work, Q, ldq, red);
}

// --------------------------------------------------------------------------
// apply the r x r factor to a tall matrix:  Q[rows] = Y[rows] T
//   mode 0: T upper triangular (T64 / T32);  mode 1: Q = Y + Y (T - I).
// If the factor step chose the Householder fallback, block 0 computes the
// Householder Q of Y instead (rank-deficient or badly conditioned Y).
// --------------------------------------------------------------------------
constexpr int APPLY_THREADS = 256;

template <typename TQ>
__global__ void __launch_bounds__(APPLY_THREADS) k_apply(
    const TQ* __restrict__ Y, long long rows, int r, int mode, const double* __restrict__ T64,
    const float* __restrict__ T32, TQ* __restrict__ Qout, const Ctl* __restrict__ ctl, int slot,
    double* __restrict__ hh_work) {
  gen_pdl_start();
  if (ctl->skip) return;
  if (ctl->fallback[slot]) {
    if (blockIdx.x == 0) {
      __shared__ double red[32];
      householder_cta<TQ, TQ>(Y, rows, r, r, hh_work, Qout, r, red);
    }
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  TQ* Ts = reinterpret_cast<TQ*>(smem_raw);
  const int rr = r * r;
  for (int e = threadIdx.x; e < rr; e += blockDim.x) {
    const int i = e / r, j = e % r;
    if (sizeof(TQ) == 8) Ts[e] = (TQ)(mode == 1 ? T64[e] - (i == j ? 1.0 : 0.0) : T64[e]);
    else Ts[e] = (TQ)T32[e];
  }
  __syncthreads();
  const long long total = rows * r;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / r;
    const int j = (int)(e % r);
    const TQ* y = Y + i * r;
    TQ s = TQ(0);
    if (mode == 0) {
      for (int k = 0; k <= j; ++k) s = fma(y[k], Ts[k * r + j], s);
    } else {
      for (int k = 0; k < r; ++k) s = fma(y[k], Ts[k * r + j], s);
      s += y[j];
    }
    Qout[e] = s;
  }
}

// --------------------------------------------------------------------------
// out[a][j] = sum_s P[s][j][a]   (transpose-reduce of split partials; r x rest)
// plus per-CTA partials of sum(out^2) when ccpart != nullptr.  Tiles of 32 values of j
// (all r values of a) are read along P's rows and written along out's rows through shared
// memory, so that both sides are coalesced.  FP32 partials are summed as float-float pairs
// (TwoSum, and TwoProd for the squares) on the FP32 pipe, FP64 ones in FP64; each in split
// order.
// --------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

template <typename TC>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_t(
    const TC* __restrict__ P, int nsplit, long long sstride, long long rest, int r,
    TC* __restrict__ out, double* __restrict__ ccpart, const Ctl* __restrict__ ctl) {
  gen_pdl_start();
  if (ctl && ctl->skip) return;
  __shared__ double red[32];
  __shared__ TC tile[32 * 65];          // 32 values of j x r (<= 64) values of a, rows padded
  const int ld = r + 1;
  double ss = 0.0;
  float sh = 0.f, sl = 0.f;             // float-float sum of squares (FP32 partials)
  const long long ntile = (rest + 31) / 32;
  for (long long t = blockIdx.x; t < ntile; t += gridDim.x) {
    const long long j0 = t * 32;
    const int nj = (int)(rest - j0 < 32 ? rest - j0 : 32);
    for (int q = threadIdx.x; q < nj * r; q += blockDim.x) {
      const long long e = j0 * r + q;
      TC o;
      if constexpr (std::is_same<TC, float>::value) {
        float h = 0.f, l = 0.f;
        for (int s = 0; s < nsplit; ++s) {
          const float p = P[(long long)s * sstride + e];
          const float u = h + p, bb = u - h;
          l += (h - (u - bb)) + (p - bb);
          h = u;
        }
        o = h + l;
        const float pr = o * o, pe = fmaf(o, o, -pr);
        const float u = sh + pr, bb = u - sh;
        sl += ((sh - (u - bb)) + (pr - bb)) + pe;
        sh = u;
      } else {
        double v = 0.0;
        for (int s = 0; s < nsplit; ++s) v += Cvt<TC>::d(P[(long long)s * sstride + e]);
        o = from_acc<TC>(v);
        const double od = Cvt<TC>::d(o);
        ss += od * od;
      }
      tile[(q / r) * ld + q % r] = o;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < r * 32; q += blockDim.x) {
      const int a = q / 32, jl = q % 32;
      if (jl < nj) out[(long long)a * rest + j0 + jl] = tile[jl * ld + a];
    }
    __syncthreads();
  }
  if (ccpart) {
    if constexpr (std::is_same<TC, float>::value) ss = (double)sh + (double)sl;
    const double tot = block_sum(ss, red);
    if (threadIdx.x == 0) ccpart[blockIdx.x] = tot;
  }
}

// First level of a split-K reduction for many splits: out[q][e] = the sum over the splits
// s in [q G, min(nsplit, (q + 1) G)) of P[s][e], in split order (float-float pairs for FP32,
// FP64 sums for FP64), one thread per (q, e): cdiv(nsplit, G) times the threads of a
// per-element sum, for outputs too small to occupy the GPU otherwise.
template <typename TC>
__global__ void k_reduce_split_groups(const TC* __restrict__ P, int nsplit, int G, long long n,
                                      TC* __restrict__ out, const Ctl* __restrict__ ctl) {
  gen_pdl_start();
  if (ctl && ctl->skip) return;
  const int ng = (nsplit + G - 1) / G;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)ng * n;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / n);
    const long long e = t - (long long)q * n;
    const int s1 = (q + 1) * G < nsplit ? (q + 1) * G : nsplit;
    if constexpr (std::is_same<TC, float>::value) {
      float h = 0.f, l = 0.f;
      for (int s = q * G; s < s1; ++s) {
        const float p = P[(long long)s * n + e];
        const float u = h + p, bb = u - h;
        l += (h - (u - bb)) + (p - bb);
        h = u;
      }
      out[t] = h + l;
    } else {
      double v = 0.0;
      for (int s = q * G; s < s1; ++s) v += Cvt<TC>::d(P[(long long)s * n + e]);
      out[t] = from_acc<TC>(v);
    }
  }
}

// out = sum of nsplit partial matrices (n elements each, split stride n), in split order
template <typename TC>
__global__ void k_reduce_rows(const TC* __restrict__ P, int nsplit, long long n, TC* __restrict__ out,
                              const Ctl* __restrict__ ctl) {
  if (ctl && ctl->skip) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<TC, float>::value) {
      float h = 0.f, l = 0.f;           // float-float (TwoSum), as in k_reduce_t
      for (int q = 0; q < nsplit; ++q) {
        const float p = P[(long long)q * n + e];
        const float u = h + p, bb = u - h;
        l += (h - (u - bb)) + (p - bb);
        h = u;
      }
      out[e] = h + l;
    } else {
      double v = 0.0;
      for (int q = 0; q < nsplit; ++q) v += Cvt<TC>::d(P[(long long)q * n + e]);
      out[e] = from_acc<TC>(v);
    }
  }
}

// ||x||^2 of the step from the level-1 solve's per-CTA partials (the Gram-form modes, which
// have no level-1 factor kernel to do it); a non-finite sum marks the step skipped
// (ENONFINITE latched) and keeps the committed value
__global__ void k_sum_xx(const double* __restrict__ sumsq, int nsum, Ctl* __restrict__ ctl) {
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nsum; i += blockDim.x) v += sumsq[i];
  const double xx = block_sum(v, red);
  if (threadIdx.x == 0) {
    if (!isfinite(xx)) { ctl->skip = 1; ctl->latched = 4; }
    else ctl->xx = xx;
  }
}

// per-CTA partials of <a, b> (FP64), written to part[blockIdx.x]
template <typename TC>
__global__ void k_dot_part(const TC* __restrict__ a, const TC* __restrict__ b, long long n, double* __restrict__ part,
                           const Ctl* __restrict__ ctl) {
  __shared__ double red[32];
  double ss = 0.0;
  if (!(ctl && ctl->skip))
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
      ss += Cvt<TC>::d(a[e]) * Cvt<TC>::d(b[e]);
  const double tot = block_sum(ss, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// --------------------------------------------------------------------------
// saturated first level (k* = 1: r_1 >= I_2...I_{n-1}): the state is the slice itself.
// --------------------------------------------------------------------------
template <typename TX, typename TC>
__global__ void k_copy_slice(const TX* __restrict__ X, long long n, TC* __restrict__ C,
                             double* __restrict__ ccpart, Ctl* __restrict__ reset) {
  gen_pdl_start();
  if (reset && blockIdx.x == 0 && threadIdx.x == 0) {
    reset->skip = 0;
    for (int i = 0; i < kMaxSlots; ++i) reset->fallback[i] = 0;
  }
  __shared__ double red[32];
  double ss = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = Cvt<TX>::d(X[e]);
    C[e] = from_acc<TC>(v);
    ss += v * v;
  }
  const double tot = block_sum(ss, red);
  if (threadIdx.x == 0) ccpart[blockIdx.x] = tot;
}

// --------------------------------------------------------------------------
// commit (one CTA): fold the step into the running statistics, or, if the step
// was skipped, restore the new state buffers from the old ones.
// --------------------------------------------------------------------------
struct CopyList {
  const void* src[kMaxLevels + 1];
  void* dst[kMaxLevels + 1];
  long long bytes[kMaxLevels + 1];
  int n;
};

__global__ void k_commit(Ctl* __restrict__ ctl, const double* __restrict__ ccpart, int ncc,
                         const double* __restrict__ xxpart, int nxx, CopyList restore) {
  gen_pdl_start();
  __shared__ double red[32];
  if (xxpart) {        // k* = 1: ||x||^2 comes from the copy kernel
    double v = 0.0;
    for (int i = threadIdx.x; i < nxx; i += blockDim.x) v += xxpart[i];
    const double xx = block_sum(v, red);
    if (threadIdx.x == 0) {
      ctl->xx = xx;
      if (!isfinite(xx)) { ctl->skip = 1; ctl->latched = 4; }
    }
    __syncthreads();
  }
  if (ctl->skip) {
    for (int q = 0; q < restore.n; ++q) {
      const uint8_t* s = (const uint8_t*)restore.src[q];
      uint8_t* d = (uint8_t*)restore.dst[q];
      for (long long b = threadIdx.x; b < restore.bytes[q]; b += blockDim.x) d[b] = s[b];
    }
    return;
  }
  double v = 0.0;
  for (int i = threadIdx.x; i < ncc; i += blockDim.x) v += ccpart[i];
  const double cc = block_sum(v, red);
  if (threadIdx.x == 0) {
    if (!isfinite(cc)) {          // overflow inside the update: keep the old state
      ctl->skip = 1;
      ctl->latched = 4;
    } else {
      const double ee = ctl->xx - cc > 0.0 ? ctl->xx - cc : 0.0;
      ctl->cc = cc;
      ctl->ee = ee;
      ctl->sum_xx += ctl->xx;
      ctl->sum_ee += ee;
      ctl->t += 1;
    }
  }
  __syncthreads();
  if (ctl->skip) {
    for (int q = 0; q < restore.n; ++q) {
      const uint8_t* s = (const uint8_t*)restore.src[q];
      uint8_t* d = (uint8_t*)restore.dst[q];
      for (long long b = threadIdx.x; b < restore.bytes[q]; b += blockDim.x) d[b] = s[b];
    }
  }
}

// element-wise conversion with a stride-1 layout
template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ in, TO* __restrict__ out, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = from_acc<TO>(Cvt<TI>::d(in[e]));
}

// sum of squares of a vector into ctl->cc (one CTA); used after set_cores
template <typename TC>
__global__ void k_norm2_to_cc(const TC* __restrict__ c, long long n, Ctl* __restrict__ ctl) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    const double v = Cvt<TC>::d(c[e]);
    s += v * v;
  }
  const double tot = block_sum(s, red);
  if (threadIdx.x == 0) ctl->cc = tot;
}

// 8-bit pixels -> the ingest type (exact: every integer 0..255 is representable in FP16,
// BF16 and FP32).  16 bytes loaded per thread and step, grid-stride; the tail of n % 16
// elements is handled element by element by the thread that owns the last chunk.
template <typename TD>
__global__ void __launch_bounds__(256) k_widen_u8(const uint8_t* __restrict__ src, TD* __restrict__ dst, long long n) {
  const long long n16 = n / 16;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n16; c += (long long)gridDim.x * blockDim.x) {
    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(src) + c);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    TD o[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) o[q] = from_acc<TD>((float)((w[q >> 2] >> (8 * (q & 3))) & 0xffu));
    constexpr int NQ = (int)sizeof(TD);            // 16-byte chunks of 16 outputs
    uint4* d = reinterpret_cast<uint4*>(dst + c * 16);
#pragma unroll
    for (int q = 0; q < NQ; ++q) d[q] = reinterpret_cast<const uint4*>(o)[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (long long e = n16 * 16; e < n; ++e) dst[e] = from_acc<TD>((float)src[e]);
}

}  // namespace ttals
