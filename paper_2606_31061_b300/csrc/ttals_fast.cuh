// ttals_fast.cuh - fused update for streams whose first level saturates the trailing
// modes (k* = 2: 3rd-order streams and the video-shaped stream) with FP16 / BF16
// slices.  One step of Algorithm 1 is three kernels chained by programmatic
// dependent launch:
//
//   K1  (solve):  Y = X_(1) B^T          (local solve, Eq. proposed-core-update, k = 1),
//                 per-tile Gram partials of W1 = Y^T Y and ||x||^2
//   K1b (factor): S = chol(D W1 D) in FP32, Q1 = Y D S^{-1} (left orthogonalisation,
//                 Sec. 3.4.2), W2 = Q1^T Q1 and Nx = W2^{-1} - I
//   K2  (env):    F  = Q1^T X_(1)        (left interface A_2^T X_t = the collapsed right
//                 part of the new state), ||x^||^2 = sum_j f_j^T (I + Nx) f_j
//
// Q1 is orthonormal up to rounding; every quantity that needs the exact orthogonal
// projector uses W2 (x^ = Q1 W2^{-1} F), and the next step needs only the row space
// of F (B = F is a left gauge of the orthonormal-gauge C = R2^{-T} F, R2 = chol(W2)).
//
// The slice is staged through the TMA engine (cp.async.bulk + mbarrier, bounded
// waits) into padded shared-memory rows; tensor cores run mma.sync.m16n8k16
// (f16/bf16 -> f32) fed by ldmatrix; thread-block clusters reduce split partial sums
// through distributed shared memory in a fixed order (deterministic).
#pragma once

#include <cuda.h>

#include "ttals_kernels.cuh"

namespace ttals {
namespace fast {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldsm_x4(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t a, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t a, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

template <typename TX>
__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, uint32_t b0, uint32_t b1);
template <>
__device__ __forceinline__ void mma16816<__half>(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma16816<__nv_bfloat16>(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// squares of the 8 halves packed in an A fragment
template <typename TX>
__device__ __forceinline__ float frag_sumsq(const uint32_t* a) {
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 v;
    if constexpr (std::is_same<TX, __half>::value) {
      v = __half22float2(*reinterpret_cast<const __half2*>(&a[i]));
    } else {
      v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&a[i]));
    }
    s = fmaf(v.x, v.x, s);
    s = fmaf(v.y, v.y, s);
  }
  return s;
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ uint32_t dsmem_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ float dsmem_ld_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];\n" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ double dsmem_ld_f64(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];\n" : "=d"(v) : "r"(a) : "memory");
  return v;
}
// programmatic dependent launch: wait for the preceding kernel's results
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// compensated addition (TwoSum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}

// mbarrier and bulk-copy (TMA) helpers -----------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on an mbarrier phase: gives up after ~100 ms and returns false (the
// caller latches TTALS_ETIMEOUT); no wait in this library is unbounded.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 100000000ull) return false;
  }
}
// 1-D bulk copy global -> shared (TMA engine); 16-byte aligned addresses, size % 16 == 0
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// sum of n (<= 8) values loaded from distributed shared memory, loads issued together
__device__ __forceinline__ float dsmem_sum8(uint32_t local_addr, int n) {
  float v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = (q < n) ? dsmem_ld_f32(dsmem_addr(local_addr, q)) : 0.f;
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += v[q];
  return s;
}

// 2-D tensor copy (TMA) global -> shared, box at element coordinates (x inner, y outer)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// byte offset of 16-byte chunk c of row `row` in a 128B-swizzled box (1024-byte aligned)
__device__ __forceinline__ uint32_t swz(int row, int c) { return (uint32_t)(row * 128 + ((c ^ (row & 7)) << 4)); }

// ================================================================ K1: local solve
// Y = X_(1) B^T for one 64-row tile of X and a k-split; the splits of a row tile form a
// thread-block cluster and reduce their partial tiles through distributed shared memory
// (fixed rank order).  Also per-cluster partials of ||x||^2 and of the Gram W1 = Y^T Y.
// X and B arrive as 64 x 64 (resp. NP x 64) boxes through the TMA engine, 128B-swizzled,
// out-of-range rows and columns zero-filled by the hardware.
constexpr int K1_THREADS = 256;
constexpr int K1_BM = 64;          // rows of X per CTA
constexpr int K1_BK = 64;          // k per pipeline stage (128 bytes of a row)
constexpr int K1_STAGES = 6;

struct SolveArgs {
  int M, r;
  long long K, kchunk;    // kchunk % 64 == 0
  float* Y;               // M x r
  float* gram_part;       // [row tiles][r*r]
  double* xx_part;        // [row tiles]
  Ctl* ctl;
};

template <int NP>
__host__ __device__ constexpr size_t k1_stage_bytes() {
  return (size_t)(K1_BM + NP) * 128;
}
template <int NP>
__host__ __device__ constexpr size_t k1_smem_bytes() {
  return (size_t)K1_STAGES * k1_stage_bytes<NP>() + 1024;   // + alignment slack
}

template <typename TX, int NP>
__global__ void __launch_bounds__(K1_THREADS, 2)
    k_fast_solve(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, SolveArgs a) {
  static_assert(NP % 16 == 0 && NP >= 16 && NP <= 64, "NP");
  constexpr int NT = NP / 16;  // n8-tiles per warp (each warp covers NP/2 columns)
  constexpr uint32_t ABYTES = K1_BM * 128, BBYTES = NP * 128;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bars[K1_STAGES];
  __shared__ double red[32];
  __shared__ double ss_sh;
  __shared__ int timeout_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wr = warp & 3, wc = warp >> 2;
  const uint32_t crank = cluster_rank();
  const int nsplit = gridDim.y;
  const int rt = blockIdx.x;
  const int m0 = rt * K1_BM;
  const int r = a.r, rr = r * r;
  const long long kbeg = (long long)blockIdx.y * a.kchunk;
  const long long kend = (kbeg + a.kchunk < a.K) ? kbeg + a.kchunk : a.K;
  const int ntk = kend > kbeg ? (int)((kend - kbeg + K1_BK - 1) / K1_BK) : 0;
  const bool tr0 = (blockIdx.x == 0 && blockIdx.y == 0);
  const uint32_t sbase = smem_u32(smem);
  auto stageA = [&](int st) { return sbase + (uint32_t)(st * k1_stage_bytes<NP>()); };
  auto stageB = [&](int st) { return stageA(st) + ABYTES; };

  if (tid == 0) {
    for (int s = 0; s < K1_STAGES; ++s) mbar_init(smem_u32(&bars[s]), 2);   // A arrival + B arrival
    mbar_fence_init();
    timeout_flag = 0;
  }
  __syncthreads();
  if (tr0) TTRACE(0);
  // A tiles do not depend on the previous kernel: start them before the dependency wait
  if (tid == 0) {
    for (int t = 0; t < K1_STAGES && t < ntk; ++t) {
      const uint32_t bar = smem_u32(&bars[t]);
      mbar_arrive_expect_tx(bar, ABYTES);
      tma_load_2d(stageA(t), &tmX, (int)(kbeg + (long long)t * K1_BK), m0, bar);
    }
  }
  pdl_wait();       // the previous step's env kernel wrote B and ctl
  pdl_trigger();    // the factor kernel may launch and wait for this grid
  const bool bzero = (a.ctl->cc == 0.0);
  if (tid == 0) {
    for (int t = 0; t < K1_STAGES && t < ntk; ++t) {
      const uint32_t bar = smem_u32(&bars[t]);
      if (bzero) {
        mbar_arrive_expect_tx(bar, 0);
      } else {
        mbar_arrive_expect_tx(bar, BBYTES);
        tma_load_2d(stageB(t), &tmB, (int)(kbeg + (long long)t * K1_BK), 0, bar);
      }
    }
  }
  if (bzero) {
    // e_1 rule for a zero temporal row: the right part becomes e_0 e_0^T
    for (int st = 0; st < K1_STAGES; ++st)
      for (int e = tid; e < (int)BBYTES / 16; e += K1_THREADS)
        *reinterpret_cast<uint4*>(smem + (stageB(st) - sbase) + e * 16) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    if (blockIdx.y == 0 && tid == 0) *reinterpret_cast<TX*>(smem + (stageB(0) - sbase)) = from_acc<TX>(1.0f);
  }
  __syncthreads();

  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  double ssd = 0.0;
  for (int t = 0; t < ntk; ++t) {
    const int st = t % K1_STAGES;
    if (!mbar_wait(smem_u32(&bars[st]), (uint32_t)((t / K1_STAGES) & 1))) timeout_flag = 1;
    const uint32_t tA = stageA(st), tB = stageB(st);
    float ss = 0.f;
#pragma unroll
    for (int kk = 0; kk < K1_BK / 16; ++kk) {
      uint32_t af[4];
      {
        const int row = wr * 16 + (lane & 15);
        ldsm_x4(tA + swz(row, kk * 2 + (lane >> 4)), af[0], af[1], af[2], af[3]);
      }
      if (wc == 0) ss += frag_sumsq<TX>(af);
#pragma unroll
      for (int p = 0; p < NT / 2; ++p) {
        uint32_t b0, b1, b2, b3;
        const int n = wc * (NP / 2) + p * 16 + (lane & 7) + ((lane >> 4) << 3);
        ldsm_x4(tB + swz(n, kk * 2 + ((lane >> 3) & 1)), b0, b1, b2, b3);
        mma16816<TX>(acc[2 * p], af, b0, b1);
        mma16816<TX>(acc[2 * p + 1], af, b2, b3);
      }
      if constexpr (NT % 2 == 1) {
        uint32_t b0, b1;
        const int n = wc * (NP / 2) + (NT - 1) * 8 + (lane & 7);
        ldsm_x2(tB + swz(n, kk * 2 + ((lane >> 3) & 1)), b0, b1);
        mma16816<TX>(acc[NT - 1], af, b0, b1);
      }
    }
    ssd += (double)ss;
    __syncthreads();          // every warp is done with stage st
    if (t == 0 && bzero && blockIdx.y == 0 && tid == 0)
      *reinterpret_cast<TX*>(smem + (stageB(0) - sbase)) = from_acc<TX>(0.f);
    if (tid == 0 && t + K1_STAGES < ntk) {
      const int tn = t + K1_STAGES;
      const uint32_t bar = smem_u32(&bars[st]);
      mbar_arrive_expect_tx(bar, ABYTES);
      tma_load_2d(stageA(st), &tmX, (int)(kbeg + (long long)tn * K1_BK), m0, bar);
      if (bzero) {
        mbar_arrive_expect_tx(bar, 0);
      } else {
        mbar_arrive_expect_tx(bar, BBYTES);
        tma_load_2d(stageB(st), &tmB, (int)(kbeg + (long long)tn * K1_BK), 0, bar);
      }
    }
  }
  if (tr0) TTRACE(1);
  // ---- partial tile -> shared memory P[BM][NP] (fp32), reusing the pipeline buffers
  float* P = reinterpret_cast<float*>(smem);
  {
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int col = wc * (NP / 2) + j * 8 + 2 * t4;
      const int row = wr * 16 + g;
      P[row * NP + col] = acc[j][0];
      P[row * NP + col + 1] = acc[j][1];
      P[(row + 8) * NP + col] = acc[j][2];
      P[(row + 8) * NP + col + 1] = acc[j][3];
    }
  }
  const double ss_cta = block_sum(ssd, red);
  float* Gs = P + K1_BM * NP;            // r x r Gram partial of this CTA's rows
  float* Ym = Gs + rr;                   // my reduced rows [rpc][r]
  if (tid == 0) {
    ss_sh = ss_cta;
    if (timeout_flag) a.ctl->latched = 5;
  }
  cluster_sync();
  if (tr0) TTRACE(2);
  // ---- rank q reduces rows [q*rpc, (q+1)*rpc) over the cluster in fixed rank order
  const int rpc = K1_BM / nsplit;
  const int rbeg = (int)crank * rpc;
  const uint32_t Pbase = smem_u32(P);
  for (int e = tid; e < rpc * r; e += K1_THREADS) {
    const int lr = e / r, c = e % r;
    const int row = rbeg + lr;
    const float s = dsmem_sum8(Pbase + (uint32_t)(row * NP + c) * 4u, nsplit);
    Ym[lr * r + c] = s;
    if (m0 + row < a.M) a.Y[(long long)(m0 + row) * r + c] = s;
  }
  __syncthreads();
  for (int e = tid; e < rr; e += K1_THREADS) {
    const int i = e / r, j = e % r;
    float s = 0.f;
    for (int lr = 0; lr < rpc; ++lr) s = fmaf(Ym[lr * r + i], Ym[lr * r + j], s);
    Gs[e] = s;
  }
  cluster_sync();
  if (crank == 0) {
    const uint32_t Gbase = smem_u32(Gs);
    for (int e = tid; e < rr; e += K1_THREADS) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (q < nsplit) ? dsmem_ld_f32(dsmem_addr(Gbase + (uint32_t)e * 4u, q)) : 0.f;
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) two_sum_acc(hi, lo, v[q]);
      a.gram_part[(size_t)rt * rr + e] = hi + lo;
    }
    if (tid < 32) {
      const uint32_t sb = smem_u32(&ss_sh);
      double v = (tid < nsplit) ? dsmem_ld_f64(dsmem_addr(sb, tid)) : 0.0;
      v = warp_sum(v);
      if (tid == 0) a.xx_part[rt] = v;
    }
  }
  cluster_sync();   // peers' shared memory stays valid until rank 0 has read it
  if (tr0) TTRACE(3);
}

// ================================================================ K1b: r x r factor
// A cluster of KB_CLUSTER CTAs.  Every CTA sums the Gram partials (W1), factors the scaled
// Gram D W1 D = L L^T (FP32, one warp) and forms T1 = D L^{-T} (blocked triangular
// inverse); CTA q then computes Q1 = Y T1 for its share of the rows (rounded to the
// ingest type: the values that multiply X in the env kernel) and the Gram partial of
// those rows on tensor cores (exact products).  Rank 0 reduces W2 = Q1^T Q1 through
// distributed shared memory and forms Nx = W2^{-1} - I = -D2 + D2^2 - D2^3 (D2 = W2 - I).
// A failed factorisation (scaled pivot <= 1e-4: rank-deficient or badly conditioned Y)
// takes the FP64 Householder QR of Y on rank 0 instead.
constexpr int K1B_THREADS = 256;
constexpr int KB_CLUSTER = 8;

// C = alpha * A B for n x n row-major shared-memory matrices (leading dims la, lb, lc), all threads
__device__ __forceinline__ void smem_mm(float* C, int lc, const float* A, int la, const float* B, int lb, int n,
                                       float alpha) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    float s0 = 0.f, s1 = 0.f;
    int k = 0;
    for (; k + 1 < n; k += 2) {
      s0 = fmaf(A[i * la + k], B[k * lb + j], s0);
      s1 = fmaf(A[i * la + k + 1], B[(k + 1) * lb + j], s1);
    }
    if (k < n) s0 = fmaf(A[i * la + k], B[k * lb + j], s0);
    C[i * lc + j] = alpha * (s0 + s1);
  }
}

// Inverse of a lower-triangular n x n matrix (n = 32 or 64, identity-padded), blocked and
// log-depth: 4 x 4 diagonal blocks by forward substitution, then for block widths
// b = 4, 8, ... the off-diagonal block of [[A,0],[B,C]]^{-1} is -C^{-1} B A^{-1}.
// X (n x n, ld n+1) receives the inverse; T is n/2 x n/2 scratch per block pair.
__device__ void tri_lower_inverse(const float* L, int ldl, int n, float* X, float* T) {
  const int ldx = n + 1;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) X[(e / n) * ldx + e % n] = 0.f;
  __syncthreads();
  // 4 x 4 diagonal blocks: thread (blk, c) forward-substitutes column c
  for (int e = threadIdx.x; e < (n / 4) * 4; e += blockDim.x) {
    const int blk = e / 4, c = e % 4, o = blk * 4;
    float x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float s = (i == c) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < i; ++k) s = fmaf(-L[(o + i) * ldl + o + k], x[k], s);
      x[i] = (i >= c) ? s / L[(o + i) * ldl + o + i] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) X[(o + i) * ldx + o + c] = x[i];
  }
  __syncthreads();
  for (int b = 4; b < n; b *= 2) {
    const int npair = n / (2 * b);
    // T = B A^{-1}  (B = L[o+b.., o..], A^{-1} = X[o.., o..]) for every pair
    for (int e = threadIdx.x; e < npair * b * b; e += blockDim.x) {
      const int pr = e / (b * b), i = (e / b) % b, j = e % b, o = pr * 2 * b;
      float s = 0.f;
      for (int k = j; k < b; ++k) s = fmaf(L[(o + b + i) * ldl + o + k], X[(o + k) * ldx + o + j], s);
      T[pr * b * b + i * b + j] = s;
    }
    __syncthreads();
    // X21 = -C^{-1} T
    for (int e = threadIdx.x; e < npair * b * b; e += blockDim.x) {
      const int pr = e / (b * b), i = (e / b) % b, j = e % b, o = pr * 2 * b;
      float s = 0.f;
      for (int k = 0; k <= i; ++k) s = fmaf(X[(o + b + i) * ldx + o + b + k], T[pr * b * b + k * b + j], s);
      X[(o + b + i) * ldx + o + j] = -s;
    }
    __syncthreads();
  }
}

struct FactorArgs {
  const float* Y;         // M x r
  const float* gram_part; // [nrt][r*r]
  const double* xx_part;  // [nrt]
  int nrt, M, r;
  void* Qh;               // M x NP ingest-type Q1 (columns >= r zero)
  float* Qst;             // state: Q1 (M x r) as float
  float* W2st;            // state: W2 (r x r)
  float* Nx;              // r x r correction of the projector
  double* hh_work;        // 2*M*r doubles (fallback)
  float* Qfb;             // M x r (fallback Q, float)
  Ctl* ctl;
};

// rows of Y handled by one CTA of the factor cluster
__host__ __device__ constexpr int k1b_rows(int M) { return ((M + KB_CLUSTER - 1) / KB_CLUSTER + 15) / 16 * 16; }
// dynamic shared memory: Y rows (padded r+1) | Q1 rows (ingest type, padded NP+8) |
// Gram partial (NP x NP) | triangular-inverse and Nx scratch
__host__ __device__ constexpr size_t k1b_smem_bytes(int M, int r, int np) {
  return (size_t)k1b_rows(M) * (r + 1) * 4 + (size_t)(k1b_rows(M) + 16) * (np + 8) * 2 + (size_t)np * np * 4 +
         (size_t)(2 * 64 * 65 + 32 * 32) * 4 + 256;
}

template <typename TX, int NP>
__global__ void __launch_bounds__(K1B_THREADS) k_fast_factor(FactorArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float W[64 * 64];
  __shared__ float L[64 * 65];
  __shared__ float dsc[64];
  __shared__ double red[32];
  __shared__ int flags[2];     // [0] non-finite, [1] factorisation failed
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = a.r, rr = r * r, LD = r + 1;
  const uint32_t crank = cluster_rank();
  const int nrows = k1b_rows(a.M);
  const int row0 = (int)crank * nrows;
  const int myrows = (a.M - row0 < nrows) ? (a.M - row0 > 0 ? a.M - row0 : 0) : nrows;
  constexpr int LQ = NP + 8;
  float* Ys = reinterpret_cast<float*>(smem);                         // [nrows][r+1]
  TX* Qs = reinterpret_cast<TX*>(Ys + (size_t)nrows * LD);            // [nrows+16][LQ]
  float* Gp = reinterpret_cast<float*>(Qs + (size_t)(nrows + 16) * LQ);   // [NP][NP]
  float* scr = Gp + NP * NP;                                          // inverse / Nx scratch
  pdl_wait();
  pdl_trigger();
  TTRACE(10);
  // my rows of Y (coalesced; independent of the factor)
  for (int e = tid; e < myrows * r; e += K1B_THREADS) Ys[(e / r) * LD + e % r] = a.Y[(long long)row0 * r + e];
  for (int e = tid; e < rr; e += K1B_THREADS) {
    float hi = 0.f, lo = 0.f;
    for (int b0 = 0; b0 < a.nrt; b0 += 8) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (b0 + q < a.nrt) ? a.gram_part[(size_t)(b0 + q) * rr + e] : 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) two_sum_acc(hi, lo, v[q]);
    }
    W[e] = hi + lo;
  }
  if (warp == 0) {
    double xs = 0.0;
    for (int b = lane; b < a.nrt; b += 32) xs += a.xx_part[b];
    xs = warp_sum(xs);
    if (lane == 0) {
      flags[0] = !isfinite(xs);
      flags[1] = 0;
      if (crank == 0) a.ctl->xx = xs;
    }
  }
  __syncthreads();
  for (int e = tid; e < rr; e += K1B_THREADS)
    if (!isfinite(W[e])) flags[0] = 1;
  if (tid < r) {
    const float d = W[tid * r + tid];
    dsc[tid] = d > 0.f ? rsqrtf(d) : 0.f;
    if (!(d > 0.f)) flags[1] = 1;
  }
  __syncthreads();
  if (crank == 0 && tid == 0) {
    a.ctl->fallback[0] = 0;
    a.ctl->skip = flags[0];
    if (flags[0]) a.ctl->latched = 4;
  }
  if (flags[0]) return;     // uniform across the cluster (same data): no cluster barrier follows
  TTRACE(11);
  // ---- Cholesky of the scaled Gram: D W D = L L^T
  if (!flags[1]) {
    if constexpr (NP <= 32) {
      if (warp == 0) {
        float l[32];
        const float di = lane < r ? dsc[lane] : 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) l[k] = 0.f;
        int ok = 1;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float wj = (lane < r && j < r) ? W[lane * r + j] * di * dsc[j] : (lane == j ? 1.f : 0.f);
          float s0 = wj, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
          for (int k = 0; k < j; k += 4) {
            s0 = fmaf(-l[k], __shfl_sync(0xffffffffu, l[k], j), s0);
            if (k + 1 < j) s1 = fmaf(-l[k + 1], __shfl_sync(0xffffffffu, l[k + 1], j), s1);
            if (k + 2 < j) s2 = fmaf(-l[k + 2], __shfl_sync(0xffffffffu, l[k + 2], j), s2);
            if (k + 3 < j) s3 = fmaf(-l[k + 3], __shfl_sync(0xffffffffu, l[k + 3], j), s3);
          }
          const float sv = (s0 + s1) + (s2 + s3);
          const float piv = __shfl_sync(0xffffffffu, sv, j);
          if (!(piv > 1e-4f)) ok = 0;
          const float rl = rsqrtf(piv > 0.f ? piv : 1.f);
          l[j] = (lane == j) ? piv * rl : (lane > j ? sv * rl : 0.f);
        }
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (lane < r && k < r) L[lane * LD + k] = l[k];
        if (lane == 0) flags[1] = ok ? 0 : 1;
      }
    } else {
      for (int e = tid; e < rr; e += K1B_THREADS) {
        const int i = e / r, j = e % r;
        L[i * LD + j] = W[e] * dsc[i] * dsc[j];
      }
      __syncthreads();
      for (int j = 0; j < r; ++j) {
        const float piv = L[j * LD + j];
        if (!(piv > 1e-4f)) {
          if (tid == 0) flags[1] = 1;
          break;                      // uniform
        }
        const float rl = rsqrtf(piv);
        for (int e = tid; e < rr; e += K1B_THREADS) {
          const int i = e / r, k = e % r;
          if (i > j && k > j && k <= i) L[i * LD + k] -= L[i * LD + j] * L[k * LD + j] / piv;
        }
        __syncthreads();
        if (tid >= j && tid < r) L[tid * LD + j] *= rl;
        __syncthreads();
      }
    }
  }
  __syncthreads();
  TTRACE(12);
  TX* Qh = (TX*)a.Qh;
  const bool fb = flags[1] != 0;      // identical in every CTA of the cluster
  if (fb) {
    if (crank == 0) householder_cta<float, float>(a.Y, a.M, r, r, a.hh_work, a.Qfb, r, red);
    cluster_sync();                   // Qfb complete before the other ranks read it
    for (int e = tid; e < myrows * r; e += K1B_THREADS) Ys[(e / r) * LD + e % r] = a.Qfb[(long long)row0 * r + e];
  }
  // T1 = D L^{-T} (identity when the Householder Q is used)
  float* T1 = W;
  if (!fb) {
    const int n = r <= 32 ? 32 : 64;
    float* Lp = scr;                       // n x (n+1)
    float* Xi = Lp + n * (n + 1);          // n x (n+1)
    float* Tt = Xi + n * (n + 1);          // (n/2)^2
    for (int e = tid; e < n * n; e += K1B_THREADS) {
      const int i = e / n, j = e % n;
      Lp[i * (n + 1) + j] = (i < r && j < r) ? (j <= i ? L[i * LD + j] : 0.f) : (i == j ? 1.f : 0.f);
    }
    __syncthreads();
    tri_lower_inverse(Lp, n + 1, n, Xi, Tt);
    for (int e = tid; e < rr; e += K1B_THREADS) {
      const int k = e / r, c = e % r;
      T1[e] = dsc[k] * Xi[c * (n + 1) + k];    // (D L^{-T})[k][c] = d_k (L^{-1})[c][k]
    }
  } else {
    for (int e = tid; e < rr; e += K1B_THREADS) T1[e] = ((e / r) == (e % r)) ? 1.f : 0.f;
  }
  __syncthreads();
  // Q1 rows = Y rows T1: 4 x 4 register blocks; a thread takes rows br + u*nbr, so the
  // lanes of a warp read consecutive padded rows (stride r+1: conflict-free)
  {
    const int nbc = (r + 3) / 4;
    const int nbr = (myrows + 3) / 4;
    for (int task = tid; task < nbr * nbc; task += K1B_THREADS) {
      const int br = task % nbr, bc = task / nbr;      // consecutive threads: consecutive row blocks
      float q[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) q[u][w] = 0.f;
      const int kmax = fb ? r - 1 : ((4 * bc + 3 < r) ? 4 * bc + 3 : r - 1);
      for (int k = 0; k <= kmax; ++k) {
        float y[4], t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = (br + u * nbr < myrows) ? Ys[(br + u * nbr) * LD + k] : 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w) t[w] = (4 * bc + w < r) ? T1[k * r + 4 * bc + w] : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int w = 0; w < 4; ++w) q[u][w] = fmaf(y[u], t[w], q[u][w]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int row = br + u * nbr;
        if (row >= myrows) continue;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int c = 4 * bc + w;
          if (c < r) Qs[row * LQ + c] = from_acc<TX>(q[u][w]);
        }
      }
    }
    // zero: padding columns and the rows past my share (read by the last k-step below)
    for (int e = tid; e < (nrows + 16) * LQ; e += K1B_THREADS) {
      const int row = e / LQ, c = e % LQ;
      if (row >= myrows || c >= r) Qs[e] = from_acc<TX>(0.f);
    }
  }
  __syncthreads();
  // write my Q1 rows (coalesced) in the ingest type and as float
  for (int e = tid; e < myrows * NP; e += K1B_THREADS) {
    const int row = e / NP, c = e % NP;
    const TX h = Qs[row * LQ + c];
    Qh[(long long)(row0 + row) * NP + c] = h;
    if (c < r) a.Qst[(long long)(row0 + row) * r + c] = Cvt<TX>::f(h);
  }
  TTRACE(13);
  // Gram partial of my rows on tensor cores: warp w takes k-steps w, w+8, ...
  {
    constexpr int MT = NP / 16, NTT = NP / 8;
    const int nw = K1B_THREADS / 32;
    const int ksteps = (myrows + 15) / 16;
    float acc[MT][NTT][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int n = 0; n < NTT; ++n) acc[m][n][0] = acc[m][n][1] = acc[m][n][2] = acc[m][n][3] = 0.f;
    for (int ks = warp; ks < ksteps; ks += nw) {
      const int k0 = ks * 16;
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        uint32_t af[4];
        {
          const int row = k0 + (lane & 7) + ((lane >> 4) << 3);
          const int col = m * 16 + ((lane >> 3) & 1) * 8;
          ldsm_x4_t(smem_u32(Qs + row * LQ + col), af[0], af[1], af[2], af[3]);
        }
#pragma unroll
        for (int p = 0; p < NTT / 2; ++p) {
          uint32_t b0, b1, b2, b3;
          const int row = k0 + (lane & 7) + (((lane >> 3) & 1) << 3);
          const int col = p * 16 + ((lane >> 4) << 3);
          ldsm_x4_t(smem_u32(Qs + row * LQ + col), b0, b1, b2, b3);
          mma16816<TX>(acc[m][2 * p], af, b0, b1);
          mma16816<TX>(acc[m][2 * p + 1], af, b2, b3);
        }
      }
    }
    // sum the warps' fragments in a fixed order into Gp
    for (int e = tid; e < NP * NP; e += K1B_THREADS) Gp[e] = 0.f;
    __syncthreads();
    const int g = lane >> 2, t4 = lane & 3;
    for (int w = 0; w < nw; ++w) {
      if (warp == w) {
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
          for (int n = 0; n < NTT; ++n) {
            const int row = m * 16 + g, col = n * 8 + 2 * t4;
            Gp[row * NP + col] += acc[m][n][0];
            Gp[row * NP + col + 1] += acc[m][n][1];
            Gp[(row + 8) * NP + col] += acc[m][n][2];
            Gp[(row + 8) * NP + col + 1] += acc[m][n][3];
          }
      }
      __syncthreads();
    }
  }
  cluster_sync();
  TTRACE(14);
  if (crank == 0) {
    // W2 = sum of the ranks' partials (fixed order), then Nx
    const uint32_t gb = smem_u32(Gp);
    for (int e = tid; e < rr; e += K1B_THREADS) {
      const int i = e / r, j = e % r;
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        v[q] = (q < KB_CLUSTER) ? dsmem_ld_f32(dsmem_addr(gb + (uint32_t)(i * NP + j) * 4u, q)) : 0.f;
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) two_sum_acc(hi, lo, v[q]);
      W[e] = hi + lo;
    }
    __syncthreads();
    float* D2 = L;                                      // r x r
    float* U = scr;                                     // D2^2
    float* V = U + rr;                                  // D2^3
    for (int e = tid; e < rr; e += K1B_THREADS) {
      a.W2st[e] = W[e];
      D2[e] = W[e] - ((e / r) == (e % r) ? 1.f : 0.f);
    }
    __syncthreads();
    smem_mm(U, r, D2, r, D2, r, r, 1.f);
    __syncthreads();
    smem_mm(V, r, D2, r, U, r, r, 1.f);
    __syncthreads();
    for (int e = tid; e < rr; e += K1B_THREADS) a.Nx[e] = -D2[e] + U[e] - V[e];
    if (tid == 0 && fb) a.ctl->fallback[0] = 1;
  }
  cluster_sync();   // peers' partials stay valid until rank 0 has read them
  TTRACE(15);
}

// ================================================================ K2: environment
// F^T = X_(1)^T Q1 for a 128-column tile of X; the row chunks of a column tile form a
// cluster and reduce through distributed shared memory.  Writes F (the state's right
// part) and its scaled ingest-type copy, and the step's ||x^||^2 = sum_j f_j^T (I + Nx) f_j.
// The X block arrives as two 64-column, 128B-swizzled TMA boxes of rch rows.
constexpr int K2_THREADS = 256;
constexpr int K2_BN = 128;            // slice columns j per CTA

struct EnvArgs {
  int M, r;
  long long J;
  int rch;              // rows per cluster rank (multiple of 16)
  const void* Qh;       // M x NP ingest-type Q1
  const float* Nx;      // r x r
  float* Cst;           // state: F (r x J)
  void* Chst;           // state: scaled ingest-type copy of F (r x J)
  int* ch_shift;        // state: power-of-two scale exponent of Chst
  double* cc_part;      // [column tiles]
  unsigned* counter;    // self-resetting
  Ctl* ctl;
  // previous state (copied into the new one when the step is skipped)
  float* Qst;
  float* W2st;
  const float* Qold;
  const float* Cold;
  const void* Chold;
  const float* W2old;
  const int* ch_shift_old;
  int is_half;          // 1: FP16 copy needs a range scale; 0: BF16
};

template <int NP>
constexpr size_t k2_smem_bytes(int rch, int r) {
  // X block (2 x rch x 128 B) | Q1 tile | partial tile P (BN x NP) | my columns F | Nx
  return 1024 + (size_t)rch * 256 + (size_t)rch * (NP + 8) * 2 + (size_t)K2_BN * NP * 4 +
         (size_t)K2_BN * (r + 1) * 4 + (size_t)r * r * 4 + 64;
}

template <typename TX, int NP>
__global__ void __launch_bounds__(K2_THREADS, 2)
    k_fast_env(const __grid_constant__ CUtensorMap tmX, EnvArgs a) {
  constexpr int NT = NP / 8;   // n8-tiles per warp (each warp covers all NP columns)
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int rch = a.rch, r = a.r, rr = r * r;
  const uint32_t xsub0 = smem_u32(smem), xsub1 = xsub0 + (uint32_t)rch * 128;   // two swizzled boxes
  TX* sQ = reinterpret_cast<TX*>(smem + (size_t)rch * 256);           // [rch][NP+8]
  float* P = reinterpret_cast<float*>(sQ + (size_t)rch * (NP + 8));  // [BN][NP]
  const int LDF = r + 1;                                             // padded: conflict-free
  float* sF = P + K2_BN * NP;                                        // [BN][r+1] (my columns)
  float* sN = sF + K2_BN * LDF;                                      // Nx
  __shared__ __align__(8) uint64_t xbar;
  __shared__ double red[32];
  __shared__ double cc_sh;
  __shared__ int last_flag;
  __shared__ int timeout_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t crank = cluster_rank();
  const int nq = gridDim.y;
  const int ct = blockIdx.x;
  const long long j0 = (long long)ct * K2_BN;
  const int i0 = (int)crank * rch;
  const int xcols = (a.J - j0 < K2_BN) ? (int)(a.J - j0) : K2_BN;
  const bool tr0 = (blockIdx.x == 0 && blockIdx.y == 0);

  // 1. this CTA's X block through the TMA engine (independent of the previous kernels)
  if (tid == 0) {
    mbar_init(smem_u32(&xbar), 1);
    mbar_fence_init();
    timeout_flag = 0;
    const uint32_t bar = smem_u32(&xbar);
    mbar_arrive_expect_tx(bar, (uint32_t)rch * 256);
    tma_load_2d(xsub0, &tmX, (int)j0, i0, bar);
    tma_load_2d(xsub1, &tmX, (int)j0 + 64, i0, bar);
  }
  if (tr0) TTRACE(20);
  // 2. wait for the factor kernel (Q1, Nx, ctl)
  pdl_wait();
  pdl_trigger();
  if (tr0) TTRACE(21);
  if (a.ctl->skip) {
    // non-finite slice: the new state is the old one
    const long long nthr = (long long)gridDim.x * gridDim.y * K2_THREADS;
    const long long me = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * K2_THREADS + tid;
    for (long long e = me; e < (long long)a.M * r; e += nthr) a.Qst[e] = a.Qold[e];
    for (long long e = me; e < (long long)r * a.J; e += nthr) {
      a.Cst[e] = a.Cold[e];
      ((TX*)a.Chst)[e] = ((const TX*)a.Chold)[e];
    }
    for (long long e = me; e < rr; e += nthr) a.W2st[e] = a.W2old[e];
    if (me == 0) *a.ch_shift = *a.ch_shift_old;
    if (!mbar_wait(smem_u32(&xbar), 0) && tid == 0) a.ctl->latched = 5;
    return;
  }
  // 3. Q1 rows of this chunk (ingest type) and Nx
  {
    const TX* Qh = (const TX*)a.Qh;
    constexpr int CPR = NP / 8;     // 16-byte chunks per row
    for (int c = tid; c < rch * CPR; c += K2_THREADS) {
      const int row = c / CPR, ch = c % CPR;
      const int gi = i0 + row;
      const bool ok = gi < a.M;
      cp_async16(smem_u32(sQ + row * (NP + 8) + ch * 8), Qh + (ok ? (long long)gi * NP + ch * 8 : 0), ok ? 16u : 0u);
    }
    cp_async_commit();
    for (int e = tid; e < rr; e += K2_THREADS) sN[e] = a.Nx[e];
    cp_async_wait<0>();
  }
  if (!mbar_wait(smem_u32(&xbar), 0)) timeout_flag = 1;
  __syncthreads();
  if (tr0) TTRACE(22);
  // 4. F^T (j x a) = X^T Q1 over this chunk: warp w -> columns j in [16w, 16w+16)
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  {
    const int jcol = warp * 16 + ((lane >> 3) & 1) * 8;       // column of this lane's 8x8 matrix
    const uint32_t xb = (jcol >> 6) ? xsub1 : xsub0;
    const int chunk = (jcol & 63) >> 3;
    for (int k0 = 0; k0 < rch; k0 += 16) {
      uint32_t af[4];
      {
        const int row = k0 + (lane & 7) + ((lane >> 4) << 3);
        ldsm_x4_t(xb + swz(row, chunk), af[0], af[1], af[2], af[3]);
      }
#pragma unroll
      for (int p = 0; p < NT / 2; ++p) {
        uint32_t b0, b1, b2, b3;
        const int row = k0 + (lane & 7) + (((lane >> 3) & 1) << 3);
        const int col = p * 16 + ((lane >> 4) << 3);
        ldsm_x4_t(smem_u32(sQ + row * (NP + 8) + col), b0, b1, b2, b3);
        mma16816<TX>(acc[2 * p], af, b0, b1);
        mma16816<TX>(acc[2 * p + 1], af, b2, b3);
      }
    }
  }
  {
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int col = j * 8 + 2 * t4;
      const int row = warp * 16 + g;
      P[row * NP + col] = acc[j][0];
      P[row * NP + col + 1] = acc[j][1];
      P[(row + 8) * NP + col] = acc[j][2];
      P[(row + 8) * NP + col + 1] = acc[j][3];
    }
  }
  if (tid == 0 && timeout_flag) a.ctl->latched = 5;
  if (tr0) TTRACE(23);
  cluster_sync();
  if (tr0) TTRACE(24);
  // 5. my share of the tile's columns, reduced over the cluster in rank order
  const int per = (K2_BN + nq - 1) / nq;
  const int jb = (int)crank * per;
  const int je = (jb + per < xcols) ? jb + per : xcols;
  const int nmy = je > jb ? je - jb : 0;
  {
    const uint32_t Pb = smem_u32(P);
    for (int e = tid; e < nmy * r; e += K2_THREADS) {
      const int jl = e / r, c = e % r;
      sF[jl * LDF + c] = dsmem_sum8(Pb + (uint32_t)((jb + jl) * NP + c) * 4u, nq);
    }
  }
  cluster_sync();   // every rank has read the peers' tiles
  if (tr0) TTRACE(25);
  // write F and its ingest-type copy (coalesced along j); ||x^||^2 of my columns
  const double xx = a.ctl->xx;
  int shift = 0;
  if (a.is_half && xx > 0.0) {
    const float nrm = sqrtf((float)xx);
    shift = nrm > 16384.f ? (int)ceilf(log2f(nrm / 16384.f)) : 0;
  }
  if (ct == 0 && crank == 0 && tid == 0) *a.ch_shift = shift;
  const float scale = ldexpf(1.0f, -shift);
  double part = 0.0;
  for (int e = tid; e < nmy * r; e += K2_THREADS) {
    const int c = e / nmy, jl = e % nmy;
    const long long gj = j0 + jb + jl;
    const float f = sF[jl * LDF + c];
    a.Cst[(long long)c * a.J + gj] = f;
    ((TX*)a.Chst)[(long long)c * a.J + gj] = from_acc<TX>(f * scale);
    // f_c * (f + Nx f)_c
    float g = f;
    for (int b = 0; b < r; ++b) g = fmaf(sN[c * r + b], sF[jl * LDF + b], g);
    part += (double)(f * g);
  }
  const double cc_cta = block_sum(part, red);
  if (tid == 0) cc_sh = cc_cta;
  if (tr0) TTRACE(26);
  cluster_sync();
  if (crank == 0 && tid < 32) {
    const uint32_t cb = smem_u32(&cc_sh);
    double v = (tid < nq) ? dsmem_ld_f64(dsmem_addr(cb, tid)) : 0.0;
    v = warp_sum(v);
    if (tid == 0) a.cc_part[ct] = v;
  }
  cluster_sync();
  if (crank != 0) return;
  __threadfence();
  if (tid == 0) {
    const unsigned done = atomicAdd(a.counter, 1u);
    last_flag = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!last_flag) return;
  TTRACE(27);
  __threadfence();
  double s = 0.0;
  for (int b = tid; b < (int)gridDim.x; b += K2_THREADS) s += a.cc_part[b];
  const double cc = block_sum(s, red);
  if (tid == 0) {
    *a.counter = 0u;
    Ctl* c = a.ctl;
    if (!isfinite(cc)) c->latched = 4;
    const double ccv = isfinite(cc) ? cc : 0.0;
    const double ee = c->xx - ccv > 0.0 ? c->xx - ccv : 0.0;
    c->cc = ccv;
    c->ee = ee;
    c->sum_xx += c->xx;
    c->sum_ee += ee;
    c->t += 1;
  }
  TTRACE(28);
}

// ------------------------------------------------ helpers for the lazy finalisation
// W2 (FP32, r x r) -> T = R2^{-1}, R2 = chol(W2) in FP64 (one CTA; output path only).
__global__ void k_chol64_inverse(const float* __restrict__ W2, int r, double* __restrict__ T64,
                                 float* __restrict__ T32) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* R = reinterpret_cast<double*>(smem);     // r x r
  double* Ti = R + r * r;                          // r x r
  const int tid = threadIdx.x, rr = r * r;
  for (int e = tid; e < rr; e += blockDim.x) R[e] = (double)W2[e];
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    const double piv = R[j * r + j];
    const double rs = piv > 0.0 ? 1.0 / sqrt(piv) : 0.0;
    for (int e = tid; e < rr; e += blockDim.x) {
      const int i = e / r, k = e % r;
      if (i > j && k >= i) R[i * r + k] -= R[j * r + i] * R[j * r + k] * (piv > 0.0 ? 1.0 / piv : 0.0);
    }
    __syncthreads();
    if (tid >= j && tid < r) R[j * r + tid] *= rs;
    __syncthreads();
  }
  if (tid < r) {
    const int c = tid;
    for (int i = 0; i < r; ++i) Ti[i * r + c] = 0.0;
    Ti[c * r + c] = R[c * r + c] != 0.0 ? 1.0 / R[c * r + c] : 0.0;
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= c; ++k) s += R[i * r + k] * Ti[k * r + c];
      Ti[i * r + c] = R[i * r + i] != 0.0 ? -s / R[i * r + i] : 0.0;
    }
  }
  __syncthreads();
  for (int e = tid; e < rr; e += blockDim.x) {
    T64[e] = Ti[e];
    T32[e] = (float)Ti[e];
  }
}

// G1 = Q1 T (T upper triangular, FP32) -- no control-block checks (output path)
__global__ void k_apply_upper(const float* __restrict__ Q, long long rows, int r, const float* __restrict__ T,
                              float* __restrict__ G) {
  const long long total = rows * r;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / r;
    const int j = (int)(e % r);
    float s = 0.f;
    for (int k = 0; k <= j; ++k) s = fmaf(Q[i * r + k], T[k * r + j], s);
    G[e] = s;
  }
}

// Ch = (ingest type) C * 2^-shift, shift chosen so that ||C||_F * 2^-shift <= 16384 (FP16 range)
template <typename TX>
__global__ void k_make_half_copy(const float* __restrict__ C, long long n, TX* __restrict__ Ch, int* __restrict__ shift,
                                 int is_half) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) s += (double)C[e] * C[e];
  const double nrm = sqrt(block_sum(s, red));
  int sh = 0;
  if (is_half)
    while (nrm * ldexp(1.0, -sh) > 16384.0 && sh < 120) ++sh;
  const float sc = ldexpf(1.0f, -sh);
  for (long long e = threadIdx.x; e < n; e += blockDim.x) Ch[e] = from_acc<TX>(C[e] * sc);
  if (threadIdx.x == 0) *shift = sh;
}

}  // namespace fast
}  // namespace ttals
