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
#include "ttals_r64.cuh"

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
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
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
// split form: every thread arrives, does independent work, then waits
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
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

// float-float sums: hi + lo, added with TwoSum on the FP32 pipe (the FP64 pipe of this
// part is narrow and its latency long; these sums need more than FP32 but not FP64 rate)
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
  two_sum_acc(hi, lo, bh);
  lo += bl;
}
// block-wide float-float sum in a fixed order; the result is valid in thread 0.
// sh: 64 floats of shared memory.
__device__ __forceinline__ float2 ff_block_sum(float hi, float lo, float* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_down_sync(0xffffffffu, hi, o), bl = __shfl_down_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, bh, bl);
  }
  __syncthreads();
  if (lane == 0) {
    sh[2 * w] = hi;
    sh[2 * w + 1] = lo;
  }
  __syncthreads();
  if (w == 0) {
    hi = lane < nw ? sh[2 * lane] : 0.f;
    lo = lane < nw ? sh[2 * lane + 1] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float bh = __shfl_down_sync(0xffffffffu, hi, o), bl = __shfl_down_sync(0xffffffffu, lo, o);
      ff_add(hi, lo, bh, bl);
    }
  }
  return make_float2(hi, lo);
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

// the float at local address `a` in cluster rank q, or 0 for q >= n: the load always targets
// a valid rank (q clamped to n-1) and the value is masked, so no remote access depends on the
// guard being compiled as a branch
__device__ __forceinline__ float dsmem_ld_rank(uint32_t a, int q, int n) {
  const float v = dsmem_ld_f32(dsmem_addr(a, (uint32_t)(q < n ? q : n - 1)));
  return q < n ? v : 0.f;
}

// sum of n (1..8) values loaded from distributed shared memory, loads issued together
__device__ __forceinline__ float dsmem_sum8(uint32_t local_addr, int n) {
  float v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = dsmem_ld_rank(local_addr, q, n);
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += v[q];
  return s;
}

// 3-D tensor copy (TMA) global -> shared: box at element coordinates (x inner, y, z outer)
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// byte offset of 16-byte chunk c of row `row` in a 128B-swizzled box (1024-byte aligned)
__device__ __forceinline__ uint32_t swz(int row, int c) { return (uint32_t)(row * 128 + ((c ^ (row & 7)) << 4)); }

__device__ __forceinline__ unsigned short tx_bits(__half v) { return __half_as_ushort(v); }
__device__ __forceinline__ unsigned short tx_bits(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }

// ================================================================ K1: local solve
// Y = X_(1) B^T for one 64-row tile of X and a k-split; the splits of a row tile form a
// thread-block cluster and reduce their partial tiles through distributed shared memory
// (fixed rank order).  Also per-CTA partials of ||x||^2.
// X and B arrive through the TMA engine in stages of two 64-column boxes (256 contiguous
// bytes of every row per stage), 128B-swizzled, out-of-range rows and columns zero-filled by
// the hardware.  Warp 8 issues the copies; warps 0-7 consume the stages and release each
// one through its `empty` barrier, so no block-wide barrier sits in the main loop.
constexpr int K1_CWARPS = 8;                        // consumer warps
constexpr int K1_THREADS = (K1_CWARPS + 1) * 32;    // + the producer warp
constexpr int K1_BM = 64;          // rows of X per CTA
constexpr int K1_BK = 128;         // k per pipeline stage: two 64-column boxes
constexpr int K1_MAXST = 4;

struct SolveArgs {
  int M, r;
  long long K, kchunk;    // kchunk % K1_BK == 0
  float* Y;               // M x r
  float2* xx_part;        // [row tiles * splits] float-float partials of ||x||^2
  float2* W1part;         // [row tiles][NP*NP] float-float Gram partials Y_t^T Y_t of the row tiles
  long long w1_stride;    // float2 elements per stream of W1part
  Ctl* ctl;
  int stall;              // fault injection (k_fast_solve): issue no copy, so that the
                          // consumers' first bounded wait runs out (0 in normal use)
  unsigned char zmap[64];      // grid plane blockIdx.z -> stream (slot) of the batch
};

// Gram of a row tile for the factor of the local solve (Sec. 3.4.2: QR of G~ through the
// Cholesky factor of G~^T G~): G = Yt^T Yt over the nrows rows of a row-major tile (row i at
// Yt + i * ldy, 16-byte aligned rows, NP columns, zero past r) by the NT threads of the block,
// in FP32 4 x 4 register blocks.  The rows are split into NRG groups whose partials (Gr: NRG
// NP x NP matrices of shared memory; Gr may be G when NRG = 1) are summed in group order into
// G.  Yt must be complete before the call; the function ends with a block barrier.
template <int NP, int NT>
__host__ __device__ constexpr int tile_gram_groups() {
  return NT / ((NP / 4) * (NP / 4)) > 0 ? NT / ((NP / 4) * (NP / 4)) : 1;
}
template <int NP, int NT>
__device__ __forceinline__ void tile_gram(const float* Yt, int ldy, int nrows, float* Gr, float* G) {
  constexpr int NB = NP / 4, NBLK = NB * NB, NRG = tile_gram_groups<NP, NT>();
  const int tid = threadIdx.x;
  for (int w = tid; w < NRG * NBLK; w += NT) {
    const int blk = w % NBLK, rg = w / NBLK, ib = blk / NB, jb = blk % NB;
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    for (int row = rg; row < nrows; row += NRG) {
      const float4 yi = *reinterpret_cast<const float4*>(Yt + row * ldy + 4 * ib);
      const float4 yj = *reinterpret_cast<const float4*>(Yt + row * ldy + 4 * jb);
      const float vi[4] = {yi.x, yi.y, yi.z, yi.w}, vj[4] = {yj.x, yj.y, yj.z, yj.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(vi[u], vj[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) Gr[rg * NP * NP + (4 * ib + u) * NP + 4 * jb + v] = acc[u][v];
  }
  __syncthreads();
  if (NRG > 1 || Gr != G) {
    for (int e = tid; e < NP * NP; e += NT) {
      float s = 0.f;
#pragma unroll
      for (int g = 0; g < NRG; ++g) s += Gr[g * NP * NP + e];
      G[e] = s;
    }
    __syncthreads();
  }
}

template <int NP>
__host__ __device__ constexpr int k1_stages() { return NP <= 32 ? 4 : 3; }
template <int NP>
__host__ __device__ constexpr size_t k1_stage_bytes() {
  return (size_t)(K1_BM + NP) * 256;
}
template <int NP>
__host__ __device__ constexpr size_t k1_smem_bytes() {
  return (size_t)k1_stages<NP>() * k1_stage_bytes<NP>() + 1024;   // + alignment slack
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

template <typename TX, int NP>
__global__ void __launch_bounds__(K1_THREADS, 2)
    k_fast_solve(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, SolveArgs a0) {
  // grid plane z serves stream zs of the batch (the planes cover the streams that step):
  // its slice and its B are plane zs of the 3-D maps
  const int zs = a0.zmap[blockIdx.z];
  SolveArgs a = a0;
  a.Y += (size_t)zs * a.M * a.r;
  a.xx_part += (size_t)zs * gridDim.x * gridDim.y;
  a.ctl += zs;
  static_assert(NP % 16 == 0 && NP >= 16 && NP <= 64, "NP");
  constexpr int ST = k1_stages<NP>();
  static_assert(ST <= K1_MAXST, "stages");
  constexpr int NT = NP / 16;  // n8-tiles per warp (each warp covers NP/2 columns)
  constexpr uint32_t ABOX = K1_BM * 128, BBOX = NP * 128;   // one 64-column box of X / of B
  constexpr uint32_t ABYTES = 2 * ABOX, BBYTES = 2 * BBOX;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[K1_MAXST];    // stage data landed (A arrival + B arrival)
  __shared__ __align__(8) uint64_t empty[K1_MAXST];   // stage released by the 8 consumer warps
  __shared__ float redf[64];
  __shared__ int timeout_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wr = warp & 3, wc = (warp >> 2) & 1;
  const uint32_t crank = cluster_rank();
  const int nsplit = gridDim.y;
  const int rt = blockIdx.x;
  const int m0 = rt * K1_BM;
  const int r = a.r;
  const long long kbeg = (long long)blockIdx.y * a.kchunk;
  const long long kend = (kbeg + a.kchunk < a.K) ? kbeg + a.kchunk : a.K;
  const int ntk = kend > kbeg ? (int)((kend - kbeg + K1_BK - 1) / K1_BK) : 0;
  const bool tr0 = (blockIdx.x == 0 && blockIdx.y == 0);
  const bool producer = (warp == K1_CWARPS);
  const uint32_t sbase = smem_u32(smem);
  auto stageA = [&](int st) { return sbase + (uint32_t)(st * k1_stage_bytes<NP>()); };
  auto stageB = [&](int st) { return stageA(st) + ABYTES; };
  auto load_a = [&](int t, int st) {
    const int x = (int)(kbeg + (long long)t * K1_BK);
    tma_load_3d(stageA(st), &tmX, x, m0, zs, smem_u32(&full[st]));
    tma_load_3d(stageA(st) + ABOX, &tmX, x + 64, m0, zs, smem_u32(&full[st]));
  };
  auto load_b = [&](int t, int st) {
    const int x = (int)(kbeg + (long long)t * K1_BK);
    tma_load_3d(stageB(st), &tmB, x, 0, zs, smem_u32(&full[st]));
    tma_load_3d(stageB(st) + BBOX, &tmB, x + 64, 0, zs, smem_u32(&full[st]));
  };

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), 2);            // A arrival + B arrival
      mbar_init(smem_u32(&empty[s]), K1_CWARPS);
    }
    mbar_fence_init();
    timeout_flag = 0;
  }
  __syncthreads();
  if (tr0) TTRACE(0);
  TTRACE_CTA(0);
  // A tiles do not depend on the previous kernel: start them before the dependency wait
  if (producer && lane == 0 && !a.stall) {
    for (int t = 0; t < ST && t < ntk; ++t) {
      mbar_arrive_expect_tx(smem_u32(&full[t]), ABYTES);
      load_a(t, t);
    }
  }
  pdl_wait();       // the previous step's env kernel wrote B and ctl
  pdl_trigger();    // the factor kernel may launch and wait for this grid
  const bool bzero = (a.ctl->cc == 0.0);
  if (bzero) {
    // e_1 rule for a zero temporal row: the right part becomes e_0 e_0^T (B stays zero, but
    // for the one element of the first split's first stage)
    for (int st = 0; st < ST; ++st)
      for (int e = tid; e < (int)BBYTES / 16; e += K1_THREADS)
        *reinterpret_cast<uint4*>(smem + (stageB(st) - sbase) + e * 16) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    if (blockIdx.y == 0 && tid == 0) *reinterpret_cast<TX*>(smem + (stageB(0) - sbase)) = from_acc<TX>(1.0f);
  }
  __syncthreads();

  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  float ssh = 0.f, ssl = 0.f;    // ||x||^2 of the tiles seen by this thread (float-float)
  if (producer) {
    if (lane == 0 && a.stall) {
      // fault injection: no copy is issued, nothing is in flight; the consumers' wait on
      // stage 0 gives up after its bound and the step is marked failed
    } else if (lane == 0) {
      int issued = ntk < ST ? ntk : ST;
      for (int t = 0; t < issued; ++t) {
        if (bzero) {
          mbar_arrive_expect_tx(smem_u32(&full[t]), 0);
        } else {
          mbar_arrive_expect_tx(smem_u32(&full[t]), BBYTES);
          load_b(t, t);
        }
      }
      for (int t = ST; t < ntk; ++t) {
        const int st = t % ST;
        if (!mbar_wait(smem_u32(&empty[st]), (uint32_t)(((t / ST) - 1) & 1)) || timeout_flag) {
          timeout_flag = 1;
          break;
        }
        if (t == ST && bzero && blockIdx.y == 0)
          *reinterpret_cast<TX*>(smem + (stageB(0) - sbase)) = from_acc<TX>(0.f);
        mbar_arrive_expect_tx(smem_u32(&full[st]), ABYTES);
        load_a(t, st);
        if (bzero) {
          mbar_arrive_expect_tx(smem_u32(&full[st]), 0);
        } else {
          mbar_arrive_expect_tx(smem_u32(&full[st]), BBYTES);
          load_b(t, st);
        }
        issued = t + 1;
      }
      if (timeout_flag) {
        // a wait gave up: wait (bounded) for the copies still in flight before the buffers
        // are reused; the step is marked failed (ETIMEOUT)
        for (int t = issued - ST > 0 ? issued - ST : 0; t < issued; ++t)
          mbar_wait(smem_u32(&full[t % ST]), (uint32_t)((t / ST) & 1));
      }
    }
  } else {
    for (int t = 0; t < ntk; ++t) {
      const int st = t % ST;
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((t / ST) & 1)) || timeout_flag) {
        timeout_flag = 1;
        break;
      }
      if (t == 0) TTRACE_CTA(1);
      float ss = 0.f;
#pragma unroll
      for (int bx = 0; bx < 2; ++bx) {
        const uint32_t tA = stageA(st) + bx * ABOX, tB = stageB(st) + bx * BBOX;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
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
      }
      two_sum_acc(ssh, ssl, ss);
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[st]));   // this warp is done with stage st
    }
  }
  __syncthreads();          // every stage consumed (or the copies in flight drained)
  if (tr0) TTRACE(1);
  TTRACE_CTA(2);
  // ---- partial tile -> shared memory P[BM][NP] (fp32), reusing the pipeline buffers
  float* P = reinterpret_cast<float*>(smem);
  if (!producer) {
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
  const float2 ss_cta = ff_block_sum(ssh, ssl, redf);
  if (tid == 0) {
    // one partial of ||x||^2 per CTA; a CTA whose wait gave up writes NaN, which makes the
    // factor kernel mark the step skipped (not committed) while ETIMEOUT stays latched
    a.xx_part[(size_t)rt * nsplit + crank] = timeout_flag ? make_float2(__int_as_float(0x7fc00000), 0.f) : ss_cta;
    if (timeout_flag) a.ctl->latched = 5;
  }
  cluster_sync();
  if (tr0) TTRACE(2);
  // ---- rank q reduces rows [q*rpc, (q+1)*rpc) over the cluster in fixed rank order, writes
  // them to Y and keeps them (Yr, zero past r and past I_1) for the Gram partial
  const int rpc = K1_BM / nsplit;
  const int rbeg = (int)crank * rpc;
  const uint32_t Pbase = smem_u32(P);
  constexpr int LDR = NP + 4;
  float* Yr = P + K1_BM * NP;                                   // [rpc][LDR]
  float* Gr = Yr + K1_BM * LDR;                                 // row-group partials
  float* G = Gr + tile_gram_groups<NP, K1_THREADS>() * NP * NP;  // Gram of my rows
  for (int e = tid; e < rpc * NP; e += K1_THREADS) {
    const int lr = e / NP, c = e % NP;
    const int row = rbeg + lr;
    const bool in = c < r && m0 + row < a.M;
    const float s = c < r ? dsmem_sum8(Pbase + (uint32_t)(row * NP + c) * 4u, nsplit) : 0.f;
    if (in) a.Y[(long long)(m0 + row) * r + c] = s;
    Yr[lr * LDR + c] = in ? s : 0.f;
  }
  __syncthreads();
  tile_gram<NP, K1_THREADS>(Yr, LDR, rpc, Gr, G);
  float2* W1t = a.W1part + (size_t)zs * a.w1_stride + (size_t)rt * NP * NP;
  if (nsplit == 1) {
    for (int e = tid; e < NP * NP; e += K1_THREADS) W1t[e] = make_float2(G[e], 0.f);
  } else {
    cluster_sync();   // every rank's Gram is complete (and every rank has read the P tiles)
    // the row tile's Gram: entries [q*per, (q+1)*per) summed over the ranks in rank order
    // (TwoSum: a float-float pair)
    const int per = NP * NP / nsplit;
    const uint32_t Gbase = smem_u32(G);
    for (int e = tid; e < per; e += K1_THREADS) {
      const int ge = (int)crank * per + e;
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = dsmem_ld_rank(Gbase + (uint32_t)ge * 4u, q, nsplit);
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) two_sum_acc(hi, lo, v[q]);
      W1t[ge] = make_float2(hi, lo);
    }
  }
  cluster_sync();   // peers' shared memory stays valid until every rank has read it
  TTRACE_CTA(3);
  if (tr0) TTRACE(3);
}

// ================================================================ K1 on tcgen05 (batches)
// Y = X_(1) B^T for one 128-row tile of X over all of rest_1 (no k-split), on the 5th-gen
// tensor cores: warp 0 issues the TMA copies (stages of two 64-column boxes of X, 128 rows,
// and of B, NP rows: 256 contiguous bytes of every row per stage); warp 1's elected lane
// issues tcgen05.mma (M = 128, N = NP, K = 16 per instruction, FP32 accumulator in TMEM;
// operands through SWIZZLE_128B K-major shared-memory descriptors) and frees each stage with
// tcgen05.commit; warps 2-5 form ||x||^2 from the staged X tiles, release the stage, and at
// the end read the accumulator (tcgen05.ld, one TMEM lane = one row of Y) and write Y.
// The stage is free when the MMAs that read it have completed and the four ||x||^2 warps
// have read it (its `empty` barrier counts 1 + 4 arrivals).
constexpr int K1T_BM = 128;
constexpr int K1T_THREADS = 192;
constexpr int K1T_MAXST = 5;
template <int NP>
__host__ __device__ constexpr int k1t_stages() { return NP <= 32 ? 5 : 4; }
template <int NP>
__host__ __device__ constexpr size_t k1t_stage_bytes() { return (size_t)(K1T_BM + NP) * 256; }
template <int NP>
__host__ __device__ constexpr size_t k1t_smem_bytes() {
  return (size_t)k1t_stages<NP>() * k1t_stage_bytes<NP>() + 1024;
}

// shared-memory matrix descriptor: K-major operand, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address (16-byte units)
  d |= (uint64_t)1u << 16;                          // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024u >> 4) << 32;                // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1u << 46;                          // descriptor version (sm_100 family)
  d |= (uint64_t)2u << 61;                          // layout: 128-byte swizzle
  return d;
}
// instruction descriptor, kind::f16: FP32 accumulator, A and B of the ingest type, both K-major
template <typename TX>
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N) {
  return (1u << 4) | ((std::is_same<TX, __nv_bfloat16>::value ? 1u : 0u) << 7) |
         ((std::is_same<TX, __nv_bfloat16>::value ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(holder), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (lane = thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// the two 16-bit values packed in w, widened to FP32
template <typename TX>
__device__ __forceinline__ float2 sq_pair(uint32_t w) {
  if constexpr (std::is_same<TX, __half>::value) return __half22float2(*reinterpret_cast<const __half2*>(&w));
  else return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
}

template <typename TX, int NP>
__global__ void __launch_bounds__(K1T_THREADS, 1)
    k_fast_solve_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, SolveArgs a0) {
  const int zs = a0.zmap[blockIdx.z];   // grid plane z serves stream zs of the batch
  SolveArgs a = a0;
  a.Y += (size_t)zs * a.M * a.r;
  a.xx_part += (size_t)zs * gridDim.x;
  a.ctl += zs;
  static_assert(NP % 16 == 0 && NP >= 16 && NP <= 64, "NP");
  constexpr int ST = k1t_stages<NP>();
  static_assert(ST <= K1T_MAXST, "stages");
  constexpr uint32_t ABOX = K1T_BM * 128, BBOX = NP * 128;     // one 64-column box of X / of B
  constexpr uint32_t ABYTES = 2 * ABOX, BBYTES = 2 * BBOX;
  constexpr uint32_t TCOLS = NP <= 32 ? 32 : 64;               // TMEM columns (power of 2 >= 32)
  constexpr uint32_t IDESC = umma_idesc_f16<TX>(K1T_BM, NP);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[K1T_MAXST];
  __shared__ __align__(8) uint64_t empty[K1T_MAXST];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_holder;
  __shared__ float redf[64];
  __shared__ int timeout_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rt = blockIdx.x;
  const int m0 = rt * K1T_BM;
  const int r = a.r;
  const long long K = a.K;
  const int ntk = (int)((K + 127) / 128);
  const uint32_t sbase = smem_u32(smem);
  auto stageA = [&](int st) { return sbase + (uint32_t)(st * k1t_stage_bytes<NP>()); };
  auto stageB = [&](int st) { return stageA(st) + ABYTES; };

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), 2);          // A arrival + B arrival (expect_tx)
      mbar_init(smem_u32(&empty[s]), 1 + 4);     // MMA commit + the four ||x||^2 warps
    }
    mbar_init(smem_u32(&done), 1);
    mbar_fence_init();
    timeout_flag = 0;
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_holder), TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  // X tiles do not depend on the previous kernel: start them before the dependency wait
  if (warp == 0 && lane == 0) {
    for (int t = 0; t < ST && t < ntk; ++t) {
      mbar_arrive_expect_tx(smem_u32(&full[t]), ABYTES);
      const int x = t * 128;
      tma_load_3d(stageA(t), &tmX, x, m0, zs, smem_u32(&full[t]));
      tma_load_3d(stageA(t) + ABOX, &tmX, x + 64, m0, zs, smem_u32(&full[t]));
    }
  }
  pdl_wait();       // the previous step's env kernel wrote B and ctl
  pdl_trigger();
  const bool bzero = (a.ctl->cc == 0.0);
  if (bzero) {
    // e_1 rule for a zero temporal row: B stays zero but for B[0][0] of the first stage
    for (int st = 0; st < ST; ++st)
      for (int e = tid; e < (int)BBYTES / 16; e += K1T_THREADS)
        *reinterpret_cast<uint4*>(smem + (stageB(st) - sbase) + e * 16) = make_uint4(0, 0, 0, 0);
    fence_proxy_async_smem();                  // each thread's writes, before the MMAs read them
    __syncthreads();
    if (tid == 0) {
      *reinterpret_cast<TX*>(smem + (stageB(0) - sbase)) = from_acc<TX>(1.0f);
      fence_proxy_async_smem();
    }
  }
  __syncthreads();

  float ssh = 0.f, ssl = 0.f;
  if (warp == 0) {
    // ---- producer
    if (lane == 0) {
      int issued = ntk < ST ? ntk : ST;
      for (int t = 0; t < issued; ++t) {
        if (bzero) {
          mbar_arrive_expect_tx(smem_u32(&full[t]), 0);
        } else {
          mbar_arrive_expect_tx(smem_u32(&full[t]), BBYTES);
          tma_load_3d(stageB(t), &tmB, t * 128, 0, zs, smem_u32(&full[t]));
          tma_load_3d(stageB(t) + BBOX, &tmB, t * 128 + 64, 0, zs, smem_u32(&full[t]));
        }
      }
      for (int t = ST; t < ntk; ++t) {
        const int st = t % ST;
        if (!mbar_wait(smem_u32(&empty[st]), (uint32_t)(((t / ST) - 1) & 1)) || timeout_flag) {
          timeout_flag = 1;
          break;
        }
        if (t == ST && bzero) {
          *reinterpret_cast<TX*>(smem + (stageB(0) - sbase)) = from_acc<TX>(0.f);
          fence_proxy_async_smem();
        }
        const int x = t * 128;
        mbar_arrive_expect_tx(smem_u32(&full[st]), ABYTES);
        tma_load_3d(stageA(st), &tmX, x, m0, zs, smem_u32(&full[st]));
        tma_load_3d(stageA(st) + ABOX, &tmX, x + 64, m0, zs, smem_u32(&full[st]));
        if (bzero) {
          mbar_arrive_expect_tx(smem_u32(&full[st]), 0);
        } else {
          mbar_arrive_expect_tx(smem_u32(&full[st]), BBYTES);
          tma_load_3d(stageB(st), &tmB, x, 0, zs, smem_u32(&full[st]));
          tma_load_3d(stageB(st) + BBOX, &tmB, x + 64, 0, zs, smem_u32(&full[st]));
        }
        issued = t + 1;
      }
      if (timeout_flag) {
        for (int t = issued - ST > 0 ? issued - ST : 0; t < issued; ++t)
          mbar_wait(smem_u32(&full[t % ST]), (uint32_t)((t / ST) & 1));
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    int t = 0;
    if (lane == 0) {
      for (; t < ntk; ++t) {
        const int st = t % ST;
        if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((t / ST) & 1)) || timeout_flag) {
          timeout_flag = 1;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int bx = 0; bx < 2; ++bx) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = umma_desc_sw128(stageA(st) + bx * ABOX + kk * 32);
            const uint64_t bd = umma_desc_sw128(stageB(st) + bx * BBOX + kk * 32);
            umma_f16(tmem, ad, bd, IDESC, (t | bx | kk) != 0 ? 1u : 0u);
          }
        }
        umma_commit(smem_u32(&empty[st]));     // the stage is free once these MMAs completed
      }
      umma_commit(smem_u32(&done));            // every MMA issued above has completed
    }
    __syncwarp();
  } else {
    // ---- ||x||^2 of the staged X tiles (thread = row of the tile)
    const int row = tid - 64;                  // 0..127
    for (int t = 0; t < ntk; ++t) {
      const int st = t % ST;
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((t / ST) & 1)) || timeout_flag) {
        timeout_flag = 1;
        break;
      }
      // shared-memory loads on 32-bit shared addresses, chunk c of the row read where the
      // 128-byte swizzle put it (c ^ row % 8: the 8 rows of a quarter-warp hit 8 different
      // bank groups; the unswizzled offset made every lane of a warp hit the same ones), eight
      // independent accumulators, summed in a fixed order
      float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f, q4 = 0.f, q5 = 0.f, q6 = 0.f, q7 = 0.f;
#pragma unroll
      for (int bx = 0; bx < 2; ++bx) {
        const uint32_t rp = stageA(st) + (uint32_t)(bx * ABOX + row * 128);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          uint32_t w0, w1, w2, w3;
          asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];\n"
                       : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3)
                       : "r"(rp + (uint32_t)((c ^ (row & 7)) * 16)));
          const float2 f0 = sq_pair<TX>(w0), f1 = sq_pair<TX>(w1), f2 = sq_pair<TX>(w2), f3 = sq_pair<TX>(w3);
          q0 = fmaf(f0.x, f0.x, q0);
          q1 = fmaf(f0.y, f0.y, q1);
          q2 = fmaf(f1.x, f1.x, q2);
          q3 = fmaf(f1.y, f1.y, q3);
          q4 = fmaf(f2.x, f2.x, q4);
          q5 = fmaf(f2.y, f2.y, q5);
          q6 = fmaf(f3.x, f3.x, q6);
          q7 = fmaf(f3.y, f3.y, q7);
        }
      }
      const float ss = ((q0 + q1) + (q2 + q3)) + ((q4 + q5) + (q6 + q7));
      two_sum_acc(ssh, ssl, ss);
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[st]));
    }
  }
  // ---- epilogue: the accumulator -> the tile Ys in shared memory over the stage buffers,
  // which are free once every MMA has completed (warps 2-5: TMEM lanes 32 (warp % 4) ..;
  // zero past r and past I_1)
  constexpr int LDY = NP + 4;
  static_assert((size_t)(K1T_BM * LDY + (tile_gram_groups<NP, K1T_THREADS>() + 1) * NP * NP) * 4 <=
                    (size_t)ST * k1t_stage_bytes<NP>(), "epilogue tiles fit the stage buffers");
  float* Ys = reinterpret_cast<float*>(smem);                  // [128][LDY]
  float* Gr = Ys + K1T_BM * LDY;                               // row-group partials
  float* G = Gr + tile_gram_groups<NP, K1T_THREADS>() * NP * NP;
  if (warp >= 2) {
    const bool ok = mbar_wait(smem_u32(&done), 0);
    if (!ok) timeout_flag = 1;
    tc_fence_after();
    const int q = warp & 3;                    // TMEM lane quarter of this warp
    const int row = q * 32 + lane;
    const bool in = m0 + row < a.M;
    float v[32];
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 32) {
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
      if (ok) {
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4)
          if (c0 + 4 * j4 < NP) {
            float4 w;
            w.x = (in && c0 + 4 * j4 + 0 < r) ? v[4 * j4 + 0] : 0.f;
            w.y = (in && c0 + 4 * j4 + 1 < r) ? v[4 * j4 + 1] : 0.f;
            w.z = (in && c0 + 4 * j4 + 2 < r) ? v[4 * j4 + 2] : 0.f;
            w.w = (in && c0 + 4 * j4 + 3 < r) ? v[4 * j4 + 3] : 0.f;
            *reinterpret_cast<float4*>(Ys + row * LDY + c0 + 4 * j4) = w;
          }
      }
    }
  }
  tc_fence_before();
  const float2 ss_cta = ff_block_sum(ssh, ssl, redf);   // (includes a block barrier)
  if (tid == 0) {
    // one partial of ||x||^2 per row tile; NaN after a wait gave up (the step is not committed)
    a.xx_part[rt] = timeout_flag ? make_float2(__int_as_float(0x7fc00000), 0.f) : ss_cta;
    if (timeout_flag) a.ctl->latched = 5;
  }
  __syncthreads();
  if (!timeout_flag) {      // block-uniform here
    // the tile's rows of Y, coalesced (rows of Y are contiguous)
    const int nrow = a.M - m0 < K1T_BM ? a.M - m0 : K1T_BM;
    for (int e = tid; e < nrow * r; e += K1T_THREADS) a.Y[(long long)m0 * r + e] = Ys[(e / r) * LDY + e % r];
    // the tile's Gram partial (FP32 over its 128 rows; lo part zero)
    tile_gram<NP, K1T_THREADS>(Ys, LDY, K1T_BM, Gr, G);
    float2* W1t = a.W1part + (size_t)zs * a.w1_stride + (size_t)rt * NP * NP;
    for (int e = tid; e < NP * NP; e += K1T_THREADS) W1t[e] = make_float2(G[e], 0.f);
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, TCOLS);
}

// ================================================================ K1b: r x r factor
// A cluster of KBC (8, or 4 for large batches) CTAs; CTA q owns rows [q*nrows, (q+1)*nrows)
// of Y.
//  1. W1 = Y^T Y: every rank sums the solve kernel's row-tile Gram partials in tile order
//     (float-float) while its rows of Y are still arriving.
//  2. Every rank factors the scaled Gram D W1 D = L L^T: in FP64 (r64::ldl_factor, the
//     default) or in FP32 (one warp).
//  3. Q1 = Y D L^{-T}: each thread forward-substitutes whole rows, z = L^{-1} (D y),
//     and rounds them to the ingest type (the values that multiply X in the env kernel).
//  4. W2 partial = (my rounded rows)^T (my rounded rows) on tensor cores (exact products),
//     written to global memory; the environment kernel sums the partials in rank order.
// A failed factorisation (scaled pivot <= 1e-4: an ill-conditioned local solve) takes an
// FP64-accurate Cholesky-QR instead (float-float Gram of Y, FP64 factor, float-float apply);
// only a pivot at FP64 rounding takes the FP64 Householder QR of Y on rank 0.
constexpr int K1B_THREADS = 256;
constexpr int KB_CLUSTER = 8;       // the largest factor cluster: W2-partial slab stride
// static shared memory of k_fast_factor (W1 as float + its rounding error, L^T, the FP64
// factor's columns, small arrays), rounded up; the launch checks dynamic + static <= 227 KB
constexpr int K1B_STATIC_SMEM = 76 * 1024;

struct FactorArgs {
  const float* Y;         // M x r
  const float2* xx_part;  // [nxx] float-float partials of ||x||^2
  const float2* W1part;   // [nw1][NP*NP] float-float Gram partials of Y's row tiles (solve kernel)
  long long w1_stride;    // float2 elements per stream of W1part
  int nw1;
  int nxx, M, r;
  void* Qh;               // M x NP ingest-type Q1 (columns >= r zero)
  float* Qst;             // state: Q1 (M x r) as float
  float* W2part;          // [KB_CLUSTER][NP*NP] W2 partials of the ranks' rows (the first KBC)
  double* hh_work;        // 2*M*r doubles (fallback)
  float* Qfb;             // M x r (fallback Q, float)
  Ctl* ctl;
  int fp64;               // 1: the r x r factor in FP64 (r64::ldl_factor), 0: FP32 (one warp)
  float* Gff;             // [KB_CLUSTER][2][NP*NP] float-float Gram partials (ill-conditioned steps)
  double* L64ws;          // [KB_CLUSTER][NP*NP] FP64 factor of each rank (ill-conditioned steps)
  unsigned char zmap[64];      // grid plane blockIdx.z -> stream (slot) of the batch
};

// rows of Y handled by one CTA of a factor cluster of kbc CTAs
__host__ __device__ constexpr int k1b_rows(int M, int kbc = KB_CLUSTER) { return ((M + kbc - 1) / kbc + 15) / 16 * 16; }
// dynamic shared memory: Y rows (fp32, stride NP+4) | Q1 rows (ingest type, stride NP+8) |
// this rank's W2 partial
__host__ __device__ constexpr size_t k1b_smem_bytes(int M, int r, int np, int kbc = KB_CLUSTER) {
  return (size_t)k1b_rows(M, kbc) * (np + 4) * 4 + (size_t)(k1b_rows(M, kbc) + 16) * (np + 8) * 2 +
         (size_t)np * np * 4 + 256 + 0 * r;
}

template <typename TX, int NP, int KBC>
__global__ void __launch_bounds__(K1B_THREADS, 1) k_fast_factor(FactorArgs a0) {
  static_assert(KBC == 4 || KBC == 8, "factor cluster of 4 or 8 CTAs");
  // grid plane z serves stream zs of the batch: its state and scratch slabs
  const int zs = a0.zmap[blockIdx.z];
  FactorArgs a = a0;
  a.Y += (size_t)zs * a.M * a.r;
  a.xx_part += (size_t)zs * a.nxx;
  a.W1part += (size_t)zs * a.w1_stride;
  a.Qh = (void*)((TX*)a.Qh + (size_t)zs * a.M * NP);
  a.Qst += (size_t)zs * a.M * a.r;
  a.W2part += (size_t)zs * KB_CLUSTER * NP * NP;
  a.hh_work += (size_t)zs * 2 * a.M * a.r;
  a.Qfb += (size_t)zs * a.M * a.r;
  a.Gff += (size_t)zs * KB_CLUSTER * 2 * NP * NP;
  a.L64ws += (size_t)zs * KB_CLUSTER * NP * NP;
  a.ctl += zs;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int LDY = NP + 4, LQ = NP + 8, LDT = NP + 4;
  __shared__ float W[64 * 64];             // W1 (FP32 rounding of its float-float sum)
  __shared__ float Wlo[64 * 64];           // W1 - W exactly: W1 = W + Wlo (the FP64 factor's input)
  __shared__ r64::Smem ldlsm;
  __shared__ __align__(16) float LT[64 * 68];   // L^T: LT[k*LDT + i] = L[i][k] (zero above)
  __shared__ float dsc[64];
  __shared__ float invd[64];               // 1 / L[i][i]
  __shared__ __align__(16) float LTlo[64 * 68];  // L - LT exactly enough for float-float (ill-conditioned steps)
  __shared__ float invdlo[64];
  __shared__ double red[32];
  __shared__ int flags[2];                 // [0] non-finite, [1] factorisation failed
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = a.r, rr = r * r;
  const uint32_t crank = cluster_rank();
  const int nrows = k1b_rows(a.M, KBC);
  const int row0 = (int)crank * nrows;
  const int myrows = (a.M - row0 < nrows) ? (a.M - row0 > 0 ? a.M - row0 : 0) : nrows;
  float* Ys = reinterpret_cast<float*>(smem);                               // [nrows][LDY]
  TX* Qs = reinterpret_cast<TX*>(Ys + (size_t)nrows * LDY);                 // [nrows+16][LQ]
  float* Wp = reinterpret_cast<float*>(Qs + (size_t)(nrows + 16) * LQ);     // [NP*NP]
  pdl_wait();
  pdl_trigger();
  TTRACE(10);
  TTRACE_CTA2(0);
  // ---- my rows of Y (asynchronous copies; padding columns r..NP-1 zero)
  if ((r & 3) == 0) {
    const int cpr = r / 4;
    for (int e = tid; e < myrows * cpr; e += K1B_THREADS) {
      const int row = e / cpr, ch = e % cpr;
      cp_async16(smem_u32(Ys + row * LDY + ch * 4), a.Y + (long long)(row0 + row) * r + ch * 4, 16u);
    }
  } else {
    for (int e = tid; e < myrows * r; e += K1B_THREADS)
      cp_async4(smem_u32(Ys + (e / r) * LDY + e % r), a.Y + (long long)row0 * r + e);
  }
  cp_async_commit();
  if (r < NP)
    for (int e = tid; e < myrows * (NP - r); e += K1B_THREADS) Ys[(e / (NP - r)) * LDY + r + e % (NP - r)] = 0.f;
  if (warp == 0) {
    float xh = 0.f, xl = 0.f;
    for (int b0 = lane; b0 < a.nxx; b0 += 32 * 8) {
      float2 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (b0 + 32 * q < a.nxx) ? a.xx_part[b0 + 32 * q] : make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 8; ++q) ff_add(xh, xl, v[q].x, v[q].y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float bh = __shfl_down_sync(0xffffffffu, xh, o), bl = __shfl_down_sync(0xffffffffu, xl, o);
      ff_add(xh, xl, bh, bl);
    }
    if (lane == 0) {
      const double xs = (double)xh + (double)xl;
      flags[0] = !isfinite(xs);
      flags[1] = 0;
      if (crank == 0 && !flags[0]) a.ctl->xx = xs;   // a skipped step keeps the committed value
    }
  }
  // ---- 1. W1 = sum of the row tiles' Gram partials in tile order (float-float).  Thread t
  // owns the packed lower-triangle entries t, t + 256, ...; all its loads of a batch of
  // partials are issued together (one L2 round trip per batch), then summed in tile order.
  {
    constexpr int NE = NP * (NP + 1) / 2, U = (NE + K1B_THREADS - 1) / K1B_THREADS;
    constexpr int PB = 54 / U > 0 ? 54 / U : 1;    // partials per batch: ~54 loads in flight
    const int ne = r * (r + 1) / 2;
    int off[U];
    float hi[U], lo[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = tid + u * K1B_THREADS;
      int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while (i > 0 && i * (i + 1) / 2 > e) --i;
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      off[u] = e < ne ? i * NP + (e - i * (i + 1) / 2) : -1;
      hi[u] = 0.f;
      lo[u] = 0.f;
    }
    for (int t0 = 0; t0 < a.nw1; t0 += PB) {
      float2 v[U][PB];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < PB; ++q)
          v[u][q] = (off[u] >= 0 && t0 + q < a.nw1) ? __ldcg(a.W1part + (size_t)(t0 + q) * NP * NP + off[u])
                                                    : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < PB; ++q) ff_add(hi[u], lo[u], v[u][q].x, v[u][q].y);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (off[u] >= 0) {
        const int i = off[u] / NP, j = off[u] % NP;
        const float w = hi[u] + lo[u], wl = (hi[u] - w) + lo[u];   // exact split (|lo| <= ulp(hi) / 2)
        W[i * r + j] = w;
        Wlo[i * r + j] = wl;
        W[j * r + i] = w;
        Wlo[j * r + i] = wl;
      }
  }
  __syncthreads();
  TTRACE(16);
  for (int e = tid; e < rr; e += K1B_THREADS)
    if (!isfinite(W[e])) flags[0] = 1;
  if (tid < 64) {
    const float d = tid < r ? W[tid * r + tid] : 0.f;
    dsc[tid] = d > 0.f ? rsqrtf(d) : 0.f;
    invd[tid] = 0.f;
    if (tid < r && !(d > 0.f)) flags[1] = 1;
  }
  __syncthreads();
  if (crank == 0 && tid == 0) {
    a.ctl->fallback[0] = 0;
    a.ctl->skip = flags[0];
    if (flags[0] && a.ctl->latched != 5) a.ctl->latched = 4;   // a solve timeout stays ETIMEOUT
  }
  if (flags[0]) {           // uniform across the cluster (identical W1 and ||x||^2)
    cp_async_wait<0>();
    return;
  }
  TTRACE(11);
  TTRACE_CTA2(1);
  // ---- 2. Cholesky of the scaled Gram: D W1 D = L L^T, stored transposed (LT)
  for (int e = tid; e < NP * LDT; e += K1B_THREADS) LT[e] = 0.f;
  __syncthreads();
  if (!flags[1] && a.fp64) {
    // FP64: W1 = W + Wlo (its float-float sum) scaled by D.  A scaled pivot D_k <= 1e-4 takes
    // the Householder path, as in the FP32 factor below: the threshold is set by the FP32 tall
    // apply z = L^{-1} (D y), whose rows each see their own rounding of L^{-1}, so that the
    // span of Q1 drifts from span(Y) by about 6e-8 cond(Y) (measured: a 1e-8 threshold let
    // streams through whose RE moved by 1e-3 from the oracle's)
    const auto load = [&](int i, int j) -> double {
      return ((double)W[i * r + j] + (double)Wlo[i * r + j]) * (double)dsc[i] * (double)dsc[j];
    };
    if (tid < 128) {
      const bool ok = r64::ldl_factor<128, NP>(r, load, 1e-4, ldlsm, LT, LDT, invd, nullptr, 0);
      if (!ok && tid == 0) flags[1] = 1;
    }
    __syncthreads();
  } else if (!flags[1]) {
    if constexpr (NP <= 32) {
      if (warp == 0) {
        float l[32];
        const float di = lane < r ? dsc[lane] : 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) l[k] = 0.f;
        int ok = 1;
        // left-looking, lane i holds row i of L; fully unrolled (register-indexed rows)
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          // W1 is symmetric: W[j][lane] = W[lane][j], read along the row (conflict-free)
          const float wj = (lane < r && j < r) ? W[j * r + lane] * di * dsc[j] : (lane == j ? 1.f : 0.f);
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
          if (j < r && !(piv > 1e-4f)) ok = 0;
          const float rl = rsqrtf(piv > 0.f ? piv : 1.f);
          l[j] = (lane == j) ? piv * rl : (lane > j ? sv * rl : 0.f);
          if (lane == j && j < r) invd[j] = rl;
        }
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (lane < r && k < r) LT[k * LDT + lane] = l[k];
        if (lane == 0) flags[1] = ok ? 0 : 1;
      }
    } else {
      float* Lw = W;                           // in place (W1 is not needed afterwards)
      const int LD = r;
      for (int e = tid; e < rr; e += K1B_THREADS) W[e] *= dsc[e / r] * dsc[e % r];
      __syncthreads();
      for (int j = 0; j < r; ++j) {
        const float piv = Lw[j * LD + j];
        if (!(piv > 1e-4f)) {
          if (tid == 0) flags[1] = 1;
          break;                      // uniform
        }
        const float rl = rsqrtf(piv);
        for (int e = tid; e < rr; e += K1B_THREADS) {
          const int i = e / r, k = e % r;
          if (i > j && k > j && k <= i) Lw[i * LD + k] -= Lw[i * LD + j] * Lw[k * LD + j] / piv;
        }
        __syncthreads();
        if (tid >= j && tid < r) Lw[tid * LD + j] *= rl;
        if (tid == j) invd[j] = rl;
        __syncthreads();
      }
      if (!flags[1])
        for (int e = tid; e < rr; e += K1B_THREADS) {
          const int i = e / r, k = e % r;
          if (k <= i) LT[k * LDT + i] = Lw[i * LD + k];
        }
    }
  }
  cp_async_wait<0>();       // my rows of Y
  __syncthreads();
  TTRACE(12);
  TX* Qh = (TX*)a.Qh;
  const bool fb = flags[1] != 0;      // identical in every CTA of the cluster
  bool hh = false;
  if (fb) {
    // A scaled pivot <= 1e-4: the local solve is ill-conditioned for the FP32 Gram and apply.
    // FP64-accurate Cholesky-QR instead: float-float Gram of my rows (TwoProd, TwoSum), the
    // cluster's partials summed in FP64 by every rank, the FP64 factor, a float-float apply.
    // Only a pivot <= 1e-14 (the columns dependent to FP64 precision) takes the Householder QR.
    float* gp = a.Gff + (size_t)crank * 2 * NP * NP;
    for (int e = tid; e < rr; e += K1B_THREADS) {
      const int i = e / r, j = e % r;
      float sh = 0.f, sl = 0.f;
      if (j <= i) {
        for (int row = 0; row < myrows; ++row) {
          const float yi = Ys[row * LDY + i], yj = Ys[row * LDY + j];
          const float pr = yi * yj;
          two_sum_acc(sh, sl, pr);
          sl += fmaf(yi, yj, -pr);                 // pr + fma error = yi yj exactly
        }
      }
      gp[e] = sh;
      gp[NP * NP + e] = sl;
    }
    cluster_sync();                   // every rank's partial is in global memory
    const auto load64 = [&](int i, int j) -> double {
      double v = 0.0;
      for (int q = 0; q < KBC; ++q) {
        const float* gq = a.Gff + (size_t)q * 2 * NP * NP;
        v += (double)__ldcg(gq + i * r + j) + (double)__ldcg(gq + NP * NP + i * r + j);
      }
      return v * (double)dsc[i] * (double)dsc[j];
    };
    double* L64 = a.L64ws + (size_t)crank * NP * NP;
    if (tid < 128) {
      const bool ok = r64::ldl_factor<128, NP>(r, load64, 1e-14, ldlsm, LT, LDT, nullptr, L64, NP);
      if (!ok && tid == 0) flags[1] = 2;
    }
    __syncthreads();
    hh = flags[1] == 2;               // identical in every rank (same sums, same factor)
    if (!hh) {
      for (int e = tid; e < rr; e += K1B_THREADS) {
        const int i = e / r, k = e % r;
        if (k <= i) LTlo[k * LDT + i] = (float)(L64[i * NP + k] - (double)LT[k * LDT + i]);
      }
      if (tid < r) {
        const double rd = 1.0 / L64[tid * NP + tid];
        invd[tid] = (float)rd;
        invdlo[tid] = (float)(rd - (double)invd[tid]);
      }
      __syncthreads();
    } else {
      if (crank == 0) householder_cta<float, float>(a.Y, a.M, r, r, a.hh_work, a.Qfb, r, red);
      cluster_sync();                 // Qfb complete before the other ranks read it
    }
  }
  // ---- 3. Q1 rows: z = L^{-1} (D y) by forward substitution, in place in the row of Ys,
  // in 8-column register blocks (Householder Q: z = q)
  const int nb8 = (r + 7) / 8;
  for (int row = tid; row < nrows + 16; row += K1B_THREADS) {
    float* zr = Ys + row * LDY;
    if (row < myrows) {
      if (!fb) {
#pragma unroll
        for (int c4 = 0; c4 < NP / 4; ++c4) {
          float4 y = *reinterpret_cast<const float4*>(zr + 4 * c4);
          y.x *= dsc[4 * c4];
          y.y *= dsc[4 * c4 + 1];
          y.z *= dsc[4 * c4 + 2];
          y.w *= dsc[4 * c4 + 3];
          *reinterpret_cast<float4*>(zr + 4 * c4) = y;
        }
        for (int kb = 0; kb < nb8; ++kb) {
          float zb[8];
          {
            const float4 u = *reinterpret_cast<const float4*>(zr + 8 * kb);
            const float4 v = *reinterpret_cast<const float4*>(zr + 8 * kb + 4);
            zb[0] = u.x; zb[1] = u.y; zb[2] = u.z; zb[3] = u.w;
            zb[4] = v.x; zb[5] = v.y; zb[6] = v.z; zb[7] = v.w;
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            zb[k] *= invd[8 * kb + k];                 // zero past r
#pragma unroll
            for (int i = k + 1; i < 8; ++i) zb[i] = fmaf(-LT[(8 * kb + k) * LDT + 8 * kb + i], zb[k], zb[i]);
          }
          *reinterpret_cast<float4*>(zr + 8 * kb) = make_float4(zb[0], zb[1], zb[2], zb[3]);
          *reinterpret_cast<float4*>(zr + 8 * kb + 4) = make_float4(zb[4], zb[5], zb[6], zb[7]);
          for (int jb = kb + 1; jb < nb8; ++jb) {
            const float4 u = *reinterpret_cast<const float4*>(zr + 8 * jb);
            const float4 v = *reinterpret_cast<const float4*>(zr + 8 * jb + 4);
            float zj[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const float4 la = *reinterpret_cast<const float4*>(LT + (8 * kb + k) * LDT + 8 * jb);
              const float4 lb = *reinterpret_cast<const float4*>(LT + (8 * kb + k) * LDT + 8 * jb + 4);
              zj[0] = fmaf(-la.x, zb[k], zj[0]);
              zj[1] = fmaf(-la.y, zb[k], zj[1]);
              zj[2] = fmaf(-la.z, zb[k], zj[2]);
              zj[3] = fmaf(-la.w, zb[k], zj[3]);
              zj[4] = fmaf(-lb.x, zb[k], zj[4]);
              zj[5] = fmaf(-lb.y, zb[k], zj[5]);
              zj[6] = fmaf(-lb.z, zb[k], zj[6]);
              zj[7] = fmaf(-lb.w, zb[k], zj[7]);
            }
            *reinterpret_cast<float4*>(zr + 8 * jb) = make_float4(zj[0], zj[1], zj[2], zj[3]);
            *reinterpret_cast<float4*>(zr + 8 * jb + 4) = make_float4(zj[4], zj[5], zj[6], zj[7]);
          }
        }
      } else if (!hh) {
        // float-float forward substitution: z = L^{-1} (D y), L = LT + LTlo, 1/L_ii = invd + invdlo;
        // the high part replaces y in place, the low part stays in zl
        float zl[NP];
        for (int i = 0; i < r; ++i) {
          const float y = zr[i];
          float sh = y * dsc[i];
          float sl = fmaf(y, dsc[i], -sh);
          for (int k = 0; k < i; ++k) {
            const float lh = LT[k * LDT + i], ll = LTlo[k * LDT + i];
            const float zh = zr[k], zlk = zl[k];
            const float pr = lh * zh;
            const float pe = fmaf(lh, zh, -pr) + (lh * zlk + ll * zh);
            two_sum_acc(sh, sl, -pr);
            sl -= pe;
          }
          const float rh = invd[i], rl = invdlo[i];
          const float q = sh * rh;
          const float qe = fmaf(sh, rh, -q) + (sh * rl + sl * rh);
          const float zh = q + qe;
          zl[i] = qe - (zh - q);
          zr[i] = zh;
        }
        for (int c = r; c < NP; ++c) zr[c] = 0.f;
      } else {
        for (int c = 0; c < NP; ++c) zr[c] = c < r ? a.Qfb[(long long)(row0 + row) * r + c] : 0.f;
      }
    }
    float z[NP];
    if (row < myrows) {
#pragma unroll
      for (int c4 = 0; c4 < NP / 4; ++c4) {
        const float4 v = *reinterpret_cast<const float4*>(zr + 4 * c4);
        z[4 * c4] = v.x; z[4 * c4 + 1] = v.y; z[4 * c4 + 2] = v.z; z[4 * c4 + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < NP; ++c) z[c] = 0.f;     // rows past my share: read by the last k-step
    }
    // rounded row -> shared memory (W2 operand; written out below)
#pragma unroll
    for (int c8 = 0; c8 < NP / 8; ++c8) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const TX lo = from_acc<TX>(z[8 * c8 + 2 * q]), hi = from_acc<TX>(z[8 * c8 + 2 * q + 1]);
        w[q] = (uint32_t)tx_bits(lo) | ((uint32_t)tx_bits(hi) << 16);
      }
      *reinterpret_cast<uint4*>(Qs + row * LQ + 8 * c8) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  TTRACE(18);
  TTRACE_CTA2(2);
  __syncthreads();
  // my rows of Q1, coalesced: ingest-type copy (16-byte chunks) and FP32 state
  for (int e = tid; e < myrows * (NP / 8); e += K1B_THREADS) {
    const int row = e / (NP / 8), c8 = e % (NP / 8);
    *reinterpret_cast<uint4*>(Qh + (long long)(row0 + row) * NP + 8 * c8) =
        *reinterpret_cast<const uint4*>(Qs + row * LQ + 8 * c8);
  }
  for (int e = tid; e < myrows * r; e += K1B_THREADS)
    a.Qst[(long long)row0 * r + e] = Cvt<TX>::f(Qs[(e / r) * LQ + e % r]);
  TTRACE(13);
  // ---- 4. W2 partial of my rows on tensor cores: warp w owns output tiles w, w+8, ...
  {
    constexpr int MT = NP / 16, NTT = NP / 8;
    const int ksteps = (myrows + 15) / 16;
    const int g = lane >> 2, t4 = lane & 3;
    for (int tile = warp; tile < MT * NTT; tile += K1B_THREADS / 32) {
      const int m = tile / NTT, n = tile % NTT;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int ks = 0; ks < ksteps; ++ks) {
        const int k0 = ks * 16;
        uint32_t af[4], b0, b1;
        ldsm_x4_t(smem_u32(Qs + (k0 + (lane & 7) + ((lane >> 4) << 3)) * LQ + m * 16 + ((lane >> 3) & 1) * 8), af[0],
                  af[1], af[2], af[3]);
        ldsm_x2_t(smem_u32(Qs + (k0 + (lane & 7) + (((lane >> 3) & 1) << 3)) * LQ + n * 8), b0, b1);
        mma16816<TX>(acc, af, b0, b1);
      }
      const int row = m * 16 + g, col = n * 8 + 2 * t4;
      Wp[row * NP + col] = acc[0];
      Wp[row * NP + col + 1] = acc[1];
      Wp[(row + 8) * NP + col] = acc[2];
      Wp[(row + 8) * NP + col + 1] = acc[3];
    }
  }
  __syncthreads();
  TTRACE(19);
  // this rank's W2 partial (its rows of Q1) to global memory; the environment kernel sums
  // the ranks' partials in rank order and forms Nx = W2^{-1} - I itself
  for (int e = tid; e < NP * NP; e += K1B_THREADS) a.W2part[(size_t)crank * NP * NP + e] = Wp[e];
  if (tid == 0 && crank == 0 && fb) a.ctl->fallback[0] = 1;
  TTRACE(15);
  TTRACE_CTA2(3);
}

constexpr int K2_THREADS = 256;
constexpr int K2_BN = 128;            // slice columns j per CTA of the clustered env kernel

// W2 = sum over the factor kernel's ranks (rank order, TwoSum) of its NP x NP partials; the
// state's W2 (r x r) is written when `write_state`.  sD receives D2 = W2 - I zero-padded to
// NP x NP and sN receives Nx = W2^{-1} - I = -D2 + D2^2 (|D2| ~ 1e-3 for a rounded
// orthonormal basis, so the D2^3 term is below 1e-8), zero past r.  D2^2 is a fully unrolled
// 2 x 2 register-blocked product.  All K2_THREADS threads; ends synchronised.
template <int NP>
__device__ __forceinline__ void env_w2_nx(const float* __restrict__ W2part, int r, float* sD, float* sN,
                                          float* W2st, bool write_state, int nparts) {
  const int tid = threadIdx.x;
  const bool worker = tid < K2_THREADS;       // extra (producer) warps only synchronise
  constexpr int PER = (NP * NP + K2_THREADS - 1) / K2_THREADS;
  constexpr int G = PER < 4 ? PER : 4;       // elements whose partials are loaded together
  for (int u0 = 0; worker && u0 < PER; u0 += G) {
  float v[G][KB_CLUSTER];
#pragma unroll
  for (int u = 0; u < G; ++u) {
    const int e = tid + (u0 + u) * K2_THREADS;
    const int ec = e < NP * NP ? e : NP * NP - 1;
#pragma unroll
    for (int q = 0; q < KB_CLUSTER; ++q) v[u][q] = q < nparts ? __ldcg(W2part + (size_t)q * NP * NP + ec) : 0.f;
  }
#pragma unroll
  for (int u = 0; u < G; ++u) {
    const int e = tid + (u0 + u) * K2_THREADS;
    if (e < NP * NP) {
      const int i = e / NP, j = e % NP;
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int q = 0; q < KB_CLUSTER; ++q) two_sum_acc(hi, lo, v[u][q]);
      const float w = hi + lo;
      const bool in = i < r && j < r;
      sD[e] = in ? w - (i == j ? 1.f : 0.f) : 0.f;
      if (write_state && in) W2st[i * r + j] = w;
    }
  }
  }
  __syncthreads();
  constexpr int HB = NP / 2;
  for (int blk = tid; worker && blk < HB * HB; blk += K2_THREADS) {
    const int i0 = 2 * (blk / HB), j0 = 2 * (blk % HB);
    float c00 = 0.f, c01 = 0.f, c10 = 0.f, c11 = 0.f;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const float a0 = sD[i0 * NP + k], a1 = sD[(i0 + 1) * NP + k];
      const float2 bk = *reinterpret_cast<const float2*>(sD + k * NP + j0);
      c00 = fmaf(a0, bk.x, c00);
      c01 = fmaf(a0, bk.y, c01);
      c10 = fmaf(a1, bk.x, c10);
      c11 = fmaf(a1, bk.y, c11);
    }
    *reinterpret_cast<float2*>(sN + i0 * NP + j0) =
        make_float2(c00 - sD[i0 * NP + j0], c01 - sD[i0 * NP + j0 + 1]);
    *reinterpret_cast<float2*>(sN + (i0 + 1) * NP + j0) =
        make_float2(c10 - sD[(i0 + 1) * NP + j0], c11 - sD[(i0 + 1) * NP + j0 + 1]);
  }
  __syncthreads();
}

// ||x^||^2 terms f_c (f + Nx f)_c of the columns of an F tile held as sF[jl*ldf + c] (c < r),
// and the state writes of those columns.  Thread t owns column jl = t % 64 (+64, ...) and
// the NP/4 rows c of group t / 64 (256 threads); Nx is NP x NP with zeros past r.  Adds to
// the thread's float-float partial (ph, pl).
template <typename TX, int NP>
__device__ __forceinline__ void env_columns_out(const float* sF, int ldf, const float* sN, int ncols, int r,
                                                long long J, long long gj0, float* Cst, TX* Chst, float scale,
                                                float& ph, float& pl) {
  const int cg = threadIdx.x / 64;
  for (int jl = threadIdx.x % 64; jl < ncols; jl += 64) {
    float fv[NP];
#pragma unroll
    for (int b = 0; b < NP; ++b) fv[b] = b < r ? sF[jl * ldf + (b < r ? b : 0)] : 0.f;
    const long long gj = gj0 + jl;
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) {
      const int c = cg * (NP / 4) + q;
      if (c < r) {
        const float* nrow = sN + c * NP;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
        for (int b4 = 0; b4 < NP / 4; ++b4) {
          const float4 nv = *reinterpret_cast<const float4*>(nrow + 4 * b4);
          g0 = fmaf(nv.x, fv[4 * b4], g0);
          g1 = fmaf(nv.y, fv[4 * b4 + 1], g1);
          g2 = fmaf(nv.z, fv[4 * b4 + 2], g2);
          g3 = fmaf(nv.w, fv[4 * b4 + 3], g3);
        }
        const float fc = sF[jl * ldf + c];
        two_sum_acc(ph, pl, fc * (fc + ((g0 + g1) + (g2 + g3))));
        Cst[(long long)c * J + gj] = fc;
        Chst[(long long)c * J + gj] = from_acc<TX>(fc * scale);
      }
    }
  }
}

// ================================================================ K2: environment
// F^T = X_(1)^T Q1 for a 128-column tile of X; the row chunks of a column tile form a
// cluster and reduce through distributed shared memory.  Writes F (the state's right
// part) and its scaled ingest-type copy, and the step's ||x^||^2 = sum_j f_j^T (I + Nx) f_j.
// The X block arrives as two 64-column, 128B-swizzled TMA boxes of rch rows.
struct EnvArgs {
  int M, r;
  long long J;
  int rch;              // rows per cluster rank (multiple of 16)
  const void* Qh;       // M x NP ingest-type Q1
  const float* W2part;  // [KB_CLUSTER][NP*NP] W2 partials of the factor kernel's ranks
  float* Cst;           // state: F (r x J)
  void* Chst;           // state: scaled ingest-type copy of F (r x J)
  int* ch_shift;        // state: power-of-two scale exponent of Chst
  float2* cc_part;      // [CTAs] float-float partials of ||x^||^2
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
  int w2_parts;         // W2 partials written by the factor kernel (its cluster size)
  unsigned char zmap[64];      // grid plane blockIdx.z -> stream (slot) of the batch
};

template <int NP>
constexpr size_t k2_smem_bytes(int rch, int r) {
  // X block (2 x rch x 128 B) | Q1 tile | partial tile P (BN x (NP+8)) | my columns F |
  // Nx (NP x NP) | W2 (NP x NP)
  return 1024 + (size_t)rch * 256 + (size_t)rch * (NP + 8) * 2 + (size_t)K2_BN * (NP + 8) * 4 +
         (size_t)K2_BN * (r + 1) * 4 + (size_t)2 * NP * NP * 4 + 64;
}

// the environment kernels' arguments for stream z of a batch: its state slabs, its cc
// partials and its ticket counter
template <typename TX, int NP>
__device__ __forceinline__ EnvArgs env_args_for_stream(const EnvArgs& a0, int z, int ncta_per_stream) {
  EnvArgs a = a0;
  const size_t mr = (size_t)a.M * a.r, rj = (size_t)a.r * a.J, rr = (size_t)a.r * a.r;
  a.Qh = (const void*)((const TX*)a.Qh + (size_t)z * a.M * NP);
  a.W2part += (size_t)z * KB_CLUSTER * NP * NP;
  a.Cst += z * rj;
  a.Chst = (void*)((TX*)a.Chst + z * rj);
  a.ch_shift += 2 * z;
  a.cc_part += (size_t)z * ncta_per_stream;
  a.counter += 2 * z;
  a.ctl += z;
  a.Qst += z * mr;
  a.W2st += z * rr;
  a.Qold += z * mr;
  a.Cold += z * rj;
  a.Chold = (const void*)((const TX*)a.Chold + z * rj);
  a.W2old += z * rr;
  a.ch_shift_old += 2 * z;
  return a;
}

template <typename TX, int NP>
__global__ void __launch_bounds__(K2_THREADS, 2)
    k_fast_env(const __grid_constant__ CUtensorMap tmX, EnvArgs a0) {
  const int zs = a0.zmap[blockIdx.z];     // grid plane z serves stream zs of the batch
  const EnvArgs a = env_args_for_stream<TX, NP>(a0, zs, gridDim.x * gridDim.y);
  constexpr int NT = NP / 8;   // n8-tiles per warp (each warp covers all NP columns)
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int rch = a.rch, r = a.r, rr = r * r;
  const uint32_t xsub0 = smem_u32(smem), xsub1 = xsub0 + (uint32_t)rch * 128;   // two swizzled boxes
  TX* sQ = reinterpret_cast<TX*>(smem + (size_t)rch * 256);           // [rch][NP+8]
  constexpr int LDP = NP + 8;                                        // float2 stores: 2 wavefronts
  float* P = reinterpret_cast<float*>(sQ + (size_t)rch * (NP + 8));  // [BN][NP+8]
  const int LDF = r + 1;                                             // padded: conflict-free
  float* sF = P + K2_BN * LDP;                                       // [BN][r+1] (my columns)
  float* sN = sF + K2_BN * LDF;                                      // Nx (NP x NP)
  float* sW = sN + NP * NP;                                          // D2 = W2 - I (NP x NP)
  __shared__ __align__(8) uint64_t xbar;
  __shared__ float redf[64];
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
  const bool W2_WRITER = (blockIdx.x == 0 && blockIdx.y == 0);   // one CTA writes the state's W2

  // 1. this CTA's X block through the TMA engine (independent of the previous kernels)
  if (tid == 0) {
    mbar_init(smem_u32(&xbar), 1);
    mbar_fence_init();
    timeout_flag = 0;
    const uint32_t bar = smem_u32(&xbar);
    mbar_arrive_expect_tx(bar, (uint32_t)rch * 256);
    tma_load_3d(xsub0, &tmX, (int)j0, i0, zs, bar);
    tma_load_3d(xsub1, &tmX, (int)j0 + 64, i0, zs, bar);
  }
  if (tr0) TTRACE(20);
  // 2. wait for the factor kernel (Q1, Nx, ctl)
  pdl_wait();
  pdl_trigger();
  if (tr0) TTRACE(21);
  const double xx = a.ctl->xx;     // ||x||^2 of this slice (factor kernel)
  double sum_xx = 0.0, sum_ee = 0.0;  // running totals (read early; used by the last CTA)
  long long tcount = 0;
  if (tid == 0) {
    sum_xx = a.ctl->sum_xx;
    sum_ee = a.ctl->sum_ee;
    tcount = a.ctl->t;
  }
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
    env_w2_nx<NP>(a.W2part, r, sW, sN, a.W2st, W2_WRITER, a.w2_parts);
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
      *reinterpret_cast<float2*>(P + row * LDP + col) = make_float2(acc[j][0], acc[j][1]);
      *reinterpret_cast<float2*>(P + (row + 8) * LDP + col) = make_float2(acc[j][2], acc[j][3]);
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
    for (int e0 = tid; e0 < nmy * r; e0 += 4 * K2_THREADS) {
      float v[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * K2_THREADS;
        const int ec = e < nmy * r ? e : nmy * r - 1;  // in-range address; value masked below
        const int jl = ec / r, c = ec % r;
        const uint32_t la = Pb + (uint32_t)((jb + jl) * LDP + c) * 4u;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float x = dsmem_ld_rank(la, q, nq);
          v[u][q] = e < nmy * r ? x : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * K2_THREADS;
        if (e < nmy * r) {
          float sum = 0.f;
#pragma unroll
          for (int q = 0; q < 8; ++q) sum += v[u][q];
          sF[(e / r) * LDF + e % r] = sum;
        }
      }
    }
  }
  cluster_sync();   // every rank has read the peers' tiles
  if (tr0) TTRACE(25);
  // write F and its ingest-type copy (coalesced along j); ||x^||^2 of my columns
  int shift = 0;
  if (a.is_half && xx > 0.0) {
    const float nrm = sqrtf((float)xx);
    shift = nrm > 16384.f ? (int)ceilf(log2f(nrm / 16384.f)) : 0;
  }
  if (ct == 0 && crank == 0 && tid == 0) *a.ch_shift = shift;
  const float scale = ldexpf(1.0f, -shift);
  float ph = 0.f, pl = 0.f;     // float-float partial of ||x^||^2
  env_columns_out<TX, NP>(sF, LDF, sN, nmy, r, a.J, j0 + jb, a.Cst, (TX*)a.Chst, scale, ph, pl);
  const float2 cc_cta = ff_block_sum(ph, pl, redf);
  if (tr0) TTRACE(26);
  // one partial per CTA; the last CTA of the grid sums them in a fixed order
  const int ncta = (int)(gridDim.x * gridDim.y);
  if (tid == 0) {
    a.cc_part[(size_t)ct * nq + crank] = cc_cta;
    __threadfence();
    const unsigned done = atomicAdd(a.counter, 1u);
    last_flag = (done == (unsigned)ncta - 1u);
  }
  __syncthreads();
  if (!last_flag) return;
  TTRACE(27);
  __threadfence();
  float sh = 0.f, sl = 0.f;
  for (int b0 = tid; b0 < ncta; b0 += 4 * K2_THREADS) {
    float2 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      v[q] = (b0 + q * K2_THREADS < ncta) ? __ldcg(a.cc_part + b0 + q * K2_THREADS) : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) ff_add(sh, sl, v[q].x, v[q].y);
  }
  const float2 ccf = ff_block_sum(sh, sl, redf);
  if (tid == 0) {
    const double cc = (double)ccf.x + (double)ccf.y;
    *a.counter = 0u;
    Ctl* c = a.ctl;
    if (!isfinite(cc)) c->latched = 4;
    const double ccv = isfinite(cc) ? cc : 0.0;
    const double ee = xx - ccv > 0.0 ? xx - ccv : 0.0;
    c->cc = ccv;
    c->ee = ee;
    c->sum_xx = sum_xx + xx;
    c->sum_ee = sum_ee + ee;
    c->t = tcount + 1;
  }
  TTRACE(28);
}

// ================================================================ K2 (single-CTA tiles)
// F^T = X_(1)^T Q1 for a 64-column tile of X over all I_1 rows in one CTA (no cluster, no
// split over rows): the tile's X block (I_1 x 128 B, 128B-swizzled TMA boxes of RB rows) is
// requested before the dependency wait and arrives while the factor kernel runs; Q1 (ingest
// type, I_1 x NP) comes from L2 into an XOR-swizzled layout (conflict-free ldmatrix).  The 8
// warps split the rows and their partial tiles are summed in shared memory in warp order.
// Used when the X block and Q1 fit in one CTA's shared memory.
constexpr int K2S_BN = 64;            // slice columns j per CTA

// byte offset of 16-byte chunk c of row `row` of the NP-wide Q1 tile
template <int NP>
__device__ __forceinline__ uint32_t qswz(int row, int c) {
  constexpr int CPR = NP / 8;         // chunks per row
  constexpr int G = 8 / CPR;          // rows per 128 bytes
  return (uint32_t)(row * NP * 2 + ((c ^ ((row / G) & (CPR - 1))) << 4));
}

// rows of X per TMA box and boxes per tile (rows padded to a multiple of 16 for the k-steps)
__host__ __device__ constexpr int k2s_box_rows(int M) {
  return (((M + ((M + 255) / 256) - 1) / ((M + 255) / 256)) + 15) / 16 * 16;
}
__host__ __device__ constexpr int k2s_boxes(int M) { return (M + 255) / 256; }
template <int NP>
__host__ __device__ constexpr size_t k2s_smem_bytes(int M, int r) {
  return 1024 + (size_t)k2s_boxes(M) * k2s_box_rows(M) * 128 + (size_t)((M + 15) / 16 * 16) * NP * 2 +
         (size_t)2 * NP * NP * 4 + 64 + 0 * r;
}
// the warp partials (8 x 64 x (NP+8)) and my columns of F (64 x (r+1)) reuse the X block
template <int NP>
__host__ __device__ constexpr bool k2s_fits(int M, int r) {
  return NP != 48 && k2s_smem_bytes<NP>(M, r) <= 225 * 1024 &&
         (size_t)8 * K2S_BN * (NP + 8) * 4 + (size_t)K2S_BN * (r + 1) * 4 <=
             (size_t)k2s_boxes(M) * k2s_box_rows(M) * 128;
}

template <typename TX, int NP>
__global__ void __launch_bounds__(K2_THREADS, 1)
    k_fast_env1(const __grid_constant__ CUtensorMap tmX, EnvArgs a0) {
  const int zs = a0.zmap[blockIdx.z];     // grid plane z serves stream zs of the batch
  const EnvArgs a = env_args_for_stream<TX, NP>(a0, zs, gridDim.x * gridDim.y);
  constexpr int NT = NP / 8;          // n8-tiles of the output per warp
  constexpr int MT = K2S_BN / 16;     // m16-tiles (64 columns)
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int M = a.M, r = a.r, rr = r * r;
  const int RB = k2s_box_rows(M), NBX = k2s_boxes(M);
  const int Mp = (M + 15) / 16 * 16;
  const uint32_t xs = smem_u32(smem);                                  // X block, row i at i*128
  unsigned char* qbase = smem + (size_t)NBX * RB * 128;               // Q1, swizzled
  const uint32_t qs = smem_u32(qbase);
  float* sN = reinterpret_cast<float*>(qbase + (size_t)Mp * NP * 2);  // Nx, NP x NP, zero past r
  float* sW = sN + NP * NP;                                            // D2 = W2 - I (NP x NP)
  constexpr int LDR = NP + 8;                                          // float2 stores: 2 wavefronts
  float* RED = reinterpret_cast<float*>(smem);                        // [8][64][NP+8] after the product
  const int LDF = r + 1;
  float* sF = RED + 8 * K2S_BN * LDR;                                  // [64][r+1]
  __shared__ __align__(8) uint64_t xbar;
  __shared__ float redf[64];
  __shared__ int last_flag;
  __shared__ int timeout_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ct = blockIdx.x;
  const long long j0 = (long long)ct * K2S_BN;
  const int xcols = (a.J - j0 < K2S_BN) ? (int)(a.J - j0) : K2S_BN;
  const bool tr0 = (blockIdx.x == 0);
  const bool W2_WRITER = (blockIdx.x == 0);   // one CTA writes the state's W2

  // 1. this CTA's X block through the TMA engine (independent of the previous kernels)
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
    mbar_init(smem_u32(&xbar), 1);
    mbar_fence_init();
    timeout_flag = 0;
    const uint32_t bar = smem_u32(&xbar);
    mbar_arrive_expect_tx(bar, (uint32_t)NBX * RB * 128);
    for (int b = 0; b < NBX; ++b) tma_load_3d(xs + (uint32_t)b * RB * 128, &tmX, (int)j0, b * RB, zs, bar);
  }
  if (tr0) TTRACE(20);
  // 2. wait for the factor kernel (Q1, Nx, ctl)
  pdl_wait();
  pdl_trigger();
  if (tr0) TTRACE(21);
  const double xx = a.ctl->xx;     // ||x||^2 of this slice (factor kernel)
  double sum_xx = 0.0, sum_ee = 0.0;  // running totals (read early; used by the last CTA)
  long long tcount = 0;
  if (tid == 0) {
    sum_xx = a.ctl->sum_xx;
    sum_ee = a.ctl->sum_ee;
    tcount = a.ctl->t;
  }
  if (a.ctl->skip) {
    // non-finite slice: the new state is the old one
    const long long nthr = (long long)gridDim.x * K2_THREADS;
    const long long me = (long long)blockIdx.x * K2_THREADS + tid;
    for (long long e = me; e < (long long)M * r; e += nthr) a.Qst[e] = a.Qold[e];
    for (long long e = me; e < (long long)r * a.J; e += nthr) {
      a.Cst[e] = a.Cold[e];
      ((TX*)a.Chst)[e] = ((const TX*)a.Chold)[e];
    }
    for (long long e = me; e < rr; e += nthr) a.W2st[e] = a.W2old[e];
    if (me == 0) *a.ch_shift = *a.ch_shift_old;
    if (!mbar_wait(smem_u32(&xbar), 0) && tid == 0) a.ctl->latched = 5;
    return;
  }
  // 3. Q1 (all rows, swizzled; rows past I_1 zero) and Nx
  {
    const TX* Qh = (const TX*)a.Qh;
    constexpr int CPR = NP / 8;
    for (int c = tid; c < Mp * CPR; c += K2_THREADS) {
      const int row = c / CPR, ch = c % CPR;
      const bool ok = row < M;
      cp_async16(qs + qswz<NP>(row, ch), Qh + (ok ? (long long)row * NP + ch * 8 : 0), ok ? 16u : 0u);
    }
    cp_async_commit();
    env_w2_nx<NP>(a.W2part, r, sW, sN, a.W2st, W2_WRITER, a.w2_parts);
    cp_async_wait<0>();
  }
  if (!mbar_wait(smem_u32(&xbar), 0)) timeout_flag = 1;
  __syncthreads();
  if (tr0) TTRACE(22);
  // 4. F^T (j x a) = X^T Q1: warp w takes the k-steps w, w+8, ... for all 64 columns
  float acc[MT][NT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[m][n][0] = acc[m][n][1] = acc[m][n][2] = acc[m][n][3] = 0.f;
  for (int ks = warp; ks < Mp / 16; ks += K2_THREADS / 32) {
    const int k0 = ks * 16;
    uint32_t bq[NT][2];
#pragma unroll
    for (int p = 0; p < NT / 2; ++p) {
      const int row = k0 + (lane & 7) + (((lane >> 3) & 1) << 3);
      ldsm_x4_t(qs + qswz<NP>(row, 2 * p + (lane >> 4)), bq[2 * p][0], bq[2 * p][1], bq[2 * p + 1][0],
                bq[2 * p + 1][1]);
    }
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      uint32_t af[4];
      const int row = k0 + (lane & 7) + ((lane >> 4) << 3);
      ldsm_x4_t(xs + swz(row, 2 * m + ((lane >> 3) & 1)), af[0], af[1], af[2], af[3]);
#pragma unroll
      for (int n = 0; n < NT; ++n) mma16816<TX>(acc[m][n], af, bq[n][0], bq[n][1]);
    }
  }
  __syncthreads();          // every warp is done with the X block before it becomes RED
  {
    const int g = lane >> 2, t4 = lane & 3;
    float* R = RED + warp * K2S_BN * LDR;
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const int row = m * 16 + g, col = n * 8 + 2 * t4;
        *reinterpret_cast<float2*>(R + row * LDR + col) = make_float2(acc[m][n][0], acc[m][n][1]);
        *reinterpret_cast<float2*>(R + (row + 8) * LDR + col) = make_float2(acc[m][n][2], acc[m][n][3]);
      }
  }
  if (tid == 0 && timeout_flag) a.ctl->latched = 5;
  __syncthreads();
  for (int o = tid; o < K2S_BN * NP; o += K2_THREADS) {
    const int jl = o / NP, c = o % NP;
    float v[K2_THREADS / 32];
#pragma unroll
    for (int w = 0; w < K2_THREADS / 32; ++w) v[w] = RED[w * K2S_BN * LDR + jl * LDR + c];
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < K2_THREADS / 32; ++w) sum += v[w];
    if (c < r) sF[jl * LDF + c] = sum;
  }
  __syncthreads();
  if (tr0) TTRACE(23);
  // 5. write F and its ingest-type copy (coalesced along j); ||x^||^2 of my columns
  int shift = 0;
  if (a.is_half && xx > 0.0) {
    const float nrm = sqrtf((float)xx);
    shift = nrm > 16384.f ? (int)ceilf(log2f(nrm / 16384.f)) : 0;
  }
  if (ct == 0 && tid == 0) *a.ch_shift = shift;
  const float scale = ldexpf(1.0f, -shift);
  float ph = 0.f, pl = 0.f;     // float-float partial of ||x^||^2
  env_columns_out<TX, NP>(sF, LDF, sN, xcols, r, a.J, j0, a.Cst, (TX*)a.Chst, scale, ph, pl);
  const float2 cc_cta = ff_block_sum(ph, pl, redf);
  if (tr0) TTRACE(24);
  // one partial per CTA; the last CTA of the grid sums them in a fixed order
  const int ncta = (int)gridDim.x;
  if (tid == 0) {
    a.cc_part[ct] = cc_cta;
    __threadfence();
    const unsigned done = atomicAdd(a.counter, 1u);
    last_flag = (done == (unsigned)ncta - 1u);
  }
  __syncthreads();
  if (!last_flag) return;
  TTRACE(27);
  __threadfence();
  float sh = 0.f, sl = 0.f;
  for (int b0 = tid; b0 < ncta; b0 += 4 * K2_THREADS) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      v[u] = (b0 + u * K2_THREADS < ncta) ? __ldcg(a.cc_part + b0 + u * K2_THREADS) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) ff_add(sh, sl, v[u].x, v[u].y);
  }
  const float2 ccf = ff_block_sum(sh, sl, redf);
  if (tid == 0) {
    const double cc = (double)ccf.x + (double)ccf.y;
    *a.counter = 0u;
    Ctl* c = a.ctl;
    if (!isfinite(cc)) c->latched = 4;
    const double ccv = isfinite(cc) ? cc : 0.0;
    const double ee = xx - ccv > 0.0 ? xx - ccv : 0.0;
    c->cc = ccv;
    c->ee = ee;
    c->sum_xx = sum_xx + xx;
    c->sum_ee = sum_ee + ee;
    c->t = tcount + 1;
  }
  TTRACE(28);
}

// ================================================================ K2 (streamed row stages)
// F^T = X_(1)^T Q1 for a 128-column tile of X, the I_1 rows streamed through a pipeline of
// 64-row stages (two 64 x 64 TMA boxes of X: 256 contiguous bytes of every row, the solve
// kernel's map; and the stage's Q1 rows by cp.async into an XOR-swizzled layout).  Warp 8
// issues the copies (the first X stages before the dependency wait) and both kinds complete
// on the stage's `full` barrier; warps 0-7 each own 16 output columns for all NP, accumulate
// over the rows in row order (no cross-warp reduction) and release stages through `empty`.
// Small shared memory (two CTAs per SM) and long row loops: the kernel for batches.
constexpr int K2P_BM = 64;            // rows of X per stage
constexpr int K2P_BN = 128;           // slice columns j per CTA
constexpr int K2P_CWARPS = 8;
constexpr int K2P_THREADS = (K2P_CWARPS + 1) * 32;
constexpr int K2P_MAXST = 4;
template <int NP>
__host__ __device__ constexpr int k2p_stages() { return NP <= 32 ? 4 : 3; }
// bytes per Q1 row in a stage: NP 16-bit values, rows of 48 padded to 64 (128 B)
template <int NP>
__host__ __device__ constexpr int k2p_qrow() { return NP == 48 ? 128 : NP * 2; }
// byte offset of 16-byte chunk c of row `row` in a Q1 stage (conflict-free ldmatrix)
template <int NP>
__device__ __forceinline__ uint32_t k2p_qaddr(int row, int c) {
  if constexpr (NP == 48) return swz(row, c);
  else return qswz<NP>(row, c);
}
template <int NP>
__host__ __device__ constexpr size_t k2p_smem_bytes() {
  // X stages (64 x 256 B: two 128B-swizzled boxes) | Q1 stages (64 rows) | Nx, D2 (NP x NP
  // each); my columns of F (128 x (r+1) floats) reuse the X stages after the loop
  return 1024 + (size_t)k2p_stages<NP>() * (K2P_BM * 256 + K2P_BM * k2p_qrow<NP>()) + (size_t)2 * NP * NP * 4;
}
__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(bar) : "memory");
}

template <typename TX, int NP>
__global__ void __launch_bounds__(K2P_THREADS, 2)
    k_fast_env_stream(const __grid_constant__ CUtensorMap tmX, EnvArgs a0) {
  const int zs = a0.zmap[blockIdx.z];     // grid plane z serves stream zs of the batch
  const EnvArgs a = env_args_for_stream<TX, NP>(a0, zs, gridDim.x * gridDim.y);
  constexpr int ST = k2p_stages<NP>();
  static_assert(ST <= K2P_MAXST, "stages");
  constexpr int NT8 = NP / 8;         // n8-tiles of the output (every warp covers all NP)
  constexpr int CPR = NP / 8;         // 16-byte chunks per Q1 row
  constexpr uint32_t XBOX = K2P_BM * 128, XB = 2 * XBOX, QB = K2P_BM * k2p_qrow<NP>();
  static_assert(NT8 % 2 == 0, "n8-tiles come in pairs");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int M = a.M, r = a.r, rr = r * r;
  const uint32_t xs = smem_u32(smem);                          // X stage s at xs + s*XB
  const uint32_t qs = xs + ST * XB;                            // Q1 stage s at qs + s*QB
  float* sN = reinterpret_cast<float*>(smem + ST * (XB + QB)); // Nx, NP x NP, zero past r
  float* sW = sN + NP * NP;                                    // D2 = W2 - I (NP x NP)
  const int LDF = r + 1;
  float* sF = reinterpret_cast<float*>(smem);                  // [128][r+1] after the loop
  __shared__ __align__(8) uint64_t full[K2P_MAXST];
  __shared__ __align__(8) uint64_t empty[K2P_MAXST];
  __shared__ float redf[64];
  __shared__ int last_flag;
  __shared__ int timeout_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool producer = (warp == K2P_CWARPS);
  const int ct = blockIdx.x;
  const long long j0 = (long long)ct * K2P_BN;
  const int xcols = (a.J - j0 < K2P_BN) ? (int)(a.J - j0) : K2P_BN;
  const int nt = (M + K2P_BM - 1) / K2P_BM;
  const bool tr0 = (blockIdx.x == 0);
  const bool W2_WRITER = (blockIdx.x == 0);   // one CTA writes the state's W2
  auto load_x = [&](int t, int st) {          // producer lane 0
    const uint32_t bar = smem_u32(&full[st]);
    mbar_arrive_expect_tx(bar, XB);
    tma_load_3d(xs + st * XB, &tmX, (int)j0, t * K2P_BM, zs, bar);
    tma_load_3d(xs + st * XB + XBOX, &tmX, (int)j0 + 64, t * K2P_BM, zs, bar);
  };
  const TX* Qh = (const TX*)a.Qh;
  auto load_q = [&](int t, int st) {          // the 32 producer lanes
    const uint32_t dst = qs + (uint32_t)st * QB;
    for (int c = lane; c < K2P_BM * CPR; c += 32) {
      const int lr = c / CPR, ch = c % CPR;
      const int row = t * K2P_BM + lr;
      const bool ok = row < M;
      cp_async16(dst + k2p_qaddr<NP>(lr, ch), Qh + (ok ? (long long)row * NP + ch * 8 : 0), ok ? 16u : 0u);
    }
    cp_async_mbar_arrive_noinc(smem_u32(&full[st]));
  };

  // 1. barriers; the first X stages (independent of the previous kernels)
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
    for (int st = 0; st < ST; ++st) {
      mbar_init(smem_u32(&full[st]), 1 + 32);      // X expect_tx arrival + 32 lanes' Q1 copies
      mbar_init(smem_u32(&empty[st]), K2P_CWARPS);
    }
    mbar_fence_init();
    timeout_flag = 0;
  }
  __syncthreads();
  if (producer && lane == 0)
    for (int t = 0; t < ST && t < nt; ++t) load_x(t, t);
  if (tr0) TTRACE(20);
  // 2. wait for the factor kernel (Q1, W2 partials, ctl)
  pdl_wait();
  pdl_trigger();
  if (tr0) TTRACE(21);
  const double xx = a.ctl->xx;     // ||x||^2 of this slice (factor kernel)
  double sum_xx = 0.0, sum_ee = 0.0;
  long long tcount = 0;
  if (tid == 0) {
    sum_xx = a.ctl->sum_xx;
    sum_ee = a.ctl->sum_ee;
    tcount = a.ctl->t;
  }
  if (a.ctl->skip) {
    // non-finite slice: the new state is the old one
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long me = (long long)blockIdx.x * blockDim.x + tid;
    for (long long e = me; e < (long long)M * r; e += nthr) a.Qst[e] = a.Qold[e];
    for (long long e = me; e < (long long)r * a.J; e += nthr) {
      a.Cst[e] = a.Cold[e];
      ((TX*)a.Chst)[e] = ((const TX*)a.Chold)[e];
    }
    for (long long e = me; e < rr; e += nthr) a.W2st[e] = a.W2old[e];
    if (me == 0) *a.ch_shift = *a.ch_shift_old;
    if (producer) {
      // the X copies in flight land before the CTA exits: the lanes stand in for the Q1
      // arrivals that never come, then lane 0 waits (bounded) for each stage's phase
      for (int st = 0; st < ST && st < nt; ++st) mbar_arrive(smem_u32(&full[st]));
      bool ok = true;
      if (lane == 0)
        for (int st = 0; st < ST && st < nt; ++st) ok = mbar_wait(smem_u32(&full[st]), 0) && ok;
      if (!ok) a.ctl->latched = 5;
    }
    return;
  }
  // Q1 of the first stages; W2 and Nx (a block-wide step) while the copies fly; then the
  // producer refills stages as they are released and the consumers run the row loop
  if (producer)
    for (int t = 0; t < ST && t < nt; ++t) load_q(t, t);
  env_w2_nx<NP>(a.W2part, r, sW, sN, a.W2st, W2_WRITER, a.w2_parts);
  if (tr0) TTRACE(22);
  if (producer) {
    int issued = nt < ST ? nt : ST;
    for (int t = ST; t < nt; ++t) {
      const int st = t % ST;
      bool ok = true;
      if (lane == 0) ok = mbar_wait(smem_u32(&empty[st]), (uint32_t)(((t / ST) - 1) & 1)) && !timeout_flag;
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) timeout_flag = 1;
        break;
      }
      load_q(t, st);
      if (lane == 0) load_x(t, st);
      issued = t + 1;
    }
    cp_async_wait<0>();
    if (lane == 0 && timeout_flag) {
      // a wait gave up: wait (bounded) for the copies still in flight before the buffers are
      // reused; the step is marked failed (ETIMEOUT)
      for (int t = issued - ST > 0 ? issued - ST : 0; t < issued; ++t)
        mbar_wait(smem_u32(&full[t % ST]), (uint32_t)((t / ST) & 1));
    }
  }
  // 3. F^T (128 x NP) = X^T Q1 over the row stages: warp w owns columns 16 w .. 16 w + 15
  float acc[NT8][4];
#pragma unroll
  for (int n = 0; n < NT8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  if (!producer) {
    const uint32_t xoff = (uint32_t)(warp >> 2) * XBOX;   // box of my columns
    const int wm = warp & 3;                              // m16-tile within the box
    for (int t = 0; t < nt; ++t) {
      const int st = t % ST;
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((t / ST) & 1)) || timeout_flag) {
        timeout_flag = 1;
        break;
      }
      const uint32_t xst = xs + st * XB + xoff, qst = qs + st * QB;
#pragma unroll
      for (int k0 = 0; k0 < K2P_BM; k0 += 16) {
        uint32_t af[4];
        {
          const int row = k0 + (lane & 7) + ((lane >> 4) << 3);
          ldsm_x4_t(xst + swz(row, 2 * wm + ((lane >> 3) & 1)), af[0], af[1], af[2], af[3]);
        }
        const int qrow = k0 + (lane & 7) + (((lane >> 3) & 1) << 3);
#pragma unroll
        for (int p = 0; p < NT8 / 2; ++p) {
          uint32_t b0, b1, b2, b3;
          ldsm_x4_t(qst + k2p_qaddr<NP>(qrow, 2 * p + (lane >> 4)), b0, b1, b2, b3);
          mma16816<TX>(acc[2 * p], af, b0, b1);
          mma16816<TX>(acc[2 * p + 1], af, b2, b3);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[st]));   // this warp is done with stage st
    }
  }
  __syncthreads();          // every stage consumed (or the copies in flight drained)
  if (!producer) {
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int n = 0; n < NT8; ++n) {
      const int c = n * 8 + 2 * t4, jl = warp * 16 + g;
      if (c < r) {
        sF[jl * LDF + c] = acc[n][0];
        sF[(jl + 8) * LDF + c] = acc[n][2];
      }
      if (c + 1 < r) {
        sF[jl * LDF + c + 1] = acc[n][1];
        sF[(jl + 8) * LDF + c + 1] = acc[n][3];
      }
    }
  }
  if (tid == 0 && timeout_flag) a.ctl->latched = 5;
  __syncthreads();
  if (tr0) TTRACE(23);
  // 4. write F and its ingest-type copy (coalesced along j); ||x^||^2 of my columns
  int shift = 0;
  if (a.is_half && xx > 0.0) {
    const float nrm = sqrtf((float)xx);
    shift = nrm > 16384.f ? (int)ceilf(log2f(nrm / 16384.f)) : 0;
  }
  if (ct == 0 && tid == 0) *a.ch_shift = shift;
  const float scale = ldexpf(1.0f, -shift);
  float ph = 0.f, pl = 0.f;     // float-float partial of ||x^||^2
  if (!producer) env_columns_out<TX, NP>(sF, LDF, sN, xcols, r, a.J, j0, a.Cst, (TX*)a.Chst, scale, ph, pl);
  const float2 cc_cta = ff_block_sum(ph, pl, redf);
  if (tr0) TTRACE(24);
  // one partial per CTA; the last CTA of the stream's grid sums them in a fixed order
  const int ncta = (int)gridDim.x;
  if (tid == 0) {
    a.cc_part[ct] = cc_cta;
    __threadfence();
    const unsigned done = atomicAdd(a.counter, 1u);
    last_flag = (done == (unsigned)ncta - 1u);
  }
  __syncthreads();
  if (!last_flag) return;
  __threadfence();
  float sh = 0.f, sl = 0.f;
  const int nthr = (int)blockDim.x;
  for (int b0 = tid; b0 < ncta; b0 += 4 * nthr) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      v[u] = (b0 + u * nthr < ncta) ? __ldcg(a.cc_part + b0 + u * nthr) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) ff_add(sh, sl, v[u].x, v[u].y);
  }
  const float2 ccf = ff_block_sum(sh, sl, redf);
  if (tid == 0) {
    const double cc = (double)ccf.x + (double)ccf.y;
    *a.counter = 0u;
    Ctl* c = a.ctl;
    if (!isfinite(cc)) c->latched = 4;
    const double ccv = isfinite(cc) ? cc : 0.0;
    const double ee = xx - ccv > 0.0 ? xx - ccv : 0.0;
    c->cc = ccv;
    c->ee = ee;
    c->sum_xx = sum_xx + xx;
    c->sum_ee = sum_ee + ee;
    c->t = tcount + 1;
  }
  TTRACE(28);
}

// ================================================================ K2 on tcgen05 (batches)
// F^T = X_(1)^T Q1 for a 128-column tile of X on the 5th-gen tensor cores: the I_1 rows stream
// through 64-row stages (two 64 x 64 X boxes and the stage's Q1 rows, both by TMA), warp 0
// issues the copies, warp 1's elected lane issues tcgen05.mma (M = 128 columns j, N = NP,
// K = 16 rows per instruction; A = X^T and B = Q1 both MN-major in the TMA's swizzled
// layouts; FP32 accumulator in TMEM) and frees each stage with tcgen05.commit.  Warps 2-5 read
// the accumulator (TMEM lane = column j) into shared memory; then all 8 warps form the
// statistics and write the state as in the other environment kernels.  Q1 of ranks padded
// to 16, 32, 64 (swizzle 32, 64, 128 B).
constexpr int K2T_BN = 128;
constexpr int K2T_THREADS = 256;
constexpr int K2T_MAXST = 4;
template <int NP>
__host__ __device__ constexpr int k2t_stages() { return NP <= 32 ? 4 : 3; }
template <int NP>
__host__ __device__ constexpr size_t k2t_smem_bytes() {
  // X stages (64 x 256 B) | Q1 stages (64 x NP) | Nx, D2 (NP x NP each); F (128 x (r+1)
  // floats) reuses the X stages after the loop
  return 1024 + (size_t)k2t_stages<NP>() * (K2P_BM * 256 + K2P_BM * NP * 2) + (size_t)2 * NP * NP * 4;
}
// MN-major shared-memory descriptor: atoms of (row pitch) bytes x 8 rows along K, `lbo` bytes
// between atoms along MN, `sbo` bytes between 8-row groups along K, swizzle code `layout`
__device__ __forceinline__ uint64_t umma_desc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)layout << 61;
  return d;
}
template <int NP>
__host__ __device__ constexpr uint32_t k2t_q_layout() { return NP == 16 ? 6u : (NP == 32 ? 4u : 2u); }

template <typename TX, int NP>
__global__ void __launch_bounds__(K2T_THREADS, 2)
    k_fast_env_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ, EnvArgs a0) {
  const int zs = a0.zmap[blockIdx.z];     // grid plane z serves stream zs of the batch
  const EnvArgs a = env_args_for_stream<TX, NP>(a0, zs, gridDim.x * gridDim.y);
  static_assert(NP == 16 || NP == 32 || NP == 64, "Q1 swizzle atoms for ranks padded to 16, 32, 64");
  constexpr int ST = k2t_stages<NP>();
  static_assert(ST <= K2T_MAXST, "stages");
  constexpr uint32_t XBOX = K2P_BM * 128, XB = 2 * XBOX, QB = K2P_BM * NP * 2;
  constexpr uint32_t QPITCH = NP * 2;                 // bytes per Q1 row
  constexpr uint32_t TCOLS = NP <= 32 ? 32 : 64;
  // M = 128 columns, N = NP, A and B MN-major (transpose bits 15 and 16)
  constexpr uint32_t IDESC = umma_idesc_f16<TX>(K2T_BN, NP) | (1u << 15) | (1u << 16);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int M = a.M, r = a.r, rr = r * r;
  const uint32_t xs = smem_u32(smem);                          // X stage s at xs + s*XB
  const uint32_t qs = xs + ST * XB;                            // Q1 stage s at qs + s*QB
  float* sN = reinterpret_cast<float*>(smem + ST * (XB + QB)); // Nx, NP x NP, zero past r
  float* sW = sN + NP * NP;                                    // D2 = W2 - I (NP x NP)
  const int LDF = r + 1;
  float* sF = reinterpret_cast<float*>(smem);                  // [128][r+1] after the loop
  __shared__ __align__(8) uint64_t full[K2T_MAXST];
  __shared__ __align__(8) uint64_t empty[K2T_MAXST];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_holder;
  __shared__ float redf[64];
  __shared__ int last_flag;
  __shared__ int timeout_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ct = blockIdx.x;
  const long long j0 = (long long)ct * K2T_BN;
  const int xcols = (a.J - j0 < K2T_BN) ? (int)(a.J - j0) : K2T_BN;
  const int nt = (M + K2P_BM - 1) / K2P_BM;
  const bool tr0 = (blockIdx.x == 0);
  const bool W2_WRITER = (blockIdx.x == 0);
  auto load_x = [&](int t, int st) {
    const uint32_t bar = smem_u32(&full[st]);
    mbar_arrive_expect_tx(bar, XB);
    tma_load_3d(xs + st * XB, &tmX, (int)j0, t * K2P_BM, zs, bar);
    tma_load_3d(xs + st * XB + XBOX, &tmX, (int)j0 + 64, t * K2P_BM, zs, bar);
  };
  auto load_q = [&](int t, int st) {
    const uint32_t bar = smem_u32(&full[st]);
    mbar_arrive_expect_tx(bar, QB);
    tma_load_3d(qs + st * QB, &tmQ, 0, t * K2P_BM, zs, bar);
  };

  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
    for (int st = 0; st < ST; ++st) {
      mbar_init(smem_u32(&full[st]), 2);           // X arrival + Q1 arrival (expect_tx)
      mbar_init(smem_u32(&empty[st]), 1);          // the MMA commit
    }
    mbar_init(smem_u32(&done), 1);
    mbar_fence_init();
    timeout_flag = 0;
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_holder), TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  if (warp == 0 && lane == 0)
    for (int t = 0; t < ST && t < nt; ++t) load_x(t, t);
  if (tr0) TTRACE(20);
  pdl_wait();
  pdl_trigger();
  if (tr0) TTRACE(21);
  const double xx = a.ctl->xx;
  double sum_xx = 0.0, sum_ee = 0.0;
  long long tcount = 0;
  if (tid == 0) {
    sum_xx = a.ctl->sum_xx;
    sum_ee = a.ctl->sum_ee;
    tcount = a.ctl->t;
  }
  if (a.ctl->skip) {
    // non-finite slice: the new state is the old one
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long me = (long long)blockIdx.x * blockDim.x + tid;
    for (long long e = me; e < (long long)M * r; e += nthr) a.Qst[e] = a.Qold[e];
    for (long long e = me; e < (long long)r * a.J; e += nthr) {
      a.Cst[e] = a.Cold[e];
      ((TX*)a.Chst)[e] = ((const TX*)a.Chold)[e];
    }
    for (long long e = me; e < rr; e += nthr) a.W2st[e] = a.W2old[e];
    if (me == 0) *a.ch_shift = *a.ch_shift_old;
    if (warp == 0 && lane == 0) {
      // the X copies in flight land before the CTA exits (the Q1 arrival stands in)
      bool ok = true;
      for (int st = 0; st < ST && st < nt; ++st) {
        mbar_arrive_expect_tx(smem_u32(&full[st]), 0);
        ok = mbar_wait(smem_u32(&full[st]), 0) && ok;
      }
      if (!ok) a.ctl->latched = 5;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, TCOLS);
    return;
  }
  if (warp == 0 && lane == 0)
    for (int t = 0; t < ST && t < nt; ++t) load_q(t, t);
  env_w2_nx<NP>(a.W2part, r, sW, sN, a.W2st, W2_WRITER, a.w2_parts);   // block-wide, while the copies fly
  if (tr0) TTRACE(22);
  if (warp == 0) {
    if (lane == 0) {
      int issued = nt < ST ? nt : ST;
      for (int t = ST; t < nt; ++t) {
        const int st = t % ST;
        if (!mbar_wait(smem_u32(&empty[st]), (uint32_t)(((t / ST) - 1) & 1)) || timeout_flag) {
          timeout_flag = 1;
          break;
        }
        load_x(t, st);
        load_q(t, st);
        issued = t + 1;
      }
      if (timeout_flag) {
        for (int t = issued - ST > 0 ? issued - ST : 0; t < issued; ++t)
          mbar_wait(smem_u32(&full[t % ST]), (uint32_t)((t / ST) & 1));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int t = 0; t < nt; ++t) {
        const int st = t % ST;
        if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((t / ST) & 1)) || timeout_flag) {
          timeout_flag = 1;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < K2P_BM / 16; ++kk) {
          // A = X^T: 64-column atoms (one per box, 8192 B apart), 8-row groups 1024 B apart
          const uint64_t ad = umma_desc_mn(xs + st * XB + kk * 2048, XBOX, 1024, 2u);
          // B = Q1: one atom of NP columns, 8-row groups 8 x QPITCH apart
          const uint64_t bd = umma_desc_mn(qs + st * QB + kk * 16 * QPITCH, 8 * QPITCH, 8 * QPITCH, k2t_q_layout<NP>());
          umma_f16(tmem, ad, bd, IDESC, (t | kk) != 0 ? 1u : 0u);
        }
        umma_commit(smem_u32(&empty[st]));
      }
      umma_commit(smem_u32(&done));
    }
    __syncwarp();
  }
  // the accumulator (lane = column j of the tile) -> sF[j][c]; the X stages are free now
  if (warp >= 2 && warp < 6) {
    const bool ok = mbar_wait(smem_u32(&done), 0);
    if (!ok) timeout_flag = 1;
    tc_fence_after();
    const int q = warp & 3;
    const int jl = q * 32 + lane;
    float v[32];
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 32) {
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < r) sF[jl * LDF + c0 + j] = v[j];
    }
  }
  tc_fence_before();
  if (tid == 0 && timeout_flag) a.ctl->latched = 5;
  __syncthreads();
  if (tr0) TTRACE(23);
  int shift = 0;
  if (a.is_half && xx > 0.0) {
    const float nrm = sqrtf((float)xx);
    shift = nrm > 16384.f ? (int)ceilf(log2f(nrm / 16384.f)) : 0;
  }
  if (ct == 0 && tid == 0) *a.ch_shift = shift;
  const float scale = ldexpf(1.0f, -shift);
  float ph = 0.f, pl = 0.f;
  env_columns_out<TX, NP>(sF, LDF, sN, xcols, r, a.J, j0, a.Cst, (TX*)a.Chst, scale, ph, pl);
  const float2 cc_cta = ff_block_sum(ph, pl, redf);
  if (tr0) TTRACE(24);
  const int ncta = (int)gridDim.x;
  if (tid == 0) {
    a.cc_part[ct] = cc_cta;
    __threadfence();
    const unsigned dn = atomicAdd(a.counter, 1u);
    last_flag = (dn == (unsigned)ncta - 1u);
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, TCOLS);
  if (!last_flag) return;
  __threadfence();
  float sh = 0.f, sl = 0.f;
  for (int b0 = tid; b0 < ncta; b0 += 4 * K2T_THREADS) {
    float2 vv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      vv[u] = (b0 + u * K2T_THREADS < ncta) ? __ldcg(a.cc_part + b0 + u * K2T_THREADS) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) ff_add(sh, sl, vv[u].x, vv[u].y);
  }
  const float2 ccf = ff_block_sum(sh, sl, redf);
  if (tid == 0) {
    const double cc = (double)ccf.x + (double)ccf.y;
    *a.counter = 0u;
    Ctl* c = a.ctl;
    if (!isfinite(cc)) c->latched = 4;
    const double ccv = isfinite(cc) ? cc : 0.0;
    const double ee = xx - ccv > 0.0 ? xx - ccv : 0.0;
    c->cc = ccv;
    c->ee = ee;
    c->sum_xx = sum_xx + xx;
    c->sum_ee = sum_ee + ee;
    c->t = tcount + 1;
  }
  TTRACE(28);
}

// ================================================================ carry (masked steps)
// Streams of a batch that take no step this time keep their state: copy it from the old
// buffers into the new ones (the batch's buffer parity flips for every stream).  Grid plane
// z serves stream zmap[z]; plain coalesced copies, no dependency on the current step.
template <typename TX, int NP>
__global__ void __launch_bounds__(256) k_fast_carry(EnvArgs a0) {
  const int zs = a0.zmap[blockIdx.z];
  const EnvArgs a = env_args_for_stream<TX, NP>(a0, zs, 0);
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const long long me = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long mr = (long long)a.M * a.r, rj = (long long)a.r * a.J, rr = (long long)a.r * a.r;
  for (long long e = me; e < mr; e += nthr) a.Qst[e] = a.Qold[e];
  for (long long e = me; e < rj; e += nthr) {
    a.Cst[e] = a.Cold[e];
    ((TX*)a.Chst)[e] = ((const TX*)a.Chold)[e];
  }
  for (long long e = me; e < rr; e += nthr) a.W2st[e] = a.W2old[e];
  if (me == 0) *a.ch_shift = *a.ch_shift_old;
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
