// ttals.cu - C ABI and per-slice orchestration of the Online TT-ALS update
// (arXiv 2606.31061, Algorithm 1) on one GPU.
//
// Gauge-reduced form of Algorithm 1.  x^_t (and the left-orthogonal cores it is
// built from) depends on the right interfaces B_k only through their row spaces:
// the LQ sweep of Sec. 3.4.1 gives B_k = L_{k+1}^{-1} B^_k with
// B^_k = G_{k+1} x ... x G_{n-1} x g_n, and L_{k+1} is invertible for generic
// data, so QR(E_k B_k^T) and QR(E_k B^_k^T) span the same space and produce the
// same A_{k+1} up to an r x r orthogonal gauge.  The device therefore skips the
// LQ sweep and uses B^_k directly.
//
// Saturation.  Let k* be the first level with r_k >= I_{k+1}...I_{n-1} (it exists:
// r_{n-1} >= 1).  From k* on the clamped ranks span every vector of the trailing
// modes, so x^_t = A_{k*} E_{k*} with E_{k*} = A_{k*}^T X_t.  The device keeps the
// cores G_1..G_{k*-1} and C = E_{k*} (the contraction G_{k*} x ... x g_n) and
// materialises G_{k*}..G_{n-1}, g_n only when they are read (ttals_cores).
// For the 3rd-order and video-shaped streams k* = 2 and one step is
//   Y = X_(1) C^T,  G_1 = orth(Y),  C = G_1^T X_(1).
#include "ttals.h"
#include "ttals_kernels.cuh"
#include "ttals_fast.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

using namespace ttals;

namespace {

thread_local std::string g_last_err;

#define TT_CUDA(x)                                                      \
  do {                                                                  \
    cudaError_t e_ = (x);                                               \
    if (e_ != cudaSuccess) {                                            \
      g_last_err = std::string(#x) + ": " + cudaGetErrorString(e_);    \
      return TTALS_ECUDA;                                               \
    }                                                                   \
  } while (0)

#define TT_TRY(x)                        \
  do {                                   \
    ttals_status s_ = (x);               \
    if (s_ != TTALS_OK) return s_;       \
  } while (0)

constexpr int kSMs = 148;

inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

// split-K choice for the generic GEMM: about target_ctas CTAs (default: two waves on 148
// SMs), at most max_split splits of at least min_kchunk (the split partials are summed
// afterwards, per output element)
struct GemmShape {
  int M, N;
  long long K;
  int nsplit;
  long long kchunk;
  dim3 grid;
};

GemmShape plan_gemm(int M, int N, long long K, bool allow_split, int max_split = 64, int target_ctas = 2 * kSMs,
                    long long min_kchunk = GB_K) {
  GemmShape g;
  g.M = M;
  g.N = N;
  g.K = K;
  const long long tiles = cdiv(M, GB_M) * cdiv(N, GB_N);
  long long ns = allow_split ? std::max<long long>(1, cdiv(target_ctas, tiles)) : 1;
  ns = std::min<long long>(ns, std::max<long long>(1, cdiv(K, min_kchunk)));
  ns = std::min<long long>(ns, max_split);
  long long kc = cdiv(cdiv(K, ns), GB_K) * GB_K;
  if (kc < GB_K) kc = GB_K;
  g.kchunk = kc;
  g.nsplit = (int)std::max<long long>(1, cdiv(K, kc));
  g.grid = dim3((unsigned)cdiv(M, GB_M), (unsigned)cdiv(N, GB_N), (unsigned)g.nsplit);
  return g;
}

// SplitMix64 (Steele, Lea & Flood 2014) and Box-Muller for the default initial cores
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double gauss() {
    const double u1 = uniform(), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 3-D map of nplanes contiguous row-major rows x cols matrices of 16-bit elements (plane z of
// a batch is stream z's matrix), box (64 cols) x box_rows x 1 plane, 128-byte swizzle;
// out-of-range elements (rows >= rows of a plane included) read as zero
bool encode_map_3d(CUtensorMap* map, const void* base, bool bf16, long long nplanes, long long rows, long long cols,
                   int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dim[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)nplanes};
  cuuint64_t stride[2] = {(cuuint64_t)cols * 2, (cuuint64_t)(rows * cols) * 2};
  cuuint32_t box[3] = {64u, (cuuint32_t)box_rows, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                   const_cast<void*>(base), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 3-D map of the rounded basis Q1 (nplanes x rows x np, 16-bit), box np x 64 rows x 1 plane,
// swizzled to the width of a row (np 16, 32, 64: 32-, 64-, 128-byte swizzle): the MN-major
// operand layout of the tensor-core environment kernel
bool encode_map_3d_q(CUtensorMap* map, const void* base, bool bf16, long long nplanes, long long rows, int np) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dim[3] = {(cuuint64_t)np, (cuuint64_t)rows, (cuuint64_t)nplanes};
  cuuint64_t stride[2] = {(cuuint64_t)np * 2, (cuuint64_t)(rows * np) * 2};
  cuuint32_t box[3] = {(cuuint32_t)np, 64u, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUtensorMapSwizzle sw = np == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                         : (np == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                   const_cast<void*>(base), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t dtype_size(ttals_dtype d) {
  switch (d) {
    case TTALS_F64: return 8;
    case TTALS_F32: return 4;
    case TTALS_F16: return 2;
    case TTALS_BF16: return 2;
  }
  return 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// stream object
// ---------------------------------------------------------------------------
struct ttals_stream {
  int m = 0;                          // n - 1 slice modes
  std::vector<long long> dims;        // I_1..I_m
  std::vector<long long> full;        // r_0..r_m (r_0 = 1)
  std::vector<long long> rest;        // rest[k] = I_{k+1}...I_m (rest[m] = 1)
  int kstar = 1;
  ttals_dtype ingest = TTALS_F64;
  int device = 0;
  int qr_passes = 1;
  cudaStream_t last = nullptr;
  bool have_last = false;
  cudaEvent_t ev = nullptr;
  Ctl* ctl = nullptr;                 // control block of the selected stream (ctl_base + sel)
  Ctl* ctl_base = nullptr;            // [nbatch] control blocks
  int nbatch = 1;                     // streams of a batch (ttals_create_batch), else 1
  int sel = 0;                        // stream that the per-stream calls refer to
  unsigned long long active_mask = ~0ull;   // streams of a batch that take the next push
  int cfg_env_kernel = 0;             // ttals_config.env_kernel (0: by shape)
  int cfg_k1_split = 0;               // ttals_config.k1_split (0: by shape and batch)
  int cfg_solve_kernel = 0;           // ttals_config.solve_kernel (0: per launch)
  int cfg_factor_cluster = 0;         // ttals_config.factor_cluster (0: by batch size)
  int cfg_factor = 0;                 // ttals_config.factor (0: FP64 r x r factor, 1: FP32)
  int mode = 0;                       // ttals_config.mode: 0 literal, 1 lsq, 2 noortho
  size_t bytes = 0;
  std::vector<void*> allocs;
  unsigned long long nlaunch = 0;      // kernels launched by this stream (host counter)
  int stall_pushes = 0;                // fault injection: pushes whose local solve issues no copy
  // optional timing of the level-1 kernels: CUDA events recorded on the launch stream
  bool profiling = false;
  // TTALS_NO_PDL=1 in the environment at creation: launch the fused kernels without
  // programmatic dependent launch (each kernel then starts after its predecessor ends);
  // used for profiler captures that replay one kernel of the chain
  bool no_pdl = false;
  std::vector<cudaEvent_t> ev_pool;    // recorded events, in groups of kProfEvents per push
  size_t ev_used = 0;
  static constexpr int kProfEvents = 6; // push begin, solve1 begin, solve1 end, env1 begin, env1 end, push end

  // host ingest of a batch (ttals_batch_ingest_init / ttals_batch_push_host): the batch owns
  // double-buffered input blocks, 8-bit staging, a copy and a compute stream and a ring of
  // completion events, so that one call per step moves the frames and steps the batch
  struct HostIngest {
    bool on = false;
    bool u8 = false;
    void* block[2] = {};              // [nbatch][slice] in the ingest type
    void* stage[2] = {};              // [nbatch][slice] bytes (8-bit wire)
    cudaStream_t copy = nullptr, comp = nullptr;
    cudaEvent_t copied[2] = {}, consumed[2] = {};
    std::vector<cudaEvent_t> done;    // ring of completion events, one per ticket
    uint64_t ticket = 0;
    int flip = 0;
  } hi;
  static constexpr int kTicketRing = 256;

  virtual ~ttals_stream() {
    if (have_last) cudaStreamSynchronize(last);
    if (hi.copy) cudaStreamSynchronize(hi.copy);
    if (hi.comp) cudaStreamSynchronize(hi.comp);
    for (void* p : allocs) cudaFree(p);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    if (ev) cudaEventDestroy(ev);
    for (int i = 0; i < 2; ++i) {
      if (hi.copied[i]) cudaEventDestroy(hi.copied[i]);
      if (hi.consumed[i]) cudaEventDestroy(hi.consumed[i]);
    }
    for (cudaEvent_t e : hi.done) cudaEventDestroy(e);
    if (hi.copy) cudaStreamDestroy(hi.copy);
    if (hi.comp) cudaStreamDestroy(hi.comp);
  }
  // event slot `i` of the current push (profiling only)
  ttals_status mark(int i, cudaStream_t s) {
    if (!profiling) return TTALS_OK;
    const size_t idx = ev_used + (size_t)i;
    while (ev_pool.size() <= idx) {
      cudaEvent_t e;
      TT_CUDA(cudaEventCreate(&e));
      ev_pool.push_back(e);
    }
    TT_CUDA(cudaEventRecord(ev_pool[idx], s));
    return TTALS_OK;
  }
  virtual ttals_status push(const void* x, cudaStream_t s) = 0;
  virtual ttals_status reconstruct(void* out, ttals_dtype dt, cudaStream_t s) = 0;
  virtual ttals_status set_cores(const double* const* cores, const double* g, long long t) = 0;
  virtual ttals_status get_core(int k, double* host, size_t n) = 0;
  virtual ttals_status allocate() = 0;
  // batches: only the fused path steps several streams per launch
  virtual bool batch_capable() const { return false; }
  virtual ttals_status select_slot(int idx) { return idx == 0 ? TTALS_OK : TTALS_EINVAL; }
  // encode (and cache) the fused path's TMA maps of a slice buffer ahead of its first push
  virtual ttals_status warm_slice(const void* x) { (void)x; return TTALS_OK; }

  long long slice_elems() const { return rest[0]; }
  long long core_elems(int k) const {   // k = 1..m
    return full[k - 1] * dims[k - 1] * full[k];
  }

  template <typename T>
  ttals_status dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
      g_last_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? TTALS_ENOMEM : TTALS_ECUDA;
    }
    allocs.push_back((void*)*p);
    bytes += n * sizeof(T);
    return TTALS_OK;
  }

  ttals_status order_after_last(cudaStream_t s) {
    if (have_last && s != last) {
      TT_CUDA(cudaEventRecord(ev, last));
      TT_CUDA(cudaStreamWaitEvent(s, ev, 0));
    }
    last = s;
    have_last = true;
    return TTALS_OK;
  }

  ttals_status sync_and_read(Ctl* h, bool clear) {
    if (have_last) TT_CUDA(cudaStreamSynchronize(last));
    TT_CUDA(cudaMemcpy(h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (clear && h->latched) {
      int zero = 0;
      TT_CUDA(cudaMemcpy(&ctl->latched, &zero, sizeof(int), cudaMemcpyHostToDevice));
    }
    return TTALS_OK;
  }
};

namespace {

template <typename TX, typename TC>
struct Impl final : ttals_stream {
  using TG = TC;                       // per-CTA Gram accumulation type
  // state, double-buffered by parity
  TC* G[2][kMaxLevels] = {};
  TC* C[2] = {};
  int par = 0;
  // scratch
  TC* Bhat[kMaxLevels] = {};           // B^_k, k = 1..k*-2 (also reconstruct temporaries)
  TC* E[kMaxLevels + 1] = {};          // E_k, k = 2..k*-1
  TC* part = nullptr;                  // split-K partials
  TC* part2 = nullptr;                 // group sums of many split-K partials (orth, pass 0)
  TC* Y = nullptr;                     // reduced local-solve matrix of a level
  TC* Qa = nullptr;                    // first-pass orthogonal factor
  TC* Wpart = nullptr;            // per-CTA Gram partials (accumulation type TG = TC)
  double* T64 = nullptr;
  float* T32 = nullptr;
  double* sumsq = nullptr;
  double* ccpart = nullptr;
  double* hh = nullptr;                // Householder work (fallback and materialisation)
  double* dcores = nullptr;            // FP64 staging of all cores (set_cores)
  double* dtmp[2] = {};                // FP64 chain temporaries (size of C)
  double* mat_q[kMaxLevels + 1] = {};  // materialised cores k*..m (FP64)
  double* mat_g = nullptr;             // materialised g_n
  double* dout = nullptr;              // FP64 staging for core readout
  bool materialised = false;
  size_t part_elems = 0, y_elems = 0, wpart_elems = 0, sumsq_elems = 0, cc_elems = 0, hh_elems = 0;
  // Gram-form modes (lsq, noortho): r x r Grams, their FP64 factor, the unweighted environment
  TC* gM[2] = {};                      // A_k^T A_k of the current and the next level (noortho)
  TC* gBB = nullptr;                   // B^_k B^_k^T
  double* gL64 = nullptr;              // FP64 Cholesky factor of the Gram being solved
  double* gRdiag = nullptr;            // 1 / L_kk
  TC* gEt = nullptr;                   // A_{k*}^T X_(k*) before the last solve (noortho statistics)

  // ---- fused tensor-core path (k* = 2, FP16 / BF16 ingest) -------------------
  static constexpr bool kHalfIngest = std::is_same<TX, __half>::value || std::is_same<TX, __nv_bfloat16>::value;
  bool fast = false;
  int np_ = 16;                 // rank padded to a multiple of 16
  int k1_rows = 0, k2_cols = 0, k2_nq = 1, k2_rch = 16;
  size_t k1_smem = 0, k2_smem = 0;
  // state slabs [nbatch][...] and views of the selected stream's slab
  float* fQb[2] = {};           // Q1 (I_1 x r)
  float* fCb[2] = {};           // F = Q1^T X (r x rest_1): right part of the state
  TX* fChb[2] = {};             // ingest-type copy of F (scaled by 2^-shift)
  float* fW2b[2] = {};          // Q1^T Q1
  int* fShiftb = nullptr;       // [nbatch][2]
  float* fQ[2] = {};
  float* fC[2] = {};
  TX* fCh[2] = {};
  float* fW2[2] = {};
  int* fShift = nullptr;
  double* fHH = nullptr;        // [nbatch][2 I_1 r] Householder work of the factor kernel's fallback
  bool finalized[2] = {true, true};
  float* fY = nullptr;
  float2* fXX = nullptr;       // float-float partials of ||x||^2 (solve CTAs)
  float2* fW1 = nullptr;       // [row tiles][NP*NP] float-float Gram partials of Y (solve CTAs)
  TX* fQh = nullptr;            // Q1 in the ingest type, I_1 x NP (operand of the env kernel)
  float* fW2part = nullptr;     // [8][NP*NP] W2 partials of the factor kernel's ranks
  float* fGff = nullptr;        // [8][2][NP*NP] float-float Gram partials (ill-conditioned steps)
  double* fL64 = nullptr;       // [8][NP*NP] FP64 factor per factor rank (ill-conditioned steps)
  float* fQfb = nullptr;
  float2* fCC = nullptr;       // float-float partials of ||x^||^2 (env CTAs)
  // environment kernel: clustered row chunks, one CTA per 64-column tile over all rows, or
  // 64-column tiles with the rows streamed through a pipeline
  enum { K2_CLUSTER = 0, K2_SINGLE = 1, K2_STREAM = 2, K2_STREAM_TC = 3 };
  int k2_kind = K2_CLUSTER;
  // local solve kernel: mma.sync with k-splits in clusters, or tcgen05 over whole rows
  // (0: chosen per launch, 1: always tcgen05, -1: never)
  int k1_tc = 0;
  unsigned* fCounter = nullptr; // [nbatch][2]
  CUtensorMap mapB[2];          // TMA maps of fChb[p] (nbatch x r x rest_1, box 64 x NP)
  CUtensorMap mapQ;             // TMA map of fQh (nbatch x I_1 x NP, box NP x 64), NP != 48

  int rows(int k) const { return (int)(full[k - 1] * dims[k - 1]); }  // r_{k-1} I_k
  int rk(int k) const { return (int)full[k]; }

  // FP32 state: splits for about 8 resident CTAs per SM (the K loop waits on one global load
  // per 32-wide step, so occupancy is what hides its latency), at least 4 K steps each, up to
  // 1024 (a long contraction with few output tiles: 32 x 32^3 or 30 x 30^5 slices; the
  // partials are summed as float-float pairs); FP64 state: two waves, up to 64 splits (its
  // partials are summed in FP64)
  static constexpr bool kF32State = std::is_same<TC, float>::value;
  static constexpr int kMaxSplit = kF32State ? 1024 : 64;
  static constexpr int kTargetCtas = kF32State ? 8 * kSMs : 2 * kSMs;
  static constexpr long long kMinChunk = kF32State ? 4 * GB_K : GB_K;
  // more than 2 kSplitGroup split partials of a local solve are first summed in groups of
  // kSplitGroup by many threads (k_reduce_split_groups) before the Gram kernel's per-element sum
  static constexpr int kSplitGroup = 16;
  GemmShape plan_solve(int k) const {      // Y = E_k B^_k^T
    return plan_gemm(rows(k), rk(k), rest[k], true, kMaxSplit, kTargetCtas, kMinChunk);
  }
  GemmShape plan_env(int k) const {        // E_{k+1}^T = E_k^T Q_k
    return plan_gemm((int)rest[k], rk(k), rows(k), true, kMaxSplit, kTargetCtas, kMinChunk);
  }
  // Gram partials of a level (the factor kernel sums them on one CTA): at most 16
  int gram_blocks(long long nrows) const { return (int)std::min<long long>(16, cdiv(nrows, 16)); }

  ttals_status allocate() override {
    const bool f64 = std::is_same<TC, double>::value;
    (void)f64;
    for (int p = 0; p < 2; ++p) {
      for (int k = 1; k < kstar; ++k) TT_TRY(dalloc(&G[p][k - 1], (size_t)core_elems(k)));
      TT_TRY(dalloc(&C[p], (size_t)(full[kstar - 1] * rest[kstar - 1])));
    }
    for (int k = 1; k + 1 < kstar; ++k) TT_TRY(dalloc(&Bhat[k], (size_t)(full[k] * rest[k])));
    for (int k = 2; k < kstar; ++k) TT_TRY(dalloc(&E[k], (size_t)(full[k - 1] * rest[k - 1])));
    // reconstruct temporaries need r_{k-1} x rest_{k-1} for k = 2..k*-1: Bhat[k-1] has it
    for (int k = 1; k < kstar; ++k) {
      GemmShape a = plan_solve(k), b = plan_env(k);
      part_elems = std::max<size_t>(part_elems, (size_t)a.nsplit * a.M * a.N);
      part_elems = std::max<size_t>(part_elems, (size_t)b.nsplit * b.M * b.N);
      y_elems = std::max<size_t>(y_elems, (size_t)rows(k) * rk(k));
      wpart_elems = std::max<size_t>(wpart_elems, (size_t)gram_blocks(rows(k)) * rk(k) * rk(k));
      cc_elems = std::max<size_t>(cc_elems, (size_t)kSMs * 4);
      if (k == 1) sumsq_elems = (size_t)a.grid.x * a.grid.z;
      hh_elems = std::max<size_t>(hh_elems, (size_t)2 * rows(k) * rk(k));
    }
    for (int k = std::max(kstar, 1); k <= m; ++k)
      hh_elems = std::max<size_t>(hh_elems, (size_t)2 * rows(k) * std::max<long long>(rest[k], full[k]));
    cc_elems = std::max<size_t>(cc_elems, (size_t)kSMs * 4);
    TT_TRY(dalloc(&part, std::max<size_t>(part_elems, 1)));
    TT_TRY(dalloc(&Y, std::max<size_t>(y_elems, 1)));
    TT_TRY(dalloc(&part2, std::max<size_t>((size_t)cdiv(kMaxSplit, kSplitGroup) * y_elems, 1)));
    TT_TRY(dalloc(&Qa, std::max<size_t>(y_elems, 1)));
    TT_TRY(dalloc(&Wpart, std::max<size_t>(wpart_elems, 1)));
    TT_TRY(dalloc(&T64, (size_t)kMaxRank * kMaxRank));
    TT_TRY(dalloc(&T32, (size_t)kMaxRank * kMaxRank));
    TT_TRY(dalloc(&sumsq, std::max<size_t>(sumsq_elems, 1)));
    TT_TRY(dalloc(&ccpart, cc_elems));
    TT_TRY(dalloc(&hh, std::max<size_t>(hh_elems, 1)));
    size_t ncores = 0;
    for (int k = 1; k <= m; ++k) ncores += (size_t)core_elems(k);
    TT_TRY(dalloc(&dcores, ncores + (size_t)full[m]));
    const size_t csz = (size_t)(full[kstar - 1] * rest[kstar - 1]);
    TT_TRY(dalloc(&dtmp[0], csz));
    TT_TRY(dalloc(&dtmp[1], csz));
    for (int k = kstar; k <= m; ++k) TT_TRY(dalloc(&mat_q[k], (size_t)core_elems(k)));
    TT_TRY(dalloc(&mat_g, (size_t)full[m]));
    size_t maxcore = 0;
    for (int k = 1; k <= m; ++k) maxcore = std::max<size_t>(maxcore, (size_t)core_elems(k));
    TT_TRY(dalloc(&dout, maxcore));
    if (mode != 0) {
      TT_TRY(dalloc(&gM[0], (size_t)kMaxRank * kMaxRank));
      TT_TRY(dalloc(&gM[1], (size_t)kMaxRank * kMaxRank));
      TT_TRY(dalloc(&gBB, (size_t)kMaxRank * kMaxRank));
      TT_TRY(dalloc(&gL64, (size_t)64 * 64));
      TT_TRY(dalloc(&gRdiag, (size_t)64));
      TT_TRY(dalloc(&gEt, csz));
    }
    TT_TRY(dalloc(&ctl, (size_t)nbatch));
    TT_CUDA(cudaMemset(ctl, 0, sizeof(Ctl) * nbatch));
    ctl_base = ctl;
    TT_CUDA(cudaFuncSetAttribute(k_factor<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    TT_CUDA(cudaFuncSetAttribute(fast::k_chol64_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    TT_TRY(setup_fast());
    return TTALS_OK;
  }

  // Each kernel's dynamic shared-memory limit is a per-kernel (not per-stream) setting: raise
  // it once to the device's opt-in maximum, so that streams of any shape (in any creation
  // order) can launch their own sizes.  The limit only validates launches; occupancy follows
  // the size a launch asks for.
  template <typename K>
  ttals_status raise_smem_limit(K kern) {
    cudaFuncAttributes fa{};
    TT_CUDA(cudaFuncGetAttributes(&fa, kern));
    int optin = 0;
    TT_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    TT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
    return TTALS_OK;
  }

  template <int NP>
  ttals_status set_fast_attrs() {
    if constexpr (kHalfIngest) {
      TT_TRY(raise_smem_limit(fast::k_fast_solve<TX, NP>));
      TT_TRY(raise_smem_limit(fast::k_fast_solve_tc<TX, NP>));
      TT_TRY(raise_smem_limit(fast::k_fast_env1<TX, NP>));
      TT_TRY(raise_smem_limit(fast::k_fast_env_stream<TX, NP>));
      if constexpr (NP != 48) TT_TRY(raise_smem_limit(fast::k_fast_env_tc<TX, NP>));
      TT_TRY(raise_smem_limit(fast::k_fast_env<TX, NP>));
      TT_TRY(raise_smem_limit(fast::k_fast_factor<TX, NP, 8>));
      TT_TRY(raise_smem_limit(fast::k_fast_factor<TX, NP, 4>));
    }
    return TTALS_OK;
  }

  // the fused path covers k* = 2 with FP16/BF16 ingest, r_1 <= 64, rows of the slice
  // 16-byte aligned (rest_1 % 8 == 0) and I_1 small enough for one cluster of row chunks
  ttals_status setup_fast() {
    if (!kHalfIngest || kstar != 2 || mode != 0) return TTALS_OK;
    const long long M = dims[0], J = rest[1];
    const int r = rk(1);
    if (J % 8 != 0 || r > 64 || M > 8 * 512) return TTALS_OK;
    np_ = ((r + 15) / 16) * 16;
    // the factor cluster holds 1/8 of Y and Q1 per CTA in shared memory (plus its static
    // shared memory, fast::K1B_STATIC_SMEM)
    if (fast::k1b_smem_bytes((int)M, r, np_) + fast::K1B_STATIC_SMEM > 227 * 1024) {
      np_ = 16;
      return TTALS_OK;
    }
    k1_rows = (int)cdiv(M, fast::K1_BM);
    k2_cols = (int)cdiv(J, fast::K2_BN);
    // row chunks per cluster: the fewest (largest chunks) that keep two env CTAs per SM
    auto k2_bytes = [&](int rch) -> size_t {
      switch (np_) {
        case 16: return fast::k2_smem_bytes<16>(rch, r);
        case 32: return fast::k2_smem_bytes<32>(rch, r);
        case 48: return fast::k2_smem_bytes<48>(rch, r);
        default: return fast::k2_smem_bytes<64>(rch, r);
      }
    };
    k2_nq = 0;
    for (int nq = (int)std::max<long long>(1, std::min<long long>(8, cdiv(M, 256))); nq <= 8; ++nq) {
      const int rch = (int)(cdiv(cdiv(M, nq), 16) * 16);
      if (k2_bytes(rch) <= 113 * 1024) {
        k2_nq = nq;
        break;
      }
    }
    if (k2_nq == 0) k2_nq = 8;
    k2_rch = (int)(cdiv(cdiv(M, k2_nq), 16) * 16);
    k2_smem = k2_bytes(k2_rch);
    {
      bool fits = false;
      size_t b1 = 0;
      switch (np_) {
        case 16: fits = fast::k2s_fits<16>((int)M, r); b1 = fast::k2s_smem_bytes<16>((int)M, r); break;
        case 32: fits = fast::k2s_fits<32>((int)M, r); b1 = fast::k2s_smem_bytes<32>((int)M, r); break;
        case 64: fits = fast::k2s_fits<64>((int)M, r); b1 = fast::k2s_smem_bytes<64>((int)M, r); break;
        default: break;
      }
      // environment kernel: for batches streamed row stages on tcgen05 (the mma.sync version
      // for ranks padded to 48); for one stream the whole-column CTA when its tile fits, else
      // the cluster kernel.  TTALS_ENV_KERNEL=cluster|single|stream|streamtc overrides (single
      // only if it fits).
      k2_kind = nbatch > 1 ? (np_ != 48 ? K2_STREAM_TC : K2_STREAM) : (fits ? K2_SINGLE : K2_CLUSTER);
      if (const char* e = std::getenv("TTALS_ENV_KERNEL")) {
        const std::string v(e);
        if (v == "cluster") k2_kind = K2_CLUSTER;
        else if (v == "stream") k2_kind = K2_STREAM;
        else if (v == "streamtc") k2_kind = K2_STREAM_TC;
        else if (v == "single" && fits) k2_kind = K2_SINGLE;
      }
      // TTALS_SOLVE_KERNEL=tc|mma fixes the local-solve kernel (else chosen per launch)
      if (const char* e = std::getenv("TTALS_SOLVE_KERNEL")) k1_tc = std::string(e) == "tc" ? 1 : -1;
      if (cfg_solve_kernel == 1) k1_tc = -1;                  // the stream's config wins
      else if (cfg_solve_kernel == 2) k1_tc = 1;
      if (cfg_env_kernel == 1) k2_kind = K2_CLUSTER;          // the stream's config wins
      else if (cfg_env_kernel == 2 && fits) k2_kind = K2_SINGLE;
      else if (cfg_env_kernel == 3) k2_kind = K2_STREAM;
      else if (cfg_env_kernel == 4) k2_kind = K2_STREAM_TC;
      if (k2_kind == K2_SINGLE) {
        k2_nq = 1;
        k2_cols = (int)cdiv(J, fast::K2S_BN);
        k2_rch = fast::k2s_box_rows((int)M);      // TMA box height of the env kernel's X map
        k2_smem = b1;
      }
      if (k2_kind == K2_STREAM_TC && np_ == 48) k2_kind = K2_STREAM;   // no swizzle atom for 48
      if (k2_kind == K2_STREAM_TC) {
        k2_nq = 1;
        k2_cols = (int)cdiv(J, fast::K2T_BN);
        k2_rch = fast::K1_BM;
        switch (np_) {
          case 16: k2_smem = fast::k2t_smem_bytes<16>(); break;
          case 32: k2_smem = fast::k2t_smem_bytes<32>(); break;
          default: k2_smem = fast::k2t_smem_bytes<64>(); break;
        }
      } else if (k2_kind == K2_STREAM) {
        k2_nq = 1;
        k2_cols = (int)cdiv(J, fast::K2P_BN);
        k2_rch = fast::K1_BM;                     // reads X through the solve kernel's map
        switch (np_) {
          case 16: k2_smem = fast::k2p_smem_bytes<16>(); break;
          case 32: k2_smem = fast::k2p_smem_bytes<32>(); break;
          case 48: k2_smem = fast::k2p_smem_bytes<48>(); break;
          default: k2_smem = fast::k2p_smem_bytes<64>(); break;
        }
      }
    }
    switch (np_) {
      case 16: k1_smem = fast::k1_smem_bytes<16>(); break;
      case 32: k1_smem = fast::k1_smem_bytes<32>(); break;
      case 48: k1_smem = fast::k1_smem_bytes<48>(); break;
      default: k1_smem = fast::k1_smem_bytes<64>(); break;
    }
    // after the main loop the solve CTA reuses its buffers: P (64 x NP), its reduced rows
    // (64 x (NP+4)), the Gram's row-group partials and the Gram (NP x NP each); + alignment
    {
      const int ng = std::max(1, fast::K1_THREADS / ((np_ / 4) * (np_ / 4)));
      k1_smem = std::max(k1_smem, (size_t)(64 * np_ + 64 * (np_ + 4) + (ng + 1) * np_ * np_) * 4 + 1024);
    }
    if (k2_smem > 226 * 1024 || k2_rch > 256) return TTALS_OK;
    if (!tensor_map_encoder()) return TTALS_OK;
    switch (np_) {
      case 16: TT_TRY(set_fast_attrs<16>()); break;
      case 32: TT_TRY(set_fast_attrs<32>()); break;
      case 48: TT_TRY(set_fast_attrs<48>()); break;
      default: TT_TRY(set_fast_attrs<64>()); break;
    }
    // every buffer below is a slab of nbatch per-stream parts; the kernels offset by blockIdx.z
    const size_t S = (size_t)nbatch;
    for (int p = 0; p < 2; ++p) {
      TT_TRY(dalloc(&fQb[p], S * M * r));
      TT_TRY(dalloc(&fCb[p], S * r * J));
      TT_TRY(dalloc(&fChb[p], S * r * J));
      TT_TRY(dalloc(&fW2b[p], S * r * r));
    }
    TT_TRY(dalloc(&fShiftb, S * 2));
    TT_TRY(dalloc(&fY, S * M * r));
    TT_TRY(dalloc(&fXX, S * k1_rows * 8));            // room for the largest k-split
    TT_TRY(dalloc(&fW1, S * k1_rows * np_ * np_));    // room for the 64-row tiles
    TT_TRY(dalloc(&fQh, S * M * np_));
    TT_TRY(dalloc(&fW2part, S * fast::KB_CLUSTER * np_ * np_));
    TT_TRY(dalloc(&fGff, S * fast::KB_CLUSTER * 2 * np_ * np_));
    TT_TRY(dalloc(&fL64, S * fast::KB_CLUSTER * np_ * np_));
    TT_TRY(dalloc(&fQfb, S * M * r));
    TT_TRY(dalloc(&fHH, S * 2 * M * r));
    TT_TRY(dalloc(&fCC, S * k2_cols * k2_nq));
    TT_TRY(dalloc(&fCounter, S * 2));
    TT_CUDA(cudaMemset(fCounter, 0, S * 2 * sizeof(unsigned)));
    const bool bf = std::is_same<TX, __nv_bfloat16>::value;
    for (int p = 0; p < 2; ++p)
      if (!encode_map_3d(&mapB[p], fChb[p], bf, nbatch, r, J, np_)) return TTALS_OK;
    if (np_ != 48 && !encode_map_3d_q(&mapQ, fQh, bf, nbatch, M, np_)) return TTALS_OK;
    TT_CUDA(cudaMemset(fShiftb, 0, S * 2 * sizeof(int)));
    fast = true;
    return select_slot(0);
  }

  bool batch_capable() const override { return fast; }

  // point the per-stream views (state, control block) at stream idx of the batch
  ttals_status select_slot(int idx) override {
    if (idx < 0 || idx >= nbatch) return TTALS_EINVAL;
    sel = idx;
    ctl = ctl_base + idx;
    if (fast) {
      const size_t M = (size_t)dims[0], J = (size_t)rest[1], r = (size_t)rk(1);
      for (int p = 0; p < 2; ++p) {
        fQ[p] = fQb[p] + idx * M * r;
        fC[p] = fCb[p] + idx * r * J;
        fCh[p] = fChb[p] + idx * r * J;
        fW2[p] = fW2b[p] + idx * r * r;
      }
      fShift = fShiftb + 2 * idx;
      finalized[0] = finalized[1] = false;
    }
    materialised = false;
    return TTALS_OK;
  }

  // per-slice-address TMA maps {solve box, env box}; cleared when it reaches its cap
  struct SliceMaps {
    CUtensorMap m[3];           // solve box 64 x 64, env box 64 x rch, tcgen05 solve box 64 x 128
  };
  std::unordered_map<const void*, SliceMaps> map_cache;
  const CUtensorMap* slice_maps(const TX* X) {
    constexpr size_t kMapCacheCap = 1024;
    auto it = map_cache.find((const void*)X);
    if (it != map_cache.end()) return it->second.m;
    if (map_cache.size() >= kMapCacheCap) map_cache.clear();
    SliceMaps sm;
    const bool bf = std::is_same<TX, __nv_bfloat16>::value;
    if (!encode_map_3d(&sm.m[0], X, bf, nbatch, dims[0], rest[1], fast::K1_BM) ||
        !encode_map_3d(&sm.m[1], X, bf, nbatch, dims[0], rest[1], k2_rch) ||
        !encode_map_3d(&sm.m[2], X, bf, nbatch, dims[0], rest[1], fast::K1T_BM))
      return nullptr;
    return map_cache.emplace((const void*)X, sm).first->second.m;
  }

  ttals_status warm_slice(const void* x) override {
    if (!fast) return TTALS_OK;
    if (!slice_maps((const TX*)x)) {
      g_last_err = "cuTensorMapEncodeTiled failed";
      return TTALS_ECUDA;
    }
    return TTALS_OK;
  }

  template <int NP>
  ttals_status launch_fast(const TX* X, cudaStream_t s) {
    if constexpr (kHalfIngest) {
      const int np = 1 - par;
      const int r = rk(1);
      cudaLaunchAttribute at[2];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 1;
      at[0].val.clusterDim.z = 1;
      at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[1].val.programmaticStreamSerializationAllowed = (profiling || no_pdl) ? 0 : 1;
      // TMA maps of this slice (box 64 x 64 for the solve, 64 x rch for the env kernel),
      // cached by slice address: a stream fed from a ring of device buffers encodes each
      // buffer's maps once
      const CUtensorMap* maps = slice_maps(X);
      if (!maps) {
        g_last_err = "cuTensorMapEncodeTiled failed";
        return TTALS_ECUDA;
      }
      const CUtensorMap& mapX1 = maps[0];
      const CUtensorMap& mapX2 = maps[1];
      // the grids' planes cover the streams that step; the others' state is carried over
      unsigned char zact[64], zidle[64];
      int n_act = 0, n_idle = 0;
      for (int b = 0; b < nbatch; ++b) {
        if ((active_mask >> b) & 1ull) zact[n_act++] = (unsigned char)b;
        else zidle[n_idle++] = (unsigned char)b;
      }
      if (n_act == 0) return TTALS_OK;
      // k-splits of the solve, for the streams that step: up to two CTAs per SM, and clusters
      // of 8 only while they fit one CTA per SM (more 8-CTA clusters do not fit the GPCs at
      // once); a batch that fills the GPU with row tiles takes none (longer CTAs, no cluster
      // reduction).  A configured split wins.
      int split = 8;
      while (split > 1 && ((long long)k1_rows * split * n_act > 2 * kSMs ||
                           (split == 8 && (long long)k1_rows * split * n_act > kSMs)))
        split >>= 1;
      if (cfg_k1_split > 0) split = cfg_k1_split;
      const long long kchunk = cdiv(cdiv(rest[1], split), fast::K1_BK) * fast::K1_BK;
      at[0].val.clusterDim.y = (unsigned)split;
      // K1: local solve
      fast::SolveArgs a1{};
      a1.M = (int)dims[0];
      a1.r = r;
      a1.K = rest[1];
      a1.kchunk = kchunk;
      a1.Y = fY;
      a1.xx_part = fXX;
      a1.W1part = fW1;
      a1.w1_stride = (long long)k1_rows * NP * NP;
      a1.ctl = ctl_base;
      std::memcpy(a1.zmap, zact, sizeof(zact));
      cudaLaunchConfig_t c1{};
      c1.gridDim = dim3((unsigned)k1_rows, (unsigned)split, (unsigned)n_act);
      c1.blockDim = dim3(fast::K1_THREADS, 1, 1);
      c1.dynamicSmemBytes = k1_smem;
      c1.stream = s;
      c1.attrs = at;
      c1.numAttrs = 2;
      TT_TRY(mark(1, s));
      int nxx = k1_rows * split;               // ||x||^2 partials per stream
      int nw1 = k1_rows;                       // Gram partials per stream (row tiles)
      // tcgen05 over whole rows once its 128-row tiles of the stepping streams cover three
      // quarters of the SMs (one CTA per SM); below that the k-split mma.sync kernel fills
      // the GPU better
      const int rows_tc = (int)cdiv(dims[0], fast::K1T_BM);
      a1.stall = stall_pushes > 0 ? 1 : 0;
      if (stall_pushes > 0) --stall_pushes;
      const bool use_tc = !a1.stall && (k1_tc > 0 || (k1_tc == 0 && 4LL * rows_tc * n_act >= 3LL * kSMs));
      if (use_tc) {
        c1.gridDim = dim3((unsigned)rows_tc, 1, (unsigned)n_act);
        c1.blockDim = dim3(fast::K1T_THREADS, 1, 1);
        c1.dynamicSmemBytes = fast::k1t_smem_bytes<NP>();
        c1.attrs = at + 1;                     // no cluster
        c1.numAttrs = 1;
        TT_CUDA(cudaLaunchKernelEx(&c1, fast::k_fast_solve_tc<TX, NP>, maps[2], mapB[par], a1));
        nxx = rows_tc;
        nw1 = rows_tc;
      } else {
        TT_CUDA(cudaLaunchKernelEx(&c1, fast::k_fast_solve<TX, NP>, mapX1, mapB[par], a1));
      }
      ++nlaunch;
      TT_TRY(mark(2, s));
      // K1b: r x r factor, Q1, W2, Nx
      fast::FactorArgs ab{};
      ab.Y = fY;
      ab.xx_part = fXX;
      ab.nxx = nxx;
      ab.W1part = fW1;
      ab.w1_stride = a1.w1_stride;
      ab.nw1 = nw1;
      ab.M = (int)dims[0];
      ab.r = r;
      ab.Qh = fQh;
      ab.Qst = fQb[np];
      ab.W2part = fW2part;
      ab.hh_work = fHH;
      ab.Qfb = fQfb;
      ab.ctl = ctl_base;
      ab.fp64 = cfg_factor == 0 ? 1 : 0;
      ab.Gff = fGff;
      ab.L64ws = fL64;
      std::memcpy(ab.zmap, zact, sizeof(zact));
      // clusters of 8 one-CTA-per-SM CTAs fit the GPCs for up to 8 streams at once; beyond
      // that clusters of 4 (twice the rows per CTA) keep the step in one wave
      const bool fits4 = fast::k1b_smem_bytes((int)dims[0], r, NP, 4) + fast::K1B_STATIC_SMEM <= 227 * 1024;
      int kbc = (n_act > 8 && fits4) ? 4 : 8;
      if (cfg_factor_cluster == 4 && fits4) kbc = 4;          // a configured cluster size wins
      else if (cfg_factor_cluster == 8) kbc = 8;
      cudaLaunchAttribute atb[2];
      atb[0] = at[0];
      atb[0].val.clusterDim.y = (unsigned)kbc;
      atb[1] = at[1];
      cudaLaunchConfig_t cb{};
      cb.gridDim = dim3(1, (unsigned)kbc, (unsigned)n_act);
      cb.blockDim = dim3(fast::K1B_THREADS, 1, 1);
      cb.dynamicSmemBytes = fast::k1b_smem_bytes((int)dims[0], r, NP, kbc);
      cb.stream = s;
      cb.attrs = atb;
      cb.numAttrs = 2;
      if (kbc == 4)
        TT_CUDA(cudaLaunchKernelEx(&cb, fast::k_fast_factor<TX, NP, 4>, ab));
      else
        TT_CUDA(cudaLaunchKernelEx(&cb, fast::k_fast_factor<TX, NP, 8>, ab));
      ++nlaunch;
      TT_TRY(mark(3, s));
      // K2: environment
      fast::EnvArgs a2{};
      a2.M = (int)dims[0];
      a2.r = r;
      a2.J = rest[1];
      a2.rch = k2_rch;
      a2.Qh = fQh;
      a2.W2part = fW2part;
      a2.Cst = fCb[np];
      a2.Chst = fChb[np];
      a2.ch_shift = fShiftb + np;
      a2.cc_part = fCC;
      a2.counter = fCounter + 1;
      a2.ctl = ctl_base;
      a2.Qst = fQb[np];
      a2.W2st = fW2b[np];
      a2.Qold = fQb[par];
      a2.Cold = fCb[par];
      a2.Chold = fChb[par];
      a2.W2old = fW2b[par];
      a2.ch_shift_old = fShiftb + par;
      a2.is_half = std::is_same<TX, __half>::value ? 1 : 0;
      a2.w2_parts = kbc;
      // the environment kernel takes the stepping streams in the reverse of the solve kernel's
      // order: the slices the solve read last (up to the L2's size) are then read again from L2
      for (int z = 0; z < n_act; ++z) a2.zmap[z] = zact[n_act - 1 - z];
      at[0].val.clusterDim.y = (unsigned)k2_nq;
      cudaLaunchConfig_t c2{};
      c2.gridDim = dim3((unsigned)k2_cols, (unsigned)k2_nq, (unsigned)n_act);
      c2.blockDim = dim3(fast::K2_THREADS, 1, 1);
      c2.dynamicSmemBytes = k2_smem;
      c2.stream = s;
      if (k2_kind == K2_SINGLE) {
        c2.attrs = at + 1;       // no cluster
        c2.numAttrs = 1;
        TT_CUDA(cudaLaunchKernelEx(&c2, fast::k_fast_env1<TX, NP>, mapX2, a2));
      } else if (k2_kind == K2_STREAM_TC) {
        if constexpr (NP != 48) {
          c2.blockDim = dim3(fast::K2T_THREADS, 1, 1);
          c2.attrs = at + 1;     // no cluster
          c2.numAttrs = 1;
          TT_CUDA(cudaLaunchKernelEx(&c2, fast::k_fast_env_tc<TX, NP>, mapX1, mapQ, a2));
        }
      } else if (k2_kind == K2_STREAM) {
        c2.blockDim = dim3(fast::K2P_THREADS, 1, 1);
        c2.attrs = at + 1;       // no cluster
        c2.numAttrs = 1;
        TT_CUDA(cudaLaunchKernelEx(&c2, fast::k_fast_env_stream<TX, NP>, mapX1, a2));
      } else {
        c2.attrs = at;
        c2.numAttrs = 2;
        TT_CUDA(cudaLaunchKernelEx(&c2, fast::k_fast_env<TX, NP>, mapX2, a2));
      }
      ++nlaunch;
      TT_TRY(mark(4, s));
      if (n_idle > 0) {
        // streams without a slice this step: their state moves to the new buffers unchanged
        fast::EnvArgs ac = a2;
        std::memcpy(ac.zmap, zidle, sizeof(zidle));
        const long long rj = (long long)r * rest[1];
        const int nb = (int)std::min<long long>(cdiv(rj, 256), 64);
        fast::k_fast_carry<TX, NP><<<dim3((unsigned)nb, 1, (unsigned)n_idle), 256, 0, s>>>(ac);
        TT_CUDA(cudaGetLastError());
        ++nlaunch;
      }
      finalized[np] = false;
      materialised = false;
      par = np;
    }
    return TTALS_OK;
  }

  ttals_status push_fast(const TX* X, cudaStream_t s) {
    switch (np_) {
      case 16: return launch_fast<16>(X, s);
      case 32: return launch_fast<32>(X, s);
      case 48: return launch_fast<48>(X, s);
      default: return launch_fast<64>(X, s);
    }
  }

  // fused-path state -> orthonormal-gauge cores G_1 = Q1 R2^{-1}, C = R2^{-T} F
  // (R2 = chol(Q1^T Q1), FP64), written to the generic state buffers of this parity
  ttals_status finalize(cudaStream_t s) {
    if (!fast || finalized[par]) return TTALS_OK;
    const int r = rk(1);
    const long long M = dims[0], J = rest[1];
    fast::k_chol64_inverse<<<1, 256, (size_t)2 * r * r * 8, s>>>(fW2[par], r, T64, T32);
    TT_CUDA(cudaGetLastError());
    const int nb = (int)std::min<long long>(cdiv(M * r, 256), 4 * kSMs);
    fast::k_apply_upper<<<nb, 256, 0, s>>>(fQ[par], M, r, T32, (float*)G[par][0]);
    TT_CUDA(cudaGetLastError());
    // C[a][j] = sum_b T[b][a] F[b][j]
    GemmShape g = plan_gemm(r, (int)J, r, false);
    TT_TRY((gemm<float, float, float, float, false, false>(g, T32, r, fC[par], J, (float*)C[par], J, 1, 0, nullptr,
                                                           nullptr, nullptr, nullptr, s)));
    finalized[par] = true;
    return TTALS_OK;
  }

  // after set_cores: mirror the generic state into the fused-path state
  ttals_status sync_fast_from_generic(cudaStream_t s) {
    if constexpr (kHalfIngest) {
      if (!fast) return TTALS_OK;
      const int r = rk(1);
      const long long M = dims[0], J = rest[1];
      static_assert(std::is_same<TC, float>::value, "the fused path keeps FP32 state");
      TT_CUDA(cudaMemcpyAsync(fQ[par], G[par][0], (size_t)(M * r) * 4, cudaMemcpyDeviceToDevice, s));
      // W2 = G1^T G1 and F = W2 C: the fused state (Q1, W2, F) stands for x^ = Q1 W2^{-1} F,
      // which is G1 C also for a first core that is not orthonormal
      TT_TRY((gemm<float, float, float, float, false, false>(plan_gemm(r, r, M, false), G[par][0], r, G[par][0], r,
                                                             fW2[par], r, 1, 0, nullptr, nullptr, nullptr, nullptr, s)));
      TT_TRY((gemm<float, float, float, float, true, false>(plan_gemm(r, (int)J, r, false), fW2[par], r, C[par], J,
                                                            fC[par], J, 1, 0, nullptr, nullptr, nullptr, nullptr, s)));
      fast::k_make_half_copy<TX><<<1, 1024, 0, s>>>(fC[par], r * J, fCh[par], fShift + par,
                                                    std::is_same<TX, __half>::value ? 1 : 0);
      TT_CUDA(cudaGetLastError());
      finalized[par] = true;
    }
    return TTALS_OK;
  }

  // ---- launch helpers --------------------------------------------------------
  // a generic-path kernel with programmatic dependent launch (each such kernel waits for its
  // predecessor at entry: gen_pdl_start), unless profiling or TTALS_NO_PDL
  template <typename... KArgs, typename... Args>
  ttals_status launch_gen(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args&&... args) {
    cudaLaunchConfig_t c{};
    c.gridDim = grid;
    c.blockDim = block;
    c.dynamicSmemBytes = smem;
    c.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = (profiling || no_pdl) ? 0 : 1;
    c.attrs = at;
    c.numAttrs = 1;
    TT_CUDA(cudaLaunchKernelEx(&c, kern, std::forward<Args>(args)...));
    return TTALS_OK;
  }

  template <typename TA, typename TB, typename TACC, typename TD, bool AK, bool BK>
  ttals_status gemm(const GemmShape& g, const TA* A, long long lda, const TB* B, long long ldb, TD* D,
                    long long sdm, long long sdn, long long sstride, double* ss,
                    const double* bzero, const Ctl* chk, Ctl* reset, cudaStream_t s) {
    TT_TRY(launch_gen(k_gemm<TA, TB, TACC, TD, AK, BK>, g.grid, dim3(G_THREADS), 0, s, A, lda, B, ldb, D, sdm,
                      sdn, sstride, g.M, g.N, g.K, g.kchunk, ss, bzero, chk, reset));
    ++nlaunch;
    return TTALS_OK;
  }

  // orthonormal basis of the level-k local solve.  Input: split partials of Y
  // (nsplit x rows x r) in `part`.  Output: Q (rows x r) in `qout`.
  ttals_status orth(int k, int nsplit, bool first, TC* qout, cudaStream_t s, const TC* src0 = nullptr) {
    const long long n = rows(k);
    const int r = rk(k);
    const int nb = gram_blocks(n);
    const long long rpb = cdiv(n, nb);
    const int nblk = (int)cdiv(n, rpb);
    const size_t gsm = (size_t)GRAM_CHUNK * r * sizeof(TG);
    const size_t fsm = (size_t)r * r * 8 + (size_t)r * 8 + (size_t)r * (r + 1) * 4;
    const size_t asm_ = (size_t)r * r * sizeof(TC);
    const int ablk = (int)std::min<long long>(4 * kSMs, std::max<long long>(1, cdiv(n * r, APPLY_THREADS)));
    const int sum_n = (int)sumsq_elems;
    for (int pass = 0; pass < qr_passes; ++pass) {
      const int slot = 2 * (k - 1) + pass;
      // pass 0 reads the split partials of the local solve (or, with src0, the reduced solve
      // already in Y) and leaves the reduced solve in Y
      const TC* src = pass == 0 ? (src0 ? src0 : (const TC*)part) : (const TC*)Qa;
      TC* dst = (pass + 1 == qr_passes) ? qout : Qa;
      int nsrc = pass == 0 ? nsplit : 1;
      if (pass == 0 && !src0 && nsplit > 2 * kSplitGroup) {
        const long long ne = n * r;
        const int ng = (int)cdiv(nsplit, kSplitGroup);
        const int nbr = (int)std::min<long long>(cdiv((long long)ng * ne, 256), 8 * kSMs);
        TT_TRY(launch_gen(k_reduce_split_groups<TC>, dim3(nbr), dim3(256), 0, s, (const TC*)part, nsplit,
                          kSplitGroup, ne, part2, (const Ctl*)ctl));
        ++nlaunch;
        src = part2;
        nsrc = ng;
      }
      TT_TRY(launch_gen(k_gram<TC, TC, TG>, dim3(nblk), dim3(GRAM_THREADS), gsm, s, src, nsrc,
                        (long long)(n * r), (long long)n, r, (pass == 0 && !src0) ? Y : (TC*)nullptr, Wpart, (long long)rpb,
                        (const Ctl*)ctl));
      TT_TRY(launch_gen(k_factor<TC>, dim3(1), dim3(FACT_THREADS), fsm, s, (const TC*)Wpart, nblk, r,
                        pass == 0 ? 0 : 1, T64, T32, ctl, slot, (const double*)sumsq, sum_n,
                        (first && pass == 0) ? 1 : 0));
      TT_TRY(launch_gen(k_apply<TC>, dim3(ablk), dim3(APPLY_THREADS), asm_, s, pass == 0 ? (const TC*)Y : (const TC*)Qa,
                        (long long)n, r, pass == 0 ? 0 : 1, (const double*)T64, (const float*)T32, dst,
                        (const Ctl*)ctl, slot, hh));
      nlaunch += 3;
    }
    return TTALS_OK;
  }

  // ---- one step of Algorithm 1 -------------------------------------------------
  ttals_status push(const void* xv, cudaStream_t s) override {
    TT_TRY(mark(0, s));
    TT_TRY(push_body(xv, s));
    TT_TRY(mark(5, s));
    if (profiling) ev_used += kProfEvents;
    return TTALS_OK;
  }

  ttals_status push_body(const void* xv, cudaStream_t s) {
    const TX* X = (const TX*)xv;
    if (fast) return push_fast(X, s);
    if (mode != 0 && kstar > 1) return push_body_gram(X, s);
    const int np = 1 - par;
    materialised = false;
    CopyList rl{};
    for (int k = 1; k < kstar; ++k) {
      rl.src[rl.n] = G[par][k - 1];
      rl.dst[rl.n] = G[np][k - 1];
      rl.bytes[rl.n] = core_elems(k) * (long long)sizeof(TC);
      ++rl.n;
    }
    rl.src[rl.n] = C[par];
    rl.dst[rl.n] = C[np];
    rl.bytes[rl.n] = full[kstar - 1] * rest[kstar - 1] * (long long)sizeof(TC);
    ++rl.n;

    if (kstar == 1) {   // r_1 >= I_2...I_{n-1}: x^_t = X_t
      const int nb = (int)std::min<long long>(cdiv(rest[0], 256), 2 * kSMs);
      TT_TRY(launch_gen(k_copy_slice<TX, TC>, dim3(nb), dim3(256), 0, s, X, (long long)rest[0], C[np], ccpart, ctl));
      TT_TRY(launch_gen(k_commit, dim3(1), dim3(256), 0, s, ctl, (const double*)ccpart, nb, (const double*)ccpart, nb,
                        rl));
      nlaunch += 2;
      par = np;
      return TTALS_OK;
    }
    bool first_launch = true;
    // right interfaces B^_k = G_{k+1} x B^_{k+1}, B^_{k*-1} = C  (old state)
    for (int k = kstar - 2; k >= 1; --k) {
      const bool fromC = (k == kstar - 2);
      const TC* Bsrc = fromC ? C[par] : Bhat[k + 1];
      GemmShape g = plan_gemm(rows(k + 1), (int)rest[k + 1], rk(k + 1), false);
      TT_TRY((gemm<TC, TC, TC, TC, true, false>(g, G[par][k], rk(k + 1), Bsrc, rest[k + 1], Bhat[k], rest[k + 1],
                                                 1, 0, nullptr, fromC ? &ctl->cc : nullptr, nullptr,
                                                 first_launch ? ctl : nullptr, s)));
      first_launch = false;
    }
    // forward sweep
    int ncc = 0;
    for (int k = 1; k < kstar; ++k) {
      const bool last_level = (k == kstar - 1);
      const TC* Bk = last_level ? C[par] : Bhat[k];
      GemmShape gs = plan_solve(k);
      if (k == 1) {
        TT_TRY(mark(1, s));
        TT_TRY(solve_level1(gs, X, Bk, last_level ? &ctl->cc : nullptr, first_launch ? ctl : nullptr, s));
        TT_TRY(mark(2, s));
      } else {
        TT_TRY((gemm<TC, TC, TC, TC, true, true>(gs, E[k], rest[k], Bk, rest[k], part, rk(k), 1,
                                                 (long long)gs.M * gs.N, nullptr,
                                                 last_level ? &ctl->cc : nullptr, ctl, nullptr, s)));
      }
      first_launch = false;
      TC* qdst = G[np][k - 1];
      TT_TRY(orth(k, gs.nsplit, k == 1, qdst, s));
      GemmShape ge = plan_env(k);
      if (k == 1) {
        TT_TRY(mark(3, s));
        TT_TRY(env_level1(ge, X, qdst, s));
        TT_TRY(mark(4, s));
      } else {
        TT_TRY((gemm<TC, TC, TC, TC, false, false>(ge, E[k], rest[k], qdst, rk(k), part, rk(k), 1,
                                                   (long long)ge.M * ge.N, nullptr, nullptr, ctl, nullptr, s)));
      }
      TC* eout = last_level ? C[np] : E[k + 1];
      const int nb = (int)std::min<long long>(cdiv(rest[k] * rk(k), RED_THREADS), 4 * kSMs);
      TT_TRY(launch_gen(k_reduce_t<TC>, dim3(nb), dim3(RED_THREADS), 0, s, (const TC*)part, ge.nsplit,
                        (long long)ge.M * ge.N, (long long)rest[k], rk(k), eout,
                        last_level ? ccpart : (double*)nullptr, (const Ctl*)ctl));
      ++nlaunch;
      if (last_level) ncc = nb;
    }
    TT_TRY(launch_gen(k_commit, dim3(1), dim3(256), 0, s, ctl, (const double*)ccpart, ncc, (const double*)nullptr, 0,
                      rl));
    ++nlaunch;
    par = np;
    return TTALS_OK;
  }

  // ---- Gram-form modes (Sec. 3.3): the normal equations of each local least-squares problem
  // S <- S^{-1} applied to n vectors of the matrix V (see k_r64_apply), S an r x r Gram in TC:
  // the batched FP64 factor kernel (one matrix here) and the FP64 apply
  ttals_status spd_solve(const TC* S, int r, TC* V, long long n, long long vstride, long long estride,
                         cudaStream_t s) {
    const int nb = (int)std::min<long long>(std::max<long long>(1, cdiv(n, 128)), 4 * kSMs);
    if (r <= 16) {
      r64::k_r64_factor<TC, 16><<<1, r64::kFactorThreads, 0, s>>>(S, 0, r, 1e-14, gL64, gRdiag, nullptr);
      r64::k_r64_apply<TC, 16><<<nb, 128, 0, s>>>(gL64, gRdiag, r, V, n, vstride, estride, &ctl->skip);
    } else if (r <= 32) {
      r64::k_r64_factor<TC, 32><<<1, r64::kFactorThreads, 0, s>>>(S, 0, r, 1e-14, gL64, gRdiag, nullptr);
      r64::k_r64_apply<TC, 32><<<nb, 128, 0, s>>>(gL64, gRdiag, r, V, n, vstride, estride, &ctl->skip);
    } else {
      r64::k_r64_factor<TC, 64><<<1, r64::kFactorThreads, 0, s>>>(S, 0, r, 1e-14, gL64, gRdiag, nullptr);
      r64::k_r64_apply<TC, 64><<<nb, 128, 0, s>>>(gL64, gRdiag, r, V, n, vstride, estride, &ctl->skip);
    }
    TT_CUDA(cudaGetLastError());
    nlaunch += 2;
    return TTALS_OK;
  }

  // One step of Algorithm 1 with every local solve in its Gram form (mode lsq, with the QR
  // left-orthogonalisation of Sec. 3.4.2 kept), or with the LQ/QR steps removed as in the
  // ablation of Sec. 5.4 (mode noortho: G_k = (A_k^T A_k)^-1 A_k^T X B_k^T (B_k B_k^T)^-1, no
  // orthogonalisation, the collapsed right part C = (A_k*^T A_k*)^-1 A_k*^T X).  In exact
  // arithmetic both give the reconstruction of the literal update.  Right interfaces as in
  // push_body (B^_k from the old cores, no LQ sweep).
  ttals_status push_body_gram(const TX* X, cudaStream_t s) {
    const int np = 1 - par;
    const bool ortho = mode == 1;
    materialised = false;
    CopyList rl{};
    for (int k = 1; k < kstar; ++k) {
      rl.src[rl.n] = G[par][k - 1];
      rl.dst[rl.n] = G[np][k - 1];
      rl.bytes[rl.n] = core_elems(k) * (long long)sizeof(TC);
      ++rl.n;
    }
    rl.src[rl.n] = C[par];
    rl.dst[rl.n] = C[np];
    rl.bytes[rl.n] = full[kstar - 1] * rest[kstar - 1] * (long long)sizeof(TC);
    ++rl.n;
    bool first_launch = true;
    for (int k = kstar - 2; k >= 1; --k) {
      const bool fromC = (k == kstar - 2);
      const TC* Bsrc = fromC ? C[par] : Bhat[k + 1];
      GemmShape g = plan_gemm(rows(k + 1), (int)rest[k + 1], rk(k + 1), false);
      TT_TRY((gemm<TC, TC, TC, TC, true, false>(g, G[par][k], rk(k + 1), Bsrc, rest[k + 1], Bhat[k], rest[k + 1],
                                                 1, 0, nullptr, fromC ? &ctl->cc : nullptr, nullptr,
                                                 first_launch ? ctl : nullptr, s)));
      first_launch = false;
    }
    int ncc = 0;
    int mc = 0;                                  // gM[mc] = A_k^T A_k (noortho); A_1 = 1
    for (int k = 1; k < kstar; ++k) {
      const bool last_level = (k == kstar - 1);
      const TC* Bk = last_level ? C[par] : Bhat[k];
      const double* bz = last_level ? &ctl->cc : nullptr;
      const int r0 = (int)full[k - 1], r1 = rk(k);
      const long long n = rows(k);
      GemmShape gs = plan_solve(k);
      if (k == 1) {
        TT_TRY(solve_level1(gs, X, Bk, bz, first_launch ? ctl : nullptr, s));
        if (!ortho) {                           // (lsq: the first orth pass sums it)
          k_sum_xx<<<1, 256, 0, s>>>(sumsq, (int)sumsq_elems, ctl);
          TT_CUDA(cudaGetLastError());
          ++nlaunch;
        }
      } else {
        TT_TRY((gemm<TC, TC, TC, TC, true, true>(gs, E[k], rest[k], Bk, rest[k], part, r1, 1,
                                                 (long long)gs.M * gs.N, nullptr, bz, ctl, nullptr, s)));
      }
      first_launch = false;
      // Y = the reduced local solve E_k B^_k^T, (r_{k-1} I_k) x r_k
      {
        const int nb = (int)std::min<long long>(cdiv(n * r1, 256), 4 * kSMs);
        k_reduce_rows<TC><<<nb, 256, 0, s>>>(part, gs.nsplit, n * r1, Y, ctl);
        TT_CUDA(cudaGetLastError());
        ++nlaunch;
      }
      // Y <- Y (B^_k B^_k^T)^-1 (the right Gram, with the zero-row rule of the literal path)
      TT_TRY((gemm<TC, TC, TC, TC, true, true>(plan_gemm(r1, r1, rest[k], false), Bk, rest[k], Bk, rest[k], gBB, r1,
                                               1, 0, nullptr, nullptr, ctl, nullptr, s)));
      TT_TRY(spd_solve(gBB, r1, Y, n, r1, 1, s));
      TC* qdst = G[np][k - 1];
      if (ortho) {
        TT_TRY(orth(k, 1, k == 1, qdst, s, Y));
      } else {
        // G_k = (A_k^T A_k)^-1 acting on the r_{k-1} index of Y: the columns of Y seen as an
        // r_{k-1} x (I_k r_k) matrix
        if (k > 1) TT_TRY(spd_solve(gM[mc], r0, Y, (long long)dims[k - 1] * r1, 1, (long long)dims[k - 1] * r1, s));
        TT_CUDA(cudaMemcpyAsync(qdst, Y, (size_t)(n * r1) * sizeof(TC), cudaMemcpyDeviceToDevice, s));
      }
      // environment E_{k+1} = G_k^T E_k (unweighted for noortho)
      GemmShape ge = plan_env(k);
      if (k == 1) {
        TT_TRY(env_level1(ge, X, qdst, s));
      } else {
        TT_TRY((gemm<TC, TC, TC, TC, false, false>(ge, E[k], rest[k], qdst, r1, part, r1, 1,
                                                   (long long)ge.M * ge.N, nullptr, nullptr, ctl, nullptr, s)));
      }
      TC* eout = last_level ? C[np] : E[k + 1];
      const int nbr = (int)std::min<long long>(cdiv(rest[k] * r1, RED_THREADS), 4 * kSMs);
      k_reduce_t<TC><<<nbr, RED_THREADS, 0, s>>>(part, ge.nsplit, (long long)ge.M * ge.N, rest[k], r1, eout,
                                                 (last_level && ortho) ? ccpart : nullptr, ctl);
      TT_CUDA(cudaGetLastError());
      ++nlaunch;
      if (last_level && ortho) ncc = nbr;
      if (!ortho) {
        // A_{k+1}^T A_{k+1} = G_k^T (A_k^T A_k (x) I) G_k
        const int mn = 1 - mc;
        if (k == 1) {
          TT_TRY((gemm<TC, TC, TC, TC, false, false>(plan_gemm(r1, r1, n, false), qdst, r1, qdst, r1, gM[mn], r1, 1,
                                                     0, nullptr, nullptr, ctl, nullptr, s)));
        } else {
          const long long w = (long long)dims[k - 1] * r1;     // H = M_k G_k (r_{k-1} x I_k r_k) in Qa
          TT_TRY((gemm<TC, TC, TC, TC, true, false>(plan_gemm(r0, (int)w, r0, false), gM[mc], r0, qdst, w, Qa, w, 1,
                                                    0, nullptr, nullptr, ctl, nullptr, s)));
          TT_TRY((gemm<TC, TC, TC, TC, false, false>(plan_gemm(r1, r1, n, false), qdst, r1, Qa, r1, gM[mn], r1, 1, 0,
                                                     nullptr, nullptr, ctl, nullptr, s)));
        }
        mc = mn;
        if (last_level) {
          // C = (A_k*^T A_k*)^-1 E~ on the columns of the r_{k*-1} x rest matrix; ||x^||^2 = <E~, C>
          const long long csz = (long long)r1 * rest[k];
          TT_CUDA(cudaMemcpyAsync(gEt, eout, (size_t)csz * sizeof(TC), cudaMemcpyDeviceToDevice, s));
          TT_TRY(spd_solve(gM[mc], r1, eout, rest[k], 1, rest[k], s));
          ncc = (int)std::min<long long>(cdiv(csz, 256), (long long)kSMs);
          k_dot_part<TC><<<ncc, 256, 0, s>>>(gEt, eout, csz, ccpart, ctl);
          TT_CUDA(cudaGetLastError());
          ++nlaunch;
        }
      }
    }
    k_commit<<<1, 256, 0, s>>>(ctl, ccpart, ncc, nullptr, 0, rl);
    TT_CUDA(cudaGetLastError());
    ++nlaunch;
    par = np;
    return TTALS_OK;
  }

  // level-1 local solve Y = X_(1) B^_1^T (split-K partials into `part`, ||x||^2 partials)
  ttals_status solve_level1(const GemmShape& gs, const TX* X, const TC* Bk, const double* bzero, Ctl* reset,
                            cudaStream_t s) {
    return gemm<TX, TC, TC, TC, true, true>(gs, X, rest[1], Bk, rest[1], part, rk(1), 1,
                                           (long long)gs.M * gs.N, sumsq, bzero, nullptr, reset, s);
  }
  // level-1 environment E_2^T = X_(1)^T G_1 (split partials into `part`)
  ttals_status env_level1(const GemmShape& ge, const TX* X, const TC* Q, cudaStream_t s) {
    return gemm<TX, TC, TC, TC, false, false>(ge, X, rest[1], Q, rk(1), part, rk(1), 1, (long long)ge.M * ge.N,
                                             nullptr, nullptr, ctl, nullptr, s);
  }

  // ---- x^_t = G_1 x ... x G_{k*-1} x C ------------------------------------------
  ttals_status reconstruct(void* out, ttals_dtype dt, cudaStream_t s) override {
    switch (dt) {
      case TTALS_F64: return recon_t<double>((double*)out, s);
      case TTALS_F32: return recon_t<float>((float*)out, s);
      case TTALS_F16: return recon_t<__half>((__half*)out, s);
      case TTALS_BF16: return recon_t<__nv_bfloat16>((__nv_bfloat16*)out, s);
    }
    return TTALS_EINVAL;
  }
  template <typename TO>
  ttals_status recon_t(TO* out, cudaStream_t s) {
    TT_TRY(finalize(s));
    if (kstar == 1) {
      const int nb = (int)std::min<long long>(cdiv(rest[0], 256), 4 * kSMs);
      k_convert<TC, TO><<<nb, 256, 0, s>>>(C[par], out, rest[0]);
      TT_CUDA(cudaGetLastError());
      return TTALS_OK;
    }
    const TC* T = C[par];
    for (int k = kstar - 1; k >= 1; --k) {
      GemmShape g = plan_gemm(rows(k), (int)rest[k], rk(k), false);
      if (k == 1) {
        TT_TRY((gemm<TC, TC, TC, TO, true, false>(g, G[par][0], rk(1), T, rest[1], out, rest[1], 1, 0, nullptr,
                                                  nullptr, nullptr, nullptr, s)));
      } else {
        TC* dst = Bhat[k - 1];
        TT_TRY((gemm<TC, TC, TC, TC, true, false>(g, G[par][k - 1], rk(k), T, rest[k], dst, rest[k], 1, 0, nullptr,
                                                  nullptr, nullptr, nullptr, s)));
        T = dst;
      }
    }
    return TTALS_OK;
  }

  // ---- initial state / resume ---------------------------------------------------
  ttals_status set_cores(const double* const* cores, const double* g, long long t) override {
    cudaStream_t s = have_last ? last : (cudaStream_t)0;
    TT_CUDA(cudaStreamSynchronize(s));
    std::vector<double*> dc(m + 1);
    size_t off = 0;
    for (int k = 1; k <= m; ++k) {
      dc[k] = dcores + off;
      TT_CUDA(cudaMemcpy(dc[k], cores[k - 1], (size_t)core_elems(k) * 8, cudaMemcpyHostToDevice));
      off += (size_t)core_elems(k);
    }
    double* dg = dcores + off;
    TT_CUDA(cudaMemcpy(dg, g, (size_t)full[m] * 8, cudaMemcpyHostToDevice));
    // C = G_{k*} x ... x G_m x g_n, FP64 chain from the right
    const double* T = dg;
    int pp = 0;
    for (int k = m; k >= kstar; --k) {
      GemmShape gg = plan_gemm(rows(k), (int)rest[k], rk(k), false);
      double* dst = dtmp[pp];
      TT_TRY((gemm<double, double, double, double, true, false>(gg, dc[k], rk(k), T, rest[k], dst, rest[k], 1, 0,
                                                                nullptr, nullptr, nullptr, nullptr, s)));
      T = dst;
      pp ^= 1;
    }
    const long long csz = full[kstar - 1] * rest[kstar - 1];
    const int nb = (int)std::min<long long>(cdiv(csz, 256), 4 * kSMs);
    k_convert<double, TC><<<nb, 256, 0, s>>>(T, C[par], csz);
    TT_CUDA(cudaGetLastError());
    for (int k = 1; k < kstar; ++k) {
      const int nb2 = (int)std::min<long long>(cdiv(core_elems(k), 256), 4 * kSMs);
      k_convert<double, TC><<<nb2, 256, 0, s>>>(dc[k], G[par][k - 1], core_elems(k));
      TT_CUDA(cudaGetLastError());
    }
    Ctl h{};
    h.t = t;
    TT_CUDA(cudaMemcpy(ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice));
    k_norm2_to_cc<TC><<<1, 1024, 0, s>>>(C[par], csz, ctl);
    TT_CUDA(cudaGetLastError());
    TT_TRY(sync_fast_from_generic(s));
    TT_CUDA(cudaStreamSynchronize(s));
    materialised = false;
    return TTALS_OK;
  }

  // ---- readout --------------------------------------------------------------------
  ttals_status materialise(cudaStream_t s) {
    // left-orthogonal TT of C with completion: for k = k*..m, Householder QR of the
    // (r_{k-1} I_k) x rest_k unfolding, completed to r_k columns; then E_{k+1} = Q^T E_k.
    const long long csz = full[kstar - 1] * rest[kstar - 1];
    const int nb = (int)std::min<long long>(cdiv(csz, 256), 4 * kSMs);
    k_convert<TC, double><<<nb, 256, 0, s>>>(C[par], dtmp[0], csz);
    TT_CUDA(cudaGetLastError());
    double* Ek = dtmp[0];
    int pp = 1;
    for (int k = kstar; k <= m; ++k) {
      const long long nr = rows(k);
      const int p = (int)rest[k];
      const int ro = rk(k);
      k_householder<double, double><<<1, HH_THREADS, 0, s>>>(Ek, nr, p, ro, hh, mat_q[k], ro);
      TT_CUDA(cudaGetLastError());
      // E_{k+1}[a][j] = sum_i Q[i][a] E_k[i][j]   (ro x p)
      double* dst = (k == m) ? mat_g : dtmp[pp];
      GemmShape gg = plan_gemm(ro, p, nr, false);
      TT_TRY((gemm<double, double, double, double, false, false>(gg, mat_q[k], ro, Ek, p, dst, p, 1, 0, nullptr,
                                                                 nullptr, nullptr, nullptr, s)));
      Ek = dst;
      pp ^= 1;
    }
    materialised = true;
    return TTALS_OK;
  }

  ttals_status get_core(int k, double* host, size_t n) override {
    cudaStream_t s = have_last ? last : (cudaStream_t)0;
    TT_TRY(finalize(s));
    if (k >= kstar && !materialised) TT_TRY(materialise(s));
    if (k < kstar) {
      const long long ne = core_elems(k);
      const int nb = (int)std::min<long long>(cdiv(ne, 256), 4 * kSMs);
      k_convert<TC, double><<<nb, 256, 0, s>>>(G[par][k - 1], dout, ne);
      TT_CUDA(cudaGetLastError());
      TT_CUDA(cudaMemcpyAsync(host, dout, n * 8, cudaMemcpyDeviceToHost, s));
    } else if (k <= m) {
      TT_CUDA(cudaMemcpyAsync(host, mat_q[k], n * 8, cudaMemcpyDeviceToHost, s));
    } else {
      TT_CUDA(cudaMemcpyAsync(host, mat_g, n * 8, cudaMemcpyDeviceToHost, s));
    }
    TT_CUDA(cudaStreamSynchronize(s));
    return TTALS_OK;
  }
};

ttals_stream* make_impl(ttals_dtype ingest) {
  switch (ingest) {
    case TTALS_F64: return new Impl<double, double>();
    case TTALS_F32: return new Impl<float, float>();
    case TTALS_F16: return new Impl<__half, float>();
    case TTALS_BF16: return new Impl<__nv_bfloat16, float>();
  }
  return nullptr;
}

ttals_status set_device(int dev) {
  int cur = -1;
  TT_CUDA(cudaGetDevice(&cur));
  if (cur != dev) TT_CUDA(cudaSetDevice(dev));
  return TTALS_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free slice error: ||x||^2 and ||x - y||^2 of two device arrays.
// For callers that cannot allocate device memory at the point of the call: a
// serving loop that checks accuracy between pushes on a stream it must not stall
// (cudaMalloc and cudaFree synchronise the device) or a process whose device memory
// is fully reserved by its own pool.  Its scratch (per-CTA partial sums and a
// completion ticket) is the static device array below, not memory of a stream.
// ---------------------------------------------------------------------------
constexpr int kErrThreads = 256;
constexpr long long kErrPerCta = 16384;           // elements per CTA
constexpr int kErrMaxCtas = 4096;                 // => at most 4096 * 16384 = 2^26 elements
constexpr size_t kErrPartBytes = (size_t)kErrMaxCtas * 2 * sizeof(double);
// [0, kErrPartBytes): partials (||x||^2, ||x-y||^2) per CTA; then the ticket counter,
// which must be zero when a call starts (each call clears it on its stream first)
static __device__ __align__(256) unsigned char g_err_scratch[kErrPartBytes + 256];

// device address of g_err_scratch, resolved once per device with that device current
constexpr int kErrMaxDevices = 64;
void* g_err_scratch_addr[kErrMaxDevices] = {};
std::mutex g_err_scratch_mu;

ttals_status err_scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  TT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kErrMaxDevices) {
    g_last_err = "ttals_slice_error_noalloc: device ordinal out of range";
    return TTALS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_err_scratch_mu);
  if (!g_err_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_err_scratch);
    if (e != cudaSuccess || !p) {
      g_last_err = std::string("cudaGetSymbolAddress(g_err_scratch): ") + cudaGetErrorString(e);
      cudaGetLastError();
      return TTALS_ECUDA;
    }
    g_err_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_err_scratch_addr[dev];
  return TTALS_OK;
}

// one CTA per kErrPerCta elements: FP64 sums in a fixed order, partials in the static
// scratch, the last CTA (ticket) sums them in CTA order and resets the ticket
template <typename TA, typename TB>
__global__ void __launch_bounds__(kErrThreads) k_slice_error_noalloc(const TA* __restrict__ x,
                                                                     const TB* __restrict__ y, long long n,
                                                                     double* part, unsigned* ticket,
                                                                     double* out) {
  __shared__ double red[32];
  __shared__ int last;
  const long long b0 = (long long)blockIdx.x * kErrPerCta;
  const long long b1 = (b0 + kErrPerCta < n) ? b0 + kErrPerCta : n;
  double sx = 0.0, se = 0.0;
  for (long long i = b0 + threadIdx.x; i < b1; i += kErrThreads) {
    const double a = Cvt<TA>::d(x[i]), d = a - Cvt<TB>::d(y[i]);
    sx = fma(a, a, sx);
    se = fma(d, d, se);
  }
  sx = block_sum(sx, red);
  se = block_sum(se, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sx;
    part[2 * blockIdx.x + 1] = se;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tx = 0.0, te = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kErrThreads) {
    tx += __ldcg(part + 2 * b);
    te += __ldcg(part + 2 * b + 1);
  }
  tx = block_sum(tx, red);
  te = block_sum(te, red);
  if (threadIdx.x == 0) {
    out[0] = tx;
    out[1] = te;
    *ticket = 0u;
  }
}

template <typename TA>
ttals_status launch_slice_error(const TA* x, const void* y, ttals_dtype yt, long long n, double* part,
                                unsigned* ticket, double* out, cudaStream_t st) {
  const unsigned grid = (unsigned)cdiv(n, kErrPerCta);
  if (yt == TTALS_F64)
    k_slice_error_noalloc<TA, double><<<grid, kErrThreads, 0, st>>>(x, (const double*)y, n, part, ticket, out);
  else
    k_slice_error_noalloc<TA, float><<<grid, kErrThreads, 0, st>>>(x, (const float*)y, n, part, ticket, out);
  TT_CUDA(cudaGetLastError());
  return TTALS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* ttals_status_string(ttals_status st) {
  switch (st) {
    case TTALS_OK: return "ok";
    case TTALS_EINVAL: return "invalid argument";
    case TTALS_ENOMEM: return "out of device memory";
    case TTALS_ECUDA: return "CUDA error";
    case TTALS_ENONFINITE: return "non-finite slice (not committed)";
    case TTALS_ETIMEOUT: return "device wait timed out";
    case TTALS_ESTATE: return "invalid state";
  }
  return "unknown status";
}

const char* ttals_last_error(void) { return g_last_err.c_str(); }

// the selected stream's state <- the next draw of the default initial cores ("Initialize
// orthogonal cores randomly", Algorithm 1): Gaussian entries in core order, then g_n; the
// push re-orthogonalises them (Sec. 3.4.1), so they need not be orthogonal here
static ttals_status set_default_cores(ttals_stream* s, SplitMix64& rng) {
  const int m = s->m;
  std::vector<std::vector<double>> cores(m);
  std::vector<const double*> ptrs(m);
  std::vector<double> g((size_t)s->full[m]);
  for (int k = 1; k <= m; ++k) {
    cores[k - 1].resize((size_t)s->core_elems(k));
    for (double& v : cores[k - 1]) v = rng.gauss();
    ptrs[k - 1] = cores[k - 1].data();
  }
  for (double& v : g) v = rng.gauss();
  return s->set_cores(ptrs.data(), g.data(), 0);
}

// one stream (nbatch = 1) or a batch of nbatch streams of one shape that share launches
static ttals_status create_streams(int nbatch, int n_slice_modes, const int64_t* dims, const int64_t* ranks,
                                   const ttals_config* cfg, ttals_stream** out) {
  if (!out) return TTALS_EINVAL;
  *out = nullptr;
  if (n_slice_modes < 2 || n_slice_modes > kMaxLevels || !dims || !ranks) return TTALS_EINVAL;
  ttals_config c{};
  c.ingest = TTALS_F64;
  c.seed = 0x5eedull;
  c.device = 0;
  if (cfg) {
    c = *cfg;
    if (c.factor != 0 && c.factor != 1) return TTALS_EINVAL;
    if (c.mode < 0 || c.mode > 2) return TTALS_EINVAL;
    if (c.env_kernel < 0 || c.env_kernel > 4) return TTALS_EINVAL;
    if (c.k1_split != 0 && c.k1_split != 1 && c.k1_split != 2 && c.k1_split != 4 && c.k1_split != 8)
      return TTALS_EINVAL;
    if (c.solve_kernel < 0 || c.solve_kernel > 2) return TTALS_EINVAL;
    if (c.factor_cluster != 0 && c.factor_cluster != 4 && c.factor_cluster != 8) return TTALS_EINVAL;
    if (c.seed == 0) c.seed = 0x5eedull;
  }
  if (c.ingest < TTALS_F64 || c.ingest > TTALS_BF16) return TTALS_EINVAL;
  if (c.qr_passes < 0 || c.qr_passes > 2) return TTALS_EINVAL;
  const int m = n_slice_modes;
  std::vector<long long> d(m), r(m);
  long long total = 1;
  for (int i = 0; i < m; ++i) {
    if (dims[i] < 1 || ranks[i] < 1) return TTALS_EINVAL;
    d[i] = dims[i];
    r[i] = ranks[i];
    if (total > (1ll << 40) / d[i]) return TTALS_EINVAL;
    total *= d[i];
  }
  // feasible ranks: r_k <= r_{k-1} I_k and r_k <= I_{k+1} r_{k+1}, to a fixed point
  for (;;) {
    std::vector<long long> old = r;
    long long prev = 1;
    for (int k = 0; k < m; ++k) {
      r[k] = std::min(r[k], prev * d[k]);
      prev = r[k];
    }
    for (int k = m - 2; k >= 0; --k) r[k] = std::min(r[k], d[k + 1] * r[k + 1]);
    if (r == old) break;
  }
  for (int k = 0; k < m; ++k)
    if (r[k] > kMaxRank) return TTALS_EINVAL;
  if (set_device(c.device) != TTALS_OK) return TTALS_ECUDA;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device >= ndev) {
    cudaGetLastError();
    g_last_err = "no CUDA device";
    return TTALS_ECUDA;
  }
  ttals_stream* s = make_impl(c.ingest);
  {
    const char* e = std::getenv("TTALS_NO_PDL");
    s->no_pdl = e && e[0] == '1';
  }
  s->m = m;
  s->dims = d;
  s->full.assign(m + 1, 1);
  for (int k = 0; k < m; ++k) s->full[k + 1] = r[k];
  s->rest.assign(m + 1, 1);
  for (int k = m - 1; k >= 0; --k) s->rest[k] = s->rest[k + 1] * d[k];
  s->kstar = m;
  for (int k = 1; k <= m; ++k)
    if (s->full[k] >= s->rest[k]) { s->kstar = k; break; }
  s->ingest = c.ingest;
  s->device = c.device;
  s->qr_passes = c.qr_passes ? c.qr_passes : 2;
  s->nbatch = nbatch;
  s->cfg_env_kernel = c.env_kernel;
  s->cfg_k1_split = c.k1_split;
  s->cfg_solve_kernel = c.solve_kernel;
  s->cfg_factor_cluster = c.factor_cluster;
  s->cfg_factor = c.factor;
  s->mode = c.mode;
  if (cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess) {
    delete s;
    return TTALS_ECUDA;
  }
  ttals_status st = s->allocate();
  if (st == TTALS_OK && nbatch > 1 && !s->batch_capable()) {
    g_last_err = "batches need the fused path: FP16/BF16 ingest, a saturated second level, r_1 <= 64, "
                 "I_2...I_{n-1} a multiple of 8";
    st = TTALS_EINVAL;
  }
  if (st != TTALS_OK) {
    delete s;
    return st;
  }
  // default initial cores: Gaussian (SplitMix64 + Box-Muller), one draw per stream of a batch
  SplitMix64 rng{c.seed};
  for (int b = 0; b < nbatch && st == TTALS_OK; ++b) {
    st = s->select_slot(b);
    if (st == TTALS_OK) st = set_default_cores(s, rng);
  }
  if (st == TTALS_OK) st = s->select_slot(0);
  if (st != TTALS_OK) {
    delete s;
    return st;
  }
  *out = s;
  return TTALS_OK;
}

ttals_status ttals_create(int n_slice_modes, const int64_t* dims, const int64_t* ranks, const ttals_config* cfg,
                          ttals_stream** out) {
  return create_streams(1, n_slice_modes, dims, ranks, cfg, out);
}

ttals_status ttals_create_batch(int n_streams, int n_slice_modes, const int64_t* dims, const int64_t* ranks,
                                const ttals_config* cfg, ttals_stream** out) {
  if (out) *out = nullptr;
  if (n_streams < 1 || n_streams > TTALS_MAX_BATCH) return TTALS_EINVAL;
  return create_streams(n_streams, n_slice_modes, dims, ranks, cfg, out);
}

ttals_status ttals_push_batch(ttals_stream* s, const void* slices_dev, ttals_dtype dtype, void* cuda_stream) {
  if (!s || !slices_dev) return TTALS_EINVAL;
  if (dtype != s->ingest) return TTALS_EINVAL;
  if (((uintptr_t)slices_dev & 15u) != 0) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TT_TRY(s->order_after_last(st));
  return s->push(slices_dev, st);
}

ttals_status ttals_push_batch_masked(ttals_stream* s, const void* slices_dev, ttals_dtype dtype,
                                     uint64_t active_mask, void* cuda_stream) {
  if (!s || !slices_dev) return TTALS_EINVAL;
  if (dtype != s->ingest) return TTALS_EINVAL;
  if (((uintptr_t)slices_dev & 15u) != 0) return TTALS_EINVAL;
  const unsigned long long all = s->nbatch >= 64 ? ~0ull : ((1ull << s->nbatch) - 1ull);
  const unsigned long long m = (unsigned long long)active_mask & all;
  if (m == 0) return TTALS_OK;
  TT_TRY(set_device(s->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TT_TRY(s->order_after_last(st));
  s->active_mask = m;
  const ttals_status r = s->push(slices_dev, st);
  s->active_mask = ~0ull;
  return r;
}

ttals_status ttals_batch_ingest_init(ttals_stream* s, int u8_wire) {
  if (!s || (u8_wire != 0 && u8_wire != 1)) return TTALS_EINVAL;
  if (s->ingest != TTALS_F16 && s->ingest != TTALS_BF16 && s->ingest != TTALS_F32) return TTALS_EINVAL;
  if (s->hi.on) return TTALS_ESTATE;
  TT_TRY(set_device(s->device));
  auto& h = s->hi;
  const size_t n = (size_t)s->nbatch * (size_t)s->slice_elems();
  for (int p = 0; p < 2; ++p) {
    if (s->ingest == TTALS_F32) {
      float* b = nullptr;
      TT_TRY(s->dalloc(&b, n));
      h.block[p] = b;
    } else {
      __half* b = nullptr;
      TT_TRY(s->dalloc(&b, n));
      h.block[p] = b;
    }
    if (u8_wire) {
      uint8_t* st = nullptr;
      TT_TRY(s->dalloc(&st, n + 16));
      h.stage[p] = st;
    }
  }
  int lo = 0, hiprio = 0;
  TT_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hiprio));
  // copies (and the widening) at high priority: queued behind other batches' compute they
  // would leave the host link idle
  TT_CUDA(cudaStreamCreateWithPriority(&h.copy, cudaStreamNonBlocking, hiprio));
  TT_CUDA(cudaStreamCreateWithPriority(&h.comp, cudaStreamNonBlocking, lo));
  for (int p = 0; p < 2; ++p) {
    TT_CUDA(cudaEventCreateWithFlags(&h.copied[p], cudaEventDisableTiming));
    TT_CUDA(cudaEventCreateWithFlags(&h.consumed[p], cudaEventDisableTiming));
    TT_CUDA(cudaEventRecord(h.consumed[p], h.comp));
  }
  h.done.resize(ttals_stream::kTicketRing, nullptr);
  for (auto& e : h.done) TT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  h.u8 = u8_wire != 0;
  // the blocks' TMA maps now, not in the first served steps
  for (int p = 0; p < 2; ++p) TT_TRY(s->warm_slice(h.block[p]));
  h.on = true;
  return TTALS_OK;
}

ttals_status ttals_batch_push_host(ttals_stream* s, int n, const int* slots, const void* const* host_frames,
                                   uint64_t* ticket_out) {
  if (!s || !s->hi.on || n < 0 || n > s->nbatch || (n > 0 && (!slots || !host_frames)) || !ticket_out)
    return TTALS_EINVAL;
  unsigned long long mask = 0;
  for (int i = 0; i < n; ++i) {
    if (slots[i] < 0 || slots[i] >= s->nbatch || !host_frames[i]) return TTALS_EINVAL;
    if ((mask >> slots[i]) & 1ull) return TTALS_EINVAL;      // one frame per stream and step
    mask |= 1ull << slots[i];
  }
  if (n == 0) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  auto& h = s->hi;
  const int p = h.flip;
  const size_t elems = (size_t)s->slice_elems();
  const size_t esz = dtype_size(s->ingest);
  TT_CUDA(cudaStreamWaitEvent(h.copy, h.consumed[p], 0));   // the block's previous step is done with it
  for (int i = 0; i < n; ++i) {
    if (h.u8) {
      TT_CUDA(cudaMemcpyAsync((uint8_t*)h.stage[p] + (size_t)slots[i] * elems, host_frames[i], elems,
                              cudaMemcpyHostToDevice, h.copy));
    } else {
      TT_CUDA(cudaMemcpyAsync((unsigned char*)h.block[p] + (size_t)slots[i] * elems * esz, host_frames[i],
                              elems * esz, cudaMemcpyHostToDevice, h.copy));
    }
  }
  if (h.u8) {
    // one widening launch for the block (slots without a frame are widened too and not read)
    TT_TRY(ttals_widen_u8(h.stage[p], h.block[p], s->ingest, (int64_t)((size_t)s->nbatch * elems), h.copy));
  }
  TT_CUDA(cudaEventRecord(h.copied[p], h.copy));
  TT_CUDA(cudaStreamWaitEvent(h.comp, h.copied[p], 0));
  TT_TRY(ttals_push_batch_masked(s, h.block[p], s->ingest, mask, h.comp));
  TT_CUDA(cudaEventRecord(h.consumed[p], h.comp));
  TT_CUDA(cudaEventRecord(h.done[h.ticket % ttals_stream::kTicketRing], h.comp));
  *ticket_out = h.ticket++;
  h.flip ^= 1;
  return TTALS_OK;
}

ttals_status ttals_batch_ticket_done(ttals_stream* s, uint64_t ticket, int* done) {
  if (!s || !s->hi.on || !done || ticket >= s->hi.ticket) return TTALS_EINVAL;
  const cudaError_t e = cudaEventQuery(s->hi.done[ticket % ttals_stream::kTicketRing]);
  if (e == cudaSuccess) {
    *done = 1;
  } else if (e == cudaErrorNotReady) {
    *done = 0;
  } else {
    g_last_err = std::string("cudaEventQuery: ") + cudaGetErrorString(e);
    return TTALS_ECUDA;
  }
  return TTALS_OK;
}

ttals_status ttals_batch_select(ttals_stream* s, int index) {
  if (!s || index < 0 || index >= s->nbatch) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  if (s->have_last) TT_CUDA(cudaStreamSynchronize(s->last));
  return s->select_slot(index);
}

int ttals_batch_size(const ttals_stream* s) { return s ? s->nbatch : 0; }

void ttals_destroy(ttals_stream* s) {
  if (!s) return;
  set_device(s->device);
  delete s;
}

ttals_status ttals_effective_ranks(const ttals_stream* s, int64_t* ranks_out) {
  if (!s || !ranks_out) return TTALS_EINVAL;
  for (int k = 0; k < s->m; ++k) ranks_out[k] = s->full[k + 1];
  return TTALS_OK;
}

ttals_status ttals_set_cores(ttals_stream* s, const double* const* cores, const double* g, int64_t t) {
  if (!s || !cores || !g || t < 0) return TTALS_EINVAL;
  for (int k = 0; k < s->m; ++k)
    if (!cores[k]) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  return s->set_cores(cores, g, t);
}

ttals_status ttals_seed_cores(ttals_stream* s, uint64_t seed) {
  if (!s) return TTALS_EINVAL;
  SplitMix64 rng{seed ? seed : 0x5eedull};
  return set_default_cores(s, rng);
}

ttals_status ttals_push_slice(ttals_stream* s, const void* slice_dev, ttals_dtype dtype, void* cuda_stream) {
  if (!s || !slice_dev) return TTALS_EINVAL;
  if (s->nbatch != 1) return TTALS_ESTATE;          // a batch steps through ttals_push_batch
  if (dtype != s->ingest) return TTALS_EINVAL;
  if (((uintptr_t)slice_dev & 15u) != 0) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TT_TRY(s->order_after_last(st));
  return s->push(slice_dev, st);
}

ttals_status ttals_reconstruct(ttals_stream* s, void* out_dev, ttals_dtype out_dtype, void* cuda_stream) {
  if (!s || !out_dev) return TTALS_EINVAL;
  if (out_dtype < TTALS_F64 || out_dtype > TTALS_BF16) return TTALS_EINVAL;
  if (((uintptr_t)out_dev & (dtype_size(out_dtype) - 1)) != 0) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TT_TRY(s->order_after_last(st));
  return s->reconstruct(out_dev, out_dtype, st);
}

ttals_status ttals_cores(ttals_stream* s, int k, double* host_out, size_t n_elems) {
  if (!s || !host_out || k < 1 || k > s->m + 1) return TTALS_EINVAL;
  const size_t want = (k <= s->m) ? (size_t)s->core_elems(k) : (size_t)s->full[s->m];
  if (n_elems != want) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  TT_TRY(s->get_core(k, host_out, n_elems));
  Ctl h;
  TT_TRY(s->sync_and_read(&h, true));
  return h.latched ? (ttals_status)h.latched : TTALS_OK;
}

ttals_status ttals_stats(ttals_stream* s, double out[4]) {
  if (!s || !out) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  Ctl h;
  TT_TRY(s->sync_and_read(&h, true));
  out[0] = h.xx;
  out[1] = h.ee;
  out[2] = h.sum_xx;
  out[3] = h.sum_ee;
  return h.latched ? (ttals_status)h.latched : TTALS_OK;
}

ttals_status ttals_step(ttals_stream* s, int64_t* t_out) {
  if (!s || !t_out) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  Ctl h;
  TT_TRY(s->sync_and_read(&h, true));
  *t_out = h.t;
  return h.latched ? (ttals_status)h.latched : TTALS_OK;
}

ttals_status ttals_sync(ttals_stream* s) {
  if (!s) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  Ctl h;
  TT_TRY(s->sync_and_read(&h, true));
  return h.latched ? (ttals_status)h.latched : TTALS_OK;
}

size_t ttals_device_bytes(const ttals_stream* s) { return s ? s->bytes : 0; }

#ifdef TTALS_TRACE
// phase timestamps of the last traced launches (builds with -DTTALS_TRACE only)
int ttals_debug_trace(unsigned long long* out, int n) {
  if (n > 128) n = 128;
  return cudaMemcpyFromSymbol(out, ttals::g_ttals_trace, (size_t)n * 8) == cudaSuccess ? 0 : 3;
}
int ttals_debug_trace_cta(unsigned long long* out, int n) {
  if (n > 4096) n = 4096;
  return cudaMemcpyFromSymbol(out, ttals::g_ttals_cta, (size_t)n * 8) == cudaSuccess ? 0 : 3;
}
#endif

uint64_t ttals_launch_count(const ttals_stream* s) { return s ? (uint64_t)s->nlaunch : 0; }

ttals_status ttals_debug_stall_solve(ttals_stream* s, int n_pushes) {
  if (!s || n_pushes < 0) return TTALS_EINVAL;
  s->stall_pushes = n_pushes;
  return TTALS_OK;
}

ttals_status ttals_stats_async(ttals_stream* s, double* out4, void* cuda_stream) {
  if (!s || !out4) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TT_TRY(s->order_after_last(st));
  TT_CUDA(cudaMemcpyAsync(out4, &s->ctl->xx, 4 * sizeof(double), cudaMemcpyDefault, st));
  return TTALS_OK;
}

ttals_status ttals_profile(ttals_stream* s, int enable) {
  if (!s) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  if (s->have_last) TT_CUDA(cudaStreamSynchronize(s->last));
  s->profiling = enable != 0;
  s->ev_used = 0;
  return TTALS_OK;
}

ttals_status ttals_profile_read(ttals_stream* s, double ms_out[4], int64_t* n_out) {
  if (!s || !ms_out || !n_out) return TTALS_EINVAL;
  TT_TRY(set_device(s->device));
  if (s->have_last) TT_CUDA(cudaStreamSynchronize(s->last));
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const size_t npush = s->ev_used / ttals_stream::kProfEvents;
  for (size_t i = 0; i < npush; ++i) {
    cudaEvent_t* e = &s->ev_pool[i * ttals_stream::kProfEvents];
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    if (s->kstar > 1) {
      TT_CUDA(cudaEventElapsedTime(&t[0], e[1], e[2]));
      TT_CUDA(cudaEventElapsedTime(&t[1], e[2], e[3]));
      TT_CUDA(cudaEventElapsedTime(&t[2], e[3], e[4]));
    }
    TT_CUDA(cudaEventElapsedTime(&t[3], e[0], e[5]));
    for (int q = 0; q < 4; ++q) acc[q] += t[q];
  }
  for (int i = 0; i < 4; ++i) ms_out[i] = acc[i];
  *n_out = (int64_t)npush;
  s->ev_used = 0;
  return TTALS_OK;
}

ttals_status ttals_widen_u8(const void* src_dev, void* dst_dev, ttals_dtype dst_dtype, int64_t n,
                            void* cuda_stream) {
  if (!src_dev || !dst_dev || n < 0) return TTALS_EINVAL;
  if (dst_dtype != TTALS_F16 && dst_dtype != TTALS_BF16 && dst_dtype != TTALS_F32 && dst_dtype != TTALS_F64)
    return TTALS_EINVAL;
  if (((uintptr_t)src_dev & 15u) != 0 || ((uintptr_t)dst_dev & 15u) != 0) return TTALS_EINVAL;
  if (n == 0) return TTALS_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const long long n16 = (n + 15) / 16;
  int dev = 0;
  TT_CUDA(cudaGetDevice(&dev));
  int nsm = 0;
  TT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int nb = (int)std::min<long long>((n16 + 255) / 256, 8LL * nsm);
  switch (dst_dtype) {
    case TTALS_F16: k_widen_u8<__half><<<nb, 256, 0, st>>>((const uint8_t*)src_dev, (__half*)dst_dev, n); break;
    case TTALS_BF16:
      k_widen_u8<__nv_bfloat16><<<nb, 256, 0, st>>>((const uint8_t*)src_dev, (__nv_bfloat16*)dst_dev, n);
      break;
    case TTALS_F32: k_widen_u8<float><<<nb, 256, 0, st>>>((const uint8_t*)src_dev, (float*)dst_dev, n); break;
    default: k_widen_u8<double><<<nb, 256, 0, st>>>((const uint8_t*)src_dev, (double*)dst_dev, n); break;
  }
  TT_CUDA(cudaGetLastError());
  return TTALS_OK;
}

ttals_status ttals_slice_error_noalloc(const void* x_dev, ttals_dtype x_dtype, const void* y_dev,
                                       ttals_dtype y_dtype, int64_t n, double* out2_dev, void* cuda_stream) {
  if (!x_dev || !y_dev || !out2_dev || n < 1) {
    g_last_err = "ttals_slice_error_noalloc: NULL pointer or n < 1";
    return TTALS_EINVAL;
  }
  if (n > (int64_t)kErrMaxCtas * kErrPerCta) {
    g_last_err = "ttals_slice_error_noalloc: n = " + std::to_string((long long)n) +
                 " exceeds the static scratch limit of " + std::to_string((long long)kErrMaxCtas * kErrPerCta) +
                 " elements";
    return TTALS_EINVAL;
  }
  if ((x_dtype < TTALS_F64 || x_dtype > TTALS_BF16) || (y_dtype != TTALS_F64 && y_dtype != TTALS_F32)) {
    g_last_err = "ttals_slice_error_noalloc: unsupported dtype";
    return TTALS_EINVAL;
  }
  const size_t xs = dtype_size(x_dtype), ys = dtype_size(y_dtype);
  if (((uintptr_t)x_dev % xs) || ((uintptr_t)y_dev % ys) || ((uintptr_t)out2_dev % 8)) {
    g_last_err = "ttals_slice_error_noalloc: misaligned pointer";
    return TTALS_EINVAL;
  }
  unsigned char* scr = nullptr;
  TT_TRY(err_scratch_for_current_device(&scr));
  double* part = (double*)scr;
  unsigned* ticket = (unsigned*)(scr + kErrPartBytes);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TT_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
  switch (x_dtype) {
    case TTALS_F64: return launch_slice_error((const double*)x_dev, y_dev, y_dtype, n, part, ticket, out2_dev, st);
    case TTALS_F32: return launch_slice_error((const float*)x_dev, y_dev, y_dtype, n, part, ticket, out2_dev, st);
    case TTALS_F16: return launch_slice_error((const __half*)x_dev, y_dev, y_dtype, n, part, ticket, out2_dev, st);
    default:
      return launch_slice_error((const __nv_bfloat16*)x_dev, y_dev, y_dtype, n, part, ticket, out2_dev, st);
  }
}

}  // extern "C"
