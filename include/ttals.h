/*
 * ttals.h - Online TT-ALS per-slice update (arXiv 2606.31061) on one B300 GPU.
 *
 * A stream delivers slices X_t of shape I_1 x ... x I_{n-1} along the last mode
 * (Sec. 2.3, streaming tensor X[t] = X[t-1] (+) X_t).  The library keeps the
 * time-t Tensor-Train decomposition {G_k[t]}_{k=1}^{n-1}, g_n[t] (Sec. 3.1,
 * Eq. proposed-objective-slice) on the device and updates it once per slice
 * with the single sweep of Algorithm 1.
 *
 * Conventions shared by every entry point:
 *  - Slices are dense, C-order (last slice mode fastest), in device memory.
 *  - Core k (1-based) has shape r_{k-1} x I_k x r_k, C-order, r_0 = 1; core n is
 *    the temporal row g_n of length r_{n-1}.
 *  - Ingest dtype F64 runs every step in FP64.  F32, F16 and BF16 ingest keep
 *    the state in FP32 and contract the slice with FP32 accumulation.  How each
 *    local solve is orthogonalised (Sec. 3.4.2) depends on the path:
 *     - the fused FP16/BF16 path (saturated second level, r_1 <= 64): the Gram of
 *       the level-1 solve is summed in FP64 from FP32 partials and factored in
 *       FP64 (cfg->factor = 0, default; 1 = FP32 factor); the tall apply runs in
 *       FP32 and is rounded to the ingest type, and the projector is made exact
 *       for that rounded basis with its own Gram (no polar pass, qr_passes is
 *       ignored);
 *     - every other F32/F16/BF16 stream: a Gram / Cholesky pass (FP32 factor,
 *       FP64 sums), followed, when qr_passes = 2 (the default), by one FP64 polar
 *       re-orthogonalisation.
 *  - Calls that take a `cuda_stream` only enqueue work on it (NULL = legacy
 *    default stream) and return without synchronising; device-side conditions
 *    (non-finite slice, rank-deficient local solve handled by the Householder
 *    path) are latched on the device and reported by the next synchronising call
 *    (ttals_sync, ttals_step, ttals_cores, ttals_stats).
 *  - The library owns every device buffer it allocates.  The caller owns slice
 *    and output buffers and keeps them alive until the enqueued work that uses
 *    them has completed on `cuda_stream`.
 *  - No entry point falls back to the CPU.  If the CUDA device or the kernels
 *    are unavailable, ttals_create fails with TTALS_ECUDA.
 *  - A ttals_stream is not thread-safe; distinct streams may be used from
 *    distinct host threads.
 */
#ifndef TTALS_H_
#define TTALS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ttals_stream ttals_stream; /* opaque, library-owned */

typedef enum {
    TTALS_F64 = 0,
    TTALS_F32 = 1,
    TTALS_F16 = 2,
    TTALS_BF16 = 3
} ttals_dtype;

typedef enum {
    TTALS_OK = 0,
    TTALS_EINVAL = 1,     /* bad argument; nothing was enqueued                      */
    TTALS_ENOMEM = 2,     /* device allocation failed                                */
    TTALS_ECUDA = 3,      /* CUDA runtime error (message: ttals_last_error)          */
    TTALS_ENONFINITE = 4, /* a pushed slice held NaN/Inf; that slice was not committed */
    TTALS_ETIMEOUT = 5,   /* a bounded device wait gave up                           */
    TTALS_ESTATE = 6      /* call not valid in the stream's current state            */
} ttals_status;

typedef struct {
    ttals_dtype ingest;  /* dtype of every slice pushed to this stream (default F64)       */
    uint64_t seed;       /* seed of the default random initial cores (default 0x5eed)     */
    int device;          /* CUDA device ordinal (default 0)                               */
    int qr_passes;       /* orthogonalisation passes per local solve on the generic path
                            (F64/F32 ingest, unsaturated levels): 1 = Cholesky-QR with an
                            FP32 factor only, 2 = followed by one FP64 polar
                            re-orthogonalisation (0 = default = 2).  The fused FP16/BF16
                            path ignores it (see `factor`)                               */
    int env_kernel;      /* fused path, environment kernel (S6): 0 = chosen by shape, 1 = the
                            clustered one, 2 = one CTA per column tile over all rows (ignored
                            when its tile does not fit), 3 = streamed row stages, 4 = streamed
                            row stages on tcgen05 (ranks padded to 16, 32 or 64; else 3)  */
    int k1_split;        /* fused path, k-splits of the local solve (S4): 0 = chosen by
                            shape and batch size, else 1, 2, 4 or 8                         */
    int factor;          /* fused path, the r x r factor of each local solve's Gram (S5):
                            0 = FP64 (default), 1 = FP32 (one warp; faster, for comparison)  */
    int mode;            /* local solves: 0 = literal (Eq. proposed-core-update under the
                            orthogonality of Sec. 3.3; default), 1 = lsq (the Gram form of
                            Sec. 3.3: G~_k = A_k^T X B_k^T (B_k B_k^T)^-1 with the r x r solve in
                            FP64, then the QR of Sec. 3.4.2), 2 = noortho (the ablation of
                            Sec. 5.4: LQ/QR removed, both Gram inverses, FP64 r x r solves).
                            1 and 2 run on the generic path (no batches).                 */
    int solve_kernel;    /* fused path, local-solve kernel and its tile shape (S4): 0 = chosen
                            per launch from the stepping streams' row tiles, 1 = mma.sync on
                            64-row tiles with k-splits (k1_split) reduced in a cluster, 2 =
                            tcgen05 on 128-row tiles over whole rows (no k-split)          */
    int factor_cluster;  /* fused path, CTAs per stream of the r x r factor kernel (S5): 0 =
                            chosen by batch size, 4 or 8 (rows of Y per CTA: I_1/4 or I_1/8;
                            4 only where its shared memory fits, else 8)                   */
} ttals_config;

/*
 * ttals_create - allocate a stream of order n = n_slice_modes + 1.
 *   dims[0..n_slice_modes-1]  = I_1..I_{n-1} (each >= 1)
 *   ranks[0..n_slice_modes-1] = requested TT ranks r_1..r_{n-1} (each >= 1)
 *   cfg may be NULL (defaults).  n_slice_modes must be in [2, 8].
 * The ranks are clamped to the feasible set r_k <= min(r_{k-1} I_k, I_{k+1} r_{k+1})
 * (r_0 = 1) that the LQ of Sec. 3.4.1 and the QR of Sec. 3.4.2 require;
 * ttals_effective_ranks reports the result.  The initial cores are random
 * ("Initialize orthogonal cores randomly", Algorithm 1): Gaussian entries from a
 * SplitMix64 / Box-Muller generator seeded with cfg->seed.  Allocates every
 * device buffer the update needs; no later call allocates.
 * env_kernel, k1_split, solve_kernel and factor_cluster fix the fused path's schedule (an
 * autotuner's choice); they change the FP32 summation order, never the arithmetic the update
 * performs.
 * Errors: EINVAL (shape, dtype, schedule fields out of range, reserved fields), ENOMEM,
 * ECUDA.  On error *out is NULL.
 */
ttals_status ttals_create(int n_slice_modes, const int64_t *dims, const int64_t *ranks,
                          const ttals_config *cfg, ttals_stream **out);

/* Release every resource of the stream (synchronises with its pending work).  NULL is a no-op. */
void ttals_destroy(ttals_stream *s);

/* Write the clamped ranks r_1..r_{n-1} to ranks_out (n_slice_modes entries). */
ttals_status ttals_effective_ranks(const ttals_stream *s, int64_t *ranks_out);

/*
 * ttals_set_cores - replace the state by host FP64 cores (initial state or resume).
 *   cores[k] (k = 0..n-2) points to r_k x I_{k+1} x r_{k+1} doubles (C-order, clamped
 *   ranks), g points to r_{n-1} doubles, t is the committed step count to report.
 * The cores need not be orthogonal: Algorithm 1 re-orthogonalises them at the next
 * push.  Synchronous.  Clears latched errors.  Errors: EINVAL, ECUDA.
 */
ttals_status ttals_set_cores(ttals_stream *s, const double *const *cores, const double *g,
                             int64_t t);

/*
 * ttals_seed_cores - replace the state by the library's default random initial cores drawn
 *   from `seed` ("Initialize orthogonal cores randomly", Algorithm 1): the generator and
 *   order of ttals_create, so ttals_seed_cores(s, x) gives the cores that ttals_create with
 *   cfg->seed = x gives its (first) stream; seed 0 means the default seed.  t becomes 0 and
 *   latched errors are cleared.  On a batch it applies to the stream chosen by
 *   ttals_batch_select (a serving loop seeds each stream it admits into a slot).
 *   Synchronous.  Errors: EINVAL (NULL), ECUDA.
 */
ttals_status ttals_seed_cores(ttals_stream *s, uint64_t seed);

/*
 * ttals_push_slice - one step of Algorithm 1 (Sec. 3.4) for the slice X_t.
 *   slice_dev: device pointer to prod(I_k) elements of `dtype` (C-order), 16-byte aligned.
 *   dtype must equal the stream's ingest dtype.
 * Enqueues the whole update on cuda_stream and returns.  If the slice holds a
 * non-finite value the state is left unchanged and TTALS_ENONFINITE is latched.
 * Errors returned immediately: EINVAL (NULL/misaligned pointer, dtype mismatch), ECUDA.
 */
ttals_status ttals_push_slice(ttals_stream *s, const void *slice_dev, ttals_dtype dtype,
                              void *cuda_stream);

/*
 * ttals_reconstruct - write x^_t = G_1 x ... x G_{n-1} x g_n (the time-t
 * reconstruction of the last committed slice, Sec. 3.1) to out_dev as prod(I_k)
 * elements of out_dtype, C-order.  Asynchronous on cuda_stream.
 * Errors: EINVAL (NULL/misaligned pointer, bad dtype), ECUDA.
 */
ttals_status ttals_reconstruct(ttals_stream *s, void *out_dev, ttals_dtype out_dtype,
                               void *cuda_stream);

/*
 * ttals_cores - copy core k (1..n-1, shape r_{k-1} x I_k x r_k) or, for k = n, the
 * temporal row g_n (r_{n-1}) of the current decomposition to host_out as doubles.
 * n_elems must equal the core's element count.  The cores are left-orthogonal
 * (Sec. 2.4) after at least one push.  Synchronising.
 * Errors: EINVAL, ECUDA, plus any latched device error (the copy is still made).
 */
ttals_status ttals_cores(ttals_stream *s, int k, double *host_out, size_t n_elems);

/*
 * ttals_stats - per-slice accuracy of the last committed step and running totals
 * (RE over the entire stream, Sec. 5.1).  out[0] = ||x_t||^2, out[1] = ||x_t - x^_t||^2,
 * out[2] = sum_t ||x_t||^2, out[3] = sum_t ||x_t - x^_t||^2 over committed steps.
 * Synchronising.  Errors: EINVAL, ECUDA, plus any latched device error.
 */
ttals_status ttals_stats(ttals_stream *s, double out[4]);

/* ttals_step - committed step count t (synchronising; reports latched errors). */
ttals_status ttals_step(ttals_stream *s, int64_t *t_out);

/* ttals_sync - wait for the stream's enqueued work; return and clear the latched error. */
ttals_status ttals_sync(ttals_stream *s);

/* Bytes of device memory the stream holds (state + scratch); for admission control. */
size_t ttals_device_bytes(const ttals_stream *s);

/*
 * Instrumentation (the paper has no counterpart; tracing and metrics of the library).
 *
 * ttals_launch_count - number of CUDA kernels this stream has launched so far
 *   (a host-side counter; no synchronisation).
 * ttals_stats_async - enqueue on cuda_stream a copy of the four ttals_stats values
 *   {||x_t||^2, ||x_t - x^_t||^2, sum ||x||^2, sum ||x - x^||^2} into out4 (host
 *   pinned or device memory, 4 doubles).  Errors: EINVAL, ECUDA.
 * ttals_profile - enable (1) or disable (0) per-push timing: CUDA events recorded on
 *   the launch stream before the level-1 local solve Y = X_(1) B_1^T, after it, before
 *   and after the level-1 environment E_2 = G_1^T X_(1), and around the whole update.
 *   While enabled, consecutive kernels are not overlapped.  Synchronising.
 * ttals_profile_read - wait, then write the summed milliseconds over the pushes timed
 *   since the last read: ms_out[0] level-1 solve, ms_out[1] level-1 factorisation
 *   (orthonormal basis of the solve's span), ms_out[2] level-1 environment, ms_out[3]
 *   whole update; *n_out = number of pushes.  Resets the totals.
 */
uint64_t ttals_launch_count(const ttals_stream *s);
/*
 * ttals_debug_stall_solve - fault injection for tests (off unless called).  The next
 *   n_pushes pushes of a stream on the fused FP16/BF16 path launch the level-1 local solve
 *   (the k-split kernel) so that it issues no copy: its bounded wait for the first stage
 *   gives up after about 100 ms, the kernel returns, the step is not committed and
 *   TTALS_ETIMEOUT is latched for the next synchronising call.  Nothing faults and the
 *   context stays usable.  n_pushes = 0 switches it off.  Errors: EINVAL.
 */
ttals_status ttals_debug_stall_solve(ttals_stream *s, int n_pushes);
ttals_status ttals_stats_async(ttals_stream *s, double *out4, void *cuda_stream);
ttals_status ttals_profile(ttals_stream *s, int enable);
ttals_status ttals_profile_read(ttals_stream *s, double ms_out[4], int64_t *n_out);

/*
 * ttals_slice_error_noalloc - allocation-free slice error (the paper has no
 *   counterpart; an evaluation helper of this library).
 *   Enqueues on cuda_stream the computation of out2_dev[0] = ||x||^2 and
 *   out2_dev[1] = ||x - y||^2 (FP64 sums in a fixed order, deterministic) for two
 *   device arrays of n elements, e.g. a slice x_t and the reconstruction written by
 *   ttals_reconstruct.  x_dtype: F64, F32, F16 or BF16; y_dtype: F64 or F32.
 *   out2_dev: 2 doubles of device memory, 8-byte aligned, owned by the caller.
 * Allocates nothing: for callers that cannot allocate device memory at the point
 *   of the call (a serving loop that checks accuracy between pushes on a stream it
 *   must not stall, as cudaMalloc/cudaFree synchronise the device; a process whose
 *   device memory is fully reserved by its own pool).  Its scratch is a static
 *   device array of 64 KiB (+256 B) per device, which limits n to 2^26 = 67,108,864
 *   elements.  The first call on each device resolves the scratch address with
 *   that device current and should precede any stream capture on that device.
 *   Each call first clears the scratch's ticket counter on cuda_stream.  Calls
 *   that overlap in time on one device (different streams or host threads) share
 *   that scratch and race: serialise them.
 * Errors (nothing enqueued): EINVAL (NULL pointer, n < 1, n > 2^26 with a message in
 *   ttals_last_error, unsupported dtype, misaligned pointer), ECUDA.
 */
ttals_status ttals_slice_error_noalloc(const void *x_dev, ttals_dtype x_dtype, const void *y_dev,
                                       ttals_dtype y_dtype, int64_t n, double *out2_dev,
                                       void *cuda_stream);

/*
 * Batches of streams.  Algorithm 1 updates one stream; a batch holds n_streams
 * independent streams of ONE shape (dims, ranks, ingest) whose updates run in the
 * same kernel launches (each launch's grid gains one plane per stream), so that a
 * step of many small streams reads their slices at full HBM rate.  Every stream of
 * a batch performs the arithmetic it performs alone; a batch may take other
 * kernel schedules (whole-row tcgen05 tiles, fewer k-splits, streamed row stages),
 * so its FP32 sums can run in another order: results agree to FP32 rounding after
 * one step, and the 16-bit state can then round differently (a stream's results do
 * not depend on its slot or on the other streams of the batch, bit for bit).
 *
 * ttals_create_batch - like ttals_create, for 1 <= n_streams <= TTALS_MAX_BATCH
 *   streams.  Stream b starts from its own default cores (the b-th draw of the
 *   seeded generator; stream 0's equal ttals_create's).  Only shapes that take the
 *   fused FP16/BF16 path batch: FP16/BF16 ingest, r_1 >= I_2...I_{n-1} (saturated
 *   second level), r_1 <= 64, I_2...I_{n-1} a multiple of 8, I_1 <= 4096.
 *   Errors: EINVAL (also for a shape that does not batch; message in
 *   ttals_last_error), ENOMEM, ECUDA.
 * ttals_push_batch - one step of every stream of the batch.  slices_dev holds
 *   n_streams slices back to back ([n_streams][I_1]...[I_{n-1}], C order, stream b's
 *   slice at element offset b * I_1...I_{n-1}), 16-byte aligned, device memory
 *   owned by the caller and kept alive until the work on cuda_stream passes the
 *   call.  Asynchronous.  Errors: EINVAL, ECUDA.
 * ttals_batch_select - wait for the batch's work, then direct the per-stream calls
 *   (ttals_set_cores, ttals_cores, ttals_reconstruct, ttals_stats, ttals_stats_async,
 *   ttals_step, ttals_sync) to stream `index`.  Errors: EINVAL, ECUDA.
 * ttals_push_batch_masked - like ttals_push_batch, but only the streams whose bit is set in
 *   active_mask (bit b for stream b) take a step; the others keep their state, step count
 *   and statistics, and their part of slices_dev is not read.  For serving loops in which
 *   not every stream has a new slice at every step.  An all-zero mask enqueues nothing.
 * ttals_batch_size - n_streams of a batch, 1 for a single stream, 0 for NULL.
 * ttals_push_slice on a batch returns ESTATE.
 */
#define TTALS_MAX_BATCH 64
ttals_status ttals_create_batch(int n_streams, int n_slice_modes, const int64_t *dims,
                                const int64_t *ranks, const ttals_config *cfg, ttals_stream **out);
ttals_status ttals_push_batch(ttals_stream *s, const void *slices_dev, ttals_dtype dtype,
                              void *cuda_stream);
ttals_status ttals_push_batch_masked(ttals_stream *s, const void *slices_dev, ttals_dtype dtype,
                                     uint64_t active_mask, void *cuda_stream);
ttals_status ttals_batch_select(ttals_stream *s, int index);
int ttals_batch_size(const ttals_stream *s);

/*
 * Host ingest of a batch, for serving loops (one call per step instead of one copy per frame
 * from the caller; the paper has no counterpart: it streams one slice at a time).
 * ttals_batch_ingest_init - give the batch its own double-buffered input blocks
 *   ([n_streams][slice] in the ingest type; with u8_wire = 1 also 8-bit staging, the frames
 *   then being 8-bit pixels widened on the device, exact), a high-priority copy stream, a
 *   compute stream and a ring of 256 completion events.  Allocates (counted by
 *   ttals_device_bytes); call once, before serving.  Ingest F16, BF16 or F32.
 *   Errors: EINVAL, ESTATE (already initialised), ENOMEM, ECUDA.
 * ttals_batch_push_host - one masked step of the batch: n frames (1 <= n <= n_streams), frame
 *   i for stream slots[i] (distinct) from host_frames[i] (pinned host memory, the slice in the
 *   ingest type, or bytes with the 8-bit wire; the caller keeps it unchanged until the step's
 *   ticket is done).  Enqueues the copies, the widening, the step of the streams given a frame
 *   (the others keep their state, as in ttals_push_batch_masked) and a completion event, and
 *   returns its ticket (0, 1, 2, ...).  Errors (nothing enqueued): EINVAL, ECUDA.
 * ttals_batch_ticket_done - *done = 1 once the step of `ticket` has completed on the device,
 *   else 0 (no synchronisation).  Only the 256 most recent tickets are tracked: an older
 *   ticket reports the completion of a later step (never earlier than its own).
 *   Errors: EINVAL (unknown ticket), ECUDA.
 */
ttals_status ttals_batch_ingest_init(ttals_stream *s, int u8_wire);
ttals_status ttals_batch_push_host(ttals_stream *s, int n, const int *slots, const void *const *host_frames,
                                   uint64_t *ticket_out);
ttals_status ttals_batch_ticket_done(ttals_stream *s, uint64_t ticket, int *done);

/*
 * ttals_widen_u8 - enqueue on cuda_stream dst[i] = src[i] for n 8-bit unsigned values,
 *   widened to dst_dtype (F16, BF16, F32 or F64; exact, since 0..255 are representable).
 *   The paper's video slices are 8-bit pixels (Sec. 5.1): a serving loop that receives
 *   them from the host can move bytes over the host link and widen on the device, half
 *   the traffic of FP16.  src and dst: device memory, 16-byte aligned, owned by the
 *   caller.  Errors (nothing enqueued): EINVAL, ECUDA.
 */
ttals_status ttals_widen_u8(const void *src_dev, void *dst_dev, ttals_dtype dst_dtype, int64_t n,
                            void *cuda_stream);

/* Static text for a status code. */
const char *ttals_status_string(ttals_status st);

/* Message of the last CUDA error seen on this thread ("" if none). */
const char *ttals_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TTALS_H_ */
