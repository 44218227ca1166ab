/*
 * tt_sketch.h -- C ABI of the GB300 (sm_103a) TensorSketch proximal TT-ALS library.
 *
 * The library computes the hot path of Algorithm 1 (TT-TS) of Chen, Jiang, Yu, Qi,
 * "Low-rank Tensor Train Decomposition Using TensorSketch" (arXiv 2309.08093):
 *   (a) the TensorSketch of the data unfolding, Y_k = S A_(k)^T           (Alg. 1, Sec. 3)
 *   (b) the FFT TensorSketch of the TT interface matrix, S H_k            (Theorems 1 and 2)
 *   (c) the proximal normal-equation update of core k                     (Eq. (ite), Sec. 3)
 * plus the orthogonalisation steps of Algorithm 1 and the relative error of Sec. 5.
 *
 * Conventions (0-based; the paper is 1-based):
 *   - tensor A has d modes of sizes n[0..d-1] and is stored densely with mode 0 fastest
 *     (linear index i = sum_s i_s prod_{t<s} n_t, the bijection of Sec. 2.2);
 *   - TT core k has shape r[k] x n[k] x r[k+1] and is stored FP32 with r[k] fastest
 *     (element (a, i, b) at a + r[k]*(i + n[k]*b)); r[0] = r[d] = 1 (Sec. 2.1);
 *   - Y_k (sketch of the mode-k unfolding) is FP32, J x n[k], column-major: Y_k[b + J*i];
 *   - S H_k is FP32, J x s_k with s_k = r[k]*r[k+1], column-major: SH[b + J*c] with column
 *     c = a + r[k]*b' (a indexes r[k], b' indexes r[k+1]; matches G_{k(2)}, Sec. 3).
 *   - The sketch size m of the paper is J: any integer in [2, 8192], or a power of two up to
 *     16384. Powers of two use radix-4 / radix-2 FFTs; other sizes (the paper's m = 45, 150,
 *     200, 1000, 2000 of Sec. 5) use direct DFTs of O(J^2) work per transform.
 *
 * Hash/sign draws (Sec. 2.2, Eqs. (eqn_h), (eqn_v)): per sweep t and mode k the library draws
 *   h_k(i) = word(seed, t, k, 0, i) mod J,  v_k(i) = 1 - 2 * (word(seed, t, k, 1, i) >> 63),
 * where word() chains SplitMix64 output steps:  step(z, f) = mix64(z + (f+1) * 0x9E3779B97F4A7C15),
 * word(seed, t, k, s, i) = step(step(step(step(seed, t), k), s), i), and mix64 is the SplitMix64
 * finaliser (Steele, Lea, Flood 2014). With TT_FLAG_FIXED_SKETCH every sweep uses t = 0.
 *
 * Ownership: every pointer named *_dev is device memory owned by the caller; the library never
 * frees it. Arrays of pointers (float* const* ...) are HOST arrays of d device pointers. The
 * context owns its hash tables, plans and workspaces (allocated in tt_sketch_init).
 *
 * Streams: all work is enqueued on the stream given to tt_sketch_init. Calls that return host
 * scalars (tt_prox_als_sweep, tt_prox_als_sweep_monitored, tt_rel_error, tt_sketch_tables)
 * synchronise that stream; the others are asynchronous.
 *
 * Errors: every int-returning call returns TT_OK (0) or a negative TT_E* code; the message of
 * the last failure is available from tt_last_error(ctx). On error no output is guaranteed.
 * Invalid arguments are rejected on the host before anything is launched.
 */
#ifndef TT_SKETCH_H
#define TT_SKETCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tt_ctx tt_ctx; /* opaque, library-owned */

/* storage type of the data tensor A */
/* TT_FP8E4M3: OCP FP8 E4M3 bytes (bias 7, no infinities, largest finite 448); the code S.1111.111
 * is the format's NaN and reaches a solve as a non-finite value (TT_ENONFINITE) */
enum { TT_F64 = 0, TT_F32 = 1, TT_BF16 = 2, TT_FP8E4M3 = 3 };

/* status codes */
enum {
  TT_OK = 0,
  TT_EINVAL = -1,      /* bad shape, rank, J, k, dtype or null pointer */
  TT_ENOMEM = -2,      /* device or host allocation failed */
  TT_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed */
  TT_ENOTSPD = -4,     /* the Gram matrix of Eq. (ite) is not positive definite (sigma = 0) */
  TT_ETIMEOUT = -5,    /* a bounded device-side wait gave up */
  TT_ENONFINITE = -6   /* a NaN or Inf reached a solve */
};

/* flags */
/* draw h_k, v_k once (t = 0) instead of once per sweep; the data sketches then depend on A alone,
 * and a multi-sweep call computes them in its first sweep and reuses them in the others */
#define TT_FLAG_FIXED_SKETCH 1u
#define TT_FLAG_FP64_SOLVE 2u   /* solve Eq. (ite) in FP64 also when sigma > 0 (see tt_prox_update) */
/* Fixed summation orders: repeated calls on the same inputs return the same bits (data sketches,
 * interface sketches, updated cores, relative errors and rel-changes of the dense-tensor calls),
 * on any device and whatever A's alignment. The data sketch then adds the fibres of each run of
 * equal hash in index order (FP32), over work spans fixed by the shape, rounds each run's sum to
 * 64-bit fixed point (one scale for the tensor, from max |A|) and adds those with integer atomics;
 * the Gram's K-chunks and all partial sums are added in a fixed order, and the CountSketch of the
 * cores adds its entries in index order. Slower: one more read of A for the scale, the plans of
 * every draw built in index order, and 8-byte integer flushes. The sparse coordinate-form calls
 * are not covered. */
#define TT_FLAG_DETERMINISTIC 4u
/* Gram and right-hand side of the FP32 update (sigma > 0) on the tensor cores (tcgen05, TF32
 * operands staged by TMA, FP32 accumulators in tensor memory), when J is a multiple of 4 and
 * r[k]*r[k+1] <= 256; otherwise the CUDA-core FP32 Gram. TT_FLAG_TC_GRAM splits every operand into
 * two TF32 parts and adds three products (about 2^-22 relative error per product, the FP32
 * form's accuracy); TT_FLAG_TF32_GRAM reads the operands once as TF32 (about 2^-11 per product:
 * the mixed-precision form). */
#define TT_FLAG_TC_GRAM 8u
#define TT_FLAG_TF32_GRAM 16u
/* Batched contexts (tt_batch_init): on the first tt_batch_sweep, time every tensor's data-sketch
 * launches alone over a few work-item counts and CTA-per-SM limits and keep the fastest. Off by
 * default: the batch sizes the work items of each tensor by its bytes (at least 1 MB of A per
 * item), which keeps small tensors' launches to a few CTAs so that many run side by side, and
 * timing each launch alone optimises its own latency rather than the batch's throughput. */
#define TT_FLAG_BATCH_AUTOTUNE 32u

typedef struct {
  int d;              /* order of the tensor, 2 <= d <= 8 */
  const int64_t* n;   /* host array of d mode sizes, each >= 1 */
  const int* r;       /* host array of d+1 TT ranks, r[0] = r[d] = 1, each >= 1;
                         each r[k] <= 160, r[k]*r[k+1] <= 512 (up to 160 by Gauss-Jordan in
                         registers, above by a one-CTA Cholesky needing 4 s (n[k] + 33) bytes of
                         shared memory <= 227 KB), r[k]*n[k]*r[k+1] <= 40000 (in-CTA QR) */
  int J;              /* sketch size m: 2..8192, or a power of two up to 16384 */
  double lambda;      /* proximal weight sigma >= 0 of Eq. (lrtt_sub_prox) */
  uint64_t seed;      /* seed of the hash/sign draws */
  int dtype;          /* TT_F64, TT_F32, TT_BF16 or TT_FP8E4M3: storage type of A */
  unsigned flags;     /* TT_FLAG_* */
} tt_params;

/*
 * Create a context for tensors of the given shape (Alg. 1 inputs: A's shape, TT ranks,
 * sketch size m, sigma). `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 * Allocates all device workspaces. Returns TT_EINVAL for inconsistent parameters.
 */
int tt_sketch_init(tt_ctx** out, const tt_params* p, void* cuda_stream);

/* Release the context and its device memory (never the caller's buffers). NULL is a no-op. */
void tt_sketch_destroy(tt_ctx* ctx);

/* Message of the last failure on this context ("" if none). Valid until the next call. */
const char* tt_last_error(const tt_ctx* ctx);

/*
 * Process-wide cap on the device memory a context may own (0 = no cap, the default); returns
 * the previous cap. The paper has no counterpart: it is memory budgeting for applications that
 * share the GPU. tt_sketch_init sums the sizes of all the workspaces it would allocate (hash
 * tables, fibre plans of two draws, FFT sketches, data sketches, Gram and solve buffers, the
 * relative error's interfaces) before any CUDA call, and returns TT_ENOMEM (message on stderr)
 * when the sum exceeds the cap; tt_prox_als_sweep_host returns TT_ENOMEM the same way before it
 * allocates its staging buffers (the tensor, the scales and the cores) beyond the cap. Contexts
 * created before a change keep what they own. Thread-safe.
 */
uint64_t tt_set_workspace_limit(uint64_t bytes);

/*
 * Copy the hash and sign tables of sweep `sweep` (Sec. 2.2; drawn on the device) to host
 * arrays of sum_k n[k] entries, mode 0 first: h_host[off_k + i] = h_k(i) in [0, J),
 * v_host[off_k + i] = v_k(i) in {+1, -1}. Synchronises the stream.
 */
int tt_sketch_tables(tt_ctx* ctx, uint64_t sweep, int32_t* h_host, int8_t* v_host);

/*
 * Replace the drawn tables by caller-given ones (host arrays laid out as in tt_sketch_tables;
 * h values must lie in [0, J), v values in {+1, -1}). From then on every sweep uses them, as
 * with TT_FLAG_FIXED_SKETCH. Used to reproduce the worked example of Sec. 2.2.
 */
int tt_sketch_set_tables(tt_ctx* ctx, const int32_t* h_host, const int8_t* v_host);

/*
 * Part (a): Y_k = S A_(k)^T (Alg. 1, "compute S A_(k)^T"; S is the TensorSketch built from
 * the CountSketches of all modes s != k, Eqs. (eqn_h), (eqn_v)). Every entry of A is read.
 *   A_dev       : the dense tensor in the storage type of the context;
 *   scales_dev  : for TT_FP8E4M3, n[0] FP32 scales (A(i) = scale[i_0] * fp8(i)); else NULL;
 *   k           : mode in [0, d), or -1 for all modes;
 *   sweep       : sweep index t selecting the hash draw;
 *   Y_dev       : host array of d device pointers; Y_dev[k] (J x n[k], column-major) is written
 *                 for each requested mode (other entries may be NULL).
 */
int tt_sketch_unfold(tt_ctx* ctx, const void* A_dev, const float* scales_dev, int k,
                     uint64_t sweep, float* const* Y_dev);

/*
 * Part (a) for a sparse tensor in coordinate form, at O(nnz) cost (Sec. 3, the discussion after
 * Theorem 3). The context's dtype is not used: values are FP32.
 *   idx_dev : device int32 array of d x nnz indices, mode-major: idx_dev[s*nnz + e] = i_s of
 *             entry e (0-based);
 *   val_dev : device FP32 array of the nnz values; repeated coordinates add up;
 *   nnz     : number of entries (>= 0; idx_dev and val_dev may be NULL when it is 0);
 *   k, sweep, Y_dev : as tt_sketch_unfold (each requested Y_k is zeroed, then accumulated).
 * Entries with an index outside [0, n[s]) are skipped and the call returns TT_EINVAL. The call
 * reads the device status back, so it synchronises. Followed by tt_prox_als_sweep_sketched with
 * the same sweep, it gives a sweep of Algorithm 1 on the sparse tensor.
 */
int tt_sketch_unfold_coo(tt_ctx* ctx, const int32_t* idx_dev, const float* val_dev, int64_t nnz,
                         int k, uint64_t sweep, float* const* Y_dev);

/*
 * Part (b): S H_k with H_k = G_{>k}^T kron G_{<k}, computed as
 * F^{-1}[(F S_{>k} G_{>k}^T) face-split (F S_{<k} G_{<k})] (Theorem 1) with the two factors
 * formed by slice-wise products of the FFT-sketched cores (Theorem 2).
 *   cores_dev : host array of d device pointers to the FP32 cores (read only);
 *   SH_dev    : J x s_k FP32 column-major output.
 */
int tt_sketch_interface(tt_ctx* ctx, float* const* cores_dev, int k, uint64_t sweep,
                        float* SH_dev);

/*
 * Part (c): the proximal update of core k by Eq. (ite) (read with S^T S):
 *   G_{k(2)} <- (Y_k^T SH_k + sigma G_{k(2)}) (SH_k^T SH_k + sigma I)^{-1}.
 * Y_dev: J x n[k] column-major; SH_dev: J x s_k column-major; core_dev is read (proximal centre)
 * and overwritten with the update. Two forms, fixed at context creation:
 *   - sigma > 0 (Alg. 1's setting: M is SPD with smallest eigenvalue >= sigma): the Gram is
 *     accumulated in FP32 and solved in FP32, by Gauss-Jordan elimination in registers
 *     (s_k <= 160; its pivots are the D of L D L^T) or a blocked Cholesky in one CTA
 *     (s_k <= 512). A pivot at or below 1e-4 of the largest diagonal entry of M is refused with
 *     TT_ENOTSPD: the FP32 Gram's rounding noise (about sqrt(J) 2^-24 of that entry) can lift
 *     the pivots of a singular system to about that level. Small sigma with a nearly singular
 *     S H_k wants TT_FLAG_FP64_SOLVE.
 *   - sigma = 0 (run in Sec. 5, where M is not SPD by construction), or TT_FLAG_FP64_SOLVE:
 *     the Gram is accumulated in FP64 (the FP32 products are exact in FP64), factored by an
 *     FP64 Cholesky and solved by FP64 triangular solves. A pivot L_jj^2 at or below 1e-10 of
 *     the largest diagonal entry of M is refused with TT_ENOTSPD (M singular to the precision
 *     of its FP32 inputs; the oracle refuses at the same ratio).
 * Returns TT_ENOTSPD (core_dev unchanged), TT_ENONFINITE if S H_k or Y_k holds a NaN or Inf
 * (core_dev unchanged) or if the solve overflows. Synchronises the stream (the status is read
 * back).
 */
int tt_prox_update(tt_ctx* ctx, const float* Y_dev, const float* SH_dev, float* core_dev, int k);

/*
 * Orthogonalisation steps of Algorithm 1, in place on the FP32 cores (host array of device
 * pointers). direction = -1: the right-to-left orthogonalisation of all cores (each G_k^R,
 * k = d-1..1, gets orthonormal rows and the triangular factor moves into core k-1).
 * direction = +1 with 0 <= k < d-1: [Q, R] = qr(G_k^L), G_k <- Q, G_{k+1} <- R G_{k+1}^R.
 * Triangular factors have a non-negative diagonal; a wide unfolding (rows < columns) gets
 * zero-padded factors so the ranks keep their sizes.
 */
int tt_orthogonalize(tt_ctx* ctx, float* const* cores_dev, int direction, int k);

/*
 * `nsweeps` outer iterations of Algorithm 1 starting at sweep index `first_sweep`: right-to-left
 * orthogonalisation, a fresh sketch, then for k = 0..d-1 parts (b), (a), (c) and (k < d-1) the QR
 * step. Cores are updated in place. If rel_change_out is not NULL it receives, per sweep,
 * max_k ||G_k^(t+1) - G_k^(t)||_F / ||G_k^(t+1)||_F (Sec. 5), where G_k^(t) is core k right
 * before its update. The call synchronises the stream at its end to report the status of the
 * solves. Returns TT_ENOTSPD if a Gram matrix is not positive definite (cores are then left as
 * they were after the last successful update).
 */
int tt_prox_als_sweep(tt_ctx* ctx, const void* A_dev, const float* scales_dev,
                      float* const* cores_dev, int nsweeps, uint64_t first_sweep,
                      double* rel_change_out);

/*
 * tt_prox_als_sweep with the relative error of Sec. 5 after every sweep: rel_error_out (host,
 * nsweeps entries, required) receives ||A - [[G^(t+1)]]||_F / ||A||_F computed right after sweep t
 * (as tt_rel_error computes it, FP64 accumulation), rel_change_out (optional) as above. Sweeps and
 * errors are enqueued back to back and copied back with one synchronisation per block of
 * sweeps, instead of one per call of each. Returns as tt_prox_als_sweep; TT_EINVAL if
 * rel_error_out is NULL.
 */
int tt_prox_als_sweep_monitored(tt_ctx* ctx, const void* A_dev, const float* scales_dev,
                                float* const* cores_dev, int nsweeps, uint64_t first_sweep,
                                double* rel_change_out, double* rel_error_out);

/*
 * One sweep of Algorithm 1 (draw `sweep`) whose data sketches are given: Y_dev[k] must hold
 * Y_k = S A_(k)^T for that draw, as tt_sketch_unfold(ctx, A, scales, -1, sweep, Y_dev) returns
 * them (J x n[k] column-major). The sketches of a sweep do not depend on the cores, so computing
 * them beforehand and reusing them is exact; the tensor itself is not read. Used when the
 * sketches were already computed for another purpose (the warm start's summary). Synchronises;
 * returns as tt_prox_als_sweep.
 */
int tt_prox_als_sweep_sketched(tt_ctx* ctx, float* const* Y_dev, float* const* cores_dev,
                               uint64_t sweep);

/*
 * Relative error ||A - [[G_1, ..., G_d]]||_F / ||A||_F (Sec. 5) with FP64 accumulation.
 * Reads every entry of A once; synchronises and writes *out on the host.
 */
int tt_rel_error(tt_ctx* ctx, const void* A_dev, const float* scales_dev,
                 float* const* cores_dev, double* out);

/*
 * The same relative error for a sparse tensor in coordinate form (idx_dev, val_dev, nnz as in
 * tt_sketch_unfold_coo, but the coordinates must be distinct: ||A||^2 is summed entry by entry,
 * so a repeated coordinate would count its parts' squares instead of its sum's):
 * ||A - X||^2 = ||A||^2 - 2 <A, X> +
 * ||X||^2, every term in FP64 (X at each nonzero from the cores, ||X||^2 from their Gram chain).
 * Costs O(nnz sum_k r_k r_{k+1} + sum_k n_k r_k^2 r_{k+1}). Ranks up to 32 (else TT_EINVAL);
 * an index outside [0, n[s]) skips its entry and returns TT_EINVAL. Synchronises.
 */
int tt_rel_error_coo(tt_ctx* ctx, const int32_t* idx_dev, const float* val_dev, int64_t nnz,
                     float* const* cores_dev, double* out);

/*
 * The same sweeps on HOST buffers: A_host (the dense tensor in the context's storage type,
 * layout as above), scales_host (FP8 only, else NULL) and the d FP32 cores (host array of host
 * pointers, updated in place). Each call copies the inputs to library-owned device buffers
 * (allocated on first use: two for the tensor, counted against tt_set_workspace_limit), runs the
 * sweeps of tt_prox_als_sweep, then (if rel_error_out is not NULL) the relative error of
 * tt_rel_error, and copies the cores back; it synchronises. It is tt_prox_als_sweep_host_async
 * followed by tt_host_sync. Host memory should be page-locked for full copy bandwidth.
 * rel_change_out as above (at most 8192 / d sweeps per call when it is given).
 */
int tt_prox_als_sweep_host(tt_ctx* ctx, const void* A_host, const float* scales_host,
                           float* const* cores_host, int nsweeps, uint64_t first_sweep,
                           double* rel_change_out, double* rel_error_out);

/*
 * The same call without waiting, for a stream of host-buffer problems: it enqueues the copy of
 * A_host (and scales_host) into one of two device buffers on a library-owned copy stream, and, on
 * the context's stream after that copy, the copy of the cores, the sweeps, the relative error and
 * the copies back of the cores and of the result sums, then returns. The next call's tensor copy
 * runs beside this call's sweeps, so a sequence of calls is bound by the host link rather than by
 * copy plus sweeps. Calls run in order; consecutive calls on the same host core arrays see each
 * other's updates. Every host buffer of a call must stay valid, and its outputs (the cores,
 * rel_change_out, rel_error_out) unread, until tt_host_sync returns; at most four calls are in
 * flight (a fifth call first waits for the oldest). Page-locked host arrays are read and written
 * by a kernel, so that only the tensor copy uses a copy engine (pageable ones by copies). Returns
 * TT_OK or an argument/launch error; the status of the sweeps (TT_ENOTSPD, TT_ENONFINITE, ...) is
 * returned by tt_host_sync.
 */
int tt_prox_als_sweep_host_async(tt_ctx* ctx, const void* A_host, const float* scales_host,
                                 float* const* cores_host, int nsweeps, uint64_t first_sweep,
                                 double* rel_change_out, double* rel_error_out);

/* Wait for every call enqueued by tt_prox_als_sweep_host_async, write their rel_change_out and
 * rel_error_out, and return the first failure among them (TT_OK if none). */
int tt_host_sync(tt_ctx* ctx);

/*
 * Allocation-free proximal update. The paper has no counterpart: this is a service for callers
 * that cannot allocate device memory -- for example an application whose memory manager has
 * already reserved the device memory it is allowed to use, or a latency-critical loop that must
 * not pay for cudaMalloc's implicit device-wide synchronisation. It computes exactly what
 * tt_prox_update computes for a core of shape r0 x n x r1, without a context:
 *   Y_dev (J x n column-major), SH_dev (J x r0*r1 column-major), core_dev (read as the proximal
 *   centre, overwritten with the update), sigma >= 0, cuda_stream (a cudaStream_t or NULL).
 * Limits: r0, r1 >= 1 with r0*r1 <= 160, and n <= 1024; larger sizes (including ranks whose
 * product would overflow an int) are rejected with TT_EINVAL (and a message on stderr) before
 * anything is launched. It always takes the FP32 register solve, whatever sigma is.
 * Memory: it never calls cudaMalloc/cudaFree or any allocating routine. Its scratch (~0.76 MB of
 * FP32 Gram accumulators and a status word) is a static array in the library's device image, so
 * every GPU that loads the library holds it until the process exits. The first call on a device
 * looks up that array's device address while the device is current; make that first call before
 * any stream capture. All calls share the one array: each call clears what it needs, but calls
 * that overlap on the GPU (other streams, other host threads) race and give wrong results.
 * Synchronises `cuda_stream`; returns TT_OK, TT_ENOTSPD (core unchanged), TT_ENONFINITE,
 * TT_EINVAL or TT_ECUDA.
 */
int tt_prox_update_noalloc(const float* Y_dev, const float* SH_dev, float* core_dev, int J, int n,
                           int r0, int r1, double sigma, void* cuda_stream);

/*
 * Batched driver (the batching pattern: many tensors of different order, size, rank and sketch
 * size swept together). tt_batch_init creates one context per tt_params entry (all validated as
 * in tt_sketch_init) and a pool of streams. tt_batch_sweep runs `nsweeps` outer iterations of
 * Algorithm 1 on every tensor i: A_dev[i] (storage of params[i]), scales_dev[i] (FP8 only; the
 * array itself may be NULL when no tensor is FP8), cores_dev[i] (host array of params[i].d device
 * core pointers, updated in place). One sweep of all tensors is captured once into a CUDA graph
 * (tensors spread over the stream pool, forked from and joined to `cuda_stream`) and replayed
 * with one graph launch per sweep; the graph is recaptured when any pointer changes. Tensors with
 * TT_FLAG_FIXED_SKETCH compute their data sketches in a call's first sweep only. With
 * TT_FLAG_BATCH_AUTOTUNE in a tensor's flags the first call also times that tensor's data-sketch
 * launch shapes on its own data and keeps the fastest. Sweep t of the call uses
 * hash draw first_sweep + t (or 0 with TT_FLAG_FIXED_SKETCH). Synchronises `cuda_stream`;
 * returns TT_ENOTSPD etc. for the first tensor whose solve failed (tt_batch_last_error).
 */
typedef struct tt_batch tt_batch;
int tt_batch_init(tt_batch** out, int count, const tt_params* params, void* cuda_stream);
void tt_batch_destroy(tt_batch* b);
const char* tt_batch_last_error(const tt_batch* b);
int tt_batch_sweep(tt_batch* b, const void* const* A_dev, const float* const* scales_dev,
                   float* const* const* cores_dev, int nsweeps, uint64_t first_sweep);
/* Relative error of every tensor (as tt_rel_error) into out[count]; synchronises. */
int tt_batch_rel_error(tt_batch* b, const void* const* A_dev, const float* const* scales_dev,
                       float* const* const* cores_dev, double* out);

/* Per-context counters for measurement (not part of the method). */
typedef struct {
  double unfold_ms;          /* summed device time of the unfold-sketch kernels (CUDA events) */
  int64_t unfold_launches;   /* number of unfold-sketch kernel launches timed */
  int64_t unfold_bytes;      /* algorithmic bytes those launches read: entries x storage size */
  int64_t kernel_launches;   /* every kernel this library launched since the reset */
  double mode_ms[8];         /* unfold device time per mode */
  int64_t mode_launches[8];
} tt_profile;

/* on != 0: reset the counters and start timing unfold launches; on == 0: stop timing. */
int tt_profile_enable(tt_ctx* ctx, int on);

/* Synchronise the stream and read the counters accumulated since the last reset. */
int tt_profile_read(tt_ctx* ctx, tt_profile* out);

#ifdef __cplusplus
}
#endif

#endif /* TT_SKETCH_H */
