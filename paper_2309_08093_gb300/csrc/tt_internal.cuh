// Internal declarations shared by the translation units of libttsketch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tt_sketch.h"

// Two FP32 FMAs in one instruction (fma.rn.f32x2, sm_100 and later): d.x = a.x * b.x + c.x and
// d.y = a.y * b.y + c.y, each rounded once to nearest, i.e. exactly what two fmaf calls give.
__device__ __forceinline__ float2 tt_ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// Two FP32 products in one instruction (mul.rn.f32x2): d.x = a.x * b.x, d.y = a.y * b.y.
__device__ __forceinline__ float2 tt_fmul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

#define TT_MAX_D 8
#define TT_MAX_S 160      // largest r[k]*r[k+1] of the register solve (and largest single rank)
#define TT_MAX_S_LARGE 512  // largest r[k]*r[k+1] of the one-CTA Cholesky solve
size_t tt_large_solve_smem(int s, int n);  // its shared memory for s unknowns, n right-hand sides
#define TT_MAX_J 16384
// Relative pivot bound of the FP32 solves: a pivot at or below TT_PIVOT_TOL32 times the largest
// diagonal entry of M + sigma I is refused. The FP32 Gram carries a rounding noise of about
// sqrt(J) 2^-24 of that entry (up to about 1e-5 at J = 16384), which can lift the pivots of a
// singular or nearly singular system to that level; below 1e-4 the FP32 update can no longer be
// told from that noise (the FP64 update, TT_FLAG_FP64_SOLVE, resolves down to 1e-10)
#define TT_PIVOT_TOL32 1e-4f
#define TT_DET_KSPLIT 8     // K-chunks of the Gram in the deterministic mode
#define TT_DET_PARTS 8192   // capacity (CTAs) of the deterministic partial-sum buffers
size_t tt_chol64_smem(int s);           // shared memory of the FP64 Cholesky for s unknowns
size_t tt_trsm64_smem(int s, int nc);   // and of its triangular solves, nc right-hand sides per CTA

// (a + b) mod J for bucket indices a, b < J (any J)
__host__ __device__ __forceinline__ int tt_modj(int x, int J) { return x >= J ? x - J : x; }
#define TT_MAX_N 65536    // largest single mode size

// OCP FP8 E4M3 byte (low 8 bits of c) -> float: the hardware conversion to FP16 (exact: every E4M3
// value is an FP16 value; the format's NaN code S.1111.111 gives NaN), then FP16 -> FP32 (exact)
__device__ __forceinline__ float tt_e4m3_to_float(uint32_t c) {
  const unsigned short x = (unsigned short)(c & 0xFFu);
  float f;
  asm("{\n .reg .b32 h;\n .reg .b16 lo, hi;\n cvt.rn.f16x2.e4m3x2 h, %1;\n mov.b32 {lo, hi}, h;\n"
      " cvt.f32.f16 %0, lo;\n}\n"
      : "=f"(f)
      : "h"(x));
  return f;
}

struct TtPlan0;

// The hash / sign tables and fibre plans of one sketch draw. A context holds two: the current draw
// (its d_h, d_v, d_rplan ... fields) and a spare that each sweep fills, on its side stream, for the
// next sweep index, so that the next sweep starts with its plans ready.
struct TtDraw {
  int32_t* h = nullptr;
  int8_t* v = nullptr;
  uint32_t* rplan[TT_MAX_D] = {nullptr};
  int32_t* ulist[TT_MAX_D] = {nullptr};
  int64_t* ustart[TT_MAX_D] = {nullptr};
  int32_t* ucount[TT_MAX_D] = {nullptr};
  bool tables_valid = false;
  uint64_t tables_sweep = 0;
  bool rplan_valid[TT_MAX_D] = {false};
};

// Library-owned state of one problem shape (see tt_sketch_init).
struct tt_ctx {
  int d = 0;
  int64_t n[TT_MAX_D] = {0};
  int r[TT_MAX_D + 1] = {0};
  int J = 0, logJ = 0;  // logJ = -1 when J is not a power of two
  double lambda = 0.0;
  uint64_t seed = 0;
  int dtype = TT_F32;
  unsigned flags = 0;
  cudaStream_t stream = nullptr;
  std::string err;

  int64_t N = 0;             // number of tensor entries
  int64_t noff[TT_MAX_D + 1];  // offsets of mode tables (prefix sums of n)
  int64_t stride[TT_MAX_D + 1];  // stride[k] = prod_{s<k} n_s
  int smax = 0;              // max_k r[k]*r[k+1]
  int64_t nmax = 0;          // max_k n[k]

  // hash / sign tables of the current draw (device), sum_k n_k entries each
  int32_t* d_h = nullptr;
  int8_t* d_v = nullptr;
  bool tables_valid = false;   // d_h/d_v hold the draw for `tables_sweep`
  uint64_t tables_sweep = 0;
  bool user_tables = false;    // tables were set by tt_sketch_set_tables

  // mode-0 fiber plan (fibers grouped by destination row of Y_0)
  int64_t M0 = 0;              // number of mode-0 fibers, N / n_0
  uint32_t* d_plan0 = nullptr; // M0 entries: fiber index | sign in bit 31 (sorted by row)
  int64_t* d_plan0_off = nullptr;  // J + 1 row offsets into d_plan0
  int32_t* d_plan0_cursor = nullptr;  // d x J plan counts / scatter cursors (one row per mode)
  bool plan0_valid = false;

  // mode-k plans: mode-0 fibres of the modes other than 0 and k ("rest" fibres r), grouped by
  // their hash c_r = (sum_{s != 0, k} h_s(i_s)) mod J. Entry = index of the fibre at i_k = 0
  // (element offset / n_0), sign in bit 31. Distinct c values listed in ulist / ustart.
  int64_t R[TT_MAX_D] = {0};          // number of rest fibres of mode k
  uint32_t* d_rplan[TT_MAX_D] = {nullptr};
  int32_t* d_ulist[TT_MAX_D] = {nullptr};   // distinct c values (J entries max)
  int64_t* d_ustart[TT_MAX_D] = {nullptr};  // J + 1 starts into d_rplan[k]
  int32_t* d_ucount[TT_MAX_D] = {nullptr};  // number of distinct c values (device scalar)
  int64_t* d_rtmp = nullptr;                 // d x (J + 1) bucket offsets of the plan build
  bool rplan_valid[TT_MAX_D] = {false};
  float* d_Ypart = nullptr;                  // unused placeholder
  TtDraw spare;                              // the next sweep's draw (see TtDraw)
  cudaEvent_t ev_spare = nullptr;            // end of the spare's build on `side`
  bool spare_pending = false;

  // FFT sketches of the cores: for core j, (J/2+1) x s_j complex, frequency-major
  float2* d_ghat = nullptr;
  int64_t ghat_off[TT_MAX_D + 1];
  float2* d_twiddle = nullptr;   // J/2 twiddles exp(-2 pi i t / J)
  float2* d_twstage = nullptr;   // radix-4 stage twiddles exp(-2 pi i r m / (4 Ns)), per stage [m][r-1]
  float2* d_suffix = nullptr;    // for each k: (J/2+1) x r[k+1] complex (suffix R_{>k})
  int64_t suffix_off[TT_MAX_D + 1];
  float2* d_prefix = nullptr;    // (J/2+1) x rmax complex: prefix L_{<k}
  float2* d_prefix_tmp = nullptr;
  int rmax = 1;

  // dense workspaces
  float* d_SH = nullptr;       // J x smax (column-major)
  float* d_Y = nullptr;        // J x nmax, scratch for the autotuner's timed data sketches
  // the sweep's data sketches run on `side`, concurrently with the interface/solve chain on the
  // caller's stream: mode k's sketch goes to d_Yall + yoff[k] and signals ev_y[k]
  cudaStream_t side = nullptr;
  // the chain itself runs on `hi`, a highest-priority stream forked from (and joined back to) the
  // caller's stream, so that its small kernels get SM slots ahead of the data-sketch CTAs
  cudaStream_t hi = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool in_sweep = false;       // data sketches launched inside a sweep: finer work items
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_y[TT_MAX_D] = {nullptr};
  float* d_Yall = nullptr;
  int64_t yoff[TT_MAX_D + 1] = {0};
  float* d_gram = nullptr;     // (smax + nmax) x smax FP32 accumulators of [SH | Y]^T SH
  bool solve64 = false;        // the FP64 update (sigma = 0 or TT_FLAG_FP64_SOLVE)
  double* d_gram64 = nullptr;  // (smax + nmax) x smax FP64 accumulators, then L, when solve64
  // deterministic summation order (TT_FLAG_DETERMINISTIC, tt_det.cu)
  bool det = false;
  int* d_det_misc = nullptr;        // [0] bits of max |A|, [1] fixed-point exponent S, [2] A not finite
  int64_t* d_y64 = nullptr;         // int64 data-sketch accumulators, mode k at yoff[k]
  int32_t* d_det_bcnt = nullptr;    // deterministic plans: per range and key, counts then first slots
  uint2* d_det_kv = nullptr;        // deterministic plans: (key, plan entry) of every rest fibre
  void* d_gram_part = nullptr;      // TT_DET_KSPLIT K-chunk partials of the Gram (FP32 or FP64)
  double* d_part_err = nullptr;     // per-CTA partial sums of the relative error (2 per CTA)
  double* d_part_chg = nullptr;     // per-CTA partial sums of the change norms (2 per CTA)
  float* d_core_old = nullptr; // proximal centre copy (nmax * smax)
  double* d_changes = nullptr; // per (sweep, k): ||dG||^2, ||G||^2
  int* d_status = nullptr;     // device error flag (0 = ok, else TT_E* code)
  double* d_err_acc = nullptr; // rel-error accumulators (2 doubles)
  double* d_errs = nullptr;    // per-sweep rel-error accumulators (2 per sweep, changes_cap / d sweeps)
  double* d_ws_acc = nullptr;  // warm-start summary accumulators (2 doubles)
  float* d_rint = nullptr;     // right interfaces of the mode-0 fibres (N / n_0 x rint_r1p), rel error
  int rint_r1p = 0;            // r_1 rounded up to a multiple of 4
  float* d_slab_u = nullptr;   // u_t = G_2(i_2)...G_{d-1}(i_{d-1}) per slab (N / (n_0 n_1) x r_2), rel error
  double* d_xgram = nullptr;   // two 32 x 32 FP64 Gram matrices of the sparse relative error
  int changes_cap = 0;

  // measurement counters (tt_profile_*)
  int64_t launches = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_mode;   // mode of each recorded pair (pairs at 2i, 2i+1)
  int ev_used = 0;            // events in use
  int64_t prof_bytes = 0;

  // graph-capture mode (batched driver): tables are drawn from the device sweep counter
  // *d_sweep_ptr and the plans are rebuilt every sweep, with no host-side state checks.
  bool capture_mode = false;
  const uint64_t* d_sweep_ptr = nullptr;

  // The data sketches in d_Yall are those of the A of the running multi-sweep call under a draw
  // that does not change from sweep to sweep (TT_FLAG_FIXED_SKETCH or tables set by the caller):
  // later sweeps of the call reuse them. Cleared at the start and the end of every call.
  bool y_reuse = false;
  // Deterministic mode: the fixed-point scale S in d_det_misc is that of the A of the running
  // multi-sweep call (set by its first sweep outside graph capture; cleared with y_reuse), so the
  // later sweeps skip the max |A| pass.
  bool det_scale_reuse = false;

  // least bytes of A per work item of a data-sketch launch (0: items sized for one tensor alone,
  // about one per CTA slot). Contexts of a batch set it, so that a small tensor's launch takes few
  // CTAs and the launches of the batch's other tensors run beside it.
  int64_t item_bytes = 0;

  // autotuned parameters of the unfold kernel per mode (0 = default)
  int tune_seg_mult[TT_MAX_D] = {0};   // multiplier of the work-item count
  int tune_cta_per_sm[TT_MAX_D] = {0}; // CTAs per SM (1 or 2)

  uint64_t ws_bytes = 0;        // bytes of the workspaces planned at creation (tt_workspace_each)

  // host-buffer entry points (tt_host.cu, allocated on first use): two staging buffers for the
  // tensor (and its scales), so that the copy of the next call's tensor runs on copy_stream beside
  // this call's sweeps; ev_copied[b] ends the copy into buffer b, ev_consumed[b] the last kernel
  // that reads it. The results of calls not yet synchronised land in pinned host slots.
  void* d_A_stage[2] = {nullptr, nullptr};
  float* d_scales_stage[2] = {nullptr, nullptr};
  float* d_cores_stage[TT_MAX_D] = {nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_consumed[2] = {nullptr, nullptr};
  bool consumed_recorded[2] = {false, false};
  int stage_next = 0;
  struct HostPending {
    double* rel_change_out;
    double* rel_error_out;
    int nsweeps;
    int slot;
  };
  std::vector<HostPending> pending;   // calls enqueued and not yet synchronised, in order
  unsigned char* h_slots = nullptr;   // pinned: TT_HOST_SLOTS result slots (status, error, changes)
  cudaEvent_t ev_slot[4] = {nullptr, nullptr, nullptr, nullptr};  // a slot's results have landed
  int slot_next = 0;
  int host_error = 0;                 // first failure of a call finished but not yet reported
};
#define TT_HOST_SLOTS 4
// least bytes of A per data-sketch work item for the tensors of a batch (tt_ctx::item_bytes)
#define TT_BATCH_ITEM_BYTES (1024 * 1024)
// bytes of one pinned result slot: the status word, the two error sums, 2 d change sums per sweep
size_t tt_host_slot_bytes(const tt_ctx* c);
// the host-buffer calls' resources (tt_host.cu)
void tt_host_free(tt_ctx* c);

// ---------------------------------------------------------------------------------------------
// hashing (SplitMix64 chain, see tt_sketch.h)

__host__ __device__ inline uint64_t tt_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t tt_step(uint64_t z, uint64_t f) {
  return tt_mix64(z + (f + 1ull) * 0x9E3779B97F4A7C15ull);
}
__host__ __device__ inline uint64_t tt_word(uint64_t seed, uint64_t sweep, uint64_t mode,
                                            uint64_t stream, uint64_t i) {
  return tt_step(tt_step(tt_step(tt_step(seed, sweep), mode), stream), i);
}

// ---------------------------------------------------------------------------------------------
// host helpers (tt_context.cu)

int tt_fail(tt_ctx* c, int code, const char* fmt, ...);
int tt_cuda_check(tt_ctx* c, cudaError_t e, const char* what);
#define TT_CUDA(ctx, call)                                   \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return tt_cuda_check(ctx, _e, #call); \
  } while (0)
#define TT_LAUNCH(ctx, what)                                          \
  do {                                                                \
    cudaError_t _e = cudaGetLastError();                              \
    if (_e != cudaSuccess) return tt_cuda_check(ctx, _e, what);       \
    ++(ctx)->launches;                                                \
  } while (0)

int tt_ensure_tables(tt_ctx* c, uint64_t sweep);
// Build the tables and plans of draw `sweep` into the spare on the side stream (no-op in graph
// capture, with user tables or a fixed sketch, or when the spare already holds that draw).
int tt_prepare_next_draw(tt_ctx* c, uint64_t sweep);
void tt_swap_draw(tt_ctx* c);
int tt_ensure_plan0(tt_ctx* c);
int tt_ensure_rplan(tt_ctx* c, int k);

// kernels' host entry points (one translation unit each)
int tt_launch_unfold(tt_ctx* c, const void* A, const float* scales, int k, float* Y);
int tt_launch_unfold_coo(tt_ctx* c, const int32_t* idx, const float* val, int64_t nnz, int k, float* const* Y);
// d_err_acc[0..2] = sum val^2, sum val X(i), ||X||^2 of a sparse tensor in coordinate form
int tt_launch_rel_error_coo(tt_ctx* c, const int32_t* idx, const float* val, int64_t nnz, float* const* cores);
int tt_launch_core_fft(tt_ctx* c, const float* core, int j);
int tt_launch_core_ffts(tt_ctx* c, float* const* cores);  // all d cores, one launch
int tt_launch_suffixes(tt_ctx* c);
int tt_launch_prefix_step(tt_ctx* c, int j);
// S H_k from the prefix and suffix chains; `zero` (nzero floats, optional) is zeroed on the side
int tt_launch_interface_from_chain(tt_ctx* c, int k, float* SH, float* zero = nullptr, int64_t nzero = 0);
int tt_launch_prox_update(tt_ctx* c, const float* Y, const float* SH, float* core, int k,
                          double* change_slot,
                          bool gram_zeroed = false);  // gram_zeroed: d_gram already zero
// deterministic mode (tt_det.cu): the data sketches of the modes in `mask` in int64 fixed point
// (Y[k] written for those modes, ev[k] recorded on c->stream after Y[k] when ev is given), the
// ordered sum of per-CTA partials into acc[0..1], and the ordered sum of the Gram's K-chunk partials
int tt_launch_unfold_det(tt_ctx* c, const void* A, const float* scales, unsigned mask, float* const* Y,
                         cudaEvent_t* ev = nullptr);
int tt_launch_sum_partials(tt_ctx* c, const double* part, int nparts, double* acc);
int tt_launch_gram_reduce(tt_ctx* c, const void* P, int nz, int64_t count, void* C, bool f64);
// tensor-core Gram of the FP32 update (tt_gram_tc.cu): whether the shape and pointers suit TMA,
// and C (zeroed, or P's ordered sum in the deterministic mode) = [S H | Y]^T S H in TF32 x 3
// (split3) or TF32 x 1
bool tt_gram_tc_fits(int J, int s, const void* SH, const void* Y);
int tt_launch_gram_tc(tt_ctx* c, const float* SH, const float* Y, int s, int n, float* C, float* P, bool split3,
                      int* nz_out);
// the same update in FP64 (FP64 Gram, Cholesky and triangular solves; tt_solve64.cu)
int tt_launch_prox_update64(tt_ctx* c, const float* Y, const float* SH, float* core, int k, double* change_slot,
                            bool gram_zeroed);
int tt_launch_qr_left(tt_ctx* c, float* core_k, float* core_k1, int k);
int tt_launch_lq_right(tt_ctx* c, float* core_km1, float* core_k, int k);
int tt_launch_lq_sweep(tt_ctx* c, float* const* cores);  // all right-to-left steps
int tt_launch_rel_error(tt_ctx* c, const void* A, const float* scales, float* const* cores,
                        double* acc = nullptr);  // acc: 2 doubles (default: the context's)
int tt_read_status(tt_ctx* c);
int tt_reset_status(tt_ctx* c);
int tt_check_cores(tt_ctx* c, float* const* cores);
// A non-null; slice scales given exactly for FP8 storage
int tt_check_data(tt_ctx* c, const void* A, const float* scales);

#define TT_TRY(x)            \
  do {                       \
    int _rc = (x);           \
    if (_rc) return _rc;     \
  } while (0)
int tt_one_sweep(tt_ctx* c, const void* A, const float* scales, float* const* cores, uint64_t sweep,
                 double* change_slots, float* const* Ygiven = nullptr);
int tt_prof_begin(tt_ctx* c, int k);   // record a start event when profiling (returns TT_OK)
int tt_prof_end(tt_ctx* c);
int tt_elem_bytes(int dtype);
// number of SMs of the current device (queried once per device; 152 if the query fails)
int tt_sm_count();
// TT_ENOMEM (with a message) when the context's workspaces plus `extra` bytes would exceed the
// process-wide cap of tt_set_workspace_limit; TT_OK otherwise
int tt_check_workspace_cap(tt_ctx* c, uint64_t extra);

// element loads of the data tensor in its storage type, converted to float
template <int DT>
struct TtElem;
