// Context lifetime, parameter validation, hash/sign draws and the mode-0 fiber plan.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <new>
#include <vector>

#include <utility>

#include "tt_internal.cuh"

int tt_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 152;
  if (dev < 64 && cache[dev] > 0) return cache[dev];
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  if (dev < 64) cache[dev] = sms;
  return sms;
}

int tt_fail(tt_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int tt_cuda_check(tt_ctx* c, cudaError_t e, const char* what) {
  int code = (e == cudaErrorMemoryAllocation) ? TT_ENOMEM : TT_ECUDA;
  return tt_fail(c, code, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------------------------
// hash / sign tables (Sec. 2.2): one thread per (mode, index)

struct TabArgs {
  int64_t noff[TT_MAX_D + 1];
  int d;
};

__global__ void k_gen_tables(uint64_t seed, uint64_t sweep, TabArgs a, int J, int32_t* h, int8_t* v) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= a.noff[a.d]) return;
  int k = 0;
  while (g >= a.noff[k + 1]) ++k;
  uint64_t i = (uint64_t)(g - a.noff[k]);
  uint64_t wh = tt_word(seed, sweep, (uint64_t)k, 0ull, i);
  uint64_t wv = tt_word(seed, sweep, (uint64_t)k, 1ull, i);
  h[g] = (int32_t)((J & (J - 1)) == 0 ? (wh & (uint64_t)(J - 1)) : wh % (uint64_t)J);
  v[g] = (wv >> 63) ? (int8_t)-1 : (int8_t)1;
}

__global__ void k_gen_tables_dev(uint64_t seed, const uint64_t* sweep_ptr, int fixed, TabArgs a, int J,
                                 int32_t* h, int8_t* v) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= a.noff[a.d]) return;
  const uint64_t sweep = fixed ? 0ull : *sweep_ptr;
  int k = 0;
  while (g >= a.noff[k + 1]) ++k;
  uint64_t i = (uint64_t)(g - a.noff[k]);
  const uint64_t wh = tt_word(seed, sweep, (uint64_t)k, 0ull, i);
  h[g] = (int32_t)((J & (J - 1)) == 0 ? (wh & (uint64_t)(J - 1)) : wh % (uint64_t)J);
  v[g] = (tt_word(seed, sweep, (uint64_t)k, 1ull, i) >> 63) ? (int8_t)-1 : (int8_t)1;
}

void tt_swap_draw(tt_ctx* c) {
  TtDraw& o = c->spare;
  std::swap(c->d_h, o.h);
  std::swap(c->d_v, o.v);
  for (int k = 0; k < TT_MAX_D; ++k) {
    std::swap(c->d_rplan[k], o.rplan[k]);
    std::swap(c->d_ulist[k], o.ulist[k]);
    std::swap(c->d_ustart[k], o.ustart[k]);
    std::swap(c->d_ucount[k], o.ucount[k]);
    std::swap(c->rplan_valid[k], o.rplan_valid[k]);
  }
  std::swap(c->tables_valid, o.tables_valid);
  std::swap(c->tables_sweep, o.tables_sweep);
}

int tt_ensure_tables(tt_ctx* c, uint64_t sweep) {
  if (c->user_tables) return TT_OK;
  if (c->capture_mode) {  // sweep index read on the device at replay time
    TabArgs a;
    for (int k = 0; k <= c->d; ++k) a.noff[k] = c->noff[k];
    a.d = c->d;
    const int64_t total = c->noff[c->d];
    k_gen_tables_dev<<<(int)((total + 255) / 256), 256, 0, c->stream>>>(
        c->seed, c->d_sweep_ptr, (c->flags & TT_FLAG_FIXED_SKETCH) ? 1 : 0, a, c->J, c->d_h, c->d_v);
    TT_LAUNCH(c, "k_gen_tables_dev");
    for (int k = 0; k < TT_MAX_D; ++k) c->rplan_valid[k] = false;
    return TT_OK;
  }
  if (c->flags & TT_FLAG_FIXED_SKETCH) sweep = 0;
  if (c->tables_valid && c->tables_sweep == sweep) return TT_OK;
  if (c->spare.tables_valid && c->spare.tables_sweep == sweep) {  // built ahead by the last sweep
    tt_swap_draw(c);
    if (c->spare_pending) TT_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_spare, 0));
    return TT_OK;
  }
  if (c->spare_pending) TT_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_spare, 0));  // shared scratch
  TabArgs a;
  for (int k = 0; k <= c->d; ++k) a.noff[k] = c->noff[k];
  a.d = c->d;
  int64_t total = c->noff[c->d];
  int threads = 256;
  int blocks = (int)((total + threads - 1) / threads);
  k_gen_tables<<<blocks, threads, 0, c->stream>>>(c->seed, sweep, a, c->J, c->d_h, c->d_v);
  TT_LAUNCH(c, "k_gen_tables");
  c->tables_valid = true;
  c->tables_sweep = sweep;
  for (int k = 0; k < TT_MAX_D; ++k) c->rplan_valid[k] = false;
  return TT_OK;
}

// ---------------------------------------------------------------------------------------------
// per-mode fibre plans. For mode k, the "rest" fibres r enumerate the modes s = 1..d-1, s != k
// (mode-0 fibres of the sub-tensor A(:, .., i_k = 0, ..)), lowest mode fastest. Each gets its hash
// c_r = (sum_s h_s(i_s)) mod J, sign prod_s v_s(i_s) and element offset sum_s i_s stride_s. The
// plan lists the fibres grouped by c_r (counting sort) plus the distinct c values in order.
// For k = 0 the groups are the rows of Y_0 (every mode-0 fibre lands in row c_r).

struct RPlanArgs {
  int64_t n[TT_MAX_D];
  int64_t stride[TT_MAX_D];
  int64_t fstride[TT_MAX_D];  // stride[s] / n[0]: mode-0 fibres per step of mode s (s >= 1)
  int64_t noff[TT_MAX_D + 1];
  int d, k, J;
  int64_t R;
};

// Mixed-radix counter over the rest modes of a plan (lowest mode fastest). A thread decomposes
// its first fibre index and its stride once (divisions), then advances with digit additions and
// carries only; hash, sign and offset are updated incrementally from per-digit table lookups.
struct RestWalker {
  int dig[TT_MAX_D];    // current digits, one per rest mode
  int sdig[TT_MAX_D];   // digits of the stride
  int nm;               // number of rest modes
  int md[TT_MAX_D];     // mode of each digit
  __device__ void init(const RPlanArgs& a, int64_t r, int64_t stride) {
    nm = 0;
    for (int s = 1; s < a.d; ++s)
      if (s != a.k) md[nm++] = s;
    int64_t rem = r, st = stride;
    for (int q = 0; q < nm; ++q) {
      const int64_t n = a.n[md[q]];
      dig[q] = (int)(rem % n);
      rem /= n;
      sdig[q] = (int)(st % n);
      st /= n;
    }
  }
  __device__ void advance(const RPlanArgs& a) {
    int carry = 0;
    for (int q = 0; q < nm; ++q) {
      const int n = (int)a.n[md[q]];
      int x = dig[q] + sdig[q] + carry;
      carry = 0;
      while (x >= n) {
        x -= n;
        ++carry;
      }
      dig[q] = x;
    }
  }
  __device__ void entry(const RPlanArgs& a, const int32_t* __restrict__ h, const int8_t* __restrict__ v,
                        int* key, int* neg, int64_t* off) const {
    int b = 0, sg = 0;
    int64_t o = 0;
    for (int q = 0; q < nm; ++q) {
      const int s = md[q], i = dig[q];
      b += h[a.noff[s] + i];
      sg ^= (v[a.noff[s] + i] < 0);
      o += (int64_t)i * a.fstride[s];
    }
    *key = (a.J & (a.J - 1)) == 0 ? (b & (a.J - 1)) : b % a.J;
    *neg = sg;
    *off = o;  // mode-0 fibre index at i_k = 0
  }
};

// Plans of all modes are built together (the hashes of a sweep are known at its start): one
// launch counts, one scans, one scatters, over a grid that concatenates the blocks of every mode.
// Modes with few rest fibres (R <= 8 J) use global atomics per fibre; the others a per-block
// shared-memory histogram (one global atomic per non-empty bucket and block), with at least J
// fibres per block (measured at J = 4096 and 10^6 fibres: J per block 632 us per sweep, 2 J
// 642 us, 4 J 682 us, 8 J 753 us -- more blocks beat fewer bucket atomics).
#define TT_PLAN_BLOCK 8192  // fibres per block in histogram mode
struct RPlanAll {
  RPlanArgs m[TT_MAX_D];
  int64_t bstart[TT_MAX_D + 1];  // first block of each mode
  int pb[TT_MAX_D];              // fibres per block
  int direct[TT_MAX_D];          // 1: global atomics, no shared histogram
  int d;
};
struct RPlanOut {
  int32_t* ulist[TT_MAX_D];
  int64_t* ustart[TT_MAX_D];
  int32_t* ucount[TT_MAX_D];
  uint32_t* plan[TT_MAX_D];
};

__device__ __forceinline__ int plan_mode(const RPlanAll& P) {
  int m = 0;
  while (m + 1 < P.d && (int64_t)blockIdx.x >= P.bstart[m + 1]) ++m;
  return m;
}

__global__ void k_rplan_count(RPlanAll P, const int32_t* h, const int8_t* v, int32_t* count) {
  extern __shared__ int hist[];
  const int m = plan_mode(P);
  const RPlanArgs& a = P.m[m];
  const int64_t r0 = ((int64_t)blockIdx.x - P.bstart[m]) * P.pb[m], r1 = min(a.R, r0 + P.pb[m]);
  int32_t* cnt = count + (int64_t)m * a.J;
  RestWalker wk;
  wk.init(a, r0 + threadIdx.x, blockDim.x);
  if (P.direct[m]) {
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x, wk.advance(a)) {
      int key, neg;
      int64_t off;
      wk.entry(a, h, v, &key, &neg, &off);
      atomicAdd(&cnt[key], 1);
    }
    return;
  }
  for (int i = threadIdx.x; i < a.J; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x, wk.advance(a)) {
    int key, neg;
    int64_t off;
    wk.entry(a, h, v, &key, &neg, &off);
    atomicAdd(&hist[key], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.J; i += blockDim.x)
    if (hist[i]) atomicAdd(&cnt[i], hist[i]);
}

// exclusive scans of the counts and of the non-empty flags (one block of 1024 threads per mode,
// warp-shuffle scans); the counts become the scatter cursors
__device__ __forceinline__ int64_t warp_incl_scan(int64_t x) {
  const int lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}
__global__ void k_rplan_scan(int J, int32_t* count_all, int64_t* off_all, RPlanOut o) {
  __shared__ int64_t wsum[32], wun[32];
  const int m = blockIdx.x;
  int32_t* count = count_all + (int64_t)m * J;
  int64_t* off = off_all + (int64_t)m * (J + 1);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int per = (J + 1023) / 1024;
  const int lo = min(J, t * per), hi = min(J, (t + 1) * per);
  int64_t s = 0, u = 0;
  for (int i = lo; i < hi; ++i) {
    s += count[i];
    u += count[i] > 0;
  }
  const int64_t si = warp_incl_scan(s), ui = warp_incl_scan(u);
  if (lane == 31) {
    wsum[warp] = si;
    wun[warp] = ui;
  }
  __syncthreads();
  if (warp == 0) {
    const int64_t a1 = warp_incl_scan(wsum[lane]), a2 = warp_incl_scan(wun[lane]);
    wsum[lane] = a1;
    wun[lane] = a2;
  }
  __syncthreads();
  int64_t base = (warp ? wsum[warp - 1] : 0) + si - s;
  int ub = (int)((warp ? wun[warp - 1] : 0) + ui - u);
  for (int i = lo; i < hi; ++i) {
    const int ci = count[i];
    off[i] = base;
    if (ci > 0) {
      o.ulist[m][ub] = i;
      o.ustart[m][ub] = base;
      ++ub;
    }
    base += ci;
    count[i] = 0;
  }
  if (t == 1023) {
    off[J] = wsum[31];
    o.ustart[m][wun[31]] = wsum[31];
    *o.ucount[m] = (int32_t)wun[31];
  }
}

// Scatter: a histogram-mode block reserves, per non-empty bucket, a range of the bucket's slots
// with one global atomic, then places its fibres with shared-memory cursors; a direct-mode block
// takes one global cursor increment per fibre.
__global__ void k_rplan_scatter(RPlanAll P, const int32_t* h, const int8_t* v, const int64_t* off_all,
                                int32_t* cursor_all, RPlanOut o) {
  extern __shared__ int hist[];
  const int m = plan_mode(P);
  const RPlanArgs& a = P.m[m];
  const int64_t r0 = ((int64_t)blockIdx.x - P.bstart[m]) * P.pb[m], r1 = min(a.R, r0 + P.pb[m]);
  int32_t* cursor = cursor_all + (int64_t)m * a.J;
  const int64_t* off = off_all + (int64_t)m * (a.J + 1);
  uint32_t* plan = o.plan[m];
  RestWalker wk;
  wk.init(a, r0 + threadIdx.x, blockDim.x);
  if (P.direct[m]) {
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x, wk.advance(a)) {
      int key, neg;
      int64_t ofs;
      wk.entry(a, h, v, &key, &neg, &ofs);
      const int pos = atomicAdd(&cursor[key], 1);
      plan[off[key] + pos] = (uint32_t)ofs | ((uint32_t)neg << 31);
    }
    return;
  }
  for (int i = threadIdx.x; i < a.J; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x, wk.advance(a)) {
    int key, neg;
    int64_t ofs;
    wk.entry(a, h, v, &key, &neg, &ofs);
    atomicAdd(&hist[key], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.J; i += blockDim.x)
    if (hist[i]) hist[i] = atomicAdd(&cursor[i], hist[i]);  // start of this block's slots
  __syncthreads();
  wk.init(a, r0 + threadIdx.x, blockDim.x);
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x, wk.advance(a)) {
    int key, neg;
    int64_t ofs;
    wk.entry(a, h, v, &key, &neg, &ofs);
    const int pos = atomicAdd(&hist[key], 1);
    plan[off[key] + pos] = (uint32_t)ofs | ((uint32_t)neg << 31);  // fibre index | sign
  }
}

// Deterministic plan (TT_FLAG_DETERMINISTIC): the fibres of each group in ascending fibre index
// (the rest index r is walked in order and the fibre offset grows with r), so that the data-sketch
// kernels sum every run in the same order on every call. A mode's rest fibres are split into
// contiguous ranges: k_rplan_dcount writes each range's key counts to its row of `bcnt` and every
// fibre's (key, plan entry) to `kv`; k_rplan_dbase turns the rows into the range's first slot per
// key (off[key] plus the counts of the earlier ranges, in range order); k_rplan_dscatter walks
// each range 32 fibres at a time (one warp), ranking equal keys by lane (__match_any_sync) on top
// of a per-key cursor in shared memory.
struct DPlan {
  int64_t bstart[TT_MAX_D + 1];  // first range (block) of each mode
  int64_t per[TT_MAX_D];         // rest fibres per range
  int64_t R[TT_MAX_D];           // rest fibres of each mode
  int64_t roff[TT_MAX_D];        // first entry of each mode in kv
};

// deterministic plans: rest fibres per range (at least 256; at most 2^21 / J ranges per mode, in
// [32, 1024], which bounds the count table to 8 MB per mode), the ranges of all modes, and the
// rest fibres of all modes (entries of kv)
static int64_t dplan_per(int64_t R, int J) {
  const int64_t nr = std::max<int64_t>(32, std::min<int64_t>(1024, (1 << 21) / J));
  return std::max<int64_t>(256, (R + nr - 1) / nr);
}
static int64_t dplan_ranges(const tt_ctx* c) {
  int64_t t = 0;
  for (int m = 0; m < c->d; ++m) {
    const int64_t per = dplan_per(c->R[m], c->J);
    t += std::max<int64_t>(1, (c->R[m] + per - 1) / per);
  }
  return t;
}
static int64_t dplan_fibres(const tt_ctx* c) {
  int64_t t = 0;
  for (int m = 0; m < c->d; ++m) t += c->R[m];
  return t;
}

__device__ __forceinline__ int dplan_mode(const DPlan& D, int d) {
  int m = 0;
  while (m + 1 < d && (int64_t)blockIdx.x >= D.bstart[m + 1]) ++m;
  return m;
}

__global__ void k_rplan_dcount(RPlanAll P, DPlan D, const int32_t* h, const int8_t* v, int32_t* bcnt, uint2* kv) {
  extern __shared__ int hist[];
  const int m = dplan_mode(D, P.d);
  const RPlanArgs& a = P.m[m];
  const int64_t r0 = ((int64_t)blockIdx.x - D.bstart[m]) * D.per[m], r1 = min(a.R, r0 + D.per[m]);
  for (int i = threadIdx.x; i < a.J; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  uint2* out = kv + D.roff[m];
  RestWalker wk;
  wk.init(a, r0 + threadIdx.x, blockDim.x);
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x, wk.advance(a)) {
    int key, neg;
    int64_t ofs;
    wk.entry(a, h, v, &key, &neg, &ofs);
    atomicAdd(&hist[key], 1);  // counts: the order of the adds does not matter
    out[r] = make_uint2((uint32_t)key, (uint32_t)ofs | ((uint32_t)neg << 31));
  }
  __syncthreads();
  int32_t* row = bcnt + (int64_t)blockIdx.x * a.J;
  for (int i = threadIdx.x; i < a.J; i += blockDim.x) row[i] = hist[i];
}

// One CTA per (mode, 32 keys), 32 x 32 threads: thread (x, y) takes key 32 t + x over the y-th
// of 32 contiguous slices of the mode's ranges. It sums its slice's counts, the slice totals are
// scanned in y order, and the slice is walked again, each count replaced by its range's first
// slot: off[key] plus the counts of all earlier ranges. Loads go eight at a time.
__global__ void __launch_bounds__(1024) k_rplan_dbase(DPlan D, int J, const int64_t* off_all, int32_t* bcnt) {
  __shared__ int64_t part[32][33];
  const int tiles = (J + 31) / 32;
  const int m = blockIdx.x / tiles;
  const int key = (blockIdx.x - m * tiles) * 32 + threadIdx.x;
  const int64_t rb = D.bstart[m], nr = D.bstart[m + 1] - rb;
  const int64_t per_t = (nr + 31) / 32;
  const int64_t b0 = min(rb + nr, rb + threadIdx.y * per_t), b1 = min(rb + nr, b0 + per_t);
  const bool ok = key < J;
  int64_t s = 0;
  if (ok)
    for (int64_t b = b0; b < b1; b += 8) {
      int32_t cnt[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) cnt[u] = b + u < b1 ? bcnt[(b + u) * J + key] : 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) s += cnt[u];
    }
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (!ok) return;
  int64_t pos = off_all[(int64_t)m * (J + 1) + key];
  for (int y = 0; y < (int)threadIdx.y; ++y) pos += part[y][threadIdx.x];
  for (int64_t b = b0; b < b1; b += 8) {
    int32_t cnt[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) cnt[u] = b + u < b1 ? bcnt[(b + u) * J + key] : 0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (b + u < b1) {
        bcnt[(b + u) * J + key] = (int32_t)pos;
        pos += cnt[u];
      }
  }
}

// one warp per range: fibres in index order, equal keys within a step of 32 ranked by lane; the
// (key, entry) pairs of four steps are loaded before the four steps run
__global__ void __launch_bounds__(32) k_rplan_dscatter(DPlan D, int d, int J, const uint2* kv, const int32_t* bbase,
                                                       RPlanOut o) {
  extern __shared__ int cur[];
  const int m = dplan_mode(D, d);
  const int64_t r0 = ((int64_t)blockIdx.x - D.bstart[m]) * D.per[m], r1 = min(D.R[m], r0 + D.per[m]);
  const int32_t* base = bbase + (int64_t)blockIdx.x * J;
  for (int i = threadIdx.x; i < J; i += 32) cur[i] = base[i];
  __syncwarp();
  const int lane = threadIdx.x;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t* plan = o.plan[m];
  const uint2* src = kv + D.roff[m];
  for (int64_t rb = r0; rb < r1; rb += 128) {
    uint2 e[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t r = rb + 32 * u + lane;
      e[u] = r < r1 ? src[r] : make_uint2(0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool ok = rb + 32 * u + lane < r1;
      const int key = ok ? (int)e[u].x : -1 - lane;  // lanes past the range: a key no other lane has
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int rank = __popc(peers & lt);
      if (ok) plan[cur[key] + rank] = e[u].y;
      __syncwarp();
      if (ok && rank == 0) cur[key] += __popc(peers);
      __syncwarp();
    }
  }
}

// Plans of every mode for the current tables. In graph-capture mode with per-sweep draws the
// plans are rebuilt at the sweep's first data sketch (mode 0) and reused by the other modes.
int tt_ensure_rplan(tt_ctx* c, int k) {
  const bool redraw = c->capture_mode && !(c->flags & TT_FLAG_FIXED_SKETCH) && !c->user_tables;
  if (redraw ? k != 0 : c->rplan_valid[k]) return TT_OK;
  RPlanAll P;
  RPlanOut o;
  P.d = c->d;
  P.bstart[0] = 0;
  for (int m = 0; m < c->d; ++m) {
    RPlanArgs& a = P.m[m];
    for (int s = 0; s < c->d; ++s) {
      a.n[s] = c->n[s];
      a.stride[s] = c->stride[s];
      a.fstride[s] = c->stride[s] / c->n[0];
    }
    for (int s = 0; s <= c->d; ++s) a.noff[s] = c->noff[s];
    a.d = c->d;
    a.k = m;
    a.J = c->J;
    a.R = c->R[m];
    P.direct[m] = a.R <= 8 * (int64_t)c->J;
    P.pb[m] = P.direct[m] ? 1024
                          : (int)std::max<int64_t>((int64_t)c->J, std::min<int64_t>(TT_PLAN_BLOCK, (a.R + 303) / 304));
    P.bstart[m + 1] = P.bstart[m] + std::max<int64_t>(1, (a.R + P.pb[m] - 1) / P.pb[m]);
    o.ulist[m] = c->d_ulist[m];
    o.ustart[m] = c->d_ustart[m];
    o.ucount[m] = c->d_ucount[m];
    o.plan[m] = c->d_rplan[m];
  }
  int32_t* count = c->d_plan0_cursor;
  if (c->spare_pending && c->stream != c->side) TT_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_spare, 0));
  TT_CUDA(c, cudaMemsetAsync(count, 0, sizeof(int32_t) * c->J * c->d, c->stream));
  const size_t hsm = sizeof(int) * c->J;
  if (hsm > 48 * 1024) {
    TT_CUDA(c, cudaFuncSetAttribute(k_rplan_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
    TT_CUDA(c, cudaFuncSetAttribute(k_rplan_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
  }
  const int blocks = (int)P.bstart[c->d];
  k_rplan_count<<<blocks, 512, hsm, c->stream>>>(P, c->d_h, c->d_v, count);
  TT_LAUNCH(c, "k_rplan_count");
  k_rplan_scan<<<c->d, 1024, 0, c->stream>>>(c->J, count, c->d_rtmp, o);
  TT_LAUNCH(c, "k_rplan_scan");
  if (c->det) {  // fibres of each group in index order
    DPlan D;
    D.bstart[0] = 0;
    int64_t roff = 0;
    for (int m = 0; m < c->d; ++m) {
      D.per[m] = dplan_per(c->R[m], c->J);
      D.bstart[m + 1] = D.bstart[m] + std::max<int64_t>(1, (c->R[m] + D.per[m] - 1) / D.per[m]);
      D.R[m] = c->R[m];
      D.roff[m] = roff;
      roff += c->R[m];
    }
    if (hsm > 48 * 1024) {
      TT_CUDA(c, cudaFuncSetAttribute(k_rplan_dcount, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
      TT_CUDA(c, cudaFuncSetAttribute(k_rplan_dscatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
    }
    const int nr = (int)D.bstart[c->d];
    k_rplan_dcount<<<nr, 256, hsm, c->stream>>>(P, D, c->d_h, c->d_v, c->d_det_bcnt, c->d_det_kv);
    TT_LAUNCH(c, "k_rplan_dcount");
    k_rplan_dbase<<<c->d * ((c->J + 31) / 32), dim3(32, 32), 0, c->stream>>>(D, c->J, c->d_rtmp, c->d_det_bcnt);
    TT_LAUNCH(c, "k_rplan_dbase");
    k_rplan_dscatter<<<nr, 32, hsm, c->stream>>>(D, c->d, c->J, c->d_det_kv, c->d_det_bcnt, o);
    TT_LAUNCH(c, "k_rplan_dscatter");
  } else {
    k_rplan_scatter<<<blocks, 512, hsm, c->stream>>>(P, c->d_h, c->d_v, c->d_rtmp, count, o);
    TT_LAUNCH(c, "k_rplan_scatter");
  }
  for (int m = 0; m < c->d; ++m) c->rplan_valid[m] = true;
  return TT_OK;
}

int tt_ensure_plan0(tt_ctx* c) { return tt_ensure_rplan(c, 0); }

int tt_prepare_next_draw(tt_ctx* c, uint64_t sweep) {
  // (the deterministic mode's plans too: tt_ensure_rplan builds them in index order)
  if (c->capture_mode || c->user_tables || (c->flags & TT_FLAG_FIXED_SKETCH)) return TT_OK;
  bool ready = c->spare.tables_valid && c->spare.tables_sweep == sweep;
  for (int k = 0; k < c->d; ++k) ready = ready && c->spare.rplan_valid[k];
  if (ready) return TT_OK;
  tt_swap_draw(c);  // build into the spare through the current-draw fields
  cudaStream_t s0 = c->stream;
  c->stream = c->side;
  c->tables_valid = false;
  int rc = tt_ensure_tables(c, sweep);
  if (rc == TT_OK) rc = tt_ensure_rplan(c, 0);
  cudaError_t e = cudaEventRecord(c->ev_spare, c->side);
  c->stream = s0;
  tt_swap_draw(c);
  if (rc == TT_OK && e != cudaSuccess) rc = tt_cuda_check(c, e, "cudaEventRecord");
  if (rc != TT_OK) {
    c->spare.tables_valid = false;
    return rc;
  }
  c->spare_pending = true;
  return TT_OK;
}

// ---------------------------------------------------------------------------------------------
// lifetime

static void free_all(tt_ctx* c) {
  void* ps[] = {c->d_h, c->d_v, c->d_plan0, c->d_plan0_off, c->d_plan0_cursor, c->d_ghat,
                c->d_twiddle, c->d_twstage, c->d_suffix, c->d_prefix, c->d_prefix_tmp, c->d_SH, c->d_Y,
                c->d_gram, c->d_core_old, c->d_changes, c->d_status, c->d_err_acc, c->d_errs, c->d_ws_acc, c->d_rint, c->d_slab_u, c->d_Yall, c->d_xgram, c->d_gram64,
                c->d_det_misc, c->d_y64, c->d_gram_part, c->d_part_err, c->d_part_chg, c->d_det_bcnt, c->d_det_kv};
  for (void* p : ps)
    if (p) cudaFree(p);
  tt_host_free(c);
  void* sp[] = {c->spare.h, c->spare.v};
  for (void* p : sp)
    if (p) cudaFree(p);
  if (c->ev_spare) cudaEventDestroy(c->ev_spare);
  for (int k = 0; k < TT_MAX_D; ++k) {
    if (c->spare.rplan[k]) cudaFree(c->spare.rplan[k]);
    if (c->spare.ulist[k]) cudaFree(c->spare.ulist[k]);
    if (c->spare.ustart[k]) cudaFree(c->spare.ustart[k]);
    if (c->spare.ucount[k]) cudaFree(c->spare.ucount[k]);
  }
  for (int k = 0; k < TT_MAX_D; ++k) {
    if (c->d_rplan[k]) cudaFree(c->d_rplan[k]);
    if (c->d_ulist[k]) cudaFree(c->d_ulist[k]);
    if (c->d_ustart[k]) cudaFree(c->d_ustart[k]);
    if (c->d_ucount[k]) cudaFree(c->d_ucount[k]);
  }
  if (c->d_rtmp) cudaFree(c->d_rtmp);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (int k = 0; k < TT_MAX_D; ++k)
    if (c->ev_y[k]) cudaEventDestroy(c->ev_y[k]);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->hi) cudaStreamDestroy(c->hi);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
}

// Every device workspace of a context, in allocation order: f(&pointer, bytes). Used twice by
// tt_sketch_init: to sum the sizes (the cap of tt_set_workspace_limit is checked before any CUDA
// call) and to allocate. Fills the size bookkeeping of the context (R, yoff, changes_cap,
// rint_r1p) as it goes.
template <typename F>
static void tt_workspace_each(tt_ctx* c, F&& A) {
  A((void**)&c->d_h, sizeof(int32_t) * c->noff[c->d]);
  A((void**)&c->d_v, sizeof(int8_t) * c->noff[c->d]);
  A((void**)&c->d_plan0_cursor, sizeof(int32_t) * c->J * c->d);
  A((void**)&c->d_rtmp, sizeof(int64_t) * (c->J + 1) * c->d);
  for (int k = 0; k < c->d; ++k) {
    c->R[k] = c->N / (c->n[0] * (k == 0 ? 1 : c->n[k]));
    A((void**)&c->d_rplan[k], sizeof(uint32_t) * c->R[k]);
    A((void**)&c->d_ulist[k], sizeof(int32_t) * c->J);
    A((void**)&c->d_ustart[k], sizeof(int64_t) * (c->J + 1));
    A((void**)&c->d_ucount[k], sizeof(int32_t));
    A((void**)&c->spare.rplan[k], sizeof(uint32_t) * c->R[k]);
    A((void**)&c->spare.ulist[k], sizeof(int32_t) * c->J);
    A((void**)&c->spare.ustart[k], sizeof(int64_t) * (c->J + 1));
    A((void**)&c->spare.ucount[k], sizeof(int32_t));
  }
  const int64_t H = c->J / 2 + 1;
  A((void**)&c->spare.h, sizeof(int32_t) * c->noff[c->d]);
  A((void**)&c->spare.v, sizeof(int8_t) * c->noff[c->d]);
  A((void**)&c->d_ghat, sizeof(float2) * c->ghat_off[c->d]);
  A((void**)&c->d_twiddle, sizeof(float2) * c->J);
  A((void**)&c->d_twstage, sizeof(float2) * c->J);
  A((void**)&c->d_suffix, sizeof(float2) * c->suffix_off[c->d]);
  A((void**)&c->d_prefix, sizeof(float2) * H * c->rmax);
  A((void**)&c->d_prefix_tmp, sizeof(float2) * H * c->rmax);
  A((void**)&c->d_SH, sizeof(float) * c->J * c->smax);
  A((void**)&c->d_Y, sizeof(float) * c->J * c->nmax);
  c->yoff[0] = 0;
  for (int k = 0; k < c->d; ++k) c->yoff[k + 1] = c->yoff[k] + (int64_t)c->J * c->n[k];
  A((void**)&c->d_Yall, sizeof(float) * c->yoff[c->d]);
  A((void**)&c->d_gram, sizeof(float) * (c->smax + c->nmax) * c->smax);
  if (c->solve64) A((void**)&c->d_gram64, sizeof(double) * (c->smax + c->nmax) * c->smax);
  if (c->det) {
    A((void**)&c->d_det_misc, sizeof(int) * 4);
    A((void**)&c->d_y64, sizeof(int64_t) * c->yoff[c->d]);
    A((void**)&c->d_gram_part, (c->solve64 ? sizeof(double) : sizeof(float)) * (size_t)TT_DET_KSPLIT *
                                   (c->smax + c->nmax) * c->smax);
    A((void**)&c->d_part_err, sizeof(double) * 2 * TT_DET_PARTS);
    A((void**)&c->d_part_chg, sizeof(double) * 2 * std::max<int64_t>(TT_DET_PARTS, c->nmax));
    A((void**)&c->d_det_bcnt, sizeof(int32_t) * (size_t)c->J * dplan_ranges(c));
    A((void**)&c->d_det_kv, sizeof(uint2) * (size_t)dplan_fibres(c));
  }
  A((void**)&c->d_core_old, sizeof(float) * c->nmax * c->smax);
  c->changes_cap = 1024 * TT_MAX_D;
  A((void**)&c->d_changes, sizeof(double) * 2 * c->changes_cap);
  A((void**)&c->d_errs, sizeof(double) * 2 * (c->changes_cap / c->d));
  A((void**)&c->d_status, sizeof(int));
  A((void**)&c->d_err_acc, sizeof(double) * 4);
  A((void**)&c->d_xgram, sizeof(double) * 2 * 32 * 32);
  A((void**)&c->d_ws_acc, sizeof(double) * 2);
  // streaming relative error (n_0 % 4 == 0, n_0 <= 1024, G_0 within 48 KB of shared memory)
  c->rint_r1p = (c->r[1] + 3) & ~3;
  if (c->n[0] % 4 == 0 && c->n[0] <= 1024 && (int64_t)c->rint_r1p * c->n[0] * 4 <= 48 * 1024) {
    A((void**)&c->d_rint, sizeof(float) * (size_t)(c->N / c->n[0]) * c->rint_r1p);
    A((void**)&c->d_slab_u, sizeof(float) * (size_t)(c->N / (c->n[0] * c->n[1])) * c->r[2]);
  }
}

static std::atomic<uint64_t> g_workspace_limit{0};

// Total bytes of the workspaces above (each allocation rounded up to the 16 bytes cudaMalloc is
// given at least); touches no device.
static uint64_t tt_workspace_plan(tt_ctx* c) {
  uint64_t total = 0;
  tt_workspace_each(c, [&](void**, size_t bytes) { total += (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255; });
  return total;
}

extern "C" uint64_t tt_set_workspace_limit(uint64_t bytes) { return g_workspace_limit.exchange(bytes); }

int tt_check_workspace_cap(tt_ctx* c, uint64_t extra) {
  const uint64_t cap = g_workspace_limit.load();
  if (cap && c->ws_bytes + extra > cap)
    return tt_fail(c, TT_ENOMEM, "workspaces need %llu bytes, above the limit of %llu bytes",
                   (unsigned long long)(c->ws_bytes + extra), (unsigned long long)cap);
  return TT_OK;
}

extern "C" int tt_sketch_init(tt_ctx** out, const tt_params* p, void* stream) {
  if (!out || !p) return TT_EINVAL;
  *out = nullptr;
  tt_ctx* c = new (std::nothrow) tt_ctx();
  if (!c) return TT_ENOMEM;
  auto bad = [&](const char* msg, long long v) {
    // keep the message readable through a context-less path: return code only
    fprintf(stderr, "tt_sketch_init: %s (%lld)\n", msg, v);
    delete c;
    return TT_EINVAL;
  };
  if (p->d < 2 || p->d > TT_MAX_D) return bad("d must be in [2, 8]", p->d);
  if (!p->n || !p->r) return bad("null n or r", 0);
  if (p->J < 2 || p->J > TT_MAX_J) return bad("J must be in [2, 16384]", p->J);
  if ((p->J & (p->J - 1)) && p->J > 8192) return bad("J above 8192 must be a power of two", p->J);
  if (!(p->lambda >= 0.0) || !std::isfinite(p->lambda)) return bad("lambda must be finite and >= 0", 0);
  if (p->dtype < TT_F64 || p->dtype > TT_FP8E4M3) return bad("unknown dtype", p->dtype);
  if (p->r[0] != 1 || p->r[p->d] != 1) return bad("r[0] and r[d] must be 1", 0);
  c->d = p->d;
  c->J = p->J;
  c->logJ = 0;
  while ((1 << c->logJ) < c->J) ++c->logJ;
  if ((1 << c->logJ) != c->J) c->logJ = -1;  // not a power of two: direct DFTs
  c->lambda = p->lambda;
  c->seed = p->seed;
  c->dtype = p->dtype;
  c->flags = p->flags;
  // sigma = 0 (Alg. 1 asks sigma > 0: M is then not SPD by construction and its conditioning is
  // unbounded) and TT_FLAG_FP64_SOLVE take the FP64 update
  c->solve64 = (p->flags & TT_FLAG_FP64_SOLVE) != 0 || p->lambda == 0.0;
  c->det = (p->flags & TT_FLAG_DETERMINISTIC) != 0;
  c->stream = (cudaStream_t)stream;
  c->N = 1;
  c->noff[0] = 0;
  c->stride[0] = 1;
  for (int k = 0; k < c->d; ++k) {
    if (p->n[k] < 1 || p->n[k] > TT_MAX_N) return bad("mode size out of [1, 65536]", p->n[k]);
    c->n[k] = p->n[k];
    c->noff[k + 1] = c->noff[k] + c->n[k];
    c->stride[k + 1] = c->stride[k] * c->n[k];
    if (c->stride[k + 1] > (1ll << 40)) return bad("tensor too large", c->stride[k + 1]);
    c->nmax = std::max<int64_t>(c->nmax, c->n[k]);
  }
  c->N = c->stride[c->d];
  for (int k = 0; k <= c->d; ++k) {
    if (p->r[k] < 1) return bad("ranks must be >= 1", p->r[k]);
    c->r[k] = p->r[k];
    c->rmax = std::max(c->rmax, c->r[k]);
  }
  for (int k = 0; k < c->d; ++k) {
    int s = c->r[k] * c->r[k + 1];
    if (s > TT_MAX_S_LARGE) return bad("r[k]*r[k+1] exceeds 512", s);
    if (s > TT_MAX_S && (p->n[k] > 100000 || tt_large_solve_smem(s, (int)p->n[k]) > 227 * 1024))
      return bad("r[k]*r[k+1]*(n[k]+33) too large for the one-CTA Cholesky solve", s);
    if (p->r[k] > TT_MAX_S) return bad("a TT rank exceeds 160", p->r[k]);
    c->smax = std::max(c->smax, s);
    // QR/LQ working sets (see tt_solve.cu): rows x cols floats in shared memory
    int64_t ql = (int64_t)c->r[k] * c->n[k] * c->r[k + 1];
    if (ql > 40000) return bad("core too large for the in-CTA QR (r_k n_k r_{k+1} > 40000)", ql);
  }
  c->M0 = c->N / c->n[0];
  if (c->M0 >= (1ll << 31)) return bad("too many mode-0 fibers", c->M0);

  int H = c->J / 2 + 1;
  c->ghat_off[0] = 0;
  for (int k = 0; k < c->d; ++k) c->ghat_off[k + 1] = c->ghat_off[k] + (int64_t)H * c->r[k] * c->r[k + 1];
  c->suffix_off[0] = 0;
  for (int k = 0; k < c->d; ++k) c->suffix_off[k + 1] = c->suffix_off[k] + (int64_t)H * c->r[k + 1];

  // The workspaces are planned (sizes summed) before anything is allocated, so that a process-wide
  // cap (tt_set_workspace_limit) is enforced before any CUDA call.
  const uint64_t planned = tt_workspace_plan(c);
  c->ws_bytes = planned;
  const uint64_t cap = g_workspace_limit.load();
  if (cap && planned > cap) {
    fprintf(stderr, "tt_sketch_init: workspaces need %llu bytes, above the limit of %llu bytes\n",
            (unsigned long long)planned, (unsigned long long)cap);
    delete c;
    return TT_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  tt_workspace_each(c, [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
  });
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->hi, cudaStreamNonBlocking, greatest);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_spare, cudaEventDisableTiming);
  for (int k = 0; k < c->d && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&c->ev_y[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_all(c);
    fprintf(stderr, "tt_sketch_init: cudaMalloc: %s\n", cudaGetErrorString(e));
    delete c;
    return e == cudaErrorMemoryAllocation ? TT_ENOMEM : TT_ECUDA;
  }
  // twiddles exp(-2 pi i t / J), t < J (the radix-2 FFT reads t < J/2, the direct DFT all),
  // evaluated in double on the host
  std::vector<float2> tw(c->J);
  for (int t = 0; t < c->J; ++t) {
    double ang = -2.0 * M_PI * (double)t / (double)c->J;
    tw[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  e = cudaMemcpyAsync(c->d_twiddle, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice, c->stream);
  // per-stage tables of the radix-4 Stockham FFT: spans Ns = Ns0, 4 Ns0, ... < J (Ns0 = 2 after
  // the radix-2 stage of an odd log J), entries exp(-2 pi i r m / (4 Ns)) at [off + 3 m + r - 1]
  std::vector<float2> tws(c->J, make_float2(1.f, 0.f));
  if (c->logJ >= 0) {
    size_t off = 0;
    for (int Ns = (c->logJ & 1) ? 2 : 1; Ns < c->J; Ns *= 4)
      for (int m = 0; m < Ns; ++m, off += 3)
        for (int r = 1; r <= 3; ++r) {
          const double ang = -2.0 * M_PI * (double)r * (double)m / (4.0 * (double)Ns);
          tws[off + r - 1] = make_float2((float)std::cos(ang), (float)std::sin(ang));
        }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_twstage, tws.data(), sizeof(float2) * tws.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free_all(c);
    fprintf(stderr, "tt_sketch_init: %s\n", cudaGetErrorString(e));
    delete c;
    return TT_ECUDA;
  }
  *out = c;
  return TT_OK;
}

extern "C" void tt_sketch_destroy(tt_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);  // a spare draw may still be in flight
  free_all(c);
  delete c;
}

extern "C" const char* tt_last_error(const tt_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" int tt_sketch_tables(tt_ctx* c, uint64_t sweep, int32_t* h_host, int8_t* v_host) {
  if (!c) return TT_EINVAL;
  if (!h_host || !v_host) return tt_fail(c, TT_EINVAL, "tt_sketch_tables: null output");
  int rc = tt_ensure_tables(c, sweep);
  if (rc) return rc;
  TT_CUDA(c, cudaMemcpyAsync(h_host, c->d_h, sizeof(int32_t) * c->noff[c->d], cudaMemcpyDeviceToHost, c->stream));
  TT_CUDA(c, cudaMemcpyAsync(v_host, c->d_v, sizeof(int8_t) * c->noff[c->d], cudaMemcpyDeviceToHost, c->stream));
  TT_CUDA(c, cudaStreamSynchronize(c->stream));
  return TT_OK;
}

extern "C" int tt_sketch_set_tables(tt_ctx* c, const int32_t* h_host, const int8_t* v_host) {
  if (!c) return TT_EINVAL;
  if (!h_host || !v_host) return tt_fail(c, TT_EINVAL, "tt_sketch_set_tables: null input");
  int64_t tot = c->noff[c->d];
  for (int64_t i = 0; i < tot; ++i) {
    if (h_host[i] < 0 || h_host[i] >= c->J) return tt_fail(c, TT_EINVAL, "h[%lld]=%d outside [0, J)", (long long)i, h_host[i]);
    if (v_host[i] != 1 && v_host[i] != -1) return tt_fail(c, TT_EINVAL, "v[%lld]=%d not +-1", (long long)i, v_host[i]);
  }
  if (c->spare_pending) TT_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_spare, 0));
  TT_CUDA(c, cudaMemcpyAsync(c->d_h, h_host, sizeof(int32_t) * tot, cudaMemcpyHostToDevice, c->stream));
  TT_CUDA(c, cudaMemcpyAsync(c->d_v, v_host, sizeof(int8_t) * tot, cudaMemcpyHostToDevice, c->stream));
  TT_CUDA(c, cudaStreamSynchronize(c->stream));
  c->user_tables = true;
  c->spare.tables_valid = false;
  c->tables_valid = true;
  for (int k = 0; k < TT_MAX_D; ++k) c->rplan_valid[k] = false;
  return TT_OK;
}
