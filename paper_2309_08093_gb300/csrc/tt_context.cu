// Context lifetime, parameter validation, hash/sign draws and the mode-0 fiber plan.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <new>
#include <vector>

#include "tt_internal.cuh"

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
  h[g] = (int32_t)(wh & (uint64_t)(J - 1));
  v[g] = (wv >> 63) ? (int8_t)-1 : (int8_t)1;
}

int tt_ensure_tables(tt_ctx* c, uint64_t sweep) {
  if (c->user_tables) return TT_OK;
  if (c->flags & TT_FLAG_FIXED_SKETCH) sweep = 0;
  if (c->tables_valid && c->tables_sweep == sweep) return TT_OK;
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
  c->plan0_valid = false;
  return TT_OK;
}

// ---------------------------------------------------------------------------------------------
// mode-0 fiber plan: fibers f = (i_1, ..., i_{d-1}) (mode 1 fastest) grouped by their row
// b_f = (sum_{s>=1} h_s(i_s)) mod J of Y_0, with sign prod_{s>=1} v_s(i_s) in bit 31.

struct PlanArgs {
  int64_t n[TT_MAX_D];
  int64_t noff[TT_MAX_D + 1];
  int d;
  int J;
  int64_t M0;
};

__device__ __forceinline__ void plan_key(const PlanArgs& a, const int32_t* __restrict__ h,
                                         const int8_t* __restrict__ v, int64_t f, int* key, int* neg) {
  int b = 0, s = 0;
  int64_t rem = f;
  for (int k = 1; k < a.d; ++k) {
    int64_t i = rem % a.n[k];
    rem /= a.n[k];
    b += h[a.noff[k] + i];
    s ^= (v[a.noff[k] + i] < 0);
  }
  *key = b & (a.J - 1);
  *neg = s;
}

__global__ void k_plan_count(PlanArgs a, const int32_t* h, const int8_t* v, int32_t* count) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < a.M0; f += (int64_t)gridDim.x * blockDim.x) {
    int key, neg;
    plan_key(a, h, v, f, &key, &neg);
    atomicAdd(&count[key], 1);
  }
}

// exclusive scan of J counts into off[0..J]; one block of 1024 threads
__global__ void k_plan_scan(int J, const int32_t* count, int64_t* off, int32_t* cursor) {
  __shared__ int64_t part[1024];
  int t = threadIdx.x;
  int per = (J + 1023) / 1024;
  int64_t s = 0;
  for (int i = t * per; i < min(J, (t + 1) * per); ++i) s += count[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t x = (t >= o) ? part[t - o] : 0;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  int64_t base = part[t] - s;
  for (int i = t * per; i < min(J, (t + 1) * per); ++i) {
    off[i] = base;
    base += count[i];
    cursor[i] = 0;
  }
  if (t == 1023) off[J] = part[1023];
}

__global__ void k_plan_scatter(PlanArgs a, const int32_t* h, const int8_t* v, const int64_t* off,
                               int32_t* cursor, uint32_t* plan) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < a.M0; f += (int64_t)gridDim.x * blockDim.x) {
    int key, neg;
    plan_key(a, h, v, f, &key, &neg);
    int pos = atomicAdd(&cursor[key], 1);
    plan[off[key] + pos] = (uint32_t)f | ((uint32_t)neg << 31);
  }
}

int tt_ensure_plan0(tt_ctx* c) {
  if (c->plan0_valid) return TT_OK;
  PlanArgs a;
  for (int k = 0; k < c->d; ++k) a.n[k] = c->n[k];
  for (int k = 0; k <= c->d; ++k) a.noff[k] = c->noff[k];
  a.d = c->d;
  a.J = c->J;
  a.M0 = c->M0;
  int32_t* count = c->d_plan0_cursor;
  TT_CUDA(c, cudaMemsetAsync(count, 0, sizeof(int32_t) * c->J, c->stream));
  int blocks = (int)std::min<int64_t>((c->M0 + 255) / 256, 152 * 16);
  k_plan_count<<<blocks, 256, 0, c->stream>>>(a, c->d_h, c->d_v, count);
  TT_LAUNCH(c, "k_plan_count");
  k_plan_scan<<<1, 1024, 0, c->stream>>>(c->J, count, c->d_plan0_off, count);
  TT_LAUNCH(c, "k_plan_scan");
  k_plan_scatter<<<blocks, 256, 0, c->stream>>>(a, c->d_h, c->d_v, c->d_plan0_off, count, c->d_plan0);
  TT_LAUNCH(c, "k_plan_scatter");
  c->plan0_valid = true;
  return TT_OK;
}

// ---------------------------------------------------------------------------------------------
// lifetime

static void free_all(tt_ctx* c) {
  void* ps[] = {c->d_h, c->d_v, c->d_plan0, c->d_plan0_off, c->d_plan0_cursor, c->d_ghat,
                c->d_twiddle, c->d_suffix, c->d_prefix, c->d_prefix_tmp, c->d_SH, c->d_Y,
                c->d_gram, c->d_core_old, c->d_changes, c->d_status, c->d_err_acc};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (c->d_A_stage) cudaFree(c->d_A_stage);
  if (c->d_scales_stage) cudaFree(c->d_scales_stage);
  for (int k = 0; k < TT_MAX_D; ++k)
    if (c->d_cores_stage[k]) cudaFree(c->d_cores_stage[k]);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
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
  if (p->J < 2 || p->J > TT_MAX_J || (p->J & (p->J - 1))) return bad("J must be a power of two in [2, 16384]", p->J);
  if (!(p->lambda >= 0.0) || !std::isfinite(p->lambda)) return bad("lambda must be finite and >= 0", 0);
  if (p->dtype < TT_F64 || p->dtype > TT_FP8E4M3) return bad("unknown dtype", p->dtype);
  if (p->r[0] != 1 || p->r[p->d] != 1) return bad("r[0] and r[d] must be 1", 0);
  c->d = p->d;
  c->J = p->J;
  c->logJ = 0;
  while ((1 << c->logJ) < c->J) ++c->logJ;
  c->lambda = p->lambda;
  c->seed = p->seed;
  c->dtype = p->dtype;
  c->flags = p->flags;
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
    if (s > TT_MAX_S) return bad("r[k]*r[k+1] exceeds 160", s);
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

  cudaError_t e = cudaSuccess;
  auto A = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
  };
  A((void**)&c->d_h, sizeof(int32_t) * c->noff[c->d]);
  A((void**)&c->d_v, sizeof(int8_t) * c->noff[c->d]);
  A((void**)&c->d_plan0, sizeof(uint32_t) * c->M0);
  A((void**)&c->d_plan0_off, sizeof(int64_t) * (c->J + 1));
  A((void**)&c->d_plan0_cursor, sizeof(int32_t) * c->J);
  A((void**)&c->d_ghat, sizeof(float2) * c->ghat_off[c->d]);
  A((void**)&c->d_twiddle, sizeof(float2) * (c->J / 2));
  A((void**)&c->d_suffix, sizeof(float2) * c->suffix_off[c->d]);
  A((void**)&c->d_prefix, sizeof(float2) * H * c->rmax);
  A((void**)&c->d_prefix_tmp, sizeof(float2) * H * c->rmax);
  A((void**)&c->d_SH, sizeof(float) * c->J * c->smax);
  A((void**)&c->d_Y, sizeof(float) * c->J * c->nmax);
  A((void**)&c->d_gram, sizeof(double) * (c->smax + c->nmax) * c->smax);
  A((void**)&c->d_core_old, sizeof(float) * c->nmax * c->smax);
  c->changes_cap = 1024 * TT_MAX_D;
  A((void**)&c->d_changes, sizeof(double) * 2 * c->changes_cap);
  A((void**)&c->d_status, sizeof(int));
  A((void**)&c->d_err_acc, sizeof(double) * 4);
  if (e != cudaSuccess) {
    free_all(c);
    fprintf(stderr, "tt_sketch_init: cudaMalloc: %s\n", cudaGetErrorString(e));
    delete c;
    return e == cudaErrorMemoryAllocation ? TT_ENOMEM : TT_ECUDA;
  }
  // FFT twiddles exp(-2 pi i t / J), t < J/2, evaluated in double on the host
  std::vector<float2> tw(c->J / 2);
  for (int t = 0; t < c->J / 2; ++t) {
    double ang = -2.0 * M_PI * (double)t / (double)c->J;
    tw[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  e = cudaMemcpyAsync(c->d_twiddle, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice, c->stream);
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
  TT_CUDA(c, cudaMemcpyAsync(c->d_h, h_host, sizeof(int32_t) * tot, cudaMemcpyHostToDevice, c->stream));
  TT_CUDA(c, cudaMemcpyAsync(c->d_v, v_host, sizeof(int8_t) * tot, cudaMemcpyHostToDevice, c->stream));
  TT_CUDA(c, cudaStreamSynchronize(c->stream));
  c->user_tables = true;
  c->tables_valid = true;
  c->plan0_valid = false;
  return TT_OK;
}
