// Part (a): Y_k = S A_(k)^T, the TensorSketch of every mode-k unfolding (Alg. 1, Sec. 3).
//
// Y_k[b, i_k] = sum over entries with that i_k of prod_{s!=k} v_s(i_s) * A(i), restricted to
// (sum_{s!=k} h_s(i_s)) mod J = b  (Eqs. (eqn_h), (eqn_v)).
//
// Mode 0 (the contiguous mode): every mode-0 fiber A(:, i_1, ..., i_{d-1}) lands in ONE row
// b_f = (sum_{s>=1} h_s(i_s)) mod J of Y_0, so Y_0[b, :] = sum_{f : b_f = b} s_f A(:, f). The
// per-sweep plan lists fibers grouped by row; a warp owns a row, gathers its fibers with
// 16-byte loads and sums them in registers. No atomics, one read of every entry.
//
// Modes k >= 1: a CTA owns column i_k of Y_k (J floats in shared memory) and streams the
// entries with that i_k, mode-0 fibers at a time; each entry is added to its bucket
// (h_0(i_0) + c_f) mod J with a shared-memory atomic. Column partials of CTAs that split
// one column are combined with global atomics.
#include <algorithm>

#include "tt_internal.cuh"

template <>
struct TtElem<TT_F64> {
  using T = double;
  static constexpr int bytes = 8;
  __device__ static float get(const void* a, int64_t i) { return (float)__ldg((const double*)a + i); }
};
template <>
struct TtElem<TT_F32> {
  using T = float;
  static constexpr int bytes = 4;
  __device__ static float get(const void* a, int64_t i) { return __ldg((const float*)a + i); }
};
template <>
struct TtElem<TT_BF16> {
  using T = unsigned short;
  static constexpr int bytes = 2;
  __device__ static float get(const void* a, int64_t i) {
    return __uint_as_float(((uint32_t)__ldg((const unsigned short*)a + i)) << 16);
  }
};

// OCP FP8 E4M3 (bias 7, no infinities): decode from the bit fields.
__device__ __forceinline__ float tt_fp8_e4m3(uint32_t c) {
  uint32_t s = (c & 0x80u) << 24;
  uint32_t e = (c >> 3) & 0xFu;
  uint32_t m = c & 7u;
  float mag = e ? __uint_as_float(((e + 120u) << 23) | (m << 20)) : (float)m * 0.001953125f;  // 2^-9
  return __uint_as_float(__float_as_uint(mag) | s);
}
template <>
struct TtElem<TT_FP8E4M3> {
  using T = unsigned char;
  static constexpr int bytes = 1;
  __device__ static float get(const void* a, int64_t i) { return tt_fp8_e4m3(__ldg((const unsigned char*)a + i)); }
};

// ---------------------------------------------------------------------------------------------
// mode 0: row-owner fiber gather

// Unpack a 16/8/4/2/1-byte vector of EPV elements of type DT into floats.
template <int DT, int VB>
struct TtVec {
  static constexpr int EPV = VB / TtElem<DT>::bytes;
  __device__ static void load(const char* p, float* out) {
    if constexpr (VB == 16) {
      uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
      unpack(reinterpret_cast<const uint32_t*>(&u), out);
    } else if constexpr (VB == 8) {
      uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
      unpack(reinterpret_cast<const uint32_t*>(&u), out);
    } else if constexpr (VB == 4) {
      uint32_t u = __ldg(reinterpret_cast<const uint32_t*>(p));
      unpack(&u, out);
    } else if constexpr (VB == 2) {
      uint32_t u = __ldg(reinterpret_cast<const unsigned short*>(p));
      unpack(&u, out);
    } else {
      uint32_t u = __ldg(reinterpret_cast<const unsigned char*>(p));
      unpack(&u, out);
    }
  }
  __device__ static void unpack(const uint32_t* w, float* out) {
    if constexpr (DT == TT_F32) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) out[e] = __uint_as_float(w[e]);
    } else if constexpr (DT == TT_F64) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) {
        unsigned long long b = ((unsigned long long)w[2 * e + 1] << 32) | w[2 * e];
        out[e] = (float)__longlong_as_double((long long)b);
      }
    } else if constexpr (DT == TT_BF16) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) out[e] = __uint_as_float(((w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu) << 16);
    } else {
#pragma unroll
      for (int e = 0; e < EPV; ++e) out[e] = tt_fp8_e4m3((w[e >> 2] >> (8 * (e & 3))) & 0xFFu);
    }
  }
};

struct GatherArgs {
  const char* A;
  const float* scales;  // n0 FP8 scales or null
  const uint32_t* plan;
  const int64_t* off;   // J+1
  float* Y;             // J x n0 row-major
  int J;
  int n0;
  int64_t fiber_bytes;
  int vpf;              // vectors per fiber
  int lpf;              // lanes per fiber slot (vpf if <= 32 else 32)
  int fpi;              // fiber slots per warp (32 / lpf)
  int nchunk;           // column chunks of 32 vectors when vpf > 32
  int parts;            // splits of each row's fiber list (atomics when > 1)
};

template <int DT, int VB, int U>
__global__ void __launch_bounds__(256) k_unfold_mode0(GatherArgs g) {
  constexpr int EPV = TtVec<DT, VB>::EPV;
  extern __shared__ float red[];  // per warp: 32 lanes x EPV partial sums
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int slot = lane / g.lpf;
  const int posl = lane - slot * g.lpf;
  const bool active = slot < g.fpi;
  const int64_t items = (int64_t)g.J * g.nchunk * g.parts;
  float* wred = red + wib * 32 * EPV;
  for (int64_t it = warp; it < items; it += nwarps) {
    const int part = (int)(it % g.parts);
    const int64_t rc = it / g.parts;
    const int chunk = (int)(rc % g.nchunk);
    const int row = (int)(rc / g.nchunk);
    const int vpos = chunk * 32 + posl;  // vector index within the fiber
    const bool lane_ok = active && vpos < g.vpf;
    float acc[EPV];
#pragma unroll
    for (int e = 0; e < EPV; ++e) acc[e] = 0.f;
    int64_t beg = g.off[row], end = g.off[row + 1];
    int64_t len = end - beg;
    int64_t pb = beg + len * part / g.parts, pe = beg + len * (part + 1) / g.parts;
    for (int64_t j0 = pb; j0 < pe; j0 += (int64_t)g.fpi * U) {
      float v[U][EPV];
      float sg[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        int64_t j = j0 + (int64_t)u * g.fpi + slot;
        sg[u] = 0.f;
        if (lane_ok && j < pe) {
          uint32_t w = __ldg(g.plan + j);
          sg[u] = (w >> 31) ? -1.f : 1.f;
          const char* p = g.A + (int64_t)(w & 0x7FFFFFFFu) * g.fiber_bytes + (int64_t)vpos * VB;
          TtVec<DT, VB>::load(p, v[u]);
        } else {
#pragma unroll
          for (int e = 0; e < EPV; ++e) v[u][e] = 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int e = 0; e < EPV; ++e) acc[e] = fmaf(sg[u], v[u][e], acc[e]);
    }
    // combine the fiber slots (lanes with equal posl) through shared memory
    if (g.fpi > 1) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) wred[lane * EPV + e] = acc[e];
      __syncwarp();
      if (slot == 0) {
        for (int s = 1; s < g.fpi; ++s)
#pragma unroll
          for (int e = 0; e < EPV; ++e) acc[e] += wred[(s * g.lpf + posl) * EPV + e];
      }
      __syncwarp();
    }
    if (slot == 0 && lane_ok) {
      float* yrow = g.Y + (int64_t)row * g.n0;
#pragma unroll
      for (int e = 0; e < EPV; ++e) {
        int i0 = vpos * EPV + e;
        float val = acc[e];
        if (g.scales) val *= __ldg(g.scales + i0);
        if (g.parts > 1)
          atomicAdd(yrow + i0, val);
        else
          yrow[i0] = val;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// modes k >= 1: column owner with shared-memory accumulation

struct ColArgs {
  const void* A;
  const float* scales;
  const int32_t* h;
  const int8_t* v;
  float* Y;  // J x n_k row-major
  int64_t n[TT_MAX_D];
  int64_t noff[TT_MAX_D + 1];
  int d, k, J;
  int64_t P;      // prod_{s<k} n_s (contiguous block per (i_k, outer))
  int64_t F;      // P / n_0 fibers per block
  int64_t Q;      // prod_{s>k} n_s outer combinations
  int nchunk;     // CTAs per column
};

template <int DT>
__global__ void __launch_bounds__(512) k_unfold_col(ColArgs a) {
  extern __shared__ float ycol[];
  const int J = a.J;
  for (int b = threadIdx.x; b < J; b += blockDim.x) ycol[b] = 0.f;
  __syncthreads();
  const int col = blockIdx.x / a.nchunk;
  const int chunk = blockIdx.x % a.nchunk;
  const int64_t pairs = a.Q * a.F;
  const int64_t pb = pairs * chunk / a.nchunk, pe = pairs * (chunk + 1) / a.nchunk;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int n0 = (int)a.n[0];
  const int32_t* h0 = a.h;
  const int8_t* v0 = a.v;
  const int hk = a.h[a.noff[a.k] + col];
  const int vk = a.v[a.noff[a.k] + col];
  for (int64_t t = pb + warp; t < pe; t += nw) {
    int64_t q = t / a.F, f = t - q * a.F;
    // bucket offset and sign of the fiber: modes 1..k-1 from f, modes k+1..d-1 from q
    int c = 0, neg = 0;
    int64_t rem = f;
    for (int s = 1; s < a.k; ++s) {
      int64_t i = rem % a.n[s];
      rem /= a.n[s];
      c += a.h[a.noff[s] + i];
      neg ^= a.v[a.noff[s] + i] < 0;
    }
    rem = q;
    for (int s = a.k + 1; s < a.d; ++s) {
      int64_t i = rem % a.n[s];
      rem /= a.n[s];
      c += a.h[a.noff[s] + i];
      neg ^= a.v[a.noff[s] + i] < 0;
    }
    (void)hk;
    (void)vk;
    float sgn = neg ? -1.f : 1.f;
    int64_t base = ((int64_t)col + a.n[a.k] * q) * a.P + f * n0;
    for (int i0 = lane; i0 < n0; i0 += 32) {
      float x = TtElem<DT>::get(a.A, base + i0);
      if (a.scales) x *= __ldg(a.scales + i0);
      int b = (__ldg(h0 + i0) + c) & (J - 1);
      float s = (__ldg(v0 + i0) < 0) ? -sgn : sgn;
      atomicAdd(&ycol[b], s * x);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < J; b += blockDim.x) {
    float val = ycol[b];
    if (val != 0.f) atomicAdd(a.Y + (int64_t)b * a.n[a.k] + col, val);
  }
}

// ---------------------------------------------------------------------------------------------
// host side

template <int DT, int VB>
static int launch_mode0_vb(tt_ctx* c, const void* A, const float* scales, float* Y) {
  constexpr int EPV = TtVec<DT, VB>::EPV;
  constexpr int U = (VB >= 8) ? 8 : 4;
  GatherArgs g;
  g.A = (const char*)A;
  g.scales = scales;
  g.plan = c->d_plan0;
  g.off = c->d_plan0_off;
  g.Y = Y;
  g.J = c->J;
  g.n0 = (int)c->n[0];
  g.fiber_bytes = (int64_t)c->n[0] * TtElem<DT>::bytes;
  g.vpf = (int)(g.fiber_bytes / VB);
  if (g.vpf <= 32) {
    g.lpf = g.vpf;
    g.fpi = 32 / g.vpf;
    g.nchunk = 1;
  } else {
    g.lpf = 32;
    g.fpi = 1;
    g.nchunk = (g.vpf + 31) / 32;
  }
  const int threads = 256;
  int dev_sms = 152;
  int64_t warps_wanted = (int64_t)dev_sms * 48;
  int64_t base_items = (int64_t)c->J * g.nchunk;
  g.parts = (int)std::max<int64_t>(1, std::min<int64_t>(64, (warps_wanted + base_items - 1) / base_items));
  if (g.parts > 1) TT_CUDA(c, cudaMemsetAsync(Y, 0, sizeof(float) * c->J * c->n[0], c->stream));
  int64_t items = base_items * g.parts;
  int blocks = (int)std::min<int64_t>((items + 7) / 8, (int64_t)dev_sms * 64);
  size_t smem = sizeof(float) * 32 * EPV * (threads / 32);
  k_unfold_mode0<DT, VB, U><<<blocks, threads, smem, c->stream>>>(g);
  TT_LAUNCH(c, "k_unfold_mode0");
  return TT_OK;
}

template <int DT>
static int launch_mode0(tt_ctx* c, const void* A, const float* scales, float* Y) {
  int64_t fb = (int64_t)c->n[0] * TtElem<DT>::bytes;
  uintptr_t al = (uintptr_t)A;
  if (fb % 16 == 0 && al % 16 == 0) return launch_mode0_vb<DT, 16>(c, A, scales, Y);
  if (fb % 8 == 0 && al % 8 == 0) return launch_mode0_vb<DT, (TtElem<DT>::bytes <= 8 ? 8 : 16)>(c, A, scales, Y);
  if constexpr (TtElem<DT>::bytes <= 4) {
    if (fb % 4 == 0 && al % 4 == 0) return launch_mode0_vb<DT, 4>(c, A, scales, Y);
  }
  if constexpr (TtElem<DT>::bytes <= 2) {
    if (fb % 2 == 0 && al % 2 == 0) return launch_mode0_vb<DT, 2>(c, A, scales, Y);
  }
  if constexpr (TtElem<DT>::bytes <= 1) return launch_mode0_vb<DT, 1>(c, A, scales, Y);
  return launch_mode0_vb<DT, TtElem<DT>::bytes>(c, A, scales, Y);
}

template <int DT>
static int launch_col(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  ColArgs a;
  a.A = A;
  a.scales = scales;
  a.h = c->d_h;
  a.v = c->d_v;
  a.Y = Y;
  for (int s = 0; s < c->d; ++s) a.n[s] = c->n[s];
  for (int s = 0; s <= c->d; ++s) a.noff[s] = c->noff[s];
  a.d = c->d;
  a.k = k;
  a.J = c->J;
  a.P = c->stride[k];
  a.F = a.P / c->n[0];
  a.Q = c->N / (c->stride[k] * c->n[k]);
  int64_t want = 152 * 4;
  a.nchunk = (int)std::max<int64_t>(1, std::min<int64_t>((want + c->n[k] - 1) / c->n[k], a.Q * a.F));
  TT_CUDA(c, cudaMemsetAsync(Y, 0, sizeof(float) * c->J * c->n[k], c->stream));
  int blocks = (int)(c->n[k] * a.nchunk);
  size_t smem = sizeof(float) * c->J;
  if (smem > 48 * 1024) TT_CUDA(c, cudaFuncSetAttribute(k_unfold_col<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_unfold_col<DT><<<blocks, 512, smem, c->stream>>>(a);
  TT_LAUNCH(c, "k_unfold_col");
  return TT_OK;
}

template <int DT>
static int unfold_dt(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  if (k == 0) {
    int rc = tt_ensure_plan0(c);
    if (rc) return rc;
    return launch_mode0<DT>(c, A, scales, Y);
  }
  return launch_col<DT>(c, A, scales, k, Y);
}

int tt_launch_unfold(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  if (k == 0) {
    int rc = tt_ensure_plan0(c);  // plan build is not part of the timed kernel
    if (rc) return rc;
  }
  int rc = tt_prof_begin(c, k);
  if (rc) return rc;
  switch (c->dtype) {
    case TT_F64: rc = unfold_dt<TT_F64>(c, A, scales, k, Y); break;
    case TT_F32: rc = unfold_dt<TT_F32>(c, A, scales, k, Y); break;
    case TT_BF16: rc = unfold_dt<TT_BF16>(c, A, scales, k, Y); break;
    default: rc = unfold_dt<TT_FP8E4M3>(c, A, scales, k, Y); break;
  }
  if (rc) return rc;
  return tt_prof_end(c);
}
