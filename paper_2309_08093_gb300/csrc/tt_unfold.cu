// Part (a): Y_k = S A_(k)^T, the TensorSketch of every mode-k unfolding (Alg. 1, Sec. 3).
//
// Y_k[b, i_k] = sum over entries with that i_k of prod_{s!=k} v_s(i_s) * A(i), restricted to
// (sum_{s!=k} h_s(i_s)) mod J = b  (Eqs. (eqn_h), (eqn_v)).
//
// Both kernels read A only as whole mode-0 fibres (contiguous runs of n_0 entries), gathered with
// 16-byte loads in the order of a small per-sweep plan (tt_context.cu) and summed in registers.
//
// Mode 0: every fibre A(:, i_1, ..., i_{d-1}) lands in ONE row c = (sum_{s>=1} h_s(i_s)) mod J of
// Y_0, so Y_0[c, :] = sum_{fibres with hash c} sign * fibre.
//
// Modes k >= 1: with Z_k[i_0, c] = sum over the fibres r of the modes != 0, k with hash c_r = c
// of sign_r * A(i_0, r, i_k), the TensorSketch definition regroups to
//     Y_k[b, i_k] = sum_{i_0} v_0(i_0) Z_k[i_0, (b - h_0(i_0)) mod J],
// i.e. column i_k is a sum of n_0 circularly rolled rows of Z_k.
//
// One kernel serves both. Each CTA owns a contiguous range of (column i_k, c) groups of the plan
// and walks it in chunks of C groups. Phase 1 builds the chunk's Z rows in shared memory: the
// chunk's fibres are split evenly over (warp, fibre-slot) pairs, each sums its runs of equal c
// in registers (plan words prefetched one round ahead, U fibres in flight), stores inner runs and
// adds its first/last run (possibly shared with a neighbour) with shared-memory atomics.
// Phase 2 (k >= 1) adds coef(i_0) * Z[c, i_0] into bucket (c + h_0(i_0)) mod J of the CTA's
// column copy; consecutive threads take consecutive c, so the shared-memory atomics hit
// consecutive banks. The column is flushed to global with 16-byte vector atomics when the CTA
// moves to the next column. For mode 0, phase 2 writes the finished rows straight to Y_0.
// Y_k is column-major (J x n_k).
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

// A VB-byte vector of EPV elements of type DT: loaded as raw 32-bit words (so that U loads in
// flight cost U * VB/4 registers whatever the element type) and unpacked to floats when used.
template <int DT, int VB>
struct TtVec {
  static constexpr int EPV = VB / TtElem<DT>::bytes;
  static constexpr int W = (VB + 3) / 4;
  struct Raw {
    uint32_t w[W];
  };
  __device__ static Raw load(const char* p) {
    Raw r;
    if constexpr (VB == 16) {
      uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
      r.w[0] = u.x; r.w[1] = u.y; r.w[2] = u.z; r.w[3] = u.w;
    } else if constexpr (VB == 8) {
      uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
      r.w[0] = u.x; r.w[1] = u.y;
    } else if constexpr (VB == 4) {
      r.w[0] = __ldg(reinterpret_cast<const uint32_t*>(p));
    } else if constexpr (VB == 2) {
      r.w[0] = __ldg(reinterpret_cast<const unsigned short*>(p));
    } else {
      r.w[0] = __ldg(reinterpret_cast<const unsigned char*>(p));
    }
    return r;
  }
  __device__ static Raw zero() {
    Raw r;
#pragma unroll
    for (int i = 0; i < W; ++i) r.w[i] = 0u;
    return r;
  }
  // acc[e] += s * element e
  __device__ static void fma_into(const Raw& r, float s, float* acc) {
    const uint32_t* w = r.w;
    if constexpr (DT == TT_F32) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) acc[e] = fmaf(s, __uint_as_float(w[e]), acc[e]);
    } else if constexpr (DT == TT_F64) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) {
        unsigned long long b = ((unsigned long long)w[2 * e + 1] << 32) | w[2 * e];
        acc[e] = fmaf(s, (float)__longlong_as_double((long long)b), acc[e]);
      }
    } else if constexpr (DT == TT_BF16) {
#pragma unroll
      for (int e = 0; e < EPV; ++e)
        acc[e] = fmaf(s, __uint_as_float(((w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu) << 16), acc[e]);
    } else {
#pragma unroll
      for (int e = 0; e < EPV; ++e) acc[e] = fmaf(s, tt_fp8_e4m3((w[e >> 2] >> (8 * (e & 3))) & 0xFFu), acc[e]);
    }
  }
};

// Vector geometry of a fibre: VB-byte loads, vpf vectors per fibre, lanes per fibre slot and
// fibre slots per warp (several short fibres share one warp instruction).
struct FibreGeom {
  int64_t fiber_bytes;
  int vpf, lpf, fpi, nchunk;
};

static FibreGeom fibre_geom(int64_t fiber_bytes, int VB) {
  FibreGeom g;
  g.fiber_bytes = fiber_bytes;
  g.vpf = (int)(fiber_bytes / VB);
  if (g.vpf <= 32) {
    g.lpf = g.vpf;
    g.fpi = 32 / g.vpf;
    g.nchunk = 1;
  } else {
    g.lpf = 32;
    g.fpi = 1;
    g.nchunk = (g.vpf + 31) / 32;
  }
  return g;
}

// ---------------------------------------------------------------------------------------------
// the gather kernel

struct GArgs {
  const char* A;
  const float* scales;    // n0 FP8 scales or null
  const int32_t* h0;      // h_0 (n0 entries)
  const int8_t* v0;
  const uint32_t* plan;   // fibre index at i_k = 0 | sign in bit 31, grouped by c
  const int32_t* ulist;   // distinct c values
  const int64_t* ustart;  // starts into plan (U + 1)
  const int32_t* ucount;  // U
  float* Y;               // J x ncol column-major (zeroed by the host when k >= 1)
  int64_t col_fibres;     // fibre-index stride of the output column (stride_k / n0); 0 for mode 0
  int J, n0, ncol;
  int C;                  // c groups per chunk
  int pitch;              // row pitch of the Z chunk (odd)
  int elem_bytes;
  FibreGeom fg;
};

template <int DT, int VB, int U, bool MODE0>
__global__ void __launch_bounds__(256, 2) k_unfold_gather(GArgs a) {
  constexpr int EPV = TtVec<DT, VB>::EPV;
  extern __shared__ float sm[];
  const int J = a.J;
  float* Ys = sm;                                       // J (k >= 1 only)
  float* Zs = Ys + (MODE0 ? 0 : J);                     // C x pitch
  float* coef = Zs + (size_t)a.C * a.pitch;             // n0
  int* h0s = reinterpret_cast<int*>(coef + a.n0);       // n0
  int* cvals = h0s + a.n0;                              // C
  int64_t* cst = reinterpret_cast<int64_t*>(sm) + ((size_t)((MODE0 ? 0 : J) + a.C * a.pitch + 2 * a.n0 + a.C + 1) / 2);
  const int T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  for (int i = threadIdx.x; i < a.n0; i += T) {
    float cf = 1.f;
    if (!MODE0 && __ldg(a.v0 + i) < 0) cf = -1.f;
    if (a.scales) cf *= __ldg(a.scales + i);
    coef[i] = cf;
    h0s[i] = MODE0 ? 0 : __ldg(a.h0 + i);
  }
  const int64_t U_ = *a.ucount;
  const int64_t total = U_ * a.ncol;
  const int64_t lo = total * blockIdx.x / gridDim.x, hi = total * (blockIdx.x + 1) / gridDim.x;
  const int slot = lane / a.fg.lpf, posl = lane - slot * a.fg.lpf;
  const int nslots = nw * a.fg.fpi;
  const int gslot = warp * a.fg.fpi + slot;
  const bool slot_ok = slot < a.fg.fpi;
  int cur_col = -1;
  for (int64_t p0 = lo; p0 < hi;) {
    const int col = (int)(p0 / U_);
    const int64_t u0 = p0 - (int64_t)col * U_;
    const int64_t cend = min(hi, (int64_t)(col + 1) * U_);
    const int nc = (int)((cend - p0) < (int64_t)a.C ? (cend - p0) : (int64_t)a.C);
    if (!MODE0 && col != cur_col) {
      if (cur_col >= 0) {  // flush the finished column
        __syncthreads();
        float* yc = a.Y + (int64_t)J * cur_col;
        if ((J & 3) == 0) {
          for (int b = threadIdx.x * 4; b < J; b += T * 4) {
            float4 v4 = make_float4(Ys[b], Ys[b + 1], Ys[b + 2], Ys[b + 3]);
            atomicAdd(reinterpret_cast<float4*>(yc + b), v4);
          }
        } else {
          for (int b = threadIdx.x; b < J; b += T) atomicAdd(yc + b, Ys[b]);
        }
        __syncthreads();
      }
      for (int i = threadIdx.x; i < J; i += T) Ys[i] = 0.f;
      cur_col = col;
    }
    for (int i = threadIdx.x; i < nc * a.pitch; i += T) Zs[i] = 0.f;
    for (int i = threadIdx.x; i <= nc; i += T) {
      cst[i] = __ldg(a.ustart + u0 + i);
      if (i < nc) cvals[i] = __ldg(a.ulist + u0 + i);
    }
    __syncthreads();
    // ---- phase 1: Z rows of the chunk by fibre gathers
    {
      const int64_t e0 = cst[0], ne = cst[nc] - e0;
      const int64_t sb = e0 + ne * gslot / nslots, se = e0 + ne * (gslot + 1) / nslots;
      const int64_t colf = (int64_t)col * a.col_fibres;
      if (slot_ok && sb < se) {
        // run containing sb: largest cu with cst[cu] <= sb
        int lo2 = 0, hi2 = nc;  // cst[lo2] <= sb < cst[hi2]
        while (hi2 - lo2 > 1) {
          const int mid = (lo2 + hi2) >> 1;
          if (cst[mid] <= sb) lo2 = mid; else hi2 = mid;
        }
        for (int ch = 0; ch < a.fg.nchunk; ++ch) {
          const int vpos = ch * 32 + posl;
          const bool lane_ok = vpos < a.fg.vpf;
          const int64_t vbyte = (int64_t)vpos * VB;
          int cu = lo2;
          int64_t next_b = cst[cu + 1];
          bool first_run = true;
          float acc[EPV];
#pragma unroll
          for (int e = 0; e < EPV; ++e) acc[e] = 0.f;
          uint32_t wn[U];
#pragma unroll
          for (int q = 0; q < U; ++q) wn[q] = (sb + q < se) ? __ldg(a.plan + sb + q) : 0u;
          for (int64_t j0 = sb; j0 < se; j0 += U) {
            typename TtVec<DT, VB>::Raw v[U];
            uint32_t w[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
              w[q] = wn[q];
              if (lane_ok && j0 + q < se) {
                const int64_t fib = (int64_t)(w[q] & 0x7FFFFFFFu) + colf;
                v[q] = TtVec<DT, VB>::load(a.A + fib * a.fg.fiber_bytes + vbyte);
              } else {
                v[q] = TtVec<DT, VB>::zero();
              }
            }
#pragma unroll
            for (int q = 0; q < U; ++q) wn[q] = (j0 + U + q < se) ? __ldg(a.plan + j0 + U + q) : 0u;
#pragma unroll
            for (int q = 0; q < U; ++q) {
              const int64_t j = j0 + q;
              if (j < se) {
                if (j >= next_b) {  // the run of group cu ended: write it
                  if (lane_ok) {
                    float* z = Zs + (size_t)cu * a.pitch + vpos * EPV;
                    if (first_run) {
#pragma unroll
                      for (int e = 0; e < EPV; ++e) atomicAdd(z + e, acc[e]);
                    } else {
#pragma unroll
                      for (int e = 0; e < EPV; ++e) z[e] = acc[e];
                    }
                  }
#pragma unroll
                  for (int e = 0; e < EPV; ++e) acc[e] = 0.f;
                  first_run = false;
                  do {
                    ++cu;
                    next_b = cst[cu + 1];
                  } while (j >= next_b);
                }
                TtVec<DT, VB>::fma_into(v[q], (w[q] >> 31) ? -1.f : 1.f, acc);
              }
            }
          }
          if (lane_ok) {  // the slot's last run may be shared with the next slot
            float* z = Zs + (size_t)cu * a.pitch + vpos * EPV;
#pragma unroll
            for (int e = 0; e < EPV; ++e) atomicAdd(z + e, acc[e]);
          }
        }
      }
    }
    __syncthreads();
    // ---- phase 2
    if (MODE0) {
      // finished rows c of Y_0: Y_0[c + J i0] = scale(i0) * Z[c, i0] (consecutive c: coalesced)
      for (int idx = threadIdx.x; idx < nc * a.n0; idx += T) {
        const int ul = idx % nc, i0 = idx / nc;
        a.Y[cvals[ul] + (int64_t)J * i0] = coef[i0] * Zs[(size_t)ul * a.pitch + i0];
      }
    } else {
      for (int idx = threadIdx.x; idx < nc * a.n0; idx += T) {
        const int ul = idx % nc, i0 = idx / nc;
        const int b = (cvals[ul] + h0s[i0]) & (J - 1);
        atomicAdd(Ys + b, coef[i0] * Zs[(size_t)ul * a.pitch + i0]);
      }
    }
    __syncthreads();
    p0 += nc;
  }
  if (!MODE0 && cur_col >= 0) {
    __syncthreads();
    float* yc = a.Y + (int64_t)J * cur_col;
    if ((J & 3) == 0) {
      for (int b = threadIdx.x * 4; b < J; b += T * 4) {
        float4 v4 = make_float4(Ys[b], Ys[b + 1], Ys[b + 2], Ys[b + 3]);
        atomicAdd(reinterpret_cast<float4*>(yc + b), v4);
      }
    } else {
      for (int b = threadIdx.x; b < J; b += T) atomicAdd(yc + b, Ys[b]);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// host side

static int pick_vb(int64_t fiber_bytes, uintptr_t base, int elem_bytes) {
  for (int vb = 16; vb >= elem_bytes; vb >>= 1)
    if (fiber_bytes % vb == 0 && base % vb == 0) return vb;
  return elem_bytes;
}

static size_t gather_smem(int J, bool mode0, int C, int pitch, int n0) {
  size_t words = (size_t)(mode0 ? 0 : J) + (size_t)C * pitch + 2 * (size_t)n0 + C + 1;
  words = (words + 1) & ~(size_t)1;  // cst is 8-byte aligned
  return words * 4 + sizeof(int64_t) * (C + 1);
}

template <int DT, int VB, bool MODE0>
static int launch_gather_vb(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  constexpr int U = 8;
  GArgs a;
  a.A = (const char*)A;
  a.scales = scales;
  a.h0 = c->d_h;
  a.v0 = c->d_v;
  a.plan = c->d_rplan[k];
  a.ulist = c->d_ulist[k];
  a.ustart = c->d_ustart[k];
  a.ucount = c->d_ucount[k];
  a.Y = Y;
  a.J = c->J;
  a.n0 = (int)c->n[0];
  a.ncol = MODE0 ? 1 : (int)c->n[k];
  a.col_fibres = MODE0 ? 0 : c->stride[k] / c->n[0];
  a.elem_bytes = TtElem<DT>::bytes;
  a.fg = fibre_geom((int64_t)c->n[0] * TtElem<DT>::bytes, VB);
  a.pitch = (a.n0 % 2 == 0) ? a.n0 + 1 : a.n0;
  // chunk size: aim at two CTAs per SM (about 105 KB of shared memory each)
  const size_t target = 105 * 1024;
  int C = 256;
  while (C > 32 && gather_smem(c->J, MODE0, C, a.pitch, a.n0) > target) C -= 32;
  while (C > 1 && gather_smem(c->J, MODE0, C, a.pitch, a.n0) > 220 * 1024) C >>= 1;
  a.C = C;
  const size_t smem = gather_smem(c->J, MODE0, C, a.pitch, a.n0);
  if (smem > 220 * 1024) return tt_fail(c, TT_EINVAL, "gather kernel needs %zu bytes of shared memory", smem);
  TT_CUDA(c, cudaMemsetAsync(Y, 0, sizeof(float) * c->J * c->n[k], c->stream));  // empty groups stay 0
  TT_CUDA(c, cudaFuncSetAttribute(k_unfold_gather<DT, VB, U, MODE0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1;
  TT_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_unfold_gather<DT, VB, U, MODE0>, 256, smem));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int blocks = std::max(1, sms * std::max(1, per_sm));
  k_unfold_gather<DT, VB, U, MODE0><<<blocks, 256, smem, c->stream>>>(a);
  TT_LAUNCH(c, "k_unfold_gather");
  return TT_OK;
}

template <int DT, bool MODE0>
static int launch_gather(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  constexpr int EB = TtElem<DT>::bytes;
  const int vb = pick_vb((int64_t)c->n[0] * EB, (uintptr_t)A, EB);
  switch (vb) {
    case 16: return launch_gather_vb<DT, 16, MODE0>(c, A, scales, k, Y);
    case 8: return launch_gather_vb<DT, (EB <= 8 ? 8 : 16), MODE0>(c, A, scales, k, Y);
    case 4: return launch_gather_vb<DT, (EB <= 4 ? 4 : EB), MODE0>(c, A, scales, k, Y);
    case 2: return launch_gather_vb<DT, (EB <= 2 ? 2 : EB), MODE0>(c, A, scales, k, Y);
    default: return launch_gather_vb<DT, EB, MODE0>(c, A, scales, k, Y);
  }
}

template <int DT>
static int unfold_dt(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  if (k == 0) return launch_gather<DT, true>(c, A, scales, k, Y);
  return launch_gather<DT, false>(c, A, scales, k, Y);
}

int tt_launch_unfold(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  int rc = tt_ensure_rplan(c, k);  // plan build is not part of the timed kernel
  if (rc) return rc;
  rc = tt_prof_begin(c, k);
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
