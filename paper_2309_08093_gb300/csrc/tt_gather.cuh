// The gather kernels of the data sketch (Alg. 1 part (a); the regrouping by mode-0 fibres is
// described in tt_unfold.cu): k_unfold_gather (one output column per work item) and
// k_unfold_cols (G neighbouring columns per work item, modes >= 1). Fibres of a per-sweep plan are
// staged with cp.async in VB-byte vectors and summed in registers run by run. Shared by
// tt_unfold.cu (FP32 flushes) and tt_det.cu (the deterministic mode's 64-bit fixed-point flushes,
// DET = true).
#pragma once

#include "tt_unfold.cuh"

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
  // acc[e] += s * element e (s = +-1, the sign of a plan entry)
  __device__ static void fma_into(const Raw& r, float s, float* acc) {
    const uint32_t* w = r.w;
    if constexpr (DT == TT_F32 && EPV % 2 == 0) {  // pairs of entries: one fma.rn.f32x2 each
#pragma unroll
      for (int e = 0; e < EPV; e += 2) {
        const float2 d = tt_ffma2(make_float2(s, s), make_float2(__uint_as_float(w[e]), __uint_as_float(w[e + 1])),
                                  make_float2(acc[e], acc[e + 1]));
        acc[e] = d.x;
        acc[e + 1] = d.y;
      }
    } else if constexpr (DT == TT_F32) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) acc[e] = fmaf(s, __uint_as_float(w[e]), acc[e]);
    } else if constexpr (DT == TT_F64) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) {
        unsigned long long b = ((unsigned long long)w[2 * e + 1] << 32) | w[2 * e];
        acc[e] = fmaf(s, (float)__longlong_as_double((long long)b), acc[e]);
      }
    } else if constexpr (DT == TT_BF16) {  // a 32-bit word holds two entries: two mixed BF16 FMAs
      const unsigned short sb = tt_bf16_sign(s);
#pragma unroll
      for (int e = 0; e < EPV; e += 2) tt_fma_bf16x2(w[e >> 1], sb, acc[e], acc[e + 1]);
    } else if constexpr (EPV % 4 == 0) {  // FP8: four entries per word, hardware conversions
      const unsigned short sh = tt_f16_sign(s);
#pragma unroll
      for (int e = 0; e < EPV; e += 4) tt_fma_e4m3x4(w[e >> 2], sh, acc[e], acc[e + 1], acc[e + 2], acc[e + 3]);
    } else {
      const unsigned short sh = tt_f16_sign(s);
#pragma unroll
      for (int e = 0; e < EPV; ++e) acc[e] = tt_fma_e4m3((unsigned short)((w[e >> 2] >> (8 * (e & 3))) & 0xFFu), sh, acc[e]);
    }
  }
};

static inline FibreGeom fibre_geom(int64_t fiber_bytes, int VB, int M) {
  FibreGeom g;
  g.fiber_bytes = fiber_bytes;
  g.m = M;
  g.vpf = (int)(fiber_bytes / VB);
  const int lanes = (g.vpf + M - 1) / M;
  if (lanes <= 32) {
    g.lpf = lanes;
    g.fpi = 32 / lanes;
    g.nchunk = 1;
  } else {
    g.lpf = 32;
    g.fpi = 1;
    g.nchunk = (g.vpf + 32 * M - 1) / (32 * M);
  }
  return g;
}

// vectors per lane for a fibre of vpf VB-byte vectors: the most fibre slots per warp (fewest warp
// instructions per fibre), ties to the smaller m; at most 16 elements per lane (registers)
static inline int pick_m(int vpf, int epv) {
  int best = 1, best_fpi = 0;
  for (int M : {1, 2, 4}) {
    if (M * epv > 16) break;
    const int lanes = (vpf + M - 1) / M;
    const int fpi = lanes <= 32 ? 32 / lanes : 0;
    if (fpi > best_fpi) {
      best = M;
      best_fpi = fpi;
    }
  }
  return best;
}

// ---------------------------------------------------------------------------------------------
// the gather kernel

__device__ __forceinline__ void cp_async_vec(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}

// One work item = a contiguous segment of c groups of one output column (mode 0: of Y_0's
// rows). The item's fibres are split evenly over the (warp, fibre-slot) pairs; each lane keeps S
// fibres of M VB-byte pieces in flight with cp.async (one commit group per fibre, the stage is
// refilled as soon as it is consumed) and sums runs of equal c in registers. When a run ends:
//   mode 0  : the finished row goes to Y_0 (plain store if the run lies inside this slot's range,
//             atomic add otherwise);
//   mode >= 1: coef(i0) * run is added into bucket (c + h_0(i0)) mod J of the CTA's column copy.
// DET (deterministic mode): a finished run's sum (its fibres added in the order of a
// deterministic plan, so the same float on every call) becomes the integer round(sum 2^S)
// (det_fixed) and is added with 64-bit integer atomics, whose order does not matter: rows of
// a.Yq (mode 0) and the CTA's int64 column copy, then a.Yq (modes >= 1).
template <int DT, int VB, int S, int M, bool MODE0, bool DET = false>
__global__ void __launch_bounds__(256, 2) k_unfold_gather(GArgs a) {
  constexpr bool ASYNC = VB >= 4;  // cp.async moves 4, 8 or 16 bytes; 1-2 byte vectors load directly
  static_assert(ASYNC || M == 1, "direct loads use one vector per lane");
  constexpr int EPV = TtVec<DT, VB>::EPV;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int J = a.J;
  const int T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  unsigned char* ring = smraw;                                           // nw x S x M x 32 x VB
  unsigned char* ysraw = ring + gather_ring_bytes(ASYNC, nw, S * M, VB);
  float* Ys = reinterpret_cast<float*>(ysraw);                           // J (mode >= 1)
  unsigned long long* Yqs = reinterpret_cast<unsigned long long*>(ysraw);  // J (mode >= 1, DET)
  int* sstart = reinterpret_cast<int*>(ysraw + (MODE0 ? 0 : (size_t)J * (DET ? 8 : 4)));  // segmax + 1
  if constexpr (DET) {
    if (a.det_S[1] != 0) return;  // {S, A not finite}: the sketches are written as NaN afterwards
  }
  const int dS = DET ? *a.det_S : 0;
  int* scval = sstart + a.segmax + 1;                                    // segmax
  const int U_ = *a.ucount;
  const int lpf = a.fg.lpf;
  const int slot = lane / lpf, posl = lane - slot * lpf;
  const bool slot_ok = slot < a.fg.fpi;
  const int nslots = nw * a.fg.fpi;
  const int gslot = warp * a.fg.fpi + slot;
  unsigned char* myring = ring + ((size_t)warp * S * M * 32 + lane) * VB;
  const int items = a.ncol * a.nseg;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int col = item / a.nseg, seg = item - col * a.nseg;
    const int ua = (int)((int64_t)U_ * seg / a.nseg), ub = (int)((int64_t)U_ * (seg + 1) / a.nseg);
    const int nu = ub - ua;
    if (nu <= 0) continue;
    const int64_t e0 = __ldg(a.ustart + ua);
    for (int i = threadIdx.x; i <= nu; i += T) {
      sstart[i] = (int)(__ldg(a.ustart + ua + i) - e0);
      if (i < nu) scval[i] = __ldg(a.ulist + ua + i);
    }
    if (!MODE0)
      for (int i = threadIdx.x; i < J; i += T) {
        if constexpr (DET) Yqs[i] = 0ull; else Ys[i] = 0.f;
      }
    __syncthreads();
    const int ne = sstart[nu];
    const char* Acol = a.A + (int64_t)col * a.col_fibres * a.fg.fiber_bytes;
    const uint32_t* plan = a.plan + e0;
    // the item's fibres split into nch spans, span t on slot t mod nslots: one span per slot in
    // the fast path; in DET a count fixed by the shape alone, so that the run sums (and so the
    // bits) do not depend on the vector width or the slots per warp
    const int nch = DET ? a.nch : nslots;
    int chk = gslot;
    do {  // once in the fast path (a plain block)
      const int sb = (int)((int64_t)ne * chk / nch), se = (int)((int64_t)ne * (chk + 1) / nch);
      if (slot_ok && sb < se) {
        int lo2 = 0, hi2 = nu;  // run containing sb: sstart[lo2] <= sb < sstart[hi2]
        while (hi2 - lo2 > 1) {
          const int mid = (lo2 + hi2) >> 1;
          if (sstart[mid] <= sb) lo2 = mid; else hi2 = mid;
        }
        const int count = se - sb;
        for (int ch = 0; ch < a.fg.nchunk; ++ch) {
          int vpos[M];
          bool vok[M];
          float coefr[M][EPV];
          int h0r[M][EPV];
  #pragma unroll
          for (int mm = 0; mm < M; ++mm) {
            vpos[mm] = ch * lpf * M + mm * lpf + posl;
            vok[mm] = vpos[mm] < a.fg.vpf;
  #pragma unroll
            for (int e = 0; e < EPV; ++e) {
              const int i0 = vpos[mm] * EPV + e;
              float cf = 1.f;
              int hh = 0;
              if (vok[mm]) {
                if (!MODE0 && __ldg(a.v0 + i0) < 0) cf = -1.f;
                if (a.scales) cf *= __ldg(a.scales + i0);
                if (!MODE0) hh = __ldg(a.h0 + i0);
              }
              coefr[mm][e] = cf;
              h0r[mm][e] = hh;
            }
          }
          const char* Alane[M];
  #pragma unroll
          for (int mm = 0; mm < M; ++mm) Alane[mm] = Acol + (int64_t)vpos[mm] * VB;
          int cu = lo2;
          int next_b = sstart[cu + 1];
          bool first_run = true;
          float acc[M][EPV];
  #pragma unroll
          for (int mm = 0; mm < M; ++mm)
  #pragma unroll
            for (int e = 0; e < EPV; ++e) acc[mm][e] = 0.f;
          // flush of the run of group cu (shared with a neighbour slot when `shared`)
          auto flush = [&](bool shared) {
            const int cv = scval[cu];
  #pragma unroll
            for (int mm = 0; mm < M; ++mm) {
              if (vok[mm]) {
                if (MODE0) {
  #pragma unroll
                  for (int e = 0; e < EPV; ++e) {
                    const float v = coefr[mm][e] * acc[mm][e];
                    if constexpr (DET) {
                      unsigned long long* dst = a.Yq + cv + (int64_t)J * (vpos[mm] * EPV + e);
                      const unsigned long long q = (unsigned long long)det_fixed(v, dS);
                      if (shared) atomicAdd(dst, q); else *dst = q;
                    } else {
                      float* dst = a.Y + cv + (int64_t)J * (vpos[mm] * EPV + e);
                      if (shared) atomicAdd(dst, v); else *dst = v;
                    }
                  }
                } else {
  #pragma unroll
                  for (int e = 0; e < EPV; ++e) {
                    const int bk = tt_modj(cv + h0r[mm][e], J);
                    if constexpr (DET)
                      atomicAdd(Yqs + bk, (unsigned long long)det_fixed(coefr[mm][e] * acc[mm][e], dS));
                    else
                      atomicAdd(Ys + bk, coefr[mm][e] * acc[mm][e]);
                  }
                }
              }
  #pragma unroll
              for (int e = 0; e < EPV; ++e) acc[mm][e] = 0.f;
            }
          };
          // pipeline: stage q of the ring holds fibre j with j % S == q (M pieces per lane)
          uint32_t wcur[S], wnext[S];
  #pragma unroll
          for (int q = 0; q < S; ++q) {
            wcur[q] = (q < count) ? __ldg(plan + sb + q) : 0u;
            if constexpr (ASYNC) {
              if (q < count) {
                const int64_t fo = (int64_t)(wcur[q] & 0x7FFFFFFFu) * a.fg.fiber_bytes;
  #pragma unroll
                for (int mm = 0; mm < M; ++mm)
                  if (vok[mm]) cp_async_vec(myring + (size_t)(q * M + mm) * 32 * VB, Alane[mm] + fo, VB);
              }
              cp_async_commit();
            }
            wnext[q] = (S + q < count) ? __ldg(plan + sb + S + q) : 0u;
          }
          for (int j0 = 0; j0 < count; j0 += S) {
  #pragma unroll
            for (int q = 0; q < S; ++q) {
              const int j = j0 + q;
              if (j < count) {
                typename TtVec<DT, VB>::Raw raw[M];
                if constexpr (ASYNC) {
                  cp_async_wait<S - 1>();
  #pragma unroll
                  for (int mm = 0; mm < M; ++mm) {
                    if (vok[mm]) {
                      const unsigned char* src = myring + (size_t)(q * M + mm) * 32 * VB;
                      if constexpr (VB == 16) {
                        const uint4 w4 = *reinterpret_cast<const uint4*>(src);
                        raw[mm].w[0] = w4.x; raw[mm].w[1] = w4.y; raw[mm].w[2] = w4.z; raw[mm].w[3] = w4.w;
                      } else {
  #pragma unroll
                        for (int t2 = 0; t2 < TtVec<DT, VB>::W; ++t2) raw[mm].w[t2] = reinterpret_cast<const uint32_t*>(src)[t2];
                      }
                    } else {
                      raw[mm] = TtVec<DT, VB>::zero();
                    }
                  }
                } else {
                  raw[0] = vok[0] ? TtVec<DT, VB>::load(Alane[0] + (int64_t)(wcur[q] & 0x7FFFFFFFu) * a.fg.fiber_bytes)
                                  : TtVec<DT, VB>::zero();
                }
                const int jr = sb + j;  // position within the item
                if (jr >= next_b) {
                  flush(first_run || (sstart[cu] < sb));
                  first_run = false;
                  do {
                    ++cu;
                    next_b = sstart[cu + 1];
                  } while (jr >= next_b);
                }
                const float sg = (wcur[q] >> 31) ? -1.f : 1.f;
  #pragma unroll
                for (int mm = 0; mm < M; ++mm) TtVec<DT, VB>::fma_into(raw[mm], sg, acc[mm]);
                // refill stage q with fibre j + S, prefetch the plan word of fibre j + 2S
                const int jn = j + S;
                if constexpr (ASYNC) {
                  if (jn < count) {
                    const int64_t fo = (int64_t)(wnext[q] & 0x7FFFFFFFu) * a.fg.fiber_bytes;
  #pragma unroll
                    for (int mm = 0; mm < M; ++mm)
                      if (vok[mm]) cp_async_vec(myring + (size_t)(q * M + mm) * 32 * VB, Alane[mm] + fo, VB);
                  }
                  cp_async_commit();
                }
                wcur[q] = wnext[q];
                wnext[q] = (jn + S < count) ? __ldg(plan + sb + jn + S) : 0u;
              }
            }
          }
          if constexpr (ASYNC) cp_async_wait<0>();
          // last run: shared with the next slot unless it ends exactly at se
          flush(first_run || sstart[cu] < sb || sstart[cu + 1] > se);
        }
      }
      chk += nslots;
    } while (DET && chk < nch);
    __syncthreads();
    if (!MODE0 && DET) {  // add the column copy to a.Yq
      unsigned long long* yc = a.Yq + (int64_t)J * col;
      for (int b = threadIdx.x; b < J; b += T)
        if (Yqs[b]) atomicAdd(yc + b, Yqs[b]);
      __syncthreads();
    } else if (!MODE0) {  // flush the column copy
      float* yc = a.Y + (int64_t)J * col;
      if (a.y_vec4) {
        for (int b = threadIdx.x * 4; b < J; b += T * 4) {
          const float4 v4 = make_float4(Ys[b], Ys[b + 1], Ys[b + 2], Ys[b + 3]);
          if (v4.x != 0.f || v4.y != 0.f || v4.z != 0.f || v4.w != 0.f) atomicAdd(reinterpret_cast<float4*>(yc + b), v4);
        }
      } else {
        for (int b = threadIdx.x; b < J; b += T) atomicAdd(yc + b, Ys[b]);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------------------------
// modes >= 1, G columns at once. The plan of mode k lists the rest fibres r by tail hash c_r and
// is the same for every output column i_k, so one work item takes G neighbouring columns
// (i_k = G g .. G g + G - 1) and one c-segment: a warp walks its slice of the segment and, per plan
// entry r, gathers the G fibres A(:, r, i_k) (neighbours in memory for mode 1). Lane l holds the
// MV vectors v = l + 32 m of the G * vpf vectors of an entry (column v / vpf, piece v % vpf), keeps
// S entries in flight with cp.async and sums runs of equal c in registers; a run's end (the same
// for every lane: all of them walk the same entries) adds coef(i_0) * sum into bucket
// (c + h_0(i_0)) mod J of the CTA's copy of the column. The G column copies are flushed to Y_k
// with 16-byte atomics at the end of the item.
// DET: as in k_unfold_gather, int64 column copies and fixed-point flushes; an item's entries are
// cut into a.nch spans (span t on warp t mod 8), the same spans as k_unfold_gather<DET> takes for
// each of the columns, so the two kernels give the same bits.
template <int DT, int VB, int S, int MV, int G, bool DET = false>
__global__ void __launch_bounds__(256, 2) k_unfold_cols(GArgs a) {
  constexpr int EPV = TtVec<DT, VB>::EPV;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int J = a.J;
  const int T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  unsigned char* ring = smraw;                                                // nw x S x MV x 32 x VB
  float* Ys = reinterpret_cast<float*>(ring + gather_ring_bytes(true, nw, S * MV, VB));  // G x J
  unsigned long long* Yqs = reinterpret_cast<unsigned long long*>(Ys);     // G x J (DET)
  int* sstart = reinterpret_cast<int*>(Ys + (size_t)G * (J + TT_YPAD) * (DET ? 2 : 1));  // segmax + 1 (relative)
  int* scval = sstart + a.segmax + 1;                                        // segmax
  if constexpr (DET) {
    if (a.det_S[1] != 0) return;  // {S, A not finite}: the sketches are written as NaN afterwards
  }
  const int dS = DET ? *a.det_S : 0;
  const int U_ = *a.ucount;
  const int vpf = a.fg.vpf;
  unsigned char* myring = ring + ((size_t)warp * S * MV * 32 + lane) * VB;
  // this lane's vectors of an entry and their coefficients (fixed for the whole kernel)
  int vg[MV], vp[MV];
  float coefr[MV][EPV];
  int h0r[MV][EPV];
#pragma unroll
  for (int m = 0; m < MV; ++m) {
    const int v = lane + 32 * m;
    const bool in = v < G * vpf;
    vg[m] = in ? v / vpf : 0;
    vp[m] = in ? v - vg[m] * vpf : 0;
#pragma unroll
    for (int e = 0; e < EPV; ++e) {
      const int i0 = vp[m] * EPV + e;
      float cf = 0.f;
      int hh = 0;
      if (in) {
        cf = __ldg(a.v0 + i0) < 0 ? -1.f : 1.f;
        if (a.scales) cf *= __ldg(a.scales + i0);
        hh = __ldg(a.h0 + i0);
      }
      coefr[m][e] = cf;
      h0r[m][e] = hh;
    }
  }
  const int ncolg = (a.ncol + G - 1) / G;
  const int items = ncolg * a.nseg;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int colg = item / a.nseg, seg = item - colg * a.nseg;
    const int col0 = colg * G;
    const int ua = (int)((int64_t)U_ * seg / a.nseg), ub = (int)((int64_t)U_ * (seg + 1) / a.nseg);
    const int nu = ub - ua;
    if (nu <= 0) continue;
    const int64_t e0 = __ldg(a.ustart + ua);
    for (int i = threadIdx.x; i <= nu; i += T) {
      sstart[i] = (int)(__ldg(a.ustart + ua + i) - e0);
      if (i < nu) scval[i] = __ldg(a.ulist + ua + i);
    }
    for (int i = threadIdx.x; i < G * (J + TT_YPAD); i += T) {
      if constexpr (DET) Yqs[i] = 0ull; else Ys[i] = 0.f;
    }
    __syncthreads();
    const int ne = sstart[nu];
    const int nch = DET ? a.nch : nw;
    const uint32_t* plan = a.plan + e0;
    bool vok[MV];
    const char* Alane[MV];
#pragma unroll
    for (int m = 0; m < MV; ++m) {
      vok[m] = lane + 32 * m < G * vpf && col0 + vg[m] < a.ncol;
      Alane[m] = a.A + ((int64_t)(col0 + vg[m]) * a.col_fibres) * a.fg.fiber_bytes + (int64_t)vp[m] * VB;
    }
    int chk = warp;
    do {  // once in the fast path (a plain block)
      const int sb = (int)((int64_t)ne * chk / nch), se = (int)((int64_t)ne * (chk + 1) / nch);
      if (sb < se) {
        int lo2 = 0, hi2 = nu;  // run containing sb: sstart[lo2] <= sb < sstart[hi2]
        while (hi2 - lo2 > 1) {
          const int mid = (lo2 + hi2) >> 1;
          if (sstart[mid] <= sb) lo2 = mid; else hi2 = mid;
        }
        const int count = se - sb;
        int cu = lo2;
        int next_b = sstart[cu + 1];
        float acc[MV][EPV];
#pragma unroll
        for (int m = 0; m < MV; ++m)
#pragma unroll
          for (int e = 0; e < EPV; ++e) acc[m][e] = 0.f;
        auto flush = [&]() {
          const int cv = scval[cu];
#pragma unroll
          for (int m = 0; m < MV; ++m) {
            if (vok[m]) {
              if constexpr (DET) {
                unsigned long long* yc = Yqs + (size_t)vg[m] * (J + TT_YPAD);
#pragma unroll
                for (int e = 0; e < EPV; ++e)
                  atomicAdd(yc + tt_modj(cv + h0r[m][e], J), (unsigned long long)det_fixed(coefr[m][e] * acc[m][e], dS));
              } else {
                float* yc = Ys + (size_t)vg[m] * (J + TT_YPAD);
#pragma unroll
                for (int e = 0; e < EPV; ++e) atomicAdd(yc + tt_modj(cv + h0r[m][e], J), coefr[m][e] * acc[m][e]);
              }
            }
#pragma unroll
            for (int e = 0; e < EPV; ++e) acc[m][e] = 0.f;
          }
        };
        // pipeline: stage q of the ring holds entry j with j % S == q (MV pieces per lane)
        uint32_t wcur[S], wnext[S];
#pragma unroll
        for (int q = 0; q < S; ++q) {
          wcur[q] = (q < count) ? __ldg(plan + sb + q) : 0u;
          if (q < count) {
            const int64_t fo = (int64_t)(wcur[q] & 0x7FFFFFFFu) * a.fg.fiber_bytes;
#pragma unroll
            for (int m = 0; m < MV; ++m)
              if (vok[m]) cp_async_vec(myring + (size_t)(q * MV + m) * 32 * VB, Alane[m] + fo, VB);
          }
          cp_async_commit();
          wnext[q] = (S + q < count) ? __ldg(plan + sb + S + q) : 0u;
        }
        for (int j0 = 0; j0 < count; j0 += S) {
#pragma unroll
          for (int q = 0; q < S; ++q) {
            const int j = j0 + q;
            if (j < count) {
              typename TtVec<DT, VB>::Raw raw[MV];
              cp_async_wait<S - 1>();
#pragma unroll
              for (int m = 0; m < MV; ++m) {
                if (vok[m]) {
                  const unsigned char* src = myring + (size_t)(q * MV + m) * 32 * VB;
                  if constexpr (VB == 16) {
                    const uint4 w4 = *reinterpret_cast<const uint4*>(src);
                    raw[m].w[0] = w4.x; raw[m].w[1] = w4.y; raw[m].w[2] = w4.z; raw[m].w[3] = w4.w;
                  } else {
#pragma unroll
                    for (int t2 = 0; t2 < TtVec<DT, VB>::W; ++t2) raw[m].w[t2] = reinterpret_cast<const uint32_t*>(src)[t2];
                  }
                } else {
                  raw[m] = TtVec<DT, VB>::zero();
                }
              }
              const int jr = sb + j;
              if (jr >= next_b) {
                flush();
                do {
                  ++cu;
                  next_b = sstart[cu + 1];
                } while (jr >= next_b);
              }
              const float sg = (wcur[q] >> 31) ? -1.f : 1.f;
#pragma unroll
              for (int m = 0; m < MV; ++m) TtVec<DT, VB>::fma_into(raw[m], sg, acc[m]);
              const int jn = j + S;
              if (jn < count) {
                const int64_t fo = (int64_t)(wnext[q] & 0x7FFFFFFFu) * a.fg.fiber_bytes;
#pragma unroll
                for (int m = 0; m < MV; ++m)
                  if (vok[m]) cp_async_vec(myring + (size_t)(q * MV + m) * 32 * VB, Alane[m] + fo, VB);
              }
              cp_async_commit();
              wcur[q] = wnext[q];
              wnext[q] = (jn + S < count) ? __ldg(plan + sb + jn + S) : 0u;
            }
          }
        }
        cp_async_wait<0>();
        flush();
      }
      chk += nw;
    } while (DET && chk < nch);
    __syncthreads();
    // flush the G column copies
    if constexpr (DET) {
      for (int g = 0; g < G && col0 + g < a.ncol; ++g) {
        unsigned long long* yc = a.Yq + (int64_t)J * (col0 + g);
        const unsigned long long* ys = Yqs + (size_t)g * (J + TT_YPAD);
        for (int b = threadIdx.x; b < J; b += T)
          if (ys[b]) atomicAdd(yc + b, ys[b]);
      }
    } else {
      for (int g = 0; g < G && col0 + g < a.ncol; ++g) {
        float* yc = a.Y + (int64_t)J * (col0 + g);
        const float* ys = Ys + (size_t)g * (J + TT_YPAD);
        if (a.y_vec4) {
          for (int b = threadIdx.x * 4; b < J; b += T * 4) {
            const float4 v4 = make_float4(ys[b], ys[b + 1], ys[b + 2], ys[b + 3]);
            if (v4.x != 0.f || v4.y != 0.f || v4.z != 0.f || v4.w != 0.f) atomicAdd(reinterpret_cast<float4*>(yc + b), v4);
          }
        } else {
          for (int b = threadIdx.x; b < J; b += T)
            if (ys[b] != 0.f) atomicAdd(yc + b, ys[b]);
        }
      }
    }
    __syncthreads();
  }
}

// the widest vector (16, 8, 4, 2 or 1 bytes) that both the fibre length and A's base allow
static inline int pick_vb(int64_t fiber_bytes, uintptr_t base, int elem_bytes) {
  for (int vb = 16; vb >= elem_bytes; vb >>= 1)
    if (fiber_bytes % vb == 0 && base % vb == 0) return vb;
  return elem_bytes;
}

