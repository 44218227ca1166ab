// Part (a) of Alg. 1, the data sketch Y_k = S A_(k)^T (Eqs. (eqn_h), (eqn_v); the regrouping by
// mode-0 fibres is that of tt_unfold.cu), for tensors whose mode-0 fibres do not start on a
// 16-byte boundary: n_0 * element bytes is not a multiple of 16, so fibre f starts at byte
// f * n_0 * element bytes, on a 1-, 2- or 4-byte boundary that changes from fibre to fibre (the
// 8-byte case keeps the 8-byte vector kernels of tt_unfold.cu).
//
// Window staging. A fibre is fetched as the 16-byte-aligned window around it: window vector w
// covers bytes [16 w, 16 w + 16) from the aligned address at or below the fibre's first byte, and
// only the window vectors that hold a byte of the fibre are copied (cp.async, 16 bytes), the last
// one clipped at the end of the tensor (the copy's source size; the rest is zero-filled). Every
// copy is thus a whole 16-byte vector inside A, whatever the fibre's alignment, where loads of
// the fibre itself could only be as wide as that alignment.
//
// The window lands in the fibre's region of a shared-memory stage; the fibre starts m = (byte
// offset of the fibre) mod 16 bytes into it. The lpf lanes that serve a fibre own fixed entries
// i_0 = posl + lpf t (t < EPT) and read entry i_0 at region + m + i_0 * element bytes: one
// shared-memory load at a fixed offset from (region + m), consecutive lanes on consecutive words.
// Lanes read vectors their neighbours copied, so the fibre's lanes synchronise (__syncwarp) after
// the copies land and before the stage is refilled. Entries t with i_0 >= n_0 are read and summed
// too (whatever the region holds there; the region is sized so those reads stay inside it) but
// never flushed, which keeps the inner loop free of per-entry tests.
#include <algorithm>

#include "tt_unfold.cuh"

namespace {

// Bytes of a fibre's region of a stage: the window (ceil(fibre bytes / 16) + 1 vectors) and every
// entry slot its lanes read (offsets below 16 + lpf * ept * element bytes), in 16-byte vectors
// whose count makes the 32-bit word offset of neighbouring regions differ by max(4, lpf) modulo 32
// (the lanes of neighbouring fibres then read different shared-memory banks).
int win_stride(int64_t fb, int eb, int lpf, int ept) {
  const int nw16 = (int)((fb + 15) / 16) + 1;
  int v = std::max(nw16, (16 + eb * lpf * ept + 15) / 16);
  const int target = std::max(4, lpf) % 32;
  while ((4 * v) % 32 != target) ++v;
  return 16 * v;
}

// window vectors a lane copies per fibre, at most (the window of an n_0 <= lpf * ept fibre)
__host__ __device__ constexpr int win_copies(int lpf, int ept, int eb) {
  return ((lpf * ept * eb + 15) / 16 + 1 + lpf - 1) / lpf;
}

// the fibre's byte offset modulo 16 from the column's and the plan word's: (colb + r fb) mod 16
__device__ __forceinline__ int win_m(int cb16, uint32_t word, int fb16) {
  return (cb16 + (int)(((word & 15u) * (uint32_t)fb16) & 15u)) & 15;
}

// acc[t] += s * entry t of the lane (entry stride lpf * element bytes from p; s = +-1)
template <int DT, int LPF, int EPT>
__device__ __forceinline__ void win_fma(const unsigned char* p, float s, float* acc) {
  constexpr int EB = TtElem<DT>::bytes;
  if constexpr (DT == TT_BF16) {
    const unsigned short sb = tt_bf16_sign(s);
#pragma unroll
    for (int t = 0; t < EPT; ++t)
      acc[t] = tt_fma_bf16(*reinterpret_cast<const unsigned short*>(p + EB * LPF * t), sb, acc[t]);
  } else if constexpr (DT == TT_FP8E4M3) {
    const unsigned short sh = tt_f16_sign(s);
#pragma unroll
    for (int t = 0; t < EPT; ++t) acc[t] = tt_fma_e4m3(*(p + EB * LPF * t), sh, acc[t]);
  } else if constexpr (DT == TT_F32 && EPT % 2 == 0) {
#pragma unroll
    for (int t = 0; t < EPT; t += 2) {
      const float2 d = tt_ffma2(make_float2(s, s),
                                make_float2(TtElem<DT>::sget(p + EB * LPF * t), TtElem<DT>::sget(p + EB * LPF * (t + 1))),
                                make_float2(acc[t], acc[t + 1]));
      acc[t] = d.x;
      acc[t + 1] = d.y;
    }
  } else {
#pragma unroll
    for (int t = 0; t < EPT; ++t) acc[t] = fmaf(s, TtElem<DT>::sget(p + EB * LPF * t), acc[t]);
  }
}

// copy the window of the fibre at byte offset fo of A into a region (this lane's share: window
// vectors posl + lpf c)
template <int LPF, int MWC>
__device__ __forceinline__ void win_issue(const GArgs& a, unsigned char* region, int posl, int64_t fo) {
  const int m = (int)(fo & 15);
  const int64_t ws = fo - m + 16 * posl;                             // this lane's first window vector
  const int nwv = (int)((m + a.fg.fiber_bytes + 15) >> 4);           // window vectors of the fibre
  const int lim = (int)min(a.total_bytes - ws, (int64_t)(1 << 30));  // bytes of A from there on
  unsigned char* dst = region + 16 * posl;
  const char* src = a.A + ws;
#pragma unroll
  for (int c = 0; c < MWC; ++c)
    if (posl + LPF * c < nwv) cp_async_16z(dst + 16 * LPF * c, src + 16 * LPF * c, min(16, lim - 16 * LPF * c));
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Modes k >= 1, G = 4 output columns per work item (the walk of k_unfold_cols): a warp walks its
// slice of the item's c-segment; per plan entry r, lanes 8 g .. 8 g + 7 stage and sum fibre
// A(:, r, col0 + g). Runs of equal c end at the same entry for every lane; their sums go, times
// coef(i_0), into bucket (c + h_0(i_0)) mod J of the CTA's copy of the column (shared-memory
// atomics), and the G copies are added to Y_k at the end of the item.
template <int DT, int S, int EPT>
__global__ void __launch_bounds__(256, 2) k_unfold_cols_win(GArgs a) {
  constexpr int G = 4, LPF = 8;
  constexpr int MWC = win_copies(LPF, EPT, TtElem<DT>::bytes);
  constexpr int EB = TtElem<DT>::bytes;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int J = a.J, T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  const int g = lane / LPF, posl = lane - g * LPF;
  float* Ys = reinterpret_cast<float*>(smraw + (size_t)nw * S * a.wstage);  // G x (J + TT_YPAD)
  int* sstart = reinterpret_cast<int*>(Ys + (size_t)G * (J + TT_YPAD));  // segmax + 1 (relative)
  int* scval = sstart + a.segmax + 1;                                        // segmax
  const int U_ = *a.ucount;
  const int n0 = a.n0;
  const int64_t fb = a.fg.fiber_bytes;
  const int fb16 = (int)(fb & 15);
  unsigned char* reg = smraw + (size_t)warp * S * a.wstage + (size_t)g * a.wstride;  // stage 0
  float coefr[EPT];
  int h0r[EPT];
#pragma unroll
  for (int t = 0; t < EPT; ++t) {
    const int i0 = posl + LPF * t;
    float cf = 0.f;
    int hh = 0;
    if (i0 < n0) {
      cf = __ldg(a.v0 + i0) < 0 ? -1.f : 1.f;
      if (a.scales) cf *= __ldg(a.scales + i0);
      hh = __ldg(a.h0 + i0);
    }
    coefr[t] = cf;
    h0r[t] = hh;
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
    for (int i = threadIdx.x; i < G * (J + TT_YPAD); i += T) Ys[i] = 0.f;
    __syncthreads();
    const int ne = sstart[nu];
    const int sb = (int)((int64_t)ne * warp / nw), se = (int)((int64_t)ne * (warp + 1) / nw);
    const uint32_t* plan = a.plan + e0;
    const bool colok = col0 + g < a.ncol;
    const int64_t colb = colok ? (int64_t)(col0 + g) * a.col_fibres * fb : 0;  // byte offset of the column
    const int cb16 = (int)(colb & 15);
    if (sb < se) {
      int lo2 = 0, hi2 = nu;  // run containing sb: sstart[lo2] <= sb < sstart[hi2]
      while (hi2 - lo2 > 1) {
        const int mid = (lo2 + hi2) >> 1;
        if (sstart[mid] <= sb) lo2 = mid; else hi2 = mid;
      }
      const int count = se - sb;
      int cu = lo2;
      int next_b = sstart[cu + 1];
      float acc[EPT];
#pragma unroll
      for (int t = 0; t < EPT; ++t) acc[t] = 0.f;
      auto flush = [&]() {
        const int cv = scval[cu];
        if (colok) {
          float* yc = Ys + (size_t)g * (J + TT_YPAD);
#pragma unroll
          for (int t = 0; t < EPT; ++t)
            if (posl + LPF * t < n0) atomicAdd(yc + tt_modj(cv + h0r[t], J), coefr[t] * acc[t]);
        }
#pragma unroll
        for (int t = 0; t < EPT; ++t) acc[t] = 0.f;
      };
      // pipeline: stage q of the ring holds entry j with j % S == q
      uint32_t wcur[S], wnext[S];
#pragma unroll
      for (int q = 0; q < S; ++q) {
        wcur[q] = (q < count) ? __ldg(plan + sb + q) : 0u;
        if (q < count && colok)
          win_issue<LPF, MWC>(a, reg + (size_t)q * a.wstage, posl, colb + (int64_t)(wcur[q] & 0x7FFFFFFFu) * fb);
        cp_async_commit();
        wnext[q] = (S + q < count) ? __ldg(plan + sb + S + q) : 0u;
      }
      for (int j0 = 0; j0 < count; j0 += S) {
#pragma unroll
        for (int q = 0; q < S; ++q) {
          const int j = j0 + q;
          if (j < count) {  // the same for every lane of the warp
            const int jr = sb + j;
            if (jr >= next_b) {
              flush();
              do {
                ++cu;
                next_b = sstart[cu + 1];
              } while (jr >= next_b);
            }
            cp_async_wait<S - 1>();
            __syncwarp();  // every lane's copies of stage q have landed
            const float sg = (wcur[q] >> 31) ? -1.f : 1.f;
            win_fma<DT, LPF, EPT>(reg + (size_t)q * a.wstage + win_m(cb16, wcur[q], fb16) + EB * posl, sg, acc);
            __syncwarp();  // every lane has read stage q before it is refilled
            const int jn = j + S;
            if (jn < count && colok)
              win_issue<LPF, MWC>(a, reg + (size_t)q * a.wstage, posl, colb + (int64_t)(wnext[q] & 0x7FFFFFFFu) * fb);
            cp_async_commit();
            wcur[q] = wnext[q];
            wnext[q] = (jn + S < count) ? __ldg(plan + sb + jn + S) : 0u;
          }
        }
      }
      cp_async_wait<0>();
      flush();
    }
    __syncthreads();
    // add the G column copies to Y_k
    for (int gg = 0; gg < G && col0 + gg < a.ncol; ++gg) {
      float* yc = a.Y + (int64_t)J * (col0 + gg);
      const float* ys = Ys + (size_t)gg * (J + TT_YPAD);
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
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// One output column per work item (mode 0: Y_0's rows; modes >= 1 when the four-column kernel
// does not apply), the walk of k_unfold_gather: the item's fibres are split evenly over the
// (warp, fibre slot) pairs, a slot of LPF lanes stages and sums one fibre at a time (S in flight)
// and flushes each run of equal c:
//   mode 0  : the run's sum is row c of Y_0 (a plain store when the run lies inside this slot's
//             range, an atomic add when a neighbour slot shares it);
//   mode >= 1: coef(i_0) * sum is added into bucket (c + h_0(i_0)) mod J of the CTA's column copy.
template <int DT, int S, int LPF, int EPT, bool MODE0>
__global__ void __launch_bounds__(256, 2) k_unfold_gather_win(GArgs a) {
  constexpr int FPI = 32 / LPF;
  constexpr int MWC = win_copies(LPF, EPT, TtElem<DT>::bytes);
  constexpr int EB = TtElem<DT>::bytes;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int J = a.J, T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  const int slot = lane / LPF, posl = lane - slot * LPF;
  const unsigned smask = LPF >= 32 ? 0xFFFFFFFFu : (((1u << LPF) - 1u) << (slot * LPF));
  float* Ys = reinterpret_cast<float*>(smraw + (size_t)nw * S * a.wstage);  // J (mode >= 1)
  int* sstart = reinterpret_cast<int*>(Ys + (MODE0 ? 0 : J));               // segmax + 1 (relative)
  int* scval = sstart + a.segmax + 1;                                        // segmax
  const int U_ = *a.ucount;
  const int n0 = a.n0;
  const int64_t fb = a.fg.fiber_bytes;
  const int fb16 = (int)(fb & 15);
  const int nslots = nw * FPI, gslot = warp * FPI + slot;
  unsigned char* reg = smraw + (size_t)warp * S * a.wstage + (size_t)slot * a.wstride;  // stage 0
  float coefr[EPT];
  int h0r[EPT];
#pragma unroll
  for (int t = 0; t < EPT; ++t) {
    const int i0 = posl + LPF * t;
    float cf = 1.f;
    int hh = 0;
    if (i0 < n0) {
      if (!MODE0 && __ldg(a.v0 + i0) < 0) cf = -1.f;
      if (a.scales) cf *= __ldg(a.scales + i0);
      if (!MODE0) hh = __ldg(a.h0 + i0);
    }
    coefr[t] = cf;
    h0r[t] = hh;
  }
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
      for (int i = threadIdx.x; i < J; i += T) Ys[i] = 0.f;
    __syncthreads();
    const int ne = sstart[nu];
    const int sb = (int)((int64_t)ne * gslot / nslots), se = (int)((int64_t)ne * (gslot + 1) / nslots);
    const int64_t colb = (int64_t)col * a.col_fibres * fb;  // byte offset of the column
    const int cb16 = (int)(colb & 15);
    const uint32_t* plan = a.plan + e0;
    if (sb < se) {  // the same for the LPF lanes of the slot
      int lo2 = 0, hi2 = nu;  // run containing sb: sstart[lo2] <= sb < sstart[hi2]
      while (hi2 - lo2 > 1) {
        const int mid = (lo2 + hi2) >> 1;
        if (sstart[mid] <= sb) lo2 = mid; else hi2 = mid;
      }
      const int count = se - sb;
      int cu = lo2;
      int next_b = sstart[cu + 1];
      bool first_run = true;
      float acc[EPT];
#pragma unroll
      for (int t = 0; t < EPT; ++t) acc[t] = 0.f;
      // flush of the run of group cu (shared with a neighbour slot when `shared`)
      auto flush = [&](bool shared) {
        const int cv = scval[cu];
#pragma unroll
        for (int t = 0; t < EPT; ++t) {
          const int i0 = posl + LPF * t;
          if (i0 < n0) {
            const float v = coefr[t] * acc[t];
            if (MODE0) {
              float* dst = a.Y + cv + (int64_t)J * i0;
              if (shared) atomicAdd(dst, v); else *dst = v;
            } else {
              atomicAdd(Ys + tt_modj(cv + h0r[t], J), v);
            }
          }
          acc[t] = 0.f;
        }
      };
      // pipeline: stage q of the ring holds fibre j with j % S == q
      uint32_t wcur[S], wnext[S];
#pragma unroll
      for (int q = 0; q < S; ++q) {
        wcur[q] = (q < count) ? __ldg(plan + sb + q) : 0u;
        if (q < count) win_issue<LPF, MWC>(a, reg + (size_t)q * a.wstage, posl, colb + (int64_t)(wcur[q] & 0x7FFFFFFFu) * fb);
        cp_async_commit();
        wnext[q] = (S + q < count) ? __ldg(plan + sb + S + q) : 0u;
      }
      for (int j0 = 0; j0 < count; j0 += S) {
#pragma unroll
        for (int q = 0; q < S; ++q) {
          const int j = j0 + q;
          if (j < count) {  // the same for the LPF lanes of the slot
            const int jr = sb + j;  // position within the item
            if (jr >= next_b) {
              flush(first_run || (sstart[cu] < sb));
              first_run = false;
              do {
                ++cu;
                next_b = sstart[cu + 1];
              } while (jr >= next_b);
            }
            cp_async_wait<S - 1>();
            __syncwarp(smask);  // the slot's copies of stage q have landed
            const float sg = (wcur[q] >> 31) ? -1.f : 1.f;
            win_fma<DT, LPF, EPT>(reg + (size_t)q * a.wstage + win_m(cb16, wcur[q], fb16) + EB * posl, sg, acc);
            __syncwarp(smask);  // the slot's lanes have read stage q before it is refilled
            const int jn = j + S;
            if (jn < count)
              win_issue<LPF, MWC>(a, reg + (size_t)q * a.wstage, posl, colb + (int64_t)(wnext[q] & 0x7FFFFFFFu) * fb);
            cp_async_commit();
            wcur[q] = wnext[q];
            wnext[q] = (jn + S < count) ? __ldg(plan + sb + jn + S) : 0u;
          }
        }
      }
      cp_async_wait<0>();
      // last run: shared with the next slot unless it ends exactly at se
      flush(first_run || sstart[cu] < sb || sstart[cu + 1] > se);
    }
    __syncthreads();
    if (!MODE0) {  // add the column copy to Y_k
      float* yc = a.Y + (int64_t)J * col;
      if (a.y_vec4) {
        for (int b = threadIdx.x * 4; b < J; b += T * 4) {
          const float4 v4 = make_float4(Ys[b], Ys[b + 1], Ys[b + 2], Ys[b + 3]);
          if (v4.x != 0.f || v4.y != 0.f || v4.z != 0.f || v4.w != 0.f) atomicAdd(reinterpret_cast<float4*>(yc + b), v4);
        }
      } else {
        for (int b = threadIdx.x; b < J; b += T)
          if (Ys[b] != 0.f) atomicAdd(yc + b, Ys[b]);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------------------------
// host side

namespace {

constexpr int WIN_THREADS = 256;

GArgs win_args(tt_ctx* c, const void* A, const float* scales, int k, float* Y, int eb, bool mode0) {
  GArgs a{};
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
  a.y_vec4 = (c->J & 3) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
  a.n0 = (int)c->n[0];
  a.ncol = mode0 ? 1 : (int)c->n[k];
  a.col_fibres = mode0 ? 0 : c->stride[k] / c->n[0];
  a.total_bytes = c->N * eb;
  a.fg.fiber_bytes = (int64_t)c->n[0] * eb;
  return a;
}

// about `slots` work items in all, four times as many beside the chain of a sweep (short CTAs
// hand SM slots to the chain kernels sooner), capped by tt_unfold_nseg
int win_nseg(tt_ctx* c, int k, int units, int slots) {
  int nseg = std::max(1, slots / units);
  if (c->tune_seg_mult[k]) nseg *= c->tune_seg_mult[k];
  else if (c->in_sweep) nseg *= 4;
  return tt_unfold_nseg(c, units, nseg);
}

template <int DT, int S, int EPT>
int cols_win_launch(tt_ctx* c, const GArgs& a, size_t smem, int blocks) {
  auto kern = k_unfold_cols_win<DT, S, EPT>;
  TT_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<blocks, WIN_THREADS, smem, c->stream>>>(a);
  TT_LAUNCH(c, "k_unfold_cols_win");
  return TT_OK;
}

// Modes >= 1, four columns per item: n_0 <= 128 (at most 16 entries per lane); four fibres in
// flight per warp when two CTAs still fit on an SM, else two.
template <int DT>
int cols_win(tt_ctx* c, const void* A, const float* scales, int k, float* Y, bool* done) {
  constexpr int G = 4, LPF = 8, EB = TtElem<DT>::bytes;
  const int n0 = (int)c->n[0];
  if (n0 > LPF * 16) return TT_OK;
  const int ept = ((n0 + LPF - 1) / LPF + 3) / 4 * 4;  // 4, 8, 12 or 16
  GArgs a = win_args(c, A, scales, k, Y, EB, false);
  a.wstride = win_stride(a.fg.fiber_bytes, EB, LPF, ept);
  a.wstage = G * a.wstride;
  const int ncolg = (a.ncol + G - 1) / G;
  a.nseg = win_nseg(c, k, ncolg, 2 * tt_sm_count());
  a.segmax = (c->J + a.nseg - 1) / a.nseg + 1;
  const size_t rest = sizeof(float) * (size_t)G * (c->J + TT_YPAD) + sizeof(int) * (2 * (size_t)a.segmax + 1);
  const size_t smem4 = (size_t)(WIN_THREADS / 32) * 4 * a.wstage + rest;
  const size_t smem2 = (size_t)(WIN_THREADS / 32) * 2 * a.wstage + rest;
  const size_t two_ctas = 113 * 1024;
  const int S = smem4 <= two_ctas ? 4 : (smem2 <= two_ctas ? 2 : 0);
  if (S == 0) return TT_OK;
  *done = true;
  TT_CUDA(c, cudaMemsetAsync(Y, 0, sizeof(float) * c->J * c->n[k], c->stream));
  const size_t smem = S == 4 ? smem4 : smem2;
  const int blocks = std::max(1, ncolg * a.nseg);
  switch (ept * 10 + S) {
    case 44: return cols_win_launch<DT, 4, 4>(c, a, smem, blocks);
    case 42: return cols_win_launch<DT, 2, 4>(c, a, smem, blocks);
    case 84: return cols_win_launch<DT, 4, 8>(c, a, smem, blocks);
    case 82: return cols_win_launch<DT, 2, 8>(c, a, smem, blocks);
    case 124: return cols_win_launch<DT, 4, 12>(c, a, smem, blocks);
    case 122: return cols_win_launch<DT, 2, 12>(c, a, smem, blocks);
    case 164: return cols_win_launch<DT, 4, 16>(c, a, smem, blocks);
    default: return cols_win_launch<DT, 2, 16>(c, a, smem, blocks);
  }
}

// One column per item, slots of LPF lanes (the smallest power of two with n_0 <= 16 LPF), four
// fibres in flight per slot.
template <int DT, int LPF, bool MODE0>
int gather_win_launch(tt_ctx* c, const void* A, const float* scales, int k, float* Y, bool* done) {
  constexpr int S = 4, EPT = 16, EB = TtElem<DT>::bytes;
  GArgs a = win_args(c, A, scales, k, Y, EB, MODE0);
  a.wstride = win_stride(a.fg.fiber_bytes, EB, LPF, EPT);
  a.wstage = (32 / LPF) * a.wstride;
  const int sms = tt_sm_count();
  const int cps = c->tune_cta_per_sm[k] ? c->tune_cta_per_sm[k] : 2;
  a.nseg = win_nseg(c, k, a.ncol, cps * sms);
  a.segmax = (c->J + a.nseg - 1) / a.nseg + 1;
  const size_t smem = (size_t)(WIN_THREADS / 32) * S * a.wstage + sizeof(float) * (MODE0 ? 0 : c->J) +
                      sizeof(int) * (2 * (size_t)a.segmax + 1);
  if (smem > 220 * 1024) return TT_OK;
  *done = true;
  TT_CUDA(c, cudaMemsetAsync(Y, 0, sizeof(float) * c->J * c->n[k], c->stream));  // empty groups stay 0
  auto kern = k_unfold_gather_win<DT, S, LPF, EPT, MODE0>;
  TT_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1;
  TT_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WIN_THREADS, smem));
  const int items = a.ncol * a.nseg;
  // one CTA per item inside a sweep (freed slots go to the high-priority chain first); otherwise
  // at most one wave
  const int blocks = (c->in_sweep && !c->tune_seg_mult[k])
                         ? std::max(1, items)
                         : std::max(1, std::min(items, sms * std::max(1, std::min(per_sm, cps))));
  kern<<<blocks, WIN_THREADS, smem, c->stream>>>(a);
  TT_LAUNCH(c, "k_unfold_gather_win");
  return TT_OK;
}

template <int DT, bool MODE0>
int gather_win(tt_ctx* c, const void* A, const float* scales, int k, float* Y, bool* done) {
  const int64_t n0 = c->n[0];
  if (n0 <= 16) return gather_win_launch<DT, 1, MODE0>(c, A, scales, k, Y, done);
  if (n0 <= 32) return gather_win_launch<DT, 2, MODE0>(c, A, scales, k, Y, done);
  if (n0 <= 64) return gather_win_launch<DT, 4, MODE0>(c, A, scales, k, Y, done);
  if (n0 <= 128) return gather_win_launch<DT, 8, MODE0>(c, A, scales, k, Y, done);
  if (n0 <= 256) return gather_win_launch<DT, 16, MODE0>(c, A, scales, k, Y, done);
  if (n0 <= 512) return gather_win_launch<DT, 32, MODE0>(c, A, scales, k, Y, done);
  return TT_OK;  // longer fibres: the vector path of tt_unfold.cu
}

template <int DT>
int win_dt(tt_ctx* c, const void* A, const float* scales, int k, float* Y, bool* done) {
  if (k == 0) return gather_win<DT, true>(c, A, scales, k, Y, done);
  if (!c->tune_seg_mult[k]) {  // the autotuner times the one-column kernel's granularities
    const int rc = cols_win<DT>(c, A, scales, k, Y, done);
    if (rc != TT_OK || *done) return rc;
  }
  return gather_win<DT, false>(c, A, scales, k, Y, done);
}

}  // namespace

int tt_launch_unfold_win(tt_ctx* c, const void* A, const float* scales, int k, float* Y, bool* done) {
  *done = false;
  if ((reinterpret_cast<uintptr_t>(A) & 15) != 0) return TT_OK;
  switch (c->dtype) {
    case TT_F64: return TT_OK;  // FP64 fibres lie on an 8-byte grid: the 8-byte vector kernels
    case TT_F32: return win_dt<TT_F32>(c, A, scales, k, Y, done);
    case TT_BF16: return win_dt<TT_BF16>(c, A, scales, k, Y, done);
    default: return win_dt<TT_FP8E4M3>(c, A, scales, k, Y, done);
  }
}
