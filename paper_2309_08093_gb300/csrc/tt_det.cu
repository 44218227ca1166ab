// Deterministic summation order (TT_FLAG_DETERMINISTIC): repeated runs of the same call on the
// same inputs give the same bits.
//
// The fast data-sketch kernels sum fibres in the order of a plan built with atomic cursors and
// add finished runs with shared- and global-memory float atomics, so their FP32 sums depend on
// timing. In this mode the data sketch Y_k = S A_(k)^T (Alg. 1, Eqs. (eqn_h), (eqn_v)) is instead
// accumulated in 64-bit fixed point:
//   - k_det_absmax: m = max_i |A(i)| (FP8: times the slice scale), by integer atomicMax on the
//     bits of non-negative floats (order-independent);
//   - k_det_exp: the binary exponent S such that every term |A(i)| 2^S < 2^(62 - L) with
//     2^(L-1) >= N, so no sum of at most N terms leaves the int64 range (a NaN or Inf in A makes
//     every sketch NaN, which the update then reports as TT_ENONFINITE);
//   - per mode, the vector gather of the fast path (tt_gather.cuh, DET = true) on a deterministic
//     plan (tt_context.cu: each group's fibres in index order). Its work items and the spans into
//     which an item's fibres are cut are fixed by the shape alone, so every run of equal hash is
//     cut at the same places and each piece summed in FP32 in the same order on every call, on any
//     device and with any vector width. Each piece's sum becomes the integer round(sum 2^S)
//     (products with powers of two, then the hardware conversion to int64, ties to even) and is
//     added to the int64 sketch by 64-bit integer atomics, which are associative: the result does
//     not depend on the order in which the adds land;
//   - k_fixed_to_float: Y_k = float(sum 2^-S).
// A piece's sum has the FP32 rounding of the fast path's run sums; its conversion adds at most
// 2^-(S+1), far below that for the data of this library. The integer total stays below 2^61 in
// magnitude: at most N terms of at most 2^(62-L), and the FP32 rounding of a piece is far below
// the remaining factor of two.
//
// The other order-dependent sums of a sweep take fixed orders in this mode: the split-K Gram
// (k_gram_reduce sums the K-chunk partials in chunk order), the relative error and the change
// sums (per-CTA partials added in CTA order by k_sum_partials), and the CountSketch of the cores
// (tt_interface.cu: one thread adds the entries in index order).
#include <algorithm>

#include "tt_gather.cuh"

template <int DT>
__device__ __forceinline__ float det_load(const void* A, int64_t i) {
  if constexpr (DT == TT_F64) return (float)__ldg((const double*)A + i);
  else if constexpr (DT == TT_F32) return __ldg((const float*)A + i);
  else if constexpr (DT == TT_BF16) return __uint_as_float(((uint32_t)__ldg((const unsigned short*)A + i)) << 16);
  else return tt_e4m3_to_float(__ldg((const unsigned char*)A + i));
}

// |A(i)| with the FP8 slice scale applied (the value the sketch adds)
template <int DT>
__device__ __forceinline__ float det_value(const void* A, const float* scales, int64_t i, int n0) {
  float x = det_load<DT>(A, i);
  if (scales) x *= __ldg(scales + (i % n0));
  return x;
}

template <int DT>
__global__ void __launch_bounds__(256) k_det_absmax(const void* A, const float* scales, int64_t N, int n0,
                                                    unsigned* out) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = fabsf(det_value<DT>(A, scales, i, n0));
    m = (x > m || x != x) ? x : m;  // a NaN propagates (its bits exceed every finite value's)
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float y = __shfl_xor_sync(0xffffffffu, m, o);
    m = (y > m || y != y) ? y : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as integers
}

// S = 62 - L - e, with max |A| < 2^e and 2^(L-1) >= N. A non-finite maximum sets misc[2]: the
// sketches are then written as NaN, so that the update that reads them raises TT_ENONFINITE in
// its own stream order (this kernel runs beside the chain and does not touch the status word).
__global__ void k_det_exp(const unsigned* absmax, int64_t N, int* S, int* nonfinite) {
  const unsigned bits = *absmax;
  const int E = (int)((bits >> 23) & 0xFFu);
  *nonfinite = E == 0xFF;
  if (E == 0xFF) {
    *S = 0;
    return;
  }
  if (bits == 0u) {
    *S = 0;
    return;
  }
  const int e = E ? E - 126 : -125;  // |x| < 2^e (subnormals: below 2^-126)
  int L = 1;
  while (L < 63 && (1ll << (L - 1)) < N) ++L;
  *S = 62 - L - e;
}


__global__ void k_fixed_to_float(const unsigned long long* Yq, int64_t count, const int* S, const int* nonfinite,
                                 float* Y) {
  const int s = *S;
  const bool nf = *nonfinite != 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    Y[i] = nf ? __int_as_float(0x7fc00000) : (float)ldexp((double)(long long)Yq[i], -s);
}

// the vectors per lane (1, 2 or 4) for a fibre of vpf vectors of epv entries: mode 0 the most
// fibre slots per warp, modes >= 1 one slot per warp (runs there are short)
static int det_m(bool mode0, int vpf, int epv, int vb) {
  if (vb < 4) return 1;
  const int m = mode0 ? pick_m(vpf, epv) : (vpf > 64 && vpf <= 128 ? 4 : vpf > 32 && vpf <= 64 ? 2 : 1);
  return m * epv <= 16 ? m : 1;
}

// spans per work item: 8 warps times the fibre slots per warp of the widest vectors that the
// fibre length allows (the launch's own count when A is aligned to them)
template <int DT, bool MODE0>
static int det_spans(const tt_ctx* c) {
  constexpr int EB = TtElem<DT>::bytes;
  const int64_t fb = (int64_t)c->n[0] * EB;
  const int vb = pick_vb(fb, 0, EB);
  const int vpf = (int)(fb / vb);
  return 8 * fibre_geom(fb, vb, det_m(MODE0, vpf, vb / EB, vb)).fpi;
}

// c-segments per output column, fixed by the shape (not by the device, the vector width, the
// batch or whether a sweep runs beside): what the fast path picks for 152 SMs inside a sweep
// (mode 0: 1216 segments; modes >= 1: 1216 / column groups of four), and at least one segment
// per 2048 c groups
static int det_nseg(const tt_ctx* c, bool mode0, int ncol) {
  const int nseg = mode0 ? 1216 : std::max(1, 1216 / ((ncol + 3) / 4));
  return std::max(nseg, (c->J + 2047) / 2048);
}

// Modes >= 1 on the column kernel (G = 2 columns per item, int64 copies, S entries in flight,
// MV vectors per lane): the same c-segments and spans as det_gather_launch, so the same bits;
// *done = false (nothing launched) when the shared memory does not allow two CTAs per SM.
template <int DT, int VB, int S, int MV>
static int det_cols_launch(tt_ctx* c, const void* A, const float* scales, int k, unsigned long long* Yq, bool* done) {
  constexpr int G = 2, THREADS = 256;
  constexpr int EB = TtElem<DT>::bytes;
  const int64_t fiber_bytes = (int64_t)c->n[0] * EB;
  GArgs a{};
  a.A = (const char*)A;
  a.scales = scales;
  a.h0 = c->d_h;
  a.v0 = c->d_v;
  a.plan = c->d_rplan[k];
  a.ulist = c->d_ulist[k];
  a.ustart = c->d_ustart[k];
  a.ucount = c->d_ucount[k];
  a.Yq = Yq;
  a.det_S = c->d_det_misc + 1;
  a.J = c->J;
  a.n0 = (int)c->n[0];
  a.ncol = (int)c->n[k];
  a.col_fibres = c->stride[k] / c->n[0];
  a.total_bytes = c->N * EB;
  a.fg = fibre_geom(fiber_bytes, VB, 1);
  a.nseg = det_nseg(c, false, a.ncol);
  a.segmax = (c->J + a.nseg - 1) / a.nseg + 1;
  a.nch = det_spans<DT, false>(c);
  const size_t smem = gather_ring_bytes(true, THREADS / 32, S * MV, VB) +
                      sizeof(int64_t) * (size_t)G * (c->J + TT_YPAD) + sizeof(int) * (2 * (size_t)a.segmax + 1);
  if (smem > 113 * 1024) return TT_OK;
  auto kern = k_unfold_cols<DT, VB, S, MV, G, true>;
  TT_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int items = (a.ncol + G - 1) / G * a.nseg;
  kern<<<std::max(1, items), THREADS, smem, c->stream>>>(a);
  TT_LAUNCH(c, "k_unfold_cols (deterministic)");
  *done = true;
  return TT_OK;
}

// The column kernel's shape for VB-byte vectors: MV = the vectors per lane that cover an entry
// of G = 2 fibres (16-byte vectors: 1 to 4; narrower ones: min(8, 16 / EPV), every lane holding
// up to 8 or 16 entries), four entries in flight for MV <= 2 and two otherwise (registers)
template <int DT, int VB>
static int det_cols(tt_ctx* c, const void* A, const float* scales, int k, unsigned long long* Yq, bool* done) {
  *done = false;
  if constexpr (VB >= 4 && VB >= TtElem<DT>::bytes) {
    constexpr int EPV = TtVec<DT, VB>::EPV;
    constexpr int MV_MAX = VB == 16 ? 4 : (16 / EPV < 8 ? 16 / EPV : 8);
    const int vpf = (int)((int64_t)c->n[0] * TtElem<DT>::bytes / VB);
    const int mv = (2 * vpf + 31) / 32;
    if (mv > MV_MAX || mv * EPV > 16) return TT_OK;  // at most 16 elements per lane
    if constexpr (VB == 16) {
      if (mv == 1) return det_cols_launch<DT, VB, 4, 1>(c, A, scales, k, Yq, done);
      if constexpr (2 * EPV <= 16)
        if (mv == 2) return det_cols_launch<DT, VB, 4, 2>(c, A, scales, k, Yq, done);
      if constexpr (3 * EPV <= 16)
        if (mv == 3) return det_cols_launch<DT, VB, 2, 3>(c, A, scales, k, Yq, done);
      if constexpr (4 * EPV <= 16)
        if (mv == 4) return det_cols_launch<DT, VB, 2, 4>(c, A, scales, k, Yq, done);
      return TT_OK;
    } else {
      return det_cols_launch<DT, VB, 2, MV_MAX>(c, A, scales, k, Yq, done);
    }
  }
  return TT_OK;
}

// The deterministic gather of mode k into the int64 sketch Yq: the fast path's vector gather
// (tt_gather.cuh) with VB-byte vectors, M per lane and S fibres in flight per slot.
template <int DT, int VB, int M, bool MODE0>
static int det_gather_launch(tt_ctx* c, const void* A, const float* scales, int k, unsigned long long* Yq) {
  constexpr int THREADS = 256, S = 12 / M;
  GArgs a{};
  a.A = (const char*)A;
  a.scales = scales;
  a.h0 = c->d_h;
  a.v0 = c->d_v;
  a.plan = c->d_rplan[k];
  a.ulist = c->d_ulist[k];
  a.ustart = c->d_ustart[k];
  a.ucount = c->d_ucount[k];
  a.Yq = Yq;
  a.det_S = c->d_det_misc + 1;
  a.J = c->J;
  a.n0 = (int)c->n[0];
  a.ncol = MODE0 ? 1 : (int)c->n[k];
  a.col_fibres = MODE0 ? 0 : c->stride[k] / c->n[0];
  a.total_bytes = c->N * TtElem<DT>::bytes;
  a.fg = fibre_geom((int64_t)c->n[0] * TtElem<DT>::bytes, VB, M);
  a.nseg = det_nseg(c, MODE0, a.ncol);
  a.segmax = (c->J + a.nseg - 1) / a.nseg + 1;
  a.nch = det_spans<DT, MODE0>(c);
  const size_t smem = gather_ring_bytes(VB >= 4, THREADS / 32, S * M, VB) + sizeof(int64_t) * (MODE0 ? 0 : c->J) +
                      sizeof(int) * (2 * (size_t)a.segmax + 1);
  if (smem > 220 * 1024) return tt_fail(c, TT_EINVAL, "gather kernel needs %zu bytes of shared memory", smem);
  auto kern = k_unfold_gather<DT, VB, S, M, MODE0, true>;
  TT_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int items = a.ncol * a.nseg;
  kern<<<std::max(1, items), THREADS, smem, c->stream>>>(a);
  TT_LAUNCH(c, "k_unfold_gather (deterministic)");
  return TT_OK;
}

template <int DT, int VB, bool MODE0>
static int det_gather_vb(tt_ctx* c, const void* A, const float* scales, int k, unsigned long long* Yq) {
  if constexpr (!MODE0) {
    bool done = false;
    TT_TRY((det_cols<DT, VB>(c, A, scales, k, Yq, &done)));
    if (done) return TT_OK;
  }
  if constexpr (VB >= 4 && VB >= TtElem<DT>::bytes) {
    constexpr int EPV = TtVec<DT, VB>::EPV;
    const int vpf = (int)(c->n[0] * TtElem<DT>::bytes / VB);
    const int m = det_m(MODE0, vpf, EPV, VB);
    if constexpr (4 * EPV <= 16)
      if (m == 4) return det_gather_launch<DT, VB, 4, MODE0>(c, A, scales, k, Yq);
    if constexpr (2 * EPV <= 16)
      if (m == 2) return det_gather_launch<DT, VB, 2, MODE0>(c, A, scales, k, Yq);
  }
  return det_gather_launch<DT, VB, 1, MODE0>(c, A, scales, k, Yq);
}

template <int DT, bool MODE0>
static int det_gather(tt_ctx* c, const void* A, const float* scales, int k, unsigned long long* Yq) {
  constexpr int EB = TtElem<DT>::bytes;
  switch (pick_vb((int64_t)c->n[0] * EB, (uintptr_t)A, EB)) {
    case 16: return det_gather_vb<DT, 16, MODE0>(c, A, scales, k, Yq);
    case 8: return det_gather_vb<DT, (EB <= 8 ? 8 : 16), MODE0>(c, A, scales, k, Yq);
    case 4: return det_gather_vb<DT, (EB <= 4 ? 4 : 16), MODE0>(c, A, scales, k, Yq);
    case 2: return det_gather_vb<DT, (EB <= 2 ? 2 : 16), MODE0>(c, A, scales, k, Yq);
    default: return det_gather_vb<DT, (EB <= 1 ? 1 : 16), MODE0>(c, A, scales, k, Yq);
  }
}

template <int DT>
static int det_gather_mode(tt_ctx* c, const void* A, const float* scales, int k, unsigned long long* Yq) {
  return k == 0 ? det_gather<DT, true>(c, A, scales, k, Yq) : det_gather<DT, false>(c, A, scales, k, Yq);
}

// S (and the non-finite flag) from max |A|: k_det_absmax, then k_det_exp, into d_det_misc
static int det_scale(tt_ctx* c, const void* A, const float* scales) {
  const int sms = tt_sm_count();
  TT_CUDA(c, cudaMemsetAsync(c->d_det_misc, 0, 3 * sizeof(int), c->stream));
  const int ablocks = (int)std::min<int64_t>((c->N + 255) / 256, (int64_t)sms * 8);
  switch (c->dtype) {
    case TT_F64: k_det_absmax<TT_F64><<<ablocks, 256, 0, c->stream>>>(A, scales, c->N, (int)c->n[0], (unsigned*)c->d_det_misc); break;
    case TT_F32: k_det_absmax<TT_F32><<<ablocks, 256, 0, c->stream>>>(A, scales, c->N, (int)c->n[0], (unsigned*)c->d_det_misc); break;
    case TT_BF16: k_det_absmax<TT_BF16><<<ablocks, 256, 0, c->stream>>>(A, scales, c->N, (int)c->n[0], (unsigned*)c->d_det_misc); break;
    default: k_det_absmax<TT_FP8E4M3><<<ablocks, 256, 0, c->stream>>>(A, scales, c->N, (int)c->n[0], (unsigned*)c->d_det_misc); break;
  }
  TT_LAUNCH(c, "k_det_absmax");
  k_det_exp<<<1, 1, 0, c->stream>>>((const unsigned*)c->d_det_misc, c->N, c->d_det_misc + 1, c->d_det_misc + 2);
  TT_LAUNCH(c, "k_det_exp");
  return TT_OK;
}

int tt_launch_unfold_det(tt_ctx* c, const void* A, const float* scales, unsigned mask, float* const* Y, cudaEvent_t* ev) {
  const int sms = tt_sm_count();
  if (!c->det_scale_reuse || c->capture_mode) TT_TRY(det_scale(c, A, scales));
  for (int k = 0; k < c->d; ++k) {
    if (!(mask & (1u << k))) continue;
    TT_TRY(tt_ensure_rplan(c, k));  // deterministic plans (all modes on the first call of a draw)
    unsigned long long* Yq = reinterpret_cast<unsigned long long*>(c->d_y64 + c->yoff[k]);
    TT_CUDA(c, cudaMemsetAsync(Yq, 0, sizeof(int64_t) * (size_t)c->J * c->n[k], c->stream));
    switch (c->dtype) {
      case TT_F64: TT_TRY(det_gather_mode<TT_F64>(c, A, scales, k, Yq)); break;
      case TT_F32: TT_TRY(det_gather_mode<TT_F32>(c, A, scales, k, Yq)); break;
      case TT_BF16: TT_TRY(det_gather_mode<TT_BF16>(c, A, scales, k, Yq)); break;
      default: TT_TRY(det_gather_mode<TT_FP8E4M3>(c, A, scales, k, Yq)); break;
    }
    const int64_t cnt = (int64_t)c->J * c->n[k];
    k_fixed_to_float<<<(int)std::min<int64_t>((cnt + 255) / 256, (int64_t)sms * 4), 256, 0, c->stream>>>(
        Yq, cnt, c->d_det_misc + 1, c->d_det_misc + 2, Y[k]);
    TT_LAUNCH(c, "k_fixed_to_float");
    if (ev) TT_CUDA(c, cudaEventRecord(ev[k], c->stream));
  }
  return TT_OK;
}

// acc[0] += sum_b part[2b], acc[1] += sum_b part[2b + 1], b = 0 .. nparts - 1 in order
__global__ void k_sum_partials(const double* part, int nparts, double* acc) {
  double t0 = 0.0, t1 = 0.0;
  for (int b = 0; b < nparts; ++b) {
    t0 += part[2 * b];
    t1 += part[2 * b + 1];
  }
  acc[0] += t0;
  acc[1] += t1;
}

int tt_launch_sum_partials(tt_ctx* c, const double* part, int nparts, double* acc) {
  k_sum_partials<<<1, 1, 0, c->stream>>>(part, nparts, acc);
  TT_LAUNCH(c, "k_sum_partials");
  return TT_OK;
}

// C[e] = sum_z P[z * count + e] for z = 0 .. nz - 1 in order (the split-K Gram partials)
template <typename T>
__global__ void k_gram_reduce(const T* P, int nz, int64_t count, T* C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int z = 0; z < nz; ++z) s += P[(int64_t)z * count + e];
    C[e] = s;
  }
}

int tt_launch_gram_reduce(tt_ctx* c, const void* P, int nz, int64_t count, void* C, bool f64) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, (int64_t)tt_sm_count() * 4));
  if (f64)
    k_gram_reduce<double><<<blocks, 256, 0, c->stream>>>((const double*)P, nz, count, (double*)C);
  else
    k_gram_reduce<float><<<blocks, 256, 0, c->stream>>>((const float*)P, nz, count, (float*)C);
  TT_LAUNCH(c, "k_gram_reduce");
  return TT_OK;
}
