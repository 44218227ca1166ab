// Shared by the data-sketch kernels of Alg. 1 part (a) (tt_unfold.cu: 16-, 8-, 4-, 2- and 1-byte
// vector loads of mode-0 fibres; tt_unfold_win.cu: window staging of fibres that do not start on
// a 16-byte boundary): element types, the kernels' argument block and the cp.async helpers.
#pragma once

#include <algorithm>

#include "tt_internal.cuh"

template <>
struct TtElem<TT_F64> {
  using T = double;
  static constexpr int bytes = 8;
  __device__ static float get(const void* a, int64_t i) { return (float)__ldg((const double*)a + i); }
  __device__ static float sget(const unsigned char* p) { return (float)*reinterpret_cast<const double*>(p); }
};
template <>
struct TtElem<TT_F32> {
  using T = float;
  static constexpr int bytes = 4;
  __device__ static float get(const void* a, int64_t i) { return __ldg((const float*)a + i); }
  __device__ static float sget(const unsigned char* p) { return *reinterpret_cast<const float*>(p); }
};
template <>
struct TtElem<TT_BF16> {
  using T = unsigned short;
  static constexpr int bytes = 2;
  __device__ static float get(const void* a, int64_t i) {
    return __uint_as_float(((uint32_t)__ldg((const unsigned short*)a + i)) << 16);
  }
  __device__ static float sget(const unsigned char* p) {
    return __uint_as_float(((uint32_t)*reinterpret_cast<const unsigned short*>(p)) << 16);
  }
};

// OCP FP8 E4M3 (bias 7, no infinities, S.1111.111 NaN)
__device__ __forceinline__ float tt_fp8_e4m3(uint32_t c) { return tt_e4m3_to_float(c); }
template <>
struct TtElem<TT_FP8E4M3> {
  using T = unsigned char;
  static constexpr int bytes = 1;
  __device__ static float get(const void* a, int64_t i) { return tt_fp8_e4m3(__ldg((const unsigned char*)a + i)); }
  __device__ static float sget(const unsigned char* p) { return tt_fp8_e4m3(*p); }
};

// Vector geometry of a fibre: VB-byte loads, vpf vectors per fibre, m vectors per lane, lanes per
// fibre slot and fibre slots per warp (several short fibres share one warp instruction). Vector v
// of a fibre is read by lane posl of its slot as (chunk ch, sub-vector mm) with
// v = ch * lpf * m + mm * lpf + posl, so each of a lane's m loads is coalesced across the slot.
struct FibreGeom {
  int64_t fiber_bytes;
  int vpf, lpf, fpi, nchunk, m;
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// acc += s x for a BF16 entry x (raw bits) and a sign s = +-1 (BF16 bits 0x3F80 / 0xBF80): the
// mixed-precision FMA multiplies exactly and rounds the sum once to FP32, so the result is the
// bits of fmaf(s, (float)x, acc) without the conversion of x to FP32
__device__ __forceinline__ float tt_fma_bf16(unsigned short x, unsigned short s, float acc) {
  asm("fma.rn.f32.bf16 %0, %1, %2, %0;\n" : "+f"(acc) : "h"(x), "h"(s));
  return acc;
}
// the same for the two BF16 entries of a 32-bit word (low half: a0, high half: a1)
__device__ __forceinline__ void tt_fma_bf16x2(uint32_t w, unsigned short s, float& a0, float& a1) {
  asm("{\n .reg .b16 lo, hi;\n mov.b32 {lo, hi}, %2;\n fma.rn.f32.bf16 %0, lo, %3, %0;\n"
      " fma.rn.f32.bf16 %1, hi, %3, %1;\n}\n"
      : "+f"(a0), "+f"(a1)
      : "r"(w), "h"(s));
}
// BF16 bits of a sign s = +-1
__device__ __forceinline__ unsigned short tt_bf16_sign(float s) { return s < 0.f ? 0xBF80 : 0x3F80; }

// acc_j += s x_j for the four E4M3 entries of a 32-bit word (byte j = entry j) and a sign s = +-1
// (FP16 bits 0x3C00 / 0xBC00): two hardware conversions of two entries each to FP16 (exact), then
// mixed-precision FMAs (exact product, one rounding to FP32): the bits of fmaf(s, decoded, acc)
__device__ __forceinline__ void tt_fma_e4m3x4(uint32_t w, unsigned short s, float& a0, float& a1, float& a2,
                                              float& a3) {
  asm("{\n .reg .b16 p0, p1, q0, q1, q2, q3;\n .reg .b32 h01, h23;\n mov.b32 {p0, p1}, %4;\n"
      " cvt.rn.f16x2.e4m3x2 h01, p0;\n cvt.rn.f16x2.e4m3x2 h23, p1;\n"
      " mov.b32 {q0, q1}, h01;\n mov.b32 {q2, q3}, h23;\n"
      " fma.rn.f32.f16 %0, q0, %5, %0;\n fma.rn.f32.f16 %1, q1, %5, %1;\n"
      " fma.rn.f32.f16 %2, q2, %5, %2;\n fma.rn.f32.f16 %3, q3, %5, %3;\n}\n"
      : "+f"(a0), "+f"(a1), "+f"(a2), "+f"(a3)
      : "r"(w), "h"(s));
}
// the same for one E4M3 entry (low byte of x)
__device__ __forceinline__ float tt_fma_e4m3(unsigned short x, unsigned short s, float acc) {
  asm("{\n .reg .b32 h;\n .reg .b16 lo, hi;\n cvt.rn.f16x2.e4m3x2 h, %1;\n mov.b32 {lo, hi}, h;\n"
      " fma.rn.f32.f16 %0, lo, %2, %0;\n}\n"
      : "+f"(acc)
      : "h"(x), "h"(s));
  return acc;
}
// FP16 bits of a sign s = +-1
__device__ __forceinline__ unsigned short tt_f16_sign(float s) { return s < 0.f ? 0xBC00 : 0x3C00; }

// round(x 2^S) as an int64, ties to even: x 2^S formed by one or two products with powers of two
// (exact, except a product below 2^-126 in magnitude, which rounds to 0 either way), then one
// hardware conversion (cvt.rni.s64.f32). |x| 2^S < 2^62 by the choice of S.
__device__ __forceinline__ long long det_fixed(float x, int S) {
  const int s1 = S < -126 ? -126 : (S > 126 ? 126 : S);
  float t = x * __int_as_float((s1 + 127) << 23);
  if (S != s1) t *= __int_as_float((S - s1 + 127) << 23);
  return __float2ll_rn(t);
}

// 16-byte copy global -> shared of `bytes` (1..16) valid source bytes, the rest of the 16
// destination bytes zero-filled; both addresses 16-byte aligned
__device__ __forceinline__ void cp_async_16z(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes));
}

struct GArgs {
  const char* A;
  const float* scales;    // n0 FP8 scales or null
  const int32_t* h0;      // h_0 (n0 entries)
  const int8_t* v0;
  const uint32_t* plan;   // fibre index at i_k = 0 | sign in bit 31, grouped by c
  const int32_t* ulist;   // distinct c values
  const int64_t* ustart;  // starts into plan (U + 1)
  const int32_t* ucount;  // U
  float* Y;               // J x ncol column-major, zeroed by the host
  int64_t col_fibres;     // fibre-index stride of the output column (stride_k / n0); 0 for mode 0
  int J, n0, ncol;
  int nseg;               // c-segments per column (work items = ncol * nseg)
  int segmax;             // capacity of the staged segment (c groups)
  int y_vec4;             // Y 16-byte aligned and J % 4 == 0: columns flushed with 16-byte atomics
  int64_t total_bytes;    // bytes of A (window staging clips its last copies here)
  unsigned long long* Yq; // deterministic mode: J x ncol int64 fixed-point accumulators (instead of Y)
  const int* det_S;       // deterministic mode: {S, A not finite}; values scaled by 2^S
  int nch;                // deterministic mode: spans per item (split at ne * t / nch), any slot count
  int wstride;            // window staging: bytes of a fibre's region of a stage (a multiple of 16)
  int wstage;             // window staging: bytes of one warp's stage
  FibreGeom fg;
};

// Bytes of the cp.async ring at the start of the gather kernel's shared memory (none when the
// vectors are loaded synchronously). Used by the kernel and by the host-side size computation.
__host__ __device__ constexpr size_t gather_ring_bytes(bool async, int nwarps, int stages, int vb) {
  return async ? (size_t)nwarps * stages * 32 * vb : 0;
}

// The G column copies of a multi-column data-sketch item lie J + TT_YPAD floats apart in shared
// memory, so that the buckets of two columns that one flush instruction touches fall on different
// banks (the flush adds of a run go to random buckets (c + h_0(i_0)) mod J).
#define TT_YPAD 8

// c-segments per column unit (column or column group) of a data-sketch launch: `nseg` as chosen
// for a tensor alone, at most (bytes of A / c->item_bytes) work items in all when the context sets
// item_bytes, and at least one segment per 2048 c groups (the staged segment's capacity).
inline int tt_unfold_nseg(const tt_ctx* c, int units, int nseg) {
  if (c->item_bytes > 0) {
    const int64_t cap = std::max<int64_t>(1, c->N * tt_elem_bytes(c->dtype) / c->item_bytes);
    nseg = (int)std::min<int64_t>(nseg, std::max<int64_t>(1, cap / units));
  }
  return std::max(nseg, (c->J + 2047) / 2048);
}

// Modes k of the data sketch whose fibres lie on a 1-, 2- or 4-byte grid (n_0 * element bytes not
// a multiple of 8; FP32, BF16 or FP8) and A 16-byte aligned: launches the window-staging kernel on
// c->stream and sets *done, or returns TT_OK with *done = false when the shape does not suit it.
int tt_launch_unfold_win(tt_ctx* c, const void* A, const float* scales, int k, float* Y, bool* done);
