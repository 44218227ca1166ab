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
//   - k_unfold_fixed: one warp per mode-0 fibre, one lane per entry; each entry A(i) becomes the
//     integer round(A(i) 2^S) (an integer conversion of the float bits, ties away from zero) and is
//     added, with its sign prod_{s != k} v_s(i_s), to Y_k[(sum_{s != k} h_s(i_s)) mod J, i_k] for
//     every requested mode k by 64-bit integer atomics, which are associative: the result does not
//     depend on the order in which the adds land. One read of A serves all modes;
//   - k_fixed_to_float: Y_k = float(sum 2^-S).
// With S chosen as above each term carries an absolute error below 2^-(S+1), far below the FP32
// rounding of the fast path for the data of this library.
//
// The other order-dependent sums of a sweep take fixed orders in this mode: the split-K Gram
// (k_gram_reduce sums the K-chunk partials in chunk order), the relative error and the change
// sums (per-CTA partials added in CTA order by k_sum_partials), and the CountSketch of the cores
// (tt_interface.cu: one thread adds the entries in index order).
#include <algorithm>

#include "tt_internal.cuh"

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

// round(x 2^S) as an int64, from the float bits: x = mant 2^e2; ties rounded away from zero
__device__ __forceinline__ long long det_fixed(float x, int S) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t ex = (b >> 23) & 0xFFu;
  const long long mant = (long long)((b & 0x7FFFFFu) | (ex ? 0x800000u : 0u));
  const int shift = (ex ? (int)ex : 1) - 150 + S;
  long long v;
  if (shift >= 0)
    v = mant << shift;  // below 2^62 by the choice of S
  else if (shift > -40)
    v = (mant + (1ll << (-shift - 1))) >> (-shift);
  else
    v = 0;
  return (b >> 31) ? -v : v;
}

struct FixedArgs {
  const void* A;
  const float* scales;  // n_0 FP8 scales or null
  const int32_t* h;     // all modes' tables, mode s at noff[s]
  const int8_t* v;
  int64_t noff[TT_MAX_D + 1];
  int64_t n[TT_MAX_D];
  int64_t M0;           // mode-0 fibres, N / n_0
  unsigned long long* Y[TT_MAX_D];  // J x n_k int64 accumulators per requested mode (null: skip)
  const int* S;
  const int* nonfinite;  // set by k_det_exp: nothing to accumulate
  int d, J;
};

template <int DT>
__global__ void __launch_bounds__(256) k_unfold_fixed(FixedArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (*a.nonfinite) return;
  const int S = *a.S;
  const int n0 = (int)a.n[0];
  for (int64_t f = warp0; f < a.M0; f += nwarps) {
    // the fibre's modes s >= 1: indices, hashes and signs (every lane computes the same values)
    int ik[TT_MAX_D], hk[TT_MAX_D];
    bool nk[TT_MAX_D];
    int Hrest = 0;
    bool nrest = false;
    int64_t rem = f;
#pragma unroll
    for (int s = 1; s < TT_MAX_D; ++s) {
      ik[s] = 0;
      hk[s] = 0;
      nk[s] = false;
      if (s < a.d) {
        const int i = (int)(rem % a.n[s]);
        rem /= a.n[s];
        ik[s] = i;
        hk[s] = __ldg(a.h + a.noff[s] + i);
        nk[s] = __ldg(a.v + a.noff[s] + i) < 0;
        Hrest += hk[s];
        nrest ^= nk[s];
      }
    }
    for (int i0 = lane; i0 < n0; i0 += 32) {
      const long long q = det_fixed(det_value<DT>(a.A, a.scales, f * n0 + i0, n0), S);
      const int h0 = __ldg(a.h + i0);
      const bool n0neg = __ldg(a.v + i0) < 0;
      if (a.Y[0]) {  // mode 0: row (sum_{s>=1} h_s) mod J, column i_0, sign prod_{s>=1} v_s
        const long long t = nrest ? -q : q;
        atomicAdd(a.Y[0] + (Hrest % a.J) + (int64_t)a.J * i0, (unsigned long long)t);
      }
#pragma unroll
      for (int k = 1; k < TT_MAX_D; ++k) {
        if (k < a.d && a.Y[k]) {
          const int b = (Hrest - hk[k] + h0) % a.J;
          const long long t = (nrest != (nk[k] != n0neg)) ? -q : q;
          atomicAdd(a.Y[k] + b + (int64_t)a.J * ik[k], (unsigned long long)t);
        }
      }
    }
  }
}

__global__ void k_fixed_to_float(const unsigned long long* Yq, int64_t count, const int* S, const int* nonfinite,
                                 float* Y) {
  const int s = *S;
  const bool nf = *nonfinite != 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    Y[i] = nf ? __int_as_float(0x7fc00000) : (float)ldexp((double)(long long)Yq[i], -s);
}

int tt_launch_unfold_det(tt_ctx* c, const void* A, const float* scales, unsigned mask, float* const* Y) {
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
  FixedArgs a;
  a.A = A;
  a.scales = scales;
  a.h = c->d_h;
  a.v = c->d_v;
  for (int s = 0; s <= c->d; ++s) a.noff[s] = c->noff[s];
  for (int s = 0; s < TT_MAX_D; ++s) {
    a.n[s] = s < c->d ? c->n[s] : 1;
    a.Y[s] = nullptr;
  }
  for (int k = 0; k < c->d; ++k)
    if (mask & (1u << k)) {
      a.Y[k] = reinterpret_cast<unsigned long long*>(c->d_y64 + c->yoff[k]);
      TT_CUDA(c, cudaMemsetAsync(a.Y[k], 0, sizeof(int64_t) * (size_t)c->J * c->n[k], c->stream));
    }
  a.M0 = c->M0;
  a.S = c->d_det_misc + 1;
  a.nonfinite = c->d_det_misc + 2;
  a.d = c->d;
  a.J = c->J;
  const int fblocks = (int)std::max<int64_t>(1, std::min<int64_t>((c->M0 + 7) / 8, (int64_t)sms * 8));
  switch (c->dtype) {
    case TT_F64: k_unfold_fixed<TT_F64><<<fblocks, 256, 0, c->stream>>>(a); break;
    case TT_F32: k_unfold_fixed<TT_F32><<<fblocks, 256, 0, c->stream>>>(a); break;
    case TT_BF16: k_unfold_fixed<TT_BF16><<<fblocks, 256, 0, c->stream>>>(a); break;
    default: k_unfold_fixed<TT_FP8E4M3><<<fblocks, 256, 0, c->stream>>>(a); break;
  }
  TT_LAUNCH(c, "k_unfold_fixed");
  for (int k = 0; k < c->d; ++k)
    if (mask & (1u << k)) {
      const int64_t cnt = (int64_t)c->J * c->n[k];
      k_fixed_to_float<<<(int)std::min<int64_t>((cnt + 255) / 256, (int64_t)sms * 4), 256, 0, c->stream>>>(
          a.Y[k], cnt, c->d_det_misc + 1, c->d_det_misc + 2, Y[k]);
      TT_LAUNCH(c, "k_fixed_to_float");
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
