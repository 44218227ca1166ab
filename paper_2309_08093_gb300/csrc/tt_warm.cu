// Learned warm start: the network's input and output on a TT-TS context (include/tt_warmstart.h).
//
//   k_ws_summary_sums / k_ws_summary_write : rows 0..p-1 of every data sketch Y_k, normalised
//                   by their root mean square, and ||Y_0||_F (grid-wide FP64 sums, then the writes)
//   k_canon_step  : one step k of the right-to-left SVD pass of the right-canonical gauge
//                   (one CTA): C = G_k^R G_k^R^T in FP64, eigen-decomposition of C by parallel
//                   cyclic Jacobi rotations (Golub and Van Loan, Matrix Computations, Sec. 8.5:
//                   the 2 x 2 symmetric Schur rotation and the round-robin ordering), singular
//                   values sqrt(eigenvalues) in decreasing order, G_k <- signed V^T,
//                   G_{k-1} <- G_{k-1} x_3 (U S)
//   k_ws_pack / k_ws_unpack : cores <-> network target vector
#include <math.h>

#include <algorithm>

#include "../../include/tt_warmstart.h"
#include "tt_internal.cuh"

namespace {

constexpr int CANON_MAX_R = 64;
constexpr int CANON_THREADS = 1024;
constexpr double CANON_TOL = 1e-6;  // singular values <= tol * largest become zero

struct CorePtrs {
  float* p[TT_MAX_D];
  int64_t off[TT_MAX_D + 1];  // offsets of the cores in the packed vector
  int r0[TT_MAX_D], n[TT_MAX_D], r1[TT_MAX_D];
  int d;
};

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

struct SummaryArgs {
  const float* Y[TT_MAX_D];
  int64_t n[TT_MAX_D];
  int64_t xoff[TT_MAX_D + 1];
  int d, J, p;
  int64_t y0_vec4;  // entries of Y_0 read as float4 (0 when Y_0 is not 16-byte aligned)
  float* x;
  float* scale;
};

__device__ __forceinline__ float summary_value(const SummaryArgs& a, int64_t e) {
  int k = 0;
  while (e >= a.xoff[k + 1]) ++k;
  const int64_t loc = e - a.xoff[k];
  return a.Y[k][(loc / a.p) * a.J + loc % a.p];
}

// acc[0] += sum of squares of the summary entries, acc[1] += ||Y_0||_F^2 (grid-wide, FP64)
__global__ void __launch_bounds__(256) k_ws_summary_sums(SummaryArgs a, double* __restrict__ acc) {
  __shared__ double red[32];
  const int64_t total = a.xoff[a.d];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double ss = 0.0, y0 = 0.0;
  for (int64_t e = t0; e < total; e += stride) {
    const double v = summary_value(a, e);
    ss += v * v;
  }
  const float4* Y0 = (const float4*)a.Y[0];
  const int64_t n4 = a.y0_vec4;
  for (int64_t e = t0; e < n4; e += stride) {
    const float4 q = Y0[e];
    y0 += (double)q.x * q.x + (double)q.y * q.y + (double)q.z * q.z + (double)q.w * q.w;
  }
  for (int64_t e = 4 * n4 + t0; e < a.n[0] * a.J; e += stride) {
    const double v = a.Y[0][e];
    y0 += v * v;
  }
  ss = block_sum(ss, red);
  y0 = block_sum(y0, red);
  if (threadIdx.x == 0) {
    if (ss != 0.0) atomicAdd(&acc[0], ss);
    if (y0 != 0.0) atomicAdd(&acc[1], y0);
  }
}

__global__ void __launch_bounds__(256) k_ws_summary_write(SummaryArgs a, const double* __restrict__ acc) {
  const int64_t total = a.xoff[a.d];
  const double inv = acc[0] > 0.0 ? 1.0 / sqrt(acc[0] / (double)total) : 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    a.x[e] = (float)((double)summary_value(a, e) * inv);
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.scale = (float)sqrt(acc[1]);
}

// One step of the right-to-left SVD pass at core k: W = G_k^R (r x m, element (a, c) at
// a + r c, m = n_k r_{k+1}); prev = core k-1 with rows rho = alpha + r_{k-1} i (rows_prev of
// them) and last index b < r at rho + rows_prev * b.
__global__ void __launch_bounds__(CANON_THREADS) k_canon_step(float* __restrict__ W, int r, int n, int m,
                                                              float* __restrict__ prev, int rows_prev,
                                                              int* __restrict__ status) {
  extern __shared__ double sh[];
  const int L = CANON_MAX_R + 1;  // padded row length
  double* C = sh;                 // r x r, row stride L
  double* U = C + CANON_MAX_R * L;
  double* rot = U + CANON_MAX_R * L;      // 2 per pair
  double* omega = rot + CANON_MAX_R;      // r first moments of the rows of W
  double* Q = omega + CANON_MAX_R;        // r x r coefficients of the new rows (row stride L)
  double* Mx = Q + CANON_MAX_R * L;       // r x r absorbed matrix (row stride L)
  double* red = Mx + CANON_MAX_R * L;     // 32
  int* order = (int*)(red + 32);          // position -> eigen index
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // C = W W^T (upper triangle computed, mirrored), first moments omega_a = sum_c (c mod n + 1) W[a, c]
  for (int pr = tid; pr < r * r; pr += blockDim.x) {
    const int a = pr / r, b = pr % r;
    if (b < a) continue;
    double s = 0.0;
    for (int c = 0; c < m; ++c) s += (double)W[a + (int64_t)r * c] * (double)W[b + (int64_t)r * c];
    C[a * L + b] = s;
    C[b * L + a] = s;
  }
  for (int a = warp; a < r; a += blockDim.x >> 5) {
    double s = 0.0;
    for (int c = lane; c < m; c += 32) s += (double)((c % n) + 1) * (double)W[a + (int64_t)r * c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) omega[a] = s;
  }
  for (int e = tid; e < r * r; e += blockDim.x) U[(e / r) * L + (e % r)] = (e / r == e % r) ? 1.0 : 0.0;
  __syncthreads();

  // parallel cyclic Jacobi, round-robin pairs over nn = r rounded up to even
  const int nn = r + (r & 1);
  const int npairs = nn / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int e = tid; e < r * r; e += blockDim.x) {
      const double v = C[(e / r) * L + (e % r)];
      if (e / r == e % r) dia += v * v; else off += v * v;
    }
    off = block_sum(off, red);
    dia = block_sum(dia, red);
    if (!(off == off) || !(dia == dia)) {  // NaN
      if (tid == 0) atomicExch(status, TT_ENONFINITE);
      return;
    }
    if (off <= 1e-30 * dia || dia == 0.0) break;
    for (int t = 0; t < nn - 1; ++t) {
      int p = -1, q = -1;
      if (warp < npairs) {
        // pair w of round t: (t, nn-1) for w = 0, else ((t + w) mod (nn-1), (t - w) mod (nn-1))
        if (warp == 0) {
          p = t;
          q = nn - 1;
        } else {
          p = (t + warp) % (nn - 1);
          q = (t - warp + (nn - 1)) % (nn - 1);
        }
        if (p > q) { const int x = p; p = q; q = x; }
        if (q >= r) p = q = -1;  // pair with the padding index
      }
      if (warp < npairs && lane == 0) {
        double c = 1.0, s = 0.0;
        if (p >= 0) {
          const double apq = C[p * L + q];
          if (fabs(apq) > 1e-300) {
            const double theta = (C[q * L + q] - C[p * L + p]) / (2.0 * apq);
            double tt;
            if (fabs(theta) > 1e100) tt = 0.5 / theta;
            else tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
        }
        rot[2 * warp] = c;
        rot[2 * warp + 1] = s;
      }
      __syncthreads();
      if (warp < npairs && p >= 0) {  // rows p, q of C (J^T C)
        const double c = rot[2 * warp], s = rot[2 * warp + 1];
        for (int j = lane; j < r; j += 32) {
          const double cp = C[p * L + j], cq = C[q * L + j];
          C[p * L + j] = c * cp - s * cq;
          C[q * L + j] = s * cp + c * cq;
        }
      }
      __syncthreads();
      if (warp < npairs && p >= 0) {  // columns p, q of C and U (. J)
        const double c = rot[2 * warp], s = rot[2 * warp + 1];
        for (int j = lane; j < r; j += 32) {
          const double cp = C[j * L + p], cq = C[j * L + q];
          C[j * L + p] = c * cp - s * cq;
          C[j * L + q] = s * cp + c * cq;
          const double up = U[j * L + p], uq = U[j * L + q];
          U[j * L + p] = c * up - s * uq;
          U[j * L + q] = s * up + c * uq;
        }
      }
      __syncthreads();
    }
  }

  // eigenvalues in decreasing order (ties by index)
  for (int a = tid; a < r; a += blockDim.x) {
    const double la = C[a * L + a];
    int pos = 0;
    for (int b = 0; b < r; ++b) {
      const double lb = C[b * L + b];
      if (lb > la || (lb == la && b < a)) ++pos;
    }
    order[pos] = a;
  }
  __syncthreads();
  const double smax = sqrt(fmax(C[order[0] * L + order[0]], 0.0));
  // Q[j][a] = sg_j u_j[a] / s_j and Mx[b][j] = U[b][a_j] s_j sg_j for kept j, zero otherwise
  for (int j = warp; j < r; j += blockDim.x >> 5) {
    const int aj = order[j];
    const double sj = sqrt(fmax(C[aj * L + aj], 0.0));
    const bool keep = smax > 0.0 && sj > CANON_TOL * smax;
    double mom = 0.0;
    for (int a = lane; a < r; a += 32) mom += U[a * L + aj] * omega[a];
    for (int o = 16; o > 0; o >>= 1) mom += __shfl_xor_sync(0xffffffffu, mom, o);
    const double sg = mom < 0.0 ? -1.0 : 1.0;
    for (int a = lane; a < r; a += 32) {
      Q[j * L + a] = keep ? sg * U[a * L + aj] / sj : 0.0;
      Mx[a * L + j] = keep ? U[a * L + aj] * sj * sg : 0.0;
    }
  }
  __syncthreads();
  // G_k <- V^T: column c of W -> column c of the new rows (in place, one thread per column)
  for (int c = tid; c < m; c += blockDim.x) {
    double w[CANON_MAX_R];
    for (int a = 0; a < r; ++a) w[a] = W[a + (int64_t)r * c];
    for (int j = 0; j < r; ++j) {
      double s = 0.0;
      for (int a = 0; a < r; ++a) s += Q[j * L + a] * w[a];
      W[j + (int64_t)r * c] = (float)s;
    }
  }
  // G_{k-1} <- G_{k-1} x_3 Mx (in place, one thread per row)
  for (int rho = tid; rho < rows_prev; rho += blockDim.x) {
    double g[CANON_MAX_R];
    for (int b = 0; b < r; ++b) g[b] = prev[rho + (int64_t)rows_prev * b];
    for (int j = 0; j < r; ++j) {
      double s = 0.0;
      for (int b = 0; b < r; ++b) s += g[b] * Mx[b * L + j];
      prev[rho + (int64_t)rows_prev * j] = (float)s;
    }
  }
}

constexpr size_t canon_smem() {
  return sizeof(double) * (4 * CANON_MAX_R * (CANON_MAX_R + 1) + 2 * CANON_MAX_R + 32) + sizeof(int) * CANON_MAX_R;
}

__global__ void k_ws_pack(CorePtrs cp, const float* __restrict__ scale, float* __restrict__ y, int unpack) {
  const float inv_scale = 1.0f / *scale;
  const float sc = *scale;
  for (int k = 0; k < cp.d; ++k) {
    const int64_t sz = cp.off[k + 1] - cp.off[k];
    const float f = sqrtf((float)cp.n[k] * (float)cp.r1[k]);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sz; e += (int64_t)gridDim.x * blockDim.x) {
      if (!unpack) {
        y[cp.off[k] + e] = cp.p[k][e] * f * (k == 0 ? inv_scale : 1.0f);
      } else {
        cp.p[k][e] = y[cp.off[k] + e] / f * (k == 0 ? sc : 1.0f);
      }
    }
  }
}

CorePtrs core_ptrs(const tt_ctx* c, float* const* cores) {
  CorePtrs cp{};
  cp.d = c->d;
  cp.off[0] = 0;
  for (int k = 0; k < c->d; ++k) {
    cp.p[k] = cores[k];
    cp.r0[k] = c->r[k];
    cp.n[k] = (int)c->n[k];
    cp.r1[k] = c->r[k + 1];
    cp.off[k + 1] = cp.off[k] + (int64_t)c->r[k] * c->n[k] * c->r[k + 1];
  }
  return cp;
}

}  // namespace

extern "C" int64_t tt_ws_summary_dim(const tt_ctx* c, int p) {
  if (!c || p < 1) return -1;
  int64_t s = 0;
  for (int k = 0; k < c->d; ++k) s += c->n[k];
  return s * p;
}

extern "C" int64_t tt_ws_core_dim(const tt_ctx* c) {
  if (!c) return -1;
  int64_t s = 0;
  for (int k = 0; k < c->d; ++k) s += (int64_t)c->r[k] * c->n[k] * c->r[k + 1];
  return s;
}

extern "C" int tt_ws_summary(tt_ctx* c, float* const* Y, int p, float* x, float* scale) {
  if (!c) return TT_EINVAL;
  if (!Y || !x || !scale) return tt_fail(c, TT_EINVAL, "null pointer");
  if (p < 1 || p > c->J) return tt_fail(c, TT_EINVAL, "p = %d outside 1..J", p);
  SummaryArgs a{};
  a.d = c->d;
  a.J = c->J;
  a.p = p;
  a.x = x;
  a.scale = scale;
  a.y0_vec4 = ((uintptr_t)Y[0] & 15) ? 0 : (c->n[0] * c->J) / 4;
  a.xoff[0] = 0;
  for (int k = 0; k < c->d; ++k) {
    if (!Y[k]) return tt_fail(c, TT_EINVAL, "null sketch pointer %d", k);
    a.Y[k] = Y[k];
    a.n[k] = c->n[k];
    a.xoff[k + 1] = a.xoff[k] + (int64_t)p * c->n[k];
  }
  int dev = 0, sms = 0;
  TT_CUDA(c, cudaGetDevice(&dev));
  TT_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  TT_CUDA(c, cudaMemsetAsync(c->d_ws_acc, 0, 2 * sizeof(double), c->stream));
  k_ws_summary_sums<<<sms, 256, 0, c->stream>>>(a, c->d_ws_acc);
  TT_LAUNCH(c, "k_ws_summary_sums");
  k_ws_summary_write<<<(unsigned)std::min<int64_t>(sms, (a.xoff[a.d] + 255) / 256), 256, 0, c->stream>>>(a, c->d_ws_acc);
  TT_LAUNCH(c, "k_ws_summary_write");
  return TT_OK;
}

extern "C" int tt_canonicalize(tt_ctx* c, float* const* cores) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_cores(c, cores));
  for (int k = 1; k < c->d; ++k) {
    if (c->r[k] > CANON_MAX_R) return tt_fail(c, TT_EINVAL, "canonical form needs r[%d] <= %d", k, CANON_MAX_R);
    if ((int64_t)c->r[k] > c->n[k] * c->r[k + 1])
      return tt_fail(c, TT_EINVAL, "canonical form needs r[%d] <= n[%d] r[%d]", k, k, k + 1);
  }
  c->err.clear();
  TT_TRY(tt_reset_status(c));
  for (int k = 0; k < c->d - 1; ++k) TT_TRY(tt_launch_qr_left(c, cores[k], cores[k + 1], k));
  static bool attr = false;
  if (!attr) {
    TT_CUDA(c, cudaFuncSetAttribute(k_canon_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)canon_smem()));
    attr = true;
  }
  for (int k = c->d - 1; k >= 1; --k) {
    const int r = c->r[k], n = (int)c->n[k];
    const int m = n * c->r[k + 1];
    const int rows_prev = c->r[k - 1] * (int)c->n[k - 1];
    k_canon_step<<<1, CANON_THREADS, canon_smem(), c->stream>>>(cores[k], r, n, m, cores[k - 1], rows_prev,
                                                                 c->d_status);
    TT_LAUNCH(c, "k_canon_step");
  }
  return tt_read_status(c);
}

extern "C" int tt_ws_pack(tt_ctx* c, float* const* cores, const float* scale, float* y) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_cores(c, cores));
  if (!scale || !y) return tt_fail(c, TT_EINVAL, "null pointer");
  k_ws_pack<<<256, 256, 0, c->stream>>>(core_ptrs(c, cores), scale, y, 0);
  TT_LAUNCH(c, "k_ws_pack");
  return TT_OK;
}

extern "C" int tt_ws_unpack(tt_ctx* c, const float* y, const float* scale, float* const* cores) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_cores(c, cores));
  if (!scale || !y) return tt_fail(c, TT_EINVAL, "null pointer");
  k_ws_pack<<<256, 256, 0, c->stream>>>(core_ptrs(c, cores), scale, const_cast<float*>(y), 1);
  TT_LAUNCH(c, "k_ws_unpack");
  return TT_OK;
}
