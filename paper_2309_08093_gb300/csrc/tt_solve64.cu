// Part (c) in FP64: the proximal update of Eq. (ite),
//   M = (S H_k)^T (S H_k) + sigma I,  B = Y_k^T (S H_k) + sigma G_{k(2)},  G_{k(2)} <- B M^{-1},
// with the Gram accumulated in FP64 and M factored by an FP64 Cholesky (M = L L^T) followed by
// two FP64 triangular solves per right-hand side. This is the form the context takes when
// sigma = 0 -- Alg. 1 asks sigma > 0, Sec. 5 runs sigma = 0, where M is not SPD by construction
// and its conditioning is unbounded -- or when TT_FLAG_FP64_SOLVE is set.
//
//   k_gram64 : [S H_k | Y_k]^T (S H_k): the FP32 inputs are widened to FP64 when staged in shared
//              memory, so every product is exact (24 + 24 significand bits < 53) and the sums
//              carry FP64 rounding only; split-K with FP64 atomics. A non-finite sum raises
//              TT_ENONFINITE before the solve runs.
//   k_chol64 : one CTA factors M + sigma I = L L^T in place (right-looking, 32-column panels
//              staged in shared memory; the trailing lower triangle stays in L2). A pivot
//              L_jj^2 <= TT_PIVOT_TOL64 * max_i (M_ii + sigma) means M is singular to the
//              precision of its inputs: TT_ENOTSPD, core unchanged.
//   k_trsm64 : one CTA per chunk of right-hand sides: L Z = B^T + sigma G_c, then L^T X = Z,
//              with L staged by 32-row or 32-column panels; the update goes to the core.
#include <stdio.h>

#include <algorithm>

#include "tt_internal.cuh"

// Relative pivot bound of the FP64 Cholesky; the oracle refuses at the same ratio.
#define TT_PIVOT_TOL64 1e-10

struct Gram64Args {
  const float* SH;  // J x s column-major
  const float* Y;   // J x n column-major
  double* C;        // accumulators (zeroed by the caller): s x s Gram, then s x n RHS, row-major
  int* status;
  double* P;        // deterministic mode: K-chunk z stores its sums at P + z (s + n) s (no atomics)
  int J, s, n, kchunk;
};

// CTA tile of 64 x 64 entries over one K-chunk, 256 threads with 4 x 4 entries each; K-steps of
// 16 rows staged as [k][column] in FP64 (the widening happens once per staged element, not per
// product); the next step's global loads are in flight during the current step's FMAs.
template <bool VEC>
__global__ void __launch_bounds__(256) k_gram64(Gram64Args a) {
  __shared__ __align__(16) double Xs[16][68];
  __shared__ __align__(16) double Bs[16][68];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int rows = a.s + a.n;
  const int r0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  const int kb = blockIdx.z * a.kchunk, ke = min(a.J, kb + a.kchunk);
  const int lc = t >> 2, lk = (t & 3) * 4;
  const int gr = r0 + lc, gc = c0 + lc;
  const float* xcol = gr < a.s ? a.SH + (int64_t)gr * a.J : (gr < rows ? a.Y + (int64_t)(gr - a.s) * a.J : nullptr);
  const float* bcol = gc < a.s ? a.SH + (int64_t)gc * a.J : nullptr;
  float xr[4], br[4];
  auto load = [&](int k0) {
    if constexpr (VEC) {
      const float4 xv = xcol ? __ldg(reinterpret_cast<const float4*>(xcol + k0 + lk)) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 bv = bcol ? __ldg(reinterpret_cast<const float4*>(bcol + k0 + lk)) : make_float4(0.f, 0.f, 0.f, 0.f);
      xr[0] = xv.x, xr[1] = xv.y, xr[2] = xv.z, xr[3] = xv.w;
      br[0] = bv.x, br[1] = bv.y, br[2] = bv.z, br[3] = bv.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool in = k0 + lk + e < ke;
        xr[e] = (xcol && in) ? __ldg(xcol + k0 + lk + e) : 0.f;
        br[e] = (bcol && in) ? __ldg(bcol + k0 + lk + e) : 0.f;
      }
    }
  };
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  if (kb < ke) load(kb);
  for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      Xs[lk + e][lc] = (double)xr[e];
      Bs[lk + e][lc] = (double)br[e];
    }
    __syncthreads();
    if (k0 + 16 < ke) load(k0 + 16);
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      const double2 x01 = *reinterpret_cast<const double2*>(&Xs[kk][ty * 4]);
      const double2 x23 = *reinterpret_cast<const double2*>(&Xs[kk][ty * 4 + 2]);
      const double2 b01 = *reinterpret_cast<const double2*>(&Bs[kk][tx * 4]);
      const double2 b23 = *reinterpret_cast<const double2*>(&Bs[kk][tx * 4 + 2]);
      const double xa[4] = {x01.x, x01.y, x23.x, x23.y};
      const double ba[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(xa[i], ba[j], acc[i][j]);
    }
    __syncthreads();
  }
  bool finite = true;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = r0 + ty * 4 + i, col = c0 + tx * 4 + j;
      if (col >= a.s || row >= rows) continue;
      finite = finite && isfinite(acc[i][j]);
      // the Gram row-major, then the right-hand side stored transposed (s x n)
      const int64_t idx = row < a.s ? (int64_t)row * a.s + col : (int64_t)a.s * a.s + (int64_t)col * a.n + (row - a.s);
      if (a.P)
        a.P[(int64_t)blockIdx.z * (a.s + a.n) * a.s + idx] = acc[i][j];
      else
        atomicAdd(a.C + idx, acc[i][j]);
    }
  if (!finite) atomicCAS(a.status, 0, TT_ENONFINITE);
}

struct Chol64Args {
  double* M;  // s x s row-major (the Gram); its lower triangle is overwritten with L
  int* status;
  double sigma;
  int s;
};

constexpr int C64_NB = 32, C64_P = 33, C64_T = 512;

__global__ void __launch_bounds__(C64_T) k_chol64(Chol64Args a) {
  extern __shared__ double csm[];  // panel: rows x C64_P
  __shared__ double red[C64_T / 32];
  __shared__ int bad;
  const int s = a.s, t = threadIdx.x, T = blockDim.x;
  double* P = csm;
  double* M = a.M;
  if (*a.status != 0) return;
  // the largest diagonal entry of M + sigma I (the scale of the pivot bound)
  double dm = 0.0;
  for (int i = t; i < s; i += T) dm = fmax(dm, M[(size_t)i * s + i] + a.sigma);
  for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if ((t & 31) == 0) red[t >> 5] = dm;
  if (t == 0) bad = 0;
  __syncthreads();
  dm = 0.0;
  for (int w = 0; w < T / 32; ++w) dm = fmax(dm, red[w]);
  const double thr = TT_PIVOT_TOL64 * dm;
  for (int p0 = 0; p0 < s; p0 += C64_NB) {
    const int pb = min(C64_NB, s - p0), rows = s - p0;
    for (int e = t; e < rows * C64_NB; e += T) {
      const int i = e / C64_NB, c = e - i * C64_NB;
      double v = 0.0;
      if (c < pb && i >= c) v = M[(size_t)(p0 + i) * s + p0 + c] + (i == c ? a.sigma : 0.0);
      P[i * C64_P + c] = v;
    }
    __syncthreads();
    for (int c = 0; c < pb; ++c) {
      const double dpiv = P[c * C64_P + c];
      if (!(dpiv > thr) || !isfinite(dpiv)) {  // every thread reads the same value
        if (t == 0) bad = isfinite(dpiv) ? TT_ENOTSPD : TT_ENONFINITE;
        break;
      }
      const double l = sqrt(dpiv), il = 1.0 / l;
      __syncthreads();  // everyone has read the pivot before column c changes
      for (int i = c + t; i < rows; i += T) P[i * C64_P + c] = i == c ? l : P[i * C64_P + c] * il;
      __syncthreads();
      for (int e = t; e < rows * C64_NB; e += T) {  // the panel's columns right of c
        const int i = e / C64_NB, c2 = e - i * C64_NB;
        if (c2 > c && c2 < pb && i >= c2) P[i * C64_P + c2] = fma(-P[i * C64_P + c], P[c2 * C64_P + c], P[i * C64_P + c2]);
      }
      __syncthreads();
    }
    __syncthreads();
    if (bad) break;  // read after a barrier: the same value in every thread
    for (int e = t; e < rows * C64_NB; e += T) {  // L back over the Gram
      const int i = e / C64_NB, c = e - i * C64_NB;
      if (c < pb && i >= c) M[(size_t)(p0 + i) * s + p0 + c] = P[i * C64_P + c];
    }
    const int tr = rows - pb;  // trailing lower triangle: M[i][k] -= sum_c L[i][c] L[k][c]
    for (int e = t; e < tr * tr; e += T) {
      const int i = e / tr, kk = e - i * tr;
      if (kk > i) continue;
      const double* pi = P + (pb + i) * C64_P;
      const double* pk = P + (pb + kk) * C64_P;
      double acc = 0.0;
#pragma unroll 8
      for (int c = 0; c < pb; ++c) acc = fma(pi[c], pk[c], acc);
      M[(size_t)(p0 + pb + i) * s + p0 + pb + kk] -= acc;
    }
    __syncthreads();
  }
  if (bad && t == 0) atomicCAS(a.status, 0, bad);
}

struct Trsm64Args {
  const double* C;  // L (lower triangle of the s x s block), then B^T (s x n), row-major
  float* core;      // r0 x n x r1: proximal centre in, update out
  double* change;   // [0] += ||G_new - G_old||^2, [1] += ||G_new||^2 (may be null)
  double* part;     // deterministic mode: CTA b stores its two change sums at part[2 b]
  int* status;
  double sigma;
  int s, n, r0, nc;
};

constexpr int T64_NB = 32, T64_T = 256;

__global__ void __launch_bounds__(T64_T) k_trsm64(Trsm64Args a) {
  extern __shared__ double tsm[];
  const int s = a.s, n = a.n, r0 = a.r0, nc = a.nc;
  const int t = threadIdx.x, T = blockDim.x;
  const int c0 = blockIdx.x * nc, ncl = min(nc, n - c0);
  double* Z = tsm;                   // s x nc, row-major
  double* P = tsm + (size_t)s * nc;  // panel of L, at most 32 x s
  const double* L = a.C;
  const double* BT = a.C + (size_t)s * s;
  __shared__ int skip;  // the status read once: other CTAs of this kernel may raise it meanwhile
  if (t == 0) skip = *a.status != 0;
  __syncthreads();
  if (skip) return;
  for (int e = t; e < s * ncl; e += T) {  // Z = B^T + sigma G_c
    const int i = e / ncl, c = e - i * ncl;
    const int be = i / r0, al = i - be * r0;
    const double g = (double)a.core[al + (int64_t)r0 * ((c0 + c) + (int64_t)n * be)];
    Z[i * nc + c] = fma(a.sigma, g, BT[(size_t)i * n + c0 + c]);
  }
  // forward substitution L Z = Z, by 32-column panels of L (rows p0..s-1)
  for (int p0 = 0; p0 < s; p0 += T64_NB) {
    const int pb = min(T64_NB, s - p0), rows = s - p0;
    for (int e = t; e < rows * T64_NB; e += T) {
      const int i = e / T64_NB, c = e - i * T64_NB;
      P[e] = (c < pb && c <= i) ? L[(size_t)(p0 + i) * s + p0 + c] : 0.0;
    }
    __syncthreads();
    for (int c = 0; c < pb; ++c) {
      const int j = p0 + c;
      for (int col = t; col < ncl; col += T) Z[j * nc + col] /= P[c * T64_NB + c];
      __syncthreads();
      for (int e = t; e < (pb - c - 1) * ncl; e += T) {
        const int i = c + 1 + e / ncl, col = e % ncl;
        Z[(p0 + i) * nc + col] = fma(-P[i * T64_NB + c], Z[j * nc + col], Z[(p0 + i) * nc + col]);
      }
      __syncthreads();
    }
    for (int e = t; e < (rows - pb) * ncl; e += T) {  // the rows below the panel
      const int i = pb + e / ncl, col = e % ncl;
      double acc = Z[(p0 + i) * nc + col];
      for (int c = 0; c < pb; ++c) acc = fma(-P[i * T64_NB + c], Z[(p0 + c) * nc + col], acc);
      Z[(p0 + i) * nc + col] = acc;
    }
    __syncthreads();
  }
  // back substitution L^T X = Z, by 32-row blocks of L from the bottom (row b0 + jj, columns
  // 0 .. b0 + pb - 1, staged as pb x w)
  for (int b0 = ((s - 1) / T64_NB) * T64_NB; b0 >= 0; b0 -= T64_NB) {
    const int pb = min(T64_NB, s - b0), w = b0 + pb;
    for (int e = t; e < pb * w; e += T) {
      const int jj = e / w, i = e - jj * w;
      P[e] = i <= b0 + jj ? L[(size_t)(b0 + jj) * s + i] : 0.0;
    }
    __syncthreads();
    for (int jj = pb - 1; jj >= 0; --jj) {
      const int j = b0 + jj;
      for (int col = t; col < ncl; col += T) Z[j * nc + col] /= P[(size_t)jj * w + j];
      __syncthreads();
      for (int e = t; e < jj * ncl; e += T) {
        const int i = b0 + e / ncl, col = e % ncl;
        Z[i * nc + col] = fma(-P[(size_t)jj * w + i], Z[j * nc + col], Z[i * nc + col]);
      }
      __syncthreads();
    }
    for (int e = t; e < b0 * ncl; e += T) {  // the rows above the block
      const int i = e / ncl, col = e % ncl;
      double acc = Z[i * nc + col];
      for (int jj = 0; jj < pb; ++jj) acc = fma(-P[(size_t)jj * w + i], Z[(b0 + jj) * nc + col], acc);
      Z[i * nc + col] = acc;
    }
    __syncthreads();
  }
  bool nonfinite = false;
  for (int e = t; e < s * ncl; e += T) nonfinite |= !isfinite(Z[(e / ncl) * nc + e % ncl]);
  if (__syncthreads_or(nonfinite)) {  // an overflow in the solve: this chunk keeps its core
    if (t == 0) atomicCAS(a.status, 0, TT_ENONFINITE);
    return;
  }
  double dsum = 0.0, nsum = 0.0;
  for (int e = t; e < s * ncl; e += T) {
    const int i = e / ncl, c = e - i * ncl;
    const int be = i / r0, al = i - be * r0;
    float* g = a.core + al + (int64_t)r0 * ((c0 + c) + (int64_t)n * be);
    const double nw = Z[i * nc + c], dd = nw - (double)*g;
    dsum = fma(dd, dd, dsum);
    nsum = fma(nw, nw, nsum);
    *g = (float)nw;
  }
  if (a.change) {  // warp sums added in warp order, then one add (or one partial) per CTA
    __shared__ double cred[2][T64_T / 32];
    for (int o = 16; o > 0; o >>= 1) {
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
      nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
    }
    if ((t & 31) == 0) {
      cred[0][t >> 5] = dsum;
      cred[1][t >> 5] = nsum;
    }
    __syncthreads();
    if (t == 0) {
      double t1 = 0.0, t2 = 0.0;
      for (int w = 0; w < (T >> 5); ++w) {
        t1 += cred[0][w];
        t2 += cred[1][w];
      }
      if (a.part) {
        a.part[2 * blockIdx.x] = t1;
        a.part[2 * blockIdx.x + 1] = t2;
      } else {
        atomicAdd(a.change, t1);
        atomicAdd(a.change + 1, t2);
      }
    }
  }
}

size_t tt_chol64_smem(int s) { return sizeof(double) * (size_t)s * C64_P; }
size_t tt_trsm64_smem(int s, int nc) { return sizeof(double) * (size_t)s * (nc + T64_NB); }

int tt_launch_prox_update64(tt_ctx* c, const float* Y, const float* SH, float* core, int k, double* change_slot,
                            bool gram_zeroed) {
  const int s = c->r[k] * c->r[k + 1];
  const int n = (int)c->n[k];
  if (!gram_zeroed) TT_CUDA(c, cudaMemsetAsync(c->d_gram64, 0, sizeof(double) * (size_t)(s + n) * s, c->stream));
  Gram64Args g;
  g.SH = SH;
  g.Y = Y;
  g.C = c->d_gram64;
  g.status = c->d_status;
  g.P = c->det ? static_cast<double*>(c->d_gram_part) : nullptr;
  g.J = c->J;
  g.s = s;
  g.n = n;
  const int mt = (s + n + 63) / 64, nt = (s + 63) / 64;
  const int sms = tt_sm_count();
  int ksplit = std::max(1, std::min(c->J / 64, (2 * sms + mt * nt - 1) / (mt * nt)));
  if (c->det) ksplit = std::min(ksplit, TT_DET_KSPLIT);
  g.kchunk = ((c->J + ksplit - 1) / ksplit + 15) & ~15;
  const dim3 grid(mt, nt, (c->J + g.kchunk - 1) / g.kchunk);
  const bool vec = c->J % 16 == 0 && ((reinterpret_cast<uintptr_t>(SH) | reinterpret_cast<uintptr_t>(Y)) & 15) == 0;
  if (vec)
    k_gram64<true><<<grid, 256, 0, c->stream>>>(g);
  else
    k_gram64<false><<<grid, 256, 0, c->stream>>>(g);
  TT_LAUNCH(c, "k_gram64");
  if (c->det) TT_TRY(tt_launch_gram_reduce(c, c->d_gram_part, (int)grid.z, (int64_t)(s + n) * s, c->d_gram64, true));
  Chol64Args ch;
  ch.M = c->d_gram64;
  ch.status = c->d_status;
  ch.sigma = c->lambda;
  ch.s = s;
  const size_t csm = tt_chol64_smem(s);
  TT_CUDA(c, cudaFuncSetAttribute(k_chol64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
  k_chol64<<<1, C64_T, csm, c->stream>>>(ch);
  TT_LAUNCH(c, "k_chol64");
  if (change_slot) TT_CUDA(c, cudaMemsetAsync(change_slot, 0, 2 * sizeof(double), c->stream));
  Trsm64Args tr;
  tr.C = c->d_gram64;
  tr.core = core;
  tr.change = change_slot;
  tr.part = (c->det && change_slot) ? c->d_part_chg : nullptr;  // grid <= n_k <= the buffer's CTAs
  tr.status = c->d_status;
  tr.sigma = c->lambda;
  tr.s = s;
  tr.n = n;
  tr.r0 = c->r[k];
  // about two chunks per SM, at most 8 right-hand sides per chunk
  tr.nc = std::max(1, std::min(8, (n + 2 * sms - 1) / (2 * sms)));
  const size_t tsm = tt_trsm64_smem(s, tr.nc);
  TT_CUDA(c, cudaFuncSetAttribute(k_trsm64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
  const int tgrid = (n + tr.nc - 1) / tr.nc;
  k_trsm64<<<tgrid, T64_T, tsm, c->stream>>>(tr);
  TT_LAUNCH(c, "k_trsm64");
  if (tr.part) TT_TRY(tt_launch_sum_partials(c, tr.part, tgrid, change_slot));
  return TT_OK;
}
