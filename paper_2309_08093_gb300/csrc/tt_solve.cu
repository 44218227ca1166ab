// Part (c): the proximal update of Eq. (ite) (read with S^T S):
//   M = (S H_k)^T (S H_k) + sigma I,  B = Y_k^T (S H_k) + sigma G_{k(2)},  G_{k(2)} <- B M^{-1},
// plus the QR / LQ orthogonalisation steps of Algorithm 1 and the relative error of Sec. 5.
//
//   k_gram        : [S H_k | Y_k]^T (S H_k) with FP32 products summed in FP32 over K-chunks of
//                   256 rows and across chunks (split-K, FP32 atomics)
//   k_prox_solve  : Gauss-Jordan elimination of [M | B^T] in registers, one barrier per pivot,
//                   one CTA per chunk of right-hand-side rows (s <= 160)
//   k_qr_left_rows, k_lq_right_rows : CholeskyQR2 with rows in registers (rank <= 16), then
//                   G_k <- Q and R absorbed into the neighbour (prefetched during the QR)
//   k_qr_left     : the same for larger ranks (Gram in shared memory), Householder fallback:
//                   G_k^L = Q R, G_k <- Q, G_{k+1} <- R G_{k+1}^R
//   k_lq_right    : the same on (G_k^R)^T: G_k^R <- Q^T, G_{k-1}^L <- G_{k-1}^L R^T
//   k_slab_u, k_rint, k_rel_error_stream : ||A - [[G]]||_F^2 and ||A||_F^2: right interfaces of
//                   all mode-0 fibres, then one pass over A in memory order (bulk copies)
//   k_rel_error   : the same for other shapes (n_0 % 4 != 0 or n_0 > 1024), slab by slab
#include <stdio.h>

#include <algorithm>
#include <type_traits>

#include "tt_internal.cuh"

// 4-byte asynchronous copies global -> shared (cp.async), committed and awaited by group
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------------------------------------
// Gram and right-hand side

struct GramArgs {
  const float* SH;  // J x s column-major
  const float* Y;   // J x n column-major
  float* C;         // accumulators (zeroed by the caller): s x s Gram, then the s x n RHS
                    // (SH^T Y, row-major) -- both row-major
  int* status;      // raised to TT_ENONFINITE when a sum is not finite (may be null)
  float* P;         // deterministic mode: K-chunk z stores its sums at P + z (s + n) s (no atomics)
  int J, s, n, kchunk;
};

// CTA tile of 64 x 64 entries of [S H_k | Y_k]^T (S H_k) over one K-chunk; 256 threads with 4 x 4
// entries each. K-steps of 16 rows are staged through shared memory as [k][column], so that a
// thread reads its 4 rows and 4 columns with two 16-byte loads per k (8 FMAs per load); the next
// step's global loads (16 bytes per thread and operand when VEC: J % 16 == 0 and aligned bases;
// else 4 bounds-checked scalars) are in flight while the current step is multiplied. Chunks are
// summed with FP32 atomics. A non-finite partial sum (a NaN or Inf in S H_k or Y_k) raises
// TT_ENONFINITE, so the solve that follows leaves the core unchanged.
template <bool VEC>
__global__ void __launch_bounds__(256) k_gram(GramArgs a) {
  __shared__ __align__(16) float Xs[16][68];
  __shared__ __align__(16) float Bs[16][68];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int rows = a.s + a.n;
  const int r0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  const int kb = blockIdx.z * a.kchunk, ke = min(a.J, kb + a.kchunk);
  // loader: tile column lc = t / 4, k offset 4 (t % 4) within the step
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
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  if (kb < ke) load(kb);
  for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      Xs[lk + e][lc] = xr[e];
      Bs[lk + e][lc] = br[e];
    }
    __syncthreads();
    if (k0 + 16 < ke) load(k0 + 16);  // in flight during the FMAs below
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float4 xv = *reinterpret_cast<const float4*>(&Xs[kk][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
      const float2 blo = make_float2(bv.x, bv.y), bhi = make_float2(bv.z, bv.w);
#pragma unroll
      for (int i = 0; i < 4; ++i) {  // pairs of outputs per fma.rn.f32x2
        const float2 x2 = make_float2(xa[i], xa[i]);
        const float2 lo = tt_ffma2(x2, blo, make_float2(acc[i][0], acc[i][1]));
        const float2 hi = tt_ffma2(x2, bhi, make_float2(acc[i][2], acc[i][3]));
        acc[i][0] = lo.x, acc[i][1] = lo.y, acc[i][2] = hi.x, acc[i][3] = hi.y;
      }
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
  if (!finite && a.status) atomicCAS(a.status, 0, TT_ENONFINITE);
}

// Gram + right-hand side (C zeroed by the caller), any J >= 1. With g.P set (deterministic mode)
// at most TT_DET_KSPLIT K-chunks store partials that the caller sums in order.
static cudaError_t launch_gram(GramArgs g, cudaStream_t st, int* nz_out = nullptr) {
  const int mt = (g.s + g.n + 63) / 64, nt = (g.s + 63) / 64;
  const int sms = tt_sm_count();
  // K-chunks: about two CTAs per SM in all, each at least 64 rows of K
  int ksplit = std::max(1, std::min(g.J / 64, (2 * sms + mt * nt - 1) / (mt * nt)));
  if (g.P) ksplit = std::min(ksplit, TT_DET_KSPLIT);
  g.kchunk = ((g.J + ksplit - 1) / ksplit + 15) & ~15;
  dim3 grid(mt, nt, (g.J + g.kchunk - 1) / g.kchunk);
  if (nz_out) *nz_out = (int)grid.z;
  const bool vec = g.J % 16 == 0 && ((reinterpret_cast<uintptr_t>(g.SH) | reinterpret_cast<uintptr_t>(g.Y)) & 15) == 0;
  if (vec)
    k_gram<true><<<grid, 256, 0, st>>>(g);
  else
    k_gram<false><<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Cholesky + triangular solves, one CTA

struct SolveArgs {
  const float* C;   // s x s Gram SH^T SH, then s x n SH^T Y (both row-major)
  float* core;      // r0 x n x r1 (read: proximal centre; written: update)
  double* change;   // [0] += ||G_new - G_old||^2, [1] += ||G_new||^2 (may be null)
  double* part;     // deterministic mode: CTA b stores its two change sums at part[2 b]
  int* status;
  double sigma;
  int s, n, r0, r1;
  int chunk_rows;
};

// Gauss-Jordan elimination without pivoting of the s x (s + nr) array W = [M | B_c^T], where B_c
// holds the nr right-hand-side rows of this CTA's chunk. Step j divides row j by its pivot
// W[j][j] (the D of M = L D L^T: positive exactly when M is SPD) and subtracts W[i][j] times it
// from every other row i; after s steps the first s columns are the identity and
// X_c[r][i] = W[i][s + r]. W lives in registers: thread (ty, tx) of a TY x 32 layout owns
// W[ty + TY a][tx + 32 b]. A warp needs column j only for its own rows, so lane j % 32 hands it
// over by shuffles; the normalised row j is published through shared memory by its warp at the
// end of step j - 1: one barrier per step. Steps run in groups of TY (template recursion over
// the group G): row j is then register block G of warp j - TY G and column j register block
// TY G / 32 of lane j % 32, both compile-time, so no register is ever selected by a runtime
// index. Column blocks wholly left of the group's pivots are dead and skipped.
// A pivot at or below `thr` (TT_PIVOT_TOL32 times the largest diagonal entry of M + sigma I: the
// system cannot be told from the FP32 Gram's rounding noise) refuses the update with TT_ENOTSPD.
template <int TY, int RA, int CB, int G>
__device__ __forceinline__ void gj_publish_row(float (&w)[RA][CB], int jn, float* rowb, int* bad, int ty, int tx,
                                               float thr) {
  constexpr int CN = (TY * G) / 32;  // column block of pivots TY G .. TY G + TY - 1
  if (ty == jn - TY * G) {           // the warp that owns row jn (register block G)
    const float p = __shfl_sync(0xffffffffu, w[G][CN], jn & 31);
    if (tx == 0 && (!(p > thr) || !isfinite(p))) atomicCAS(bad, 0, isfinite(p) ? TT_ENOTSPD : TT_ENONFINITE);
    const float ip = 1.f / p;
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) {
      const float v = w[G][cb] * ip;
      w[G][cb] = v;
      rowb[tx + 32 * cb] = v;
    }
  }
}

template <int TY, int RA, int CB, int G>
__device__ __forceinline__ void gj_groups(float (&w)[RA][CB], int s, float (*rowbuf)[CB * 32], int* bad, int& bs,
                                          int ty, int tx, float thr) {
  if constexpr (G < RA) {
    constexpr int CN = (TY * G) / 32;  // column block of this group's pivots = first live block
    const int j0 = TY * G;
    if (j0 >= s) return;
    const int jend = min(TY, s - j0);
    for (int jj = 0; jj < jend; ++jj) {
      const int jl = (j0 + jj) & 31;  // the lane that holds column j
      float f[RA], rv[CB];
#pragma unroll
      for (int ra = 0; ra < RA; ++ra) f[ra] = __shfl_sync(0xffffffffu, w[ra][CN], jl);
      if (ty == jj) f[G] = 0.f;  // row j itself (already normalised) is left alone
#pragma unroll
      for (int cb = CN & ~1; cb < CB; ++cb) rv[cb] = rowbuf[bs][tx + 32 * cb];
      // pairs of column blocks per fma.rn.f32x2 (a dead block left of CN may be updated too: it
      // is never read again)
      constexpr int CP = CN & ~1;
#pragma unroll
      for (int cb = CP; cb < CB; cb += 2) {
        if (cb + 1 < CB) {
#pragma unroll
          for (int ra = 0; ra < RA; ++ra) {
            const float2 d = tt_ffma2(make_float2(-f[ra], -f[ra]), make_float2(rv[cb], rv[cb + 1]),
                                      make_float2(w[ra][cb], w[ra][cb + 1]));
            w[ra][cb] = d.x;
            w[ra][cb + 1] = d.y;
          }
        } else {
#pragma unroll
          for (int ra = 0; ra < RA; ++ra) w[ra][cb] = fmaf(-f[ra], rv[cb], w[ra][cb]);
        }
      }
      const int jn = j0 + jj + 1;
      if (jn < s) {
        if (jj + 1 < TY)
          gj_publish_row<TY, RA, CB, G>(w, jn, rowbuf[bs ^ 1], bad, ty, tx, thr);
        else if constexpr (G + 1 < RA)
          gj_publish_row<TY, RA, CB, G + 1>(w, jn, rowbuf[bs ^ 1], bad, ty, tx, thr);
      }
      __syncthreads();
      bs ^= 1;
    }
    gj_groups<TY, RA, CB, G + 1>(w, s, rowbuf, bad, bs, ty, tx, thr);
  }
}

template <int TY, int RA, int CB>
__global__ void __launch_bounds__(TY * 32) k_prox_solve(SolveArgs a) {
  constexpr int T = TY * 32;
  __shared__ __align__(16) float rowbuf[2][CB * 32];
  __shared__ float gsm[RA * TY][33];  // this chunk of G_{k(2)}^T: proximal centre, then the update
  __shared__ float red[2][TY];
  __shared__ int bad;
  __shared__ int dmax_bits;  // largest diagonal entry of M + sigma I (a positive float's bits)
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  const int s = a.s, r0 = a.r0, n = a.n;
  const int i0 = blockIdx.x * a.chunk_rows;
  const int nr = min(a.chunk_rows, n - i0);
  const int ncol = s + nr;
  const float sigma = (float)a.sigma;
  __shared__ int skip;  // the status read once: other CTAs of this kernel may raise it meanwhile
  if (t == 0) skip = *a.status != 0;
  __syncthreads();
  if (skip) return;
  // M and the transposed right-hand side: unconditional loads (clamped addresses) so that many
  // are in flight at once; row-major rows of both are read along the lanes
  float w[RA][CB];
#pragma unroll
  for (int ra = 0; ra < RA; ++ra) {
    const int ic = min(ty + TY * ra, s - 1);
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) {
      const int l = tx + 32 * cb;
      const int r = min(max(l - s, 0), nr - 1);
      const int64_t ci = (l < s) ? (int64_t)ic * s + l : (int64_t)s * s + (int64_t)ic * n + i0 + r;
      w[ra][cb] = __ldg(a.C + ci);
    }
  }
  // the chunk's proximal centre, coalesced and asynchronous: gsm[al + r0 be][r] = G(al, i0 + r, be)
  const int rn = r0 * nr;
  for (int idx = t; idx < s * nr; idx += T) {
    const int be = idx / rn, rem = idx - be * rn, r = rem / r0, al = rem - r * r0;
    cp_async4(&gsm[al + r0 * be][r], a.core + al + (int64_t)r0 * ((i0 + r) + (int64_t)n * be));
  }
  cp_async_commit();
  if (t == 0) {
    bad = 0;
    dmax_bits = 0;
  }
  cp_async_wait<0>();
  __syncthreads();
  float dloc = 0.f;
#pragma unroll
  for (int ra = 0; ra < RA; ++ra) {
    const int i = ty + TY * ra;
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) {
      const int l = tx + 32 * cb;
      const bool in = i < s && l < ncol;
      float v = w[ra][cb];
      if (l == i) v += sigma;
      if (in && l >= s) v = fmaf(sigma, gsm[i][l - s], v);
      if (in && l == i) dloc = fmaxf(dloc, v);
      w[ra][cb] = in ? v : 0.f;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dloc = fmaxf(dloc, __shfl_xor_sync(0xffffffffu, dloc, o));
  if (tx == 0 && dloc > 0.f) atomicMax(&dmax_bits, __float_as_int(dloc));  // positive floats order as ints
  __syncthreads();
  const float thr = TT_PIVOT_TOL32 * __int_as_float(dmax_bits);
  gj_publish_row<TY, RA, CB, 0>(w, 0, rowbuf[0], &bad, ty, tx, thr);
  __syncthreads();
  int bs = 0;
  gj_groups<TY, RA, CB, 0>(w, s, rowbuf, &bad, bs, ty, tx, thr);
  if (bad) {  // read after the last step's barrier: the same value in every thread
    if (t == 0) atomicCAS(a.status, 0, bad);
    return;
  }
  // change sums against the proximal centre, the update into gsm, then coalesced stores
  float dsum = 0.f, nsum = 0.f;
#pragma unroll
  for (int ra = 0; ra < RA; ++ra) {
    const int i = ty + TY * ra;
    if (i >= s) continue;
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) {
      const int l = tx + 32 * cb;
      if (l < s || l >= ncol) continue;
      const float nw = w[ra][cb], d = nw - gsm[i][l - s];
      dsum = fmaf(d, d, dsum);
      nsum = fmaf(nw, nw, nsum);
      gsm[i][l - s] = nw;
    }
  }
  if (a.change) {  // slot zeroed by the host
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
      nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
    }
    if (tx == 0) {
      red[0][ty] = dsum;
      red[1][ty] = nsum;
    }
  }
  __syncthreads();
  for (int idx = t; idx < s * nr; idx += T) {
    const int be = idx / rn, rem = idx - be * rn, r = rem / r0, al = rem - r * r0;
    a.core[al + (int64_t)r0 * ((i0 + r) + (int64_t)n * be)] = gsm[al + r0 * be][r];
  }
  if (a.change && t == 0) {
    float t1 = 0.f, t2 = 0.f;
    for (int u = 0; u < TY; ++u) {
      t1 += red[0][u];
      t2 += red[1][u];
    }
    if (a.part) {
      a.part[2 * blockIdx.x] = (double)t1;
      a.part[2 * blockIdx.x + 1] = (double)t2;
    } else {
      atomicAdd(a.change, (double)t1);
      atomicAdd(a.change + 1, (double)t2);
    }
  }
}

// Register shapes of the solve (TY x 32 threads, RA row blocks of TY, CB column blocks of 32):
// the first that holds s rows and s + 1 columns; its spare columns carry right-hand-side rows.
struct SolveShape {
  int ty, ra, cb;
};
static const SolveShape kSolveShapes[] = {{8, 4, 2}, {8, 14, 4}, {16, 10, 6}};

static cudaError_t launch_prox_solve(SolveArgs a, cudaStream_t st, int* grid_out = nullptr) {
  for (const SolveShape& sh : kSolveShapes) {
    if (a.s > sh.ty * sh.ra || a.s + 1 > 32 * sh.cb) continue;
    a.chunk_rows = std::max(1, std::min(a.n, std::min(32, 32 * sh.cb - a.s)));
    const int grid = (a.n + a.chunk_rows - 1) / a.chunk_rows;
    if (grid_out) *grid_out = grid;
    if (sh.ra == 4)
      k_prox_solve<8, 4, 2><<<grid, 256, 0, st>>>(a);
    else if (sh.ra == 14)
      k_prox_solve<8, 14, 4><<<grid, 256, 0, st>>>(a);
    else
      k_prox_solve<16, 10, 6><<<grid, 512, 0, st>>>(a);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;  // s above TT_MAX_S, rejected at context creation
}

// Large systems (TT_MAX_S < s <= TT_MAX_S_LARGE): one CTA of 1024 threads factors
// M + sigma I = L L^T (Cholesky, right-looking by 32-column panels) and solves for all n
// right-hand sides. A panel (rows p0..s-1, 32 columns) is staged in shared memory, factored there
// column by column, written back over the Gram (L2-resident) and applied to the trailing lower
// triangle; while it is in shared memory it also carries out its part of the forward substitution
// L Z = B^T + sigma G_c on Z (s x n, shared). The back substitution L^T X^T = Z then walks row
// blocks of L from the bottom, staged in shared memory. A non-positive or non-finite pivot raises
// the status (TT_ENOTSPD / TT_ENONFINITE) and leaves the core unchanged. Shared memory:
// 4 (33 s + s n) bytes.
constexpr int LS_NB = 32, LS_P = 33;
__global__ void __launch_bounds__(1024) k_prox_solve_large(SolveArgs a) {
  extern __shared__ float lsm[];
  __shared__ int bad;
  __shared__ int dmax_bits;  // largest diagonal entry of M + sigma I (a positive float's bits)
  const int s = a.s, n = a.n, r0 = a.r0;
  const int t = threadIdx.x, T = blockDim.x;
  float* P = lsm;                       // panel, rows x LS_P
  float* Z = lsm + (size_t)s * LS_P;    // s x n right-hand sides, then solutions
  float* M = const_cast<float*>(a.C);   // factored in place (recomputed by every update)
  const float* BT = a.C + (size_t)s * s;
  const float sigma = (float)a.sigma;
  if (*a.status != 0) return;
  if (t == 0) {
    bad = 0;
    dmax_bits = 0;
  }
  __syncthreads();
  float dloc = 0.f;
  for (int i = t; i < s; i += T) dloc = fmaxf(dloc, M[(size_t)i * s + i] + sigma);
  for (int o = 16; o > 0; o >>= 1) dloc = fmaxf(dloc, __shfl_xor_sync(0xffffffffu, dloc, o));
  if ((t & 31) == 0 && dloc > 0.f) atomicMax(&dmax_bits, __float_as_int(dloc));
  for (int e = t; e < s * n; e += T) {  // Z = B^T + sigma G_c
    const int i = e / n, r = e - i * n;
    const int be = i / r0, al = i - be * r0;
    Z[e] = fmaf(sigma, a.core[al + (int64_t)r0 * (r + (int64_t)n * be)], BT[e]);
  }
  __syncthreads();
  const float thr = TT_PIVOT_TOL32 * __int_as_float(dmax_bits);
  for (int p0 = 0; p0 < s; p0 += LS_NB) {
    const int pb = min(LS_NB, s - p0), rows = s - p0;
    for (int e = t; e < rows * LS_NB; e += T) {
      const int i = e / LS_NB, c = e - i * LS_NB;
      float v = 0.f;
      if (c < pb && i >= c) v = M[(size_t)(p0 + i) * s + p0 + c] + (i == c ? sigma : 0.f);
      P[i * LS_P + c] = v;
    }
    __syncthreads();
    for (int c = 0; c < pb; ++c) {
      const float d = P[c * LS_P + c];
      if (!(d > thr) || !isfinite(d)) {
        if (t == 0) bad = isfinite(d) ? TT_ENOTSPD : TT_ENONFINITE;
        break;  // every thread reads the same d
      }
      const float l = sqrtf(d), il = 1.f / l;
      __syncthreads();  // everyone has read d before column c changes
      for (int i = c + t; i < rows; i += T) P[i * LS_P + c] = i == c ? l : P[i * LS_P + c] * il;
      __syncthreads();
      for (int e = t; e < rows * LS_NB; e += T) {  // the panel's columns right of c
        const int i = e / LS_NB, c2 = e - i * LS_NB;
        if (c2 > c && c2 < pb && i >= c2) P[i * LS_P + c2] = fmaf(-P[i * LS_P + c], P[c2 * LS_P + c], P[i * LS_P + c2]);
      }
      // forward substitution of this column: Z[p0 + c] /= l, then the rows below it
      for (int r = t; r < n; r += T) Z[(size_t)(p0 + c) * n + r] *= il;
      __syncthreads();
      for (int e = t; e < (rows - c - 1) * n; e += T) {
        const int i = c + 1 + e / n, r = e % n;
        Z[(size_t)(p0 + i) * n + r] = fmaf(-P[i * LS_P + c], Z[(size_t)(p0 + c) * n + r], Z[(size_t)(p0 + i) * n + r]);
      }
      __syncthreads();
    }
    __syncthreads();
    if (bad) break;  // read after a barrier: the same value in every thread
    for (int e = t; e < rows * LS_NB; e += T) {  // L back over the Gram
      const int i = e / LS_NB, c = e - i * LS_NB;
      if (c < pb && i >= c) M[(size_t)(p0 + i) * s + p0 + c] = P[i * LS_P + c];
    }
    const int tr = rows - pb;  // trailing lower triangle: M[i][k] -= sum_c L[i][c] L[k][c]
    for (int e = t; e < tr * tr; e += T) {
      const int i = e / tr, kk = e - i * tr;
      if (kk > i) continue;
      const float* pi = P + (pb + i) * LS_P;
      const float* pk = P + (pb + kk) * LS_P;
      float acc = 0.f;
      for (int c = 0; c < pb; ++c) acc = fmaf(pi[c], pk[c], acc);
      float* m = M + (size_t)(p0 + pb + i) * s + p0 + pb + kk;
      *m -= acc;
    }
    __syncthreads();
  }
  if (bad) {
    if (t == 0) atomicCAS(a.status, 0, bad);
    return;
  }
  // back substitution L^T X^T = Z, row blocks of L from the bottom (rows b0..b0+pb-1, columns
  // 0..b0+pb-1 staged as pb x (b0 + pb))
  for (int b0 = ((s - 1) / LS_NB) * LS_NB; b0 >= 0; b0 -= LS_NB) {
    const int pb = min(LS_NB, s - b0), w = b0 + pb;
    for (int e = t; e < pb * w; e += T) {
      const int j = e / w, i = e - j * w;
      P[e] = i <= b0 + j ? M[(size_t)(b0 + j) * s + i] : 0.f;
    }
    __syncthreads();
    for (int j = pb - 1; j >= 0; --j) {
      const float* Lj = P + (size_t)j * w;  // row b0 + j of L
      const float il = 1.f / Lj[b0 + j];
      for (int r = t; r < n; r += T) Z[(size_t)(b0 + j) * n + r] *= il;
      __syncthreads();
      for (int e = t; e < (b0 + j) * n; e += T) {
        const int i = e / n, r = e - i * n;
        Z[e] = fmaf(-Lj[i], Z[(size_t)(b0 + j) * n + r], Z[e]);
      }
      __syncthreads();
    }
  }
  // the update into the core, with the change sums against the proximal centre
  float dsum = 0.f, nsum = 0.f;
  for (int e = t; e < s * n; e += T) {
    const int i = e / n, r = e - i * n;
    const int be = i / r0, al = i - be * r0;
    float* g = a.core + al + (int64_t)r0 * (r + (int64_t)n * be);
    const float nw = Z[e], dd = nw - *g;
    dsum = fmaf(dd, dd, dsum);
    nsum = fmaf(nw, nw, nsum);
    *g = nw;
  }
  if (a.change) {  // one CTA: warp sums added in warp order (the same bits on every run)
    __shared__ float cred[2][32];
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
      atomicAdd(a.change, t1);
      atomicAdd(a.change + 1, t2);
    }
  }
}

size_t tt_large_solve_smem(int s, int n) { return sizeof(float) * ((size_t)s * LS_P + (size_t)s * n); }

int tt_launch_prox_update(tt_ctx* c, const float* Y, const float* SH, float* core, int k,
                          double* change_slot, bool gram_zeroed) {
  if (c->solve64) return tt_launch_prox_update64(c, Y, SH, core, k, change_slot, gram_zeroed);
  const int s = c->r[k] * c->r[k + 1];
  const int n = (int)c->n[k];
  if (!gram_zeroed) TT_CUDA(c, cudaMemsetAsync(c->d_gram, 0, sizeof(float) * (s + n) * s, c->stream));
  GramArgs g;
  g.SH = SH;
  g.Y = Y;
  g.C = c->d_gram;
  g.status = c->d_status;
  g.P = c->det ? static_cast<float*>(c->d_gram_part) : nullptr;
  g.J = c->J;
  g.s = s;
  g.n = n;
  int nz = 1;
  if ((c->flags & (TT_FLAG_TC_GRAM | TT_FLAG_TF32_GRAM)) && tt_gram_tc_fits(c->J, s, SH, Y)) {
    TT_TRY(tt_launch_gram_tc(c, SH, Y, s, n, c->d_gram, g.P, !(c->flags & TT_FLAG_TF32_GRAM), &nz));
  } else {
    TT_CUDA(c, launch_gram(g, c->stream, &nz));
    TT_LAUNCH(c, "k_gram");
  }
  if (c->det) TT_TRY(tt_launch_gram_reduce(c, c->d_gram_part, nz, (int64_t)(s + n) * s, c->d_gram, false));
  SolveArgs a;
  a.C = c->d_gram;
  a.core = core;
  a.change = change_slot;
  a.status = c->d_status;
  a.sigma = c->lambda;
  a.s = s;
  a.n = n;
  a.r0 = c->r[k];
  a.r1 = c->r[k + 1];
  a.part = nullptr;
  if (change_slot) TT_CUDA(c, cudaMemsetAsync(change_slot, 0, 2 * sizeof(double), c->stream));
  if (s > TT_MAX_S) {  // Cholesky in one CTA (sizes checked at context creation)
    const size_t smem = tt_large_solve_smem(s, n);
    TT_CUDA(c, cudaFuncSetAttribute(k_prox_solve_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_prox_solve_large<<<1, 1024, smem, c->stream>>>(a);
    TT_LAUNCH(c, "k_prox_solve_large");
    return TT_OK;
  }
  if (c->det && change_slot) a.part = c->d_part_chg;  // grid <= n_k <= the buffer's CTAs
  int grid = 0;
  TT_CUDA(c, launch_prox_solve(a, c->stream, &grid));
  TT_LAUNCH(c, "k_prox_solve");
  if (a.part) TT_TRY(tt_launch_sum_partials(c, a.part, grid, change_slot));
  return TT_OK;
}

// ---------------------------------------------------------------------------------------------
// Householder QR of an m x q column-major matrix held in shared memory (q small).
// On exit: A holds Q (m x p, p = min(m, q)) in its first p columns, R (p x q) in Rm (q x q,
// row-major, rows >= p zero), with diag(R) >= 0.

__device__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ void block_householder_qr(float* A, int m, int q, float* Rm, float* tau, float* colsc) {
  const int p = min(m, q);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < p; ++j) {
    float* x = A + (int64_t)j * m;
    // norm of x[j+1 : m]
    if (warp == 0) {
      float ss = 0.f;
      for (int i = j + 1 + lane; i < m; i += 32) ss = fmaf(x[i], x[i], ss);
      ss = warp_sum(ss);
      if (lane == 0) {
        float alpha = x[j];
        float xn = sqrtf(ss);
        if (xn == 0.f) {
          tau[j] = 0.f;
          colsc[0] = 0.f;
        } else {
          float beta = -copysignf(hypotf(alpha, xn), alpha);
          tau[j] = (beta - alpha) / beta;
          colsc[0] = 1.f / (alpha - beta);
          x[j] = beta;
        }
      }
    }
    __syncthreads();
    const float sc = colsc[0];
    const float tj = tau[j];
    if (tj != 0.f)
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) x[i] *= sc;
    __syncthreads();
    if (tj != 0.f) {
      // apply H_j = I - tau v v^T (v_j = 1) to columns j+1..q-1, one warp per column
      for (int cc = j + 1 + warp; cc < q; cc += nw) {
        float* y = A + (int64_t)cc * m;
        float w = 0.f;
        for (int i = j + 1 + lane; i < m; i += 32) w = fmaf(x[i], y[i], w);
        w = warp_sum(w) + y[j];
        w *= tj;
        if (lane == 0) y[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) y[i] = fmaf(-w, x[i], y[i]);
      }
    }
    __syncthreads();
  }
  // R (upper trapezoid) out, zero below
  for (int idx = threadIdx.x; idx < q * q; idx += blockDim.x) {
    int i = idx / q, jj = idx - i * q;
    Rm[idx] = (i < p && jj >= i) ? A[(int64_t)jj * m + i] : 0.f;
  }
  __syncthreads();
  // form Q in place (backward accumulation of the reflectors), columns 0..p-1
  for (int j = p - 1; j >= 0; --j) {
    float* x = A + (int64_t)j * m;
    const float tj = tau[j];
    for (int cc = j + 1 + warp; cc < p; cc += nw) {
      float* y = A + (int64_t)cc * m;
      float w = 0.f;
      for (int i = j + 1 + lane; i < m; i += 32) w = fmaf(x[i], y[i], w);
      w = (warp_sum(w) + y[j]) * tj;
      if (lane == 0) y[j] -= w;
      for (int i = j + 1 + lane; i < m; i += 32) y[i] = fmaf(-w, x[i], y[i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      if (i < j)
        x[i] = 0.f;
      else if (i == j)
        x[i] = 1.f - tj;
      else
        x[i] = -tj * x[i];
    }
    __syncthreads();
  }
  // non-negative diagonal of R
  for (int j = 0; j < p; ++j) {
    if (Rm[j * q + j] < 0.f) {
      for (int t = threadIdx.x; t < q; t += blockDim.x) Rm[j * q + t] = -Rm[j * q + t];
      for (int i = threadIdx.x; i < m; i += blockDim.x) A[(int64_t)j * m + i] = -A[(int64_t)j * m + i];
    }
    __syncthreads();
  }
}

// CholeskyQR2 of the m x q column-major matrix A (pitch lda) in shared memory: two passes of
// W = A^T A (threads own (i, j, row-group) partial sums), W = R^T R (one warp, FP32 Cholesky),
// A <- A R^{-1} (one thread per row). With rows >= q and a well-conditioned A the result is the
// unique QR factorisation with positive diagonal; a non-positive or relatively tiny pivot
// (rank deficiency, a wide matrix, a very ill-conditioned core) returns false and the caller
// falls back to Householder. On success A holds Q and Rm (q x q row-major) holds R.
__device__ bool block_cholqr2(float* A, int m, int q, int lda, float* Rm, float* W, float* Rp, int* flag) {
  const int t = threadIdx.x, T = blockDim.x;
  const int lane = t & 31, warp = t >> 5;
  const int pairs = q * q;
  const int tri = q * (q + 1) / 2;  // lower-triangle pairs (i >= j), p = i (i + 1) / 2 + j
  const int G = max(1, min(32, T / max(1, tri)));
  for (int pass = 0; pass < 2; ++pass) {
    // W = A^T A on the lower triangle, partial sums over G row groups
    for (int idx = t; idx < tri * G; idx += T) {
      const int p = idx % tri, g = idx / tri;
      int i = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);
      while (i * (i + 1) / 2 > p) --i;
      while ((i + 1) * (i + 2) / 2 <= p) ++i;
      const int j = p - i * (i + 1) / 2;
      float acc = 0.f;
      for (int r = g; r < m; r += G) acc = fmaf(A[r + lda * i], A[r + lda * j], acc);
      W[idx] = acc;
    }
    __syncthreads();
    if (warp == 0) {
      // reduce the groups, then Cholesky W = L L^T (lower, row-major in Rp); R = L^T
      for (int pr = lane; pr < pairs; pr += 32) {
        const int i = pr / q, j = pr - i * q;
        float acc = 0.f;
        if (j <= i) {
          const int p = i * (i + 1) / 2 + j;
          for (int g = 0; g < G; ++g) acc += W[p + tri * g];
        }
        Rp[pr] = acc;
      }
      __syncwarp();
      float dmax = 0.f;
      for (int i = 0; i < q; ++i) dmax = fmaxf(dmax, Rp[i * q + i]);
      int ok = (dmax > 0.f && isfinite(dmax)) ? 1 : 0;
      for (int j = 0; j < q && ok; ++j) {
        const float pj = Rp[j * q + j];
        if (!(pj > 1e-6f * dmax) || !isfinite(pj)) {  // kappa(A) above ~1e3: use Householder
          ok = 0;
          break;
        }
        const float lj = sqrtf(pj);
        __syncwarp();
        for (int i = j + lane; i < q; i += 32) Rp[i * q + j] = (i == j) ? lj : Rp[i * q + j] / lj;
        __syncwarp();
        for (int i = j + 1 + lane; i < q; i += 32) {
          const float lij = Rp[i * q + j];
          for (int l = j + 1; l <= i; ++l) Rp[i * q + l] -= lij * Rp[l * q + j];
        }
        __syncwarp();
      }
      if (lane == 0) *flag = ok;
    }
    __syncthreads();
    if (!*flag) return false;
    // A <- A R^{-1} with R = L^T: row r solves x L^T = a_r (x_j = (a_j - sum_{l<j} x_l L[j][l]) / L[j][j])
    for (int r = t; r < m; r += T) {
      for (int j = 0; j < q; ++j) {
        float v = A[r + lda * j];
        for (int l = 0; l < j; ++l) v -= A[r + lda * l] * Rp[j * q + l];
        A[r + lda * j] = v / Rp[j * q + j];
      }
    }
    // R_total = R_pass * R_total  (R_pass = L^T upper)
    if (warp == 1 || (T == 32 && warp == 0)) {
      for (int pr = lane; pr < pairs; pr += 32) {
        const int i = pr / q, j = pr - i * q;
        float acc = 0.f;
        if (pass == 0) {
          acc = (j >= i) ? Rp[j * q + i] : 0.f;
        } else {
          for (int l = i; l <= j; ++l) acc = fmaf(Rp[l * q + i], Rm[l * q + j], acc);
        }
        W[pr] = acc;
      }
      __syncwarp();
      for (int pr = lane; pr < pairs; pr += 32) Rm[pr] = W[pr];
    }
    __syncthreads();
  }
  return true;
}

// Shared-memory layout of the QR kernels: A (lda x q) | Rm (q x q) | tau (q) | colsc (4) |
// W (max(q*q, 512)) | Rp (q*q). CholeskyQR2 is used for q <= 32; otherwise, or when it reports a
// tiny pivot, Householder runs on a dense copy (pitch m) of the input.
struct QrSmem {
  float *A, *Rm, *tau, *colsc, *W, *Rp;
  int lda;
};
__device__ QrSmem qr_layout(float* sm, int m, int q, int use_chol) {
  QrSmem L;
  L.lda = use_chol ? (m | 1) : m;
  L.A = sm;
  L.Rm = L.A + (int64_t)L.lda * q;
  L.tau = L.Rm + q * q;
  L.colsc = L.tau + q;
  L.W = L.colsc + 4;
  L.Rp = L.W + max(q * q, 512);
  return L;
}

// Copy `total` floats from global into shared memory with UB independent loads in flight per
// thread: the loads of a batch are issued before any of its stores (a plain copy loop waits for
// each global load in turn). src(idx) / dst(idx) give the source and destination addresses.
template <typename Src, typename Dst>
__device__ __forceinline__ void stage_batched(int total, Src src, Dst dst) {
  constexpr int UB = 8;
  for (int b0 = threadIdx.x; b0 < total; b0 += UB * blockDim.x) {
    float v[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int idx = b0 + u * blockDim.x;
      v[u] = idx < total ? *src(idx) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int idx = b0 + u * blockDim.x;
      if (idx < total) *dst(idx) = v[u];
    }
  }
}

// G_k^L (m = r0 n rows, q = r1 cols) = Q R; G_k <- Q (zero-padded); G_{k+1} <- R G_{k+1}^R
__global__ void __launch_bounds__(512) k_qr_left(float* core, float* next, int r0, int n, int r1,
                                                 int ncols_next, int use_chol, const int* status) {
  extern __shared__ float sm[];
  __shared__ int flag;
  if (*status != 0) return;
  const int m = r0 * n, q = r1;
  const QrSmem L = qr_layout(sm, m, q, use_chol);
  bool ok = false;
  if (use_chol && m >= q) {
    stage_batched(m * q, [&](int idx) { return core + idx; },
                  [&](int idx) { return L.A + (idx % m) + (int64_t)L.lda * (idx / m); });
    __syncthreads();
    ok = block_cholqr2(L.A, m, q, L.lda, L.Rm, L.W, L.Rp, &flag);
    __syncthreads();
    if (ok)
      for (int idx = threadIdx.x; idx < m * q; idx += blockDim.x) {
        const int r = idx % m, j = idx / m;
        core[idx] = L.A[r + L.lda * j];
      }
  }
  if (!ok) {  // Householder on a dense copy of the input (G_k^L is column-major, pitch m)
    stage_batched(m * q, [&](int idx) { return core + idx; }, [&](int idx) { return L.A + idx; });
    __syncthreads();
    block_householder_qr(L.A, m, q, L.Rm, L.tau, L.colsc);
    const int p = min(m, q);
    for (int idx = threadIdx.x; idx < m * q; idx += blockDim.x) core[idx] = (idx / m < p) ? L.A[idx] : 0.f;
  }
  __syncthreads();
  // G_{k+1}^R <- R G_{k+1}^R (r1 x ncols_next, column-major), staged through the free A region
  // in pieces that fit it
  const int64_t cap = (int64_t)L.lda * q;  // floats available in A
  const int cols_per = (int)(cap / r1 > 1 ? cap / r1 : 1);
  for (int c0 = 0; c0 < ncols_next; c0 += cols_per) {
    const int nc = min(cols_per, ncols_next - c0);
    float* g = next + (int64_t)c0 * r1;
    stage_batched(nc * r1, [&](int idx) { return g + idx; }, [&](int idx) { return L.A + idx; });
    __syncthreads();
    for (int idx = threadIdx.x; idx < nc * r1; idx += blockDim.x) {
      const int cc = idx / r1, a2 = idx - cc * r1;
      const float* col = L.A + (size_t)cc * r1;
      float acc = 0.f;
      for (int b = a2; b < r1; ++b) acc = fmaf(L.Rm[a2 * q + b], col[b], acc);
      g[idx] = acc;
    }
    __syncthreads();
  }
}

// (G_k^R)^T (m = n r1 rows, q = r0 cols) = Q R; G_k^R <- Q^T; G_{k-1}^L <- G_{k-1}^L R^T
__global__ void __launch_bounds__(512) k_lq_right(float* prev, float* core, int r0, int n, int r1,
                                                  int nrows_prev, int use_chol, const int* status) {
  extern __shared__ float sm[];
  __shared__ int flag;
  if (*status != 0) return;
  const int m = n * r1, q = r0;
  const QrSmem L = qr_layout(sm, m, q, use_chol);
  bool ok = false;
  if (use_chol && m >= q) {
    stage_batched(m * q, [&](int idx) { return core + (idx / m) + (int64_t)r0 * (idx % m); },
                  [&](int idx) { return L.A + (idx % m) + (int64_t)L.lda * (idx / m); });
    __syncthreads();
    ok = block_cholqr2(L.A, m, q, L.lda, L.Rm, L.W, L.Rp, &flag);
    __syncthreads();
    if (ok)
      for (int idx = threadIdx.x; idx < m * q; idx += blockDim.x) {
        const int i = idx % m, a2 = idx / m;
        core[a2 + (int64_t)r0 * i] = L.A[i + L.lda * a2];
      }
  }
  if (!ok) {
    stage_batched(m * q, [&](int idx) { return core + (idx / m) + (int64_t)r0 * (idx % m); },
                  [&](int idx) { return L.A + idx; });  // dense, pitch m
    __syncthreads();
    block_householder_qr(L.A, m, q, L.Rm, L.tau, L.colsc);
    const int p = min(m, q);
    for (int idx = threadIdx.x; idx < m * q; idx += blockDim.x) {
      const int i = idx % m, a2 = idx / m;
      core[a2 + (int64_t)r0 * i] = (a2 < p) ? L.A[idx] : 0.f;
    }
  }
  __syncthreads();
  // G_{k-1}^L <- G_{k-1}^L R^T (nrows_prev x r0, column-major), staged through the free A region
  const int64_t cap = (int64_t)L.lda * q;
  const int rows_per = (int)(cap / r0 > 1 ? cap / r0 : 1);
  for (int t0 = 0; t0 < nrows_prev; t0 += rows_per) {
    const int nr = min(rows_per, nrows_prev - t0);
    stage_batched(nr * r0, [&](int idx) { return prev + t0 + (idx % nr) + (int64_t)nrows_prev * (idx / nr); },
                  [&](int idx) { return L.A + idx; });  // A[a2 * nr + tt]
    __syncthreads();
    for (int idx = threadIdx.x; idx < nr * r0; idx += blockDim.x) {
      const int b = idx / nr, tt = idx - b * nr;
      float acc = 0.f;
      for (int a2 = b; a2 < r0; ++a2) acc = fmaf(L.A[a2 * nr + tt], L.Rm[b * q + a2], acc);  // (G R^T)[t, b]
      prev[t0 + tt + (int64_t)nrows_prev * b] = acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// CholeskyQR2 with rows in registers, for q <= 16 columns (Q = q rounded up to 4, 8, 12 or 16),
// 256 threads. A (m x Q, row-major, pitch QP) is in shared memory; thread t owns rows t, t + 256,
// ... Per pass: every thread sums the outer products a a^T of its rows (Q (Q+1) / 2 packed
// lower-triangle values in registers); each warp folds its 32 copies with a reduce-scatter of
// shuffles (each step halves the values a lane holds), the 8 warp sums are added in a fixed
// order; every thread then factors W = L L^T itself (FP32 Cholesky, so no further barrier) and
// replaces each of its rows a by the solution x of x L^T = a. Padded columns (q <= j < Q) are
// zero and get a unit pivot, so they stay zero. A pivot <= 1e-6 times the largest diagonal entry
// of W (condition number above ~1e3, rank deficiency) returns false: the caller falls back to
// Householder. On success Rm (q x q row-major) holds R = L_2^T L_1^T.

constexpr int QR_T = 256;

template <int Q>
struct QrShape {
  static constexpr int QP = (Q % 8 == 0) ? Q + 4 : Q;  // row pitch: conflict-free 16-byte loads
  static constexpr int V = Q * (Q + 1) / 2;            // packed lower triangle, p = i (i+1)/2 + j
};

// Sum v[0..V) over the 32 lanes of a warp; on return lane `lane` holds the sums of the packed
// indices base + k, k < kept (written to out[base + k] for base + k < V).
// One step of the fold: N values per lane become H = (N + 1) / 2; a lane with the OFF bit set
// keeps the upper half (and adds H to its base index), its partner the lower half. `cnt` counts
// the leading slots that hold real indices; the rest are zero padding (odd N), which must not be
// stored: their index belongs to another lane.
template <int N, int OFF, int V>
__device__ __forceinline__ void warp_fold_step(float (&v)[V], int lane, int& base, int& cnt) {
  constexpr int H = (N + 1) / 2;
  const bool up = (lane & OFF) != 0;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float lo = v[k];
    const float hi = (H + k < N) ? v[H + k] : 0.f;
    const float got = __shfl_xor_sync(0xffffffffu, up ? lo : hi, OFF);
    v[k] = (up ? hi : lo) + got;
  }
  if (up) {
    base += H;
    cnt = max(cnt - H, 0);
  } else {
    cnt = min(cnt, H);
  }
}

// Sum v[0..V) over the 32 lanes of a warp (a reduce-scatter: 5 steps, each halving the values a
// lane holds) and store the sums to out[0..V): lane `lane` ends with indices base + k.
template <int V>
__device__ __forceinline__ void warp_fold_store(float (&v)[V], float* out) {
  const int lane = threadIdx.x & 31;
  int base = 0, cnt = V;
  constexpr int N1 = (V + 1) / 2, N2 = (N1 + 1) / 2, N3 = (N2 + 1) / 2, N4 = (N3 + 1) / 2, N5 = (N4 + 1) / 2;
  warp_fold_step<V, 16>(v, lane, base, cnt);
  warp_fold_step<N1, 8>(v, lane, base, cnt);
  warp_fold_step<N2, 4>(v, lane, base, cnt);
  warp_fold_step<N3, 2>(v, lane, base, cnt);
  warp_fold_step<N4, 1>(v, lane, base, cnt);
#pragma unroll
  for (int k = 0; k < N5; ++k)
    if (k < cnt) out[base + k] = v[k];
}

template <int Q>
__device__ __forceinline__ void qr_load_row(const float* As, int r, float (&a)[Q]) {
  const float4* p = reinterpret_cast<const float4*>(As + (size_t)r * QrShape<Q>::QP);
#pragma unroll
  for (int u = 0; u < Q / 4; ++u) {
    const float4 x = p[u];
    a[4 * u] = x.x;
    a[4 * u + 1] = x.y;
    a[4 * u + 2] = x.z;
    a[4 * u + 3] = x.w;
  }
}

template <int Q>
__device__ __forceinline__ void qr_store_row(float* As, int r, const float (&a)[Q]) {
  float4* p = reinterpret_cast<float4*>(As + (size_t)r * QrShape<Q>::QP);
#pragma unroll
  for (int u = 0; u < Q / 4; ++u) p[u] = make_float4(a[4 * u], a[4 * u + 1], a[4 * u + 2], a[4 * u + 3]);
}

// Shared scratch of cholqr2_rows: part (8 x V) | Wsum (V) | Ls (2 x V)
template <int Q>
__device__ bool cholqr2_rows(float* As, int m, int q, float* scratch, float* Rm) {
  constexpr int V = QrShape<Q>::V;
  float* part = scratch;
  float* Wsum = part + 8 * V;
  float* Ls = Wsum + V;
  const int t = threadIdx.x, warp = t >> 5;
  for (int pass = 0; pass < 2; ++pass) {
    float acc[V];
#pragma unroll
    for (int p = 0; p < V; ++p) acc[p] = 0.f;
    for (int r = t; r < m; r += QR_T) {
      float a[Q];
      qr_load_row<Q>(As, r, a);
#pragma unroll
      for (int i = 0; i < Q; ++i) {  // row i of the packed triangle: pairs (j, j+1) per fma.rn.f32x2
        const int pi = i * (i + 1) / 2;
        const float2 ai = make_float2(a[i], a[i]);
#pragma unroll
        for (int j = 0; j + 1 <= i; j += 2) {
          const float2 d = tt_ffma2(ai, make_float2(a[j], a[j + 1]), make_float2(acc[pi + j], acc[pi + j + 1]));
          acc[pi + j] = d.x;
          acc[pi + j + 1] = d.y;
        }
        if ((i & 1) == 0) acc[pi + i] = fmaf(a[i], a[i], acc[pi + i]);  // odd count: the diagonal alone
      }
    }
    warp_fold_store<V>(acc, part + warp * V);
    __syncthreads();
    if (t < V) {
      float sum = 0.f;
#pragma unroll
      for (int u = 0; u < QR_T / 32; ++u) sum += part[u * V + t];
      Wsum[t] = sum;
    }
    __syncthreads();
    float L[V], dinv[Q];
    float dmax = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) dmax = fmaxf(dmax, i < q ? Wsum[i * (i + 1) / 2 + i] : 0.f);
    bool ok = dmax > 0.f && isfinite(dmax);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const int pj = j * (j + 1) / 2;
      float d = (j < q) ? Wsum[pj + j] : 1.f;
#pragma unroll
      for (int l = 0; l < Q; ++l)
        if (l < j) d = fmaf(-L[pj + l], L[pj + l], d);
      if (j < q && (!(d > 1e-6f * dmax) || !isfinite(d))) ok = false;
      const float ljj = sqrtf(fmaxf(d, 1e-30f));
      L[pj + j] = ljj;
      dinv[j] = 1.f / ljj;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (i <= j) continue;
        const int pi = i * (i + 1) / 2;
        float v = (i < q && j < q) ? Wsum[pi + j] : 0.f;
#pragma unroll
        for (int l = 0; l < Q; ++l)
          if (l < j) v = fmaf(-L[pi + l], L[pj + l], v);
        L[pi + j] = v * dinv[j];
      }
    }
    if (!ok) return false;  // the same values in every thread: a uniform exit
    for (int r = t; r < m; r += QR_T) {
      float a[Q];
      qr_load_row<Q>(As, r, a);
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const int pj = j * (j + 1) / 2;
        float v = a[j];
#pragma unroll
        for (int l = 0; l < Q; ++l)
          if (l < j) v = fmaf(-a[l], L[pj + l], v);
        a[j] = v * dinv[j];
      }
      qr_store_row<Q>(As, r, a);
    }
    if (t == 0) {
#pragma unroll
      for (int p = 0; p < V; ++p) Ls[pass * V + p] = L[p];
    }
  }
  __syncthreads();
  // R = R_2 R_1, R_p = L_p^T: R[i][j] = sum_{l = i..j} L_2[l][i] L_1[j][l]
  for (int e = t; e < q * q; e += QR_T) {
    const int i = e / q, j = e - i * q;
    float acc = 0.f;
    for (int l = i; l <= j; ++l) acc = fmaf(Ls[V + l * (l + 1) / 2 + i], Ls[j * (j + 1) / 2 + l], acc);
    Rm[e] = acc;
  }
  __syncthreads();
  return true;
}


// Shared-memory layout of k_qr_left_rows / k_lq_right_rows (floats): As (m x QP) | NX (the
// neighbour core, when prefetched) | scratch (8 V + 3 V) | Rm (q x q) | tau (Q) | colsc (4)
template <int Q>
static size_t qr_rows_smem(int m, int64_t nx) {
  constexpr int V = QrShape<Q>::V;
  return sizeof(float) * ((size_t)m * QrShape<Q>::QP + (size_t)nx + 11 * V + Q * Q + Q + 4);
}

// G_k^L (m = r0 n rows, q = r1 <= Q cols) = Q R; G_k <- Q; G_{k+1} <- R G_{k+1}^R. The
// neighbour G_{k+1} (r1 x ncols_next) is prefetched with cp.async while the QR runs when
// `prefetch` is set (the launcher reserved room for it).
template <int Q>
__global__ void __launch_bounds__(QR_T, 1) k_qr_left_rows(float* core, float* next, int r0, int n, int r1,
                                                      int ncols_next, int prefetch, const int* status) {
  extern __shared__ __align__(16) float sm[];
  constexpr int QP = QrShape<Q>::QP, V = QrShape<Q>::V;
  if (*status != 0) return;
  const int m = r0 * n, q = r1, t = threadIdx.x;
  const int64_t nx = prefetch ? (int64_t)r1 * ncols_next : 0;
  float* As = sm;
  float* NX = As + (size_t)m * QP;
  float* scratch = NX + nx;
  float* Rm = scratch + 11 * V;
  float* tau = Rm + Q * Q;
  float* colsc = tau + Q;
  bool ok = false;
  if (m >= q) {
    for (int j = 0; j < q; ++j)  // G_k^L column-major -> rows
      for (int r = t; r < m; r += QR_T) cp_async4(As + (size_t)r * QP + j, core + (size_t)j * m + r);
  }
  cp_async_commit();  // group 0: the matrix (empty when m < q)
  for (int64_t idx = t; idx < nx; idx += QR_T) cp_async4(NX + idx, next + idx);
  cp_async_commit();  // group 1: the neighbour core
  if (m >= q) {
    for (int r = t; r < m; r += QR_T)  // zero padding columns
#pragma unroll
      for (int j = 0; j < QP; ++j)
        if (j >= q) As[(size_t)r * QP + j] = 0.f;
    cp_async_wait<1>();
    __syncthreads();
    ok = cholqr2_rows<Q>(As, m, q, scratch, Rm);
    if (ok)
      for (int j = 0; j < q; ++j)
        for (int r = t; r < m; r += QR_T) core[(size_t)j * m + r] = As[(size_t)r * QP + j];
  }
  cp_async_wait<0>();
  __syncthreads();
  if (!ok) {  // Householder on a dense column-major copy (pitch m)
    stage_batched(m * q, [&](int idx) { return core + idx; }, [&](int idx) { return As + idx; });
    __syncthreads();
    block_householder_qr(As, m, q, Rm, tau, colsc);
    const int p = min(m, q);
    for (int idx = t; idx < m * q; idx += QR_T) core[idx] = (idx / m < p) ? As[idx] : 0.f;
    __syncthreads();
  }
  // G_{k+1}^R <- R G_{k+1}^R (r1 x ncols_next, column-major): one thread per column, the upper
  // triangle of R in registers
  float R[QrShape<Q>::V];
#pragma unroll
  for (int a2 = 0; a2 < Q; ++a2)
#pragma unroll
    for (int b = 0; b < Q; ++b)
      if (b >= a2) R[b * (b + 1) / 2 + a2] = (a2 < q && b < q) ? Rm[a2 * q + b] : 0.f;
  // with the neighbour prefetched, each thread overwrites its own columns of the shared copy and
  // the CTA then stores the copy with coalesced writes (columns are r1 floats apart)
  float* dstc = prefetch ? NX : next;
  for (int cc = t; cc < ncols_next; cc += QR_T) {
    float x[Q];
    const float* src = prefetch ? NX + (size_t)cc * r1 : next + (size_t)cc * r1;
#pragma unroll
    for (int b = 0; b < Q; ++b) x[b] = b < q ? src[b] : 0.f;
#pragma unroll
    for (int a2 = 0; a2 < Q; ++a2) {
      if (a2 >= q) break;
      float acc = 0.f;
#pragma unroll
      for (int b = 0; b < Q; ++b)
        if (b >= a2) acc = fmaf(R[b * (b + 1) / 2 + a2], x[b], acc);
      dstc[(size_t)cc * r1 + a2] = acc;
    }
  }
  if (prefetch) {
    __syncthreads();
    const int64_t nx = (int64_t)r1 * ncols_next;
    for (int64_t idx = t; idx < nx; idx += QR_T) next[idx] = NX[idx];
  }
}

// (G_k^R)^T (m = n r1 rows, q = r0 <= Q cols) = Q R; G_k^R <- Q^T; G_{k-1}^L <- G_{k-1}^L R^T.
// The neighbour G_{k-1} (nrows_prev x r0) is prefetched as in k_qr_left_rows.
template <int Q>
__device__ void lq_right_body(float* sm, float* prev, float* core, int r0, int n, int r1, int nrows_prev,
                              int prefetch) {
  constexpr int QP = QrShape<Q>::QP, V = QrShape<Q>::V;
  const int m = n * r1, q = r0, t = threadIdx.x;
  const int64_t nx = prefetch ? (int64_t)nrows_prev * r0 : 0;
  float* As = sm;
  float* NX = As + (size_t)m * QP;
  float* scratch = NX + nx;
  float* Rm = scratch + 11 * V;
  float* tau = Rm + Q * Q;
  float* colsc = tau + Q;
  bool ok = false;
  if (m >= q) {
    for (int i = t; i < m; i += QR_T)  // row i of (G_k^R)^T = core[q i .. q i + q)
#pragma unroll
      for (int a2 = 0; a2 < Q; ++a2)
        if (a2 < q) cp_async4(As + (size_t)i * QP + a2, core + (size_t)i * q + a2);
  }
  cp_async_commit();  // group 0: the matrix (empty when m < q)
  for (int64_t idx = t; idx < nx; idx += QR_T) cp_async4(NX + idx, prev + idx);
  cp_async_commit();  // group 1: the neighbour core
  if (m >= q) {
    for (int r = t; r < m; r += QR_T)  // zero padding columns
#pragma unroll
      for (int j = 0; j < QP; ++j)
        if (j >= q) As[(size_t)r * QP + j] = 0.f;
    cp_async_wait<1>();
    __syncthreads();
    ok = cholqr2_rows<Q>(As, m, q, scratch, Rm);
    if (ok)
      for (int i = t; i < m; i += QR_T)
#pragma unroll
        for (int a2 = 0; a2 < Q; ++a2)
          if (a2 < q) core[(size_t)i * q + a2] = As[(size_t)i * QP + a2];
  }
  cp_async_wait<0>();
  __syncthreads();
  if (!ok) {
    stage_batched(m * q, [&](int idx) { return core + (idx / m) + (int64_t)r0 * (idx % m); },
                  [&](int idx) { return As + idx; });  // dense, pitch m
    __syncthreads();
    block_householder_qr(As, m, q, Rm, tau, colsc);
    const int p = min(m, q);
    for (int idx = t; idx < m * q; idx += QR_T) {
      const int i = idx % m, a2 = idx / m;
      core[a2 + (int64_t)r0 * i] = (a2 < p) ? As[idx] : 0.f;
    }
    __syncthreads();
  }
  // G_{k-1}^L <- G_{k-1}^L R^T (nrows_prev x r0, column-major): one thread per row, the upper
  // triangle of R in registers
  float R[QrShape<Q>::V];
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int a2 = 0; a2 < Q; ++a2)
      if (a2 >= b) R[a2 * (a2 + 1) / 2 + b] = (a2 < q && b < q) ? Rm[b * q + a2] : 0.f;
  for (int tt = t; tt < nrows_prev; tt += QR_T) {
    float x[Q];
    const float* src = prefetch ? NX : prev;
#pragma unroll
    for (int a2 = 0; a2 < Q; ++a2) x[a2] = a2 < q ? src[tt + (size_t)nrows_prev * a2] : 0.f;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      if (b >= q) break;
      float acc = 0.f;
#pragma unroll
      for (int a2 = 0; a2 < Q; ++a2)
        if (a2 >= b) acc = fmaf(x[a2], R[a2 * (a2 + 1) / 2 + b], acc);
      prev[tt + (size_t)nrows_prev * b] = acc;
    }
  }
}

template <int Q>
__global__ void __launch_bounds__(QR_T, 1) k_lq_right_rows(float* prev, float* core, int r0, int n, int r1,
                                                       int nrows_prev, int prefetch, const int* status) {
  extern __shared__ __align__(16) float sm[];
  if (*status != 0) return;
  lq_right_body<Q>(sm, prev, core, r0, n, r1, nrows_prev, prefetch);
}

// The right-to-left orthogonalisation of Algorithm 1 (k = d-1 .. 1) in one CTA: each step is the
// body of k_lq_right_rows on the cores left by the previous one (a barrier between the steps).
struct LqSweepArgs {
  float* core[TT_MAX_D];
  int r[TT_MAX_D + 1];
  int n[TT_MAX_D];
  int d;
  int prefetch;
};

template <int Q>
__global__ void __launch_bounds__(QR_T, 1) k_lq_sweep_rows(LqSweepArgs a, const int* status) {
  extern __shared__ __align__(16) float sm[];
  if (*status != 0) return;
  for (int k = a.d - 1; k >= 1; --k) {
    lq_right_body<Q>(sm, a.core[k - 1], a.core[k], a.r[k], a.n[k], a.r[k + 1], a.r[k - 1] * a.n[k - 1], a.prefetch);
    __syncthreads();
  }
}

template <int Q>
static bool launch_lq_sweep_q(tt_ctx* c, float* const* cores, cudaError_t* err) {
  LqSweepArgs a;
  a.d = c->d;
  size_t with = 0, without = 0;
  for (int k = 0; k < c->d; ++k) {
    a.core[k] = cores[k];
    a.n[k] = (int)c->n[k];
  }
  for (int k = 0; k <= c->d; ++k) a.r[k] = c->r[k];
  for (int k = c->d - 1; k >= 1; --k) {
    const int m = (int)c->n[k] * c->r[k + 1];
    const int64_t nx = (int64_t)c->r[k - 1] * c->n[k - 1] * c->r[k];
    with = std::max(with, qr_rows_smem<Q>(m, nx));
    without = std::max(without, qr_rows_smem<Q>(m, 0));
  }
  a.prefetch = with <= 200 * 1024;
  const size_t smem = a.prefetch ? with : without;
  if (smem > 200 * 1024) return false;
  *err = cudaFuncSetAttribute(k_lq_sweep_rows<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (*err != cudaSuccess) return true;
  k_lq_sweep_rows<Q><<<1, QR_T, smem, c->stream>>>(a, c->d_status);
  *err = cudaGetLastError();
  return true;
}

// Launch a rows kernel for q <= 16 when its shared memory fits; false = use the generic kernels.
template <int Q, bool LEFT>
static bool launch_qr_rows_q(float* a0, float* a1, int r0, int n, int r1, int nbr, int m, int64_t nx,
                             const int* status, cudaStream_t st, cudaError_t* err) {
  size_t smem = qr_rows_smem<Q>(m, nx);
  int prefetch = 1;
  if (smem > 200 * 1024) {
    prefetch = 0;
    smem = qr_rows_smem<Q>(m, 0);
    if (smem > 200 * 1024) return false;
  }
  auto kern = LEFT ? k_qr_left_rows<Q> : k_lq_right_rows<Q>;
  *err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (*err != cudaSuccess) return true;
  kern<<<1, QR_T, smem, st>>>(a0, a1, r0, n, r1, nbr, prefetch, status);
  *err = cudaGetLastError();
  return true;
}

template <bool LEFT>
static bool launch_qr_rows(float* a0, float* a1, int r0, int n, int r1, int nbr, const int* status,
                           cudaStream_t st, cudaError_t* err) {
  const int q = LEFT ? r1 : r0, m = LEFT ? r0 * n : n * r1;
  const int64_t nx = (int64_t)nbr * q;
  if (q <= 4) return launch_qr_rows_q<4, LEFT>(a0, a1, r0, n, r1, nbr, m, nx, status, st, err);
  if (q <= 8) return launch_qr_rows_q<8, LEFT>(a0, a1, r0, n, r1, nbr, m, nx, status, st, err);
  if (q <= 12) return launch_qr_rows_q<12, LEFT>(a0, a1, r0, n, r1, nbr, m, nx, status, st, err);
  if (q <= 16) return launch_qr_rows_q<16, LEFT>(a0, a1, r0, n, r1, nbr, m, nx, status, st, err);
  return false;
}

static size_t qr_smem(int m, int q, int use_chol) {
  const size_t lda = use_chol ? (size_t)(m | 1) : (size_t)m;
  return sizeof(float) * (lda * q + (size_t)q * q + q + 4 + (size_t)std::max(q * q, 512) + (size_t)q * q);
}

int tt_launch_qr_left(tt_ctx* c, float* core_k, float* core_k1, int k) {
  int r0 = c->r[k], n = (int)c->n[k], r1 = c->r[k + 1];
  int ncols = (int)(c->n[k + 1] * c->r[k + 2]);
  cudaError_t e = cudaSuccess;
  if (launch_qr_rows<true>(core_k, core_k1, r0, n, r1, ncols, c->d_status, c->stream, &e)) {
    TT_CUDA(c, e);
    TT_LAUNCH(c, "k_qr_left_rows");
    return TT_OK;
  }
  const int use_chol = (r1 <= 32) ? 1 : 0;
  size_t smem = qr_smem(r0 * n, r1, use_chol);
  TT_CUDA(c, cudaFuncSetAttribute(k_qr_left, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_qr_left<<<1, 512, smem, c->stream>>>(core_k, core_k1, r0, n, r1, ncols, use_chol, c->d_status);
  TT_LAUNCH(c, "k_qr_left");
  return TT_OK;
}

// Right-to-left orthogonalisation of all cores: one launch when every rank r_1 .. r_{d-1} is at
// most 16 (and shared memory allows), else one launch per step.
int tt_launch_lq_sweep(tt_ctx* c, float* const* cores) {
  int q = 1;
  for (int k = 1; k < c->d; ++k) q = std::max(q, c->r[k]);
  cudaError_t e = cudaSuccess;
  bool done = false;
  if (c->d >= 2 && q <= 16) {
    if (q <= 4)
      done = launch_lq_sweep_q<4>(c, cores, &e);
    else if (q <= 8)
      done = launch_lq_sweep_q<8>(c, cores, &e);
    else if (q <= 12)
      done = launch_lq_sweep_q<12>(c, cores, &e);
    else
      done = launch_lq_sweep_q<16>(c, cores, &e);
  }
  if (done) {
    TT_CUDA(c, e);
    TT_LAUNCH(c, "k_lq_sweep_rows");
    return TT_OK;
  }
  for (int kk = c->d - 1; kk >= 1; --kk) TT_TRY(tt_launch_lq_right(c, cores[kk - 1], cores[kk], kk));
  return TT_OK;
}

int tt_launch_lq_right(tt_ctx* c, float* core_km1, float* core_k, int k) {
  int r0 = c->r[k], n = (int)c->n[k], r1 = c->r[k + 1];
  int nrows = (int)(c->r[k - 1] * c->n[k - 1]);
  cudaError_t e = cudaSuccess;
  if (launch_qr_rows<false>(core_km1, core_k, r0, n, r1, nrows, c->d_status, c->stream, &e)) {
    TT_CUDA(c, e);
    TT_LAUNCH(c, "k_lq_right_rows");
    return TT_OK;
  }
  const int use_chol = (r0 <= 32) ? 1 : 0;
  size_t smem = qr_smem(n * r1, r0, use_chol);
  TT_CUDA(c, cudaFuncSetAttribute(k_lq_right, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_lq_right<<<1, 512, smem, c->stream>>>(core_km1, core_k, r0, n, r1, nrows, use_chol, c->d_status);
  TT_LAUNCH(c, "k_lq_right");
  return TT_OK;
}

// ---------------------------------------------------------------------------------------------
// relative error. The tensor is walked in slabs of modes (0, 1) (contiguous n_0 x n_1 blocks):
// for the slab's tail indices (i_2, .., i_{d-1}) one warp forms u = G_2(i_2) ... G_{d-1}(i_{d-1})
// (r_2 entries), the CTA forms W(:, i_1) = G_1(:, i_1, :) u for the slab's i_1 range, and every
// entry is then reconstructed as G_0(0, i_0, :) . W(:, i_1) and compared with A, reading A in
// order. Work items are (slab, i_1-chunk) so that order-2 tensors still spread over all SMs.

struct ErrArgs {
  const void* A;
  const float* scales;
  const float* core[TT_MAX_D];
  int64_t n[TT_MAX_D];
  int r[TT_MAX_D + 1];
  int d;
  int64_t slabs;      // prod_{s>=2} n_s
  int i1chunk;        // i_1 values per work item
  int nchunks;        // ceil(n_1 / i1chunk)
  int g0_in_smem;     // G_0 (n_0 x r_1) staged in shared memory
  double* acc;        // [0] += ||A - [[G]]||^2, [1] += ||A||^2
  double* part;       // deterministic mode: CTA b stores its two sums at part[2 b] (no atomics)
};

template <int DT>
__device__ __forceinline__ float err_elem(const void* A, int64_t idx) {
  if constexpr (DT == TT_F64) return (float)__ldg((const double*)A + idx);
  if constexpr (DT == TT_F32) return __ldg((const float*)A + idx);
  if constexpr (DT == TT_BF16) return __uint_as_float(((uint32_t)__ldg((const unsigned short*)A + idx)) << 16);
  if constexpr (DT == TT_FP8E4M3) return tt_e4m3_to_float(__ldg((const unsigned char*)A + idx));
  return 0.f;
}

// four consecutive entries starting at a multiple of 4 (vector load in the storage type)
template <int DT>
__device__ __forceinline__ void err_load4(const void* A, int64_t idx, float* x) {
  if constexpr (DT == TT_F32) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(A) + idx / 4);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else if constexpr (DT == TT_F64) {
    const double2 v0 = __ldg(reinterpret_cast<const double2*>(A) + idx / 2);
    const double2 v1 = __ldg(reinterpret_cast<const double2*>(A) + idx / 2 + 1);
    x[0] = (float)v0.x; x[1] = (float)v0.y; x[2] = (float)v1.x; x[3] = (float)v1.y;
  } else if constexpr (DT == TT_BF16) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(A) + idx / 4);
    x[0] = __uint_as_float(v.x << 16); x[1] = __uint_as_float(v.x & 0xFFFF0000u);
    x[2] = __uint_as_float(v.y << 16); x[3] = __uint_as_float(v.y & 0xFFFF0000u);
  } else {
    const uint32_t v = __ldg(reinterpret_cast<const uint32_t*>(A) + idx / 4);
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = tt_e4m3_to_float(v >> (8 * c));
  }
}

template <int DT>
__global__ void __launch_bounds__(256) k_rel_error(ErrArgs a) {
  extern __shared__ float sm[];
  __shared__ float ubuf[2][TT_MAX_S];
  __shared__ double red[2][8];
  const int n0 = (int)a.n[0], n1 = (int)a.n[1], r1 = a.r[1], r2 = a.r[2];
  const int WP = a.i1chunk;                        // W pitch (multiple of 4)
  float* W = sm;                                   // r1 x WP
  float* G0 = sm + (size_t)r1 * WP;                // r1 x n0 (G_0(0, i0, al) at al * n0 + i0)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < n0 * r1; i += blockDim.x) G0[i] = a.core[0][i];
  double e2 = 0.0, x2 = 0.0;
  const int64_t items = a.slabs * a.nchunks;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t t = it / a.nchunks;
    const int ch = (int)(it - t * a.nchunks);
    const int j0 = ch * a.i1chunk, j1 = min(n1, j0 + a.i1chunk);
    if (warp == 0) {  // u = G_2(i_2) ... G_{d-1}(i_{d-1}), or [1] when d == 2
      int64_t idx[TT_MAX_D];
      int64_t rem = t;
      for (int s2 = 2; s2 < a.d; ++s2) {
        idx[s2] = rem % a.n[s2];
        rem /= a.n[s2];
      }
      float* u = ubuf[0];
      float* un = ubuf[1];
      if (a.d == 2) {
        if (lane == 0) u[0] = 1.f;
      } else {
        const int s2 = a.d - 1, ra = a.r[s2];
        for (int al = lane; al < ra; al += 32) u[al] = a.core[s2][al + (int64_t)ra * idx[s2]];
      }
      __syncwarp();
      for (int s2 = a.d - 2; s2 >= 2; --s2) {
        const int ra = a.r[s2], rb = a.r[s2 + 1];
        const float* G = a.core[s2] + (int64_t)ra * idx[s2];
        const int64_t bstride = (int64_t)ra * a.n[s2];
        for (int al = lane; al < ra; al += 32) {
          float acc = 0.f;
          for (int be = 0; be < rb; ++be) acc = fmaf(G[al + bstride * be], u[be], acc);
          un[al] = acc;
        }
        __syncwarp();
        for (int al = lane; al < ra; al += 32) u[al] = un[al];
        __syncwarp();
      }
    }
    __syncthreads();
    // W(al, i1) = sum_be G_1(al, i1, be) u(be), zero-padded to a multiple of 4 columns
    const float* g1 = a.core[1];
    const int wcols = (j1 - j0 + 3) & ~3;
    for (int q = threadIdx.x; q < r1 * wcols; q += blockDim.x) {
      const int al = q / wcols, c = q - al * wcols, i1 = j0 + c;
      float acc = 0.f;
      if (i1 < j1)
        for (int be = 0; be < r2; ++be) acc = fmaf(g1[al + (int64_t)r1 * (i1 + (int64_t)n1 * be)], ubuf[0][be], acc);
      W[(size_t)al * WP + c] = acc;
    }
    __syncthreads();
    // tiles of 4 consecutive i0 for one i1 (when n0 % 4 == 0): one vector load of A (issued before
    // the reconstruction so its latency overlaps the FMAs), one 16-byte G_0 load and one broadcast
    // W load per rank index feed 4 FMAs. Otherwise tiles of 4 consecutive i1 for one i0.
    const int64_t base = t * (int64_t)n0 * n1 + (int64_t)j0 * n0;
    float fe = 0.f, fa = 0.f;
    if ((n0 & 3) == 0) {
      const int q4 = n0 >> 2;
      const int tiles = q4 * (j1 - j0);
      constexpr int UT = 4;  // tiles per thread in flight
      for (int qb = threadIdx.x; qb < tiles; qb += UT * blockDim.x) {
        float x[UT][4];
        int i1s[UT], i0s[UT];
#pragma unroll
        for (int u = 0; u < UT; ++u) {
          const int q = qb + u * blockDim.x;
          i1s[u] = q / q4;
          i0s[u] = (q - i1s[u] * q4) * 4;
          if (q < tiles)
            err_load4<DT>(a.A, base + (int64_t)i1s[u] * n0 + i0s[u], x[u]);
        }
#pragma unroll
        for (int u = 0; u < UT; ++u) {
          if (qb + u * blockDim.x >= tiles) break;
          const int i1 = i1s[u], i0 = i0s[u];
          float r4[4] = {0.f, 0.f, 0.f, 0.f};
          for (int al = 0; al < r1; ++al) {
            const float4 g4 = *reinterpret_cast<const float4*>(G0 + al * n0 + i0);
            const float w = W[(size_t)al * WP + i1];
            r4[0] = fmaf(g4.x, w, r4[0]);
            r4[1] = fmaf(g4.y, w, r4[1]);
            r4[2] = fmaf(g4.z, w, r4[2]);
            r4[3] = fmaf(g4.w, w, r4[3]);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float xv = a.scales ? x[u][c] * __ldg(a.scales + i0 + c) : x[u][c];
            const float dl = xv - r4[c];
            fe = fmaf(dl, dl, fe);
            fa = fmaf(xv, xv, fa);
          }
        }
      }
    } else {
      const int ngroups = wcols >> 2;
      const int tiles = ngroups * n0;
      for (int q = threadIdx.x; q < tiles; q += blockDim.x) {
        const int gq = q / n0, i0 = q - gq * n0;
        float r4[4] = {0.f, 0.f, 0.f, 0.f};
        const float* wp = W + 4 * gq;
        for (int al = 0; al < r1; ++al) {
          const float g = G0[al * n0 + i0];
          const float4 w4 = *reinterpret_cast<const float4*>(wp + (size_t)al * WP);
          r4[0] = fmaf(g, w4.x, r4[0]);
          r4[1] = fmaf(g, w4.y, r4[1]);
          r4[2] = fmaf(g, w4.z, r4[2]);
          r4[3] = fmaf(g, w4.w, r4[3]);
        }
        const float sc = a.scales ? __ldg(a.scales + i0) : 1.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i1 = 4 * gq + c;
          if (j0 + i1 < j1) {
            const float x = err_elem<DT>(a.A, base + (int64_t)i1 * n0 + i0) * sc;
            const float dl = x - r4[c];
            fe = fmaf(dl, dl, fe);
            fa = fmaf(x, x, fa);
          }
        }
      }
    }
    e2 += fe;
    x2 += fa;
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
  }
  if (lane == 0) {
    red[0][warp] = e2;
    red[1][warp] = x2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t1 += red[0][w];
      t2 += red[1][w];
    }
    if (a.part) {
      a.part[2 * blockIdx.x] = t1;
      a.part[2 * blockIdx.x + 1] = t2;
    } else {
      atomicAdd(a.acc, t1);
      atomicAdd(a.acc + 1, t2);
    }
  }
}

// Right interface of every mode-0 fibre f = i_1 + n_1 t (t = slab index over modes 2..d-1):
// R[f * r1p + al] = (G_1(i_1) u_t)[al], zero for r1 <= al < r1p, with
// u_t = G_2(i_2) ... G_{d-1}(i_{d-1}) (r_2 values; [1] when d == 2). k_slab_u forms u_t (one
// thread per slab), k_rint one output per thread (coalesced writes).
__global__ void __launch_bounds__(256) k_slab_u(ErrArgs a, float* __restrict__ Uo) {
  const int r2 = a.r[2];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.slabs; t += (int64_t)gridDim.x * blockDim.x) {
    float u[TT_MAX_S], un[TT_MAX_S];
    if (a.d == 2) {
      u[0] = 1.f;
    } else {
      int64_t idx[TT_MAX_D];
      int64_t rem = t;
      for (int s2 = 2; s2 < a.d; ++s2) {
        idx[s2] = rem % a.n[s2];
        rem /= a.n[s2];
      }
      const int s2 = a.d - 1, ra = a.r[s2];
      for (int al = 0; al < ra; ++al) u[al] = a.core[s2][al + (int64_t)ra * idx[s2]];
      for (int s3 = a.d - 2; s3 >= 2; --s3) {
        const int rA = a.r[s3], rB = a.r[s3 + 1];
        const float* G = a.core[s3] + (int64_t)rA * idx[s3];
        const int64_t bstride = (int64_t)rA * a.n[s3];
        for (int al = 0; al < rA; ++al) {
          float acc = 0.f;
          for (int be = 0; be < rB; ++be) acc = fmaf(G[al + bstride * be], u[be], acc);
          un[al] = acc;
        }
        for (int al = 0; al < rA; ++al) u[al] = un[al];
      }
    }
    for (int be = 0; be < r2; ++be) Uo[t * r2 + be] = u[be];
  }
}

// The same right interfaces with G_1 in registers: a CTA takes a run of slabs; thread x owns the
// output positions ol = x + blockDim.x k (k < RINT_KP; ol = i_1 r1p + al) of every slab of the
// run and keeps their G_1(al, i_1, :) entries (RB >= r_2 of them) in registers, so each output
// costs r_2 FMAs with u_t broadcast from shared memory; the stores of a slab are contiguous.
// The CTA first forms the u_t of its own slabs, one level (core) at a time with its threads over
// (slab, entry) pairs: entry al of G_s(i_s) u takes r_{s+1} loads issued in batches of eight; the
// vectors pass through shared memory.
constexpr int RINT_KP = 4;
template <int RB>
__global__ void __launch_bounds__(512, 1) k_rint_reg(ErrArgs a, float* __restrict__ R, int r1p, int slabs_per_cta) {
  extern __shared__ float us[];  // slabs_per_cta x r_2, then two slabs_per_cta x max(r_2..r_{d-1}) buffers
  const int n1 = (int)a.n[1], r1 = a.r[1], r2 = a.r[2];
  const int per = n1 * r1p;
  const int64_t t0 = (int64_t)blockIdx.x * slabs_per_cta;
  if (t0 >= a.slabs) return;
  const int nsl = (int)min((int64_t)slabs_per_cta, a.slabs - t0);
  const float* g1 = a.core[1];
  float g[RINT_KP][RB];
#pragma unroll
  for (int k = 0; k < RINT_KP; ++k) {
    const int ol = threadIdx.x + blockDim.x * k;
    const int i1 = ol / r1p, al = ol - i1 * r1p;
    const bool valid = ol < per && al < r1;
#pragma unroll
    for (int be = 0; be < RB; ++be)
      g[k][be] = (valid && be < r2) ? __ldg(g1 + al + r1 * (i1 + n1 * be)) : 0.f;
  }
  if (a.d == 2) {
    for (int sl = threadIdx.x; sl < nsl; sl += blockDim.x) us[sl] = 1.f;
  } else {  // u_t level by level, the CTA's threads over (slab, entry) pairs
    int rmax = 1;
    for (int q = 2; q < a.d; ++q) rmax = max(rmax, a.r[q]);
    float* bufs[2] = {us + slabs_per_cta * r2, us + slabs_per_cta * (r2 + rmax)};
    int64_t stride = 1;  // prod_{2 <= q < s} n_q for the mode s of the level
    for (int q = 2; q < a.d - 1; ++q) stride *= a.n[q];
    const int sl1 = a.d - 1, rl = a.r[sl1];  // the last core: u = G_{d-1}(:, i_{d-1}, 0)
    float* cur = sl1 == 2 ? us : bufs[0];
    const int pc = sl1 == 2 ? r2 : rmax;
    for (int e = threadIdx.x; e < nsl * rl; e += blockDim.x) {
      const int sl = e / rl, al = e - sl * rl;
      const int64_t i = ((t0 + sl) / stride) % a.n[sl1];
      cur[sl * pc + al] = __ldg(a.core[sl1] + al + (int64_t)rl * i);
    }
    int pcur = pc;
    for (int s3 = a.d - 2; s3 >= 2; --s3) {
      __syncthreads();
      stride /= a.n[s3];
      const int rA = a.r[s3], rB = a.r[s3 + 1];
      const int64_t bstride = (int64_t)rA * a.n[s3];
      float* nxt = s3 == 2 ? us : (cur == bufs[0] ? bufs[1] : bufs[0]);
      const int pn = s3 == 2 ? r2 : rmax;
      for (int e = threadIdx.x; e < nsl * rA; e += blockDim.x) {
        const int sl = e / rA, al = e - sl * rA;
        const int64_t i = ((t0 + sl) / stride) % a.n[s3];
        const float* G = a.core[s3] + al + (int64_t)rA * i;
        const float* uc = cur + sl * pcur;
        float acc = 0.f;
        for (int be0 = 0; be0 < rB; be0 += 8) {  // eight loads in flight per batch
          float gv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) gv[q] = be0 + q < rB ? __ldg(G + bstride * (be0 + q)) : 0.f;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (be0 + q < rB) acc = fmaf(gv[q], uc[be0 + q], acc);
        }
        nxt[sl * pn + al] = acc;
      }
      cur = nxt;
      pcur = pn;
    }
  }
  __syncthreads();
  for (int sl = 0; sl < nsl; ++sl) {
    float u[RB];
#pragma unroll
    for (int be = 0; be < RB; ++be) u[be] = be < r2 ? us[sl * r2 + be] : 0.f;
    float* out = R + (t0 + sl) * (int64_t)per;
#pragma unroll
    for (int k = 0; k < RINT_KP; ++k) {
      const int ol = threadIdx.x + blockDim.x * k;
      float acc = 0.f;
#pragma unroll
      for (int be = 0; be < RB; ++be) acc = fmaf(g[k][be], u[be], acc);
      if (ol < per) out[ol] = acc;
    }
  }
}

__global__ void __launch_bounds__(256) k_rint(ErrArgs a, const float* __restrict__ Uv, float* __restrict__ R, int r1p) {
  __shared__ float u[TT_MAX_S];
  const int n1 = (int)a.n[1], r1 = a.r[1], r2 = a.r[2];
  const int per = n1 * r1p;  // outputs of one slab (al fastest: G_1 reads and R writes contiguous)
  const float* g1 = a.core[1];
  for (int64_t t = blockIdx.x; t < a.slabs; t += gridDim.x) {
    for (int be = threadIdx.x; be < r2; be += blockDim.x) u[be] = Uv[t * r2 + be];
    __syncthreads();
    float* out = R + t * (int64_t)per;
    for (int ol = threadIdx.x; ol < per; ol += blockDim.x) {
      const int i1 = ol / r1p, al = ol - i1 * r1p;
      float acc = 0.f;
      if (al < r1)
        for (int be = 0; be < r2; ++be) acc = fmaf(__ldg(g1 + al + r1 * (i1 + n1 * be)), u[be], acc);
      out[ol] = acc;
    }
    __syncthreads();
  }
}

template <int DT>
struct ElemSize {
  static constexpr int value = DT == TT_F64 ? 8 : DT == TT_F32 ? 4 : DT == TT_BF16 ? 2 : 1;
};


// four consecutive entries from shared memory (storage type DT, 4-entry aligned)
template <int DT>
__device__ __forceinline__ void smem_load4(const unsigned char* p, float* x) {
  if constexpr (DT == TT_F32) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else if constexpr (DT == TT_F64) {
    const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 16);
    x[0] = (float)v0.x; x[1] = (float)v0.y; x[2] = (float)v1.x; x[3] = (float)v1.y;
  } else if constexpr (DT == TT_BF16) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    x[0] = __uint_as_float(v.x << 16); x[1] = __uint_as_float(v.x & 0xFFFF0000u);
    x[2] = __uint_as_float(v.y << 16); x[3] = __uint_as_float(v.y & 0xFFFF0000u);
  } else {
    const uint32_t v = *reinterpret_cast<const uint32_t*>(p);
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = tt_e4m3_to_float(v >> (8 * c));
  }
}

constexpr int REL_U = 4;   // fibres per thread per tile (three CTAs per SM at 100-entry FP32 fibres)
constexpr int REL_NS = 3;  // tiles in flight per CTA

__device__ __forceinline__ bool rel_mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
               : "=r"(ok) : "r"(addr), "r"(parity) : "memory");
  return ok != 0;
}
// bounded wait (2 s by %globaltimer) for the completion of phase `parity`
__device__ __forceinline__ bool rel_mbar_wait(uint32_t addr, uint32_t parity) {
  if (rel_mbar_try(addr, parity)) return true;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  do {
    if (rel_mbar_try(addr, parity)) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  } while (t - t0 < 2000000000ull);
  return false;
}
// 1-D bulk copy global -> shared (16-byte aligned, a multiple of 16 bytes), counted on an mbarrier
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

// ||A - [[G]]||^2 and ||A||^2 by streaming A in memory order. A tile is FT = P * REL_U consecutive
// mode-0 fibres (FT * n_0 entries, contiguous) with their rows of R; one thread moves each tile
// into shared memory with two bulk copies (cp.async.bulk, counted on the buffer's mbarrier),
// REL_NS tiles in flight per CTA, while the CTA reduces the oldest one.
// Thread (q, p) owns entries 4q..4q+3 of the tile's fibres p + P u; the reconstruction is
// G_0 (shared, float4 along i_0) times the fibre's R row (shared, float4 broadcast).
// Needs n_0 % 4 == 0 and n_0 <= 1024.
template <int DT>
__global__ void __launch_bounds__(256, 2) k_rel_error_stream(const void* __restrict__ A, const float* __restrict__ scales,
                                                          const float* __restrict__ g0, const float* __restrict__ R,
                                                          int n0, int r1, int r1p, int64_t M0, double* acc,
                                                          double* part) {
  constexpr int ES = ElemSize<DT>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[2][8];
  const int Q = n0 >> 2, P = blockDim.x / Q, FT = P * REL_U;
  float* G0 = reinterpret_cast<float*>(smraw);  // r1p x n0, rows >= r1 zero
  unsigned char* bufA = smraw + (size_t)r1p * n0 * 4;
  const int tileA = FT * n0 * ES;               // bytes (a multiple of 16)
  float* bufR = reinterpret_cast<float*>(bufA + REL_NS * (size_t)tileA);
  const int tileR = FT * r1p;                   // floats
  uint64_t* mb = reinterpret_cast<uint64_t*>(bufR + REL_NS * (size_t)tileR);  // one per buffer
  for (int i = threadIdx.x; i < r1p * n0; i += blockDim.x) G0[i] = i < r1 * n0 ? g0[i] : 0.f;
  const int qi = threadIdx.x % Q, pi = threadIdx.x / Q;
  const bool active = pi < P;
  float sc[4] = {1.f, 1.f, 1.f, 1.f};
  if (scales && active)
    for (int c = 0; c < 4; ++c) sc[c] = __ldg(scales + 4 * qi + c);
  const int64_t ntiles = (M0 + FT - 1) / FT;
  // thread 0: both bulk copies of a tile on the buffer's mbarrier; the bytes of a partial last
  // tile past the last multiple of 16 are copied by plain loads (read after a CTA barrier)
  auto issue = [&](int64_t tile, int b) {
    const int64_t f0 = tile * FT;
    const int nf = (int)min((int64_t)FT, M0 - f0);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(A) + f0 * n0 * ES;
    const uint32_t bytes = (uint32_t)nf * n0 * ES, bulk = bytes & ~15u;
    const uint32_t bytesR = (uint32_t)nf * r1p * 4;
    unsigned char* dA = bufA + (size_t)b * tileA;
    const uint32_t m = (uint32_t)__cvta_generic_to_shared(&mb[b]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(m), "r"(bulk + bytesR) : "memory");
    if (bulk) bulk_copy((uint32_t)__cvta_generic_to_shared(dA), src, bulk, m);
    bulk_copy((uint32_t)__cvta_generic_to_shared(bufR + (size_t)b * tileR), R + f0 * r1p, bytesR, m);
    for (uint32_t t2 = bulk; t2 < bytes; ++t2) dA[t2] = src[t2];
  };
  if (threadIdx.x == 0) {
    for (int i = 0; i < REL_NS; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"((uint32_t)__cvta_generic_to_shared(&mb[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    for (int i = 0; i < REL_NS - 1; ++i)
      if (blockIdx.x + (int64_t)i * gridDim.x < ntiles) issue(blockIdx.x + (int64_t)i * gridDim.x, i);
  }
  __syncthreads();
  double e2 = 0.0, x2 = 0.0;
  bool timed_out = false;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it % REL_NS;
    if (threadIdx.x == 0) {  // tile it + REL_NS - 1 goes into the buffer read in iteration it - 1
      const int64_t nx = tile + (int64_t)(REL_NS - 1) * gridDim.x;
      if (nx < ntiles) issue(nx, (it + REL_NS - 1) % REL_NS);
    }
    if (!rel_mbar_wait((uint32_t)__cvta_generic_to_shared(&mb[b]), (uint32_t)((it / REL_NS) & 1))) timed_out = true;
    const int64_t f0 = tile * FT;
    const unsigned char* tA = bufA + (size_t)b * tileA;
    const float* tR = bufR + (size_t)b * tileR;
    float fe = 0.f, fa = 0.f;
    if (active) {
      // fibres innermost: every G_0 float4 read from shared memory serves REL_U fibres
      // the reconstruction in pairs of entries: one fma.rn.f32x2 per two FMAs
      float x[REL_U][4];
      float2 r2[REL_U][2];
#pragma unroll
      for (int u = 0; u < REL_U; ++u) smem_load4<DT>(tA + ((size_t)(pi + P * u) * n0 + 4 * qi) * ES, x[u]);
      // ranks al0 .. al0 + 3; the first block's first rank starts the sums with a product (r1 >= 1)
      auto ranks = [&](int al0, auto first) {
        float4 w[REL_U];
#pragma unroll
        for (int u = 0; u < REL_U; ++u) w[u] = *reinterpret_cast<const float4*>(tR + (size_t)(pi + P * u) * r1p + al0);
#pragma unroll
        for (int aa = 0; aa < 4; ++aa) {
          if (al0 + aa >= r1) break;  // rows r1 .. r1p - 1 of G_0 are padding (zero)
          const float4 g4 = *reinterpret_cast<const float4*>(G0 + (al0 + aa) * n0 + 4 * qi);
          const float2 glo = make_float2(g4.x, g4.y), ghi = make_float2(g4.z, g4.w);
#pragma unroll
          for (int u = 0; u < REL_U; ++u) {
            const float ww = aa == 0 ? w[u].x : aa == 1 ? w[u].y : aa == 2 ? w[u].z : w[u].w;
            const float2 w2 = make_float2(ww, ww);
            if (decltype(first)::value && aa == 0) {
              r2[u][0] = tt_fmul2(glo, w2);
              r2[u][1] = tt_fmul2(ghi, w2);
            } else {
              r2[u][0] = tt_ffma2(glo, w2, r2[u][0]);
              r2[u][1] = tt_ffma2(ghi, w2, r2[u][1]);
            }
          }
        }
      };
      ranks(0, std::true_type{});
      for (int al0 = 4; al0 < r1p; al0 += 4) ranks(al0, std::false_type{});
      float2 fe2 = make_float2(0.f, 0.f), fa2 = make_float2(0.f, 0.f);
      const bool full = f0 + FT <= M0;  // every fibre of the tile exists (all tiles but the last)
#pragma unroll
      for (int u = 0; u < REL_U; ++u) {
        if (!full && f0 + pi + P * u >= M0) continue;  // past the last fibre (stale buffer entries)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float2 xv = make_float2(x[u][2 * h], x[u][2 * h + 1]);
          if constexpr (DT == TT_FP8E4M3) xv = make_float2(xv.x * sc[2 * h], xv.y * sc[2 * h + 1]);  // slice scales
          const float2 dl = make_float2(xv.x - r2[u][h].x, xv.y - r2[u][h].y);
          fe2 = tt_ffma2(dl, dl, fe2);
          fa2 = tt_ffma2(xv, xv, fa2);
        }
      }
      fe = fe2.x + fe2.y;
      fa = fa2.x + fa2.y;
    }
    e2 += fe;
    x2 += fa;
    __syncthreads();  // buffer b is refilled by the next iteration's issue
  }
  if (timed_out) e2 = __longlong_as_double(0x7ff8000000000000ll);  // a wait gave up: the result reads NaN
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
  }
  if (lane == 0) {
    red[0][warp] = e2;
    red[1][warp] = x2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t1 += red[0][w];
      t2 += red[1][w];
    }
    if (part) {
      part[2 * blockIdx.x] = t1;
      part[2 * blockIdx.x + 1] = t2;
    } else {
      atomicAdd(acc, t1);
      atomicAdd(acc + 1, t2);
    }
  }
}

// shared memory of k_rel_error_stream for this context (0 if the shape does not fit)
static size_t rel_stream_smem(const tt_ctx* c, int es) {
  const int64_t n0 = c->n[0];
  if (n0 % 4 != 0 || n0 > 1024) return 0;
  const int64_t Q = n0 / 4, P = 256 / Q, FT = P * REL_U;
  const size_t bytes = (size_t)c->rint_r1p * n0 * 4 + REL_NS * (size_t)FT * n0 * es +
                       REL_NS * (size_t)FT * c->rint_r1p * 4 + REL_NS * sizeof(uint64_t);
  return bytes <= 200 * 1024 ? bytes : 0;
}

template <int DT>
static int launch_rel_stream(tt_ctx* c, const void* A, const float* scales, const float* g0, size_t smem,
                             double* acc) {
  static bool attr = false;
  if (!attr) {
    TT_CUDA(c, cudaFuncSetAttribute(k_rel_error_stream<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  int per_sm = 0;
  TT_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rel_error_stream<DT>, 256, smem));
  const int sms = tt_sm_count();
  const int64_t M0 = c->N / c->n[0];
  const int64_t Q = c->n[0] / 4, FT = (256 / Q) * REL_U;
  const int64_t ntiles = (M0 + FT - 1) / FT;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)std::max(1, per_sm) * sms));
  double* part = c->det ? c->d_part_err : nullptr;  // at most TT_DET_PARTS CTAs: a few per SM
  k_rel_error_stream<DT><<<blocks, 256, smem, c->stream>>>(A, scales, g0, c->d_rint, (int)c->n[0], c->r[1],
                                                          c->rint_r1p, M0, acc, part);
  TT_LAUNCH(c, "k_rel_error_stream");
  if (part) TT_TRY(tt_launch_sum_partials(c, part, blocks, acc));
  return TT_OK;
}

int tt_launch_rel_error(tt_ctx* c, const void* A, const float* scales, float* const* cores, double* acc) {
  if (!acc) acc = c->d_err_acc;
  ErrArgs a;
  a.A = A;
  a.scales = scales;
  for (int k = 0; k < c->d; ++k) {
    a.core[k] = cores[k];
    a.n[k] = c->n[k];
  }
  for (int k = 0; k <= c->d; ++k) a.r[k] = c->r[k];
  a.d = c->d;
  a.acc = acc;
  a.part = nullptr;
  a.slabs = c->N / (c->n[0] * c->n[1]);
  // i_1 chunk (multiple of 4): W (r1 x chunk) plus G_0 (r1 x n0) within ~200 KB, at most ~16K
  // entries per item, and at least ~4 items per SM overall
  const int64_t g0sz = (int64_t)c->n[0] * c->r[1];
  int64_t chunk = std::max<int64_t>(4, std::min<int64_t>(c->n[1], 16384 / std::max<int64_t>(1, c->n[0])));
  chunk = (chunk + 3) & ~3ll;
  while (chunk > 4 && (int64_t)c->r[1] * chunk + g0sz > 50 * 1024) chunk -= 4;
  while (chunk > 4 && a.slabs * ((c->n[1] + chunk - 1) / chunk) < (int64_t)tt_sm_count() * 4) chunk = ((chunk / 2) + 3) & ~3ll;
  a.i1chunk = (int)chunk;
  a.nchunks = (int)((c->n[1] + chunk - 1) / chunk);
  a.g0_in_smem = 1;
  const size_t smem = sizeof(float) * ((size_t)c->r[1] * a.i1chunk + (size_t)g0sz);
  TT_CUDA(c, cudaMemsetAsync(acc, 0, sizeof(double) * 2, c->stream));
  const int es = c->dtype == TT_F64 ? 8 : c->dtype == TT_F32 ? 4 : c->dtype == TT_BF16 ? 2 : 1;
  const size_t ssm = c->d_rint ? rel_stream_smem(c, es) : 0;
  if (ssm) {  // streaming form: right interfaces first, then one pass over A in memory order
    const int per = (int)c->n[1] * c->rint_r1p;
    const int r2 = c->r[2];
    const int rthreads = ((per + RINT_KP - 1) / RINT_KP + 31) & ~31;
    if (rthreads <= 512 && r2 <= 16) {  // G_1 entries in registers, u_t formed in the same kernel
      const int sms = tt_sm_count();
      // one slab run per SM (one CTA fits per SM: a single wave pays the G_1 and u_t prologue once
      // per SM); a run's u_t and the two level buffers within the default 48 KB of shared memory
      int rmax = 1;
      for (int q = 2; q < c->d; ++q) rmax = std::max(rmax, c->r[q]);
      const int64_t per_slab = r2 + (c->d > 2 ? 2 * rmax : 0);
      const int64_t spc_max = std::max<int64_t>(1, 12 * 1024 / per_slab);
      const int spc = (int)std::min(spc_max, std::max<int64_t>(1, (a.slabs + sms - 1) / sms));
      const int rgrid = (int)((a.slabs + spc - 1) / spc);
      const size_t rsm = sizeof(float) * (size_t)spc * per_slab;
      if (r2 <= 4)
        k_rint_reg<4><<<rgrid, rthreads, rsm, c->stream>>>(a, c->d_rint, c->rint_r1p, spc);
      else if (r2 <= 8)
        k_rint_reg<8><<<rgrid, rthreads, rsm, c->stream>>>(a, c->d_rint, c->rint_r1p, spc);
      else if (r2 <= 12)
        k_rint_reg<12><<<rgrid, rthreads, rsm, c->stream>>>(a, c->d_rint, c->rint_r1p, spc);
      else
        k_rint_reg<16><<<rgrid, rthreads, rsm, c->stream>>>(a, c->d_rint, c->rint_r1p, spc);
      TT_LAUNCH(c, "k_rint_reg");
    } else {
      const int ublocks = (int)std::max<int64_t>(1, std::min<int64_t>((a.slabs + 255) / 256, 4096));
      k_slab_u<<<ublocks, 256, 0, c->stream>>>(a, c->d_slab_u);
      TT_LAUNCH(c, "k_slab_u");
      const int rblocks = (int)std::max<int64_t>(1, std::min<int64_t>(a.slabs, (int64_t)tt_sm_count() * 8));
      k_rint<<<rblocks, 256, 0, c->stream>>>(a, c->d_slab_u, c->d_rint, c->rint_r1p);
      TT_LAUNCH(c, "k_rint");
    }
    switch (c->dtype) {
      case TT_F64: return launch_rel_stream<TT_F64>(c, A, scales, cores[0], ssm, acc);
      case TT_F32: return launch_rel_stream<TT_F32>(c, A, scales, cores[0], ssm, acc);
      case TT_BF16: return launch_rel_stream<TT_BF16>(c, A, scales, cores[0], ssm, acc);
      default: return launch_rel_stream<TT_FP8E4M3>(c, A, scales, cores[0], ssm, acc);
    }
  }
  const int64_t items = a.slabs * a.nchunks;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)tt_sm_count() * 8));
  a.part = c->det ? c->d_part_err : nullptr;  // blocks <= 8 per SM <= TT_DET_PARTS
  switch (c->dtype) {
    case TT_F64:
      TT_CUDA(c, cudaFuncSetAttribute(k_rel_error<TT_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_rel_error<TT_F64><<<blocks, 256, smem, c->stream>>>(a);
      break;
    case TT_F32:
      TT_CUDA(c, cudaFuncSetAttribute(k_rel_error<TT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_rel_error<TT_F32><<<blocks, 256, smem, c->stream>>>(a);
      break;
    case TT_BF16:
      TT_CUDA(c, cudaFuncSetAttribute(k_rel_error<TT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_rel_error<TT_BF16><<<blocks, 256, smem, c->stream>>>(a);
      break;
    default:
      TT_CUDA(c, cudaFuncSetAttribute(k_rel_error<TT_FP8E4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_rel_error<TT_FP8E4M3><<<blocks, 256, smem, c->stream>>>(a);
      break;
  }
  TT_LAUNCH(c, "k_rel_error");
  if (a.part) TT_TRY(tt_launch_sum_partials(c, a.part, blocks, acc));
  return TT_OK;
}

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of the proximal update (see tt_prox_update_noalloc in tt_sketch.h).
//
// Its only scratch -- the FP32 accumulators of [SH | Y]^T SH and the status word -- lives in the
// file-scope array below, sized for s = r0*r1 <= 160 and n <= 1024: (160 + 1024) x 160 floats and
// the status word, about 0.76 MB that every GPU loading the library holds until the process
// exits. In host code `g_noalloc_scratch` only names a host-side stand-in, so the device address
// is looked up once per device with cudaGetSymbolAddress (on the first call made while that
// device is current).

#include <mutex>

#define TT_NOALLOC_MAX_S 160
#define TT_NOALLOC_MAX_N 1024
#define TT_NOALLOC_GRAM ((TT_NOALLOC_MAX_S + TT_NOALLOC_MAX_N) * TT_NOALLOC_MAX_S)
#define TT_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) float g_noalloc_scratch[TT_NOALLOC_GRAM + 64];  // Gram, then the status word

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[TT_NOALLOC_MAX_DEVICES];

static int noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TT_NOALLOC_MAX_DEVICES) return TT_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TT_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return TT_OK;
}

extern "C" int tt_prox_update_noalloc(const float* Y_dev, const float* SH_dev, float* core_dev, int J, int n,
                                      int r0, int r1, double sigma, void* cuda_stream) {
  if (!Y_dev || !SH_dev || !core_dev) return TT_EINVAL;
  // each rank is bounded before the product is formed (in 64 bits), so that no pair of ranks can
  // wrap r0 * r1 into the accepted range
  const bool ranks_ok = r0 >= 1 && r1 >= 1 && r0 <= TT_NOALLOC_MAX_S && r1 <= TT_NOALLOC_MAX_S &&
                        (int64_t)r0 * r1 <= TT_NOALLOC_MAX_S;
  const int s = ranks_ok ? r0 * r1 : 0;
  if (J < 1 || n < 1 || !ranks_ok || n > TT_NOALLOC_MAX_N || !(sigma >= 0.0)) {
    fprintf(stderr,
            "tt_prox_update_noalloc: sizes outside the static scratch (need J >= 1, 1 <= n <= %d, "
            "r0*r1 <= %d, sigma >= 0; got J=%d n=%d r0=%d r1=%d)\n",
            TT_NOALLOC_MAX_N, TT_NOALLOC_MAX_S, J, n, r0, r1);
    return TT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  void* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  float* gram = (float*)base;
  int* status = (int*)(gram + TT_NOALLOC_GRAM);
  // the array keeps the previous call's contents: clear the accumulators and the status word
  if (cudaMemsetAsync(gram, 0, sizeof(float) * (size_t)(s + n) * s, st) != cudaSuccess) return TT_ECUDA;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return TT_ECUDA;
  GramArgs g;
  g.SH = SH_dev;
  g.Y = Y_dev;
  g.C = gram;
  g.status = status;
  g.P = nullptr;
  g.J = J;
  g.s = s;
  g.n = n;
  if (launch_gram(g, st) != cudaSuccess) return TT_ECUDA;
  SolveArgs a;
  a.C = gram;
  a.core = core_dev;
  a.change = nullptr;
  a.part = nullptr;
  a.status = status;
  a.sigma = sigma;
  a.s = s;
  a.n = n;
  a.r0 = r0;
  a.r1 = r1;
  if (launch_prox_solve(a, st) != cudaSuccess) return TT_ECUDA;
  int hst = 0;
  if (cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return TT_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TT_ECUDA;
  return hst;  // TT_OK, TT_ENOTSPD or TT_ENONFINITE
}

// ---------------------------------------------------------------------------------------------
// Relative error of a sparse tensor in coordinate form (Sec. 5's relative error; the nonzeros of
// the discussion after Theorem 3): ||A - X||^2 = ||A||^2 - 2 <A, X> + ||X||^2 with
// X = [[G_0, ..., G_{d-1}]]. The expanded form cancels (about four digits at a 1% residual), so
// every term is formed in FP64: X at each nonzero by the chain of slice products
// G_0(i_0) G_1(i_1) ... G_{d-1}(i_{d-1}) (one thread per entry, the row vector in registers: the
// loops over ranks run to RB with a predicate), and ||X||^2 by the Gram chain
// Gamma_0 = 1, Gamma_{k+1} = sum_i G_k(i)^T Gamma_k G_k(i) (one CTA per slice i, FP64 atomics).
// Ranks up to 32; the coordinates must be distinct (||A||^2 is summed entry by entry). An index
// outside [0, n_s) skips its entry and raises TT_EINVAL.

struct CooErrArgs {
  const int32_t* idx;
  const float* val;
  int64_t nnz;
  int d;
  const float* core[TT_MAX_D];
  int64_t n[TT_MAX_D];
  int r[TT_MAX_D + 1];
  double* acc;  // [0] += sum val^2, [1] += sum val X(i)
  int* status;
};

template <int RB>
__global__ void __launch_bounds__(256) k_coo_inner(CooErrArgs a) {
  double sa = 0.0, sx = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.nnz; e += (int64_t)gridDim.x * blockDim.x) {
    double u[RB], w[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) u[b] = b == 0 ? 1.0 : 0.0;  // r_0 = 1
    bool bad = false;
    for (int k = 0; k < a.d; ++k) {
      const int i = __ldg(a.idx + (int64_t)k * a.nnz + e);
      if (i < 0 || i >= a.n[k]) {
        bad = true;
        break;
      }
      const int ra = a.r[k], rb = a.r[k + 1];
      const float* G = a.core[k] + (int64_t)ra * i;
      const int64_t bstride = (int64_t)ra * a.n[k];
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        double acc = 0.0;
        if (b < rb) {
#pragma unroll
          for (int c = 0; c < RB; ++c)
            if (c < ra) acc = fma(u[c], (double)__ldg(G + c + bstride * b), acc);
        }
        w[b] = acc;
      }
#pragma unroll
      for (int b = 0; b < RB; ++b) u[b] = w[b];
    }
    if (bad) {
      atomicCAS(a.status, 0, TT_EINVAL);
      continue;
    }
    const double v = (double)__ldg(a.val + e);
    sa = fma(v, v, sa);
    sx = fma(v, u[0], sx);  // r_d = 1
  }
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(a.acc, sa);
    atomicAdd(a.acc + 1, sx);
  }
}

// Gamma_out += G(i)^T Gamma_in G(i) for the slice i = blockIdx.x of a ra x n x rb core
// (Gamma_in ra x ra, Gamma_out rb x rb, row-major, FP64)
__global__ void __launch_bounds__(256) k_tt_gram_step(const float* __restrict__ G, int n, int ra, int rb,
                                                      const double* __restrict__ Gin, double* Gout) {
  extern __shared__ double gsd[];
  double* S = gsd;            // the slice, S[a + ra b]
  double* T = gsd + ra * rb;  // Gamma_in S, same layout
  const int i = blockIdx.x;
  for (int e = threadIdx.x; e < ra * rb; e += blockDim.x) {
    const int al = e % ra, b = e / ra;
    S[e] = (double)G[al + (int64_t)ra * (i + (int64_t)n * b)];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ra * rb; e += blockDim.x) {
    const int al = e % ra, b = e / ra;
    double acc = 0.0;
    for (int c = 0; c < ra; ++c) acc = fma(Gin[al * ra + c], S[c + ra * b], acc);
    T[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rb * rb; e += blockDim.x) {
    const int b1 = e / rb, b2 = e - b1 * rb;
    double acc = 0.0;
    for (int al = 0; al < ra; ++al) acc = fma(S[al + ra * b1], T[al + ra * b2], acc);
    atomicAdd(Gout + e, acc);
  }
}

__global__ void k_set_one(double* p) { *p = 1.0; }

int tt_launch_rel_error_coo(tt_ctx* c, const int32_t* idx, const float* val, int64_t nnz, float* const* cores) {
  int rmax = 1;
  for (int k = 0; k <= c->d; ++k) rmax = std::max(rmax, c->r[k]);
  if (rmax > 32) return tt_fail(c, TT_EINVAL, "the sparse relative error supports ranks up to 32");
  CooErrArgs a;
  a.idx = idx;
  a.val = val;
  a.nnz = nnz;
  a.d = c->d;
  for (int k = 0; k < c->d; ++k) {
    a.core[k] = cores[k];
    a.n[k] = c->n[k];
  }
  for (int k = 0; k <= c->d; ++k) a.r[k] = c->r[k];
  a.acc = c->d_err_acc;
  a.status = c->d_status;
  TT_CUDA(c, cudaMemsetAsync(c->d_err_acc, 0, sizeof(double) * 3, c->stream));
  if (nnz > 0) {
    const int sms = tt_sm_count();
    const int blocks = (int)std::min<int64_t>((nnz + 255) / 256, (int64_t)sms * 8);
    if (rmax <= 8)
      k_coo_inner<8><<<blocks, 256, 0, c->stream>>>(a);
    else if (rmax <= 16)
      k_coo_inner<16><<<blocks, 256, 0, c->stream>>>(a);
    else
      k_coo_inner<32><<<blocks, 256, 0, c->stream>>>(a);
    TT_LAUNCH(c, "k_coo_inner");
  }
  double* g[2] = {c->d_xgram, c->d_xgram + 32 * 32};
  k_set_one<<<1, 1, 0, c->stream>>>(g[0]);  // Gamma_0 = 1 (r_0 = 1)
  TT_LAUNCH(c, "k_set_one");
  for (int k = 0; k < c->d; ++k) {
    const int ra = c->r[k], rb = c->r[k + 1];
    double* gin = g[k & 1];
    double* gout = g[(k + 1) & 1];
    TT_CUDA(c, cudaMemsetAsync(gout, 0, sizeof(double) * rb * rb, c->stream));
    k_tt_gram_step<<<(int)c->n[k], 256, sizeof(double) * 2 * ra * rb, c->stream>>>(cores[k], (int)c->n[k], ra, rb,
                                                                                    gin, gout);
    TT_LAUNCH(c, "k_tt_gram_step");
  }
  TT_CUDA(c, cudaMemcpyAsync(c->d_err_acc + 2, g[c->d & 1], sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return TT_OK;
}
