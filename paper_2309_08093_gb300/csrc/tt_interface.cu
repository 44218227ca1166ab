// Part (b): S H_k = F^{-1}[(F S_{>k} G_{>k}^T) face-split (F S_{<k} G_{<k})]   (Theorem 1)
// with F S_{<k} G_{<k} and F S_{>k} G_{>k}^T formed by slice-wise products of the
// FFT-sketched cores G_j x_2 (F S_j)                                            (Theorem 2).
//
// Every core is real, so each DFT is Hermitian and only the H = J/2+1 frequencies 0..J/2 are
// kept. Spectra are stored rank-major with the frequency fastest -- Ghat_j[(a + r_j b) H + w],
// R_{>k}[b H + w], L_{<k}[a H + w] -- so that every kernel below reads and writes them coalesced.
//   k_core_fft2    : CountSketch of two (a, b) fibres of a core into J buckets (real and imaginary
//                    parts) + radix-4 Stockham FFT, the fibres of several cores in one launch;
//                    k_core_fft (radix-2, one fibre) for J = 16384
//   k_suffix_chain : R_{>k}(w) = Ghat_{k+1}(w) ... Ghat_{d-1}(w) for all k, and L_{<0} = 1
//   k_prefix_step  : L_{<j+1}(w) = L_{<j}(w) Ghat_j(w)                      (one thread per w, b)
//   k_face_ifft2   : two columns c = a + r_k b of S H_k: inverse FFT of L_{<k}(w)[a] R_{>k}(w)[b]
//                    (k_face_ifft, one column with radix-2, for J = 16384)
#include "tt_internal.cuh"

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // a*b + c
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// In-place radix-2 decimation-in-time FFT of length J = 2^logJ held in shared memory, input in
// natural order (bit-reversal done here). Forward transform uses w = exp(-2 pi i / J) (Sec. 3).
__device__ void block_fft(float2* buf, const float2* __restrict__ tw, int J, int logJ) {
  for (int t = threadIdx.x; t < J; t += blockDim.x) {
    int r = (int)(__brev((unsigned)t) >> (32 - logJ));
    if (r > t) {
      float2 x = buf[t];
      buf[t] = buf[r];
      buf[r] = x;
    }
  }
  __syncthreads();
  for (int len = 2, lg = 1; len <= J; len <<= 1, ++lg) {
    int half = len >> 1;
    int step = J >> lg;  // twiddle stride
    for (int t = threadIdx.x; t < J / 2; t += blockDim.x) {
      int grp = t / half, pos = t - grp * half;
      int i = grp * len + pos, j = i + half;
      float2 w = __ldg(tw + pos * step);
      float2 u = buf[i], v = cmul(buf[j], w);
      buf[i] = make_float2(u.x + v.x, u.y + v.y);
      buf[j] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
}

// Self-sorting (Stockham) FFT of length J = 2^logJ, forward (w = exp(-2 pi i / J)), with the
// radix-4 iteration of Govindaraju et al. ("High performance discrete Fourier transforms on
// graphics processors", SC 2008): at span Ns, butterfly j reads x[j + r J/4] (r < 4), applies
// the twiddles exp(-2 pi i r (j mod Ns) / (4 Ns)), takes a 4-point DFT and writes
// y[(j / Ns) 4 Ns + (j mod Ns) + r Ns]; a radix-2 stage first when logJ is odd. x and y are
// J-entry shared buffers (ping-pong); returns the buffer holding the result. One barrier per stage.
// twst: the per-stage twiddle tables (tt_ctx::d_twstage): span Ns reads exp(-2 pi i r m / (4 Ns))
// at [off + 3 m + r - 1], consecutive butterflies consecutive entries.
// Direct DFT of any length J, for the sketch sizes that are not powers of two (logJ < 0): y[w] =
// sum_t x[t] tw[(t w) mod J] with tw[m] = exp(-2 pi i m / J), m < J; (t w) mod J is carried along t
// by one add and one conditional subtract. O(J^2) work: these are the paper's small sketch sizes.
__device__ float2* block_dft(const float2* x, float2* y, const float2* __restrict__ tw, int J) {
  for (int w = threadIdx.x; w < J; w += blockDim.x) {
    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);  // even and odd t
    int m = 0;
    int t = 0;
    for (; t + 1 < J; t += 2) {
      const float2 x0 = x[t], w0 = __ldg(tw + m);
      m = tt_modj(m + w, J);
      const float2 x1 = x[t + 1], w1 = __ldg(tw + m);
      m = tt_modj(m + w, J);
      s0 = make_float2(fmaf(x0.x, w0.x, fmaf(-x0.y, w0.y, s0.x)), fmaf(x0.x, w0.y, fmaf(x0.y, w0.x, s0.y)));
      s1 = make_float2(fmaf(x1.x, w1.x, fmaf(-x1.y, w1.y, s1.x)), fmaf(x1.x, w1.y, fmaf(x1.y, w1.x, s1.y)));
    }
    if (t < J) {
      const float2 x0 = x[t], w0 = __ldg(tw + m);
      s0 = make_float2(fmaf(x0.x, w0.x, fmaf(-x0.y, w0.y, s0.x)), fmaf(x0.x, w0.y, fmaf(x0.y, w0.x, s0.y)));
    }
    y[w] = make_float2(s0.x + s1.x, s0.y + s1.y);
  }
  __syncthreads();
  return y;
}

// For logJ < 0 the call is a direct DFT (block_dft) with twst the J-entry table tw.
__device__ float2* block_fft_stockham(float2* x, float2* y, const float2* __restrict__ twst, int J, int logJ) {
  int Ns = 1;
  __syncthreads();
  if (logJ < 0) return block_dft(x, y, twst, J);
  if (logJ & 1) {
    const int h = J >> 1;
    for (int j = threadIdx.x; j < h; j += blockDim.x) {
      const float2 v0 = x[j], v1 = x[j + h];
      y[2 * j] = make_float2(v0.x + v1.x, v0.y + v1.y);
      y[2 * j + 1] = make_float2(v0.x - v1.x, v0.y - v1.y);
    }
    float2* t = x; x = y; y = t;
    Ns = 2;
    __syncthreads();
  }
  int off = 0;
  const int q = J >> 2;
  for (; Ns < J; off += 3 * Ns, Ns <<= 2) {
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
      const int jm = j & (Ns - 1);
      float2 v0 = x[j], v1 = x[j + q], v2 = x[j + 2 * q], v3 = x[j + 3 * q];
      if (Ns > 1) {
        const float2* w = twst + off + 3 * jm;
        v1 = cmul(v1, __ldg(w));
        v2 = cmul(v2, __ldg(w + 1));
        v3 = cmul(v3, __ldg(w + 2));
      }
      const float2 a = make_float2(v0.x + v2.x, v0.y + v2.y), b = make_float2(v0.x - v2.x, v0.y - v2.y);
      const float2 c = make_float2(v1.x + v3.x, v1.y + v3.y), d = make_float2(v1.x - v3.x, v1.y - v3.y);
      const int o = (j - jm) * 4 + jm;
      y[o] = make_float2(a.x + c.x, a.y + c.y);
      y[o + Ns] = make_float2(b.x + d.y, b.y - d.x);       // b - i d
      y[o + 2 * Ns] = make_float2(a.x - c.x, a.y - c.y);
      y[o + 3 * Ns] = make_float2(b.x - d.y, b.y + d.x);   // b + i d
    }
    float2* t = x; x = y; y = t;
    __syncthreads();
  }
  return x;
}

// The fibres (a, b) of up to TT_MAX_D cores: core q owns fibre pairs [pair0[q], pair0[q + 1]).
struct CoreFftArgs {
  const float* core[TT_MAX_D];  // r0 x n x r1, r0 fastest
  const int32_t* h[TT_MAX_D];   // h_j, n entries
  const int8_t* v[TT_MAX_D];
  float2* out[TT_MAX_D];        // (r0 r1) x H, frequency fastest
  int r0[TT_MAX_D], r1[TT_MAX_D], n[TT_MAX_D];
  int pair0[TT_MAX_D + 1];
  int ncores;
  const float2* tw;    // J/2 twiddles (radix-2 path)
  const float2* twst;  // per-stage twiddles (Stockham path)
  int J, logJ;
  int det;             // deterministic mode: one thread adds the CountSketch entries in index order
};

__device__ __forceinline__ int fft_core_of(const CoreFftArgs& a, int pair) {
  int q = 0;
  while (q + 1 < a.ncores && pair >= a.pair0[q + 1]) ++q;
  return q;
}

__global__ void k_core_fft(CoreFftArgs a) {  // one fibre per CTA (pair0 counts fibres here)
  extern __shared__ float2 buf[];
  const int q = fft_core_of(a, blockIdx.x);
  const int fib = blockIdx.x - a.pair0[q];  // a + r0 * b
  const int r0 = a.r0[q], n = a.n[q];
  const int al = fib % r0, be = fib / r0;
  for (int t = threadIdx.x; t < a.J; t += blockDim.x) buf[t] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = a.det ? (threadIdx.x == 0 ? 0 : n) : threadIdx.x; i < n; i += a.det ? 1 : blockDim.x) {
    float g = a.core[q][al + (int64_t)r0 * (i + (int64_t)n * be)];
    float s = a.v[q][i] < 0 ? -g : g;
    if (a.det)
      buf[a.h[q][i]].x += s;
    else
      atomicAdd(&buf[a.h[q][i]].x, s);
  }
  __syncthreads();
  block_fft(buf, a.tw, a.J, a.logJ);
  const int H = a.J / 2 + 1;
  for (int w = threadIdx.x; w < H; w += blockDim.x) a.out[q][(int64_t)fib * H + w] = buf[w];
}

// Two CountSketched fibres per CTA, packed as z = x0 + i x1: one complex FFT, then
// X0[w] = (Z[w] + conj Z[J-w]) / 2 and X1[w] = (Z[w] - conj Z[J-w]) / 2i for w <= J/2.
__global__ void __launch_bounds__(512) k_core_fft2(CoreFftArgs a) {
  extern __shared__ float2 fbuf[];
  float2* x = fbuf;
  float2* y = fbuf + a.J;
  const int q = fft_core_of(a, blockIdx.x);
  const int r0 = a.r0[q], n = a.n[q], S = r0 * a.r1[q];
  const int f0 = 2 * (blockIdx.x - a.pair0[q]), f1 = f0 + 1;
  const bool has1 = f1 < S;
  for (int t = threadIdx.x; t < a.J; t += blockDim.x) x[t] = make_float2(0.f, 0.f);
  __syncthreads();
  const int al0 = f0 % r0, be0 = f0 / r0, al1 = f1 % r0, be1 = f1 / r0;
  const float* core = a.core[q];
  if (a.det) {  // index order: thread 0 the first fibre, thread 32 the second
    if (threadIdx.x == 0 || (has1 && threadIdx.x == 32)) {
      const int fb = threadIdx.x == 0 ? 0 : 1;
      const int al = fb ? al1 : al0, be = fb ? be1 : be0;
      for (int i = 0; i < n; ++i) {
        const float g = core[al + (int64_t)r0 * (i + (int64_t)n * be)];
        const float sg = a.v[q][i] < 0 ? -g : g;
        if (fb) x[a.h[q][i]].y += sg; else x[a.h[q][i]].x += sg;
      }
    }
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int hb = a.h[q][i];
      const bool neg = a.v[q][i] < 0;
      const float g0 = core[al0 + (int64_t)r0 * (i + (int64_t)n * be0)];
      atomicAdd(&x[hb].x, neg ? -g0 : g0);
      if (has1) {
        const float g1 = core[al1 + (int64_t)r0 * (i + (int64_t)n * be1)];
        atomicAdd(&x[hb].y, neg ? -g1 : g1);
      }
    }
  }
  const float2* Z = block_fft_stockham(x, y, a.twst, a.J, a.logJ);
  const int H = a.J / 2 + 1;
  float2* o0 = a.out[q] + (int64_t)f0 * H;
  for (int w = threadIdx.x; w < H; w += blockDim.x) {
    const float2 z = Z[w], zc = Z[w ? a.J - w : 0];
    o0[w] = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
    if (has1) o0[H + w] = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
  }
}

// FFT sketches of cores j0 .. j1-1 in one launch
static int launch_core_ffts(tt_ctx* c, float* const* cores, int j0, int j1) {
  CoreFftArgs a;
  const bool two = c->J <= 8192;  // two J-entry ping-pong buffers fit in shared memory
  a.ncores = j1 - j0;
  a.pair0[0] = 0;
  for (int q = 0; q < a.ncores; ++q) {
    const int j = j0 + q;
    a.core[q] = cores[q];
    a.h[q] = c->d_h + c->noff[j];
    a.v[q] = c->d_v + c->noff[j];
    a.out[q] = c->d_ghat + c->ghat_off[j];
    a.r0[q] = c->r[j];
    a.r1[q] = c->r[j + 1];
    a.n[q] = (int)c->n[j];
    const int S = a.r0[q] * a.r1[q];
    a.pair0[q + 1] = a.pair0[q] + (two ? (S + 1) / 2 : S);
  }
  a.tw = c->d_twiddle;
  a.twst = c->logJ >= 0 ? c->d_twstage : c->d_twiddle;  // per-stage tables, or the DFT table
  a.J = c->J;
  a.logJ = c->logJ;
  a.det = c->det ? 1 : 0;
  if (two) {
    const size_t smem = 2 * sizeof(float2) * c->J;  // ping-pong buffers
    static bool attr = false;
    if (!attr) {
      TT_CUDA(c, cudaFuncSetAttribute(k_core_fft2, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * (int)sizeof(float2) * 8192));
      attr = true;
    }
    k_core_fft2<<<a.pair0[a.ncores], 512, smem, c->stream>>>(a);
    TT_LAUNCH(c, "k_core_fft2");
    return TT_OK;
  }
  size_t smem = sizeof(float2) * c->J;
  if (smem > 48 * 1024) TT_CUDA(c, cudaFuncSetAttribute(k_core_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_core_fft<<<a.pair0[a.ncores], 512, smem, c->stream>>>(a);
  TT_LAUNCH(c, "k_core_fft");
  return TT_OK;
}

int tt_launch_core_fft(tt_ctx* c, const float* core, int j) {
  float* cs[1] = {const_cast<float*>(core)};
  return launch_core_ffts(c, cs, j, j + 1);
}

int tt_launch_core_ffts(tt_ctx* c, float* const* cores) { return launch_core_ffts(c, cores, 0, c->d); }

// ---------------------------------------------------------------------------------------------
// chain products (slice-wise products of Theorem 2), one thread per frequency

struct ChainArgs {
  const float2* ghat;
  int64_t ghat_off[TT_MAX_D + 1];
  float2* prefix;  // L_{<0} = [1] is written here too (the prefix chain restarts with the suffixes)
  float2* suffix;
  int64_t suffix_off[TT_MAX_D + 1];
  int r[TT_MAX_D + 1];
  int d, H;
};

// Block (32 frequencies) x (min(max rank, 32) rows): thread (w, y) forms R_{>k}[al][w] for
// al = y, y + blockDim.y, ... and k = d-2 .. 0; the rows of R_{>k+1} it reads were written by
// its own block before the barrier.
__global__ void k_suffix_chain(ChainArgs a) {
  const int w = blockIdx.x * 32 + threadIdx.x;
  const bool live = w < a.H;
  const int64_t H = a.H;
  if (live && threadIdx.y == 0) {
    a.suffix[a.suffix_off[a.d - 1] + w] = make_float2(1.f, 0.f);  // R_{>d-1} = [1]
    a.prefix[w] = make_float2(1.f, 0.f);                          // L_{<0} = [1]
  }
  __syncthreads();
  constexpr int U = 8;
  for (int k = a.d - 2; k >= 0; --k) {
    const int ra = a.r[k + 1], rb = a.r[k + 2];
    for (int al = threadIdx.y; live && al < ra; al += blockDim.y) {
      const float2* G = a.ghat + a.ghat_off[k + 1] + (int64_t)al * H + w;  // Ghat_{k+1}[(al + ra b) H + w]
      const float2* Rn = a.suffix + a.suffix_off[k + 1] + w;
      float2 acc = make_float2(0.f, 0.f);
      for (int b0 = 0; b0 < rb; b0 += U) {
        float2 g[U], rn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int be = min(b0 + u, rb - 1);
          g[u] = G[(int64_t)ra * be * H];
          rn[u] = Rn[(int64_t)be * H];
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (b0 + u < rb) acc = cfma(g[u], rn[u], acc);
      }
      a.suffix[a.suffix_off[k] + (int64_t)al * H + w] = acc;
    }
    __syncthreads();
  }
}

int tt_launch_suffixes(tt_ctx* c) {
  ChainArgs a;
  a.ghat = c->d_ghat;
  for (int k = 0; k <= c->d; ++k) {
    a.ghat_off[k] = c->ghat_off[k];
    a.suffix_off[k] = c->suffix_off[k];
    a.r[k] = c->r[k];
  }
  a.suffix = c->d_suffix;
  a.prefix = c->d_prefix;
  a.d = c->d;
  a.H = c->J / 2 + 1;
  int rmax = 1;
  for (int k = 1; k < c->d; ++k) rmax = std::max(rmax, c->r[k]);
  k_suffix_chain<<<(a.H + 31) / 32, dim3(32, std::min(rmax, 32)), 0, c->stream>>>(a);
  TT_LAUNCH(c, "k_suffix_chain");
  return TT_OK;
}

// L_new(w)[b] = sum_a L(w)[a] Ghat_j(w)[a + ra b]; L has ra = r[j] entries per frequency. One
// thread per (w, b): b = blockIdx.y.
__global__ void k_prefix_step(const float2* __restrict__ L, const float2* __restrict__ G, float2* Ln,
                              int ra, int H) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x, be = blockIdx.y;
  if (w >= H) return;
  constexpr int U = 8;  // loads in flight together
  float2 acc = make_float2(0.f, 0.f);
  const float2* Gb = G + (int64_t)ra * be * H + w;
  for (int a0 = 0; a0 < ra; a0 += U) {
    float2 l[U], g[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int al = min(a0 + u, ra - 1);
      l[u] = __ldg(L + (int64_t)al * H + w);
      g[u] = __ldg(Gb + (int64_t)al * H);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (a0 + u < ra) acc = cfma(l[u], g[u], acc);
  }
  Ln[(int64_t)be * H + w] = acc;
}

int tt_launch_prefix_step(tt_ctx* c, int j) {
  int H = c->J / 2 + 1;
  dim3 grid((H + 127) / 128, c->r[j + 1]);
  k_prefix_step<<<grid, 128, 0, c->stream>>>(c->d_prefix, c->d_ghat + c->ghat_off[j], c->d_prefix_tmp, c->r[j], H);
  TT_LAUNCH(c, "k_prefix_step");
  std::swap(c->d_prefix, c->d_prefix_tmp);
  return TT_OK;
}

// ---------------------------------------------------------------------------------------------
// face-split + inverse FFT: one CTA per column c = a + r_k b of S H_k

struct FaceArgs {
  const float2* L;  // ra x H (prefix L_{<k})
  const float2* R;  // rb x H (suffix R_{>k})
  const float2* tw;
  const float2* twst;
  float* zero;      // zeroed by the grid on the side (the Gram accumulators of the next kernel)
  int64_t nzero;
  float* SH;        // J x (ra rb), column-major
  int ra, rb, J, logJ;
};

// Two columns per CTA: their Hermitian spectra X, Y packed as Z = X + i Y; the inverse DFT of Z is
// x + i y, obtained as conj(FFT(conj Z)) / J.
__device__ __forceinline__ void face_zero(const FaceArgs& a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.nzero; i += (int64_t)gridDim.x * blockDim.x)
    a.zero[i] = 0.f;
}

__global__ void __launch_bounds__(256) k_face_ifft2(FaceArgs a) {
  extern __shared__ float2 fbuf[];
  face_zero(a);
  float2* x = fbuf;
  float2* y = fbuf + a.J;
  const int S = a.ra * a.rb;
  const int c0 = 2 * blockIdx.x, c1 = c0 + 1;
  const bool has1 = c1 < S;
  const int al0 = c0 % a.ra, be0 = c0 / a.ra, al1 = has1 ? c1 % a.ra : al0, be1 = has1 ? c1 / a.ra : be0;
  const int H = a.J / 2 + 1;
  const float2 *L0 = a.L + (int64_t)al0 * H, *R0 = a.R + (int64_t)be0 * H;
  const float2 *L1 = a.L + (int64_t)al1 * H, *R1 = a.R + (int64_t)be1 * H;
  constexpr int U = 4;  // frequencies per thread whose loads are in flight together
  for (int w0 = threadIdx.x; w0 < a.J; w0 += U * blockDim.x) {
    float2 l0[U], r0[U], l1[U], r1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int w = min(w0 + u * (int)blockDim.x, a.J - 1);
      const int ws = (w < H) ? w : a.J - w;
      l0[u] = __ldg(L0 + ws);
      r0[u] = __ldg(R0 + ws);
      l1[u] = __ldg(L1 + ws);
      r1[u] = __ldg(R1 + ws);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int w = w0 + u * blockDim.x;
      if (w >= a.J) break;
      float2 X = cmul(l0[u], r0[u]);
      float2 Y = has1 ? cmul(l1[u], r1[u]) : make_float2(0.f, 0.f);
      if (w >= H) {
        X.y = -X.y;
        Y.y = -Y.y;
      }
      x[w] = make_float2(X.x - Y.y, -(X.y + Y.x));  // conj(X + i Y)
    }
  }
  const float2* F = block_fft_stockham(x, y, a.twst, a.J, a.logJ);
  const float inv = 1.f / (float)a.J;
  for (int t = threadIdx.x; t < a.J; t += blockDim.x) {
    const float2 f = F[t];
    a.SH[(int64_t)c0 * a.J + t] = f.x * inv;
    if (has1) a.SH[(int64_t)c1 * a.J + t] = -f.y * inv;
  }
}

__global__ void k_face_ifft(FaceArgs a) {
  extern __shared__ float2 buf[];
  face_zero(a);
  const int col = blockIdx.x;
  const int al = col % a.ra, be = col / a.ra;
  const int H = a.J / 2 + 1;
  // conj of the full Hermitian spectrum: X[w] = L[w][a] R[w][b] for w <= J/2,
  // X[w] = conj(X[J - w]) above; forward FFT of conj(X) then real part / J = inverse DFT.
  for (int w = threadIdx.x; w < a.J; w += blockDim.x) {
    int ws = (w < H) ? w : a.J - w;
    float2 x = cmul(a.L[(int64_t)al * H + ws], a.R[(int64_t)be * H + ws]);
    if (w >= H) x.y = -x.y;
    buf[w] = make_float2(x.x, -x.y);
  }
  __syncthreads();
  block_fft(buf, a.tw, a.J, a.logJ);
  const float inv = 1.f / (float)a.J;
  for (int t = threadIdx.x; t < a.J; t += blockDim.x) a.SH[(int64_t)col * a.J + t] = buf[t].x * inv;
}

int tt_launch_interface_from_chain(tt_ctx* c, int k, float* SH, float* zero, int64_t nzero) {
  FaceArgs a;
  a.zero = zero;
  a.nzero = zero ? nzero : 0;
  a.L = c->d_prefix;
  a.R = c->d_suffix + c->suffix_off[k];
  a.tw = c->d_twiddle;
  a.twst = c->logJ >= 0 ? c->d_twstage : c->d_twiddle;  // per-stage tables, or the DFT table
  a.SH = SH;
  a.ra = c->r[k];
  a.rb = c->r[k + 1];
  a.J = c->J;
  a.logJ = c->logJ;
  if (c->J <= 8192) {  // two columns per CTA, radix-4 Stockham
    const size_t smem = 2 * sizeof(float2) * c->J;  // ping-pong buffers
    static bool attr = false;
    if (!attr) {
      TT_CUDA(c, cudaFuncSetAttribute(k_face_ifft2, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * (int)sizeof(float2) * 8192));
      attr = true;
    }
    k_face_ifft2<<<(a.ra * a.rb + 1) / 2, 256, smem, c->stream>>>(a);
    TT_LAUNCH(c, "k_face_ifft2");
    return TT_OK;
  }
  size_t smem = sizeof(float2) * c->J;
  if (smem > 48 * 1024) TT_CUDA(c, cudaFuncSetAttribute(k_face_ifft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_face_ifft<<<a.ra * a.rb, 512, smem, c->stream>>>(a);
  TT_LAUNCH(c, "k_face_ifft");
  return TT_OK;
}
