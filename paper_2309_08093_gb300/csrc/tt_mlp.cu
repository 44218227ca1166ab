// Learned warm start: the MLP's kernels and its C ABI (include/tt_warmstart.h).
//
//   k_gemm_tn<EPI>  : C = A B^T, A (M x K) and B (N x K) row-major BF16, one 128 x BN tile per
//                     CTA (BN = 128 or 256). Operands arrive by TMA (2-D tiled cp.async.bulk.tensor
//                     loads, 128-byte swizzle, rows past the end zero-filled) in the swizzled K-major
//                     layout; one thread is producer and MMA issuer: tcgen05.mma (kind::f16,
//                     BF16 x BF16 -> FP32) into a BN-column tensor-memory accumulator, a "full"
//                     mbarrier per stage counts the TMA bytes and the MMAs of a stage commit to its
//                     "empty" mbarrier. Four stages: a stage is refilled as soon as its MMAs
//                     released it. The
//                     epilogue reads the accumulator with tcgen05.ld (warp w owns lanes 32w..32w+31)
//                     and applies one of three fused epilogues:
//                       EPI_F32   : C (+ bias) -> FP32
//                       EPI_GELU  : Z = C + bias -> FP32 (kept for the backward pass),
//                                   H = GELU(Z) -> BF16 row-major and BF16 transposed
//                       EPI_DGELU : dZ = C * GELU'(Z) -> FP32, BF16 row-major, BF16 transposed
//   k_input         : gather rows of X, round to BF16 (row-major and transposed), zero padding
//   k_loss          : dY = 2 (Y - T) / (B out) and the squared-error sum (FP64)
//   k_colsum        : bias gradients (column sums, fixed order)
//   k_adam          : Adam update of FP32 masters, BF16 copies (and transposed copies)
//
// Padded shapes: in_p = roundup(in, 64), out_p = roundup(out, 64), batch rows padded to Bp =
// roundup(batch, 64) inside the batch_max buffers. Padding entries of weights and inputs are zero
// and receive zero gradients, so they stay zero.
#include <cuda.h>  // CUtensorMap (the encoder is fetched through the runtime: no libcuda link)
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/tt_warmstart.h"
#include "tt_tc.cuh"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int GM = 128, GK = 64, GSTAGES = 4;  // tile N (BN) is 128 or 256, per launch
constexpr int A_STAGE = GM * GK * 2;  // bytes per stage of A
template <int BN>
constexpr int b_stage() { return BN * GK * 2; }
template <int BN>
constexpr int gemm_smem() { return GSTAGES * (A_STAGE + b_stage<BN>()) + 1024 + 128; }

enum { EPI_F32 = 0, EPI_GELU = 1, EPI_DGELU = 2 };

struct GemmArgs {
  const bf16* A;
  int lda;
  const bf16* B;
  int ldb;
  int M, N, K;
  // epilogue
  const float* bias;  // per column (EPI_F32 optional, EPI_GELU required)
  float* f32;         // FP32 output (C, Z or dZ)
  int ldf;
  const float* zin;   // EPI_DGELU: pre-activation Z, row stride ldf
  bf16* hb;           // BF16 row-major output (EPI_GELU / EPI_DGELU)
  int ldh;
  bf16* ht;           // BF16 transposed output: ht[col * ldt + row]
  int ldt;
  int* err;           // device flag set to 1 when a bounded wait gave up
  int kchunk;         // split-K: columns of K per blockIdx.z (multiple of GK)
  int64_t slab;       // split-K: element offset between the FP32 outputs of consecutive splits
};

using namespace ttc;

// Instruction descriptor of the BF16 MMAs (kind::f16): 128 x BN tiles.
template <int BN>
constexpr uint32_t idesc() {
  return tc_idesc(1u, GM, BN);
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

template <int EPI, int BN>
__global__ void __launch_bounds__(128, 1) k_gemm_tn(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, GemmArgs g) {
  constexpr int B_STAGE = b_stage<BN>();
  constexpr uint32_t TMEM_COLS = BN;  // the 128 x BN FP32 accumulator
  constexpr uint32_t STAGE_BYTES = A_STAGE + B_STAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + GSTAGES * A_STAGE;
  uint64_t* full = (uint64_t*)(sB + GSTAGES * B_STAGE);  // TMA bytes of a stage have landed
  uint64_t* empty = full + GSTAGES;                        // the MMAs reading a stage are done
  uint32_t* s_tmem = (uint32_t*)(empty + GSTAGES);
  volatile int* s_err = (volatile int*)(s_tmem + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * g.kchunk;
  const int KT = (min(g.K, kbeg + g.kchunk) - kbeg) / GK;

  if (tid == 0) {
    for (int s = 0; s < GSTAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);

  // One thread is producer and MMA issuer: tiles go in flight up to GSTAGES ahead; after the MMAs
  // of tile kt are issued, the stage of tile kt-1 is refilled once those MMAs have released it.
  if (tid == 0) {
    auto load = [&](int t) {
      const int s = t % GSTAGES;
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, STAGE_BYTES);
      tma_load_2d(a0 + s * A_STAGE, &tmA, kbeg + t * GK, m0, fb);
      tma_load_2d(b0 + s * B_STAGE, &tmB, kbeg + t * GK, n0, fb);
    };
    for (int t = 0; t < GSTAGES && t < KT; ++t) load(t);
    int err = 0;
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % GSTAGES;
      if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((kt / GSTAGES) & 1))) { err = 1; break; }
      tc_fence_after();
      const uint32_t sa = a0 + s * A_STAGE, sb = b0 + s * B_STAGE;
#pragma unroll
      for (int kk = 0; kk < GK / 16; ++kk)
        tc_mma_f16(tmem, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), idesc<BN>(),
               (kt > 0 || kk > 0) ? 1u : 0u);
      tc_commit(smem_u32(&empty[s]));
      const int t = kt - 1 + GSTAGES;  // refill the stage of tile kt-1
      if (kt >= 1 && t < KT) {
        if (!mbar_wait(smem_u32(&empty[(kt - 1) % GSTAGES]), (uint32_t)(((kt - 1) / GSTAGES) & 1))) { err = 1; break; }
        load(t);
      }
    }
    if (!err && KT > 0) {
      const int t = KT - 1;  // the last commit covers every earlier MMA of this thread
      if (!mbar_wait(smem_u32(&empty[t % GSTAGES]), (uint32_t)((t / GSTAGES) & 1))) err = 1;
    }
    *s_err = err;
  }
  __syncthreads();
  const bool failed = *s_err != 0;
  tc_fence_after();

  if (!failed) {
    const int row = m0 + 32 * warp + lane;
    const bool row_ok = row < g.M;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      if (n0 + c0 >= g.N) break;  // uniform over the CTA
      uint32_t r[32];
      tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, r);
      const int col0 = n0 + c0;
      if (EPI == EPI_F32) {
        if (row_ok) {
          float* out = g.f32 + blockIdx.z * g.slab + (int64_t)row * g.ldf + col0;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col0 + j < g.N) out[j] = __uint_as_float(r[j]) + (g.bias ? g.bias[col0 + j] : 0.0f);
        }
      } else {
        // full 32-column chunks (N % 32 == 0 is checked on the host)
        float v[32];
        if (EPI == EPI_GELU) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) + g.bias[col0 + j];
          if (row_ok) {
            float* zo = g.f32 + (int64_t)row * g.ldf + col0;
#pragma unroll
            for (int j = 0; j < 32; j += 4) *(float4*)(zo + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = gelu_f(v[j]);
        } else {
          float zz[32];
          if (row_ok) {
            const float* zi = g.zin + (int64_t)row * g.ldf + col0;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              const float4 q = *(const float4*)(zi + j);
              zz[j] = q.x; zz[j + 1] = q.y; zz[j + 2] = q.z; zz[j + 3] = q.w;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) zz[j] = 0.0f;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) * gelu_grad_f(zz[j]);
          if (row_ok) {
            float* zo = g.f32 + (int64_t)row * g.ldf + col0;
#pragma unroll
            for (int j = 0; j < 32; j += 4) *(float4*)(zo + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          }
        }
        if (row_ok) {
          uint32_t pk[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            pk[j] = *(const uint32_t*)&h2;
          }
          uint4* ho = (uint4*)(g.hb + (int64_t)row * g.ldh + col0);
#pragma unroll
          for (int j = 0; j < 4; ++j) ho[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
#pragma unroll
          for (int j = 0; j < 32; ++j) g.ht[(int64_t)(col0 + j) * g.ldt + row] = __float2bfloat16_rn(v[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  if (failed && tid == 0 && g.err) atomicExch(g.err, 1);
}

// Split-K epilogue: v = sum of the nsplit FP32 partial products (fixed order), then the fused
// epilogue of EPI as in k_gemm_tn. 32 x 32 tiles; transposed BF16 stores go through shared memory.
template <int EPI>
__global__ void k_splitk_epi(const float* __restrict__ ws, int nsplit, int64_t slab, GemmArgs g) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int row = r0 + y, col = c0 + threadIdx.x;
    float v = 0.0f;
    if (row < g.M && col < g.N) {
      for (int z = 0; z < nsplit; ++z) v += ws[z * slab + (int64_t)row * g.N + col];
      if (EPI == EPI_F32) {
        g.f32[(int64_t)row * g.ldf + col] = v + (g.bias ? g.bias[col] : 0.0f);
      } else if (EPI == EPI_GELU) {
        const float z = v + g.bias[col];
        g.f32[(int64_t)row * g.ldf + col] = z;
        v = gelu_f(z);
        g.hb[(int64_t)row * g.ldh + col] = __float2bfloat16_rn(v);
      } else {
        v = v * gelu_grad_f(g.zin[(int64_t)row * g.ldf + col]);
        g.f32[(int64_t)row * g.ldf + col] = v;
        g.hb[(int64_t)row * g.ldh + col] = __float2bfloat16_rn(v);
      }
    }
    tile[y][threadIdx.x] = v;
  }
  if (EPI == EPI_F32) return;
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int col = c0 + y, row = r0 + threadIdx.x;
    if (col < g.N && row < g.M) g.ht[(int64_t)col * g.ldt + row] = __float2bfloat16_rn(tile[threadIdx.x][y]);
  }
}

// ---------------------------------------------------------------------------------------------
// elementwise kernels

// Rows of X (optionally gathered) -> BF16 row-major Xb (Bp x in_p) and transposed XbT
// (in_p x ldt); rows >= batch and columns >= in are zero.
__global__ void k_input(const float* __restrict__ X, int ldx, const int* __restrict__ rows, int batch, int in,
                        int in_p, int Bp, bf16* __restrict__ Xb, bf16* __restrict__ XbT, int ldt) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int row = r0 + y, col = c0 + threadIdx.x;
    float v = 0.0f;
    if (row < batch && col < in) {
      const int64_t src = rows ? (int64_t)rows[row] : (int64_t)row;
      v = X[src * ldx + col];
    }
    if (row < Bp && col < in_p) Xb[(int64_t)row * in_p + col] = __float2bfloat16_rn(v);
    tile[y][threadIdx.x] = v;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int col = c0 + y, row = r0 + threadIdx.x;
    if (col < in_p && row < Bp) XbT[(int64_t)col * ldt + row] = __float2bfloat16_rn(tile[threadIdx.x][y]);
  }
}

// dY = 2 (Y - T) / (batch * out) for valid entries, 0 in the padding; the sum of (Y - T)^2 is
// accumulated in FP64.
__global__ void k_loss(const float* __restrict__ Y, int ldy, const float* __restrict__ T, int ldt_in,
                       const int* __restrict__ rows, int batch, int out, int out_p, int Bp, float inv,
                       float* __restrict__ dY, bf16* __restrict__ dYb, bf16* __restrict__ dYbT, int ldbt,
                       double* __restrict__ loss) {
  __shared__ float tile[32][33];
  __shared__ double red[8];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  double acc = 0.0;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int row = r0 + y, col = c0 + threadIdx.x;
    float d = 0.0f;
    if (row < batch && col < out) {
      const int64_t src = rows ? (int64_t)rows[row] : (int64_t)row;
      const float res = Y[(int64_t)row * ldy + col] - T[src * ldt_in + col];
      acc += (double)res * (double)res;
      d = 2.0f * res * inv;
    }
    if (row < Bp && col < out_p) {
      dY[(int64_t)row * out_p + col] = d;
      dYb[(int64_t)row * out_p + col] = __float2bfloat16_rn(d);
    }
    tile[y][threadIdx.x] = d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) red[threadIdx.y] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)blockDim.y; ++i) s += red[i];
    if (s != 0.0) atomicAdd(loss, s);
  }
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int col = c0 + y, row = r0 + threadIdx.x;
    if (col < out_p && row < Bp) dYbT[(int64_t)col * ldbt + row] = __float2bfloat16_rn(tile[threadIdx.x][y]);
  }
}

// g[j] = sum_{row < rows} D[row * ld + j] (one thread per column, fixed order).
__global__ void k_colsum(const float* __restrict__ D, int ld, int rows, int cols, float* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.0f;
  for (int r = 0; r < rows; ++r) s += D[(int64_t)r * ld + j];
  g[j] = s;
}

// Adam on a rows x cols FP32 matrix (row-major, leading dimension cols), then BF16 copies:
// wb (row-major, optional) and wt (transposed, wt[c * rows + r], optional). pack_only skips the
// update and only refreshes the copies.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, int rows, int cols, float lr, float b1, float b2, float eps,
                       float c1, float c2, int pack_only, bf16* __restrict__ wb, bf16* __restrict__ wt) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int row = r0 + y, col = c0 + threadIdx.x;
    float x = 0.0f;
    if (row < rows && col < cols) {
      const int64_t i = (int64_t)row * cols + col;
      x = w[i];
      if (!pack_only) {
        const float gi = gr[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mhat = mi / c1, vhat = vi / c2;
        x = x - lr * mhat / (sqrtf(vhat) + eps);
        w[i] = x;
      }
      if (wb) wb[i] = __float2bfloat16_rn(x);
    }
    tile[y][threadIdx.x] = x;
  }
  if (!wt) return;
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int col = c0 + y, row = r0 + threadIdx.x;
    if (col < cols && row < rows) wt[(int64_t)col * rows + row] = __float2bfloat16_rn(tile[threadIdx.x][y]);
  }
}

// Copy a rows x cols block between row-major matrices of different leading dimensions.
__global__ void k_copy2d(const float* __restrict__ src, int lds, float* __restrict__ dst, int ldd, int rows,
                         int cols) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols, c = i % cols;
    dst[r * ldd + c] = src[r * lds + c];
  }
}

int roundup(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// ---------------------------------------------------------------------------------------------
// the network object

struct tt_mlp {
  int in = 0, hid = 0, out = 0, bmax = 0;
  int in_p = 0, out_p = 0, bmax_p = 0;
  float lr = 0, b1 = 0, b2 = 0, eps = 0;
  int t = 0;
  cudaStream_t stream = nullptr;
  std::string err;

  // FP32 masters (padded), Adam moments, gradients: index 0..5 = W1, b1, W2, b2, W3, b3
  float* P[6] = {nullptr};
  float* Mo[6] = {nullptr};
  float* Vo[6] = {nullptr};
  float* G[6] = {nullptr};
  int prow[6] = {0}, pcol[6] = {0};  // padded shapes (rows x cols; biases 1 x len)
  bf16 *W1b = nullptr, *W2b = nullptr, *W2t = nullptr, *W3b = nullptr, *W3t = nullptr;
  // activations
  bf16 *Xb = nullptr, *XbT = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *dY = nullptr, *dZ1 = nullptr, *dZ2 = nullptr;
  bf16 *H1b = nullptr, *H1t = nullptr, *H2b = nullptr, *H2t = nullptr;
  bf16 *dYb = nullptr, *dYt = nullptr, *dZ1b = nullptr, *dZ1t = nullptr, *dZ2b = nullptr, *dZ2t = nullptr;
  double* d_loss = nullptr;
  int* d_err = nullptr;
  float* ws = nullptr;      // split-K partial products
  int64_t ws_cap = 0;       // floats
  int64_t launches = 0;
};

namespace {

int mfail(tt_mlp* m, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (m) m->err = buf;
  return code;
}

#define MLP_CUDA(m, call)                                                                  \
  do {                                                                                     \
    cudaError_t _e = (call);                                                               \
    if (_e != cudaSuccess) return mfail(m, TT_ECUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
  } while (0)
#define MLP_LAUNCH(m, what)                                                                  \
  do {                                                                                       \
    cudaError_t _e = cudaGetLastError();                                                     \
    if (_e != cudaSuccess) return mfail(m, TT_ECUDA, "%s: %s", what, cudaGetErrorString(_e)); \
    if (m) ++(m)->launches;                                                                  \
  } while (0)
#define MLP_TRY(x)              \
  do {                          \
    int _r = (x);               \
    if (_r != TT_OK) return _r; \
  } while (0)

// Tensor map of a row-major BF16 matrix (rows x K, row stride ld elements): boxes of 64 K columns
// (128 bytes, the swizzle span) by box_rows rows, 128-byte swizzle, rows past the end read as 0.
int make_tmap(tt_mlp* m, CUtensorMap* tm, const bf16* base, int rows, int K, int ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return mfail(m, TT_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
  const cuuint32_t box[2] = {(cuuint32_t)GK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return mfail(m, TT_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TT_OK;
}

template <int EPI, int BN>
int launch_tiles_bn(tt_mlp* m, const GemmArgs& g, int nsplit, cudaStream_t s) {
  static bool attr_done = false;  // per template instance; the attribute is per function
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tn<EPI, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_smem<BN>());
    if (e != cudaSuccess) return mfail(m, TT_ECUDA, "gemm smem attribute: %s", cudaGetErrorString(e));
    attr_done = true;
  }
  CUtensorMap tmA, tmB;
  MLP_TRY(make_tmap(m, &tmA, g.A, g.M, g.K, g.lda, GM));
  MLP_TRY(make_tmap(m, &tmB, g.B, g.N, g.K, g.ldb, BN));
  dim3 grid((g.N + BN - 1) / BN, (g.M + GM - 1) / GM, nsplit);
  k_gemm_tn<EPI, BN><<<grid, 128, gemm_smem<BN>(), s>>>(tmA, tmB, g);
  MLP_LAUNCH(m, "k_gemm_tn");
  return TT_OK;
}

// 128 x 256 tiles when that still gives every SM a CTA (fewer operand re-reads per FLOP),
// 128 x 128 otherwise
template <int EPI>
int launch_tiles(tt_mlp* m, const GemmArgs& g, int nsplit, cudaStream_t s) {
  const int64_t wide = (int64_t)((g.N + 255) / 256) * ((g.M + GM - 1) / GM) * nsplit;
  if (wide >= 148) return launch_tiles_bn<EPI, 256>(m, g, nsplit, s);
  return launch_tiles_bn<EPI, 128>(m, g, nsplit, s);
}

// Number of K splits: enough CTAs to cover the SMs when the tile grid is small, at least four
// K tiles per split, at most 32 splits, and partial products that fit the workspace.
int choose_split(int M, int N, int K, int64_t cap) {
  const int tiles = ((M + GM - 1) / GM) * ((N + 127) / 128);
  const int KT = K / GK;
  if (tiles >= 100 || KT < 8) return 1;
  int s = std::min(KT / 4, (148 + tiles - 1) / tiles);
  s = std::min(s, 32);
  while (s > 1 && (int64_t)s * M * N > cap) --s;
  return std::max(s, 1);
}

template <int EPI>
int launch_gemm(tt_mlp* m, const GemmArgs& g, cudaStream_t s) {
  const int split = m ? choose_split(g.M, g.N, g.K, m->ws_cap) : 1;
  if (split <= 1) return launch_tiles<EPI>(m, g, 1, s);
  const int KT = g.K / GK;
  const int kchunk = ((KT + split - 1) / split) * GK;
  const int nsplit = (g.K + kchunk - 1) / kchunk;
  GemmArgs p = g;
  p.kchunk = kchunk;
  p.slab = (int64_t)g.M * g.N;
  p.f32 = m->ws;
  p.ldf = g.N;
  p.bias = nullptr;
  MLP_TRY(launch_tiles<EPI_F32>(m, p, nsplit, s));
  dim3 grid((g.N + 31) / 32, (g.M + 31) / 32), blk(32, 8);
  k_splitk_epi<EPI><<<grid, blk, 0, s>>>(m->ws, nsplit, p.slab, g);
  MLP_LAUNCH(m, "k_splitk_epi");
  return TT_OK;
}

GemmArgs gemm_args(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, int* err) {
  GemmArgs g{};
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.M = M; g.N = N; g.K = K; g.err = err;
  g.kchunk = K;
  g.slab = 0;
  return g;
}

int check_err_flag(tt_mlp* m) {
  int h = 0;
  MLP_CUDA(m, cudaMemcpyAsync(&h, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  MLP_CUDA(m, cudaStreamSynchronize(m->stream));
  if (h) return mfail(m, TT_ETIMEOUT, "a bounded wait in the GEMM kernel gave up");
  return TT_OK;
}

int pack_weights(tt_mlp* m) {
  dim3 blk(32, 8);
  bf16* wb[6] = {m->W1b, nullptr, m->W2b, nullptr, m->W3b, nullptr};
  bf16* wt[6] = {nullptr, nullptr, m->W2t, nullptr, m->W3t, nullptr};
  for (int i = 0; i < 6; i += 2) {
    dim3 grid((m->pcol[i] + 31) / 32, (m->prow[i] + 31) / 32);
    k_adam<<<grid, blk, 0, m->stream>>>(m->P[i], nullptr, nullptr, nullptr, m->prow[i], m->pcol[i], 0, 0, 0, 0, 1,
                                        1, 1, wb[i], wt[i]);
    MLP_LAUNCH(m, "k_adam(pack)");
  }
  return TT_OK;
}

// forward pass for `batch` rows; leaves Z1, Z2, H*, Y in the network's buffers
int forward(tt_mlp* m, const float* X, int ldx, const int* rows, int batch) {
  const int Bp = roundup(batch, 64);
  {
    dim3 grid((m->in_p + 31) / 32, (Bp + 31) / 32), blk(32, 8);
    k_input<<<grid, blk, 0, m->stream>>>(X, ldx, rows, batch, m->in, m->in_p, Bp, m->Xb, m->XbT, m->bmax_p);
    MLP_LAUNCH(m, "k_input");
  }
  GemmArgs g = gemm_args(m->Xb, m->in_p, m->W1b, m->in_p, Bp, m->hid, m->in_p, m->d_err);
  g.bias = m->P[1]; g.f32 = m->Z1; g.ldf = m->hid; g.hb = m->H1b; g.ldh = m->hid; g.ht = m->H1t; g.ldt = m->bmax_p;
  MLP_TRY(launch_gemm<EPI_GELU>(m, g, m->stream));
  g = gemm_args(m->H1b, m->hid, m->W2b, m->hid, Bp, m->hid, m->hid, m->d_err);
  g.bias = m->P[3]; g.f32 = m->Z2; g.ldf = m->hid; g.hb = m->H2b; g.ldh = m->hid; g.ht = m->H2t; g.ldt = m->bmax_p;
  MLP_TRY(launch_gemm<EPI_GELU>(m, g, m->stream));
  g = gemm_args(m->H2b, m->hid, m->W3b, m->hid, Bp, m->out_p, m->hid, m->d_err);
  g.bias = m->P[5]; g.f32 = m->Y; g.ldf = m->out_p;
  MLP_TRY(launch_gemm<EPI_F32>(m, g, m->stream));
  return TT_OK;
}

// loss gradient and backward pass into m->G[*]
int backward(tt_mlp* m, const float* T, int ldt, const int* rows, int batch) {
  const int Bp = roundup(batch, 64);
  MLP_CUDA(m, cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->stream));
  {
    dim3 grid((m->out_p + 31) / 32, (Bp + 31) / 32), blk(32, 8);
    const float inv = (float)(1.0 / ((double)batch * (double)m->out));
    k_loss<<<grid, blk, 0, m->stream>>>(m->Y, m->out_p, T, ldt, rows, batch, m->out, m->out_p, Bp, inv, m->dY,
                                        m->dYb, m->dYt, m->bmax_p, m->d_loss);
    MLP_LAUNCH(m, "k_loss");
  }
  // dW3 = dY^T H2, db3 = colsum(dY)
  GemmArgs g = gemm_args(m->dYt, m->bmax_p, m->H2t, m->bmax_p, m->out_p, m->hid, Bp, m->d_err);
  g.f32 = m->G[4]; g.ldf = m->hid;
  MLP_TRY(launch_gemm<EPI_F32>(m, g, m->stream));
  k_colsum<<<(m->out_p + 255) / 256, 256, 0, m->stream>>>(m->dY, m->out_p, Bp, m->out_p, m->G[5]);
  MLP_LAUNCH(m, "k_colsum");
  // dZ2 = (dY W3) * GELU'(Z2)
  g = gemm_args(m->dYb, m->out_p, m->W3t, m->out_p, Bp, m->hid, m->out_p, m->d_err);
  g.f32 = m->dZ2; g.ldf = m->hid; g.zin = m->Z2; g.hb = m->dZ2b; g.ldh = m->hid; g.ht = m->dZ2t; g.ldt = m->bmax_p;
  MLP_TRY(launch_gemm<EPI_DGELU>(m, g, m->stream));
  // dW2 = dZ2^T H1, db2
  g = gemm_args(m->dZ2t, m->bmax_p, m->H1t, m->bmax_p, m->hid, m->hid, Bp, m->d_err);
  g.f32 = m->G[2]; g.ldf = m->hid;
  MLP_TRY(launch_gemm<EPI_F32>(m, g, m->stream));
  k_colsum<<<(m->hid + 255) / 256, 256, 0, m->stream>>>(m->dZ2, m->hid, Bp, m->hid, m->G[3]);
  MLP_LAUNCH(m, "k_colsum");
  // dZ1 = (dZ2 W2) * GELU'(Z1)
  g = gemm_args(m->dZ2b, m->hid, m->W2t, m->hid, Bp, m->hid, m->hid, m->d_err);
  g.f32 = m->dZ1; g.ldf = m->hid; g.zin = m->Z1; g.hb = m->dZ1b; g.ldh = m->hid; g.ht = m->dZ1t; g.ldt = m->bmax_p;
  MLP_TRY(launch_gemm<EPI_DGELU>(m, g, m->stream));
  // dW1 = dZ1^T X, db1
  g = gemm_args(m->dZ1t, m->bmax_p, m->XbT, m->bmax_p, m->hid, m->in_p, Bp, m->d_err);
  g.f32 = m->G[0]; g.ldf = m->in_p;
  MLP_TRY(launch_gemm<EPI_F32>(m, g, m->stream));
  k_colsum<<<(m->hid + 255) / 256, 256, 0, m->stream>>>(m->dZ1, m->hid, Bp, m->hid, m->G[1]);
  MLP_LAUNCH(m, "k_colsum");
  return TT_OK;
}

int check_batch(tt_mlp* m, const float* X, int ldx, int batch) {
  if (!X) return mfail(m, TT_EINVAL, "null input");
  if (batch < 1 || batch > m->bmax) return mfail(m, TT_EINVAL, "batch %d outside 1..%d", batch, m->bmax);
  if (ldx < m->in) return mfail(m, TT_EINVAL, "ldx %d < in_dim %d", ldx, m->in);
  return TT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// C ABI

extern "C" int tt_mlp_init(tt_mlp** out, const tt_mlp_params* p, void* cuda_stream) {
  if (!out || !p) return TT_EINVAL;
  *out = nullptr;
  if (p->in_dim < 1 || p->in_dim > 65536 || p->hidden < 64 || p->hidden > 2048 || p->hidden % 64 != 0 ||
      p->out_dim < 1 || p->out_dim > 262144 || p->batch_max < 1 || p->batch_max > 1024 || !(p->beta1 >= 0.0f) ||
      !(p->beta1 < 1.0f) || !(p->beta2 >= 0.0f) || !(p->beta2 < 1.0f) || !(p->eps > 0.0f) || !std::isfinite(p->lr)) {
    fprintf(stderr, "tt_mlp_init: invalid parameters\n");
    return TT_EINVAL;
  }
  tt_mlp* m = new tt_mlp();
  m->in = p->in_dim; m->hid = p->hidden; m->out = p->out_dim; m->bmax = p->batch_max;
  m->in_p = roundup(m->in, 64); m->out_p = roundup(m->out, 64); m->bmax_p = roundup(m->bmax, 64);
  m->lr = p->lr; m->b1 = p->beta1; m->b2 = p->beta2; m->eps = p->eps;
  m->stream = (cudaStream_t)cuda_stream;
  const int R[6] = {m->hid, 1, m->hid, 1, m->out_p, 1};
  const int C[6] = {m->in_p, m->hid, m->hid, m->hid, m->hid, m->out_p};
  auto fail = [&](const char* what) {
    fprintf(stderr, "tt_mlp_init: allocation of %s failed\n", what);
    tt_mlp_destroy(m);
    return TT_ENOMEM;
  };
  for (int i = 0; i < 6; ++i) {
    m->prow[i] = R[i];
    m->pcol[i] = C[i];
    const size_t bytes = (size_t)R[i] * C[i] * sizeof(float);
    if (cudaMalloc(&m->P[i], bytes) != cudaSuccess || cudaMalloc(&m->Mo[i], bytes) != cudaSuccess ||
        cudaMalloc(&m->Vo[i], bytes) != cudaSuccess || cudaMalloc(&m->G[i], bytes) != cudaSuccess)
      return fail("parameters");
    cudaMemset(m->P[i], 0, bytes);
    cudaMemset(m->Mo[i], 0, bytes);
    cudaMemset(m->Vo[i], 0, bytes);
    cudaMemset(m->G[i], 0, bytes);
  }
  const size_t h = m->hid, ip = m->in_p, op = m->out_p, bp = m->bmax_p;
  struct {
    void** p;
    size_t bytes;
  } bufs[] = {{(void**)&m->W1b, h * ip * 2}, {(void**)&m->W2b, h * h * 2}, {(void**)&m->W2t, h * h * 2},
              {(void**)&m->W3b, op * h * 2}, {(void**)&m->W3t, op * h * 2}, {(void**)&m->Xb, bp * ip * 2},
              {(void**)&m->XbT, ip * bp * 2}, {(void**)&m->Z1, bp * h * 4}, {(void**)&m->Z2, bp * h * 4},
              {(void**)&m->Y, bp * op * 4}, {(void**)&m->dY, bp * op * 4}, {(void**)&m->dZ1, bp * h * 4},
              {(void**)&m->dZ2, bp * h * 4}, {(void**)&m->H1b, bp * h * 2}, {(void**)&m->H1t, h * bp * 2},
              {(void**)&m->H2b, bp * h * 2}, {(void**)&m->H2t, h * bp * 2}, {(void**)&m->dYb, bp * op * 2},
              {(void**)&m->dYt, op * bp * 2}, {(void**)&m->dZ1b, bp * h * 2}, {(void**)&m->dZ1t, h * bp * 2},
              {(void**)&m->dZ2b, bp * h * 2}, {(void**)&m->dZ2t, h * bp * 2}, {(void**)&m->d_loss, 8},
              {(void**)&m->d_err, 4}, {(void**)&m->ws, (size_t)32 * bp * h * 4}};
  m->ws_cap = (int64_t)32 * bp * h;
  for (auto& b : bufs) {
    if (cudaMalloc(b.p, b.bytes) != cudaSuccess) return fail("activations");
    cudaMemset(*b.p, 0, b.bytes);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return fail("initialisation");
  *out = m;
  return TT_OK;
}

extern "C" int tt_mlp_destroy(tt_mlp* m) {
  if (!m) return TT_OK;
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (int i = 0; i < 6; ++i) {
    cudaFree(m->P[i]); cudaFree(m->Mo[i]); cudaFree(m->Vo[i]); cudaFree(m->G[i]);
  }
  void* ps[] = {m->W1b, m->W2b, m->W2t, m->W3b, m->W3t, m->Xb, m->XbT, m->Z1, m->Z2, m->Y, m->dY, m->dZ1, m->dZ2,
                m->H1b, m->H1t, m->H2b, m->H2t, m->dYb, m->dYt, m->dZ1b, m->dZ1t, m->dZ2b, m->dZ2t, m->d_loss,
                m->d_err, m->ws};
  for (void* p : ps) cudaFree(p);
  delete m;
  return TT_OK;
}

extern "C" const char* tt_mlp_last_error(tt_mlp* m) { return m ? m->err.c_str() : "null network"; }

extern "C" int tt_mlp_set_weights(tt_mlp* m, const float* W1, const float* b1, const float* W2, const float* b2,
                                  const float* W3, const float* b3) {
  if (!m) return TT_EINVAL;
  if (!W1 || !b1 || !W2 || !b2 || !W3 || !b3) return mfail(m, TT_EINVAL, "null weight pointer");
  const float* src[6] = {W1, b1, W2, b2, W3, b3};
  const int rows[6] = {m->hid, 1, m->hid, 1, m->out, 1};
  const int cols[6] = {m->in, m->hid, m->hid, m->hid, m->hid, m->out};
  for (int i = 0; i < 6; ++i) {
    const size_t bytes = (size_t)m->prow[i] * m->pcol[i] * sizeof(float);
    MLP_CUDA(m, cudaMemsetAsync(m->P[i], 0, bytes, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->Mo[i], 0, bytes, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->Vo[i], 0, bytes, m->stream));
    k_copy2d<<<256, 256, 0, m->stream>>>(src[i], cols[i], m->P[i], m->pcol[i], rows[i], cols[i]);
    MLP_LAUNCH(m, "k_copy2d");
  }
  m->t = 0;
  return pack_weights(m);
}

extern "C" int tt_mlp_get_weights(tt_mlp* m, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3) {
  if (!m) return TT_EINVAL;
  if (!W1 || !b1 || !W2 || !b2 || !W3 || !b3) return mfail(m, TT_EINVAL, "null weight pointer");
  float* dst[6] = {W1, b1, W2, b2, W3, b3};
  const int rows[6] = {m->hid, 1, m->hid, 1, m->out, 1};
  const int cols[6] = {m->in, m->hid, m->hid, m->hid, m->hid, m->out};
  for (int i = 0; i < 6; ++i) {
    k_copy2d<<<256, 256, 0, m->stream>>>(m->P[i], m->pcol[i], dst[i], cols[i], rows[i], cols[i]);
    MLP_LAUNCH(m, "k_copy2d");
  }
  return TT_OK;
}

extern "C" int tt_mlp_forward(tt_mlp* m, const float* X, int ldx, const int* rows, int batch, float* Y, int ldy) {
  if (!m) return TT_EINVAL;
  MLP_TRY(check_batch(m, X, ldx, batch));
  if (!Y || ldy < m->out) return mfail(m, TT_EINVAL, "bad output (ldy %d < out_dim %d or null)", ldy, m->out);
  MLP_CUDA(m, cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream));
  MLP_TRY(forward(m, X, ldx, rows, batch));
  k_copy2d<<<256, 256, 0, m->stream>>>(m->Y, m->out_p, Y, ldy, batch, m->out);
  MLP_LAUNCH(m, "k_copy2d");
  return TT_OK;
}

extern "C" int tt_mlp_loss_grads(tt_mlp* m, const float* X, int ldx, const float* T, int ldt, const int* rows,
                                 int batch, double* loss_out, float* gW1, float* gb1, float* gW2, float* gb2,
                                 float* gW3, float* gb3) {
  if (!m) return TT_EINVAL;
  MLP_TRY(check_batch(m, X, ldx, batch));
  if (!T || ldt < m->out) return mfail(m, TT_EINVAL, "bad targets (ldt %d < out_dim %d or null)", ldt, m->out);
  MLP_CUDA(m, cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream));
  MLP_TRY(forward(m, X, ldx, rows, batch));
  MLP_TRY(backward(m, T, ldt, rows, batch));
  float* dst[6] = {gW1, gb1, gW2, gb2, gW3, gb3};
  const int r[6] = {m->hid, 1, m->hid, 1, m->out, 1};
  const int c[6] = {m->in, m->hid, m->hid, m->hid, m->hid, m->out};
  for (int i = 0; i < 6; ++i) {
    if (!dst[i]) continue;
    k_copy2d<<<256, 256, 0, m->stream>>>(m->G[i], m->pcol[i], dst[i], c[i], r[i], c[i]);
    MLP_LAUNCH(m, "k_copy2d");
  }
  MLP_TRY(check_err_flag(m));
  if (loss_out) {
    double s = 0.0;
    MLP_CUDA(m, cudaMemcpyAsync(&s, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    *loss_out = s / ((double)batch * (double)m->out);
  }
  return TT_OK;
}

extern "C" int tt_mlp_train_step(tt_mlp* m, const float* X, int ldx, const float* T, int ldt, const int* rows,
                                 int batch, double* loss_out) {
  if (!m) return TT_EINVAL;
  MLP_TRY(check_batch(m, X, ldx, batch));
  if (!T || ldt < m->out) return mfail(m, TT_EINVAL, "bad targets (ldt %d < out_dim %d or null)", ldt, m->out);
  MLP_CUDA(m, cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream));
  MLP_TRY(forward(m, X, ldx, rows, batch));
  MLP_TRY(backward(m, T, ldt, rows, batch));
  m->t += 1;
  const double c1 = 1.0 - std::pow((double)m->b1, (double)m->t);
  const double c2 = 1.0 - std::pow((double)m->b2, (double)m->t);
  bf16* wb[6] = {m->W1b, nullptr, m->W2b, nullptr, m->W3b, nullptr};
  bf16* wt[6] = {nullptr, nullptr, m->W2t, nullptr, m->W3t, nullptr};
  dim3 blk(32, 8);
  for (int i = 0; i < 6; ++i) {
    dim3 grid((m->pcol[i] + 31) / 32, (m->prow[i] + 31) / 32);
    k_adam<<<grid, blk, 0, m->stream>>>(m->P[i], m->G[i], m->Mo[i], m->Vo[i], m->prow[i], m->pcol[i], m->lr, m->b1,
                                        m->b2, m->eps, (float)c1, (float)c2, 0, wb[i], wt[i]);
    MLP_LAUNCH(m, "k_adam");
  }
  if (loss_out) {
    MLP_TRY(check_err_flag(m));
    double s = 0.0;
    MLP_CUDA(m, cudaMemcpyAsync(&s, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    *loss_out = s / ((double)batch * (double)m->out);
  }
  return TT_OK;
}

extern "C" int tt_mlp_gemm_bf16(const uint16_t* A, int lda, const uint16_t* B, int ldb, int M, int N, int K,
                                float* C, int ldc, int check, void* cuda_stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < GK || K % GK != 0 || lda < K || ldb < K || lda % 8 != 0 ||
      ldb % 8 != 0 || ldc < N || ((uintptr_t)A & 15) || ((uintptr_t)B & 15)) {
    fprintf(stderr, "tt_mlp_gemm_bf16: invalid arguments\n");
    return TT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  static int* d_flag = nullptr;  // one flag for the standalone entry point
  if (!d_flag && cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess) return TT_ENOMEM;
  if (cudaMemsetAsync(d_flag, 0, sizeof(int), s) != cudaSuccess) return TT_ECUDA;
  GemmArgs g = gemm_args((const bf16*)A, lda, (const bf16*)B, ldb, M, N, K, d_flag);
  g.f32 = C;
  g.ldf = ldc;
  int rc = launch_gemm<EPI_F32>(nullptr, g, s);
  if (rc != TT_OK) return rc;
  if (check) {
    int h = 0;
    if (cudaMemcpyAsync(&h, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return TT_ECUDA;
    if (h) return TT_ETIMEOUT;
  }
  return TT_OK;
}
