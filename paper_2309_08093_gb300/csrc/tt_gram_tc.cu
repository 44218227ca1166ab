// Gram and right-hand side of the proximal update (Eq. (ite)) on the tensor cores:
//   M = (S H_k)^T (S H_k)   (s x s)   and   B^T = (S H_k)^T Y_k   (s x n),
// both as D = A B^T with K = J (the sketch rows) contiguous in memory for every operand row:
// A = (S H_k)^T for the Gram tiles or Y_k^T for the right-hand-side tiles, B = (S H_k)^T.
//
// k_gram_tc: one CTA per (128-row output tile, K-chunk). Operand tiles of 32 FP32 entries of K
// (128 bytes) arrive by TMA (2-D tiled cp.async.bulk.tensor, 128-byte swizzle, rows and K past
// the end zero-filled) into four stages counted by "full" mbarriers; one thread issues
// tcgen05.mma kind::tf32 (M = 128, N = s rounded up to 16, K = 8 per instruction) into an FP32
// accumulator in tensor memory and commits each stage to its "empty" mbarrier, which releases the
// stage for the next TMA. The epilogue reads the accumulator with tcgen05.ld (warp w owns rows
// 32w .. 32w + 31) and adds the K-chunk's sums into the FP32 Gram buffer with atomics (or stores
// them as partials in the deterministic mode). Waits are bounded (2 s): a wait that gives up
// raises TT_ETIMEOUT and the CTA frees its tensor memory and returns.
//
// Two precisions:
//   TF32 x 1 : each operand read as TF32 (10 explicit mantissa bits): products carry a relative
//              error up to about 2^-11 (the mixed-precision form);
//   TF32 x 3 : every staged tile is split in shared memory into hi = tf32(x) and lo = tf32(x - hi)
//              (both rounded to nearest), and the MMAs add hi*hi + hi*lo + lo*hi: the dropped
//              lo*lo term and the rounding of lo leave a relative error of about 2^-22 per
//              product, the FP32 form's accuracy.
#include <stdio.h>

#include <algorithm>

#include "tt_internal.cuh"
#include "tt_tc.cuh"

using namespace ttc;

namespace {

constexpr int TG_M = 128, TG_BK = 32, TG_T = 128;
// pipeline depth: four stages of raw tiles, or three of raw + lo tiles (shared memory)
template <bool SPLIT3>
constexpr int tg_stages() { return SPLIT3 ? 3 : 4; }
constexpr int TG_A_BYTES = TG_M * TG_BK * 4;  // 16 KB per stage of A

struct GramTcArgs {
  float* C;      // Gram (s x s row-major), then the right-hand side transposed (s x n)
  float* P;      // deterministic mode: K-chunk z stores its sums at P + z (s + n) s (no atomics)
  int* status;
  int s, n, np;  // np = s rounded up to 16 (the MMA's N)
  int mt_gram;   // output tiles of the Gram part; the rest are right-hand-side tiles
  int J, kchunk;
};

__host__ __device__ constexpr size_t tg_b_bytes(int np) { return (size_t)np * TG_BK * 4; }
__host__ __device__ constexpr size_t tg_stage_bytes(int np, bool split3) {
  return (TG_A_BYTES + tg_b_bytes(np)) * (split3 ? 2 : 1);
}
__host__ constexpr size_t tg_smem(int np, bool split3) {
  return (split3 ? tg_stages<true>() : tg_stages<false>()) * tg_stage_bytes(np, split3) + 1024 + 256;
}

// x rounded to the nearest TF32 value (ties away from zero): a 32-bit word whose low 13 mantissa
// bits are zero
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// hi = tf32(x), lo = tf32(x - hi) (x - hi is exact in FP32): hi in place, lo into `lo` at the same
// offset (the elementwise split keeps the swizzled layout). |x - hi - lo| <= 2^-22 |x| about.
__device__ __forceinline__ void tf32_split(uint8_t* tile, uint8_t* lo, int bytes, int t) {
  for (int o = t * 16; o < bytes; o += TG_T * 16) {
    float4 x = *reinterpret_cast<float4*>(tile + o);
    float4 h, l;
    h.x = to_tf32(x.x), h.y = to_tf32(x.y), h.z = to_tf32(x.z), h.w = to_tf32(x.w);
    l.x = to_tf32(x.x - h.x), l.y = to_tf32(x.y - h.y), l.z = to_tf32(x.z - h.z), l.w = to_tf32(x.w - h.w);
    *reinterpret_cast<float4*>(tile + o) = h;
    *reinterpret_cast<float4*>(lo + o) = l;
  }
}

template <bool SPLIT3>
__global__ void __launch_bounds__(TG_T, 1) k_gram_tc(const __grid_constant__ CUtensorMap tmSHa,
                                                      const __grid_constant__ CUtensorMap tmYa,
                                                      const __grid_constant__ CUtensorMap tmSHb, GramTcArgs g) {
  constexpr int TG_STAGES = tg_stages<SPLIT3>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int np = g.np;
  const uint32_t b_bytes = (uint32_t)tg_b_bytes(np);
  const uint32_t stage = (uint32_t)tg_stage_bytes(np, SPLIT3);
  uint64_t* full = (uint64_t*)(smem + TG_STAGES * stage);
  uint64_t* empty = full + TG_STAGES;
  uint32_t* s_tmem = (uint32_t*)(empty + TG_STAGES);
  volatile int* s_err = (volatile int*)(s_tmem + 2);
  volatile int* s_skip = s_err + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool rhs = (int)blockIdx.x >= g.mt_gram;
  const int row0 = (rhs ? (int)blockIdx.x - g.mt_gram : (int)blockIdx.x) * TG_M;
  const int kbeg = blockIdx.y * g.kchunk;
  const int KT = (min(g.J, kbeg + g.kchunk) - kbeg + TG_BK - 1) / TG_BK;
  const CUtensorMap* tmA = rhs ? &tmYa : &tmSHa;
  uint32_t cols = 32;
  while ((int)cols < np) cols <<= 1;  // tensor-memory columns: a power of two >= 32
  const uint32_t idesc = tc_idesc(2u, TG_M, np);
  if (tid == 0) {
    *s_skip = *g.status != 0;  // read once: other CTAs of this kernel may raise it meanwhile
    for (int s = 0; s < TG_STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (*s_skip) return;  // uniform, before anything is allocated
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(s_tmem)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t base = smem_u32(smem);
  auto sa = [&](int s) { return base + (uint32_t)s * stage; };
  auto sb = [&](int s) { return sa(s) + TG_A_BYTES; };
  int issued = 0;  // thread 0: TMA tiles issued (tiles 0 .. issued-1)
  auto load = [&](int t) {  // thread 0
    issued = t + 1;
    const int s = t % TG_STAGES;
    const uint32_t fb = smem_u32(&full[s]);
    mbar_expect_tx(fb, TG_A_BYTES + b_bytes);
    tma_load_2d(sa(s), tmA, kbeg + t * TG_BK, row0, fb);
    tma_load_2d(sb(s), &tmSHb, kbeg + t * TG_BK, 0, fb);
  };
  auto mmas = [&](int s, bool first) {  // thread 0: the 4 K-steps of 8 entries of one stage
#pragma unroll
    for (int kk = 0; kk < TG_BK / 8; ++kk) {
      const uint64_t ah = smem_desc_sw128(sa(s) + kk * 32), bh = smem_desc_sw128(sb(s) + kk * 32);
      tc_mma_tf32(tmem, ah, bh, idesc, (!first || kk > 0) ? 1u : 0u);
      if constexpr (SPLIT3) {
        const uint32_t lo = sa(s) + TG_A_BYTES + b_bytes;  // A lo, then B lo
        tc_mma_tf32(tmem, ah, smem_desc_sw128(lo + TG_A_BYTES + kk * 32), idesc, 1u);
        tc_mma_tf32(tmem, smem_desc_sw128(lo + kk * 32), bh, idesc, 1u);
      }
    }
    tc_commit(smem_u32(&empty[s]));
  };

  // After a wait gave up: wait (bounded) for the TMA tiles still in flight from tile `from` on, so
  // that no copy lands in shared memory after the CTA has left (thread 0).
  auto drain = [&](int from) {
    for (int t = from; t < issued; ++t)
      if (!mbar_wait(smem_u32(&full[t % TG_STAGES]), (uint32_t)((t / TG_STAGES) & 1))) break;
  };
  int err = 0;
  if (!SPLIT3) {
    if (tid == 0) {
      for (int t = 0; t < TG_STAGES && t < KT; ++t) load(t);
      for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % TG_STAGES;
        if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((kt / TG_STAGES) & 1))) { err = 1; drain(kt); break; }
        tc_fence_after();
        mmas(s, kt == 0);
        const int t = kt - 1 + TG_STAGES;  // refill the stage of tile kt-1 once its MMAs are done
        if (kt >= 1 && t < KT) {
          if (!mbar_wait(smem_u32(&empty[(kt - 1) % TG_STAGES]), (uint32_t)(((kt - 1) / TG_STAGES) & 1))) {
            err = 1;
            drain(kt + 1);
            break;
          }
          load(t);
        }
      }
      if (!err && KT > 0) {
        const int t = KT - 1;  // the last commit covers every earlier MMA of this thread
        if (!mbar_wait(smem_u32(&empty[t % TG_STAGES]), (uint32_t)((t / TG_STAGES) & 1))) err = 1;
      }
      *s_err = err;
    }
  } else {
    if (tid == 0)
      for (int t = 0; t < TG_STAGES && t < KT; ++t) load(t);
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % TG_STAGES;
      // every thread waits for the stage's bytes, splits its share, and hands it to the async proxy
      const bool ok = mbar_wait(smem_u32(&full[s]), (uint32_t)((kt / TG_STAGES) & 1));
      if (__syncthreads_or(!ok)) {
        if (tid == 0) drain(kt);
        err = 1;
        break;
      }
      uint8_t* st = smem + (size_t)s * stage;
      tf32_split(st, st + TG_A_BYTES + b_bytes, TG_A_BYTES, tid);
      tf32_split(st + TG_A_BYTES, st + 2 * TG_A_BYTES + b_bytes, (int)b_bytes, tid);
      fence_async_smem();
      __syncthreads();
      int e2 = 0;
      if (tid == 0) {
        tc_fence_after();
        mmas(s, kt == 0);
        const int t = kt - 1 + TG_STAGES;
        if (kt >= 1 && t < KT) {
          if (!mbar_wait(smem_u32(&empty[(kt - 1) % TG_STAGES]), (uint32_t)(((kt - 1) / TG_STAGES) & 1))) {
            e2 = 1;
            drain(kt + 1);
          } else {
            load(t);
          }
        }
      }
      if (__syncthreads_or(e2)) { err = 1; break; }
    }
    if (tid == 0) {
      if (!err && KT > 0) {
        const int t = KT - 1;
        if (!mbar_wait(smem_u32(&empty[t % TG_STAGES]), (uint32_t)((t / TG_STAGES) & 1))) err = 1;
      }
      *s_err = err;
    }
  }
  __syncthreads();
  const bool failed = *s_err != 0;
  tc_fence_after();
  if (!failed) {
    const int r = row0 + 32 * warp + lane;  // this thread's output row (a column of S H_k or of Y_k)
    const bool row_ok = r < (rhs ? g.n : g.s);
    const int64_t cnt = (int64_t)(g.s + g.n) * g.s;
    bool finite = true;
    for (int c0 = 0; c0 < np; c0 += 32) {
      uint32_t v[32];
      tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      if (!row_ok) continue;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = c0 + j;
        if (col >= g.s) break;
        const float x = __uint_as_float(v[j]);
        finite = finite && isfinite(x);
        const int64_t idx = rhs ? (int64_t)g.s * g.s + (int64_t)col * g.n + r : (int64_t)r * g.s + col;
        if (g.P)
          g.P[(int64_t)blockIdx.y * cnt + idx] = x;
        else
          atomicAdd(g.C + idx, x);
      }
    }
    if (!finite) atomicCAS(g.status, 0, TT_ENONFINITE);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols) : "memory");
  if (failed && tid == 0) atomicCAS(g.status, 0, TT_ETIMEOUT);
}

// Tensor map of a column-major J x rows FP32 matrix read as `rows` rows of J entries: boxes of 32
// entries of K (128 bytes, the swizzle span) by box_rows rows, rows and K past the end read as 0.
int make_map(tt_ctx* c, CUtensorMap* tm, const float* base, int J, int rows, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return tt_fail(c, TT_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {(cuuint64_t)J, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)J * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)TG_BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return tt_fail(c, TT_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TT_OK;
}

}  // namespace

// The tensor-core Gram applies when the operands meet TMA's rules (J a multiple of 4, so that
// rows start on 16-byte boundaries; 16-byte aligned bases) and N = s rounded up to 16 is at most
// 256 (one MMA's N).
bool tt_gram_tc_fits(int J, int s, const void* SH, const void* Y) {
  return J >= TG_BK && J % 4 == 0 && s >= 1 && s <= 256 &&
         ((reinterpret_cast<uintptr_t>(SH) | reinterpret_cast<uintptr_t>(Y)) & 15) == 0;
}

// C (zeroed by the caller, or filled by the ordered reduction of the partials P) = [S H | Y]^T S H
int tt_launch_gram_tc(tt_ctx* c, const float* SH, const float* Y, int s, int n, float* C, float* P, bool split3,
                      int* nz_out) {
  GramTcArgs g;
  g.C = C;
  g.P = P;
  g.status = c->d_status;
  g.s = s;
  g.n = n;
  g.np = (s + 15) & ~15;
  g.mt_gram = (s + TG_M - 1) / TG_M;
  g.J = c->J;
  const int mt = g.mt_gram + (n + TG_M - 1) / TG_M;
  const int sms = tt_sm_count();
  // K-chunks: about one CTA per SM in all, each at least four tiles (128 entries) of K
  const int ktiles = (c->J + TG_BK - 1) / TG_BK;
  int ksplit = std::max(1, std::min(ktiles / 4, (sms + mt - 1) / mt));
  if (P) ksplit = std::min(ksplit, TT_DET_KSPLIT);
  g.kchunk = ((ktiles + ksplit - 1) / ksplit) * TG_BK;
  const int nz = (c->J + g.kchunk - 1) / g.kchunk;
  if (nz_out) *nz_out = nz;
  CUtensorMap tA, tY, tB;
  TT_TRY(make_map(c, &tA, SH, c->J, s, TG_M));
  TT_TRY(make_map(c, &tY, Y, c->J, n, TG_M));
  TT_TRY(make_map(c, &tB, SH, c->J, s, g.np));
  const size_t smem = tg_smem(g.np, split3);
  if (smem > 227 * 1024) return tt_fail(c, TT_EINVAL, "tensor-core Gram: %zu bytes of shared memory", smem);
  if (split3) {
    TT_CUDA(c, cudaFuncSetAttribute(k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gram_tc<true><<<dim3(mt, nz), TG_T, smem, c->stream>>>(tA, tY, tB, g);
  } else {
    TT_CUDA(c, cudaFuncSetAttribute(k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gram_tc<false><<<dim3(mt, nz), TG_T, smem, c->stream>>>(tA, tY, tB, g);
  }
  TT_LAUNCH(c, "k_gram_tc");
  return TT_OK;
}
