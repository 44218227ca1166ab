// Part (a): Y_k = S A_(k)^T, the TensorSketch of every mode-k unfolding (Alg. 1, Sec. 3).
//
// Y_k[b, i_k] = sum over entries with that i_k of prod_{s!=k} v_s(i_s) * A(i), restricted to
// (sum_{s!=k} h_s(i_s)) mod J = b  (Eqs. (eqn_h), (eqn_v)).
//
// Both kernels read A only as whole mode-0 fibres (contiguous runs of n_0 entries), gathered with
// 16-byte loads in the order of a small per-sweep plan (tt_context.cu) and summed in registers.
//
// Mode 0: every fibre A(:, i_1, ..., i_{d-1}) lands in ONE row c = (sum_{s>=1} h_s(i_s)) mod J of
// Y_0, so Y_0[c, :] = sum_{fibres with hash c} sign * fibre.
//
// Modes k >= 1: with Z_k[i_0, c] = sum over the fibres r of the modes != 0, k with hash c_r = c
// of sign_r * A(i_0, r, i_k), the TensorSketch definition regroups to
//     Y_k[b, i_k] = sum_{i_0} v_0(i_0) Z_k[i_0, (b - h_0(i_0)) mod J],
// i.e. column i_k is a sum of n_0 circularly rolled rows of Z_k.
//
// The plan of mode k (tt_context.cu) lists the fibres at i_k = 0 grouped by their tail hash c, so
// fibres of equal c are walked one after the other and summed in registers (a "run"), and a run's
// sum is flushed once:
//   k_unfold_gather (mode 0; modes >= 1 when the kernel below does not apply): one output column
//     per work item; the item's fibres are split over (warp, fibre slot) pairs, several short
//     fibres per warp; mode 0 writes a finished run as row c of Y_0, modes >= 1 add
//     coef(i_0) * run into bucket (c + h_0(i_0)) mod J of the CTA's column copy;
//   k_unfold_cols (modes >= 1): G = 4 neighbouring columns per work item, one plan entry (four
//     fibres) per warp step, every lane on the same entries, so runs end together across the warp.
// Fibres are staged with cp.async rings (S fibres in flight per slot) in VB-byte vectors, VB the
// widest that both the fibre length and A's base allow. Column copies live in shared memory and
// are added to Y_k (column-major, J x n_k) with 16-byte vector atomics at the end of an item.
// Fibres on a 1-, 2- or 4-byte grid take the window-staging kernels of tt_unfold_win.cu instead.
#include <algorithm>

#include "tt_gather.cuh"


// Modes >= 1 with G columns per item: VB-byte vectors, S entries in flight, MV vectors per lane;
// returns false (nothing launched) when the shape does not suit it. 16-byte vectors take the
// smallest MV that covers an entry (up to 4); fibres whose length is not a multiple of 16 bytes
// (8- or 4-byte vectors) take MV = 16 / EPV, every lane holding up to 16 elements (so the plan is
// walked once per item and 128 bytes per lane stay in flight, rather than one 4-byte vector per
// lane and a walk of the plan per 32 of them).
template <int DT, int VB, int S>
static int launch_cols_s(tt_ctx* c, const void* A, const float* scales, int k, float* Y, bool* done, size_t smax) {
  *done = false;
  constexpr int G = 4, THREADS = 256;
  constexpr int EB = TtElem<DT>::bytes;
  const int64_t fiber_bytes = (int64_t)c->n[0] * EB;
  const int vpf = (int)(fiber_bytes / VB);
  const int mv = (G * vpf + 31) / 32;
  constexpr int EPV = TtVec<DT, VB>::EPV;
  constexpr int MV_MAX = VB == 16 ? 4 : 16 / EPV;
  if (mv > MV_MAX || mv * EPV > 16 || (c->J & 3) != 0) return TT_OK;  // at most 16 elements per lane
  GArgs a;
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
  a.ncol = (int)c->n[k];
  a.col_fibres = c->stride[k] / c->n[0];
  a.total_bytes = c->N * EB;
  a.fg = fibre_geom(fiber_bytes, VB, 1);
  const int sms = tt_sm_count();
  const int ncolg = (a.ncol + G - 1) / G;
  const int slots = 2 * sms;
  // one item per CTA slot; four times as many beside the chain (shorter CTAs hand SM slots to
  // the chain kernels sooner; measured best of 1, 2, 4, 8 at 100^4)
  int nseg = std::max(1, slots / ncolg);
  if (c->in_sweep) nseg *= 4;
  a.nseg = tt_unfold_nseg(c, ncolg, nseg);
  a.segmax = (c->J + a.nseg - 1) / a.nseg + 1;
  const size_t smem = gather_ring_bytes(true, THREADS / 32, S * MV_MAX, VB) + sizeof(float) * (size_t)G * (c->J + TT_YPAD) +
                      sizeof(int) * (2 * (size_t)a.segmax + 1);
  if (smem > smax) return TT_OK;
  *done = true;
  TT_CUDA(c, cudaMemsetAsync(Y, 0, sizeof(float) * c->J * c->n[k], c->stream));
  void (*kern)(GArgs) = k_unfold_cols<DT, VB, S, MV_MAX, G>;
  if constexpr (VB == 16) {
    kern = k_unfold_cols<DT, VB, S, 1, G>;
    if constexpr (2 * EPV <= 16)
      if (mv == 2) kern = k_unfold_cols<DT, VB, S, 2, G>;
    if constexpr (3 * EPV <= 16)
      if (mv == 3) kern = k_unfold_cols<DT, VB, S, 3, G>;
    if constexpr (4 * EPV <= 16)
      if (mv == 4) kern = k_unfold_cols<DT, VB, S, 4, G>;
  }
  TT_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int items = ncolg * a.nseg;
  kern<<<std::max(1, items), THREADS, smem, c->stream>>>(a);
  TT_LAUNCH(c, "k_unfold_cols");
  return TT_OK;
}

template <int DT, int VB>
static int launch_cols(tt_ctx* c, const void* A, const float* scales, int k, float* Y, bool* done) {
  return launch_cols_s<DT, VB, 2>(c, A, scales, k, Y, done, 113 * 1024);  // two CTAs per SM
}

// ---------------------------------------------------------------------------------------------
// host side


// S fibres in flight per slot (S * M pieces of VB bytes per lane); ONE_CTA: the in-sweep mode-0
// shape that runs one CTA per SM beside the chain
template <int DT, int VB, int M, bool MODE0, int S = 12 / M, bool ONE_CTA = false>
static int launch_gather_vbm(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  constexpr int THREADS = 256;
  GArgs a;
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
  a.ncol = MODE0 ? 1 : (int)c->n[k];
  a.col_fibres = MODE0 ? 0 : c->stride[k] / c->n[0];
  a.total_bytes = c->N * TtElem<DT>::bytes;
  a.fg = fibre_geom((int64_t)c->n[0] * TtElem<DT>::bytes, VB, M);
  const int sms = tt_sm_count();
  // work items (column, c-segment): at most one per CTA slot (two CTAs per SM) when the columns
  // allow it, so that every CTA gets the same amount of work; segments of at most 2048 c groups
  // CTAs per SM: two (the kernel is latency-bound and needs the warps), also when the sweep runs
  // the sketches beside the chain kernels
  const int cps = c->tune_cta_per_sm[k] ? c->tune_cta_per_sm[k] : 2;
  const int slots = cps * sms;
  int nseg = std::max(1, slots / a.ncol);
  if (c->tune_seg_mult[k]) nseg *= c->tune_seg_mult[k];
  else if (c->in_sweep) nseg *= 4;  // beside the chain: short CTAs free SM slots often
  a.nseg = tt_unfold_nseg(c, a.ncol, nseg);
  a.segmax = (c->J + a.nseg - 1) / a.nseg + 1;
  const size_t ring = gather_ring_bytes(VB >= 4, THREADS / 32, S * M, VB);
  const size_t smem = ring + sizeof(float) * (MODE0 ? 0 : c->J) + sizeof(int) * (2 * (size_t)a.segmax + 1);
  if (smem > 220 * 1024) return tt_fail(c, TT_EINVAL, "gather kernel needs %zu bytes of shared memory", smem);
  TT_CUDA(c, cudaMemsetAsync(Y, 0, sizeof(float) * c->J * c->n[k], c->stream));  // empty groups stay 0
  // ONE_CTA: beside the chain of a single-tensor sweep, the mode-0 kernel with packed fibres (four
  // or more slots per warp) runs one CTA per SM (its shared-memory request is raised to more than
  // half an SM's): the packed slots keep enough bytes in flight, and the registers and shared
  // memory of the second CTA stay free for the chain kernels, which otherwise wait for sketch CTAs
  // to leave (measured at 100^4: -5% per step). Not in graph capture, where other tensors share
  // the SMs.
  const size_t smem_l = ONE_CTA ? std::max(smem, (size_t)116 * 1024) : smem;
  TT_CUDA(c, cudaFuncSetAttribute(k_unfold_gather<DT, VB, S, M, MODE0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l));
  int per_sm = 1;
  TT_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_unfold_gather<DT, VB, S, M, MODE0>, THREADS, smem));
  const int items = a.ncol * a.nseg;
  // one CTA per item inside a sweep (the scheduler hands freed slots to the high-priority chain
  // first); otherwise at most one wave
  const int blocks = (c->in_sweep && !c->tune_seg_mult[k])
                         ? std::max(1, items)
                         : std::max(1, std::min(items, sms * std::max(1, std::min(per_sm, cps))));
  k_unfold_gather<DT, VB, S, M, MODE0><<<blocks, THREADS, smem_l, c->stream>>>(a);
  TT_LAUNCH(c, "k_unfold_gather");
  return TT_OK;
}

template <int DT, int VB, bool MODE0>
static int launch_gather_vb(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  if constexpr (!MODE0 && (VB == 4 || VB == 8 || VB == 16) && VB >= TtElem<DT>::bytes) {
    if (!c->tune_seg_mult[k]) {  // the autotuner times the one-column kernel's granularities
      bool done = false;
      const int rc = launch_cols<DT, VB>(c, A, scales, k, Y, &done);
      if (rc != TT_OK || done) return rc;
    }
  }
  // Several fibres per warp pay off in mode 0, whose runs are long (one flush per row); in modes
  // >= 1 a run is a few fibres and the fibre slots of a warp would flush divergently.
  if constexpr ((VB == 16 || VB == 8 || VB == 4) && VB >= TtElem<DT>::bytes && MODE0) {
    constexpr int EPV = TtVec<DT, VB>::EPV;  // pick_m keeps M * EPV <= 16: only those are compiled
    const int m = pick_m((int)(c->n[0] * TtElem<DT>::bytes / VB), EPV);
    if constexpr (4 * EPV <= 16) {
      if (m == 4) {
        const FibreGeom fg = fibre_geom((int64_t)c->n[0] * TtElem<DT>::bytes, VB, 4);
        // beside the chain of a single-tensor sweep: one CTA per SM with six fibres in flight per
        // slot instead of three (measured at 100^4: sweep 671 -> 655 us; 4 stages: 661 us)
        if (c->in_sweep && !c->capture_mode && fg.fpi >= 4)
          return launch_gather_vbm<DT, VB, 4, MODE0, 6, true>(c, A, scales, k, Y);
        return launch_gather_vbm<DT, VB, 4, MODE0>(c, A, scales, k, Y);
      }
    }
    if constexpr (2 * EPV <= 16)
      if (m == 2) return launch_gather_vbm<DT, VB, 2, MODE0>(c, A, scales, k, Y);
    return launch_gather_vbm<DT, VB, 1, MODE0>(c, A, scales, k, Y);
  } else {
    if constexpr (!MODE0 && VB >= 4 && VB >= TtElem<DT>::bytes) {
      // one fibre per warp covered by one pass of the plan: M vectors per lane (M * EPV <= 16)
      constexpr int EPV = TtVec<DT, VB>::EPV;
      const int vpf = (int)(c->n[0] * TtElem<DT>::bytes / VB);
      if constexpr (4 * EPV <= 16)
        if (vpf > 64 && vpf <= 128) return launch_gather_vbm<DT, VB, 4, MODE0>(c, A, scales, k, Y);
      if constexpr (2 * EPV <= 16)
        if (vpf > 32 && vpf <= 64) return launch_gather_vbm<DT, VB, 2, MODE0>(c, A, scales, k, Y);
    }
    return launch_gather_vbm<DT, VB, 1, MODE0>(c, A, scales, k, Y);
  }
}

template <int DT, bool MODE0>
static int launch_gather(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  constexpr int EB = TtElem<DT>::bytes;
  const int vb = pick_vb((int64_t)c->n[0] * EB, (uintptr_t)A, EB);
  if (vb <= 4 && ((int64_t)c->n[0] * EB) % 16 != 0) {
    // fibres on a 1-, 2- or 4-byte grid: window staging keeps every copy 16 bytes wide (on an
    // 8-byte grid the 8-byte vectors measured as fast for FP32 and faster for BF16)
    bool done = false;
    const int rc = tt_launch_unfold_win(c, A, scales, k, Y, &done);
    if (rc != TT_OK || done) return rc;
  }
  switch (vb) {
    case 16: return launch_gather_vb<DT, 16, MODE0>(c, A, scales, k, Y);
    case 8: return launch_gather_vb<DT, (EB <= 8 ? 8 : 16), MODE0>(c, A, scales, k, Y);
    case 4: return launch_gather_vb<DT, (EB <= 4 ? 4 : 16), MODE0>(c, A, scales, k, Y);
    case 2: return launch_gather_vb<DT, (EB <= 2 ? 2 : 16), MODE0>(c, A, scales, k, Y);
    default: return launch_gather_vb<DT, (EB <= 1 ? 1 : 16), MODE0>(c, A, scales, k, Y);
  }
}

template <int DT>
static int unfold_dt(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  if (k == 0) return launch_gather<DT, true>(c, A, scales, k, Y);
  return launch_gather<DT, false>(c, A, scales, k, Y);
}

// ---------------------------------------------------------------------------------------------
// sparse tensors in coordinate form (Sec. 3, the discussion after Theorem 3: for sparse A the
// sketch of the unfolding costs O(nnz)). Entry e, with indices i_s = idx[s nnz + e] and value
// val[e], adds prod_{s != k} v_s(i_s) val[e] to Y_k[(sum_{s != k} h_s(i_s)) mod J, i_k] for every
// requested mode k. One thread per entry (grid-stride): the index loads of a warp are coalesced
// (mode-major indices), the hash and sign lookups hit the small per-mode tables, and the adds are
// FP32 atomics into the J x n_k sketches (L2-resident at the sizes of interest). The per-mode
// values live in registers: the loops over modes run to TT_MAX_D with a predicate. An index
// outside [0, n_s) skips its entry and raises TT_EINVAL in the device status.

struct CooArgs {
  const int32_t* idx;
  const float* val;
  int64_t nnz;
  int d, J;
  const int32_t* h;
  const int8_t* v;
  int64_t noff[TT_MAX_D + 1];
  int64_t n[TT_MAX_D];
  float* Y[TT_MAX_D];  // null: mode not requested
  int* status;
};

__global__ void __launch_bounds__(256) k_unfold_coo(CooArgs a) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.nnz; e += (int64_t)gridDim.x * blockDim.x) {
    int ii[TT_MAX_D], hh[TT_MAX_D];
    bool ng[TT_MAX_D];
    int H = 0;
    bool neg = false, bad = false;
#pragma unroll
    for (int s = 0; s < TT_MAX_D; ++s) {
      ii[s] = 0;
      hh[s] = 0;
      ng[s] = false;
      if (s < a.d) {
        const int i = __ldg(a.idx + (int64_t)s * a.nnz + e);
        if (i < 0 || i >= a.n[s]) {
          bad = true;
        } else {
          ii[s] = i;
          hh[s] = __ldg(a.h + a.noff[s] + i);
          ng[s] = __ldg(a.v + a.noff[s] + i) < 0;
          H += hh[s];
          neg ^= ng[s];
        }
      }
    }
    if (bad) {
      atomicCAS(a.status, 0, TT_EINVAL);
      continue;
    }
    const float x = __ldg(a.val + e);
#pragma unroll
    for (int k = 0; k < TT_MAX_D; ++k) {
      if (k < a.d && a.Y[k]) {
        int b = H - hh[k];  // sum over s != k: below (d - 1) J
        while (b >= a.J) b -= a.J;
        atomicAdd(a.Y[k] + b + (int64_t)a.J * ii[k], (neg != ng[k]) ? -x : x);
      }
    }
  }
}

int tt_launch_unfold_coo(tt_ctx* c, const int32_t* idx, const float* val, int64_t nnz, int k, float* const* Y) {
  CooArgs a;
  a.idx = idx;
  a.val = val;
  a.nnz = nnz;
  a.d = c->d;
  a.J = c->J;
  a.h = c->d_h;
  a.v = c->d_v;
  a.status = c->d_status;
  for (int s = 0; s <= c->d; ++s) a.noff[s] = c->noff[s];
  for (int s = 0; s < TT_MAX_D; ++s) {
    a.n[s] = s < c->d ? c->n[s] : 1;
    a.Y[s] = (s < c->d && (k == -1 || k == s)) ? Y[s] : nullptr;
    if (a.Y[s]) TT_CUDA(c, cudaMemsetAsync(a.Y[s], 0, sizeof(float) * (size_t)c->J * c->n[s], c->stream));
  }
  if (nnz == 0) return TT_OK;
  const int sms = tt_sm_count();
  const int64_t blocks = std::min<int64_t>((nnz + 255) / 256, (int64_t)sms * 8);
  k_unfold_coo<<<(int)blocks, 256, 0, c->stream>>>(a);
  TT_LAUNCH(c, "k_unfold_coo");
  return TT_OK;
}

int tt_launch_unfold(tt_ctx* c, const void* A, const float* scales, int k, float* Y) {
  if (c->det) {  // the fixed-point sketch of this mode alone
    float* ys[TT_MAX_D] = {nullptr};
    ys[k] = Y;
    return tt_launch_unfold_det(c, A, scales, 1u << k, ys);
  }
  int rc = tt_ensure_rplan(c, k);  // plan build is not part of the timed kernel
  if (rc) return rc;
  rc = tt_prof_begin(c, k);
  if (rc) return rc;
  switch (c->dtype) {
    case TT_F64: rc = unfold_dt<TT_F64>(c, A, scales, k, Y); break;
    case TT_F32: rc = unfold_dt<TT_F32>(c, A, scales, k, Y); break;
    case TT_BF16: rc = unfold_dt<TT_BF16>(c, A, scales, k, Y); break;
    default: rc = unfold_dt<TT_FP8E4M3>(c, A, scales, k, Y); break;
  }
  if (rc) return rc;
  return tt_prof_end(c);
}
