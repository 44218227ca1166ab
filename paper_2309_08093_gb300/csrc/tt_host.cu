// Host-buffer entry points: Algorithm 1's sweeps on a tensor and cores that live in host memory.
//
// tt_prox_als_sweep_host_async enqueues one call and returns: the tensor goes into one of two
// library-owned device buffers by a copy on copy_stream; then, on the context's stream after that
// copy, the cores go in, the sweeps and the relative error run, and the cores and the raw result
// sums come back (the sums into a pinned host slot). The next call copies its tensor into the
// other buffer while this call's sweeps run, so a stream of calls is bound by the host link, not
// by copy + sweep. The cores of consecutive calls stay ordered on the context's stream (a call's
// copy-in of a host core array comes after the previous call's copy-out of it). tt_host_sync waits
// for every enqueued call and turns the raw sums into rel-changes and relative errors.
// tt_prox_als_sweep_host is one asynchronous call followed by tt_host_sync.
#include <math.h>

#include <algorithm>
#include <vector>

#include "tt_internal.cuh"

// The small transfers of a call (the cores in and out, the status and result sums out) are made
// by a kernel that reads and writes page-locked host memory directly, not by the copy engines: a
// copy-out queued behind a call's sweeps would otherwise hold up the copy engine's queue, and the
// next call's tensor copy with it (measured: the pipelined step went from 1.95 to 2.42 ms).
// Pageable host arrays fall back to cudaMemcpyAsync.
struct WordCopies {
  const uint32_t* src[TT_MAX_D + 3];
  uint32_t* dst[TT_MAX_D + 3];
  int64_t words[TT_MAX_D + 3];
  int count;
};

__global__ void k_copy_words(WordCopies w) {
  for (int q = 0; q < w.count; ++q)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < w.words[q]; i += (int64_t)gridDim.x * blockDim.x)
      w.dst[q][i] = w.src[q][i];
}

// the device address of a page-locked host array (null if it is not page-locked)
static void* pinned_device_ptr(const void* h) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
    cudaGetLastError();  // clear the error of a pointer the runtime does not know
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

static int launch_copies(tt_ctx* c, const WordCopies& w) {
  int64_t most = 0;
  for (int q = 0; q < w.count; ++q) most = std::max(most, w.words[q]);
  if (!most) return TT_OK;
  k_copy_words<<<(int)std::min<int64_t>((most + 255) / 256, 64), 256, 0, c->stream>>>(w);
  TT_LAUNCH(c, "k_copy_words");
  return TT_OK;
}

// slot layout (bytes): status word (8), the two error sums (16), 2 d change sums per sweep
size_t tt_host_slot_bytes(const tt_ctx* c) { return 24 + sizeof(double) * 2 * (size_t)c->changes_cap; }

void tt_host_free(tt_ctx* c) {
  for (int b = 0; b < 2; ++b) {
    if (c->d_A_stage[b]) cudaFree(c->d_A_stage[b]);
    if (c->d_scales_stage[b]) cudaFree(c->d_scales_stage[b]);
    if (c->ev_copied[b]) cudaEventDestroy(c->ev_copied[b]);
    if (c->ev_consumed[b]) cudaEventDestroy(c->ev_consumed[b]);
    c->d_A_stage[b] = nullptr;
    c->d_scales_stage[b] = nullptr;
  }
  for (int k = 0; k < TT_MAX_D; ++k) {
    if (c->d_cores_stage[k]) cudaFree(c->d_cores_stage[k]);
    c->d_cores_stage[k] = nullptr;
  }
  for (int q = 0; q < TT_HOST_SLOTS; ++q) {
    if (c->ev_slot[q]) cudaEventDestroy(c->ev_slot[q]);
    c->ev_slot[q] = nullptr;
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->h_slots) cudaFreeHost(c->h_slots);
  c->copy_stream = nullptr;
  c->h_slots = nullptr;
}

static size_t core_bytes(const tt_ctx* c, int k) { return sizeof(float) * (size_t)c->r[k] * c->n[k] * c->r[k + 1]; }

// staging buffers, the copy stream, its events and the pinned result slots, on first use
static int host_setup(tt_ctx* c, bool scales) {
  const size_t abytes = (size_t)c->N * tt_elem_bytes(c->dtype);
  if (!c->d_A_stage[0]) {  // the staging buffers count against the workspace cap
    uint64_t extra = 2 * (abytes + sizeof(float) * c->n[0]);
    for (int k = 0; k < c->d; ++k) extra += core_bytes(c, k);
    TT_TRY(tt_check_workspace_cap(c, extra));
    for (int b = 0; b < 2; ++b) {
      TT_CUDA(c, cudaMalloc(&c->d_A_stage[b], abytes));
      TT_CUDA(c, cudaEventCreateWithFlags(&c->ev_copied[b], cudaEventDisableTiming));
      TT_CUDA(c, cudaEventCreateWithFlags(&c->ev_consumed[b], cudaEventDisableTiming));
    }
    for (int k = 0; k < c->d; ++k) TT_CUDA(c, cudaMalloc((void**)&c->d_cores_stage[k], core_bytes(c, k)));
    TT_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    TT_CUDA(c, cudaHostAlloc((void**)&c->h_slots, TT_HOST_SLOTS * tt_host_slot_bytes(c), cudaHostAllocDefault));
    for (int q = 0; q < TT_HOST_SLOTS; ++q) TT_CUDA(c, cudaEventCreateWithFlags(&c->ev_slot[q], cudaEventDisableTiming));
  }
  if (scales && !c->d_scales_stage[0])
    for (int b = 0; b < 2; ++b) TT_CUDA(c, cudaMalloc((void**)&c->d_scales_stage[b], sizeof(float) * c->n[0]));
  return TT_OK;
}

// The outputs of a finished call from its slot; its failure is kept until tt_host_sync reports it.
static void host_finish(tt_ctx* c, const tt_ctx::HostPending& p) {
  const unsigned char* slot = c->h_slots + (size_t)p.slot * tt_host_slot_bytes(c);
  const int st = *reinterpret_cast<const int*>(slot);
  const double* err = reinterpret_cast<const double*>(slot + 8);
  const double* chg = reinterpret_cast<const double*>(slot + 24);
  if (st != 0 && c->host_error == TT_OK) c->host_error = st;
  if (p.rel_error_out) *p.rel_error_out = err[1] > 0 ? sqrt(err[0] / err[1]) : 0.0;
  for (int t = 0; t < p.nsweeps && p.rel_change_out; ++t) {
    double mx = 0.0;
    for (int k = 0; k < c->d; ++k) {
      const double dd = chg[2 * (c->d * t + k)], nn = chg[2 * (c->d * t + k) + 1];
      if (nn > 0) mx = std::max(mx, sqrt(dd / nn));
    }
    p.rel_change_out[t] = mx;
  }
}

extern "C" int tt_host_sync(tt_ctx* c) {
  if (!c) return TT_EINVAL;
  TT_CUDA(c, cudaStreamSynchronize(c->stream));
  for (const tt_ctx::HostPending& p : c->pending) host_finish(c, p);
  c->pending.clear();
  const int first = c->host_error;
  c->host_error = TT_OK;
  if (first == TT_ENOTSPD) return tt_fail(c, first, "Gram matrix of the proximal update is not positive definite");
  if (first == TT_ENONFINITE) return tt_fail(c, first, "non-finite value reached the proximal solve");
  if (first != TT_OK) return tt_fail(c, first, "device status %d", first);
  return TT_OK;
}

extern "C" int tt_prox_als_sweep_host_async(tt_ctx* c, const void* A_host, const float* scales_host,
                                            float* const* cores_host, int nsweeps, uint64_t first_sweep,
                                            double* rel_change_out, double* rel_error_out) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_data(c, A_host, scales_host));
  TT_TRY(tt_check_cores(c, cores_host));
  if (nsweeps < 0) return tt_fail(c, TT_EINVAL, "nsweeps < 0");
  if (rel_change_out && nsweeps > c->changes_cap / c->d)
    return tt_fail(c, TT_EINVAL, "at most %d sweeps per call when rel-changes are requested", c->changes_cap / c->d);
  c->err.clear();
  TT_TRY(host_setup(c, scales_host != nullptr));
  if ((int)c->pending.size() == TT_HOST_SLOTS) {  // at most four calls in flight: finish the oldest
    TT_CUDA(c, cudaEventSynchronize(c->ev_slot[c->pending.front().slot]));
    host_finish(c, c->pending.front());
    c->pending.erase(c->pending.begin());
  }
  const int b = c->stage_next, slot = c->slot_next;
  c->stage_next ^= 1;
  c->slot_next = (c->slot_next + 1) % TT_HOST_SLOTS;
  const size_t abytes = (size_t)c->N * tt_elem_bytes(c->dtype);
  // the tensor, on the copy stream, once the kernels that read this buffer two calls ago are done
  if (c->consumed_recorded[b]) TT_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_consumed[b], 0));
  TT_CUDA(c, cudaMemcpyAsync(c->d_A_stage[b], A_host, abytes, cudaMemcpyHostToDevice, c->copy_stream));
  if (scales_host)
    TT_CUDA(c, cudaMemcpyAsync(c->d_scales_stage[b], scales_host, sizeof(float) * c->n[0], cudaMemcpyHostToDevice,
                               c->copy_stream));
  TT_CUDA(c, cudaEventRecord(c->ev_copied[b], c->copy_stream));
  // the cores on the context's stream (ordered after the previous call's copy-out)
  void* cores_dp[TT_MAX_D];
  bool pinned = true;
  for (int k = 0; k < c->d; ++k) pinned = pinned && (cores_dp[k] = pinned_device_ptr(cores_host[k])) != nullptr;
  if (pinned) {
    WordCopies w;
    w.count = c->d;
    for (int k = 0; k < c->d; ++k) {
      w.src[k] = static_cast<const uint32_t*>(cores_dp[k]);
      w.dst[k] = reinterpret_cast<uint32_t*>(c->d_cores_stage[k]);
      w.words[k] = (int64_t)(core_bytes(c, k) / 4);
    }
    TT_TRY(launch_copies(c, w));
  } else {
    for (int k = 0; k < c->d; ++k)
      TT_CUDA(c, cudaMemcpyAsync(c->d_cores_stage[k], cores_host[k], core_bytes(c, k), cudaMemcpyHostToDevice, c->stream));
  }
  TT_TRY(tt_reset_status(c));
  TT_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_copied[b], 0));
  const void* A = c->d_A_stage[b];
  const float* sc = scales_host ? c->d_scales_stage[b] : nullptr;
  c->y_reuse = c->det_scale_reuse = false;  // the sketches (and scale) of this call's tensor, reused by its later sweeps
  for (int t = 0; t < nsweeps; ++t) {
    double* slots = rel_change_out ? c->d_changes + (size_t)2 * c->d * t : nullptr;
    const int rc = tt_one_sweep(c, A, sc, c->d_cores_stage, first_sweep + t, slots);
    if (rc != TT_OK) {
      c->y_reuse = c->det_scale_reuse = false;
      return rc;
    }
  }
  c->y_reuse = c->det_scale_reuse = false;
  if (rel_error_out) TT_TRY(tt_launch_rel_error(c, A, sc, c->d_cores_stage, c->d_err_acc));
  TT_CUDA(c, cudaEventRecord(c->ev_consumed[b], c->stream));
  c->consumed_recorded[b] = true;
  unsigned char* hs = c->h_slots + (size_t)slot * tt_host_slot_bytes(c);  // page-locked, mapped
  WordCopies w;
  w.count = 0;
  auto add = [&](const void* src, void* dst, size_t bytes) {
    w.src[w.count] = static_cast<const uint32_t*>(src);
    w.dst[w.count] = static_cast<uint32_t*>(dst);
    w.words[w.count++] = (int64_t)(bytes / 4);
  };
  add(c->d_status, pinned_device_ptr(hs), sizeof(int));
  if (rel_error_out) add(c->d_err_acc, pinned_device_ptr(hs + 8), 2 * sizeof(double));
  if (rel_change_out && nsweeps > 0) add(c->d_changes, pinned_device_ptr(hs + 24), sizeof(double) * 2 * c->d * (size_t)nsweeps);
  if (pinned) {
    for (int k = 0; k < c->d; ++k) add(c->d_cores_stage[k], cores_dp[k], core_bytes(c, k));
  } else {
    for (int k = 0; k < c->d; ++k)
      TT_CUDA(c, cudaMemcpyAsync(cores_host[k], c->d_cores_stage[k], core_bytes(c, k), cudaMemcpyDeviceToHost, c->stream));
  }
  TT_TRY(launch_copies(c, w));
  TT_CUDA(c, cudaEventRecord(c->ev_slot[slot], c->stream));
  c->pending.push_back({rel_change_out, rel_error_out, nsweeps, slot});
  return TT_OK;
}

extern "C" int tt_prox_als_sweep_host(tt_ctx* c, const void* A_host, const float* scales_host,
                                      float* const* cores_host, int nsweeps, uint64_t first_sweep,
                                      double* rel_change_out, double* rel_error_out) {
  if (!c) return TT_EINVAL;
  const int rc = tt_prox_als_sweep_host_async(c, A_host, scales_host, cores_host, nsweeps, first_sweep,
                                              rel_change_out, rel_error_out);
  if (rc != TT_OK) {
    cudaStreamSynchronize(c->stream);  // whatever was enqueued before the failure
    c->pending.clear();
    return rc;
  }
  return tt_host_sync(c);
}
