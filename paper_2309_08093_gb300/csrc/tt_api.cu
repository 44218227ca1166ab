// Public entry points of tt_sketch.h and the sweep driver of Algorithm 1.
#include <math.h>

#include <algorithm>
#include <vector>

#include "tt_internal.cuh"

int tt_check_data(tt_ctx* c, const void* A, const float* scales) {
  if (!A) return tt_fail(c, TT_EINVAL, "null tensor pointer");
  if (c->dtype == TT_FP8E4M3 && !scales) return tt_fail(c, TT_EINVAL, "FP8 storage needs n[0] slice scales");
  if (c->dtype != TT_FP8E4M3 && scales) return tt_fail(c, TT_EINVAL, "slice scales are only used with FP8 storage");
  return TT_OK;
}

int tt_check_cores(tt_ctx* c, float* const* cores) {
  if (!cores) return tt_fail(c, TT_EINVAL, "null core array");
  for (int k = 0; k < c->d; ++k)
    if (!cores[k]) return tt_fail(c, TT_EINVAL, "null core pointer %d", k);
  return TT_OK;
}

int tt_read_status(tt_ctx* c) {
  int st = 0;
  TT_CUDA(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  TT_CUDA(c, cudaStreamSynchronize(c->stream));
  if (st == TT_ENOTSPD) return tt_fail(c, TT_ENOTSPD, "Gram matrix of the proximal update is not positive definite");
  if (st == TT_ENONFINITE) return tt_fail(c, TT_ENONFINITE, "non-finite value reached the proximal solve");
  if (st != 0) return tt_fail(c, st, "device status %d", st);
  return TT_OK;
}

int tt_reset_status(tt_ctx* c) {
  TT_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
  return TT_OK;
}

extern "C" int tt_sketch_unfold(tt_ctx* c, const void* A, const float* scales, int k, uint64_t sweep,
                                float* const* Y) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_data(c, A, scales));
  if (!Y) return tt_fail(c, TT_EINVAL, "null output array");
  if (k < -1 || k >= c->d) return tt_fail(c, TT_EINVAL, "mode %d outside [-1, %d)", k, c->d);
  for (int kk = 0; kk < c->d; ++kk)
    if ((k == -1 || k == kk) && !Y[kk]) return tt_fail(c, TT_EINVAL, "null output for mode %d", kk);
  c->err.clear();
  TT_TRY(tt_ensure_tables(c, sweep));
  if (c->det)  // fixed-point sketches of the requested modes (one scale for all)
    return tt_launch_unfold_det(c, A, scales, k == -1 ? (1u << c->d) - 1u : 1u << k, Y);
  for (int kk = 0; kk < c->d; ++kk)
    if (k == -1 || k == kk) TT_TRY(tt_launch_unfold(c, A, scales, kk, Y[kk]));
  return TT_OK;
}

extern "C" int tt_sketch_unfold_coo(tt_ctx* c, const int32_t* idx, const float* val, int64_t nnz, int k,
                                    uint64_t sweep, float* const* Y) {
  if (!c) return TT_EINVAL;
  if (nnz < 0) return tt_fail(c, TT_EINVAL, "nnz < 0");
  if (nnz > 0 && (!idx || !val)) return tt_fail(c, TT_EINVAL, "null coordinates or values");
  if (!Y) return tt_fail(c, TT_EINVAL, "null output array");
  if (k < -1 || k >= c->d) return tt_fail(c, TT_EINVAL, "mode %d outside [-1, %d)", k, c->d);
  for (int kk = 0; kk < c->d; ++kk)
    if ((k == -1 || k == kk) && !Y[kk]) return tt_fail(c, TT_EINVAL, "null output for mode %d", kk);
  c->err.clear();
  TT_TRY(tt_ensure_tables(c, sweep));
  TT_TRY(tt_reset_status(c));
  TT_TRY(tt_launch_unfold_coo(c, idx, val, nnz, k, Y));
  const int rc = tt_read_status(c);  // synchronises
  if (rc == TT_EINVAL) return tt_fail(c, TT_EINVAL, "a coordinate lies outside its mode size (entry skipped)");
  return rc;
}

static int build_all_ghat(tt_ctx* c, float* const* cores) { return tt_launch_core_ffts(c, cores); }

extern "C" int tt_sketch_interface(tt_ctx* c, float* const* cores, int k, uint64_t sweep, float* SH) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_cores(c, cores));
  if (!SH) return tt_fail(c, TT_EINVAL, "null output");
  if (k < 0 || k >= c->d) return tt_fail(c, TT_EINVAL, "mode %d outside [0, %d)", k, c->d);
  c->err.clear();
  TT_TRY(tt_ensure_tables(c, sweep));
  TT_TRY(build_all_ghat(c, cores));
  TT_TRY(tt_launch_suffixes(c));  // also restarts the prefix chain
  for (int j = 0; j < k; ++j) TT_TRY(tt_launch_prefix_step(c, j));
  TT_TRY(tt_launch_interface_from_chain(c, k, SH));
  return TT_OK;
}

extern "C" int tt_prox_update(tt_ctx* c, const float* Y, const float* SH, float* core, int k) {
  if (!c) return TT_EINVAL;
  if (!Y || !SH || !core) return tt_fail(c, TT_EINVAL, "null pointer");
  if (k < 0 || k >= c->d) return tt_fail(c, TT_EINVAL, "mode %d outside [0, %d)", k, c->d);
  c->err.clear();
  TT_TRY(tt_reset_status(c));
  TT_TRY(tt_launch_prox_update(c, Y, SH, core, k, nullptr));
  return tt_read_status(c);
}

extern "C" int tt_orthogonalize(tt_ctx* c, float* const* cores, int direction, int k) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_cores(c, cores));
  c->err.clear();
  TT_TRY(tt_reset_status(c));
  if (direction == -1) {
    TT_TRY(tt_launch_lq_sweep(c, cores));
  } else if (direction == 1) {
    if (k < 0 || k >= c->d - 1) return tt_fail(c, TT_EINVAL, "QR step needs 0 <= k < d-1 (k=%d)", k);
    TT_TRY(tt_launch_qr_left(c, cores[k], cores[k + 1], k));
  } else {
    return tt_fail(c, TT_EINVAL, "direction must be -1 or +1");
  }
  return tt_read_status(c);
}

// One outer iteration of Algorithm 1; change slots receive ||dG_k||^2, ||G_k||^2 per core.
static int sweep_body(tt_ctx* c, const void* A, const float* scales, float* const* cores, uint64_t sweep,
                      double* change_slots, float* const* Ygiven) {
  const int d = c->d;
  TT_TRY(tt_ensure_tables(c, sweep));
  // The data sketches Y_k do not depend on the cores: all d of them are launched now on the side
  // stream (plans built there too) and run concurrently with the orthogonalisation, interface
  // and solve kernels below, which use few SMs; core k's update waits only for Y_k.
  const bool fork = Ygiven == nullptr;
  // a fixed draw: the data sketches depend on A alone, so the call's first sweep computes them and
  // its later sweeps reuse them (the chain's waits on the Y_k events of that sweep are met)
  const bool fixed_draw = ((c->flags & TT_FLAG_FIXED_SKETCH) != 0 || c->user_tables) && !c->capture_mode;
  if (fork && !c->y_reuse) {
    TT_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
    TT_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    cudaStream_t main_stream = c->stream;
    c->stream = c->side;
    c->in_sweep = true;
    int rc = TT_OK;
    if (c->det) {  // every mode in fixed point (one scale for all), Y_k's event as it is done
      float* ys[TT_MAX_D];
      for (int k = 0; k < d; ++k) ys[k] = c->d_Yall + c->yoff[k];
      rc = tt_launch_unfold_det(c, A, scales, (1u << d) - 1u, ys, c->ev_y);
      if (rc == TT_OK && !c->capture_mode) c->det_scale_reuse = true;
    }
    for (int k = 0; k < d && rc == TT_OK && !c->det; ++k) {
      rc = tt_launch_unfold(c, A, scales, k, c->d_Yall + c->yoff[k]);
      if (rc == TT_OK) {
        const cudaError_t e = cudaEventRecord(c->ev_y[k], c->side);
        if (e != cudaSuccess) rc = tt_cuda_check(c, e, "cudaEventRecord");
      }
    }
    c->stream = main_stream;
    c->in_sweep = false;
    if (rc == TT_OK && fixed_draw) c->y_reuse = true;
    // the next sweep's draw and plans, behind this sweep's data sketches on the side stream (not
    // joined: it overlaps the rest of this sweep and whatever the caller does next)
    if (rc == TT_OK) rc = tt_prepare_next_draw(c, sweep + 1);
    if (rc != TT_OK) {
      cudaEventRecord(c->ev_fork, c->side);  // join whatever was launched before returning
      cudaStreamWaitEvent(c->stream, c->ev_fork, 0);
      return rc;
    }
  }
  auto chain = [&]() -> int {
    TT_TRY(tt_launch_lq_sweep(c, cores));
    TT_TRY(build_all_ghat(c, cores));
    TT_TRY(tt_launch_suffixes(c));  // also restarts the prefix chain
    for (int k = 0; k < d; ++k) {
      // the interface kernel also zeroes the Gram accumulators of this core's update
      const int64_t sk = (int64_t)c->r[k] * c->r[k + 1];
      if (c->solve64)
        TT_TRY(tt_launch_interface_from_chain(c, k, c->d_SH, reinterpret_cast<float*>(c->d_gram64),
                                              2 * (sk + c->n[k]) * sk));
      else
        TT_TRY(tt_launch_interface_from_chain(c, k, c->d_SH, c->d_gram, (sk + c->n[k]) * sk));
      const float* Yk = fork ? c->d_Yall + c->yoff[k] : Ygiven[k];
      if (fork) TT_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_y[k], 0));
      TT_TRY(tt_launch_prox_update(c, Yk, c->d_SH, cores[k], k, change_slots ? change_slots + 2 * k : nullptr,
                                   true));
      if (k < d - 1) {
        TT_TRY(tt_launch_qr_left(c, cores[k], cores[k + 1], k));
        TT_TRY(tt_launch_core_fft(c, cores[k], k));
        TT_TRY(tt_launch_prefix_step(c, k));
      }
    }
    return TT_OK;
  };
  const int rc = chain();
  if (fork) TT_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_y[d - 1], 0));  // joined on every path
  return rc;
}

// One outer iteration of Algorithm 1 on the context's high-priority stream, ordered after the
// caller's stream and joined back into it on every return path.
int tt_one_sweep(tt_ctx* c, const void* A, const float* scales, float* const* cores, uint64_t sweep,
                 double* change_slots, float* const* Ygiven) {
  cudaStream_t caller = c->stream;
  TT_CUDA(c, cudaEventRecord(c->ev_in, caller));
  TT_CUDA(c, cudaStreamWaitEvent(c->hi, c->ev_in, 0));
  c->stream = c->hi;
  const int rc = sweep_body(c, A, scales, cores, sweep, change_slots, Ygiven);
  c->stream = caller;
  TT_CUDA(c, cudaEventRecord(c->ev_out, c->hi));
  TT_CUDA(c, cudaStreamWaitEvent(caller, c->ev_out, 0));
  return rc;
}

extern "C" int tt_prox_als_sweep_sketched(tt_ctx* c, float* const* Y, float* const* cores, uint64_t sweep) {
  if (!c) return TT_EINVAL;
  if (!Y) return tt_fail(c, TT_EINVAL, "null sketch array");
  for (int k = 0; k < c->d; ++k)
    if (!Y[k]) return tt_fail(c, TT_EINVAL, "null sketch pointer %d", k);
  TT_TRY(tt_check_cores(c, cores));
  c->err.clear();
  TT_TRY(tt_reset_status(c));
  TT_TRY(tt_one_sweep(c, nullptr, nullptr, cores, sweep, nullptr, Y));
  return tt_read_status(c);
}

// nsweeps outer iterations; per sweep (optional) the rel-change and the relative error of the
// updated cores, copied back in blocks of changes_cap / d sweeps with one synchronisation each.
static int run_sweeps_body(tt_ctx* c, const void* A, const float* scales, float* const* cores, int nsweeps,
                           uint64_t first_sweep, double* rel_change_out, double* rel_error_out);

static int run_sweeps(tt_ctx* c, const void* A, const float* scales, float* const* cores, int nsweeps,
                      uint64_t first_sweep, double* rel_change_out, double* rel_error_out) {
  c->y_reuse = c->det_scale_reuse = false;  // reused within one call only (A may change between calls)
  const int rc = run_sweeps_body(c, A, scales, cores, nsweeps, first_sweep, rel_change_out, rel_error_out);
  c->y_reuse = c->det_scale_reuse = false;
  return rc;
}

static int run_sweeps_body(tt_ctx* c, const void* A, const float* scales, float* const* cores, int nsweeps,
                           uint64_t first_sweep, double* rel_change_out, double* rel_error_out) {
  TT_TRY(tt_reset_status(c));
  const int per_block = c->changes_cap / c->d;
  std::vector<double> host, herr;
  for (int t0 = 0; t0 < nsweeps; t0 += per_block) {
    const int nt = std::min(per_block, nsweeps - t0);
    for (int t = 0; t < nt; ++t) {
      double* slots = rel_change_out ? c->d_changes + (size_t)2 * c->d * t : nullptr;
      TT_TRY(tt_one_sweep(c, A, scales, cores, first_sweep + t0 + t, slots));
      if (rel_error_out) TT_TRY(tt_launch_rel_error(c, A, scales, cores, c->d_errs + 2 * t));
    }
    if (rel_change_out) {
      host.resize((size_t)2 * c->d * nt);
      TT_CUDA(c, cudaMemcpyAsync(host.data(), c->d_changes, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, c->stream));
    }
    if (rel_error_out) {
      herr.resize((size_t)2 * nt);
      TT_CUDA(c, cudaMemcpyAsync(herr.data(), c->d_errs, sizeof(double) * herr.size(), cudaMemcpyDeviceToHost, c->stream));
    }
    if (rel_change_out || rel_error_out) {
      TT_TRY(tt_read_status(c));  // synchronises
      for (int t = 0; t < nt && rel_change_out; ++t) {
        double mx = 0.0;
        for (int k = 0; k < c->d; ++k) {
          double dd = host[(size_t)2 * (c->d * t + k)], nn = host[(size_t)2 * (c->d * t + k) + 1];
          if (nn > 0) mx = std::max(mx, sqrt(dd / nn));
        }
        rel_change_out[t0 + t] = mx;
      }
      for (int t = 0; t < nt && rel_error_out; ++t)
        rel_error_out[t0 + t] = herr[2 * t + 1] > 0 ? sqrt(herr[2 * t] / herr[2 * t + 1]) : 0.0;
    }
  }
  if (!rel_change_out && !rel_error_out) {
    // surface a failed solve (one synchronisation at the end of the call)
    int st = 0;
    TT_CUDA(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (st != 0) return tt_read_status(c);
  }
  return TT_OK;
}

extern "C" int tt_prox_als_sweep(tt_ctx* c, const void* A, const float* scales, float* const* cores,
                                 int nsweeps, uint64_t first_sweep, double* rel_change_out) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_data(c, A, scales));
  TT_TRY(tt_check_cores(c, cores));
  if (nsweeps < 0) return tt_fail(c, TT_EINVAL, "nsweeps < 0");
  c->err.clear();
  return run_sweeps(c, A, scales, cores, nsweeps, first_sweep, rel_change_out, nullptr);
}

extern "C" int tt_prox_als_sweep_monitored(tt_ctx* c, const void* A, const float* scales, float* const* cores,
                                           int nsweeps, uint64_t first_sweep, double* rel_change_out,
                                           double* rel_error_out) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_data(c, A, scales));
  TT_TRY(tt_check_cores(c, cores));
  if (nsweeps < 0) return tt_fail(c, TT_EINVAL, "nsweeps < 0");
  if (!rel_error_out) return tt_fail(c, TT_EINVAL, "null rel_error_out");
  c->err.clear();
  return run_sweeps(c, A, scales, cores, nsweeps, first_sweep, rel_change_out, rel_error_out);
}

extern "C" int tt_rel_error_coo(tt_ctx* c, const int32_t* idx, const float* val, int64_t nnz,
                                float* const* cores, double* out) {
  if (!c) return TT_EINVAL;
  if (nnz < 0) return tt_fail(c, TT_EINVAL, "nnz < 0");
  if (nnz > 0 && (!idx || !val)) return tt_fail(c, TT_EINVAL, "null coordinates or values");
  TT_TRY(tt_check_cores(c, cores));
  if (!out) return tt_fail(c, TT_EINVAL, "null output");
  c->err.clear();
  TT_TRY(tt_reset_status(c));
  TT_TRY(tt_launch_rel_error_coo(c, idx, val, nnz, cores));
  double h[3];
  TT_CUDA(c, cudaMemcpyAsync(h, c->d_err_acc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  const int rc = tt_read_status(c);  // synchronises
  if (rc == TT_EINVAL) return tt_fail(c, TT_EINVAL, "a coordinate lies outside its mode size (entry skipped)");
  TT_TRY(rc);
  const double e2 = h[0] - 2.0 * h[1] + h[2];
  *out = h[0] > 0 ? sqrt(std::max(0.0, e2) / h[0]) : 0.0;
  return TT_OK;
}

extern "C" int tt_rel_error(tt_ctx* c, const void* A, const float* scales, float* const* cores, double* out) {
  if (!c) return TT_EINVAL;
  TT_TRY(tt_check_data(c, A, scales));
  TT_TRY(tt_check_cores(c, cores));
  if (!out) return tt_fail(c, TT_EINVAL, "null output");
  c->err.clear();
  TT_TRY(tt_launch_rel_error(c, A, scales, cores));
  double h[2];
  TT_CUDA(c, cudaMemcpyAsync(h, c->d_err_acc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  TT_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = (h[1] > 0) ? sqrt(h[0] / h[1]) : 0.0;
  return TT_OK;
}

// ---------------------------------------------------------------------------------------------
// host-buffer sweep

int tt_elem_bytes(int dtype) {
  switch (dtype) {
    case TT_F64: return 8;
    case TT_F32: return 4;
    case TT_BF16: return 2;
    default: return 1;
  }
}

// ---------------------------------------------------------------------------------------------
// measurement counters

int tt_prof_begin(tt_ctx* c, int k) {
  if (!c->profiling) return TT_OK;
  while ((int)c->ev_pool.size() < c->ev_used + 2) {
    cudaEvent_t e;
    TT_CUDA(c, cudaEventCreate(&e));
    c->ev_pool.push_back(e);
  }
  TT_CUDA(c, cudaEventRecord(c->ev_pool[c->ev_used], c->stream));
  c->ev_mode.push_back(k);
  c->ev_used += 1;
  return TT_OK;
}

int tt_prof_end(tt_ctx* c) {
  if (!c->profiling) return TT_OK;
  TT_CUDA(c, cudaEventRecord(c->ev_pool[c->ev_used], c->stream));
  c->ev_used += 1;
  // algorithmic bytes of one data-sketch launch: every entry once, plus the FP8 slice scales
  c->prof_bytes += (int64_t)c->N * tt_elem_bytes(c->dtype) + (c->dtype == TT_FP8E4M3 ? 4 * c->n[0] : 0);
  return TT_OK;
}

extern "C" int tt_profile_enable(tt_ctx* c, int on) {
  if (!c) return TT_EINVAL;
  if (on) {
    TT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->ev_used = 0;
    c->ev_mode.clear();
    c->prof_bytes = 0;
    c->launches = 0;
  }
  c->profiling = on != 0;
  return TT_OK;
}

extern "C" int tt_profile_read(tt_ctx* c, tt_profile* out) {
  if (!c || !out) return TT_EINVAL;
  TT_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = tt_profile{};
  for (int i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    TT_CUDA(c, cudaEventElapsedTime(&ms, c->ev_pool[i], c->ev_pool[i + 1]));
    int k = c->ev_mode[i / 2];
    out->unfold_ms += ms;
    out->unfold_launches += 1;
    if (k >= 0 && k < 8) {
      out->mode_ms[k] += ms;
      out->mode_launches[k] += 1;
    }
  }
  out->unfold_bytes = c->prof_bytes;
  out->kernel_launches = c->launches;
  return TT_OK;
}
