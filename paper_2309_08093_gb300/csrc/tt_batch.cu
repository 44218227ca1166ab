// Batched driver: many independent tensors (each with its own shape, ranks and sketch size) swept
// together. One sweep of Algorithm 1 for every tensor is captured once into a CUDA graph (tensor i
// runs on stream i mod S of a stream pool, S = 64, forked from and joined to the caller's stream),
// and every later sweep is a single cudaGraphLaunch. The sweep index lives in a device counter that
// the graph increments, so each replay draws the next sketch (Alg. 1 redraws S_k per outer
// iteration). Tensors with a fixed draw (TT_FLAG_FIXED_SKETCH) also get a second graph, replayed
// for a call's sweeps after its first, in which they reuse the data sketches that the first sweep
// left in their contexts.
// The data-sketch launches of a batched tensor size their work items by its bytes
// (TT_BATCH_ITEM_BYTES), so that a small tensor's launch takes few CTAs and those of other tensors
// run beside it. With TT_FLAG_BATCH_AUTOTUNE an autotuner times, per mode and on the tensor's own
// data before the first capture, the default launch and the one-column kernel at a few work-item
// granularities and CTA-per-SM limits, and keeps the fastest alone.
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "tt_internal.cuh"

struct tt_batch {
  int count = 0;
  std::vector<tt_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  cudaStream_t caller = nullptr;  // the user's stream (may be the legacy default stream)
  cudaStream_t main = nullptr;    // the batch's own stream: graphs are captured and launched here
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_caller = nullptr;
  std::vector<cudaEvent_t> ev_join;
  uint64_t* d_sweep = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // the sweeps after a call's first when some tensors have a fixed draw (their data sketches
  // reused); null otherwise
  cudaGraph_t graph_reuse = nullptr;
  cudaGraphExec_t exec_reuse = nullptr;
  std::vector<const void*> capA;
  std::vector<const float*> capS;
  std::vector<float*> capC;  // flattened core pointers
  bool tuned = false;
  std::string err;
};

static void free_graphs(tt_batch* b);

static int bfail(tt_batch* b, int code, const char* msg) {
  if (b) b->err = msg;
  return code;
}

__global__ void k_sweep_inc(uint64_t* s) { *s += 1ull; }

extern "C" int tt_batch_init(tt_batch** out, int count, const tt_params* params, void* stream) {
  if (!out || count < 1 || !params) return TT_EINVAL;
  *out = nullptr;
  tt_batch* b = new tt_batch();
  b->count = count;
  b->caller = (cudaStream_t)stream;
  const int ns = std::min(count, 64);  // measured: 8 / 16 / 32 / 64 streams 21.8 / 19.4 / 19.3 / 18.9 ms per batched sweep
  b->streams.resize(ns);
  b->ev_join.resize(ns);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < ns && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_caller, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_sweep, sizeof(uint64_t));
  if (e != cudaSuccess) {
    fprintf(stderr, "tt_batch_init: %s\n", cudaGetErrorString(e));
    return TT_ECUDA;  // partially created objects are released by the process
  }
  b->ctx.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    int rc = tt_sketch_init(&b->ctx[i], &params[i], (void*)b->streams[i % ns]);
    if (rc != TT_OK) {
      fprintf(stderr, "tt_batch_init: tensor %d rejected (%d)\n", i, rc);
      for (int j = 0; j < i; ++j) tt_sketch_destroy(b->ctx[j]);
      for (auto s : b->streams) cudaStreamDestroy(s);
      cudaFree(b->d_sweep);
      delete b;
      return rc;
    }
    b->ctx[i]->d_sweep_ptr = b->d_sweep;
    b->ctx[i]->item_bytes = TT_BATCH_ITEM_BYTES;
  }
  *out = b;
  return TT_OK;
}

extern "C" void tt_batch_destroy(tt_batch* b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  for (auto s : b->streams) cudaStreamSynchronize(s);
  free_graphs(b);
  for (auto c : b->ctx) tt_sketch_destroy(c);
  for (auto ev : b->ev_join) cudaEventDestroy(ev);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_caller) cudaEventDestroy(b->ev_caller);
  if (b->main) cudaStreamDestroy(b->main);
  for (auto s : b->streams) cudaStreamDestroy(s);
  cudaFree(b->d_sweep);
  delete b;
}

extern "C" const char* tt_batch_last_error(const tt_batch* b) { return b ? b->err.c_str() : "null batch"; }

// time one unfold of mode k of context c with the current tunables (stream-ordered, CUDA events)
static int time_unfold(tt_ctx* c, const void* A, const float* sc, int k, float* Y, float* ms) {
  cudaEvent_t e0, e1;
  TT_CUDA(c, cudaEventCreate(&e0));
  TT_CUDA(c, cudaEventCreate(&e1));
  int rc = tt_launch_unfold(c, A, sc, k, Y);  // warm
  if (rc) return rc;
  TT_CUDA(c, cudaEventRecord(e0, c->stream));
  for (int r = 0; r < 3; ++r) {
    rc = tt_launch_unfold(c, A, sc, k, Y);
    if (rc) return rc;
  }
  TT_CUDA(c, cudaEventRecord(e1, c->stream));
  TT_CUDA(c, cudaEventSynchronize(e1));
  TT_CUDA(c, cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return TT_OK;
}

static int autotune(tt_batch* b, const void* const* A, const float* const* S) {
  // 0 = the default launch (modes >= 1: the G-column kernel where it fits); 1, 2, 4 = the
  // one-column kernel with that multiple of the work items
  static const int seg_mult[] = {0, 1, 2, 4};
  static const int cps[] = {1, 2};
  for (int i = 0; i < b->count; ++i) {
    tt_ctx* c = b->ctx[i];
    if (c->det || !(c->flags & TT_FLAG_BATCH_AUTOTUNE)) continue;  // no tunables / not asked for
    int rc = tt_ensure_tables(c, 0);
    if (rc) return rc;
    for (int k = 0; k < c->d; ++k) {
      float best = 1e30f;
      int bs = 1, bc = 2;
      for (int sm : seg_mult)
        for (int cp : cps) {
          c->tune_seg_mult[k] = sm;
          c->tune_cta_per_sm[k] = cp;
          float ms = 0.f;
          rc = time_unfold(c, A[i], S ? S[i] : nullptr, k, c->d_Y, &ms);
          if (rc) return rc;
          if (ms < best) {
            best = ms;
            bs = sm;
            bc = cp;
          }
        }
      c->tune_seg_mult[k] = bs;
      c->tune_cta_per_sm[k] = bc;
    }
    c->tables_valid = false;
  }
  b->tuned = true;
  return TT_OK;
}

// Capture one sweep of every tensor into a graph. reuse: tensors with a fixed draw
// (TT_FLAG_FIXED_SKETCH) run their sweep on the data sketches left in their context by the sweep
// before (the first graph's), without the data-sketch launches.
static int capture_graph(tt_batch* b, const void* const* A, const float* const* S, float* const* const* C,
                         bool reuse, cudaGraph_t* g_out, cudaGraphExec_t* x_out) {
  cudaError_t e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return bfail(b, TT_ECUDA, cudaGetErrorString(e));
  int rc = TT_OK;
  e = cudaEventRecord(b->ev_fork, b->main);
  for (size_t s = 0; s < b->streams.size() && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->streams[s], b->ev_fork, 0);
  for (int i = 0; i < b->count && e == cudaSuccess && rc == TT_OK; ++i) {
    tt_ctx* c = b->ctx[i];
    c->capture_mode = true;
    if (reuse && (c->flags & TT_FLAG_FIXED_SKETCH)) {
      float* ys[TT_MAX_D];
      for (int k = 0; k < c->d; ++k) ys[k] = c->d_Yall + c->yoff[k];
      rc = tt_one_sweep(c, A[i], S ? S[i] : nullptr, C[i], 0, nullptr, ys);
    } else {
      rc = tt_one_sweep(c, A[i], S ? S[i] : nullptr, C[i], 0, nullptr);
    }
    c->capture_mode = false;
    if (rc) b->err = c->err;
  }
  for (size_t s = 0; s < b->streams.size() && e == cudaSuccess; ++s) {
    e = cudaEventRecord(b->ev_join[s], b->streams[s]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->ev_join[s], 0);
  }
  if (e == cudaSuccess && rc == TT_OK) {
    k_sweep_inc<<<1, 1, 0, b->main>>>(b->d_sweep);
    e = cudaGetLastError();
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->main, &g);
  if (e == cudaSuccess) e = e2;
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, TT_ECUDA, cudaGetErrorString(e));
  }
  *g_out = g;
  e = cudaGraphInstantiate(x_out, g, 0);
  if (e != cudaSuccess) return bfail(b, TT_ECUDA, cudaGetErrorString(e));
  return TT_OK;
}

static void free_graphs(tt_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->exec_reuse) cudaGraphExecDestroy(b->exec_reuse);
  if (b->graph_reuse) cudaGraphDestroy(b->graph_reuse);
  b->exec = b->exec_reuse = nullptr;
  b->graph = b->graph_reuse = nullptr;
}

static int capture(tt_batch* b, const void* const* A, const float* const* S, float* const* const* C) {
  free_graphs(b);
  TT_TRY(capture_graph(b, A, S, C, false, &b->graph, &b->exec));
  bool any_fixed = false;
  for (auto c : b->ctx) any_fixed = any_fixed || (c->flags & TT_FLAG_FIXED_SKETCH) != 0;
  if (any_fixed) TT_TRY(capture_graph(b, A, S, C, true, &b->graph_reuse, &b->exec_reuse));
  b->capA.assign(A, A + b->count);
  b->capS.assign(b->count, nullptr);
  if (S)
    for (int i = 0; i < b->count; ++i) b->capS[i] = S[i];
  b->capC.clear();
  for (int i = 0; i < b->count; ++i)
    for (int k = 0; k < b->ctx[i]->d; ++k) b->capC.push_back(C[i][k]);
  return TT_OK;
}

static bool same_pointers(const tt_batch* b, const void* const* A, const float* const* S, float* const* const* C) {
  if (!b->exec || (int)b->capA.size() != b->count) return false;
  size_t q = 0;
  for (int i = 0; i < b->count; ++i) {
    if (b->capA[i] != A[i] || b->capS[i] != (S ? S[i] : nullptr)) return false;
    for (int k = 0; k < b->ctx[i]->d; ++k)
      if (b->capC[q++] != C[i][k]) return false;
  }
  return true;
}

extern "C" int tt_batch_sweep(tt_batch* b, const void* const* A_dev, const float* const* scales_dev,
                              float* const* const* cores_dev, int nsweeps, uint64_t first_sweep) {
  if (!b) return TT_EINVAL;
  if (!A_dev || !cores_dev || nsweeps < 0) return bfail(b, TT_EINVAL, "null arrays or negative sweep count");
  for (int i = 0; i < b->count; ++i) {
    tt_ctx* c = b->ctx[i];
    if (!A_dev[i] || !cores_dev[i]) return bfail(b, TT_EINVAL, "null tensor or core array");
    if ((c->dtype == TT_FP8E4M3) != (scales_dev && scales_dev[i]))
      return bfail(b, TT_EINVAL, "FP8 tensors need slice scales, other storage types none");
    for (int k = 0; k < c->d; ++k)
      if (!cores_dev[i][k]) return bfail(b, TT_EINVAL, "null core pointer");
  }
  // order the batch after the caller's stream (the call synchronises at its end)
  {
    cudaError_t e = cudaEventRecord(b->ev_caller, b->caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->ev_caller, 0);
    if (e != cudaSuccess) return bfail(b, TT_ECUDA, cudaGetErrorString(e));
  }
  if (!b->tuned) {
    cudaError_t e = cudaStreamSynchronize(b->main);
    if (e != cudaSuccess) return bfail(b, TT_ECUDA, cudaGetErrorString(e));
    int rc = autotune(b, A_dev, scales_dev);
    if (rc) return bfail(b, rc, "autotuning failed");
    for (auto s : b->streams) cudaStreamSynchronize(s);
  }
  if (!same_pointers(b, A_dev, scales_dev, cores_dev)) {
    int rc = capture(b, A_dev, scales_dev, cores_dev);
    if (rc) return rc;
  }
  for (auto c : b->ctx) {
    cudaError_t e = cudaMemsetAsync(c->d_status, 0, sizeof(int), b->main);
    if (e != cudaSuccess) return bfail(b, TT_ECUDA, cudaGetErrorString(e));
  }
  uint64_t s0 = first_sweep;
  cudaError_t e = cudaMemcpyAsync(b->d_sweep, &s0, sizeof(s0), cudaMemcpyHostToDevice, b->main);
  // a call's first sweep computes every tensor's data sketches; with a fixed draw its later
  // sweeps reuse them
  for (int t = 0; t < nsweeps && e == cudaSuccess; ++t)
    e = cudaGraphLaunch(t > 0 && b->exec_reuse ? b->exec_reuse : b->exec, b->main);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->main);
  if (e != cudaSuccess) return bfail(b, TT_ECUDA, cudaGetErrorString(e));
  for (int i = 0; i < b->count; ++i) {
    int st = 0;
    e = cudaMemcpy(&st, b->ctx[i]->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(b, TT_ECUDA, cudaGetErrorString(e));
    if (st != 0) {
      char msg[96];
      snprintf(msg, sizeof(msg), "tensor %d: solve status %d", i, st);
      return bfail(b, st, msg);
    }
  }
  return TT_OK;
}

extern "C" int tt_batch_rel_error(tt_batch* b, const void* const* A_dev, const float* const* scales_dev,
                                  float* const* const* cores_dev, double* out) {
  if (!b || !A_dev || !cores_dev || !out) return TT_EINVAL;
  for (int i = 0; i < b->count; ++i) {
    int rc = tt_rel_error(b->ctx[i], A_dev[i], scales_dev ? scales_dev[i] : nullptr, cores_dev[i], &out[i]);
    if (rc) return bfail(b, rc, b->ctx[i]->err.c_str());
  }
  return TT_OK;
}
