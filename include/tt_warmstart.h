/*
 * tt_warmstart.h -- C ABI of the learned warm start of the TT-TS library (same libttsketch.so).
 *
 * Algorithm 1 of the paper (Chen, Jiang, Yu, Qi, arXiv 2309.08093) takes initial cores as an
 * input; its experiments start from zero or random cores (Sec. 5). The paper has no learned
 * initialisation: these entry points add one. A multilayer perceptron
 *     in -> hidden -> hidden -> out, GELU after each hidden layer (Hendrycks and Gimpel, 2016),
 * maps a summary of the data sketch Y_k = S A_(k)^T (Alg. 1, Sec. 3) to initial TT cores. It is
 * trained on the GPU by the library's own kernels: BF16 tcgen05 GEMMs with FP32 accumulation in
 * tensor memory, FP32 master weights and Adam (Kingma and Ba, ICLR 2015, Algorithm 1) on the
 * mean squared error. Training pairs come from the method itself: a converged TT-TS solve,
 * brought to the right-canonical SVD gauge (tt_canonicalize) so that targets are unique.
 *
 * Conventions follow tt_sketch.h: cores FP32 with r[k] fastest, Y_k FP32 J x n[k] column-major,
 * *_dev pointers are caller-owned device memory, arrays of pointers are host arrays. Matrices of
 * the network are row-major FP32: X (batch x in), T and Y (batch x out), W1 (hidden x in),
 * W2 (hidden x hidden), W3 (out x hidden), b1, b2 (hidden), b3 (out). BF16 arguments are raw
 * 16-bit patterns (uint16_t). Every call returns TT_OK or a negative TT_E* code (tt_sketch.h);
 * invalid arguments are rejected on the host before any launch; the message of the last failure
 * of a network is in tt_mlp_last_error, of a context in tt_last_error.
 */
#ifndef TT_WARMSTART_H
#define TT_WARMSTART_H

#include <stdint.h>

#include "tt_sketch.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tt_mlp tt_mlp; /* opaque, library-owned */

typedef struct {
  int in_dim;      /* network input width, 1..65536 */
  int hidden;      /* hidden width, a multiple of 64, 64..2048 */
  int out_dim;     /* network output width, 1..262144 */
  int batch_max;   /* largest batch passed to any call, 1..1024 */
  float lr;        /* Adam step size */
  float beta1;     /* Adam first-moment decay, in [0, 1) */
  float beta2;     /* Adam second-moment decay, in [0, 1) */
  float eps;       /* Adam denominator offset, > 0 */
} tt_mlp_params;

/*
 * Create a network with all weights zero (set them with tt_mlp_set_weights). All work of the
 * network is enqueued on `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * Allocates every buffer for batch_max rows; no call allocates afterwards.
 */
int tt_mlp_init(tt_mlp** out, const tt_mlp_params* p, void* cuda_stream);
int tt_mlp_destroy(tt_mlp* m);
const char* tt_mlp_last_error(tt_mlp* m);

/* Load FP32 weights from device arrays (layouts above) and reset Adam's moments and step count. */
int tt_mlp_set_weights(tt_mlp* m, const float* W1_dev, const float* b1_dev, const float* W2_dev,
                       const float* b2_dev, const float* W3_dev, const float* b3_dev);
/* Copy the FP32 master weights to device arrays (layouts above). Asynchronous. */
int tt_mlp_get_weights(tt_mlp* m, float* W1_dev, float* b1_dev, float* W2_dev, float* b2_dev,
                       float* W3_dev, float* b3_dev);

/*
 * Y = MLP(X) for `batch` rows (1 <= batch <= batch_max). Row b of the input is
 * X_dev[rows[b] * ldx ...] when rows_dev (device int array of `batch` indices) is non-NULL,
 * else X_dev[b * ldx ...]. Y_dev receives batch x out_dim with row stride ldy. GEMM operands
 * are rounded to BF16 (nearest even); accumulation, biases and GELU are FP32. Asynchronous.
 */
int tt_mlp_forward(tt_mlp* m, const float* X_dev, int ldx, const int* rows_dev, int batch,
                   float* Y_dev, int ldy);

/*
 * Loss L = mean over the batch x out_dim entries of (Y - T)^2 and its gradients, without
 * updating the weights. Rows are selected as in tt_mlp_forward, for X and T alike. The
 * gradients go to the device arrays g*_dev (layouts of the weights) when non-NULL; the loss to
 * *loss_out (host) when non-NULL, which synchronises the stream.
 */
int tt_mlp_loss_grads(tt_mlp* m, const float* X_dev, int ldx, const float* T_dev, int ldt,
                      const int* rows_dev, int batch, double* loss_out, float* gW1_dev,
                      float* gb1_dev, float* gW2_dev, float* gb2_dev, float* gW3_dev,
                      float* gb3_dev);

/*
 * One training step: forward, backward and one Adam update of every parameter (the step count
 * t increases by one). *loss_out (host, optional) receives the loss before the update and then
 * the call synchronises; with loss_out == NULL the call is asynchronous.
 */
int tt_mlp_train_step(tt_mlp* m, const float* X_dev, int ldx, const float* T_dev, int ldt,
                      const int* rows_dev, int batch, double* loss_out);

/*
 * The network's GEMM on its own: C (M x N, FP32, row stride ldc) = A (M x K) B (N x K)^T with A
 * and B row-major BF16 (raw 16-bit patterns, row strides lda, ldb). K must be a multiple of 64;
 * lda and ldb multiples of 8 and every row 16-byte aligned; M, N >= 1. One tcgen05 kernel:
 * 128 x 256 tiles, FP32 accumulators in tensor memory. Asynchronous on `cuda_stream`; returns
 * TT_ETIMEOUT (after synchronising) only if a bounded wait inside the kernel gave up, which the
 * call checks when `check` is non-zero.
 */
int tt_mlp_gemm_bf16(const uint16_t* A_dev, int lda, const uint16_t* B_dev, int ldb, int M, int N,
                     int K, float* C_dev, int ldc, int check, void* cuda_stream);

/* ------------------------------------------------------------------------------------------
 * Warm-start data on a TT-TS context (tt_sketch.h)
 */

/* Width of the summary of tt_ws_summary: p * (n[0] + ... + n[d-1]). */
int64_t tt_ws_summary_dim(const tt_ctx* c, int p);
/* Width of the core vector of tt_ws_pack: sum_k r[k] n[k] r[k+1]. */
int64_t tt_ws_core_dim(const tt_ctx* c);

/*
 * Summary of the data sketches: x[o_k + i*p + b] = Y_k[b, i] for b < p, i < n[k], with
 * o_k = p * (n[0] + ... + n[k-1]), divided by its root mean square; *scale_dev = ||Y_0||_F, an
 * estimate of ||A||_F (E[S^T S] = I, Sec. 2.2). Y_dev[k] are the d sketches of tt_sketch_unfold
 * (J x n[k] column-major); bucket row b of Y_k is A_(k) times one random sparse sign vector, a
 * randomized range sample of A_(k). 1 <= p <= J. x_dev receives tt_ws_summary_dim(c, p) floats.
 * Asynchronous.
 */
int tt_ws_summary(tt_ctx* c, float* const* Y_dev, int p, float* x_dev, float* scale_dev);

/*
 * Right-canonical SVD gauge, in place: a left-to-right QR pass (Algorithm 1's orthogonalisation
 * step for k = 0..d-2, zero-padded where r[k] n[k] < r[k+1]), then for k = d-1..1 the thin SVD
 * of the right unfolding G_k^R = U S V^T (computed from the eigen-decomposition of G_k^R G_k^R^T
 * in FP64 by cyclic Jacobi rotations), G_k <- V^T with each row signed so that its first moment
 * sum_{i,b} (i + 1) V^T[j, i + n[k] b] is non-negative, G_{k-1} <- G_{k-1} x_3 (U S). Singular
 * values <= 1e-6 times the largest become zero together with their rows. The tensor [[G]] is
 * unchanged (up to those), and the result does not depend on the input gauge. Requires
 * r[k] <= 64 and r[k] <= n[k] r[k+1] for k >= 1 (else TT_EINVAL). Synchronises; returns TT_OK,
 * TT_ENONFINITE or TT_ECUDA.
 */
int tt_canonicalize(tt_ctx* c, float* const* cores_dev);

/*
 * Network target from cores and back: y = concat_k vec(G_k) * sqrt(n[k] r[k+1]) in the core
 * layout order, core 0 additionally divided by *scale_dev (tt_ws_pack); tt_ws_unpack inverts it.
 * y_dev holds tt_ws_core_dim(c) floats. Asynchronous.
 */
int tt_ws_pack(tt_ctx* c, float* const* cores_dev, const float* scale_dev, float* y_dev);
int tt_ws_unpack(tt_ctx* c, const float* y_dev, const float* scale_dev, float* const* cores_dev);

#ifdef __cplusplus
}
#endif

#endif /* TT_WARMSTART_H */
