"""CPU FP64 oracle for the learned warm start of TT-TS.

TEST INFRASTRUCTURE ONLY. Like ``tt_oracle``, this module is the independent reference that the
CUDA library is checked against. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import it; the library never calls it and shares no code
with it.

The paper's Algorithm 1 takes initial cores as an input and its experiments start from zero or
random cores (Sec. 5). The learned warm start replaces that input with the output of a small
network, so this module has no passage of the paper to follow for the network itself. It follows
published definitions instead:
  * GELU(z) = z Phi(z), Phi the standard normal CDF (Hendrycks and Gimpel, 2016);
  * Adam with bias correction (Kingma and Ba, ICLR 2015, Algorithm 1);
  * a multilayer perceptron in -> H -> H -> out with GELU after each hidden layer, trained on the
    mean squared error;
  * the TT gauge fixed by a left-to-right QR pass (Algorithm 1's orthogonalisation step) and a
    right-to-left pass of SVDs of the right unfoldings: the right-canonical form of Sec. 2.1's
    TT format, whose rows are the singular vectors of the tensor's unfoldings, one sign per row.

Where the CUDA path rounds GEMM operands to BF16 (round to nearest, ties to even), the functions
below take ``bf16=True`` and round at exactly the same points, in float64 arithmetic otherwise, so
the two differ only by FP32 accumulation order. With ``bf16=False`` they are the plain FP64
definitions, which the pins check against finite differences and library routines.

Parity status: every public function is pinned by tests/test_oracle_warmstart.py (closed forms,
finite differences, library routines, gauge invariance, round trips). No function is unpinned.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np
from scipy.special import erf

import tt_oracle as O

# ---------------------------------------------------------------------------------------------
# number formats and the activation


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to BF16 (8 exponent bits, 7 fraction bits), nearest, ties to even, returned as
    float64. Values are first taken to float32 (the CUDA path rounds FP32 values). Finite inputs
    only."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64).reshape(np.shape(x))


def gelu(z: np.ndarray) -> np.ndarray:
    """GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2."""
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z: np.ndarray) -> np.ndarray:
    """d GELU / dz = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


# ---------------------------------------------------------------------------------------------
# the network: params = {"W1": (H, In), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (Out, H),
# "b3": (Out,)}; rows of X and T are samples


def _q(x, bf16):
    return round_bf16(x) if bf16 else np.asarray(x, dtype=np.float64)


def mlp_forward(P: Dict[str, np.ndarray], X: np.ndarray, bf16: bool = False):
    """Y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3 for every row x of X. Returns Y and the cache
    (pre-activations Z1, Z2 and activations H1, H2) used by the backward pass."""
    Z1 = _q(X, bf16) @ _q(P["W1"], bf16).T + P["b1"]
    H1 = gelu(Z1)
    Z2 = _q(H1, bf16) @ _q(P["W2"], bf16).T + P["b2"]
    H2 = gelu(Z2)
    Y = _q(H2, bf16) @ _q(P["W3"], bf16).T + P["b3"]
    return Y, {"X": X, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2}


def mlp_loss_grads(P: Dict[str, np.ndarray], X: np.ndarray, T: np.ndarray, bf16: bool = False):
    """Mean squared error L = mean_{b,j} (Y_bj - T_bj)^2 and its gradient with respect to every
    parameter, by the chain rule written out layer by layer."""
    B, out = T.shape
    Y, c = mlp_forward(P, X, bf16)
    R = Y - T
    loss = float(np.mean(R * R))
    dY = 2.0 * R / (B * out)
    g = {}
    g["W3"] = _q(dY, bf16).T @ _q(c["H2"], bf16)
    g["b3"] = dY.sum(axis=0)
    dH2 = _q(dY, bf16) @ _q(P["W3"], bf16)
    dZ2 = dH2 * gelu_grad(c["Z2"])
    g["W2"] = _q(dZ2, bf16).T @ _q(c["H1"], bf16)
    g["b2"] = dZ2.sum(axis=0)
    dH1 = _q(dZ2, bf16) @ _q(P["W2"], bf16)
    dZ1 = dH1 * gelu_grad(c["Z1"])
    g["W1"] = _q(dZ1, bf16).T @ _q(X, bf16)
    g["b1"] = dZ1.sum(axis=0)
    return loss, g, Y


def adam_step(theta, grad, m, v, t: int, lr: float, beta1: float, beta2: float, eps: float):
    """One Adam update (Kingma and Ba, Algorithm 1), t = 1 for the first step. Returns the new
    (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ---------------------------------------------------------------------------------------------
# TT gauge fixing: the right-canonical SVD form


def _right_unfold(G):
    r0, n, r1 = G.shape
    return G.reshape(r0, n * r1, order="F")  # column i + n * b


def canonicalize_right(cores: Sequence[np.ndarray], tol: float = 1e-6) -> List[np.ndarray]:
    """Right-canonical TT with the SVD gauge, cores (r_{k-1}, n_k, r_k).

    1. Left-to-right QR pass (the orthogonalisation step of Algorithm 1 applied for k = 0..d-2):
       cores 0..d-2 become left-orthonormal, zero-padded where r_{k-1} n_k < r_k. A sweep of
       Algorithm 1 already leaves its cores in this state.
    2. For k = d-1 down to 1: thin SVD of the right unfolding G_k^R = U S V^T. Because everything
       left of core k is left-orthonormal and everything right of it right-orthonormal, S and V
       are the singular values and (coordinates of the) right singular vectors of the tensor's
       unfolding between modes k-1 and k, so the result does not depend on the input gauge.
       Singular values <= tol * S[0] are set to zero together with their rows of V^T. Each kept
       row of V^T gets the sign that makes its first moment along the mode index,
       sum_{i,b} (i + 1) V^T[j, i + n_k b], non-negative. G_k <- V^T, G_{k-1} <- G_{k-1} x_3 (U S).

    The tensor is unchanged up to the dropped singular values; cores 1..d-1 have orthonormal (or
    zero) rows in decreasing singular-value order. Requires r_{k-1} <= n_k r_k for k >= 1."""
    cs = [np.array(G, dtype=np.float64) for G in cores]
    d = len(cs)
    for k in range(d - 1):
        O.left_orthogonalize_step(cs, k)
    for k in range(d - 1, 0, -1):
        r0, n, r1 = cs[k].shape
        assert r0 <= n * r1, "right unfolding must have r_{k-1} <= n_k r_k"
        U, s, Vt = np.linalg.svd(_right_unfold(cs[k]), full_matrices=False)
        keep = s > tol * s[0] if s[0] > 0 else np.zeros_like(s, dtype=bool)
        s = np.where(keep, s, 0.0)
        Vt = Vt * keep[:, None]
        w = np.tile(np.arange(1, n + 1, dtype=np.float64), r1)  # column i + n b has weight i + 1
        sg = np.where(Vt @ w < 0, -1.0, 1.0)
        Vt = Vt * sg[:, None]
        US = U * (s * sg)[None, :]
        cs[k] = Vt.reshape(r0, n, r1, order="F")
        cs[k - 1] = np.einsum("aib,bc->aic", cs[k - 1], US)
    return cs


# ---------------------------------------------------------------------------------------------
# the network's input and output


def ws_summary(Y: Sequence[np.ndarray], p: int) -> Tuple[np.ndarray, float]:
    """Sketch summary. Y[k] is the data sketch Y_k = S A_(k)^T (J x n_k) of Sec. 3; its bucket
    row b is A_(k) times one random signed sparse vector, a randomized range sample of A_(k).
    The summary keeps rows 0..p-1 of every Y_k, laid out x[o_k + i p + b] = Y_k[b, i]
    (o_k = p sum_{t<k} n_t), divided by its root mean square. The scale returned is ||Y_0||_F,
    an unbiased-in-square estimate of ||A||_F (E[S^T S] = I, Sec. 2.2)."""
    parts = [np.asarray(Yk, dtype=np.float64)[:p, :].T.reshape(-1) for Yk in Y]
    x = np.concatenate(parts)
    rms = math.sqrt(float(np.mean(x * x)))
    return x / rms, float(np.linalg.norm(np.asarray(Y[0], dtype=np.float64)))


def ws_targets(cores: Sequence[np.ndarray], scale: float) -> np.ndarray:
    """Network target: vec(G_k) in the (alpha fastest, then i, then beta) order, times
    sqrt(n_k r_k), concatenated over k; core 0 is first divided by ``scale``. For right-canonical
    cores this puts every core's entries at unit root mean square."""
    out = []
    for k, G in enumerate(cores):
        r0, n, r1 = G.shape
        g = np.asarray(G, dtype=np.float64) / (scale if k == 0 else 1.0)
        out.append(g.reshape(-1, order="F") * math.sqrt(n * r1))
    return np.concatenate(out)


def ws_cores(y: np.ndarray, scale: float, dims: Sequence[int], ranks: Sequence[int]) -> List[np.ndarray]:
    """Inverse of ws_targets: network output -> initial cores."""
    cs, o = [], 0
    for k, n in enumerate(dims):
        r0, r1 = ranks[k], ranks[k + 1]
        sz = r0 * n * r1
        g = np.asarray(y[o:o + sz], dtype=np.float64) / math.sqrt(n * r1)
        cs.append(g.reshape(r0, n, r1, order="F") * (scale if k == 0 else 1.0))
        o += sz
    return cs
