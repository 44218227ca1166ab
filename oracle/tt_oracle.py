"""CPU FP64 oracle for randomized proximal TT-ALS with TensorSketch (TT-TS).

TEST INFRASTRUCTURE ONLY. This module is the independent reference that the CUDA library is
checked against. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import it; the library never calls it and shares no code with it.

It is written to be read against the paper (Chen, Jiang, Yu, Qi, "Low-rank Tensor Train
Decomposition Using TensorSketch"): every function states which passage it follows. Equations
are cited by their LaTeX labels, e.g. Eq. (ite) is the closed-form proximal update of Sec. 3.
Everything is float64 numpy; library primitives (matmul, FFT, QR, Cholesky, bincount) serve as
single steps, with no blocking or fusion beyond what the paper's formulas state.

Conventions (0-based indices throughout; the paper is 1-based):
  * tensor A of shape (n_0, ..., n_{d-1}); linear index i = sum_s i_s prod_{t<s} n_t, i.e. the
    first index fastest (Sec. 2.2, the bijection used to define TensorSketch);
  * TT core G_k of shape (r_{k-1}, n_k, r_k) (Sec. 2.1);
  * left unfolding G^L (r_{k-1} n_k x r_k), right unfolding G^R (r_{k-1} x n_k r_k) (Sec. 1.2);
  * mode-k matricization A_(k) (n_k x prod_{i!=k} n_i), remaining modes first-fastest
    (Sec. 1.2; the printed column formula has a garbled product index, read as t<s, t!=k);
  * G_{k(2)} = mode-2 matricization of core k: n_k x r_{k-1} r_k, column a + r_{k-1} b.

Hash/sign draws (Sec. 2.2, Eqs. (eqn_h), (eqn_v)): the paper asks for 3-wise independent
h_k : [n_k] -> [m] and 4-wise independent v_k : [n_k] -> {+1,-1}. Both sides of this project
draw them from one counter-based generator built on the published SplitMix64 output function
(Steele, Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
    step(z, f) = mix64(z + (f + 1) * 0x9E3779B97F4A7C15  mod 2^64)
    word(seed, sweep, mode, stream, i) = step(step(step(step(seed, sweep), mode), stream), i)
    h_k(i) = word(seed, sweep, k, 0, i) mod J
    v_k(i) = +1 if the top bit of word(seed, sweep, k, 1, i) is 0 else -1
where mix64 is SplitMix64's finaliser. This is stronger than the required k-wise independence.

Parity status: every public function here is pinned by tests/test_oracle_pins.py against the
paper's worked example, its identities (Lemma 1, Cor. 1-2, Thm 1-2, Thm 5's augmented form),
closed forms, invariants or brute force. No function is unpinned.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


# ---------------------------------------------------------------------------------------------
# Hash / sign draws (Sec. 2.2)

def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def splitmix64_sequence(seed: int, count: int) -> List[int]:
    """First `count` outputs of SplitMix64 started from state `seed` (for the published test vector)."""
    out = []
    x = seed & _M64
    for _ in range(count):
        x = (x + _GOLDEN) & _M64
        out.append(int(_mix64(np.array([x], dtype=np.uint64))[0]))
    return out


def _step(z: np.ndarray, field) -> np.ndarray:
    f = np.asarray(field, dtype=np.uint64)
    inc = (f + np.uint64(1)) * np.uint64(_GOLDEN)
    return _mix64(z + inc)


def hash_words(seed: int, sweep: int, mode: int, stream: int, index: np.ndarray) -> np.ndarray:
    """word(seed, sweep, mode, stream, i) for an array of indices i (uint64 result)."""
    index = np.asarray(index, dtype=np.uint64)
    z = np.full(index.shape, seed & _M64, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _step(z, sweep & _M64)
        z = _step(z, mode)
        z = _step(z, stream)
        z = _step(z, index)
    return z


def draw_sketch(seed: int, sweep: int, dims: Sequence[int], J: int) -> Tuple[List[np.ndarray], List[np.ndarray]]:
    """Per-mode CountSketch tables (h_k, v_k), k = 0..d-1, for one sweep (Sec. 2.2, Alg. 1).

    h_k takes values in [0, J) (the paper's h_k - 1), v_k in {+1, -1}.
    """
    hs, vs = [], []
    for k, n in enumerate(dims):
        idx = np.arange(n, dtype=np.uint64)
        h = (hash_words(seed, sweep, k, 0, idx) % np.uint64(J)).astype(np.int64)
        top = hash_words(seed, sweep, k, 1, idx) >> np.uint64(63)
        v = np.where(top == 0, 1.0, -1.0)
        hs.append(h)
        vs.append(v)
    return hs, vs


# ---------------------------------------------------------------------------------------------
# Sketch matrices by definition (Sec. 2.2)

def countsketch_matrix(h: np.ndarray, v: np.ndarray, J: int) -> np.ndarray:
    """S = Omega D (Definition of CountSketch): S[h(i), i] = v(i), zero elsewhere."""
    n = len(h)
    S = np.zeros((J, n))
    for i in range(n):
        S[h[i], i] = v[i]
    return S


def tensorsketch_matrix(hs: Sequence[np.ndarray], vs: Sequence[np.ndarray], J: int) -> np.ndarray:
    """Dense order-q TensorSketch S (J x prod n_k) from Eqs. (eqn_h), (eqn_v). Tiny shapes only.

    Column i <-> tuple (i_1..i_q) with the first index fastest; row h(i) = (sum_k h_k(i_k)) mod J;
    entry v(i) = prod_k v_k(i_k).
    """
    dims = [len(h) for h in hs]
    total = int(np.prod(dims)) if dims else 1
    S = np.zeros((J, total))
    for lin in range(total):
        rem = lin
        b = 0
        s = 1.0
        for k, n in enumerate(dims):
            ik = rem % n
            rem //= n
            b += int(hs[k][ik])
            s *= vs[k][ik]
        S[b % J, lin] = s
    return S


def dft_matrix(J: int) -> np.ndarray:
    """F of Sec. 3: F[s, j] = w^(s j), w = exp(-2 pi i / J)."""
    s = np.arange(J)
    return np.exp(-2j * np.pi * np.outer(s, s) / J)


def face_split(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Face-splitting product A [] B (Definition in Sec. 1.2): row i is A(i,:) kron B(i,:)."""
    assert A.shape[0] == B.shape[0]
    return np.stack([np.kron(A[i], B[i]) for i in range(A.shape[0])])


# ---------------------------------------------------------------------------------------------
# Tensor / TT bookkeeping (Secs. 1.2, 2.1, 3)

def unfold(A: np.ndarray, k: int) -> np.ndarray:
    """Mode-k matricization A_(k): n_k x prod_{i != k} n_i, remaining indices first-fastest."""
    return np.moveaxis(A, k, 0).reshape(A.shape[k], -1, order="F")


def left_unfold(G: np.ndarray) -> np.ndarray:
    """G^L(a + r0 * i, b) = G(a, i, b)."""
    r0, n, r1 = G.shape
    return G.reshape(r0 * n, r1, order="F")


def right_unfold(G: np.ndarray) -> np.ndarray:
    """G^R(a, i + n * b) = G(a, i, b)."""
    r0, n, r1 = G.shape
    return G.reshape(r0, n * r1, order="F")


def mode2_unfold(G: np.ndarray) -> np.ndarray:
    """G_{k(2)}: n_k x r_{k-1} r_k with column a + r_{k-1} b."""
    return unfold(G, 1)


def mode2_fold(G2: np.ndarray, r0: int, r1: int) -> np.ndarray:
    n = G2.shape[0]
    return np.moveaxis(G2.reshape(n, r0, r1, order="F"), 0, 1).copy(order="F")


def tt_full(cores: Sequence[np.ndarray]) -> np.ndarray:
    """[[G_1, ..., G_d]] (Sec. 2.1): A(i_1..i_d) = G_1(i_1) G_2(i_2) ... G_d(i_d)."""
    dims = [G.shape[1] for G in cores]
    T = left_unfold(cores[0])  # n_0 x r_1
    for G in cores[1:]:
        T = (T @ right_unfold(G)).reshape(T.shape[0] * G.shape[1], G.shape[2], order="F")
    return T.reshape(dims, order="F")


def interface_left(cores: Sequence[np.ndarray], k: int) -> np.ndarray:
    """G_{<k} = reshape([[G_1..G_{k-1}]], prod_{i<k} n_i, r_{k-1}) (Sec. 3); G_{<1} = 1."""
    if k == 0:
        return np.ones((1, 1))
    T = left_unfold(cores[0])
    for G in cores[1:k]:
        T = (T @ right_unfold(G)).reshape(T.shape[0] * G.shape[1], G.shape[2], order="F")
    return T


def interface_right(cores: Sequence[np.ndarray], k: int) -> np.ndarray:
    """G_{>k} = reshape([[G_{k+1}..G_d]], r_k, prod_{i>k} n_i) (Sec. 3); G_{>d} = 1."""
    d = len(cores)
    if k == d - 1:
        return np.ones((1, 1))
    R = right_unfold(cores[d - 1])
    for G in reversed(cores[k + 1:d - 1]):
        r0, n, r1 = G.shape
        R = (left_unfold(G) @ R).reshape(r0, n * R.shape[1], order="F")
    return R


def interface_matrix(cores: Sequence[np.ndarray], k: int) -> np.ndarray:
    """H_k = G_{>k}^T kron G_{<k} (Eq. (lrtt_sub4)). Small shapes only."""
    return np.kron(interface_right(cores, k).T, interface_left(cores, k))


# ---------------------------------------------------------------------------------------------
# Part (a): the data sketch S A_(k)^T

def sketch_unfolding_column(A: np.ndarray, hs, vs, J: int, k: int, ik: int) -> np.ndarray:
    """Column i_k of Y_k = S A_(k)^T by the TensorSketch definition (Eqs. (eqn_h), (eqn_v)).

    Y_k[b, i_k] = sum over all entries with that i_k of prod_{s!=k} v_s(i_s) * A(i),
    restricted to (sum_{s!=k} h_s(i_s)) mod J = b. S is built from the modes s != k.
    """
    d = A.ndim
    sub = A[(slice(None),) * k + (ik,)]  # remaining modes, in order (a view)
    others = [s for s in range(d) if s != k]
    bucket = np.zeros(sub.shape, dtype=np.int64)
    sign = np.ones(sub.shape)
    for ax, s in enumerate(others):
        shape = [1] * len(others)
        shape[ax] = sub.shape[ax]
        bucket = bucket + hs[s].reshape(shape)
        sign = sign * vs[s].reshape(shape)
    bucket %= J
    return np.bincount(bucket.ravel(), weights=(sign * sub).ravel(), minlength=J)


def sketch_unfolding_coo(idx: np.ndarray, vals: np.ndarray, dims: Sequence[int], hs, vs, J: int,
                         k: int) -> np.ndarray:
    """Y_k = S A_(k)^T for a sparse A given as coordinates (Sec. 3, the discussion after Theorem
    3: for sparse A the sketch of the unfolding costs O(nnz)). idx is d x nnz (0-based indices,
    idx[s, e] = i_s of entry e), vals the nnz values; repeated coordinates add up. Entry e adds
    prod_{s != k} v_s(i_s) * val_e to Y_k[(sum_{s != k} h_s(i_s)) mod J, i_k], which is the
    definition of Eqs. (eqn_h), (eqn_v) restricted to the nonzeros."""
    d = len(dims)
    idx = np.asarray(idx, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    bucket = np.zeros(vals.shape[0], dtype=np.int64)
    sign = np.ones(vals.shape[0])
    for s in range(d):
        if s != k:
            bucket += hs[s][idx[s]]
            sign *= vs[s][idx[s]]
    Y = np.zeros((J, dims[k]))
    np.add.at(Y, (bucket % J, idx[k]), sign * vals)
    return Y


def sketch_unfolding(A: np.ndarray, hs, vs, J: int, k: int) -> np.ndarray:
    """Y_k = S A_(k)^T (J x n_k), every column by its definition (Alg. 1, 'compute S A_(k)^T')."""
    return np.stack([sketch_unfolding_column(A, hs, vs, J, k, i) for i in range(A.shape[k])], axis=1)


def sketch_unfolding_dense(A: np.ndarray, hs, vs, J: int, k: int) -> np.ndarray:
    """Same quantity as a dense product S_{-k} @ A_(k)^T (brute force, tiny shapes)."""
    others = [s for s in range(A.ndim) if s != k]
    S = tensorsketch_matrix([hs[s] for s in others], [vs[s] for s in others], J)
    return S @ unfold(A, k).T


# ---------------------------------------------------------------------------------------------
# Part (b): the interface sketch S H_k = S (G_{>k}^T kron G_{<k})

def sketch_interface_dense(cores, hs, vs, J: int, k: int) -> np.ndarray:
    """S_{-k} H_k by explicit matrices (brute force, tiny shapes)."""
    d = len(cores)
    others = [s for s in range(d) if s != k]
    S = tensorsketch_matrix([hs[s] for s in others], [vs[s] for s in others], J)
    return S @ interface_matrix(cores, k)


def _bucket_prefix(cores, hs, vs, J: int, k: int) -> np.ndarray:
    """P_{<k} = S_{<k} G_{<k} (J x r_{k-1}) in the bucket domain, built core by core.

    P_0 = e_0 (the sketch of the empty product); P_j[b, :] = sum_i v_j(i) P_{j-1}[(b - h_j(i)) mod J, :] G_j(i).
    """
    P = np.zeros((J, 1))
    P[0, 0] = 1.0
    for j in range(k):
        G = cores[j]
        Pn = np.zeros((J, G.shape[2]))
        for i in range(G.shape[1]):
            Pn += vs[j][i] * (np.roll(P, int(hs[j][i]), axis=0) @ G[:, i, :])
        P = Pn
    return P


def _bucket_suffix(cores, hs, vs, J: int, k: int) -> np.ndarray:
    """Q_{>k} = (S_{>k} G_{>k}^T)^T (r_k x J) in the bucket domain, built core by core from the right."""
    d = len(cores)
    Q = np.zeros((1, J))
    Q[0, 0] = 1.0
    for j in range(d - 1, k, -1):
        G = cores[j]
        Qn = np.zeros((G.shape[0], J))
        for i in range(G.shape[1]):
            Qn += vs[j][i] * (G[:, i, :] @ np.roll(Q, int(hs[j][i]), axis=1))
        Q = Qn
    return Q


def sketch_interface_conv(cores, hs, vs, J: int, k: int) -> np.ndarray:
    """S H_k without any FFT: circular convolution of P_{<k} and Q_{>k} along the bucket axis.

    SH_k[b, a + r_{k-1} c] = sum_{b1} P_{<k}[b1, a] Q_{>k}[c, (b - b1) mod J]: Theorem 1 read in
    the bucket domain (the TensorSketch hash of Eq. (eqn_h) adds the partial hashes mod J).
    """
    P = _bucket_prefix(cores, hs, vs, J, k)
    Q = _bucket_suffix(cores, hs, vs, J, k)
    r0, r1 = P.shape[1], Q.shape[0]
    SH = np.zeros((J, r0 * r1))
    for b1 in range(J):
        rolled = np.roll(Q, b1, axis=1)  # rolled[c, b] = Q[c, (b - b1) mod J]
        SH += np.einsum("a,cb->bca", P[b1], rolled).reshape(J, r1 * r0)
    return SH


def core_fft_sketch(G: np.ndarray, h: np.ndarray, v: np.ndarray, J: int) -> np.ndarray:
    """G x_2 (F S) (Theorem 2): CountSketch along the middle mode, then DFT. Shape (r0, J, r1)."""
    r0, n, r1 = G.shape
    cs = np.zeros((r0, J, r1))
    for i in range(n):
        cs[:, h[i], :] += v[i] * G[:, i, :]
    return np.fft.fft(cs, axis=1)


def sketch_interface_fft(cores, hs, vs, J: int, k: int) -> np.ndarray:
    """S H_k = F^{-1}[(F S_{>k} G_{>k}^T) [] (F S_{<k} G_{<k})] (Theorem 1), with the two factors
    formed by slice-wise products of the FFT-sketched cores (Theorem 2)."""
    d = len(cores)
    L = np.ones((J, 1), dtype=complex)  # F S_{<k} G_{<k}, row s = prefix product at frequency s
    for j in range(k):
        Gh = core_fft_sketch(cores[j], hs[j], vs[j], J)
        L = np.einsum("sa,asb->sb", L, Gh)
    R = np.ones((J, 1), dtype=complex)  # F S_{>k} G_{>k}^T, row s = suffix product at frequency s
    for j in range(d - 1, k, -1):
        Gh = core_fft_sketch(cores[j], hs[j], vs[j], J)
        R = np.einsum("asb,sb->sa", Gh, R)
    FSH = face_split(R, L)  # column c * r_{k-1} + a
    return np.real(np.fft.ifft(FSH, axis=0))


# ---------------------------------------------------------------------------------------------
# Part (c): the proximal update, Eq. (ite)

def prox_gram_rhs(Yk: np.ndarray, SHk: np.ndarray, Gk: np.ndarray, sigma: float):
    """M = (S H_k)^T (S H_k) + sigma I and B = Y_k^T (S H_k) + sigma G_{k(2)} of Eq. (ite)
    (read with S^T S; the printed S S^T does not conform)."""
    s = SHk.shape[1]
    M = SHk.T @ SHk + sigma * np.eye(s)
    B = Yk.T @ SHk + sigma * mode2_unfold(Gk)
    return M, B


class NotSPD(Exception):
    pass


# Eq. (ite) needs M SPD, which Alg. 1 guarantees through sigma > 0; Sec. 5 also runs sigma = 0,
# where the sketched Gram can be singular (for instance when two indices of a mode whose core is
# square share a bucket, S H_k loses rank). Reading taken: a Cholesky pivot L_jj^2 at or below
# PIVOT_TOL times the largest diagonal entry of M means M is singular to the precision of its
# inputs, and the update is refused.
PIVOT_TOL = 1e-10


def cholesky_lower(M: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor of M, refusing (NotSPD) a factorization that fails or whose smallest
    pivot L_jj^2 is at most PIVOT_TOL * max_i M_ii."""
    try:
        L = np.linalg.cholesky(M)
    except np.linalg.LinAlgError as e:
        raise NotSPD(str(e))
    piv = np.diag(L) ** 2
    if piv.size and piv.min() <= PIVOT_TOL * np.max(np.diag(M)):
        raise NotSPD(f"pivot ratio {piv.min() / np.max(np.diag(M)):.3e} <= {PIVOT_TOL:g}")
    return L


def prox_update(Yk: np.ndarray, SHk: np.ndarray, Gk: np.ndarray, sigma: float) -> np.ndarray:
    """New core by Eq. (ite): G_{k(2)} <- B M^{-1}, solved through the Cholesky factor of M."""
    r0, n, r1 = Gk.shape
    M, B = prox_gram_rhs(Yk, SHk, Gk, sigma)
    L = cholesky_lower(M)
    Z = np.linalg.solve(L, B.T)  # L Z = B^T
    X = np.linalg.solve(L.T, Z)  # L^T X = Z  ->  M X = B^T
    return mode2_fold(X.T, r0, r1)


def prox_update_augmented(Yk: np.ndarray, SHk: np.ndarray, Gk: np.ndarray, sigma: float) -> np.ndarray:
    """The same update as the least-squares problem of Thm 5's proof:
    min_X || [S H_k; sqrt(sigma) I] X - [Y_k; sqrt(sigma) G_{k(2)}^T] ||_F (Eq. (lrtt_sub4))."""
    r0, n, r1 = Gk.shape
    s = SHk.shape[1]
    P = np.vstack([SHk, math.sqrt(sigma) * np.eye(s)])
    Bt = np.vstack([Yk, math.sqrt(sigma) * mode2_unfold(Gk).T])
    X, *_ = np.linalg.lstsq(P, Bt, rcond=None)
    return mode2_fold(X.T, r0, r1)


# ---------------------------------------------------------------------------------------------
# Orthogonalisation (Alg. 1)

def qr_nonneg(M: np.ndarray):
    """Reduced QR with diag(R) >= 0. For a wide M (m < n) the factors are zero-padded to
    Q (m x n) and R (n x n) so that the TT ranks keep their sizes (Q R = M still holds)."""
    m, n = M.shape
    Q, R = np.linalg.qr(M, mode="reduced")
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    Q = Q * sgn
    R = sgn[:, None] * R
    if m < n:
        Q = np.hstack([Q, np.zeros((m, n - m))])
        R = np.vstack([R, np.zeros((n - m, n))])
    return Q, R


def left_orthogonalize_step(cores: List[np.ndarray], k: int) -> None:
    """Alg. 1 for k < d: [Q, R] = qr(G_k^L); G_k <- reshape(Q); G_{k+1} <- reshape(R G_{k+1}^R)."""
    G = cores[k]
    r0, n, r1 = G.shape
    Q, R = qr_nonneg(left_unfold(G))
    cores[k] = Q.reshape(r0, n, r1, order="F")
    Gn = cores[k + 1]
    cores[k + 1] = (R @ right_unfold(Gn)).reshape(Gn.shape, order="F")


def right_orthogonalize_step(cores: List[np.ndarray], k: int) -> None:
    """One step of the right-to-left orthogonalisation of Alg. 1: G_k^R = L Q^T with orthonormal
    rows Q^T and lower-triangular L (non-negative diagonal); G_k <- Q^T, G_{k-1}^L <- G_{k-1}^L L."""
    G = cores[k]
    r0, n, r1 = G.shape
    Q, R = qr_nonneg(right_unfold(G).T)  # (n r1) x r0
    cores[k] = Q.T.reshape(r0, n, r1, order="F")
    Gp = cores[k - 1]
    cores[k - 1] = (left_unfold(Gp) @ R.T).reshape(Gp.shape, order="F")


def orthogonalize_right_to_left(cores: Sequence[np.ndarray]) -> List[np.ndarray]:
    out = [np.array(G, dtype=np.float64, order="F") for G in cores]
    for k in range(len(out) - 1, 0, -1):
        right_orthogonalize_step(out, k)
    return out


# ---------------------------------------------------------------------------------------------
# Algorithm 1 (TT-TS) and the deterministic comparison (proximal TT-ALS)

def tt_ts_sweep(A: np.ndarray, cores: Sequence[np.ndarray], seed: int, sweep: int, J: int,
                sigma: float, interface: str = "fft"):
    """One outer iteration of Algorithm 1. Returns (new cores, rel-change of Sec. 5).

    The proximal centre G_k^(t) is core k right before its update (after the right-to-left
    orthogonalisation and after R from step k-1 was absorbed). Rel-change is
    max_k ||G_k^(t+1) - G_k^(t)||_F / ||G_k^(t+1)||_F over the updates of this sweep.
    """
    d = A.ndim
    cores = orthogonalize_right_to_left(cores)
    hs, vs = draw_sketch(seed, sweep, A.shape, J)
    sk = {"fft": sketch_interface_fft, "conv": sketch_interface_conv, "dense": sketch_interface_dense}[interface]
    rel_change = 0.0
    for k in range(d):
        SH = sk(cores, hs, vs, J, k)
        Y = sketch_unfolding(A, hs, vs, J, k)
        Gn = prox_update(Y, SH, cores[k], sigma)
        nrm = np.linalg.norm(Gn.ravel())
        if nrm > 0:
            rel_change = max(rel_change, np.linalg.norm((Gn - cores[k]).ravel()) / nrm)
        cores[k] = Gn
        if k < d - 1:
            left_orthogonalize_step(cores, k)
    return cores, rel_change


def tt_ts(A: np.ndarray, cores0: Sequence[np.ndarray], seed: int, J: int, sigma: float,
          nsweeps: int, first_sweep: int = 0, interface: str = "fft"):
    """Algorithm 1 for a fixed number of outer iterations; a fresh sketch is drawn per sweep."""
    cores = [np.array(G, dtype=np.float64, order="F") for G in cores0]
    changes = []
    for t in range(nsweeps):
        cores, rc = tt_ts_sweep(A, cores, seed, first_sweep + t, J, sigma, interface)
        changes.append(rc)
    return cores, changes


def prox_als_sweep(A: np.ndarray, cores: Sequence[np.ndarray], sigma: float):
    """One sweep of unsketched proximal TT-ALS, subproblem Eq. (lrtt_sub_prox), same order and
    orthogonalisation as Algorithm 1 (the TT-ALS comparison of Sec. 5)."""
    d = A.ndim
    cores = orthogonalize_right_to_left(cores)
    for k in range(d):
        H = interface_matrix(cores, k)
        r0, n, r1 = cores[k].shape
        M = H.T @ H + sigma * np.eye(H.shape[1])
        B = unfold(A, k) @ H + sigma * mode2_unfold(cores[k])
        X = np.linalg.solve(M, B.T)
        cores[k] = mode2_fold(X.T, r0, r1)
        if k < d - 1:
            left_orthogonalize_step(cores, k)
    return cores


def tt_svd(A: np.ndarray, ranks: Sequence[int]) -> List[np.ndarray]:
    """TT-SVD (Oseledets 2011, cited in Sec. 1): successive truncated SVDs of the unfoldings."""
    d = A.ndim
    dims = A.shape
    C = A.reshape(-1, order="F")
    cores = []
    rp = 1
    for k in range(d - 1):
        C = C.reshape(rp * dims[k], -1, order="F")
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        r = min(ranks[k + 1], len(s))
        cores.append(U[:, :r].reshape(rp, dims[k], r, order="F"))
        C = s[:r, None] * Vt[:r]
        rp = r
    cores.append(C.reshape(rp, dims[d - 1], 1, order="F"))
    return cores


def rel_error(A: np.ndarray, cores: Sequence[np.ndarray]) -> float:
    """||A - [[G]]||_F / ||A||_F (the 'relative error' of Sec. 5)."""
    return float(np.linalg.norm((A - tt_full(cores)).ravel()) / np.linalg.norm(A.ravel()))
