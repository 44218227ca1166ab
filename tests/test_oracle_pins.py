"""Pins for the CPU oracle: each check compares the oracle with something other than itself
(the paper's worked example, its identities, closed forms, invariants, brute force).

CPU only (no GPU marker)."""
import math

import numpy as np
import pytest

import tt_oracle as O
from conftest import read_golden
from paper_2309_08093_gb300 import synth


def _rng(seed):
    return np.random.default_rng(seed)


def _rand_tables(rng, dims, J):
    hs = [rng.integers(0, J, size=n) for n in dims]
    vs = [rng.choice([-1.0, 1.0], size=n) for n in dims]
    return hs, vs


# ---------------------------------------------------------------------------------------------
# Sec. 2.2 worked example

def test_worked_example_tensorsketch_matrix():
    g = read_golden("tensorsketch_worked_example.txt")
    m = int(g["m"][0][0])
    h1 = np.array([int(x) - 1 for x in g["h1"][0]])
    h2 = np.array([int(x) - 1 for x in g["h2"][0]])
    v1 = np.array([float(x) for x in g["v1"][0]])
    v2 = np.array([float(x) for x in g["v2"][0]])
    S_printed = np.array([[float(x) for x in row] for row in g["S"]])
    Omega_printed = np.array([[float(x) for x in row] for row in g["Omega"]])
    v_printed = np.array([float(x) for x in g["v"][0]])
    h_printed = np.array([int(x) - 1 for x in g["h"][0]])
    S = O.tensorsketch_matrix([h1, h2], [v1, v2], m)
    assert np.array_equal(S, S_printed)
    assert np.array_equal(np.abs(S), Omega_printed)
    assert np.array_equal(S.sum(axis=0), v_printed)
    assert np.array_equal(np.argmax(np.abs(S), axis=0), h_printed)


def test_worked_example_through_data_sketch():
    """A 2 x 2 x 1 tensor sketched along its last (singleton) mode: Y = S vec(A)."""
    g = read_golden("tensorsketch_worked_example.txt")
    S_printed = np.array([[float(x) for x in row] for row in g["S"]])
    hs = [np.array([0, 1]), np.array([0, 1]), np.array([0])]
    vs = [np.array([1.0, -1.0]), np.array([-1.0, 1.0]), np.array([1.0])]
    A = np.asfortranarray(np.arange(1.0, 5.0).reshape(2, 2, 1, order="F"))
    Y = O.sketch_unfolding(A, hs, vs, 2, 2)
    assert np.array_equal(Y[:, 0], S_printed @ A.ravel(order="F"))


# ---------------------------------------------------------------------------------------------
# hash / sign draws

def test_splitmix64_published_vector():
    g = read_golden("splitmix64_vectors.txt")
    seed = int(g["seed"][0][0])
    expect = [int(x) for x in g["out"][0]]
    assert O.splitmix64_sequence(seed, 3) == expect


def test_hash_words_match_python_integers():
    """numpy uint64 wrapping arithmetic vs exact Python integers mod 2^64."""
    M = (1 << 64) - 1

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    def word(seed, sweep, mode, stream, i):
        z = seed
        for f in (sweep, mode, stream, i):
            z = mix((z + (f + 1) * 0x9E3779B97F4A7C15) & M)
        return z

    idx = np.arange(50)
    got = O.hash_words(987654321123, 7, 3, 1, idx)
    assert [int(x) for x in got] == [word(987654321123, 7, 3, 1, int(i)) for i in idx]


def test_hash_tables_distribution():
    """h_k uniform on [0, J) and v_k balanced (chi-square / binomial bounds)."""
    J, n = 64, 64 * 400
    hs, vs = O.draw_sketch(12345, 0, [n], J)
    counts = np.bincount(hs[0], minlength=J)
    chi2 = ((counts - n / J) ** 2 / (n / J)).sum()
    assert chi2 < J + 6 * math.sqrt(2 * J)  # ~6 sigma above the mean of chi2(J-1)
    assert abs(vs[0].sum()) < 6 * math.sqrt(n)
    # pairwise: h(i) and h(i+1) independent -> joint counts on a 8x8 grid close to uniform
    a, b = hs[0][:-1] % 8, hs[0][1:] % 8
    joint = np.bincount(a * 8 + b, minlength=64)
    e = (n - 1) / 64
    assert ((joint - e) ** 2 / e).sum() < 64 + 6 * math.sqrt(128)


def test_hash_tables_change_with_sweep_and_mode():
    h_a, v_a = O.draw_sketch(5, 0, [100, 100], 4096)
    h_b, v_b = O.draw_sketch(5, 1, [100, 100], 4096)
    assert not np.array_equal(h_a[0], h_b[0])
    assert not np.array_equal(h_a[0], h_a[1])
    assert np.all((h_a[0] >= 0) & (h_a[0] < 4096))
    assert set(np.unique(v_a[0])) <= {-1.0, 1.0}


# ---------------------------------------------------------------------------------------------
# unfoldings and the TT format

def test_unfold_matches_index_formula():
    A = synth.random_tensor((3, 4, 2, 5), 1)
    for k in range(4):
        Ak = O.unfold(A, k)
        others = [s for s in range(4) if s != k]
        for idx in np.ndindex(A.shape):
            j, stride = 0, 1
            for s in others:
                j += idx[s] * stride
                stride *= A.shape[s]
            assert Ak[idx[k], j] == A[idx]


def test_tt_full_elementwise_products():
    cores = synth.random_tt((3, 2, 4, 2), (1, 2, 3, 2, 1), 2)
    T = O.tt_full(cores)
    for idx in np.ndindex(T.shape):
        p = np.ones((1, 1))
        for k, i in enumerate(idx):
            p = p @ cores[k][:, i, :]
        assert abs(T[idx] - p[0, 0]) < 1e-12


def test_interface_reproduces_unfolding():
    """(G_{>k}^T kron G_{<k}) G_{k(2)}^T = A_(k)^T for A = [[G]] (Eq. (lrtt_sub) at zero residual)."""
    cores = synth.random_tt((3, 4, 2, 3), (1, 2, 3, 2, 1), 3)
    A = O.tt_full(cores)
    for k in range(4):
        H = O.interface_matrix(cores, k)
        assert np.allclose(H @ O.mode2_unfold(cores[k]).T, O.unfold(A, k).T, atol=1e-12)
        r0, n, r1 = cores[k].shape
        assert np.array_equal(O.mode2_fold(O.mode2_unfold(cores[k]), r0, r1), cores[k])


def test_left_right_unfold_index_formula():
    G = synth.random_tensor((2, 3, 4), 4)
    L, R = O.left_unfold(G), O.right_unfold(G)
    for a, i, b in np.ndindex(G.shape):
        assert L[a + 2 * i, b] == G[a, i, b]
        assert R[a, i + 3 * b] == G[a, i, b]


@pytest.mark.parametrize("J", [45, 150, 1000])
def test_hash_tables_distribution_any_sketch_size(J):
    """The same uniformity for sketch sizes that are not powers of two (h = word mod J)."""
    n = J * 200
    hs, vs = O.draw_sketch(777, 3, [n], J)
    assert hs[0].min() >= 0 and hs[0].max() < J
    counts = np.bincount(hs[0], minlength=J)
    chi2 = ((counts - n / J) ** 2 / (n / J)).sum()
    assert chi2 < J + 6 * math.sqrt(2 * J)
    assert abs(vs[0].sum()) < 6 * math.sqrt(n)


# ---------------------------------------------------------------------------------------------
# part (a): Y_k = S A_(k)^T

@pytest.mark.parametrize("dims,J", [((3, 4, 5), 8), ((2, 3, 2, 4), 16), ((5, 2), 4), ((4, 3, 2, 2, 3), 32),
                                    ((3, 4, 5), 7), ((2, 3, 2, 4), 45)])
def test_data_sketch_definition_vs_dense(dims, J):
    rng = _rng(sum(dims) + J)
    A = synth.random_tensor(dims, J)
    hs, vs = _rand_tables(rng, dims, J)
    for k in range(len(dims)):
        Y = O.sketch_unfolding(A, hs, vs, J, k)
        assert Y.shape == (J, dims[k])
        assert np.allclose(Y, O.sketch_unfolding_dense(A, hs, vs, J, k), atol=1e-13)


@pytest.mark.parametrize("dims,J,density", [((5, 4, 6), 8, 0.3), ((3, 4, 2, 5), 45, 0.2), ((6, 7), 16, 1.0)])
def test_coo_sketch_equals_dense_definition(dims, J, density):
    """The coordinate form on the nonzeros of a sparse tensor (with repeated coordinates, whose
    values add up) equals the dense definition on the densified tensor, and an empty list gives 0."""
    rng = _rng(len(dims) * 7 + J)
    hs, vs = _rand_tables(rng, dims, J)
    A = synth.random_tensor(dims, J) * (rng.random(dims) < density)
    nz = np.nonzero(A)
    idx = np.stack(nz)
    vals = A[nz]
    # split every value into two repeated coordinates
    idx2 = np.concatenate([idx, idx], axis=1)
    vals2 = np.concatenate([0.25 * vals, 0.75 * vals])
    for k in range(len(dims)):
        dense = O.sketch_unfolding(A, hs, vs, J, k)
        assert np.allclose(O.sketch_unfolding_coo(idx, vals, dims, hs, vs, J, k), dense, atol=1e-13)
        assert np.allclose(O.sketch_unfolding_coo(idx2, vals2, dims, hs, vs, J, k), dense, atol=1e-13)
        empty = O.sketch_unfolding_coo(np.zeros((len(dims), 0), np.int64), np.zeros(0), dims, hs, vs, J, k)
        assert empty.shape == (J, dims[k]) and not empty.any()


def test_data_sketch_injective_hash_is_a_transpose():
    """With J = n_2, h_2 a permutation and v = +1, S is a permutation and Y_1 = P A^T."""
    A = synth.random_tensor((6, 7), 11)
    perm = np.random.default_rng(3).permutation(7)
    Y = O.sketch_unfolding(A, [np.zeros(6, int), perm], [np.ones(6), np.ones(7)], 7, 0)
    expect = np.zeros((7, 6))
    expect[perm, :] = A.T
    assert np.array_equal(Y, expect)


# ---------------------------------------------------------------------------------------------
# part (b): Lemma 1, Cor. 1, Cor. 2, Thm 1/2

def test_lemma1_and_corollaries():
    rng = _rng(7)
    J = 8
    F = O.dft_matrix(J)
    Finv = np.linalg.inv(F)
    dims = (3, 5, 4)
    hs, vs = _rand_tables(rng, dims, J)
    S1 = O.countsketch_matrix(hs[0], vs[0], J)
    S2 = O.countsketch_matrix(hs[1], vs[1], J)
    S3 = O.countsketch_matrix(hs[2], vs[2], J)
    # Lemma 1
    S12 = O.tensorsketch_matrix(hs[:2], vs[:2], J)
    assert np.allclose(S12, Finv @ O.face_split(F @ S2, F @ S1), atol=1e-12)
    # Corollary 1 (three factors)
    S123 = O.tensorsketch_matrix(hs, vs, J)
    assert np.allclose(S123, Finv @ O.face_split(O.face_split(F @ S3, F @ S2), F @ S1), atol=1e-12)
    # Corollary 2: S (B kron A) = F^{-1}[(F S2 B) [] (F S1 A)]
    A = rng.standard_normal((3, 2))
    B = rng.standard_normal((5, 3))
    assert np.allclose(S12 @ np.kron(B, A), Finv @ O.face_split(F @ S2 @ B, F @ S1 @ A), atol=1e-12)


def test_mixed_product_rule():
    rng = _rng(8)
    A, B = rng.standard_normal((3, 2)), rng.standard_normal((4, 5))
    C, D = rng.standard_normal((6, 3)), rng.standard_normal((6, 4))
    assert np.allclose(O.face_split(D, C) @ np.kron(B, A), O.face_split(D @ B, C @ A), atol=1e-12)


@pytest.mark.parametrize("dims,ranks,J", [((3, 4, 2), (1, 2, 3, 1), 8), ((2, 3, 4, 3), (1, 2, 2, 3, 1), 16),
                                          ((4, 2, 3, 2, 3), (1, 3, 2, 2, 2, 1), 16), ((5, 4), (1, 3, 1), 4),
                                          ((3, 4, 2), (1, 2, 3, 1), 9), ((2, 3, 4, 3), (1, 2, 2, 3, 1), 15)])
def test_interface_sketch_three_routes(dims, ranks, J):
    rng = _rng(len(dims) * 31 + J)
    cores = synth.random_tt(dims, ranks, J)
    hs, vs = _rand_tables(rng, dims, J)
    for k in range(len(dims)):
        dense = O.sketch_interface_dense(cores, hs, vs, J, k)
        conv = O.sketch_interface_conv(cores, hs, vs, J, k)
        fft = O.sketch_interface_fft(cores, hs, vs, J, k)
        assert dense.shape == (J, ranks[k] * ranks[k + 1])
        assert np.allclose(conv, dense, atol=1e-12)
        assert np.allclose(fft, dense, atol=1e-12)


def test_interface_sketch_conv_vs_fft_medium():
    dims, ranks, J = (20, 30, 25, 10), (1, 4, 5, 3, 1), 256
    cores = synth.random_tt(dims, ranks, 9)
    hs, vs = O.draw_sketch(99, 0, dims, J)
    for k in range(4):
        a = O.sketch_interface_conv(cores, hs, vs, J, k)
        b = O.sketch_interface_fft(cores, hs, vs, J, k)
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)


def test_data_sketch_of_tt_tensor_equals_interface_sketch():
    """For A = [[G]]: S A_(k)^T = (S H_k) G_{k(2)}^T, linking parts (a) and (b)."""
    dims, ranks, J = (6, 5, 7, 4), (1, 3, 2, 3, 1), 32
    cores = synth.random_tt(dims, ranks, 12)
    A = O.tt_full(cores)
    hs, vs = O.draw_sketch(4, 2, dims, J)
    for k in range(4):
        Y = O.sketch_unfolding(A, hs, vs, J, k)
        SH = O.sketch_interface_fft(cores, hs, vs, J, k)
        assert np.allclose(Y, SH @ O.mode2_unfold(cores[k]).T, atol=1e-10)


# ---------------------------------------------------------------------------------------------
# part (c): Eq. (ite)

def test_prox_update_vs_augmented_least_squares():
    rng = _rng(21)
    J, n, r0, r1 = 40, 7, 3, 4
    Y = rng.standard_normal((J, n))
    SH = rng.standard_normal((J, r0 * r1))
    G = rng.standard_normal((r0, n, r1))
    for sigma in (1e-3, 0.5, 3.0):
        a = O.prox_update(Y, SH, G, sigma)
        b = O.prox_update_augmented(Y, SH, G, sigma)
        assert np.allclose(a, b, atol=1e-10)


def test_prox_update_sigma_zero_is_least_squares():
    rng = _rng(22)
    Y, SH = rng.standard_normal((30, 5)), rng.standard_normal((30, 6))
    G = rng.standard_normal((2, 5, 3))
    X, *_ = np.linalg.lstsq(SH, Y, rcond=None)
    assert np.allclose(O.mode2_unfold(O.prox_update(Y, SH, G, 0.0)), X.T, atol=1e-10)


def test_prox_update_sigma_zero_singular_raises():
    Y = np.ones((4, 2))
    SH = np.zeros((4, 3))
    with pytest.raises(O.NotSPD):
        O.prox_update(Y, SH, np.zeros((1, 2, 3)), 0.0)


def test_prox_update_refuses_numerically_singular_grams():
    """Two equal columns of S H_k, or a column within 1e-9 of the span of the others, make M
    singular to working precision (pivot ratios near 1e-16 and 1e-18): refused at sigma = 0,
    accepted with sigma > 0. A system with cond(M) = 1e8 is kept and equals lstsq."""
    rng = _rng(23)
    J, n = 60, 5
    Y = rng.standard_normal((J, n))
    G = rng.standard_normal((2, n, 3))
    base = rng.standard_normal((J, 6))
    dup = base.copy()
    dup[:, 4] = dup[:, 1]
    near = base.copy()
    near[:, 5] = base[:, :5] @ rng.standard_normal(5) + 1e-9 * rng.standard_normal(J)
    for SH in (dup, near):
        with pytest.raises(O.NotSPD):
            O.prox_update(Y, SH, G, 0.0)
        a = O.prox_update(Y, SH, G, 0.5)
        assert np.allclose(a, O.prox_update_augmented(Y, SH, G, 0.5), atol=1e-9)
    U, _ = np.linalg.qr(rng.standard_normal((J, 6)))
    V, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    SH = U @ np.diag(np.logspace(0, -4, 6)) @ V.T  # cond(SH) = 1e4, cond(M) = 1e8
    X, *_ = np.linalg.lstsq(SH, Y, rcond=None)
    got = O.mode2_unfold(O.prox_update(Y, SH, G, 0.0)).T
    assert np.linalg.norm(got - X) <= 1e-6 * np.linalg.norm(X)


def test_sigma_zero_gram_is_singular_after_a_collision_in_a_square_last_core():
    """The last core G_{d-1} (r_{d-1} x n_{d-1} x 1) is square when n_{d-1} = r_{d-1}. For
    k = d-2 the sketched right interface is the CountSketch of that core's right unfolding
    (Theorem 2 with one factor); two indices sharing a bucket add two of its rows, so S H_{d-2}
    loses r_{d-2} columns of rank (checked by SVD) and the sigma = 0 Gram of Eq. (ite) is
    singular: the oracle refuses it. Distinct buckets keep full rank and the update goes through."""
    dims, ranks = (3, 5, 4), (1, 3, 4, 1)
    cores = synth.random_tt(dims, ranks, 31)
    A = synth.random_tensor(dims, 32)
    J, k = 16, 1
    vs = [np.ones(3), np.array([1.0, -1.0, 1.0, 1.0, -1.0]), np.array([1.0, -1.0, -1.0, 1.0])]
    for h2, singular in (([0, 3, 3, 9], True), ([0, 3, 6, 9], False)):  # h_0 + h_2 distinct in the second
        hs = [np.array([0, 1, 2]), np.array([3, 1, 4, 1, 5]), np.array(h2)]
        SH = O.sketch_interface_dense(cores, hs, vs, J, k)
        Y = O.sketch_unfolding(A, hs, vs, J, k)
        sv = np.linalg.svd(SH, compute_uv=False)
        s = ranks[k] * ranks[k + 1]
        rank = int(np.sum(sv > 1e-12 * sv[0]))
        if singular:
            assert rank == s - ranks[k]
            with pytest.raises(O.NotSPD):
                O.prox_update(Y, SH, cores[k], 0.0)
        else:
            assert rank == s
            X, *_ = np.linalg.lstsq(SH, Y, rcond=None)
            got = O.mode2_unfold(O.prox_update(Y, SH, cores[k], 0.0)).T
            assert np.linalg.norm(got - X) <= 1e-8 * np.linalg.norm(X)
        O.prox_update(Y, SH, cores[k], 0.5)  # the proximal term keeps M SPD


def test_identity_sketch_reduces_to_exact_prox_als():
    """m = prod_{i!=k} n_i, injective hash, v = +1: S is a permutation, so (ite) equals the exact
    proximal update of Eq. (lrtt_sub_prox)."""
    dims, ranks = (3, 4, 2), (1, 2, 2, 1)
    cores = synth.random_tt(dims, ranks, 5)
    A = synth.random_tensor(dims, 6)
    k, sigma = 1, 0.3
    J = dims[0] * dims[2]
    hs = [np.arange(3), np.zeros(4, int), np.arange(2) * 3]  # h_0(i)+h_2(j) = i + 3 j: a bijection
    vs = [np.ones(3), np.ones(4), np.ones(2)]
    Y = O.sketch_unfolding(A, hs, vs, J, k)
    SH = O.sketch_interface_dense(cores, hs, vs, J, k)
    got = O.prox_update(Y, SH, cores[k], sigma)
    H = O.interface_matrix(cores, k)
    X = np.linalg.solve(H.T @ H + sigma * np.eye(4), (O.unfold(A, k) @ H + sigma * O.mode2_unfold(cores[k])).T)
    assert np.allclose(O.mode2_unfold(got), X.T, atol=1e-12)


# ---------------------------------------------------------------------------------------------
# orthogonalisation

@pytest.mark.parametrize("shape", [(12, 4), (5, 5), (3, 7)])
def test_qr_nonneg(shape):
    M = _rng(sum(shape)).standard_normal(shape)
    Q, R = O.qr_nonneg(M)
    assert np.allclose(Q @ R, M, atol=1e-12)
    assert np.allclose(np.triu(R), R)
    assert np.all(np.diag(R) >= 0)
    m, n = shape
    q = min(m, n)
    assert np.allclose(Q[:, :q].T @ Q[:, :q], np.eye(q), atol=1e-12)
    assert Q.shape == (m, n) and R.shape == (n, n)


def test_orthogonalization_invariants():
    cores = synth.random_tt((4, 5, 3, 6), (1, 3, 4, 3, 1), 13)
    T = O.tt_full(cores)
    oc = O.orthogonalize_right_to_left(cores)
    assert np.allclose(O.tt_full(oc), T, atol=1e-10 * np.abs(T).max())
    for k in range(1, 4):
        R = O.right_unfold(oc[k])
        assert np.allclose(R @ R.T, np.eye(R.shape[0]), atol=1e-12)
    # ||[[G]]|| lives in the first core after right-to-left orthogonalisation
    assert abs(np.linalg.norm(oc[0].ravel()) - np.linalg.norm(T.ravel())) < 1e-10 * np.linalg.norm(T.ravel())
    oc2 = list(oc)
    O.left_orthogonalize_step(oc2, 0)
    L = O.left_unfold(oc2[0])
    assert np.allclose(L.T @ L, np.eye(L.shape[1]), atol=1e-12)
    assert np.allclose(O.tt_full(oc2), T, atol=1e-10 * np.abs(T).max())


# ---------------------------------------------------------------------------------------------
# whole method

def test_exact_tt_is_a_fixed_point():
    """If A = [[G*]] then G* is a fixed point of Eq. (ite) for any sigma (Y = S H G*^T)."""
    dims, ranks = (6, 7, 5, 6), (1, 3, 3, 2, 1)
    cores = synth.random_tt(dims, ranks, 14)
    A = O.tt_full(cores)
    for sigma in (0.0, 0.5):
        new, rc = O.tt_ts_sweep(A, cores, 77, 0, 64, sigma)
        assert O.rel_error(A, new) < 1e-11
        assert rc < 1e-10


def test_rel_change_by_hand_on_a_two_by_two_matrix():
    """One sweep on A = [[3, 1], [1, 2]] with rank-1 cores g0 = (1, 0), g1 = (1, 1), sigma = 1/2,
    and a draw whose hashes are injective at J = 2, so that S is a signed permutation and
    S^T S = I. Worked by hand:
      right-to-left orthogonalisation: q1 = g1 / |g1|, centre c0 = |g1| g0;
      core 0: (S H_0)^T (S H_0) = 1, Y_0^T S H_0 = A S^T S q1 = A q1, so
              G0 = (A q1 + sigma c0) / (1 + sigma); QR: q0 = G0 / |G0|, centre c1 = |G0| q1;
      core 1: G1 = (A^T q0 + sigma c1) / (1 + sigma);
      rel-change (Sec. 5) = max(|G0 - c0| / |G0|, |G1 - c1| / |G1|), each over the NEW core's norm."""
    A = np.array([[3.0, 1.0], [1.0, 2.0]])
    g0, g1, sigma, J = np.array([1.0, 0.0]), np.array([1.0, 1.0]), 0.5, 2
    seed = next(sd for sd in range(1000)
                if all(len(set(h.tolist())) == 2 for h in O.draw_sketch(sd, 0, (2, 2), J)[0]))
    q1 = g1 / np.linalg.norm(g1)
    c0 = np.linalg.norm(g1) * g0
    G0 = (A @ q1 + sigma * c0) / (1 + sigma)
    q0 = G0 / np.linalg.norm(G0)
    c1 = np.linalg.norm(G0) * q1
    G1 = (A.T @ q0 + sigma * c1) / (1 + sigma)
    ch = max(np.linalg.norm(G0 - c0) / np.linalg.norm(G0), np.linalg.norm(G1 - c1) / np.linalg.norm(G1))
    cores = [g0.reshape(1, 2, 1), g1.reshape(1, 2, 1)]
    new, rc = O.tt_ts_sweep(A, cores, seed, 0, J, sigma)
    assert abs(rc - ch) <= 1e-12, (rc, ch)
    assert np.allclose(new[0].ravel(), q0, atol=1e-12) and np.allclose(new[1].ravel(), G1, atol=1e-12)
    # the normalisation matters here: over the old cores' norms the value differs
    wrong = max(np.linalg.norm(G0 - c0) / np.linalg.norm(c0), np.linalg.norm(G1 - c1) / np.linalg.norm(c1))
    assert abs(wrong - ch) > 1e-2


def test_exact_recovery_from_random_init():
    dims, ranks = (8, 9, 7, 8), (1, 3, 3, 3, 1)
    A = O.tt_full(synth.random_tt(dims, ranks, 15))
    init = synth.random_tt(dims, ranks, 16)
    cores, ch = O.tt_ts(A, init, 31, 128, 1e-3, 30)
    assert O.rel_error(A, cores) < 1e-8


def test_unsketched_prox_als_monotone_and_vs_ttsvd():
    dims, ranks = (6, 7, 6, 5), (1, 3, 4, 3, 1)
    rng = np.random.default_rng(17)
    A = synth.add_noise(O.tt_full(synth.random_tt(dims, ranks, 17)), 0.05, rng)
    svd_cores = O.tt_svd(A, ranks)
    e_svd = O.rel_error(A, svd_cores)
    cores = svd_cores
    errs = [e_svd]
    for _ in range(6):
        cores = O.prox_als_sweep(A, cores, 0.1)
        errs.append(O.rel_error(A, cores))
    assert all(errs[i + 1] <= errs[i] + 1e-12 for i in range(len(errs) - 1))
    # TT-SVD quasi-optimality: e_svd <= sqrt(d-1) * e_best <= sqrt(d-1) * e_als
    assert e_svd <= math.sqrt(len(dims) - 1) * errs[-1] + 1e-12


def test_ttsvd_exact_on_tt_tensor():
    dims, ranks = (5, 6, 4, 3), (1, 2, 3, 2, 1)
    A = O.tt_full(synth.random_tt(dims, ranks, 18))
    assert O.rel_error(A, O.tt_svd(A, ranks)) < 1e-12


def test_sketched_gram_unbiased():
    """E_S[(S H)^T (S H)] = H^T H (TensorSketch preserves inner products in expectation)."""
    dims, ranks, J = (4, 5, 3), (1, 2, 2, 1), 16
    cores = synth.random_tt(dims, ranks, 19)
    k = 1
    H = O.interface_matrix(cores, k)
    acc = np.zeros((4, 4))
    acc2 = np.zeros((4, 4))
    T = 600
    for t in range(T):
        hs, vs = O.draw_sketch(1000 + t, 0, dims, J)
        SH = O.sketch_interface_fft(cores, hs, vs, J, k)
        G = SH.T @ SH
        acc += G
        acc2 += G * G
    mean = acc / T
    sd = np.sqrt(np.maximum(acc2 / T - mean ** 2, 0) / T)
    assert np.all(np.abs(mean - H.T @ H) <= 5 * sd + 1e-9)


def test_rel_error_closed_forms():
    cores = synth.random_tt((3, 4, 5), (1, 2, 2, 1), 20)
    T = O.tt_full(cores)
    assert O.rel_error(T, cores) < 1e-14
    assert abs(O.rel_error(2 * T, cores) - 0.5) < 1e-14
