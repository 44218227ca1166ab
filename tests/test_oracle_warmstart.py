"""Pins for the warm-start oracle: each check compares it with something other than itself
(closed forms, finite differences, library routines, gauge invariance, round trips). CPU only."""
import math

import numpy as np
import pytest

import tt_oracle as O
import tt_warmstart as W

torch = pytest.importorskip("torch")


# ---------------------------------------------------------------------------------------------
# BF16 rounding and GELU

def test_round_bf16_closed_form_ties_and_torch():
    u = 2.0 ** -7  # BF16 spacing just above 1
    assert W.round_bf16(np.array([1.0]))[0] == 1.0
    assert W.round_bf16(np.array([1.0 + u / 2]))[0] == 1.0                 # tie -> even (1.0)
    assert W.round_bf16(np.array([1.0 + 3 * u / 2]))[0] == 1.0 + 2 * u      # tie -> even (1 + 2u)
    assert W.round_bf16(np.array([1.0 + 0.6 * u]))[0] == 1.0 + u
    assert W.round_bf16(np.array([-1.0 - 0.4 * u]))[0] == -1.0
    x = np.random.default_rng(1).standard_normal(10000) * np.exp(np.random.default_rng(2).uniform(-20, 20, 10000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(W.round_bf16(x), ref)


def test_gelu_identities_library_and_derivative():
    z = np.linspace(-6, 6, 241)
    g = W.gelu(z)
    np.testing.assert_allclose(g - W.gelu(-z), z, atol=1e-14)               # GELU(z) - GELU(-z) = z
    assert W.gelu(np.array([0.0]))[0] == 0.0
    assert abs(W.gelu(np.array([10.0]))[0] - 10.0) < 1e-20 + 1e-15
    ref = torch.nn.functional.gelu(torch.from_numpy(z)).numpy()             # exact (erf) GELU
    np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-14)
    h = 1e-6
    fd = (W.gelu(z + h) - W.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(W.gelu_grad(z), fd, rtol=1e-7, atol=1e-8)
    assert abs(W.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


# ---------------------------------------------------------------------------------------------
# the network

def _params(rng, n_in, h, n_out, scale=0.3):
    return {"W1": rng.standard_normal((h, n_in)) * scale, "b1": rng.standard_normal(h) * 0.1,
            "W2": rng.standard_normal((h, h)) * scale, "b2": rng.standard_normal(h) * 0.1,
            "W3": rng.standard_normal((n_out, h)) * scale, "b3": rng.standard_normal(n_out) * 0.1}


def test_mlp_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    P = _params(rng, 7, 6, 5)
    X = rng.standard_normal((4, 7))
    T = rng.standard_normal((4, 5))
    loss, g, _ = W.mlp_loss_grads(P, X, T)
    h = 1e-6
    for name, p in P.items():
        fd = np.zeros_like(p)
        for idx in np.ndindex(p.shape):
            old = p[idx]
            p[idx] = old + h
            lp, _, _ = W.mlp_loss_grads(P, X, T)
            p[idx] = old - h
            lm, _, _ = W.mlp_loss_grads(P, X, T)
            p[idx] = old
            fd[idx] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g[name], fd, rtol=1e-6, atol=1e-9, err_msg=name)


def test_mlp_matches_torch_autograd():
    rng = np.random.default_rng(4)
    P = _params(rng, 11, 9, 13)
    X = rng.standard_normal((6, 11))
    T = rng.standard_normal((6, 13))
    loss, g, Y = W.mlp_loss_grads(P, X, T)
    tp = {k: torch.tensor(v, requires_grad=True) for k, v in P.items()}
    xt = torch.tensor(X)
    a = torch.nn.functional.gelu(xt @ tp["W1"].T + tp["b1"])
    a = torch.nn.functional.gelu(a @ tp["W2"].T + tp["b2"])
    y = a @ tp["W3"].T + tp["b3"]
    lt = ((y - torch.tensor(T)) ** 2).mean()
    lt.backward()
    assert abs(loss - float(lt.detach())) < 1e-12
    for k in P:
        np.testing.assert_allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-13, err_msg=k)


def test_mlp_bf16_rounding_points():
    """With every operand already BF16-representable and the GELU outputs rounded by hand, the
    BF16 form must equal the FP64 form on the rounded inputs; in general it stays within the
    BF16 error."""
    rng = np.random.default_rng(5)
    P = _params(rng, 16, 8, 12)
    X = rng.standard_normal((5, 16))
    T = rng.standard_normal((5, 12))
    l64, g64, _ = W.mlp_loss_grads(P, X, T)
    l16, g16, _ = W.mlp_loss_grads(P, X, T, bf16=True)
    assert abs(l16 - l64) <= 2e-2 * l64
    for k in P:
        assert np.linalg.norm(g16[k] - g64[k]) <= 3e-2 * np.linalg.norm(g64[k]), k
    # exactness: forward with BF16-representable operands equals the plain forward
    Pq = {k: (W.round_bf16(v) if k.startswith("W") else v) for k, v in P.items()}
    Xq = W.round_bf16(X)
    Yq, c = W.mlp_forward(Pq, Xq, bf16=True)
    Z1 = Xq @ Pq["W1"].T + Pq["b1"]
    Z2 = W.round_bf16(W.gelu(Z1)) @ Pq["W2"].T + Pq["b2"]
    Y = W.round_bf16(W.gelu(Z2)) @ Pq["W3"].T + Pq["b3"]
    np.testing.assert_allclose(Yq, Y, rtol=0, atol=1e-13)


def test_adam_first_step_closed_form_and_torch():
    rng = np.random.default_rng(6)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    new, m, v = W.adam_step(th, g, np.zeros(50), np.zeros(50), 1, lr, b1, b2, eps)
    np.testing.assert_allclose(new, th - lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
    # several steps against torch.optim.Adam
    tt = torch.tensor(th, requires_grad=True)
    opt = torch.optim.Adam([tt], lr=lr, betas=(b1, b2), eps=eps)
    cur, m, v = th.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        gt = rng.standard_normal(50)
        cur, m, v = W.adam_step(cur, gt, m, v, t, lr, b1, b2, eps)
        tt.grad = torch.tensor(gt)
        opt.step()
    np.testing.assert_allclose(cur, tt.detach().numpy(), rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------------------------
# gauge fixing

def _random_tt(rng, dims, ranks):
    return [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(len(dims))]


def test_canonicalize_reconstruction_orthonormality_order_sign():
    rng = np.random.default_rng(7)
    dims, ranks = (5, 6, 3, 4), (1, 4, 3, 4, 1)
    cs = _random_tt(rng, dims, ranks)
    cc = W.canonicalize_right(cs)
    np.testing.assert_allclose(O.tt_full(cc), O.tt_full(cs), rtol=1e-12, atol=1e-12)
    for k in range(1, len(dims)):
        R = cc[k].reshape(ranks[k], -1, order="F")
        np.testing.assert_allclose(R @ R.T, np.eye(ranks[k]), atol=1e-12)
        w = np.tile(np.arange(1, dims[k] + 1), ranks[k + 1])
        assert np.all(R @ w > 0)
    # rows of every canonical core are the right singular vectors of the tensor unfolding
    # between modes k-1 and k, in decreasing order (checked on the full tensor by brute force)
    A = O.tt_full(cs)
    for k in range(1, len(dims)):
        Ak = A.reshape(int(np.prod(dims[:k])), -1, order="F")
        _, s, Vt = np.linalg.svd(Ak, full_matrices=False)
        # row space of Ak in the coordinates of G_k^R: contract the right-canonical tail
        tail = cc[k]
        for j in range(k + 1, len(dims)):
            tail = np.einsum("aib,bjc->aijc", tail, cc[j]).reshape(tail.shape[0], -1, cc[j].shape[2], order="F")
        rows = tail.reshape(ranks[k], -1, order="F")
        np.testing.assert_allclose(np.abs(rows), np.abs(Vt[:ranks[k]]), atol=1e-10)
        assert np.all(np.diff(s[:ranks[k]]) < 0)


def test_canonicalize_is_gauge_invariant():
    """Inserting M M^{-1} between neighbouring cores changes no tensor; the canonical form must not
    change either."""
    rng = np.random.default_rng(8)
    dims, ranks = (6, 5, 4, 7), (1, 3, 4, 2, 1)
    cs = _random_tt(rng, dims, ranks)
    gauged = [c.copy() for c in cs]
    for k in range(len(dims) - 1):
        r = ranks[k + 1]
        M = rng.standard_normal((r, r)) + 2 * np.eye(r)
        gauged[k] = np.einsum("aib,bc->aic", gauged[k], M)
        gauged[k + 1] = np.einsum("cb,bid->cid", np.linalg.inv(M), gauged[k + 1])
    np.testing.assert_allclose(O.tt_full(gauged), O.tt_full(cs), rtol=1e-10, atol=1e-10)
    a, b = W.canonicalize_right(cs), W.canonicalize_right(gauged)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-8, atol=1e-9)


def test_canonicalize_matches_tt_svd_order3():
    """A rank-(1, r, r, 1) TT of a generic tensor: the canonical last core's rows span the top
    right singular subspace of the last unfolding (the TT-SVD from the right)."""
    rng = np.random.default_rng(9)
    dims, ranks = (4, 5, 6), (1, 4, 6, 1)
    A = rng.standard_normal(dims)
    cs = O.tt_svd(A, ranks)
    cc = W.canonicalize_right(cs)
    last = cc[-1].reshape(ranks[-2], -1, order="F")
    Ak = A.reshape(-1, dims[-1], order="F").T           # n_last x rest
    U, s, Vt = np.linalg.svd(Ak, full_matrices=False)
    P1 = last.T @ last
    P2 = U[:, :ranks[-2]] @ U[:, :ranks[-2]].T
    np.testing.assert_allclose(P1, P2, atol=1e-10)


# ---------------------------------------------------------------------------------------------
# summary and targets

def test_canonicalize_zero_pads_rank_deficient_splits():
    """Ranks (1, 4, 2, 4, 1) with n_2 = 1: the split after mode 2 has rank <= 2 < 4, so two rows of
    the last core must come out zero and the tensor unchanged."""
    rng = np.random.default_rng(13)
    dims, ranks = (5, 4, 1, 6), (1, 4, 2, 4, 1)
    cs = _random_tt(rng, dims, ranks)
    cc = W.canonicalize_right(cs)
    np.testing.assert_allclose(O.tt_full(cc), O.tt_full(cs), rtol=1e-10, atol=1e-10)
    last = cc[-1].reshape(4, -1, order="F")
    np.testing.assert_allclose(last[2:], 0.0, atol=0)
    np.testing.assert_allclose(last[:2] @ last[:2].T, np.eye(2), atol=1e-12)


def test_summary_layout_scale_and_rms():
    rng = np.random.default_rng(10)
    Y = [rng.standard_normal((16, n)) for n in (3, 5, 2)]
    x, s = W.ws_summary(Y, 4)
    assert x.shape == (4 * 10,)
    assert abs(float(np.mean(x * x)) - 1.0) < 1e-12
    raw = np.concatenate([Y[0][:4].T.ravel(), Y[1][:4].T.ravel(), Y[2][:4].T.ravel()])
    np.testing.assert_allclose(x, raw / math.sqrt(np.mean(raw ** 2)), rtol=1e-14)
    assert x[4 * 3 + 2 * 4 + 1] * math.sqrt(np.mean(raw ** 2)) == pytest.approx(Y[1][1, 2])
    assert s == pytest.approx(math.sqrt(float((Y[0] ** 2).sum())))


def test_summary_scale_estimates_the_norm():
    """E ||S a||^2 = ||a||^2 for the TensorSketch of Sec. 2.2: the mean of ||Y_0||^2 over draws
    approaches ||A||^2."""
    rng = np.random.default_rng(11)
    dims, J = (6, 5, 4), 64
    A = rng.standard_normal(dims)
    vals = []
    for sweep in range(200):
        hs, vs = O.draw_sketch(3, sweep, dims, J)
        vals.append(float(np.sum(O.sketch_unfolding(A, hs, vs, J, 0) ** 2)))
    assert abs(np.mean(vals) / np.sum(A ** 2) - 1.0) < 0.05


def test_targets_round_trip_and_unit_rms():
    rng = np.random.default_rng(12)
    dims, ranks = (7, 6, 3, 5), (1, 4, 3, 4, 1)
    cc = W.canonicalize_right(_random_tt(rng, dims, ranks))
    y = W.ws_targets(cc, 2.5)
    assert y.size == sum(ranks[k] * dims[k] * ranks[k + 1] for k in range(4))
    back = W.ws_cores(y, 2.5, dims, ranks)
    for a, b in zip(back, cc):
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-15)
    o = ranks[0] * dims[0] * ranks[1]
    for k in range(1, 4):  # right-orthonormal cores -> unit RMS after scaling
        sz = ranks[k] * dims[k] * ranks[k + 1]
        assert abs(float(np.mean(y[o:o + sz] ** 2)) - 1.0) < 1e-12
        o += sz
