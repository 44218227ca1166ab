"""The FP64 form of the proximal update (Eq. (ite)): an FP64 Gram of the FP32 sketches, an FP64
Cholesky and FP64 triangular solves. A context takes it when sigma = 0 (Sec. 5 runs sigma = 0,
where M is not SPD by construction and its conditioning is unbounded) or with
TT_FLAG_FP64_SOLVE. Checked through the C ABI against the CPU FP64 oracle:
  * single updates, including ill-conditioned systems (cond(M) = 1e6) that the FP32 form cannot
    resolve, to 1e-6 relative: both sides solve the same FP32-rounded inputs in FP64;
  * the first sigma = 0 update of the paper's sinc tensor (Sec. 5, m = 45), which is numerically
    of rank 2 (so later sigma = 0 iterates depend on how a QR treats rounding noise);
  * refusals: TT_ENOTSPD exactly where the oracle's Cholesky refuses. On the oscillatory
    function (rank 20, m = 1000) the first sweep's draw puts two indices of the last, square,
    core into one bucket, so S H_4 loses rank and the sigma = 0 Gram of core 4 is singular; the
    GPU must refuse that update and hold the cores the oracle holds at that point."""
import numpy as np
import pytest

import tt_oracle as O
from paper_2309_08093_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_08093_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2309_08093_gb300 import lib  # noqa: E402


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def _system(J, n, r0, r1, cond, seed):
    """S H_k with singular values spread from 1 to 1/cond, a random right-hand side and centre."""
    rng = np.random.default_rng(seed)
    s = r0 * r1
    U, _ = np.linalg.qr(rng.standard_normal((J, s)))
    V, _ = np.linalg.qr(rng.standard_normal((s, s)))
    SH = (U @ np.diag(np.logspace(0, -np.log10(cond), s)) @ V.T).astype(np.float32)
    Y = rng.standard_normal((J, n)).astype(np.float32)
    G = rng.standard_normal((r0, n, r1)).astype(np.float32)
    return SH, Y, G


def _gpu_update(SH, Y, G, sigma, flags):
    J, s = SH.shape
    r0, n, r1 = G.shape
    dims = (n, 4, 3) if r0 == 1 else (5, n, 3)
    k = 0 if r0 == 1 else 1
    ranks = (1, r1, 1, 1) if k == 0 else (1, r0, r1, 1)
    ctx = lib.Context(dims, ranks, J, sigma, 5, "f32", flags=flags)
    Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda()
    SHd = torch.from_numpy(np.ascontiguousarray(SH.T)).cuda()
    core = torch.from_numpy(np.ascontiguousarray(G.ravel(order="F"))).cuda()
    before = core.clone()
    try:
        ctx.tt_prox_update(Yd, SHd, core, k)
        code = lib.TT_OK
    except lib.TtError as e:
        code = e.code
    out = core.cpu().numpy().astype(np.float64).reshape(r0, n, r1, order="F")
    unchanged = bool(torch.equal(core, before))
    ctx.close()
    return code, out, unchanged


@pytest.mark.parametrize("J,n,r0,r1,sigma,cond,flags", [
    (1024, 50, 5, 5, 0.0, 2.0, 0),             # sigma = 0: the FP64 form by default
    (1024, 50, 5, 5, 0.0, 1e3, 0),             # cond(M) = 1e6
    (4096, 100, 10, 10, 1e-3, 10.0, lib.TT_FLAG_FP64_SOLVE),
    (45, 10, 5, 5, 0.0, 30.0, 0),              # the paper's m = 45 (Sec. 5)
    (1000, 10, 20, 20, 0.0, 50.0, 0),          # 400 unknowns (the oscillatory function's cores)
    (2000, 37, 12, 13, 0.0, 1e2, 0),           # ragged: 156 unknowns, n not a multiple of the chunk
    (512, 300, 1, 7, 0.0, 5.0, 0),             # first core (r0 = 1), many right-hand sides
])
def test_fp64_update_matches_oracle(J, n, r0, r1, sigma, cond, flags):
    SH, Y, G = _system(J, n, r0, r1, cond, J + n + r0)
    code, got, _ = _gpu_update(SH, Y, G, sigma, flags)
    assert code == lib.TT_OK
    ref = O.prox_update(Y.astype(np.float64), SH.astype(np.float64), G.astype(np.float64), sigma)
    assert rel(got, ref) <= 1e-6, rel(got, ref)


def test_fp32_form_refuses_what_it_cannot_resolve():
    """sigma = 1e-9 with cond(S H) = 1e4 (cond(M) = 1e8): the FP32 form's pivots fall below 1e-4
    of the largest diagonal entry and it refuses (core unchanged); the FP64 form solves the same
    system."""
    SH, Y, G = _system(1024, 30, 4, 5, 1e4, 3)
    code, _, unchanged = _gpu_update(SH, Y, G, 1e-9, 0)
    assert code == lib.TT_ENOTSPD and unchanged
    code, got, _ = _gpu_update(SH, Y, G, 1e-9, lib.TT_FLAG_FP64_SOLVE)
    assert code == lib.TT_OK
    ref = O.prox_update(Y.astype(np.float64), SH.astype(np.float64), G.astype(np.float64), 1e-9)
    assert rel(got, ref) <= 1e-5, rel(got, ref)


@pytest.mark.parametrize("kind", ["duplicate", "zero"])
def test_fp64_form_refuses_singular_grams_like_the_oracle(kind):
    SH, Y, G = _system(512, 20, 3, 4, 3.0, 9)
    if kind == "duplicate":
        SH[:, 7] = SH[:, 2]
    else:
        SH[:, 0] = 0.0
    with pytest.raises(O.NotSPD):
        O.prox_update(Y.astype(np.float64), SH.astype(np.float64), G.astype(np.float64), 0.0)
    code, _, unchanged = _gpu_update(SH, Y, G, 0.0, 0)
    assert code == lib.TT_ENOTSPD and unchanged


def _oracle_sweep_until_refusal(A, cores, seed, sweep, J, sigma):
    """Algorithm 1's sweep (orthogonalise right to left, then update and QR core by core), stopping
    at the first update the oracle's Cholesky refuses. Returns (cores at that point, refused k or
    None)."""
    d = A.ndim
    cores = O.orthogonalize_right_to_left(cores)
    hs, vs = O.draw_sketch(seed, sweep, A.shape, J)
    for k in range(d):
        SH = O.sketch_interface_fft(cores, hs, vs, J, k)
        Y = O.sketch_unfolding(A, hs, vs, J, k)
        try:
            cores[k] = O.prox_update(Y, SH, cores[k], sigma)
        except O.NotSPD:
            return cores, k
        if k < d - 1:
            O.left_orthogonalize_step(cores, k)
    return cores, None


def test_sigma_zero_refusal_matches_the_oracle_on_the_oscillatory_function():
    dims, ranks, J, seed = (10,) * 6, (1, 10, 20, 20, 20, 10, 1), 1000, 20230917
    A = np.asarray(synth.paper_function_tensor("osc"), np.float32)
    init = synth.random_tt(dims, ranks, 100)
    ref, k_ref = _oracle_sweep_until_refusal(A.astype(np.float64), init, seed, 0, J, 0.0)
    assert k_ref == 4  # the mode-5 collision of this draw
    hs, _ = O.draw_sketch(seed, 0, dims, J)
    assert len(set(hs[5].tolist())) < dims[5]
    ctx = lib.Context(dims, ranks, J, 0.0, seed, "f32")
    Ad = lib.device_tensor(A.ravel(order="F"), "f32")
    dc = lib.device_cores(init)
    with pytest.raises(lib.TtError) as e:
        ctx.tt_prox_als_sweep(Ad, dc, 1, 0, rel_change=False)
    assert e.value.code == lib.TT_ENOTSPD
    got = lib.host_cores(dc, ranks, dims)
    ctx.close()
    assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4, rel(O.tt_full(got), O.tt_full(ref))
    for k in range(5):  # cores 0..3 updated and left-orthogonal, core 4 holding the absorbed R
        assert rel(got[k], ref[k]) <= 1e-3, (k, rel(got[k], ref[k]))


def test_sigma_zero_update_on_the_sinc_tensor_matches_the_oracle():
    """The first sigma = 0 update of the paper's sinc tensor (m = 45; Sec. 5), through the C ABI
    step by step: right-to-left orthogonalisation, S H_0, Y_0, the FP64 update. It is the least
    squares solution for core 0, unique, and matches the oracle's (1e-5). It is also numerically
    of rank 2, as the data are: the tensor's first unfolding has singular values 1, 5.1e-5,
    6.8e-9, ... So the QR that follows takes three columns of Q from rounding, in the oracle and on
    the GPU alike, and later sigma = 0 iterates of two correct implementations part ways; what
    both must agree on are the update and its singular values (to the level of that noise)."""
    dims, ranks, J, seed = (10,) * 6, (1, 5, 5, 5, 5, 5, 1), 45, 20230917
    A32 = np.asarray(synth.paper_function_tensor("sinc"), np.float32)
    A = A32.astype(np.float64)
    init = synth.random_tt(dims, ranks, 100)
    ref = O.orthogonalize_right_to_left([np.asarray(g, np.float32).astype(np.float64) for g in init])
    hs, vs = O.draw_sketch(seed, 0, dims, J)
    SH_ref = O.sketch_interface_fft(ref, hs, vs, J, 0)
    Y_ref = O.sketch_unfolding(A, hs, vs, J, 0)
    G_ref = O.prox_update(Y_ref, SH_ref, ref[0], 0.0)
    ctx = lib.Context(dims, ranks, J, 0.0, seed, "f32")
    Ad = lib.device_tensor(A32.ravel(order="F"), "f32")
    dc = lib.device_cores(init)
    ctx.tt_orthogonalize(dc, -1)
    SH = torch.zeros(J * ranks[1], device="cuda")
    ctx.tt_sketch_interface(dc, 0, 0, SH)
    Y = [torch.zeros(J * n, device="cuda") for n in dims]
    ctx.tt_sketch_unfold(Ad, 0, 0, Y)
    ctx.tt_prox_update(Y[0], SH, dc[0], 0)
    got = lib.host_cores(dc, ranks, dims)[0]
    ctx.close()
    assert rel(got, G_ref) <= 1e-5, rel(got, G_ref)
    sv_got = np.linalg.svd(O.left_unfold(got), compute_uv=False)
    sv_ref = np.linalg.svd(O.left_unfold(G_ref), compute_uv=False)
    # Weyl: every singular value moves by at most ||G_gpu - G_ref||_2 <= 1e-5 ||G_ref||_F
    assert np.abs(sv_got - sv_ref).max() <= 1e-5 * np.linalg.norm(G_ref.ravel())
    assert sv_ref[2] / sv_ref[0] < 1e-7 and sv_got[2] / sv_got[0] < 1e-6  # rank 2 to working precision
