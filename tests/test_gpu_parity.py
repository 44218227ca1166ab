"""GPU parity: the CUDA library (called through the C ABI) against the CPU FP64 oracle on the
same seeded inputs and hash draws. Floating-point outputs are compared in relative Frobenius
norm (sums in different orders) and, for the data and interface sketches, entry by entry
against a bound that any summation order meets: for Y_k, 1e-5 of (the largest |entry| plus the
sum of |terms| of the bucket), so a dropped or mis-signed term of a small bucket still fails;
for S H_k, 1e-5 of each column's largest |entry|. Buckets with cancellation make a plain
element-wise relative error meaningless. Tolerance 1e-5 for FP32 work; integer tables
bit-exact."""
import numpy as np
import pytest

import tt_oracle as O
from conftest import read_golden
from paper_2309_08093_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_08093_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2309_08093_gb300 import lib  # noqa: E402

TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


def oracle_tables(ctx_dims, seed, sweep, J):
    hs, vs = O.draw_sketch(seed, sweep, ctx_dims, J)
    return np.concatenate(hs).astype(np.int32), np.concatenate(vs).astype(np.int8)


def split_tables(h, v, dims):
    hs, vs, o = [], [], 0
    for n in dims:
        hs.append(h[o:o + n].astype(np.int64))
        vs.append(v[o:o + n].astype(np.float64))
        o += n
    return hs, vs


# ---------------------------------------------------------------------------------------------
# a0: hash / sign tables

@pytest.mark.parametrize("dims,J,seed,sweep", [((50, 50, 50), 1024, 935972268168698347, 0),
                                               ((100, 100, 100, 100), 4096, 7, 19),
                                               ((3, 1, 7), 2, 2**63 + 5, 3),
                                               ((40,) * 5, 8192, 123, 2**40 + 1),
                                               ((256, 256, 3, 128), 16384, 0, 0),
                                               ((50, 50, 50), 150, 11, 2), ((40,) * 4, 2000, 5, 1),
                                               ((3, 1, 7), 3, 9, 0), ((10,) * 6, 45, 2**62 + 1, 7)])
def test_tables_bit_exact(dims, J, seed, sweep):
    ranks = (1,) + (1,) * (len(dims) - 1) + (1,)
    ctx = lib.Context(dims, ranks, J, 1e-3, seed, "f32")
    h, v = ctx.tt_sketch_tables(sweep)
    ho, vo = oracle_tables(dims, seed, sweep, J)
    assert np.array_equal(h, ho)
    assert np.array_equal(v, vo)
    ctx.close()


def test_fixed_sketch_flag_ignores_sweep():
    ctx = lib.Context((5, 6, 7), (1, 2, 2, 1), 64, 1e-3, 99, "f32", flags=lib.TT_FLAG_FIXED_SKETCH)
    h0, v0 = ctx.tt_sketch_tables(0)
    h1, v1 = ctx.tt_sketch_tables(5)
    assert np.array_equal(h0, h1) and np.array_equal(v0, v1)
    ctx.close()


# ---------------------------------------------------------------------------------------------
# worked example of Sec. 2.2 on the GPU

def test_worked_example_on_gpu():
    g = read_golden("tensorsketch_worked_example.txt")
    S = np.array([[float(x) for x in row] for row in g["S"]])
    ctx = lib.Context((2, 2, 1), (1, 1, 1, 1), 2, 0.0, 0, "f32")
    h = np.array([int(x) - 1 for x in g["h1"][0]] + [int(x) - 1 for x in g["h2"][0]] + [0], np.int32)
    v = np.array([int(x) for x in g["v1"][0]] + [int(x) for x in g["v2"][0]] + [1], np.int8)
    ctx.tt_sketch_set_tables(h, v)
    A = np.arange(1.0, 5.0)
    Ad = torch.tensor(A, dtype=torch.float32, device="cuda")
    Y = [torch.zeros(2, 2, device="cuda"), torch.zeros(2, 2, device="cuda"), torch.zeros(2, 1, device="cuda")]
    ctx.tt_sketch_unfold(Ad, -1, 0, Y)
    torch.cuda.synchronize()
    assert np.array_equal(Y[2].cpu().numpy()[:, 0], S @ A)
    ctx.close()


# ---------------------------------------------------------------------------------------------
# a1: data sketch Y_k = S A_(k)^T

CASES_A = [((7, 5, 9), 64, "f32"), ((3, 5, 7, 2), 16, "f32"), ((50, 50, 50), 1024, "f64"),
           ((33, 17, 9, 5), 512, "bf16"), ((40, 12, 10, 6), 256, "fp8"), ((64, 3, 1, 20), 128, "f32"),
           ((1, 6, 8), 32, "f32"), ((100, 30, 20), 4096, "f32"), ((130, 7, 11), 2, "f32"),
           ((300, 4, 5), 16384, "bf16"), ((12, 10, 8, 6, 4), 8192, "bf16"), ((41, 23, 6), 256, "f32"),
           # sketch sizes that are not powers of two (the paper's m of Sec. 5)
           ((7, 5, 9), 45, "f32"), ((20, 18, 16), 150, "bf16"), ((16, 12, 10, 8), 1000, "f32"),
           ((33, 17, 9, 5), 200, "fp8"), ((12, 10, 8), 2000, "f64"), ((10,) * 6, 45, "f32"),
           # fibres whose length is not a multiple of 16 bytes (8- and 4-byte vectors, up to 16 per lane)
           ((62, 9, 7), 512, "f32"), ((30, 7, 11), 256, "bf16"), ((123, 8, 6), 1024, "f32"),
           ((126, 5, 4, 3), 2048, "f32"), ((67, 12, 5), 512, "fp8"),
           # FP64 with odd n_0 (8-byte grid); window staging with long fibres (one fibre per slot of
           # 32 lanes), fibres too long for it (the narrow-vector path), J not a multiple of 4
           ((25, 6, 7), 512, "f64"), ((301, 5, 3), 1024, "f32"), ((509, 3, 2), 256, "f32"),
           ((515, 3, 2), 256, "f32"), ((600, 3, 2), 128, "fp8"), ((45, 9, 4), 150, "bf16")]


def _data(dims, storage, seed):
    a = synth.random_tensor(dims, seed)
    flat, scales, exact = synth.quantize(a, storage)
    return flat, scales, exact


@pytest.mark.parametrize("dims,J,storage", CASES_A)
def test_unfold_sketch_parity(dims, J, storage):
    seed = 1000 + sum(dims) + J
    flat, scales, exact = _data(dims, storage, seed)
    ranks = (1,) * (len(dims) + 1)
    ctx = lib.Context(dims, ranks, J, 1e-3, seed, storage)
    Ad = lib.device_tensor(flat, storage)
    sd = torch.tensor(scales, device="cuda") if scales is not None else None
    Y = [torch.zeros(J * n, device="cuda") for n in dims]
    for sweep in (0, 3):
        ctx.tt_sketch_unfold(Ad, -1, sweep, Y, scales=sd)
        torch.cuda.synchronize()
        hs, vs = O.draw_sketch(seed, sweep, dims, J)
        ones = [np.ones_like(v) for v in vs]
        for k in range(len(dims)):
            ref = O.sketch_unfolding(exact, hs, vs, J, k)
            got = Y[k].cpu().numpy().reshape(dims[k], J).T  # column-major J x n_k
            assert rel(got, ref) <= TOL, (k, rel(got, ref))
            # entrywise: the sum of |terms| of each bucket (the sketch of |A| with unit signs)
            # bounds what any FP32 summation order can move it by
            mass = O.sketch_unfolding(np.abs(exact), hs, ones, J, k)
            assert np.all(np.abs(got - ref) <= TOL * (np.abs(ref).max() + mass)), k
    # single-mode call writes only that mode
    Y1 = [None] * len(dims)
    Y1[1] = torch.zeros(J * dims[1], device="cuda")
    ctx.tt_sketch_unfold(Ad, 1, 0, Y1, scales=sd)
    hs, vs = O.draw_sketch(seed, 0, dims, J)
    assert rel(Y1[1].cpu().numpy().reshape(dims[1], J).T, O.sketch_unfolding(exact, hs, vs, J, 1)) <= TOL
    ctx.close()


@pytest.mark.parametrize("n0", [256, 254])
def test_fp8_every_finite_code(n0):
    """Every finite OCP FP8-E4M3 code (all but S.1111.111, the format's NaN) as an entry of the
    data, with unit scales: the data sketches against the oracle's sketch of the decoded tensor
    (synth's decode table: subnormals m 2^-9, normals (1 + m/8) 2^(e-7), up to 448). n_0 = 256
    takes the 16-byte vector kernels (four entries per word), n_0 = 254 window staging."""
    dims, J = (n0, 5, 3), 512
    finite = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], np.uint8)
    rng = np.random.default_rng(n0)
    codes = finite[(np.arange(int(np.prod(dims))) + rng.integers(0, 254)) % finite.size]
    exact = synth.fp8_e4m3_decode(codes).reshape(dims, order="F")
    ctx = lib.Context(dims, (1, 1, 1, 1), J, 1e-3, 31, "fp8")
    Ad = lib.device_tensor(codes, "fp8")
    sd = torch.ones(n0, device="cuda")
    Y = [torch.zeros(J * n, device="cuda") for n in dims]
    ctx.tt_sketch_unfold(Ad, -1, 0, Y, scales=sd)
    hs, vs = O.draw_sketch(31, 0, dims, J)
    for k in range(3):
        ref = O.sketch_unfolding(exact, hs, vs, J, k)
        got = Y[k].cpu().numpy().reshape(dims[k], J).T
        assert rel(got, ref) <= TOL, (k, rel(got, ref))
    ctx.close()


def test_fp8_nan_code_reaches_the_status():
    """Code 0x7F (S.1111.111, E4M3's NaN) decodes as NaN: a sweep over data holding one returns
    TT_ENONFINITE with finite cores (the refused update writes nothing); with the code replaced
    the same context sweeps."""
    dims, ranks, J = (24, 20, 18), (1, 4, 4, 1), 256
    a = synth.random_tensor(dims, 5)
    flat, scales, _ = synth.quantize(a, "fp8")
    bad = flat.copy()
    bad[1000] = 0x7F
    ctx = lib.Context(dims, ranks, J, 1e-3, 9, "fp8")
    sd = torch.tensor(scales, device="cuda")
    init = synth.random_tt(dims, ranks, 6)
    dc = lib.device_cores(init)
    before = [t.clone() for t in dc]
    with pytest.raises(lib.TtError) as e:
        ctx.tt_prox_als_sweep(lib.device_tensor(bad, "fp8"), dc, 1, 0, rel_change=False, scales=sd)
    assert e.value.code == lib.TT_ENONFINITE
    for t in dc:
        assert bool(torch.isfinite(t).all())
    ctx.tt_prox_als_sweep(lib.device_tensor(flat, "fp8"), dc, 1, 0, rel_change=False, scales=sd)
    ctx.close()


@pytest.mark.parametrize("offset", [1, 3, 4])
def test_unfold_sketch_offset_base(offset):
    """A tensor that starts `offset` FP32 entries into its allocation: 4 and 12 bytes off the
    16-byte grid (the narrow-vector path) and 16 bytes (the window staging of 61-entry fibres)."""
    dims, J, storage = (61, 9, 7), 512, "f32"
    seed = 77 + offset
    flat, _, exact = _data(dims, storage, seed)
    ctx = lib.Context(dims, (1, 1, 1, 1), J, 1e-3, seed, storage)
    buf = torch.zeros(flat.size + offset, dtype=torch.float32, device="cuda")
    buf[offset:] = torch.from_numpy(np.ascontiguousarray(flat, dtype=np.float32)).cuda()
    Ad = buf[offset:]
    Y = [torch.zeros(J * n, device="cuda") for n in dims]
    ctx.tt_sketch_unfold(Ad, -1, 0, Y)
    hs, vs = O.draw_sketch(seed, 0, dims, J)
    for k in range(len(dims)):
        ref = O.sketch_unfolding(exact, hs, vs, J, k)
        got = Y[k].cpu().numpy().reshape(dims[k], J).T
        assert rel(got, ref) <= TOL, (k, rel(got, ref))
    ctx.close()


@pytest.mark.parametrize("dims,J,density", [((30, 20, 10), 1024, 0.05), ((12, 10, 8, 6), 150, 0.2),
                                            ((100, 100, 100), 4096, 0.01), ((9, 8, 7, 6, 5), 45, 0.1)])
def test_unfold_coo_parity(dims, J, density):
    """Sparse tensors in coordinate form (with repeated coordinates) against the oracle's dense
    definition on the densified tensor, every mode and one mode alone; an empty list gives zeros."""
    seed = 300 + J
    rng = np.random.default_rng(seed)
    A = synth.random_tensor(dims, seed) * (rng.random(dims) < density)
    A = np.asarray(A, np.float32).astype(np.float64)
    nz = np.nonzero(A)
    idx = np.stack(nz).astype(np.int32)
    vals = A[nz]
    half = idx.shape[1] // 2  # the first half of the entries repeated with their value split
    idx2 = np.concatenate([idx, idx[:, :half]], axis=1)
    vals2 = np.concatenate([np.where(np.arange(vals.size) < half, 0.5 * vals, vals), 0.5 * vals[:half]])
    nnz = idx2.shape[1]
    perm = rng.permutation(nnz)  # arbitrary entry order
    idx_d = torch.from_numpy(np.ascontiguousarray(idx2[:, perm])).cuda()
    val_d = torch.from_numpy(vals2[perm].astype(np.float32)).cuda()
    ranks = (1,) * (len(dims) + 1)
    ctx = lib.Context(dims, ranks, J, 1e-3, seed, "f32")
    Y = [torch.full((J * n,), 7.0, device="cuda") for n in dims]  # overwritten
    ctx.tt_sketch_unfold_coo(idx_d, val_d, nnz, -1, 2, Y)
    hs, vs = O.draw_sketch(seed, 2, dims, J)
    for k in range(len(dims)):
        got = Y[k].cpu().numpy().reshape(dims[k], J).T
        ref = O.sketch_unfolding(A, hs, vs, J, k)
        assert rel(got, ref) <= TOL, (k, rel(got, ref))
    Y1 = [None] * len(dims)
    Y1[1] = torch.zeros(J * dims[1], device="cuda")
    ctx.tt_sketch_unfold_coo(idx_d, val_d, nnz, 1, 2, Y1)
    assert rel(Y1[1].cpu().numpy().reshape(dims[1], J).T, O.sketch_unfolding(A, hs, vs, J, 1)) <= TOL
    Y[0].fill_(3.0)
    ctx.tt_sketch_unfold_coo(None, None, 0, 0, 2, Y)
    assert not Y[0].any()
    ctx.close()


def test_unfold_coo_rejects_bad_coordinates():
    dims = (4, 5, 6)
    ctx = lib.Context(dims, (1, 1, 1, 1), 16, 1e-3, 1, "f32")
    Y = [torch.zeros(16 * n, device="cuda") for n in dims]
    idx = torch.tensor([[0, 3], [1, 5], [2, 0]], dtype=torch.int32, device="cuda")  # i_1 = 5 >= n_1
    val = torch.ones(2, device="cuda")
    with pytest.raises(lib.TtError) as e:
        ctx.tt_sketch_unfold_coo(idx, val, 2, -1, 0, Y)
    assert e.value.code == lib.TT_EINVAL
    # the valid entry was still added, the bad one skipped
    hs, vs = O.draw_sketch(1, 0, dims, 16)
    A = np.zeros(dims)
    A[0, 1, 2] = 1.0
    assert rel(Y[0].cpu().numpy().reshape(dims[0], 16).T, O.sketch_unfolding(A, hs, vs, 16, 0)) <= TOL
    with pytest.raises(lib.TtError):
        ctx.tt_sketch_unfold_coo(idx, val, -1, -1, 0, Y)
    ctx.close()


def test_sparse_sweep_equals_dense_sweep():
    """A sweep on the coordinate-form sketches (tt_sketch_unfold_coo + tt_prox_als_sweep_sketched)
    equals the ordinary sweep on the densified tensor (the same draw)."""
    dims, ranks, J = (20, 18, 16, 14), (1, 4, 5, 4, 1), 512
    rng = np.random.default_rng(5)
    A = np.asarray(synth.random_tensor(dims, 5) * (rng.random(dims) < 0.1), np.float32)
    nz = np.nonzero(A)
    idx_d = torch.from_numpy(np.stack(nz).astype(np.int32)).cuda()
    val_d = torch.from_numpy(A[nz]).cuda()
    init = synth.random_tt(dims, ranks, 6)
    ctx = lib.Context(dims, ranks, J, 1e-3, 77, "f32")
    c_dense, c_sparse = lib.device_cores(init), lib.device_cores(init)
    ctx.tt_prox_als_sweep(lib.device_tensor(A.ravel(order="F"), "f32"), c_dense, 1, 4, rel_change=False)
    Y = [torch.zeros(J * n, device="cuda") for n in dims]
    ctx.tt_sketch_unfold_coo(idx_d, val_d, idx_d.shape[1], -1, 4, Y)
    ctx.tt_prox_als_sweep_sketched(Y, c_sparse, 4)
    a = O.tt_full(lib.host_cores(c_dense, ranks, dims))
    b = O.tt_full(lib.host_cores(c_sparse, ranks, dims))
    assert rel(b, a) <= 1e-4, rel(b, a)
    ctx.close()


def test_unfold_sketch_rejects_bad_calls():
    ctx = lib.Context((4, 5, 6), (1, 1, 1, 1), 16, 1e-3, 1, "f32")
    A = torch.zeros(120, device="cuda")
    Y = [torch.zeros(16 * n, device="cuda") for n in (4, 5, 6)]
    with pytest.raises(lib.TtError) as e:
        ctx.tt_sketch_unfold(A, 3, 0, Y)
    assert e.value.code == lib.TT_EINVAL
    with pytest.raises(lib.TtError) as e:
        ctx.tt_sketch_unfold(A, 0, 0, Y, scales=torch.ones(4, device="cuda"))
    assert e.value.code == lib.TT_EINVAL
    ctx.close()


# ---------------------------------------------------------------------------------------------
# a2-a4: interface sketch S H_k

CASES_B = [((6, 5, 7), (1, 2, 3, 1), 32), ((4, 3, 5, 6), (1, 3, 4, 2, 1), 64), ((9, 8), (1, 4, 1), 16),
           ((20, 30, 25, 10), (1, 4, 5, 3, 1), 256), ((50, 50, 50), (1, 5, 5, 1), 1024),
           ((10, 12, 3, 9), (1, 8, 3, 8, 1), 2048), ((7, 7, 7, 7, 7), (1, 3, 3, 3, 3, 1), 4096),
           ((5, 6, 4), (1, 2, 2, 1), 2), ((30, 20, 10), (1, 12, 10, 1), 16384),
           # sketch sizes that are not powers of two: direct DFTs
           ((6, 5, 7), (1, 2, 3, 1), 45), ((10, 12, 3, 9), (1, 8, 3, 8, 1), 2000),
           ((20, 30, 25, 10), (1, 4, 5, 3, 1), 150), ((9, 8), (1, 4, 1), 3), ((50, 50, 50), (1, 5, 5, 1), 1000),
           ((10,) * 6, (1, 5, 5, 5, 5, 5, 1), 200)]


@pytest.mark.parametrize("dims,ranks,J", CASES_B)
def test_interface_sketch_parity(dims, ranks, J):
    seed = 77 + J
    cores = synth.random_tt(dims, ranks, seed)
    ctx = lib.Context(dims, ranks, J, 1e-3, seed, "f32")
    dc = lib.device_cores(cores)
    c32 = [np.asarray(g, np.float32).astype(np.float64) for g in cores]
    for sweep in (0, 2):
        hs, vs = O.draw_sketch(seed, sweep, dims, J)
        for k in range(len(dims)):
            s = ranks[k] * ranks[k + 1]
            SH = torch.zeros(J * s, device="cuda")
            ctx.tt_sketch_interface(dc, k, sweep, SH)
            torch.cuda.synchronize()
            got = SH.cpu().numpy().reshape(s, J).T
            ref = O.sketch_interface_fft(c32, hs, vs, J, k)
            assert rel(got, ref) <= TOL, (k, rel(got, ref))
            # entrywise, column by column (columns of S H_k differ in scale)
            colmax = np.abs(ref).max(axis=0, keepdims=True)
            assert np.all(np.abs(got - ref) <= TOL * colmax + 1e-30), (k, np.max(np.abs(got - ref) / colmax))
    ctx.close()


# ---------------------------------------------------------------------------------------------
# a5-a6: proximal update

@pytest.mark.parametrize("J,n,r0,r1,sigma", [(256, 7, 3, 4, 1e-3), (4096, 100, 10, 10, 1e-3), (2048, 256, 1, 20, 0.5),
                                             (1024, 50, 5, 5, 0.0), (8192, 40, 8, 8, 1e-3), (512, 128, 12, 12, 1e-3),
                                             (64, 3, 1, 1, 2.0), (45, 7, 3, 4, 1e-3), (1000, 100, 10, 10, 1e-3),
                                             (150, 10, 5, 5, 1e-3),
                                             # s > 160: the one-CTA Cholesky solve
                                             (2048, 10, 20, 20, 0.5), (1024, 30, 12, 16, 1e-3), (4096, 50, 16, 30, 1e-3)])
def test_prox_update_parity(J, n, r0, r1, sigma):
    rng = np.random.default_rng(J + n)
    s = r0 * r1
    # well-conditioned sketched interface: orthonormal columns scaled to a near-isometry
    SH = np.linalg.qr(rng.standard_normal((J, s)))[0] * (1.0 + 0.1 * rng.standard_normal(s))
    Y = rng.standard_normal((J, n))
    G = rng.standard_normal((r0, n, r1))
    SH32, Y32, G32 = (x.astype(np.float32) for x in (SH, Y, G))
    dims = (n, 4, 3) if r0 == 1 else (5, n, 3)
    k = 0 if r0 == 1 else 1
    ranks = (1, r1, 1, 1) if k == 0 else (1, r0, r1, 1)
    ctx = lib.Context(dims, ranks, J, sigma, 5, "f32")
    Yd = torch.from_numpy(np.ascontiguousarray(Y32.T)).cuda()  # J x n column-major
    SHd = torch.from_numpy(np.ascontiguousarray(SH32.T)).cuda()  # column-major J x s
    core = torch.from_numpy(np.ascontiguousarray(G32.ravel(order="F"))).cuda()
    ctx.tt_prox_update(Yd, SHd, core, k)
    got = core.cpu().numpy().astype(np.float64).reshape(r0, n, r1, order="F")
    ref = O.prox_update(Y32.astype(np.float64), SH32.astype(np.float64), G32.astype(np.float64), sigma)
    assert rel(got, ref) <= TOL, rel(got, ref)
    ctx.close()


@pytest.mark.parametrize("dims,ranks,k", [((6, 4, 3), (1, 2, 2, 1), 0), ((5, 10, 3), (1, 20, 20, 1), 1)])
def test_prox_update_not_spd_leaves_core(dims, ranks, k):
    """sigma = 0 and a zero sketched interface: the register solve (s = 2) and the Cholesky solve
    (s = 400) both refuse the singular Gram and leave the core as it was."""
    J = 512
    ctx = lib.Context(dims, ranks, J, 0.0, 5, "f32")
    s, n = ranks[k] * ranks[k + 1], dims[k]
    Yd = torch.randn(J, n, device="cuda")
    SHd = torch.zeros(J * s, device="cuda")
    core = torch.randn(s * n, device="cuda")
    before = core.clone()
    with pytest.raises(lib.TtError) as e:
        ctx.tt_prox_update(Yd, SHd, core, k)
    assert e.value.code == lib.TT_ENOTSPD
    assert torch.equal(core, before)
    ctx.close()


# ---------------------------------------------------------------------------------------------
# a7-a8: orthogonalisation

@pytest.mark.parametrize("dims,ranks", [((6, 7, 5, 4), (1, 3, 4, 2, 1)), ((256, 256, 3, 128), (1, 20, 3, 20, 1)),
                                        ((10, 12, 3, 9), (1, 8, 3, 8, 1)), ((40, 40, 40), (1, 8, 8, 1)),
                                        ((30, 24, 20, 16), (1, 10, 12, 10, 1)), ((32, 20, 18), (1, 16, 9, 1))])
def test_orthogonalization_parity(dims, ranks):
    cores = synth.random_tt(dims, ranks, 31)
    c32 = [np.asarray(g, np.float32).astype(np.float64) for g in cores]
    ctx = lib.Context(dims, ranks, 64, 1e-3, 5, "f32")
    dc = lib.device_cores(cores)
    ctx.tt_orthogonalize(dc, -1)
    got = lib.host_cores(dc, ranks, dims)
    ref = O.orthogonalize_right_to_left(c32)
    for k in range(len(dims)):
        assert rel(got[k], ref[k]) <= 1e-4, (k, rel(got[k], ref[k]))
    for k in range(len(dims) - 1):
        ctx.tt_orthogonalize(dc, +1, k)
        O.left_orthogonalize_step(ref, k)
        got = lib.host_cores(dc, ranks, dims)
        assert rel(got[k], ref[k]) <= 1e-4, (k, rel(got[k], ref[k]))
        assert rel(got[k + 1], ref[k + 1]) <= 1e-4
    assert rel(O.tt_full(got), O.tt_full(c32)) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("case", ["rank_deficient", "wide"])
def test_orthogonalization_fallback(case):
    """CholeskyQR2 gives way to Householder when G_k^L is rank deficient (a repeated column) or
    wider than tall; either way [[G]] is unchanged and G_k^L gets orthonormal columns (zero
    columns past its row count in the wide case)."""
    if case == "rank_deficient":
        dims, ranks = (9, 7, 6), (1, 5, 6, 1)
    else:
        dims, ranks = (2, 3, 6), (1, 2, 8, 1)
    cores = synth.random_tt(dims, ranks, 41)
    if case == "rank_deficient":
        cores[1][:, :, 4] = cores[1][:, :, 1]
    c32 = [np.asarray(g, np.float32).astype(np.float64) for g in cores]
    ctx = lib.Context(dims, ranks, 64, 1e-3, 5, "f32")
    dc = lib.device_cores(cores)
    ctx.tt_orthogonalize(dc, +1, 1)
    got = lib.host_cores(dc, ranks, dims)
    assert rel(O.tt_full(got), O.tt_full(c32)) <= 1e-5
    m, q = ranks[1] * dims[1], ranks[2]
    GL = got[1].reshape(m, q, order="F")
    p = min(m, q)
    assert np.allclose(GL[:, :p].T @ GL[:, :p], np.eye(p), atol=1e-5)
    assert np.all(GL[:, p:] == 0)
    ctx.close()


# ---------------------------------------------------------------------------------------------
# a9: relative error

@pytest.mark.parametrize("dims,ranks,storage", [((20, 18, 16), (1, 4, 5, 1), "f32"), ((9, 8, 7, 6), (1, 3, 4, 2, 1), "f64"),
                                                ((33, 17, 9, 5), (1, 3, 3, 3, 1), "bf16"), ((40, 12, 10, 6), (1, 2, 3, 2, 1), "fp8"),
                                                ((64, 48), (1, 7, 1), "f32"), ((12, 5, 4, 3, 3), (1, 3, 4, 3, 2, 1), "f32"),
                                                ((8, 6, 10, 40), (1, 2, 4, 36, 1), "f32")])
def test_rel_error_parity(dims, ranks, storage):
    true = synth.random_tt(dims, ranks, 3)
    a = synth.add_noise(synth.contract_cores(true), 0.05, np.random.default_rng(4))
    flat, scales, exact = synth.quantize(a, storage)
    est = synth.random_tt(dims, ranks, 5)
    c32 = [np.asarray(g, np.float32).astype(np.float64) for g in est]
    ctx = lib.Context(dims, ranks, 64, 1e-3, 5, storage)
    sd = torch.tensor(scales, device="cuda") if scales is not None else None
    e = ctx.tt_rel_error(lib.device_tensor(flat, storage), lib.device_cores(est), scales=sd)
    ref = O.rel_error(exact, c32)
    assert abs(e - ref) <= 1e-5 * ref, (e, ref)
    ctx.close()


@pytest.mark.parametrize("dims,ranks,density", [((12, 10, 8, 6), (1, 3, 4, 2, 1), 0.1), ((20, 18, 16), (1, 12, 20, 1), 0.05),
                                                ((9, 8, 7, 6, 5), (1, 4, 5, 6, 3, 1), 0.2), ((40, 30), (1, 32, 1), 0.3)])
def test_rel_error_coo_parity(dims, ranks, density):
    """The sparse relative error (coordinate form, distinct coordinates in shuffled order) against
    the oracle's relative error of the densified tensor. Every term is FP64 on FP32 inputs:
    bound 1e-8."""
    rng = np.random.default_rng(sum(dims))
    A = np.asarray(synth.random_tensor(dims, 4) * (rng.random(dims) < density), np.float32).astype(np.float64)
    est = synth.random_tt(dims, ranks, 5)
    c32 = [np.asarray(g, np.float32).astype(np.float64) for g in est]
    nz = np.nonzero(A)
    idx = np.stack(nz).astype(np.int32)
    vals = A[nz]
    perm = rng.permutation(vals.size)
    idx2, vals2 = np.ascontiguousarray(idx[:, perm]), vals[perm]
    ctx = lib.Context(dims, ranks, 64, 1e-3, 5, "f32")
    e = ctx.tt_rel_error_coo(torch.from_numpy(idx2).cuda(), torch.from_numpy(vals2.astype(np.float32)).cuda(),
                             idx2.shape[1], lib.device_cores(est))
    ref = O.rel_error(A, c32)
    assert abs(e - ref) <= 1e-8 * ref, (e, ref)
    ctx.close()


def test_rel_error_coo_small_residual():
    """Every entry listed, A = X + 1e-4 relative noise: the expanded form cancels about eight
    digits, which FP64 keeps (1e-6 against the oracle); the dense call agrees to 1e-5."""
    dims, ranks = (16, 14, 12, 10), (1, 4, 5, 3, 1)
    est = synth.random_tt(dims, ranks, 8)
    c32 = [np.asarray(g, np.float32).astype(np.float64) for g in est]
    X = O.tt_full(c32)
    A = np.asarray(X + 1e-4 * np.linalg.norm(X) / np.sqrt(X.size) * np.random.default_rng(9).standard_normal(X.shape),
                   np.float32).astype(np.float64)
    idx = np.stack(np.unravel_index(np.arange(A.size), dims, order="F")).astype(np.int32)
    vals = A.ravel(order="F")
    ctx = lib.Context(dims, ranks, 64, 1e-3, 5, "f32")
    dc = lib.device_cores(est)
    e = ctx.tt_rel_error_coo(torch.from_numpy(idx).cuda(), torch.from_numpy(vals.astype(np.float32)).cuda(), A.size, dc)
    ref = O.rel_error(A, c32)
    assert abs(e - ref) <= 1e-6 * ref, (e, ref)
    e_dense = ctx.tt_rel_error(lib.device_tensor(vals.astype(np.float32), "f32"), dc)
    assert abs(e_dense - ref) <= 1e-5 * ref, (e_dense, ref)
    ctx.close()


def test_rel_error_coo_rejects():
    ctx = lib.Context((5, 40, 3), (1, 5, 40, 1), 64, 1e-3, 5, "f32")  # a rank above 32
    est = synth.random_tt((5, 40, 3), (1, 5, 40, 1), 1)
    idx = torch.zeros(3, 1, dtype=torch.int32, device="cuda")
    val = torch.ones(1, device="cuda")
    with pytest.raises(lib.TtError) as e:
        ctx.tt_rel_error_coo(idx, val, 1, lib.device_cores(est))
    assert e.value.code == lib.TT_EINVAL
    ctx.close()
    ctx = lib.Context((5, 4, 3), (1, 2, 2, 1), 64, 1e-3, 5, "f32")
    est = synth.random_tt((5, 4, 3), (1, 2, 2, 1), 1)
    idx = torch.tensor([[0], [4], [0]], dtype=torch.int32, device="cuda")  # i_1 = 4 >= n_1
    with pytest.raises(lib.TtError) as e:
        ctx.tt_rel_error_coo(idx, val, 1, lib.device_cores(est))
    assert e.value.code == lib.TT_EINVAL
    ctx.close()


# ---------------------------------------------------------------------------------------------
# whole sweeps (Algorithm 1)

def _run_sweeps(w, storage, nsweeps):
    p = synth.make_problem(w, storage=storage)
    ctx = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, storage)
    A = lib.device_tensor(p.storage, storage)
    sd = torch.tensor(p.scales, device="cuda") if p.scales is not None else None
    dc = lib.device_cores(p.init_cores)
    changes = ctx.tt_prox_als_sweep(A, dc, nsweeps, 0, scales=sd)
    err = ctx.tt_rel_error(A, dc, scales=sd)
    got = lib.host_cores(dc, p.ranks, w.dims)
    ref, ref_changes = O.tt_ts(p.tensor, p.init_cores, p.sketch_seed, w.J, w.lam, nsweeps)
    ctx.close()
    return p, got, err, changes, ref, ref_changes


def test_sweeps_order3_50_r5_parity():
    """The order-3 50^3 workload (ranks (1,5,5,1), J=1024, lambda=1e-3, 10 sweeps)."""
    w = synth.WORKLOADS["order3-50-r5"]
    p, got, err, changes, ref, ref_changes = _run_sweeps(w, "f64", w.sweeps)
    err_ref = O.rel_error(p.tensor, ref)
    assert abs(err - err_ref) <= 1e-5 * err_ref, (err, err_ref)
    assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4
    assert abs(changes[-1] - ref_changes[-1]) <= 1e-3 * max(ref_changes[-1], 1e-9) + 1e-7


def test_sweeps_scaled_order4_parity():
    w = synth.WORKLOADS["order4-100-r10"].scaled((24, 20, 18, 16), J=512)
    p, got, err, changes, ref, ref_changes = _run_sweeps(w, "f32", 4)
    err_ref = O.rel_error(p.tensor, ref)
    assert abs(err - err_ref) <= 1e-5 * err_ref, (err, err_ref)


@pytest.mark.parametrize("dims,ranks,J,nsw", [((10,) * 6, (1, 5, 5, 5, 5, 5, 1), 45, 1),
                                              ((10,) * 6, (1, 5, 5, 5, 5, 5, 1), 150, 1),
                                              ((30, 28, 26), (1, 4, 4, 1), 200, 3), ((12, 10, 8), (1, 3, 3, 1), 1000, 3)])
def test_sweeps_non_power_of_two_sketch_sizes(dims, ranks, J, nsw):
    """Whole sweeps at sketch sizes that are not powers of two, among them the shape of the
    paper's first synthetic experiment (order 6, n = 10, ranks 5, m = 45 and 150; Sec. 5). With
    25 unknowns per core and 45 or 150 sketch rows the iteration is far from converged and
    amplifies rounding: the FP64 oracle itself moves its result after one sweep by 69x (m = 45)
    and 12x (m = 150) a 1e-7 relative perturbation of the initial cores, and after three sweeps
    by 2.3e5x and 650x. So the order-6 cases take one sweep, and the bound on the reconstructed
    tensor is 1e-4 plus the oracle's own change under two perturbations of the size of the GPU's
    FP32 rounding: the initial cores by 1e-6 (about ten FP32 ulps), and every entry of the data by
    eps = 2^-24 log2(N / J) relative: a data-sketch bucket sums about N / J terms as a tree (runs
    of equal hash in registers, then the runs' sums by atomic adds), whose error is about log2 of
    the term count in roundings of the bucket's size (8.6e-7 for N = 10^6, J = 45); the relative
    error of the GPU's cores keeps 1e-5."""
    cores = synth.random_tt(dims, ranks, 3)
    a = synth.add_noise(synth.contract_cores(cores), 1e-2, np.random.default_rng(8))
    flat, _, exact = synth.quantize(a, "f32")
    init = synth.random_tt(dims, ranks, 9)
    ctx = lib.Context(dims, ranks, J, 1e-3, 31, "f32")
    A = lib.device_tensor(flat, "f32")
    dc = lib.device_cores(init)
    ctx.tt_prox_als_sweep(A, dc, nsw, 0, rel_change=False)
    err = ctx.tt_rel_error(A, dc)
    got = lib.host_cores(dc, ranks, dims)
    ctx.close()
    ref, _ = O.tt_ts(exact, init, 31, J, 1e-3, nsw)
    xi = np.random.default_rng(1)
    pert = [g * (1.0 + 1e-6 * xi.standard_normal(g.shape)) for g in init]
    ref_p, _ = O.tt_ts(exact, pert, 31, J, 1e-3, nsw)
    eps = 2.0 ** -24 * np.log2(max(2.0, exact.size / J))
    ref_d, _ = O.tt_ts(exact * (1.0 + eps * xi.standard_normal(exact.shape)), init, 31, J, 1e-3, nsw)
    full_ref = O.tt_full(ref)
    tol = 1e-4 + rel(O.tt_full(ref_p), full_ref) + rel(O.tt_full(ref_d), full_ref)
    assert rel(O.tt_full(got), full_ref) <= tol, (rel(O.tt_full(got), full_ref), tol)
    e_ref = O.rel_error(exact, [np.asarray(g, np.float32).astype(np.float64) for g in got])
    assert abs(err - e_ref) <= 1e-5 * e_ref, (err, e_ref)


@pytest.mark.parametrize("dims,ranks,J", [
    ((3, 4, 2, 3, 2, 3, 2, 4), (1, 2, 2, 2, 2, 2, 2, 2, 1), 64),  # order 8, the largest
    ((50, 40), (1, 6, 1), 128),                                  # order 2, the smallest
    ((40000, 3, 2), (1, 1, 1, 1), 256),  # the largest mode size a core allows (r n r' <= 40000), first
    ((3, 40000, 2), (1, 1, 1, 1), 256),  # ... and inner (40,000 output columns; 12-byte fibres)
])
def test_extreme_shapes(dims, ranks, J):
    """The limits of the context: every mode's data sketch against the oracle (1e-5), then two
    sweeps against the oracle's (reconstruction 1e-4) and the relative error of the GPU's cores
    (1e-5)."""
    seed = 60 + len(dims) + J
    cores = synth.random_tt(dims, ranks, seed)
    a = synth.add_noise(synth.contract_cores(cores), 1e-2, np.random.default_rng(seed + 1))
    flat, _, exact = synth.quantize(a, "f32")
    ctx = lib.Context(dims, ranks, J, 1e-3, seed, "f32")
    A = lib.device_tensor(flat, "f32")
    Y = [torch.zeros(J * n, device="cuda") for n in dims]
    ctx.tt_sketch_unfold(A, -1, 0, Y)
    hs, vs = O.draw_sketch(seed, 0, dims, J)
    for k in range(len(dims)):
        ref = O.sketch_unfolding(exact, hs, vs, J, k)
        got = Y[k].cpu().numpy().reshape(dims[k], J).T
        assert rel(got, ref) <= TOL, (k, rel(got, ref))
    init = synth.random_tt(dims, ranks, seed + 2)
    dc = lib.device_cores(init)
    ctx.tt_prox_als_sweep(A, dc, 2, 0, rel_change=False)
    err = ctx.tt_rel_error(A, dc)
    got = lib.host_cores(dc, ranks, dims)
    ctx.close()
    ref, _ = O.tt_ts(exact, init, seed, J, 1e-3, 2)
    assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4, rel(O.tt_full(got), O.tt_full(ref))
    e_ref = O.rel_error(exact, [np.asarray(g, np.float32).astype(np.float64) for g in got])
    assert abs(err - e_ref) <= 1e-5 * e_ref, (err, e_ref)


def test_fixed_sketch_reuses_the_data_sketches_within_a_call():
    """With TT_FLAG_FIXED_SKETCH every sweep uses sweep 0's draw, so the data sketches depend on A
    alone: a call's first sweep computes them (d launches) and its later sweeps reuse them. Four
    sweeps against the oracle's four sweeps with sweep 0's draw (reconstruction 1e-4, relative
    error 1e-5); the launch count shows the reuse; a second call on other data recomputes them
    (a stale reuse would give the first tensor's sweeps)."""
    dims, ranks, J, lam, seed = (24, 20, 18, 16), (1, 4, 5, 4, 1), 512, 1e-3, 57
    probs = []
    for s0 in (1, 2):
        cores = synth.random_tt(dims, ranks, 10 * s0)
        a = synth.add_noise(synth.contract_cores(cores), 1e-2, np.random.default_rng(10 * s0 + 1))
        flat, _, exact = synth.quantize(a, "f32")
        probs.append((lib.device_tensor(flat, "f32"), exact))
    init = synth.random_tt(dims, ranks, 33)
    ctx = lib.Context(dims, ranks, J, lam, seed, "f32", flags=lib.TT_FLAG_FIXED_SKETCH)
    dc = lib.device_cores(init)
    ctx.tt_profile_enable(True)
    ctx.tt_prox_als_sweep(probs[0][0], dc, 4, 7, rel_change=False)
    launches = ctx.tt_profile_read()["unfold_launches"]
    ctx.tt_profile_enable(False)
    assert launches == len(dims), launches
    ref = [np.asarray(g, np.float64) for g in init]
    for _ in range(4):
        ref, _ = O.tt_ts_sweep(probs[0][1], ref, seed, 0, J, lam)
    got = lib.host_cores(dc, ranks, dims)
    assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4, rel(O.tt_full(got), O.tt_full(ref))
    err = ctx.tt_rel_error(probs[0][0], dc)
    e_ref = O.rel_error(probs[0][1], [np.asarray(g, np.float32).astype(np.float64) for g in got])
    assert abs(err - e_ref) <= 1e-5 * e_ref, (err, e_ref)
    ctx.tt_prox_als_sweep(probs[1][0], dc, 2, 0, rel_change=False)  # the second tensor
    for _ in range(2):
        ref, _ = O.tt_ts_sweep(probs[1][1], ref, seed, 0, J, lam)
    got = lib.host_cores(dc, ranks, dims)
    ctx.close()
    assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4, rel(O.tt_full(got), O.tt_full(ref))


def test_sweeps_with_large_cores():
    """Cores with r_k r_{k+1} = 180 > 160 unknowns (the Cholesky solve) in whole sweeps: the
    tensor after two sweeps against the oracle's (1e-4) and its relative error (1e-5)."""
    dims, ranks, J = (6, 8, 8, 6), (1, 6, 30, 6, 1), 1024
    cores = synth.random_tt(dims, ranks, 21)
    a = synth.add_noise(synth.contract_cores(cores), 1e-2, np.random.default_rng(22))
    flat, _, exact = synth.quantize(a, "f32")
    init = synth.random_tt(dims, ranks, 23)
    ctx = lib.Context(dims, ranks, J, 1e-3, 41, "f32")
    A = lib.device_tensor(flat, "f32")
    dc = lib.device_cores(init)
    ctx.tt_prox_als_sweep(A, dc, 2, 0, rel_change=False)
    err = ctx.tt_rel_error(A, dc)
    got = lib.host_cores(dc, ranks, dims)
    ctx.close()
    ref, _ = O.tt_ts(exact, init, 41, J, 1e-3, 2)
    assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4, rel(O.tt_full(got), O.tt_full(ref))
    e_ref = O.rel_error(exact, [np.asarray(g, np.float32).astype(np.float64) for g in got])
    assert abs(err - e_ref) <= 1e-5 * e_ref, (err, e_ref)


def test_monitored_sweeps_match_separate_calls():
    """tt_prox_als_sweep_monitored = per sweep, tt_prox_als_sweep then tt_rel_error. Two contexts
    with the same draws differ only by FP32 summation order in the data-sketch atomics, which
    unconverged sweeps amplify to ~1e-5: the bound is 1e-4."""
    w = synth.WORKLOADS["order4-100-r10"].scaled((24, 20, 18, 16), J=512)
    p = synth.make_problem(w, storage="f32")
    A = lib.device_tensor(p.storage, "f32")
    ctx_a = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, "f32")
    ctx_b = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, "f32")
    ca, cb = lib.device_cores(p.init_cores), lib.device_cores(p.init_cores)
    errs, changes = ctx_a.tt_prox_als_sweep_monitored(A, ca, 3, 0, rel_change=True)
    for t in range(3):
        ch = ctx_b.tt_prox_als_sweep(A, cb, 1, t)[0]
        e = ctx_b.tt_rel_error(A, cb)
        assert abs(errs[t] - e) <= 1e-4 * e, (t, errs[t], e)
        assert abs(changes[t] - ch) <= 1e-4 * ch, (t, changes[t], ch)
    ga, gb = lib.host_cores(ca, p.ranks, w.dims), lib.host_cores(cb, p.ranks, w.dims)
    assert rel(O.tt_full(ga), O.tt_full(gb)) <= 1e-4
    rc = ctx_a.lib.tt_prox_als_sweep_monitored(ctx_a.ctx, lib._ptr(A), None, lib._ptr_array(ca), 1, 0, None, None)
    assert rc == lib.TT_EINVAL  # the per-sweep errors are the point of the call
    ctx_a.close()
    ctx_b.close()


def test_sweeps_with_jumps_in_the_sweep_index():
    """Each sweep builds the next sweep index's draw and plans ahead; a call with another index
    (a jump, a step back, a repeat) must draw its own, and the data-sketch entry point must see
    the draw of the index it is given, whichever of the two buffers holds it."""
    w = synth.WORKLOADS["order3-50-r5"]
    p = synth.make_problem(w, storage="f32")
    ctx = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, "f32")
    A = lib.device_tensor(p.storage, "f32")
    dc = lib.device_cores(p.init_cores)
    ref = [np.array(g, np.float64) for g in p.init_cores]
    for first in (0, 5, 1, 2, 2):  # a jump ahead, a step back, the spare's index, a repeat
        ctx.tt_prox_als_sweep(A, dc, 1, first, rel_change=False)
        ref, _ = O.tt_ts(p.tensor, ref, p.sketch_seed, w.J, w.lam, 1, first_sweep=first)
    got = lib.host_cores(dc, p.ranks, w.dims)
    assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4
    Y = [torch.zeros(w.J * n, device="cuda") for n in w.dims]
    for sweep in (3, 2, 3):  # the spare built by the last sweep, the current draw, the spare again
        ctx.tt_sketch_unfold(A, -1, sweep, Y)
        torch.cuda.synchronize()
        hs, vs = O.draw_sketch(p.sketch_seed, sweep, w.dims, w.J)
        for k in range(len(w.dims)):
            refk = O.sketch_unfolding(p.tensor, hs, vs, w.J, k)
            gotk = Y[k].cpu().numpy().reshape(w.dims[k], w.J).T
            assert rel(gotk, refk) <= 1e-5, (sweep, k, rel(gotk, refk))
    ctx.close()


def test_sweep_exact_tt_recovery_on_gpu():
    dims, ranks = (12, 10, 11, 9), (1, 3, 3, 3, 1)
    A = synth.contract_cores(synth.random_tt(dims, ranks, 15))
    init = synth.random_tt(dims, ranks, 16)
    ctx = lib.Context(dims, ranks, 256, 1e-3, 31, "f32")
    Ad = lib.device_tensor(A.ravel(order="F"), "f32")
    dc = lib.device_cores(init)
    ctx.tt_prox_als_sweep(Ad, dc, 30, 0)
    assert ctx.tt_rel_error(Ad, dc) < 1e-5
    ctx.close()
