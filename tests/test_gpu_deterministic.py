"""The deterministic mode (TT_FLAG_DETERMINISTIC): fixed summation orders, so that repeated runs
of the same seeded call give the same bits, and the same parity with the CPU FP64 oracle as the
fast path. Its data sketch Y_k = S A_(k)^T (Alg. 1, Eqs. (eqn_h), (eqn_v)) sums each run of fibres
with equal hash in index order over work spans fixed by the shape and adds the run sums in 64-bit
fixed point; the Gram's K-chunks, the relative error and the change norms are summed in fixed
orders, and the CountSketch of the cores adds its entries in index order.

Checks: the data sketch against the oracle in every storage type (relative Frobenius and
entrywise, as for the fast path), bit-identical on a second call and for the tensor placed off
the 16-byte grid; the interface sketch against the oracle; a multi-sweep call against single-sweep
calls and a call on a rescaled tensor; whole sweeps run twice on two contexts (FP32 update and
sigma = 0 FP64 update, the latter on the paper's sinc tensor for 30 sweeps) agree bit for bit in
cores, relative errors and rel-changes, and with the oracle."""
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

DET = lib.TT_FLAG_DETERMINISTIC
TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("dims,J,storage", [((24, 20, 18, 16), 512, "f32"), ((30, 7, 11), 4096, "bf16"),
                                            ((12, 10, 8, 6, 4), 1000, "fp8"), ((12, 10, 8), 45, "f64"),
                                            ((100, 50, 40), 4096, "f32"), ((10,) * 6, 150, "f32")])
def test_det_data_sketch_matches_oracle_and_repeats_bit_for_bit(dims, J, storage):
    seed = 3000 + sum(dims) + J
    a = synth.random_tensor(dims, seed)
    flat, scales, exact = synth.quantize(a, storage)
    ctx = lib.Context(dims, (1,) * (len(dims) + 1), J, 1e-3, seed, storage, flags=DET)
    Ad = lib.device_tensor(flat, storage)
    sd = torch.tensor(scales, device="cuda") if scales is not None else None
    Y = [torch.zeros(J * n, device="cuda") for n in dims]
    Y2 = [torch.zeros(J * n, device="cuda") for n in dims]
    ctx.tt_sketch_unfold(Ad, -1, 2, Y, scales=sd)
    ctx.tt_sketch_unfold(Ad, -1, 2, Y2, scales=sd)
    torch.cuda.synchronize()
    hs, vs = O.draw_sketch(seed, 2, dims, J)
    ones = [np.ones_like(v) for v in vs]
    for k in range(len(dims)):
        assert torch.equal(Y[k], Y2[k]), k
        got = Y[k].cpu().numpy().reshape(dims[k], J).T
        ref = O.sketch_unfolding(exact, hs, vs, J, k)
        assert rel(got, ref) <= TOL, (k, rel(got, ref))
        mass = O.sketch_unfolding(np.abs(exact), hs, ones, J, k)
        assert np.all(np.abs(got - ref) <= TOL * (np.abs(ref).max() + mass)), k
    # one mode alone: the same bits as in the all-mode call
    Y1 = [None] * len(dims)
    Y1[1] = torch.zeros(J * dims[1], device="cuda")
    ctx.tt_sketch_unfold(Ad, 1, 2, Y1, scales=sd)
    torch.cuda.synchronize()
    assert torch.equal(Y1[1], Y[1])
    ctx.close()


@pytest.mark.parametrize("storage,offsets", [("f32", (1, 2, 3)), ("bf16", (1, 2, 4))])
def test_det_data_sketch_bits_do_not_depend_on_alignment(storage, offsets):
    """The same tensor starting 16-byte aligned and `offset` entries into its allocation: the
    kernels then load 4-, 8- or 2-byte vectors with fewer fibre slots per warp, but the work spans
    are fixed by the shape, so every mode's sketch has the same bits."""
    dims, J = (64, 9, 7), 512
    seed = 4100 + len(storage)
    a = synth.random_tensor(dims, seed)
    flat, _, exact = synth.quantize(a, storage)
    ctx = lib.Context(dims, (1,) * (len(dims) + 1), J, 1e-3, seed, storage, flags=DET)
    base = lib.device_tensor(flat, storage)
    Y0 = [torch.zeros(J * n, device="cuda") for n in dims]
    ctx.tt_sketch_unfold(base, -1, 0, Y0)
    hs, vs = O.draw_sketch(seed, 0, dims, J)
    for k in range(len(dims)):
        ref = O.sketch_unfolding(exact, hs, vs, J, k)
        assert rel(Y0[k].cpu().numpy().reshape(dims[k], J).T, ref) <= TOL, k
    for off in offsets:
        buf = torch.zeros(base.numel() + off, dtype=base.dtype, device="cuda")
        buf[off:] = base
        Y = [torch.zeros(J * n, device="cuda") for n in dims]
        ctx.tt_sketch_unfold(buf[off:], -1, 0, Y)
        torch.cuda.synchronize()
        for k in range(len(dims)):
            assert torch.equal(Y[k], Y0[k]), (off, k)
    ctx.close()


@pytest.mark.parametrize("dims,ranks,J", [((30, 20, 10), (1, 12, 10, 1), 1024), ((6, 5, 7), (1, 2, 3, 1), 45),
                                          ((20, 30, 25, 10), (1, 4, 5, 3, 1), 16384)])
def test_det_interface_sketch_matches_oracle(dims, ranks, J):
    seed = 91 + J
    cores = synth.random_tt(dims, ranks, seed)
    c32 = [np.asarray(g, np.float32).astype(np.float64) for g in cores]
    ctx = lib.Context(dims, ranks, J, 1e-3, seed, "f32", flags=DET)
    dc = lib.device_cores(cores)
    hs, vs = O.draw_sketch(seed, 1, dims, J)
    for k in range(len(dims)):
        s = ranks[k] * ranks[k + 1]
        SH = torch.zeros(J * s, device="cuda")
        SH2 = torch.zeros(J * s, device="cuda")
        ctx.tt_sketch_interface(dc, k, 1, SH)
        ctx.tt_sketch_interface(dc, k, 1, SH2)
        torch.cuda.synchronize()
        assert torch.equal(SH, SH2)
        got = SH.cpu().numpy().reshape(s, J).T
        assert rel(got, O.sketch_interface_fft(c32, hs, vs, J, k)) <= TOL
    ctx.close()


def _two_runs(dims, ranks, J, sigma, A_flat, init, nsweeps, seed):
    out = []
    for _ in range(2):
        ctx = lib.Context(dims, ranks, J, sigma, seed, "f32", flags=DET)
        Ad = lib.device_tensor(A_flat, "f32")
        dc = lib.device_cores(init)
        errs, changes = ctx.tt_prox_als_sweep_monitored(Ad, dc, nsweeps, 0, rel_change=True)
        out.append(([g.clone() for g in dc], list(errs), list(changes)))
        ctx.close()
    return out


def test_det_sweeps_repeat_bit_for_bit_and_match_the_oracle():
    dims, ranks, J, sigma, seed = (24, 20, 18, 16), (1, 4, 5, 4, 1), 512, 1e-3, 77
    cores = synth.random_tt(dims, ranks, 5)
    a = synth.add_noise(synth.contract_cores(cores), 1e-2, np.random.default_rng(6))
    flat, _, exact = synth.quantize(a, "f32")
    init = synth.random_tt(dims, ranks, 7)
    (c1, e1, ch1), (c2, e2, ch2) = _two_runs(dims, ranks, J, sigma, flat, init, 4, seed)
    assert all(torch.equal(x, y) for x, y in zip(c1, c2))
    assert e1 == e2 and ch1 == ch2
    ref, ref_ch = O.tt_ts(exact, init, seed, J, sigma, 4)
    got = [t.cpu().numpy().astype(np.float64).reshape(ranks[k], dims[k], ranks[k + 1], order="F")
           for k, t in enumerate(c1)]
    assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4
    e_ref = O.rel_error(exact, got)
    assert abs(e1[-1] - e_ref) <= 1e-5 * e_ref, (e1[-1], e_ref)
    assert abs(ch1[-1] - ref_ch[-1]) <= 1e-3 * ref_ch[-1] + 1e-7


def test_det_multi_sweep_call_matches_single_sweep_calls_and_rescales_per_call():
    """A multi-sweep call computes the fixed-point scale of A in its first sweep and reuses it: its
    cores have the same bits as the same sweeps made one call at a time. A later call on another
    tensor (2^40 A, whose entries at the first tensor's scale would leave the int64 range) gets
    that tensor's scale: the same bits as a fresh context's sweep on it."""
    dims, ranks, J, seed = (24, 20, 18, 16), (1, 4, 5, 4, 1), 512, 78
    a = synth.add_noise(synth.contract_cores(synth.random_tt(dims, ranks, 5)), 1e-2, np.random.default_rng(8))
    flat, _, _ = synth.quantize(a, "f32")
    init = synth.random_tt(dims, ranks, 9)
    Ad = lib.device_tensor(flat, "f32")
    Abig = Ad * 2.0 ** 40

    def ctx():
        return lib.Context(dims, ranks, J, 1e-3, seed, "f32", flags=DET)

    c1, c3 = ctx(), ctx()
    one, three = lib.device_cores(init), lib.device_cores(init)
    c1.tt_prox_als_sweep(Ad, one, 3, 0, rel_change=False)
    for t in range(3):
        c3.tt_prox_als_sweep(Ad, three, 1, t, rel_change=False)
    torch.cuda.synchronize()
    assert all(torch.equal(x, y) for x, y in zip(one, three))
    after = [x.clone() for x in one]
    c1.tt_prox_als_sweep(Abig, one, 1, 3, rel_change=False)
    fresh = ctx()
    fresh.tt_prox_als_sweep(Abig, after, 1, 3, rel_change=False)
    torch.cuda.synchronize()
    assert all(bool(torch.isfinite(x).all()) for x in one)
    assert all(torch.equal(x, y) for x, y in zip(one, after))
    for c in (c1, c3, fresh):
        c.close()


def test_det_sigma_zero_sinc_runs_repeat_bit_for_bit():
    """The sigma = 0 sinc case of Sec. 5 (m = 45, FP64 update): without fixed orders its 100-sweep
    errors differed between runs of one seeded test; here 30 sweeps run twice give the same bits."""
    dims, ranks, J, seed = (10,) * 6, (1, 5, 5, 5, 5, 5, 1), 45, 20230917
    A = np.asarray(synth.paper_function_tensor("sinc"), np.float32).ravel(order="F")
    init = synth.random_tt(dims, ranks, 100)
    (c1, e1, ch1), (c2, e2, ch2) = _two_runs(dims, ranks, J, 0.0, A, init, 30, seed)
    assert all(torch.equal(x, y) for x, y in zip(c1, c2))
    assert e1 == e2 and ch1 == ch2
    print(f"\nsinc sigma=0 m=45, deterministic: error after 30 sweeps {e1[-1]:.6e}")
