"""Parity at full size against the CPU FP64 oracle on the same seeded tensor, initial cores and
draws.

Order-4 100^4 workload (J = 4096, TT ranks (1,10,10,10,1), lambda = 1e-3): the 400 MB FP32
tensor the benchmark streams, in the launch configuration it times.

- One sweep of Algorithm 1 through tt_prox_als_sweep_monitored, the benchmark's call (its data
  sketches then run in their in-sweep launch shapes beside the chain kernels): every entry of
  every updated core against the oracle's sweep (relative Frobenius per core, 1e-4: orthogonalised
  cores, whose gauge amplifies rounding), and the relative error the call reports against the
  oracle's relative error of the same (GPU) cores (1e-5).
- The data sketches alone (tt_sketch_unfold, the launch shapes of the isolated roofline), FP32
  and BF16 storage: sampled columns Y_k[:, i_k] of every mode, first, middle and last index,
  against the oracle's column by definition (1e-5 relative per column).

Order-5 40^5 workload (J = 8192, TT ranks (1,8,8,8,8,1) with 0.8^k-decaying cores, 1e-3 noise),
stored BF16 and FP8-E4M3 with per-mode-1-slice scales: five sweeps through the same call from
random cores, to the noise level, against the oracle's five sweeps on the same quantised tensor
(reconstruction 1e-4, relative error 1e-4 of itself), and the error against the unquantised FP64
tensor within 2 delta of the oracle's FP64 run (delta = ||A_q - A|| / ||A||: the
best-approximation error moves by at most delta when A is replaced by A_q).

Warm-start family member 256 x 256 x 3 x 128 (J = 2048, TT ranks (1,20,3,20,1), cumulative-sum
cores, 1% noise; the CPU recipe of the family): the sketch summary the network reads (p = 8 bucket
rows per mode) against the oracle's summary of its own data sketches (1e-5), one sweep against
the oracle's (1e-4 per core, error 1e-5), then the right-canonical gauge of the swept cores and
their packed targets against the warm-start oracle (1e-4 per core relative to its norm, 1e-5).

Batched workload (256 tensors of order 3-4, modes 16-128, ranks 4-12, FP32 and BF16 storage,
12.2 GB): ten batched sweeps (the capture and nine graph replays, as the benchmark times them),
converged to the noise floor, against the single-tensor path on every tensor (relative error; the
two differ only by FP32 summation order: 1e-4 + 1e-7; after two unconverged sweeps that order
alone moved tensor 0 by 1.1e-4), and against the oracle's ten sweeps on the three smallest
tensors and the median one (the reconstructed tensor, 1e-4; the relative error of the same cores,
1e-5 + 1e-7).
"""
import numpy as np
import pytest

import tt_oracle as O
import tt_warmstart as WS
from paper_2309_08093_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_08093_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2309_08093_gb300 import lib  # noqa: E402

W = synth.WORKLOADS["order4-100-r10"]
COLUMNS = (0, 57, 99)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def problem():
    return synth.make_problem(W, storage="f32")


def test_full_size_sweep_matches_oracle(problem):
    p = problem
    assert p.storage.nbytes == 4 * 100 ** 4
    ctx = lib.Context(W.dims, p.ranks, W.J, W.lam, p.sketch_seed, "f32")
    A = lib.device_tensor(p.storage, "f32")
    dc = lib.device_cores(p.init_cores)
    errs, _ = ctx.tt_prox_als_sweep_monitored(A, dc, 1, 0)
    got = lib.host_cores(dc, p.ranks, W.dims)
    ctx.close()
    del A
    ref, _ = O.tt_ts(p.tensor, p.init_cores, p.sketch_seed, W.J, W.lam, 1)
    for k in range(W.d):
        assert rel(got[k], ref[k]) <= 1e-4, (k, rel(got[k], ref[k]))
    e_ref = O.rel_error(p.tensor, [np.asarray(g, np.float32).astype(np.float64) for g in got])
    assert abs(errs[0] - e_ref) <= 1e-5 * e_ref, (errs[0], e_ref)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_full_size_data_sketch_columns(problem, storage):
    p = problem
    if storage == "f32":
        flat, scales, exact = p.storage, None, p.tensor
    else:
        flat, scales, exact = synth.quantize(p.tensor, storage)
    ctx = lib.Context(W.dims, p.ranks, W.J, W.lam, p.sketch_seed, storage)
    A = lib.device_tensor(flat, storage)
    sd = torch.tensor(scales, device="cuda") if scales is not None else None
    Y = [torch.zeros(W.J * n, device="cuda") for n in W.dims]
    sweep = 3
    ctx.tt_sketch_unfold(A, -1, sweep, Y, scales=sd)
    torch.cuda.synchronize()
    hs, vs = O.draw_sketch(p.sketch_seed, sweep, W.dims, W.J)
    for k in range(W.d):
        Yk = Y[k].cpu().numpy()
        for ik in COLUMNS:
            ref = O.sketch_unfolding_column(exact, hs, vs, W.J, k, ik)
            got = Yk[ik * W.J:(ik + 1) * W.J]  # column-major J x n_k
            assert rel(got, ref) <= 1e-5, (storage, k, ik, rel(got, ref))
    ctx.close()


W5 = synth.WORKLOADS["order5-40-r8"]
W5_SWEEPS = 5  # from random cores: 1.0007, 0.654, 0.140, 7.6e-3, 1.03e-3 (FP64 oracle), the noise level


def test_full_size_order5_at_convergence_per_precision():
    """The order-5 40^5 workload (J = 8192, ranks (1,8,8,8,8,1), cores with singular values
    0.8^j, 1e-3 noise) stored BF16 and FP8-E4M3 with slice scales, five sweeps from random cores
    (the error reaches the noise level). Each GPU run is compared with the oracle's five sweeps
    on the same decoded tensor (relative error 1e-4 of itself, reconstruction 1e-4), and its
    error against the unquantised FP64 tensor lies within 2 delta of the FP64 oracle's, delta =
    ||A_q - A|| / ||A||. The three oracle runs (FP64, BF16, FP8: about 40 s per sweep each) run in
    spawned worker processes beside the GPU work."""
    import multiprocessing as mp

    import oracle_runs

    pool = mp.get_context("spawn").Pool(3)
    jobs = pool.starmap_async(oracle_runs.order5_trajectory, [("f64", W5_SWEEPS), ("bf16", W5_SWEEPS),
                                                              ("fp8", W5_SWEEPS)])
    p = synth.make_problem(W5, storage="f64")
    a64 = p.tensor
    assert a64.size == 40 ** 5
    gpu = {}
    for storage in ("bf16", "fp8"):
        flat, scales, exact_q = synth.quantize(a64, storage)
        delta = rel(exact_q, a64)
        del exact_q
        ctx = lib.Context(W5.dims, p.ranks, W5.J, W5.lam, p.sketch_seed, storage)
        A = lib.device_tensor(flat, storage)
        sd = torch.tensor(scales, device="cuda") if scales is not None else None
        dc = lib.device_cores(p.init_cores)
        errs, _ = ctx.tt_prox_als_sweep_monitored(A, dc, W5_SWEEPS, 0, scales=sd)
        got = lib.host_cores(dc, p.ranks, W5.dims)
        ctx.close()
        del A
        got64 = [np.asarray(g, np.float32).astype(np.float64) for g in got]
        gpu[storage] = (got64, errs, delta, O.rel_error(a64, got64))
    try:
        (_, e64, _), (ref_b, eb_q, _), (ref_f, ef_q, _) = jobs.get(timeout=1800)
    finally:
        pool.close()
        pool.join()
    for storage, ref, e_ref in (("bf16", ref_b, eb_q), ("fp8", ref_f, ef_q)):
        got64, errs, delta, e_gpu64 = gpu[storage]
        dev = rel(O.tt_full(got64), O.tt_full(ref))
        print(f"\n{storage}: delta={delta:.3e}; after {W5_SWEEPS} sweeps: error on the decoded tensor gpu="
              f"{errs[-1]:.6e} oracle={e_ref:.6e}; against the FP64 tensor gpu={e_gpu64:.6e}, FP64 oracle "
              f"{e64:.6e}; reconstruction deviation from the oracle {dev:.2e}")
        assert abs(errs[-1] - e_ref) <= 1e-4 * e_ref, (storage, errs[-1], e_ref)
        assert dev <= 1e-4, (storage, dev)
        assert abs(e_gpu64 - e64) <= 2 * delta, (storage, e_gpu64, e64, delta)
        assert e_gpu64 < 0.1  # a converged point, not the first sweep's error of about 1


WW = synth.WORKLOADS["order4-256x256x3x128-r20"]


def test_full_size_warmstart_member():
    p = synth.make_problem(WW)
    dims, J = WW.dims, WW.J
    ctx = lib.Context(dims, p.ranks, J, WW.lam, p.sketch_seed, "f32")
    A = lib.device_tensor(p.storage, "f32")
    # the summary of sweep 0's data sketches
    Y = [torch.zeros(J * n, device="cuda") for n in dims]
    ctx.tt_sketch_unfold(A, -1, 0, Y)
    x = torch.zeros(ctx.tt_ws_summary_dim(8), device="cuda")
    sc = torch.zeros(1, device="cuda")
    ctx.tt_ws_summary(Y, 8, x, sc)
    hs, vs = O.draw_sketch(p.sketch_seed, 0, dims, J)
    x_ref, s_ref = WS.ws_summary([O.sketch_unfolding(p.tensor, hs, vs, J, k) for k in range(WW.d)], 8)
    assert x.numel() == 8 * sum(dims)
    assert rel(x.cpu().numpy(), x_ref) <= 1e-5
    assert abs(float(sc.item()) - s_ref) <= 1e-5 * s_ref
    # one sweep
    dc = lib.device_cores(p.init_cores)
    errs, _ = ctx.tt_prox_als_sweep_monitored(A, dc, 1, 0)
    got = lib.host_cores(dc, p.ranks, dims)
    ref, _ = O.tt_ts(p.tensor, p.init_cores, p.sketch_seed, J, WW.lam, 1)
    for k in range(WW.d):
        assert rel(got[k], ref[k]) <= 1e-4, (k, rel(got[k], ref[k]))
    got64 = [np.asarray(g, np.float32).astype(np.float64) for g in got]
    e_ref = O.rel_error(p.tensor, got64)
    assert abs(errs[0] - e_ref) <= 1e-5 * e_ref, (errs[0], e_ref)
    # gauge and targets
    ctx.tt_canonicalize(dc)
    can = lib.host_cores(dc, p.ranks, dims)
    can_ref = WS.canonicalize_right(got64)
    for k in range(WW.d):
        scale = max(np.linalg.norm(can_ref[k]), 1e-30)
        assert np.linalg.norm(can[k] - can_ref[k]) <= 1e-4 * scale, k
    y = torch.zeros(ctx.tt_ws_core_dim(), device="cuda")
    ctx.tt_ws_pack(dc, sc, y)
    canc = [np.asarray(g, np.float32).astype(np.float64) for g in can]
    assert rel(y.cpu().numpy(), WS.ws_targets(canc, float(sc.item()))) <= 1e-5
    ctx.close()


def test_full_size_batched_workload():
    specs = synth.batched_specs()
    assert len(specs) == 256
    As, inits = [], []
    for sp in specs:
        a, init = synth.batched_tensor_gpu(sp)
        As.append(a)
        inits.append(init)
    cores_b = [lib.device_cores(c) for c in inits]
    batch = lib.Batch(specs)
    batch.tt_batch_sweep(As, cores_b, 1, 0)  # autotune, capture, first sweep
    batch.tt_batch_sweep(As, cores_b, 9, 1)  # graph replays
    errs_b = batch.tt_batch_rel_error(As, cores_b)
    batch.close()
    bad = []
    for i, sp in enumerate(specs):
        ctx = lib.Context(sp["dims"], sp["ranks"], sp["J"], sp["lam"], sp["seed"], sp["dtype"])
        cs = lib.device_cores(inits[i])
        ctx.tt_prox_als_sweep(As[i], cs, 10, 0, rel_change=False)
        e = ctx.tt_rel_error(As[i], cs)
        ctx.close()
        if not abs(errs_b[i] - e) <= 1e-4 * e + 1e-7:
            bad.append((i, errs_b[i], e))
    assert not bad, bad
    size = [int(np.prod(sp["dims"])) for sp in specs]
    order = sorted(range(len(specs)), key=lambda i: size[i])
    for i in order[:3] + [order[len(order) // 2]]:
        sp = specs[i]
        exact = As[i].float().cpu().numpy().astype(np.float64).reshape(sp["dims"], order="F")
        ref, _ = O.tt_ts(exact, inits[i], sp["seed"], sp["J"], sp["lam"], 10)
        got = [np.asarray(g, np.float32).astype(np.float64)
               for g in lib.host_cores(cores_b[i], sp["ranks"], sp["dims"])]
        assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4, (i, sp["dims"], sp["ranks"])
        e_ref = O.rel_error(exact, got)
        assert abs(errs_b[i] - e_ref) <= 1e-5 * e_ref + 1e-7, (i, errs_b[i], e_ref)
