"""Batched driver: many tensors of different order, size, rank, sketch size and storage swept by
one graph launch per sweep must give what the single-tensor path gives (and the oracle)."""
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


def _setup(specs):
    As, inits, flats = [], [], []
    for sp in specs:
        a, init = synth.batched_tensor_cpu(sp)
        flat, _, exact = synth.quantize(a, sp["dtype"])
        As.append(lib.device_tensor(flat, sp["dtype"]))
        inits.append(init)
        flats.append(exact)
    return As, inits, flats


@pytest.mark.parametrize("autotune", [False, True])
def test_batched_matches_single_tensor_path_and_oracle(autotune):
    """Batched vs single-tensor GPU runs differ only by FP32 summation order (fibres reach a
    group in a nondeterministic order, and the batch sizes its work items by bytes); before
    convergence the iteration amplifies that, so the comparison uses 1e-4. The oracle comparison
    keeps the FP32 tolerance 1e-5 (+1e-7 absolute). With TT_FLAG_BATCH_AUTOTUNE on every other
    tensor, those tensors' data sketches run in the launch shapes the autotuner picked."""
    nsw = 8
    specs = synth.batched_specs(count=7, dims_range=(6, 18), rank_range=(2, 5))
    if autotune:
        for sp in specs[::2]:
            sp["flags"] = lib.TT_FLAG_BATCH_AUTOTUNE
    As, inits, exact = _setup(specs)
    cores_b = [lib.device_cores(c) for c in inits]
    batch = lib.Batch(specs)
    batch.tt_batch_sweep(As, cores_b, nsw, 0)
    errs_b = batch.tt_batch_rel_error(As, cores_b)
    bad = []
    for i, sp in enumerate(specs):
        ctx = lib.Context(sp["dims"], sp["ranks"], sp["J"], sp["lam"], sp["seed"], sp["dtype"])
        cs = lib.device_cores(inits[i])
        ctx.tt_prox_als_sweep(As[i], cs, nsw, 0, rel_change=False)
        e_single = ctx.tt_rel_error(As[i], cs)
        ctx.close()
        if abs(errs_b[i] - e_single) > 1e-4 * e_single + 1e-7:
            bad.append((i, errs_b[i], e_single))
    assert not bad, bad
    for i in (0, 1):  # against the oracle on the same (quantized) input
        ref_cores, _ = O.tt_ts(exact[i], inits[i], specs[i]["seed"], specs[i]["J"], specs[i]["lam"], nsw)
        e_ref = O.rel_error(exact[i], ref_cores)
        got = O.rel_error(exact[i], lib.host_cores(cores_b[i], specs[i]["ranks"], specs[i]["dims"]))
        # near the noise floor the relative error is a difference of nearly equal norms, so its
        # FP32 perturbation is absolute (at most ||X' - X|| / ||A||): 1e-5 relative + 1e-7
        assert abs(got - e_ref) <= 1e-5 * e_ref + 1e-7, (i, got, e_ref)
        # the same cores evaluated by the GPU (FP32 reconstruction X') and in FP64 (X): by the
        # triangle inequality they differ by at most ||X' - X|| / ||A||, a few units of FP32
        # rounding: absolute, not relative to the (small) error itself
        assert abs(errs_b[i] - got) <= 1e-6 * got + 1e-7, (i, errs_b[i], got)
    batch.close()


def test_batched_sweeps_continue_and_recapture():
    """Replays draw sweep first_sweep + t; new core buffers force a recapture. After 4 sweeps the
    iterates are not converged: summation-order differences show up at ~1e-4 relative, while a
    wrong draw sequence changes the error at ~1e-2, so the bound is 1e-3."""
    specs = synth.batched_specs(count=3, dims_range=(8, 14), rank_range=(2, 4))
    As, inits, _ = _setup(specs)
    batch = lib.Batch(specs)
    c1 = [lib.device_cores(c) for c in inits]
    batch.tt_batch_sweep(As, c1, 2, 0)
    batch.tt_batch_sweep(As, c1, 2, 2)          # continue: sweeps 2, 3
    c2 = [lib.device_cores(c) for c in inits]   # new buffers: recapture
    batch.tt_batch_sweep(As, c2, 4, 0)
    e1 = batch.tt_batch_rel_error(As, c1)
    e2 = batch.tt_batch_rel_error(As, c2)
    for a, b in zip(e1, e2):
        assert abs(a - b) <= 1e-3 * b
    batch.close()


def test_batched_fixed_draw_reuses_data_sketches():
    """Tensors with TT_FLAG_FIXED_SKETCH (every other one) sweep their later sweeps of a call on the
    data sketches of its first sweep (a second graph): four sweeps in one call against the
    single-tensor path with the same flag (1e-4 on the relative error) and, for tensor 0, the
    oracle's four sweeps with sweep 0's draw (reconstruction 1e-4). A second call continues with
    fresh sketches of the same data (first graph, then the reuse graph again)."""
    specs = synth.batched_specs(count=5, dims_range=(6, 16), rank_range=(2, 4))
    for sp in specs[::2]:
        sp["flags"] = lib.TT_FLAG_FIXED_SKETCH
    As, inits, exact = _setup(specs)
    cores_b = [lib.device_cores(c) for c in inits]
    batch = lib.Batch(specs)
    batch.tt_batch_sweep(As, cores_b, 4, 0)
    batch.tt_batch_sweep(As, cores_b, 2, 4)
    errs_b = batch.tt_batch_rel_error(As, cores_b)
    batch.close()
    for i, sp in enumerate(specs):
        ctx = lib.Context(sp["dims"], sp["ranks"], sp["J"], sp["lam"], sp["seed"], sp["dtype"], flags=sp.get("flags", 0))
        cs = lib.device_cores(inits[i])
        ctx.tt_prox_als_sweep(As[i], cs, 4, 0, rel_change=False)
        ctx.tt_prox_als_sweep(As[i], cs, 2, 4, rel_change=False)
        e_single = ctx.tt_rel_error(As[i], cs)
        ctx.close()
        assert abs(errs_b[i] - e_single) <= 1e-4 * e_single + 1e-7, (i, errs_b[i], e_single)
    ref = [np.asarray(g, np.float64) for g in inits[0]]
    for _ in range(6):
        ref, _ = O.tt_ts_sweep(exact[0], ref, specs[0]["seed"], 0, specs[0]["J"], specs[0]["lam"])
    got = lib.host_cores(cores_b[0], specs[0]["ranks"], specs[0]["dims"])
    d = np.linalg.norm((O.tt_full(got) - O.tt_full(ref)).ravel()) / np.linalg.norm(O.tt_full(ref).ravel())
    assert d <= 1e-4, d


def test_batched_deterministic_repeats_and_matches_single_tensor_bits():
    """TT_FLAG_DETERMINISTIC on every tensor of a batch: two batches over the same inputs give the
    same bits, and so does each tensor's single-tensor deterministic sweep (its data sketch takes
    work spans fixed by the shape, so the batch's own item sizes and the graph change nothing);
    tensor 0 agrees with the oracle (reconstruction 1e-4, as above)."""
    nsw = 4
    specs = synth.batched_specs(count=4, dims_range=(6, 18), rank_range=(2, 5))
    for sp in specs:
        sp["flags"] = lib.TT_FLAG_DETERMINISTIC
    As, inits, exact = _setup(specs)
    runs = []
    for _ in range(2):
        cores_b = [lib.device_cores(c) for c in inits]
        batch = lib.Batch(specs)
        batch.tt_batch_sweep(As, cores_b, nsw, 0)
        torch.cuda.synchronize()
        batch.close()
        runs.append(cores_b)
    for i in range(len(specs)):
        assert all(torch.equal(x, y) for x, y in zip(runs[0][i], runs[1][i])), i
    for i, sp in enumerate(specs):
        ctx = lib.Context(sp["dims"], sp["ranks"], sp["J"], sp["lam"], sp["seed"], sp["dtype"], flags=sp["flags"])
        cs = lib.device_cores(inits[i])
        ctx.tt_prox_als_sweep(As[i], cs, nsw, 0, rel_change=False)
        torch.cuda.synchronize()
        ctx.close()
        assert all(torch.equal(x, y) for x, y in zip(runs[0][i], cs)), i
    ref, _ = O.tt_ts(exact[0], inits[0], specs[0]["seed"], specs[0]["J"], specs[0]["lam"], nsw)
    got = lib.host_cores(runs[0][0], specs[0]["ranks"], specs[0]["dims"])
    d = np.linalg.norm((O.tt_full(got) - O.tt_full(ref)).ravel()) / np.linalg.norm(O.tt_full(ref).ravel())
    assert d <= 1e-4, d
