"""Mixed-precision forms against the FP64 oracle.

The tensor is stored in BF16 (round to nearest even) or FP8-E4M3 with one FP32 scale per mode-1
slice; the GPU sketches in FP32. Two kinds of checks:
  * parity: on the SAME quantized tensor the GPU matches the oracle to the FP32 tolerance;
  * error against the unquantized FP64 problem, within bounds stated from the formats:
      - a sketch is a signed sum of entries, so its relative Frobenius error is about the
        entries' relative rounding error u / sqrt(3) (u = 2^-9 for BF16, 2^-4 for E4M3 with the
        slice scale mapping the slice maximum to 448); the bounds below are 2u;
      - the best TT approximation error moves by at most delta = ||A_q - A|| / ||A|| when A is
        replaced by A_q (triangle inequality); for the ALS iterates the bound used is 2 delta.
Observed values are printed (pytest -s)."""
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

U = {"bf16": 2.0 ** -9, "fp8": 2.0 ** -4}


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_sketch_error_against_fp64(storage):
    w = synth.WORKLOADS["order4-100-r10"].scaled((40, 36, 32, 28), J=1024)
    p = synth.make_problem(w, storage="f64")
    a64 = p.tensor
    flat, scales, exact_q = synth.quantize(a64, storage)
    ctx = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, storage)
    Y = [torch.zeros(w.J * n, device="cuda") for n in w.dims]
    sd = torch.tensor(scales, device="cuda") if scales is not None else None
    ctx.tt_sketch_unfold(lib.device_tensor(flat, storage), -1, 0, Y, scales=sd)
    hs, vs = O.draw_sketch(p.sketch_seed, 0, w.dims, w.J)
    errs = []
    for k in range(w.d):
        got = Y[k].cpu().numpy().reshape(w.dims[k], w.J).T
        # parity on the same quantized data
        assert rel(got, O.sketch_unfolding(exact_q, hs, vs, w.J, k)) <= 1e-5
        errs.append(rel(got, O.sketch_unfolding(a64, hs, vs, w.J, k)))
    print(f"\n{storage}: sketch relative error vs FP64 per mode {['%.3e' % e for e in errs]} (bound {2 * U[storage]:.3e})")
    assert max(errs) <= 2 * U[storage]
    ctx.close()


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_sweeps_error_against_fp64(storage):
    """Order-5 tensor with 0.8^k-decaying cores (the recipe of the 40^5 workload, scaled)."""
    w = synth.WORKLOADS["order5-40-r8"].scaled((16, 14, 12, 12, 10), J=1024)
    p = synth.make_problem(w, storage="f64")
    a64 = p.tensor
    flat, scales, exact_q = synth.quantize(a64, storage)
    delta = rel(exact_q, a64)
    nsw = 6
    ctx = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, storage)
    dc = lib.device_cores(p.init_cores)
    sd = torch.tensor(scales, device="cuda") if scales is not None else None
    ctx.tt_prox_als_sweep(lib.device_tensor(flat, storage), dc, nsw, 0, scales=sd)
    got = lib.host_cores(dc, p.ranks, w.dims)
    ref_q, _ = O.tt_ts(exact_q, p.init_cores, p.sketch_seed, w.J, w.lam, nsw)  # same quantized input
    ref_64, _ = O.tt_ts(a64, p.init_cores, p.sketch_seed, w.J, w.lam, nsw)   # FP64 problem
    e_gpu = O.rel_error(a64, got)
    e_q = O.rel_error(a64, ref_q)
    e_64 = O.rel_error(a64, ref_64)
    print(f"\n{storage}: delta={delta:.3e} rel error vs FP64 tensor: gpu={e_gpu:.6e} oracle(quantized)={e_q:.6e} "
          f"oracle(fp64)={e_64:.6e}")
    assert abs(e_gpu - e_q) <= 1e-5 * e_q + 1e-7      # FP32 parity on the same input
    assert abs(e_gpu - e_64) <= 2 * delta + 1e-4      # stated precision bound
    ctx.close()
