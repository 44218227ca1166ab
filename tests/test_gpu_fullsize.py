"""Parity at the full size of the order-4 100^4 workload (J = 4096, TT ranks (1,10,10,10,1),
lambda = 1e-3): the 400 MB FP32 tensor the benchmark streams, in the launch configuration it
times, against the CPU FP64 oracle on the same seeded tensor, initial cores and draws.

- One sweep of Algorithm 1 through tt_prox_als_sweep_monitored, the benchmark's call (its data
  sketches then run in their in-sweep launch shapes beside the chain kernels): every entry of
  every updated core against the oracle's sweep (relative Frobenius per core, 1e-4: orthogonalised
  cores, whose gauge amplifies rounding), and the relative error the call reports against the
  oracle's relative error of the same (GPU) cores (1e-5).
- The data sketches alone (tt_sketch_unfold, the launch shapes of the isolated roofline), FP32
  and BF16 storage: sampled columns Y_k[:, i_k] of every mode, first, middle and last index,
  against the oracle's column by definition (1e-5 relative per column).
"""
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
