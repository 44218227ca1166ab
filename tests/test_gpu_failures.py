"""Failure paths through the C ABI, made on the host: a NaN written into the data, a NaN in a
sketch, a workspace cap. No GPU fault is involved: the kernels raise a status word that the
host reads back, and the cores are left as they were before the refused update."""
import numpy as np
import pytest

from paper_2309_08093_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_08093_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2309_08093_gb300 import lib  # noqa: E402

DIMS, RANKS, J = (24, 20, 18, 16), (1, 4, 5, 4, 1), 512


def _host_problem(seed):
    cores = synth.random_tt(DIMS, RANKS, seed)
    a = synth.add_noise(synth.contract_cores(cores), 1e-2, np.random.default_rng(seed + 1))
    A = np.ascontiguousarray(a.ravel(order="F").astype(np.float32))
    init = [np.ascontiguousarray(np.asarray(g, np.float32).ravel(order="F")) for g in synth.random_tt(DIMS, RANKS, seed + 2)]
    return A, init


@pytest.mark.parametrize("sigma", [1e-3, 0.0])  # the FP32 and the FP64 update
def test_nan_in_host_tensor_gives_enonfinite(sigma):
    A, init = _host_problem(3)
    A[12345] = np.nan
    ctx = lib.Context(DIMS, RANKS, J, sigma, 7, "f32")
    cores = [g.copy() for g in init]
    with pytest.raises(lib.TtError) as e:
        ctx.tt_prox_als_sweep_host(A, cores, 1, 0)
    assert e.value.code == lib.TT_ENONFINITE
    assert all(np.all(np.isfinite(g)) for g in cores)  # the refused update wrote nothing
    A[12345] = 0.0  # the same context recovers on clean data
    ctx.tt_prox_als_sweep_host(A, cores, 2, 0)
    ctx.close()


@pytest.mark.parametrize("sigma", [1e-3, 0.0])
@pytest.mark.parametrize("where", ["Y", "SH"])
def test_nan_in_a_sketch_gives_enonfinite_and_keeps_the_core(sigma, where):
    n, r0, r1 = 20, 4, 5
    ctx = lib.Context(DIMS, RANKS, J, sigma, 7, "f32")
    rng = np.random.default_rng(4)
    SH = torch.from_numpy(np.linalg.qr(rng.standard_normal((J, r0 * r1)))[0].T.astype(np.float32).ravel()).cuda()
    Y = torch.randn(n * J, device="cuda")
    (Y if where == "Y" else SH)[77] = float("nan")
    core = torch.randn(r0 * n * r1, device="cuda")
    before = core.clone()
    with pytest.raises(lib.TtError) as e:
        ctx.tt_prox_update(Y, SH, core, 1)
    assert e.value.code == lib.TT_ENONFINITE
    assert torch.equal(core, before)
    ctx.close()


def test_workspace_cap_stops_the_host_entry_point_before_it_allocates():
    """A context made before the cap keeps its workspaces; the host-buffer sweep's staging
    buffers (the tensor and the cores) would exceed the cap, so it returns TT_ENOMEM and
    leaves the host cores alone."""
    A, init = _host_problem(5)
    ctx = lib.Context(DIMS, RANKS, J, 1e-3, 7, "f32")
    cores = [g.copy() for g in init]
    prev = lib.tt_set_workspace_limit(1 << 20)
    try:
        with pytest.raises(lib.TtError) as e:
            ctx.tt_prox_als_sweep_host(A, cores, 1, 0)
        assert e.value.code == lib.TT_ENOMEM
        assert all(np.array_equal(a, b) for a, b in zip(cores, init))
        lib.tt_set_workspace_limit(1 << 16)  # below this shape's workspaces (about 0.4 MB)
        with pytest.raises(lib.TtError) as e:  # a new context above the cap
            lib.Context(DIMS, RANKS, J, 1e-3, 7, "f32")
        assert e.value.code == lib.TT_ENOMEM
    finally:
        lib.tt_set_workspace_limit(prev)
    ctx.tt_prox_als_sweep_host(A, cores, 1, 0)  # without the cap it runs
    ctx.close()
