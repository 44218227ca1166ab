"""Host-buffer entry points: tt_prox_als_sweep_host (synchronous) and
tt_prox_als_sweep_host_async + tt_host_sync (a stream of calls whose tensor copies run beside the
previous call's sweeps). Checked through the C ABI with page-locked host arrays: queued calls give
the results of the same calls made one at a time and of the oracle's sweeps, calls on two tensors
alternate correctly through the two device buffers, and a failing call in a queue is reported by
tt_host_sync while the other calls' results are still written."""
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

DIMS, RANKS, J, LAM = (24, 20, 18, 16), (1, 4, 5, 4, 1), 512, 1e-3


def rel(a, b):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel())


def _pinned(x):
    t = torch.empty(x.shape, dtype=torch.from_numpy(x[:1].copy()).dtype, pin_memory=True)
    t.copy_(torch.from_numpy(np.ascontiguousarray(x)))
    return t.numpy()


def _problem(seed):
    cores = synth.random_tt(DIMS, RANKS, seed)
    a = synth.add_noise(synth.contract_cores(cores), 1e-2, np.random.default_rng(seed + 1))
    flat, _, exact = synth.quantize(a, "f32")
    init = synth.random_tt(DIMS, RANKS, seed + 2)
    return _pinned(flat), exact, init


def _host_cores(init):
    return [_pinned(np.asarray(g, np.float32).ravel(order="F")) for g in init]


def _as_cores(hc):
    return [g.astype(np.float64).reshape(RANKS[k], DIMS[k], RANKS[k + 1], order="F") for k, g in enumerate(hc)]


def test_queued_calls_match_single_calls_and_the_oracle():
    A, exact, init = _problem(11)
    ctx = lib.Context(DIMS, RANKS, J, LAM, 21, "f32")
    hc = _host_cores(init)
    outs = [ctx.tt_prox_als_sweep_host_async(A, hc, 1, t, rel_change=True) for t in range(5)]
    ctx.tt_host_sync()
    ctx2 = lib.Context(DIMS, RANKS, J, LAM, 21, "f32")
    hc2 = _host_cores(init)
    errs2 = [ctx2.tt_prox_als_sweep_host(A, hc2, 1, t)[1] for t in range(5)]
    ref, ref_ch = O.tt_ts(exact, init, 21, J, LAM, 5)
    assert rel(O.tt_full(_as_cores(hc)), O.tt_full(_as_cores(hc2))) <= 1e-4
    assert rel(O.tt_full(_as_cores(hc)), O.tt_full(ref)) <= 1e-4
    for t, (chg, err) in enumerate(outs):
        assert abs(err[0] - errs2[t]) <= 1e-4 * errs2[t], (t, err[0], errs2[t])
    assert abs(outs[-1][0][0] - ref_ch[-1]) <= 1e-3 * ref_ch[-1] + 1e-7
    assert abs(outs[-1][1][0] - O.rel_error(exact, _as_cores(hc))) <= 1e-5 * outs[-1][1][0]
    ctx.close()
    ctx2.close()


def test_two_tensors_alternate_through_the_two_buffers():
    (A1, ex1, in1), (A2, ex2, in2) = _problem(31), _problem(41)
    ctx = lib.Context(DIMS, RANKS, J, LAM, 22, "f32")
    h1, h2 = _host_cores(in1), _host_cores(in2)
    outs = []
    for t in range(3):  # six calls in flight-order: tensor 1, tensor 2, tensor 1, ...
        outs.append(ctx.tt_prox_als_sweep_host_async(A1, h1, 1, t))
        outs.append(ctx.tt_prox_als_sweep_host_async(A2, h2, 1, t))
    ctx.tt_host_sync()
    for hc, ex, ini, k in ((h1, ex1, in1, 0), (h2, ex2, in2, 1)):
        ref, _ = O.tt_ts(ex, ini, 22, J, LAM, 3)
        assert rel(O.tt_full(_as_cores(hc)), O.tt_full(ref)) <= 1e-4
        e = outs[4 + k][1][0]
        assert abs(e - O.rel_error(ex, _as_cores(hc))) <= 1e-5 * e
    ctx.close()


def test_a_failing_call_in_a_queue_is_reported():
    A, exact, init = _problem(51)
    bad = A.copy()
    bad[100] = np.nan
    bad = _pinned(bad)
    ctx = lib.Context(DIMS, RANKS, J, LAM, 23, "f32")
    h_ok, h_bad = _host_cores(init), _host_cores(init)
    o1 = ctx.tt_prox_als_sweep_host_async(A, h_ok, 1, 0)
    ctx.tt_prox_als_sweep_host_async(bad, h_bad, 1, 0)
    with pytest.raises(lib.TtError) as e:
        ctx.tt_host_sync()
    assert e.value.code == lib.TT_ENONFINITE
    ref, _ = O.tt_ts(exact, init, 23, J, LAM, 1)
    assert rel(O.tt_full(_as_cores(h_ok)), O.tt_full(ref)) <= 1e-4  # the good call's results stand
    assert abs(o1[1][0] - O.rel_error(exact, _as_cores(h_ok))) <= 1e-5 * o1[1][0]
    o3 = ctx.tt_prox_als_sweep_host_async(A, h_ok, 1, 1)  # and the context goes on
    ctx.tt_host_sync()
    assert np.isfinite(o3[1][0])
    ctx.close()
