"""The allocation-free proximal update (tt_prox_update_noalloc) is for callers that cannot
allocate device memory: an application whose memory manager already holds all the device memory
it may use, or a latency-critical loop that cannot pay for cudaMalloc's implicit device-wide
synchronisation. It must give the core that the oracle's Eq. (ite) update gives, and the same
core as the context-based tt_prox_update.

It lives in its own file, named to be collected last, so that a run stopping at the first
failure has already run every other test. It passes alone in a fresh process as well as after
the rest of the suite: every call clears the part of the shared static scratch that it uses."""
import ctypes

import numpy as np
import pytest

import tt_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_08093_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2309_08093_gb300 import lib  # noqa: E402

TOL = 1e-5
CASES = [(4096, 100, 10, 10, 1e-3, 1), (512, 37, 3, 5, 0.5, 2)]


def _host_inputs(J, n, r0, r1, seed):
    rng = np.random.default_rng(seed)
    s = r0 * r1
    SH = np.linalg.qr(rng.standard_normal((J, s)))[0] * (1.0 + 0.1 * rng.standard_normal(s))
    Y = rng.standard_normal((J, n))
    G = rng.standard_normal((r0, n, r1))
    return Y.astype(np.float32), SH.astype(np.float32), G.astype(np.float32)


def _device(Y, SH, G):
    return (torch.from_numpy(np.ascontiguousarray(Y.T.ravel())).cuda(),  # J x n column-major
            torch.from_numpy(np.ascontiguousarray(SH.T.ravel())).cuda(),  # J x s column-major
            torch.from_numpy(np.ascontiguousarray(G.ravel(order="F"))).cuda())


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _with_context(Y, SH, core, J, n, r0, r1, sigma):
    dims, ranks = (5, n, 3), (1, r0, r1, 1)
    ctx = lib.Context(dims, ranks, J, sigma, 1, "f32")
    out = core.clone()
    ctx.tt_prox_update(Y, SH, out, 1)
    ctx.close()
    return out


def _oracle(Yh, SHh, Gh, sigma):
    return O.prox_update(Yh.astype(np.float64), SHh.astype(np.float64), Gh.astype(np.float64), sigma)


def test_noalloc_matches_oracle_and_context_update_on_repeated_calls():
    """Three calls in a row (the first case again after the second, so the second call's scratch
    contents are there when the third starts), the last on a non-default stream."""
    side = torch.cuda.Stream()
    for i, (J, n, r0, r1, sigma, seed) in enumerate(CASES + CASES[:1]):
        Yh, SHh, Gh = _host_inputs(J, n, r0, r1, seed)
        Y, SH, core = _device(Yh, SHh, Gh)
        ref_ctx = _with_context(Y, SH, core, J, n, r0, r1, sigma).cpu().numpy()
        ref = _oracle(Yh, SHh, Gh, sigma)
        got = core.clone()
        if i == len(CASES):
            side.wait_stream(torch.cuda.current_stream())
            rc = lib.tt_prox_update_noalloc(Y, SH, got, J, n, r0, r1, sigma,
                                            stream=ctypes.c_void_p(side.cuda_stream))
            torch.cuda.current_stream().wait_stream(side)
        else:
            rc = lib.tt_prox_update_noalloc(Y, SH, got, J, n, r0, r1, sigma)
        assert rc == lib.TT_OK
        g = got.cpu().numpy()
        assert _rel(g.reshape(r0, n, r1, order="F"), ref) <= TOL
        assert _rel(g, ref_ctx) <= TOL


def test_noalloc_refuses_a_singular_gram_and_leaves_the_core_unchanged():
    """sigma = 0 with a zero column of S H_k: the Gram has a zero pivot, which the oracle's
    Cholesky refuses too; the call returns TT_ENOTSPD and the core keeps its bits."""
    J, n, r0, r1 = 256, 20, 3, 4
    Yh, SHh, Gh = _host_inputs(J, n, r0, r1, 7)
    SHh[:, 5] = 0.0
    with pytest.raises(O.NotSPD):
        _oracle(Yh, SHh, Gh, 0.0)
    Y, SH, core = _device(Yh, SHh, Gh)
    before = core.clone()
    assert lib.tt_prox_update_noalloc(Y, SH, core, J, n, r0, r1, 0.0) == lib.TT_ENOTSPD
    assert torch.equal(core, before)
    # the next call starts from a cleared status word
    Yh, SHh, Gh = _host_inputs(J, n, r0, r1, 8)
    Y, SH, core = _device(Yh, SHh, Gh)
    assert lib.tt_prox_update_noalloc(Y, SH, core, J, n, r0, r1, 0.0) == lib.TT_OK
    assert _rel(core.cpu().numpy().reshape(r0, n, r1, order="F"), _oracle(Yh, SHh, Gh, 0.0)) <= 1e-4


def test_noalloc_rejects_sizes_beyond_its_scratch():
    Yh, SHh, Gh = _host_inputs(64, 8, 2, 2, 3)
    Y, SH, core = _device(Yh, SHh, Gh)
    before = core.clone()
    assert lib.tt_prox_update_noalloc(Y, SH, core, 64, 2000, 2, 2, 1e-3) == lib.TT_EINVAL
    assert lib.tt_prox_update_noalloc(Y, SH, core, 64, 8, 13, 13, 1e-3) == lib.TT_EINVAL
    # 65536 * 65536 wraps to 0 in 32-bit arithmetic: refused before any launch
    assert lib.tt_prox_update_noalloc(Y, SH, core, 64, 8, 65536, 65536, 1e-3) == lib.TT_EINVAL
    assert lib.tt_prox_update_noalloc(Y, SH, core, 64, 8, 0, 4, 1e-3) == lib.TT_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(core, before)
