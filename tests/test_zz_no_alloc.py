"""The allocation-free proximal update (tt_prox_update_noalloc), for callers that cannot
allocate device memory, must give the same core as the context-based tt_prox_update.

It lives in its own file, named to be collected last, so that a run stopping at the first
failure has already run every other test. It passes alone in a fresh process as well as after
the rest of the suite (the shared static scratch is cleared by every call)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_08093_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2309_08093_gb300 import lib  # noqa: E402

TOL = 1e-5


def _inputs(J, n, r0, r1, seed):
    rng = np.random.default_rng(seed)
    s = r0 * r1
    SH = np.linalg.qr(rng.standard_normal((J, s)))[0] * (1.0 + 0.1 * rng.standard_normal(s))
    Y = rng.standard_normal((J, n))
    G = rng.standard_normal((r0, n, r1))
    return (torch.from_numpy(np.ascontiguousarray(Y.astype(np.float32))).cuda(),
            torch.from_numpy(np.ascontiguousarray(SH.T.astype(np.float32))).cuda(),
            torch.from_numpy(np.ascontiguousarray(G.astype(np.float32).ravel(order="F"))).cuda())


def _with_context(Y, SH, core, J, n, r0, r1, sigma):
    dims, ranks = (5, n, 3), (1, r0, r1, 1)
    ctx = lib.Context(dims, ranks, J, sigma, 1, "f32")
    out = core.clone()
    ctx.tt_prox_update(Y, SH, out, 1)
    ctx.close()
    return out


def test_noalloc_matches_context_update_twice_in_a_row():
    cases = [(4096, 100, 10, 10, 1e-3, 1), (512, 37, 3, 5, 0.5, 2)]
    for J, n, r0, r1, sigma, seed in cases:
        Y, SH, core = _inputs(J, n, r0, r1, seed)
        ref = _with_context(Y, SH, core, J, n, r0, r1, sigma)
        got = core.clone()
        rc = lib.tt_prox_update_noalloc(Y, SH, got, J, n, r0, r1, sigma)
        assert rc == lib.TT_OK
        a, b = got.cpu().double().numpy(), ref.cpu().double().numpy()
        assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    Y, SH, core = _inputs(64, 8, 2, 2, 3)
    assert lib.tt_prox_update_noalloc(Y, SH, core, 64, 2000, 2, 2, 1e-3) == lib.TT_EINVAL
    assert lib.tt_prox_update_noalloc(Y, SH, core, 64, 8, 13, 13, 1e-3) == lib.TT_EINVAL
