"""The tensor-core Gram of the proximal update (Eq. (ite)): [S H_k | Y_k]^T (S H_k) by tcgen05.mma
kind::tf32 with TMA-staged operands and FP32 accumulators in tensor memory. Checked through the
C ABI against the CPU FP64 oracle's update:
  * TF32 x 3 (TT_FLAG_TC_GRAM, operands split into two TF32 parts): the FP32 form's 1e-5, over
    shapes with one and two output tiles, ragged K, the deterministic mode, and whole sweeps;
  * TF32 x 1 (TT_FLAG_TF32_GRAM, the mixed-precision form): its error against the oracle is
    printed and bounded by 1e-2 (operands read with 10 explicit mantissa bits; the bound holds
    for the well-conditioned M of these systems, cond(M) <= 2)."""
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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _update(J, n, r0, r1, sigma, flags, seed):
    rng = np.random.default_rng(seed)
    s = r0 * r1
    SH = (np.linalg.qr(rng.standard_normal((J, s)))[0] * (1.0 + 0.1 * rng.standard_normal(s))).astype(np.float32)
    Y = rng.standard_normal((J, n)).astype(np.float32)
    G = rng.standard_normal((r0, n, r1)).astype(np.float32)
    dims = (n, 4, 3) if r0 == 1 else (5, n, 3)
    k = 0 if r0 == 1 else 1
    ranks = (1, r1, 1, 1) if k == 0 else (1, r0, r1, 1)
    ctx = lib.Context(dims, ranks, J, sigma, 5, "f32", flags=flags)
    Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda()
    SHd = torch.from_numpy(np.ascontiguousarray(SH.T)).cuda()
    core = torch.from_numpy(np.ascontiguousarray(G.ravel(order="F"))).cuda()
    ctx.tt_prox_update(Yd, SHd, core, k)
    got = core.cpu().numpy().astype(np.float64).reshape(r0, n, r1, order="F")
    ctx.close()
    ref = O.prox_update(Y.astype(np.float64), SH.astype(np.float64), G.astype(np.float64), sigma)
    return rel(got, ref)


CASES = [(4096, 100, 10, 10, 1e-3), (2048, 256, 1, 20, 0.5), (8192, 40, 8, 8, 1e-3), (512, 128, 12, 12, 1e-3),
         (1000, 100, 10, 10, 1e-3), (4096, 200, 12, 13, 1e-3), (64, 3, 1, 1, 2.0), (4100, 33, 4, 5, 1e-2)]


@pytest.mark.parametrize("J,n,r0,r1,sigma", CASES)
def test_tc_gram_split3_matches_oracle(J, n, r0, r1, sigma):
    e = _update(J, n, r0, r1, sigma, lib.TT_FLAG_TC_GRAM, J + n)
    assert e <= 1e-5, e
    e = _update(J, n, r0, r1, sigma, lib.TT_FLAG_TC_GRAM | lib.TT_FLAG_DETERMINISTIC, J + n)
    assert e <= 1e-5, e


@pytest.mark.parametrize("J,n,r0,r1,sigma", CASES[:5])
def test_tc_gram_tf32_error_bound(J, n, r0, r1, sigma):
    e = _update(J, n, r0, r1, sigma, lib.TT_FLAG_TF32_GRAM, J + n)
    print(f"\nTF32 x 1 Gram: J={J} n={n} s={r0 * r1}: update error against the FP64 oracle {e:.3e}")
    assert e <= 1e-2, e


def test_tc_gram_sweeps_match_oracle():
    w = synth.WORKLOADS["order4-100-r10"].scaled((24, 20, 18, 16), J=512)
    p = synth.make_problem(w, storage="f32")
    ctx = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, "f32", flags=lib.TT_FLAG_TC_GRAM)
    A = lib.device_tensor(p.storage, "f32")
    dc = lib.device_cores(p.init_cores)
    ctx.tt_prox_als_sweep(A, dc, 4, 0, rel_change=False)
    err = ctx.tt_rel_error(A, dc)
    got = lib.host_cores(dc, p.ranks, w.dims)
    ctx.close()
    ref, _ = O.tt_ts(p.tensor, p.init_cores, p.sketch_seed, w.J, w.lam, 4)
    assert rel(O.tt_full(got), O.tt_full(ref)) <= 1e-4
    e_ref = O.rel_error(p.tensor, ref)
    assert abs(err - e_ref) <= 1e-5 * e_ref + 1e-7
