"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/*.h declares (no compute calls: CPU only)."""
import ctypes
import os
import re
import shutil

import pytest

from conftest import ROOT


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:u?int64_t|int|void|const char\*)\s+(tt_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2309_08093_gb300 import build

    return build.build()


def test_header_declares_the_api():
    names = _declared()
    for n in ["tt_sketch_init", "tt_sketch_unfold", "tt_sketch_interface", "tt_prox_als_sweep",
              "tt_rel_error", "tt_sketch_destroy", "tt_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in sorted(_declared()):
        assert hasattr(lib, n), n


def test_binding_mirrors_declared_names(libpath):
    from paper_2309_08093_gb300 import lib

    assert set(lib.EXPORTS) == _declared()
    L = lib.load(libpath)
    assert L is not None


def test_init_rejects_bad_parameters(libpath):
    """Parameter validation runs on the host before any device work."""
    from paper_2309_08093_gb300 import lib

    L = lib.load(libpath)

    def init(dims, ranks, J, lam=1e-3, dtype=1):
        n = (ctypes.c_int64 * len(dims))(*dims)
        r = (ctypes.c_int * len(ranks))(*ranks)
        p = lib.TtParams(len(dims), n, r, J, lam, 1, dtype, 0)
        ctx = ctypes.c_void_p()
        return L.tt_sketch_init(ctypes.byref(ctx), ctypes.byref(p), None)

    assert init((4, 5, 6), (1, 2, 2, 1), 12000) == lib.TT_EINVAL    # above 8192, not a power of two
    assert init((4, 5, 6), (1, 2, 2, 1), 1) == lib.TT_EINVAL        # J < 2
    assert init((4, 5, 6), (1, 2, 2, 1), 32768) == lib.TT_EINVAL    # J too large
    assert init((4, 5, 6), (2, 2, 2, 1), 16) == lib.TT_EINVAL       # r[0] != 1
    assert init((4,), (1, 1), 16) == lib.TT_EINVAL                  # d < 2
    assert init((4, 5, 6), (1, 2, 2, 1), 16, lam=-1.0) == lib.TT_EINVAL
    assert init((4, 5, 6), (1, 2, 2, 1), 16, dtype=7) == lib.TT_EINVAL
    assert init((4, 5, 6), (1, 30, 20, 1), 16) == lib.TT_EINVAL     # r_k r_{k+1} > 512
    assert init((4, 500, 6), (1, 4, 100, 1), 16) == lib.TT_EINVAL   # s = 400 with n = 500: no room
    assert init((200, 5, 6), (1, 200, 2, 1), 16) == lib.TT_EINVAL   # a rank above 160


def test_workspace_cap_gives_enomem_before_any_device_call(libpath):
    """A cap below the planned workspaces makes tt_sketch_init return TT_ENOMEM on the host (this
    runs without a GPU: no CUDA call is made before the check); the cap is process-wide and
    returns its previous value."""
    from paper_2309_08093_gb300 import lib

    L = lib.load(libpath)
    dims, ranks = (40, 30, 20), (1, 4, 4, 1)
    n = (ctypes.c_int64 * 3)(*dims)
    r = (ctypes.c_int * 4)(*ranks)
    p = lib.TtParams(3, n, r, 256, 1e-3, 1, lib.TT_F32, 0)
    ctx = ctypes.c_void_p()
    assert lib.tt_set_workspace_limit(1 << 16) == 0
    try:
        assert L.tt_sketch_init(ctypes.byref(ctx), ctypes.byref(p), None) == lib.TT_ENOMEM
        assert not ctx.value
        # bad parameters are still reported as such, whatever the cap
        r_bad = (ctypes.c_int * 4)(2, 4, 4, 1)
        p_bad = lib.TtParams(3, n, r_bad, 256, 1e-3, 1, lib.TT_F32, 0)
        assert L.tt_sketch_init(ctypes.byref(ctx), ctypes.byref(p_bad), None) == lib.TT_EINVAL
    finally:
        assert lib.tt_set_workspace_limit(0) == 1 << 16


def test_binding_constants_match_the_header():
    """Every TT_FLAG_* / storage-type / status constant of the Python binding has the value the
    header defines."""
    from paper_2309_08093_gb300 import lib

    src = open(os.path.join(ROOT, "include", "tt_sketch.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(TT_FLAG_\w+)\s+(\d+)u", src)}
    enums = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(TT_\w+)\s*=\s*(-?\d+)", src)}
    assert len(defs) >= 6
    for name, val in {**defs, **enums}.items():
        if hasattr(lib, name):
            assert getattr(lib, name) == val, name
    for name in defs:
        assert hasattr(lib, name), name
