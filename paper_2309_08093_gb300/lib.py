"""Thin ctypes binding to libttsketch.so (declared in include/tt_sketch.h).

Function names mirror the C ABI. This module only marshals arguments (torch CUDA tensors or
host numpy arrays to raw pointers); every step of the computation runs in the CUDA library.
Loading fails loudly if the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libttsketch.so")

TT_F64, TT_F32, TT_BF16, TT_FP8E4M3 = 0, 1, 2, 3
DTYPES = {"f64": TT_F64, "f32": TT_F32, "bf16": TT_BF16, "fp8": TT_FP8E4M3}
TT_OK, TT_EINVAL, TT_ENOMEM, TT_ECUDA, TT_ENOTSPD, TT_ETIMEOUT, TT_ENONFINITE = 0, -1, -2, -3, -4, -5, -6
TT_FLAG_FIXED_SKETCH = 1
TT_FLAG_FP64_SOLVE = 2
TT_FLAG_DETERMINISTIC = 4
TT_FLAG_TC_GRAM = 8
TT_FLAG_TF32_GRAM = 16
TT_FLAG_BATCH_AUTOTUNE = 32

EXPORTS = ["tt_sketch_init", "tt_sketch_destroy", "tt_last_error", "tt_sketch_tables",
           "tt_sketch_set_tables", "tt_sketch_unfold", "tt_sketch_unfold_coo", "tt_rel_error_coo", "tt_sketch_interface", "tt_prox_update",
           "tt_orthogonalize", "tt_prox_als_sweep", "tt_rel_error", "tt_prox_als_sweep_host",
           "tt_profile_enable", "tt_profile_read", "tt_prox_update_noalloc", "tt_batch_init",
           "tt_batch_destroy", "tt_batch_last_error", "tt_batch_sweep", "tt_batch_rel_error",
           "tt_prox_als_sweep_sketched", "tt_prox_als_sweep_monitored", "tt_set_workspace_limit",
           "tt_prox_als_sweep_host_async", "tt_host_sync",
           # learned warm start (include/tt_warmstart.h)
           "tt_mlp_init", "tt_mlp_destroy", "tt_mlp_last_error", "tt_mlp_set_weights", "tt_mlp_get_weights",
           "tt_mlp_forward", "tt_mlp_loss_grads", "tt_mlp_train_step", "tt_mlp_gemm_bf16",
           "tt_ws_summary_dim", "tt_ws_core_dim", "tt_ws_summary", "tt_canonicalize", "tt_ws_pack",
           "tt_ws_unpack"]
_NOT_INT = {"tt_sketch_destroy", "tt_set_workspace_limit", "tt_last_error", "tt_batch_destroy", "tt_batch_last_error", "tt_mlp_last_error",
            "tt_ws_summary_dim", "tt_ws_core_dim"}


class TtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tt error {code}: {msg}")
        self.code = code


class TtProfile(ctypes.Structure):
    _fields_ = [("unfold_ms", ctypes.c_double), ("unfold_launches", ctypes.c_int64),
                ("unfold_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("mode_ms", ctypes.c_double * 8), ("mode_launches", ctypes.c_int64 * 8)]


class TtMlpParams(ctypes.Structure):
    _fields_ = [("in_dim", ctypes.c_int), ("hidden", ctypes.c_int), ("out_dim", ctypes.c_int),
                ("batch_max", ctypes.c_int), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


class TtParams(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.POINTER(ctypes.c_int64)),
                ("r", ctypes.POINTER(ctypes.c_int)), ("J", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("dtype", ctypes.c_int), ("flags", ctypes.c_uint)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libttsketch.so not found at {path}; run paper_2309_08093_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
    L.tt_sketch_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(TtParams), vp]
    L.tt_sketch_destroy.argtypes = [vp]
    L.tt_sketch_destroy.restype = None
    L.tt_last_error.argtypes = [vp]
    L.tt_last_error.restype = ctypes.c_char_p
    L.tt_sketch_tables.argtypes = [vp, u64, vp, vp]
    L.tt_sketch_set_tables.argtypes = [vp, vp, vp]
    L.tt_sketch_unfold.argtypes = [vp, vp, vp, i, u64, ctypes.POINTER(vp)]
    L.tt_sketch_unfold_coo.argtypes = [vp, vp, vp, ctypes.c_int64, i, u64, ctypes.POINTER(vp)]
    L.tt_rel_error_coo.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double)]
    L.tt_sketch_interface.argtypes = [vp, ctypes.POINTER(vp), i, u64, vp]
    L.tt_prox_update.argtypes = [vp, vp, vp, vp, i]
    L.tt_orthogonalize.argtypes = [vp, ctypes.POINTER(vp), i, i]
    L.tt_prox_als_sweep.argtypes = [vp, vp, vp, ctypes.POINTER(vp), i, u64, ctypes.POINTER(ctypes.c_double)]
    L.tt_rel_error.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double)]
    L.tt_prox_als_sweep_sketched.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), u64]
    L.tt_prox_als_sweep_monitored.argtypes = [vp, vp, vp, ctypes.POINTER(vp), i, u64, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]
    L.tt_prox_als_sweep_host.argtypes = [vp, vp, vp, ctypes.POINTER(vp), i, u64, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
    L.tt_prox_update_noalloc.argtypes = [vp, vp, vp, i, i, i, i, ctypes.c_double, vp]
    L.tt_prox_als_sweep_host_async.argtypes = [vp, vp, vp, ctypes.POINTER(vp), i, u64, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double)]
    L.tt_host_sync.argtypes = [vp]
    L.tt_set_workspace_limit.argtypes = [u64]
    L.tt_set_workspace_limit.restype = u64
    L.tt_profile_enable.argtypes = [vp, i]
    L.tt_profile_read.argtypes = [vp, ctypes.POINTER(TtProfile)]
    L.tt_batch_init.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(TtParams), vp]
    L.tt_batch_destroy.argtypes = [vp]
    L.tt_batch_destroy.restype = None
    L.tt_batch_last_error.argtypes = [vp]
    L.tt_batch_last_error.restype = ctypes.c_char_p
    L.tt_batch_sweep.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i, u64]
    L.tt_batch_rel_error.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(ctypes.c_double)]
    f32p, dp, ip = vp, ctypes.POINTER(ctypes.c_double), vp
    L.tt_mlp_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(TtMlpParams), vp]
    L.tt_mlp_destroy.argtypes = [vp]
    L.tt_mlp_last_error.argtypes = [vp]
    L.tt_mlp_last_error.restype = ctypes.c_char_p
    L.tt_mlp_set_weights.argtypes = [vp] + [f32p] * 6
    L.tt_mlp_get_weights.argtypes = [vp] + [f32p] * 6
    L.tt_mlp_forward.argtypes = [vp, f32p, i, ip, i, f32p, i]
    L.tt_mlp_loss_grads.argtypes = [vp, f32p, i, f32p, i, ip, i, dp] + [f32p] * 6
    L.tt_mlp_train_step.argtypes = [vp, f32p, i, f32p, i, ip, i, dp]
    L.tt_mlp_gemm_bf16.argtypes = [vp, i, vp, i, i, i, i, f32p, i, i, vp]
    L.tt_ws_summary_dim.argtypes = [vp, i]
    L.tt_ws_summary_dim.restype = ctypes.c_int64
    L.tt_ws_core_dim.argtypes = [vp]
    L.tt_ws_core_dim.restype = ctypes.c_int64
    L.tt_ws_summary.argtypes = [vp, ctypes.POINTER(vp), i, f32p, f32p]
    L.tt_canonicalize.argtypes = [vp, ctypes.POINTER(vp)]
    L.tt_ws_pack.argtypes = [vp, ctypes.POINTER(vp), f32p, f32p]
    L.tt_ws_unpack.argtypes = [vp, f32p, f32p, ctypes.POINTER(vp)]
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in _NOT_INT:
            f.restype = ctypes.c_int
    _lib = L
    return L


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _ptr_array(ts: Sequence) -> ctypes.Array:
    arr = (ctypes.c_void_p * len(ts))()
    for j, t in enumerate(ts):
        arr[j] = _ptr(t)
    return arr


def _current_stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """Owns one tt_ctx. Arguments are torch CUDA tensors (device buffers) unless stated."""

    def __init__(self, dims: Sequence[int], ranks: Sequence[int], J: int, lam: float, seed: int,
                 dtype: str = "f32", flags: int = 0, stream=None):
        self.lib = load()
        self.dims = tuple(int(x) for x in dims)
        self.ranks = tuple(int(x) for x in ranks)
        self.d = len(self.dims)
        self.J = int(J)
        self._n = (ctypes.c_int64 * self.d)(*self.dims)
        self._r = (ctypes.c_int * (self.d + 1))(*self.ranks)
        self.params = TtParams(self.d, self._n, self._r, self.J, float(lam), int(seed) & (2**64 - 1),
                               DTYPES[dtype], int(flags))
        self.ctx = ctypes.c_void_p()
        stream = _current_stream() if stream is None else stream
        rc = self.lib.tt_sketch_init(ctypes.byref(self.ctx), ctypes.byref(self.params), stream)
        if rc != TT_OK:
            raise TtError(rc, "tt_sketch_init failed (see stderr)")

    def close(self):
        if self.ctx:
            self.lib.tt_sketch_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != TT_OK:
            raise TtError(rc, self.lib.tt_last_error(self.ctx).decode())

    # -- C ABI mirrors ---------------------------------------------------------------------
    def tt_sketch_tables(self, sweep: int):
        tot = sum(self.dims)
        h = np.zeros(tot, dtype=np.int32)
        v = np.zeros(tot, dtype=np.int8)
        self._check(self.lib.tt_sketch_tables(self.ctx, int(sweep), h.ctypes.data, v.ctypes.data))
        return h, v

    def tt_sketch_set_tables(self, h: np.ndarray, v: np.ndarray):
        h = np.ascontiguousarray(h, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.int8)
        self._check(self.lib.tt_sketch_set_tables(self.ctx, h.ctypes.data, v.ctypes.data))

    def tt_sketch_unfold(self, A, k: int, sweep: int, Y: Sequence, scales=None):
        arr = _ptr_array(Y)
        self._check(self.lib.tt_sketch_unfold(self.ctx, _ptr(A), _ptr(scales), int(k), int(sweep), arr))

    def tt_sketch_unfold_coo(self, idx, val, nnz: int, k: int, sweep: int, Y: Sequence):
        """idx: device int32 (d, nnz) mode-major indices; val: device FP32 (nnz,) values."""
        arr = _ptr_array(Y)
        self._check(self.lib.tt_sketch_unfold_coo(self.ctx, _ptr(idx), _ptr(val), int(nnz), int(k), int(sweep),
                                                  arr))

    def tt_rel_error_coo(self, idx, val, nnz: int, cores: Sequence) -> float:
        out = ctypes.c_double()
        self._check(self.lib.tt_rel_error_coo(self.ctx, _ptr(idx), _ptr(val), int(nnz), _ptr_array(cores),
                                              ctypes.byref(out)))
        return out.value

    def tt_sketch_interface(self, cores: Sequence, k: int, sweep: int, SH):
        self._check(self.lib.tt_sketch_interface(self.ctx, _ptr_array(cores), int(k), int(sweep), _ptr(SH)))

    def tt_prox_update(self, Y, SH, core, k: int):
        self._check(self.lib.tt_prox_update(self.ctx, _ptr(Y), _ptr(SH), _ptr(core), int(k)))

    def tt_orthogonalize(self, cores: Sequence, direction: int, k: int = 0):
        self._check(self.lib.tt_orthogonalize(self.ctx, _ptr_array(cores), int(direction), int(k)))

    def tt_prox_als_sweep(self, A, cores: Sequence, nsweeps: int, first_sweep: int = 0, scales=None,
                          rel_change: bool = True):
        out = (ctypes.c_double * max(1, nsweeps))() if rel_change else None
        self._check(self.lib.tt_prox_als_sweep(self.ctx, _ptr(A), _ptr(scales), _ptr_array(cores),
                                               int(nsweeps), int(first_sweep), out))
        return list(out)[:nsweeps] if rel_change else None

    def tt_prox_als_sweep_monitored(self, A, cores: Sequence, nsweeps: int, first_sweep: int = 0, scales=None,
                                    rel_change: bool = False):
        """Sweeps with the relative error after each one (one synchronisation per call).
        Returns (rel_errors, rel_changes or None)."""
        err = (ctypes.c_double * max(1, nsweeps))()
        out = (ctypes.c_double * max(1, nsweeps))() if rel_change else None
        self._check(self.lib.tt_prox_als_sweep_monitored(self.ctx, _ptr(A), _ptr(scales), _ptr_array(cores),
                                                         int(nsweeps), int(first_sweep), out, err))
        return list(err)[:nsweeps], (list(out)[:nsweeps] if rel_change else None)

    def tt_prox_als_sweep_host(self, A_host: np.ndarray, cores_host: Sequence[np.ndarray], nsweeps: int,
                               first_sweep: int = 0, scales_host: Optional[np.ndarray] = None,
                               rel_change: bool = True):
        """Host-buffer variant: A_host / cores_host are (pinned) host arrays, cores updated in place."""
        out = (ctypes.c_double * max(1, nsweeps))() if rel_change else None
        err = ctypes.c_double()
        self._check(self.lib.tt_prox_als_sweep_host(self.ctx, _ptr(A_host), _ptr(scales_host),
                                                    _ptr_array(cores_host), int(nsweeps), int(first_sweep), out,
                                                    ctypes.byref(err)))
        return (list(out)[:nsweeps] if rel_change else None), err.value

    def tt_prox_als_sweep_host_async(self, A_host: np.ndarray, cores_host: Sequence[np.ndarray], nsweeps: int,
                                     first_sweep: int = 0, scales_host: Optional[np.ndarray] = None,
                                     rel_change: bool = False, rel_error: bool = True):
        """Enqueue a host-buffer call; returns the output arrays (filled by tt_host_sync). The host
        arrays must stay alive and unread until then."""
        chg = np.zeros(max(1, nsweeps)) if rel_change else None
        err = np.zeros(1) if rel_error else None
        keep = _ptr_array(cores_host)
        self._check(self.lib.tt_prox_als_sweep_host_async(
            self.ctx, _ptr(A_host), _ptr(scales_host), keep, int(nsweeps), int(first_sweep),
            chg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if chg is not None else None,
            err.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if err is not None else None))
        return chg, err

    def tt_host_sync(self):
        self._check(self.lib.tt_host_sync(self.ctx))

    def tt_profile_enable(self, on: bool = True):
        self._check(self.lib.tt_profile_enable(self.ctx, 1 if on else 0))

    def tt_profile_read(self) -> dict:
        p = TtProfile()
        self._check(self.lib.tt_profile_read(self.ctx, ctypes.byref(p)))
        return {"unfold_ms": p.unfold_ms, "unfold_launches": p.unfold_launches, "unfold_bytes": p.unfold_bytes,
                "kernel_launches": p.kernel_launches, "mode_ms": list(p.mode_ms)[:self.d],
                "mode_launches": list(p.mode_launches)[:self.d]}

    def tt_rel_error(self, A, cores: Sequence, scales=None) -> float:
        out = ctypes.c_double()
        self._check(self.lib.tt_rel_error(self.ctx, _ptr(A), _ptr(scales), _ptr_array(cores), ctypes.byref(out)))
        return out.value


def _ctx_ws_methods():
    """Warm-start entry points on a context (include/tt_warmstart.h)."""

    def tt_ws_summary_dim(self, p: int) -> int:
        return int(self.lib.tt_ws_summary_dim(self.ctx, int(p)))

    def tt_ws_core_dim(self) -> int:
        return int(self.lib.tt_ws_core_dim(self.ctx))

    def tt_ws_summary(self, Y: Sequence, p: int, x, scale):
        self._check(self.lib.tt_ws_summary(self.ctx, _ptr_array(Y), int(p), _ptr(x), _ptr(scale)))

    def tt_prox_als_sweep_sketched(self, Y: Sequence, cores: Sequence, sweep: int):
        self._check(self.lib.tt_prox_als_sweep_sketched(self.ctx, _ptr_array(Y), _ptr_array(cores), int(sweep)))

    def tt_canonicalize(self, cores: Sequence):
        self._check(self.lib.tt_canonicalize(self.ctx, _ptr_array(cores)))

    def tt_ws_pack(self, cores: Sequence, scale, y):
        self._check(self.lib.tt_ws_pack(self.ctx, _ptr_array(cores), _ptr(scale), _ptr(y)))

    def tt_ws_unpack(self, y, scale, cores: Sequence):
        self._check(self.lib.tt_ws_unpack(self.ctx, _ptr(y), _ptr(scale), _ptr_array(cores)))

    for f in (tt_ws_summary_dim, tt_ws_core_dim, tt_ws_summary, tt_prox_als_sweep_sketched, tt_canonicalize,
              tt_ws_pack, tt_ws_unpack):
        setattr(Context, f.__name__, f)


_ctx_ws_methods()


class Mlp:
    """Owns one tt_mlp (the warm-start network). Matrices are torch CUDA tensors, row-major FP32."""

    def __init__(self, in_dim: int, hidden: int, out_dim: int, batch_max: int, lr: float = 1e-3,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
        self.lib = load()
        self.in_dim, self.hidden, self.out_dim, self.batch_max = in_dim, hidden, out_dim, batch_max
        p = TtMlpParams(in_dim, hidden, out_dim, batch_max, lr, beta1, beta2, eps)
        self.m = ctypes.c_void_p()
        stream = _current_stream() if stream is None else stream
        rc = self.lib.tt_mlp_init(ctypes.byref(self.m), ctypes.byref(p), stream)
        if rc != TT_OK:
            raise TtError(rc, "tt_mlp_init failed (see stderr)")

    def close(self):
        if self.m:
            self.lib.tt_mlp_destroy(self.m)
            self.m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != TT_OK:
            raise TtError(rc, self.lib.tt_mlp_last_error(self.m).decode())

    def tt_mlp_set_weights(self, W1, b1, W2, b2, W3, b3):
        self._check(self.lib.tt_mlp_set_weights(self.m, *[_ptr(t) for t in (W1, b1, W2, b2, W3, b3)]))

    def tt_mlp_get_weights(self, W1, b1, W2, b2, W3, b3):
        self._check(self.lib.tt_mlp_get_weights(self.m, *[_ptr(t) for t in (W1, b1, W2, b2, W3, b3)]))

    def tt_mlp_forward(self, X, batch: int, Y, rows=None, ldx: Optional[int] = None, ldy: Optional[int] = None):
        self._check(self.lib.tt_mlp_forward(self.m, _ptr(X), int(ldx or self.in_dim), _ptr(rows), int(batch),
                                            _ptr(Y), int(ldy or self.out_dim)))

    def tt_mlp_loss_grads(self, X, T, batch: int, grads=None, rows=None, ldx=None, ldt=None) -> float:
        loss = ctypes.c_double(0.0)
        g = [_ptr(t) for t in grads] if grads is not None else [None] * 6
        self._check(self.lib.tt_mlp_loss_grads(self.m, _ptr(X), int(ldx or self.in_dim), _ptr(T),
                                               int(ldt or self.out_dim), _ptr(rows), int(batch),
                                               ctypes.byref(loss), *g))
        return loss.value

    def tt_mlp_train_step(self, X, T, batch: int, rows=None, ldx=None, ldt=None, want_loss: bool = False):
        loss = ctypes.c_double(0.0)
        self._check(self.lib.tt_mlp_train_step(self.m, _ptr(X), int(ldx or self.in_dim), _ptr(T),
                                               int(ldt or self.out_dim), _ptr(rows), int(batch),
                                               ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None


def tt_mlp_gemm_bf16(A, B, C, M: int, N: int, K: int, lda: int, ldb: int, ldc: int, check: bool = True,
                     stream=None) -> int:
    """C = A B^T on BF16 row-major device tensors (torch.bfloat16 or int16 views); returns the status."""
    L = load()
    stream = _current_stream() if stream is None else stream
    return L.tt_mlp_gemm_bf16(_ptr(A), int(lda), _ptr(B), int(ldb), int(M), int(N), int(K), _ptr(C), int(ldc),
                              1 if check else 0, stream)


def tt_set_workspace_limit(nbytes: int) -> int:
    """Process-wide cap on a context's device workspaces (0 = none); returns the previous cap."""
    return int(load().tt_set_workspace_limit(int(nbytes)))


def tt_prox_update_noalloc(Y, SH, core, J: int, n: int, r0: int, r1: int, sigma: float, stream=None) -> int:
    """Context-free proximal update that allocates no device memory (see tt_sketch.h).

    For callers that cannot allocate device memory; returns the TT_* status code."""
    L = load()
    stream = _current_stream() if stream is None else stream
    return L.tt_prox_update_noalloc(_ptr(Y), _ptr(SH), _ptr(core), int(J), int(n), int(r0), int(r1),
                                    float(sigma), stream)


class Batch:
    """Owns one tt_batch: many tensors, each given as a dict(dims, ranks, J, lam, seed, dtype)."""

    def __init__(self, specs: Sequence[dict], stream=None):
        self.lib = load()
        self.specs = list(specs)
        self.count = len(self.specs)
        self._keep = []
        params = (TtParams * self.count)()
        for i, sp in enumerate(self.specs):
            d = len(sp["dims"])
            n = (ctypes.c_int64 * d)(*[int(x) for x in sp["dims"]])
            r = (ctypes.c_int * (d + 1))(*[int(x) for x in sp["ranks"]])
            self._keep += [n, r]
            params[i] = TtParams(d, n, r, int(sp["J"]), float(sp["lam"]), int(sp["seed"]) & (2**64 - 1),
                                 DTYPES[sp.get("dtype", "f32")], int(sp.get("flags", 0)))
        self._params = params
        self.b = ctypes.c_void_p()
        stream = _current_stream() if stream is None else stream
        rc = self.lib.tt_batch_init(ctypes.byref(self.b), self.count, params, stream)
        if rc != TT_OK:
            raise TtError(rc, "tt_batch_init failed (see stderr)")

    def close(self):
        if self.b:
            self.lib.tt_batch_destroy(self.b)
            self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arrays(self, A_list, cores_list, scales_list):
        A = _ptr_array(A_list)
        S = _ptr_array(scales_list) if scales_list is not None else None
        inner = [_ptr_array(c) for c in cores_list]
        C = (ctypes.c_void_p * self.count)()
        for i, arr in enumerate(inner):
            C[i] = ctypes.cast(arr, ctypes.c_void_p)
        return A, S, C, inner

    def tt_batch_sweep(self, A_list, cores_list, nsweeps: int, first_sweep: int = 0, scales_list=None):
        A, S, C, inner = self._arrays(A_list, cores_list, scales_list)
        rc = self.lib.tt_batch_sweep(self.b, A, S, C, int(nsweeps), int(first_sweep))
        if rc != TT_OK:
            raise TtError(rc, self.lib.tt_batch_last_error(self.b).decode())

    def tt_batch_rel_error(self, A_list, cores_list, scales_list=None):
        A, S, C, inner = self._arrays(A_list, cores_list, scales_list)
        out = (ctypes.c_double * self.count)()
        rc = self.lib.tt_batch_rel_error(self.b, A, S, C, out)
        if rc != TT_OK:
            raise TtError(rc, self.lib.tt_batch_last_error(self.b).decode())
        return list(out)


# ---------------------------------------------------------------------------------------------
# helpers to move synthetic inputs to the device in the ABI's layouts

def device_tensor(storage: np.ndarray, dtype: str, device="cuda"):
    """Flat storage array (memory order) -> torch CUDA tensor holding the same bytes."""
    import torch

    if dtype == "f64":
        t = torch.from_numpy(np.ascontiguousarray(storage, dtype=np.float64))
    elif dtype == "f32":
        t = torch.from_numpy(np.ascontiguousarray(storage, dtype=np.float32))
    elif dtype == "bf16":
        t = torch.from_numpy(np.ascontiguousarray(storage, dtype=np.uint16).view(np.int16)).view(torch.bfloat16)
    elif dtype == "fp8":
        t = torch.from_numpy(np.ascontiguousarray(storage, dtype=np.uint8))
    else:
        raise ValueError(dtype)
    return t.to(device)


def device_cores(cores: Sequence[np.ndarray], device="cuda") -> List:
    """FP32 device copies of TT cores in the ABI layout (r_{k-1} fastest)."""
    import torch

    return [torch.from_numpy(np.ascontiguousarray(np.asarray(g, dtype=np.float32).ravel(order="F"))).to(device)
            for g in cores]


def host_cores(dev_cores: Sequence, ranks: Sequence[int], dims: Sequence[int]) -> List[np.ndarray]:
    out = []
    for k, t in enumerate(dev_cores):
        a = t.detach().cpu().numpy().astype(np.float64)
        out.append(a.reshape(ranks[k], dims[k], ranks[k + 1], order="F"))
    return out
