"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the CPU oracle.

This module holds no arithmetic of the sketched ALS method itself: it only draws random
TT cores, contracts them into a dense tensor (the data model of Sec. 2.1, used here purely
to manufacture test tensors), adds Gaussian noise and encodes the result in the storage
formats the library reads (FP64, FP32, BF16, FP8-E4M3 with one scale per mode-1 slice).

All arrays follow the paper's column-major conventions (Sec. 1.2): a tensor of shape
(n_1, ..., n_d) is stored with the first index fastest, a TT core G_k of shape
(r_{k-1}, n_k, r_k) with r_{k-1} fastest. Numpy arrays returned here are Fortran-ordered
so that ``a.ravel(order="F")`` is the memory image handed to the library.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Sub-stream identifiers for np.random.default_rng([base_seed, stream]).
STREAM_CORES = 1
STREAM_NOISE = 2
STREAM_INIT = 3
STREAM_SKETCH = 4


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic problem: a noisy low-TT-rank tensor and the method's parameters."""

    name: str
    dims: Tuple[int, ...]
    ranks: Tuple[int, ...]  # r_0 .. r_d with r_0 = r_d = 1
    J: int  # sketch size m of the paper
    lam: float  # proximal weight sigma
    sweeps: int
    noise: float  # relative Frobenius noise level
    storage: str  # "f64", "f32", "bf16", "fp8"
    core_kind: str  # "normal", "decay", "cumsum"
    seed: int

    @property
    def d(self) -> int:
        return len(self.dims)

    @property
    def numel(self) -> int:
        return int(np.prod(self.dims, dtype=np.int64))

    def sketch_seed(self) -> int:
        """64-bit seed of the per-sweep hash/sign draws (a plain integer input)."""
        rng = np.random.default_rng([self.seed, STREAM_SKETCH])
        return int(rng.integers(0, 2**63 - 1, dtype=np.int64))

    def scaled(self, dims: Sequence[int], J: Optional[int] = None, name: Optional[str] = None) -> "Workload":
        """Same recipe on smaller mode sizes (ranks are capped where a mode gets too small)."""
        return dataclasses.replace(self, dims=tuple(int(x) for x in dims), J=int(J or self.J),
                                   name=name or f"{self.name}-scaled")


# The five synthetic workloads (sizes, ranks, sketch sizes and noise levels as specified for
# the benchmark; they stand in for the paper's Sec. 5 experiments, whose datasets are absent).
WORKLOADS = {
    "order3-50-r5": Workload("order3-50-r5", (50, 50, 50), (1, 5, 5, 1), 1024, 1e-3, 10, 1e-3,
                             "f64", "normal", 20230916),
    "order4-100-r10": Workload("order4-100-r10", (100, 100, 100, 100), (1, 10, 10, 10, 1), 4096,
                               1e-3, 20, 1e-2, "f32", "normal", 20230917),
    "order5-40-r8": Workload("order5-40-r8", (40, 40, 40, 40, 40), (1, 8, 8, 8, 8, 1), 8192,
                             1e-3, 10, 1e-3, "bf16", "decay", 20230918),
    "order4-256x256x3x128-r20": Workload("order4-256x256x3x128-r20", (256, 256, 3, 128),
                                         (1, 20, 3, 20, 1), 2048, 1e-3, 20, 1e-2, "f32", "cumsum",
                                         20230920),
}


def _haar_orthonormal(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    """m x n matrix with Haar-distributed orthonormal columns (m >= n)."""
    g = rng.standard_normal((m, n))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s


def random_cores(dims: Sequence[int], ranks: Sequence[int], rng: np.random.Generator,
                 kind: str = "normal") -> List[np.ndarray]:
    """Random TT cores G_k of shape (r_{k-1}, n_k, r_k), Fortran-ordered float64."""
    d = len(dims)
    assert len(ranks) == d + 1 and ranks[0] == 1 and ranks[-1] == 1
    cores = []
    for k in range(d):
        r0, n, r1 = ranks[k], dims[k], ranks[k + 1]
        if kind == "normal":
            g = rng.standard_normal((r0, n, r1))
        elif kind == "cumsum":
            g = np.cumsum(rng.standard_normal((r0, n, r1)), axis=1)
        elif kind == "decay":
            # left unfolding (right unfolding for the last core) = U diag(0.8^j) V^T
            if k < d - 1:
                m, c = r0 * n, r1
            else:
                m, c = n * r1, r0
            q = min(m, c)
            u = _haar_orthonormal(rng, m, q)
            v = _haar_orthonormal(rng, c, q)
            mat = (u * (0.8 ** np.arange(q))) @ v.T  # m x c
            if k < d - 1:
                g = mat.reshape(r0, n, r1, order="F")
            else:
                g = mat.T.reshape(r0, n, r1, order="F")
        else:
            raise ValueError(kind)
        cores.append(np.asfortranarray(g))
    return cores


def contract_cores(cores: Sequence[np.ndarray]) -> np.ndarray:
    """Dense tensor [[G_1, ..., G_d]] (Sec. 2.1) as a Fortran-ordered float64 array.

    Used only to manufacture test tensors; the library never forms it.
    """
    dims = [g.shape[1] for g in cores]
    t = np.asarray(cores[0], dtype=np.float64).reshape(dims[0], cores[0].shape[2], order="F")
    rows = dims[0]
    for g in cores[1:]:
        r0, n, r1 = g.shape
        gr = np.asarray(g, dtype=np.float64).reshape(r0, n * r1, order="F")
        t = (t @ gr).reshape(rows * n, r1, order="F")
        rows *= n
    return t.reshape(dims, order="F")


def add_noise(t: np.ndarray, eta: float, rng: np.random.Generator) -> np.ndarray:
    """A = T + eta * ||T||_F * E / ||E||_F with E ~ N(0, 1) entrywise."""
    if eta == 0.0:
        return np.asfortranarray(t)
    e = rng.standard_normal(t.shape)
    out = t + (eta * np.linalg.norm(t.ravel()) / np.linalg.norm(e.ravel())) * e
    return np.asfortranarray(out)


# ---------------------------------------------------------------------------------------------
# storage formats

def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest, ties to even); returns uint16 bits."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))
    return ((b + bias) >> np.uint64(16)).astype(np.uint16)


def bf16_to_f64(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def _e4m3_table() -> np.ndarray:
    """Values of the 128 non-negative OCP FP8-E4M3 codes (code 0x7F is NaN -> inf here)."""
    vals = np.empty(128, dtype=np.float64)
    for c in range(128):
        e, m = c >> 3, c & 7
        if e == 0:
            vals[c] = (m / 8.0) * 2.0 ** -6
        else:
            vals[c] = (1.0 + m / 8.0) * 2.0 ** (e - 7)
    vals[127] = np.inf  # S.1111.111 is NaN; never produced
    return vals


E4M3_MAX = 448.0


def fp8_e4m3_encode(x: np.ndarray) -> np.ndarray:
    """Encode (already scaled, |x| <= 448) values as E4M3 bytes, nearest with ties to even."""
    table = _e4m3_table()[:127]  # finite magnitudes, increasing
    ax = np.minimum(np.abs(np.asarray(x, dtype=np.float64)), E4M3_MAX)
    hi = np.clip(np.searchsorted(table, ax, side="left"), 0, 126)
    lo = np.clip(hi - 1, 0, 126)
    dlo = ax - table[lo]
    dhi = table[hi] - ax
    pick_hi = (dhi < dlo) | ((dhi == dlo) & ((hi & 1) == 0))
    code = np.where(pick_hi, hi, lo).astype(np.uint8)
    sign = (np.signbit(np.asarray(x, dtype=np.float64)) & (code != 0)).astype(np.uint8) << 7
    return (code | sign).astype(np.uint8)


def fp8_e4m3_decode(codes: np.ndarray) -> np.ndarray:
    table = _e4m3_table()
    c = np.asarray(codes, dtype=np.uint8)
    mag = table[c & 0x7F]
    return np.where(c & 0x80, -mag, mag)


def quantize(a: np.ndarray, storage: str):
    """Encode a Fortran-ordered float64 tensor for the library.

    Returns (flat storage array in memory order, slice scales or None, exact decoded values as a
    Fortran-ordered float64 tensor). FP8 uses one FP32 scale per mode-1 slice
    (scale[i_1] = max |A(i_1, :, ..., :)| / 448).
    """
    flat = a.ravel(order="F")
    if storage == "f64":
        return flat.astype(np.float64), None, np.asfortranarray(a, dtype=np.float64)
    if storage == "f32":
        f = flat.astype(np.float32)
        return f, None, f.astype(np.float64).reshape(a.shape, order="F")
    if storage == "bf16":
        b = bf16_bits(flat)
        return b, None, bf16_to_f64(b).reshape(a.shape, order="F")
    if storage == "fp8":
        n1 = a.shape[0]
        amax = np.abs(a.reshape(n1, -1, order="F")).max(axis=1)
        scales = np.where(amax > 0, amax / E4M3_MAX, 1.0).astype(np.float32)
        scaled = (a.reshape(n1, -1, order="F") / scales.astype(np.float64)[:, None])
        codes = fp8_e4m3_encode(scaled)  # (n1, rest)
        dec = fp8_e4m3_decode(codes) * scales.astype(np.float64)[:, None]
        return (codes.ravel(order="F"), scales,
                np.asfortranarray(dec.reshape(a.shape, order="F")))
    raise ValueError(storage)


@dataclasses.dataclass
class Problem:
    workload: Workload
    ranks: Tuple[int, ...]  # ranks actually used (capped for scaled-down shapes)
    tensor: np.ndarray  # exact float64 values the library sees (decoded storage), Fortran order
    storage: np.ndarray  # flat memory image in the storage dtype
    scales: Optional[np.ndarray]
    true_cores: List[np.ndarray]
    init_cores: List[np.ndarray]
    sketch_seed: int


def make_problem(w: Workload, storage: Optional[str] = None) -> Problem:
    """Build the seeded noisy tensor and the seeded N(0,1) initial cores of a workload."""
    storage = storage or w.storage
    ranks = list(w.ranks)
    for k in range(1, w.d):  # cap ranks that exceed an unfolding (scaled-down variants)
        ranks[k] = min(ranks[k], int(np.prod(w.dims[:k])), int(np.prod(w.dims[k:])))
    rng_c = np.random.default_rng([w.seed, STREAM_CORES])
    true_cores = random_cores(w.dims, ranks, rng_c, w.core_kind)
    t = contract_cores(true_cores)
    a = add_noise(t, w.noise, np.random.default_rng([w.seed, STREAM_NOISE]))
    flat, scales, exact = quantize(a, storage)
    init = random_cores(w.dims, ranks, np.random.default_rng([w.seed, STREAM_INIT]), "normal")
    return Problem(w, tuple(ranks), exact, flat, scales, true_cores, init, w.sketch_seed())


def random_tensor(dims: Sequence[int], seed: int) -> np.ndarray:
    """Plain N(0,1) dense tensor (Fortran order), for shape/edge-case tests."""
    return np.asfortranarray(np.random.default_rng([seed, 0]).standard_normal(tuple(dims)))


def random_tt(dims: Sequence[int], ranks: Sequence[int], seed: int, kind: str = "normal"):
    return random_cores(dims, ranks, np.random.default_rng([seed, STREAM_CORES]), kind)


# ---------------------------------------------------------------------------------------------
# batched workload: 256 tensors of order 3-4, mode sizes in [16, 128], TT ranks in [4, 12],
# 1e-3 relative noise, J = next power of two >= 8 max_k r_{k-1} r_k; storage alternates FP32 / BF16

def batched_specs(count: int = 256, seed: int = 20230919, dims_range=(16, 128), rank_range=(4, 12),
                  storages=("f32", "bf16")):
    """Shapes, ranks and sketch sizes of the batched workload (numpy RNG, fully determined by seed)."""
    rng = np.random.default_rng([seed, 5])
    specs = []
    for i in range(count):
        d = int(rng.integers(3, 5))
        dims = [int(x) for x in rng.integers(dims_range[0], dims_range[1] + 1, size=d)]
        ranks = [1] + [int(x) for x in rng.integers(rank_range[0], rank_range[1] + 1, size=d - 1)] + [1]
        for k in range(1, d):
            ranks[k] = min(ranks[k], int(np.prod(dims[:k])), int(np.prod(dims[k:])))
        smax = max(ranks[k] * ranks[k + 1] for k in range(d))
        J = 1
        while J < 8 * smax:
            J *= 2
        specs.append({"dims": dims, "ranks": ranks, "J": J, "lam": 1e-3, "noise": 1e-3,
                      "seed": int(rng.integers(0, 2**62)), "dtype": storages[i % len(storages)],
                      "tensor_seed": int(seed * 1000 + i)})
    return specs


def batched_tensor_cpu(spec):
    """Noisy tensor of one batched spec on the host (numpy, for small test batches)."""
    cores = random_tt(spec["dims"], spec["ranks"], spec["tensor_seed"])
    a = add_noise(contract_cores(cores), spec["noise"], np.random.default_rng([spec["tensor_seed"], STREAM_NOISE]))
    init = random_cores(spec["dims"], spec["ranks"], np.random.default_rng([spec["tensor_seed"], STREAM_INIT]))
    return a, init


def batched_tensor_gpu(spec, device="cuda"):
    """The same recipe generated on the device with torch (large batches): seeded numpy cores,
    TT contraction in FP32 (TF32 disabled) and torch-generated Gaussian noise. Returns the flat
    device tensor in memory order (mode 0 fastest) in the spec's storage type (BF16 by round to
    nearest even from FP32) and the initial cores (numpy)."""
    import torch

    torch.backends.cuda.matmul.allow_tf32 = False
    cores = random_tt(spec["dims"], spec["ranks"], spec["tensor_seed"])
    q = None  # Q[beta, i] with i = linear index of the modes so far (first fastest)
    for g in cores:
        gt = torch.as_tensor(np.ascontiguousarray(g), dtype=torch.float32, device=device)
        if q is None:
            q = gt[0].transpose(0, 1).contiguous()  # (r1, n0)
        else:
            q = torch.einsum("aib,ax->bix", gt, q).reshape(gt.shape[2], -1)
    t = q.reshape(-1)
    gen = torch.Generator(device=device)
    gen.manual_seed(spec["tensor_seed"])
    e = torch.randn(t.numel(), generator=gen, device=device, dtype=torch.float32)
    a = t + (spec["noise"] * torch.linalg.vector_norm(t) / torch.linalg.vector_norm(e)) * e
    if spec["dtype"] == "bf16":
        a = a.to(torch.bfloat16)
    elif spec["dtype"] != "f32":
        raise ValueError("device generation covers f32 and bf16 storage")
    init = random_cores(spec["dims"], spec["ranks"], np.random.default_rng([spec["tensor_seed"], STREAM_INIT]))
    return a, init


# ---------------------------------------------------------------------------------------------
# learned warm start: a family of order-4 tensors with smooth (cumulative-sum) TT cores and 1%
# noise, one member per seed; plus the seeded initial weights of the network

def warmstart_spec(dims=(256, 256, 3, 128), ranks=(1, 20, 3, 20, 1), J=2048, lam=1e-3, noise=1e-2):
    return {"dims": list(dims), "ranks": list(ranks), "J": J, "lam": lam, "noise": noise, "dtype": "f32"}


def warmstart_tensor_gpu(spec, tensor_seed: int, device="cuda"):
    """One member of the family on the device: seeded cumsum cores (numpy), their FP32 TT
    contraction (TF32 off), Gaussian noise at spec['noise'] relative Frobenius norm (torch,
    seeded). Returns (A, T, init) with A the noisy and T the noise-free flat FP32 tensor (mode 0
    fastest) and init the seeded N(0,1) random initial cores (numpy)."""
    import torch

    torch.backends.cuda.matmul.allow_tf32 = False
    dims, ranks = spec["dims"], spec["ranks"]
    cores = random_cores(dims, ranks, np.random.default_rng([tensor_seed, STREAM_CORES]), "cumsum")
    q = None
    for g in cores:
        gt = torch.as_tensor(np.ascontiguousarray(g), dtype=torch.float32, device=device)
        q = gt[0].transpose(0, 1).contiguous() if q is None else torch.einsum("aib,ax->bix", gt, q).reshape(gt.shape[2], -1)
    t = q.reshape(-1)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(tensor_seed) & (2**63 - 1))
    e = torch.randn(t.numel(), generator=gen, device=device, dtype=torch.float32)
    a = t + (spec["noise"] * torch.linalg.vector_norm(t) / torch.linalg.vector_norm(e)) * e
    init = random_cores(dims, ranks, np.random.default_rng([tensor_seed, STREAM_INIT]), "normal")
    return a, t, init


def mlp_init(in_dim: int, hidden: int, out_dim: int, seed: int):
    """Seeded initial weights of the in -> hidden -> hidden -> out network (numpy FP32, row-major):
    hidden layers N(0, 2 / fan_in) (He et al., 2015), output layer N(0, 1 / fan_in), zero biases."""
    rng = np.random.default_rng([seed, 11])
    f32 = np.float32
    W1 = (rng.standard_normal((hidden, in_dim)) * np.sqrt(2.0 / in_dim)).astype(f32)
    W2 = (rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden)).astype(f32)
    W3 = (rng.standard_normal((out_dim, hidden)) * np.sqrt(1.0 / hidden)).astype(f32)
    return [W1, np.zeros(hidden, f32), W2, np.zeros(hidden, f32), W3, np.zeros(out_dim, f32)]


# ---------------------------------------------------------------------------------------------
# the paper's synthetic experiments (Sec. 5), formula-generated

def paper_tt_tensor(sd: float, seed: int, dims=(10,) * 6, rank: int = 5):
    """First synthetic experiment: a sixth-order 10 x ... x 10 tensor in TT format with equal
    ranks and N(0,1) core entries, plus Gaussian noise of standard deviation sd (absolute).
    Returns the noisy tensor (Fortran order, float64)."""
    ranks = (1,) + (rank,) * (len(dims) - 1) + (1,)
    t = contract_cores(random_tt(dims, ranks, seed))
    return t + sd * np.random.default_rng([seed, STREAM_NOISE]).standard_normal(t.shape)


def paper_function_tensor(name: str, dims=(10,) * 6):
    """Second experiment: a one-dimensional function sampled at prod(dims) equispaced points and
    reshaped column-major (first index fastest) into a tensor: 'sinc' = sin(pi x)/(pi x) on
    [-5, 5] (the normalised sinc of the MATLAB the paper used, numpy's sinc), 'osc' =
    sin(4/x) cos(x^2) on [0, 1] (first point excluded: x > 0)."""
    npts = int(np.prod(dims))
    if name == "sinc":
        x = np.linspace(-5.0, 5.0, npts)
        y = np.sinc(x)
    elif name == "osc":
        x = np.linspace(0.0, 1.0, npts + 1)[1:]
        y = np.sin(4.0 / x) * np.cos(x * x)
    else:
        raise ValueError(name)
    return y.reshape(dims, order="F")
