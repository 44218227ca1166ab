"""Oracle runs that the full-size GPU tests start in spawned worker processes, so that several
long CPU trajectories proceed side by side while the GPU work runs. Imports no GPU code.

Test infrastructure: calls only the oracle and the seeded input generators."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for _p in (ROOT, os.path.join(ROOT, "oracle")):
    if _p not in sys.path:
        sys.path.insert(0, _p)


def order5_trajectory(storage: str, nsweeps: int):
    """Algorithm 1 for `nsweeps` sweeps of the oracle on the order-5 40^5 workload, the tensor
    decoded from `storage` ("f64" = unquantised). Returns (cores, relative error against the
    decoded tensor, relative error against the FP64 tensor)."""
    import numpy as np

    import tt_oracle as O
    from paper_2309_08093_gb300 import synth

    w = synth.WORKLOADS["order5-40-r8"]
    p = synth.make_problem(w, storage="f64")
    a64 = p.tensor
    if storage == "f64":
        a = a64
    else:
        _, _, a = synth.quantize(a64, storage)
    cores, _ = O.tt_ts(a, p.init_cores, p.sketch_seed, w.J, w.lam, nsweeps)
    cores = [np.ascontiguousarray(g) for g in cores]
    return cores, O.rel_error(a, cores), O.rel_error(a64, cores)
