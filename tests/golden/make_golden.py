"""Writes oracle reference values for the GPU parity tests at full size.

Calls only the CPU oracle (``oracle/``) on inputs from ``synth``; nothing here
touches the CUDA path.  Stored per ADC order: the 4 lowest Davidson roots and
their residual norms, the 1p/1p block, and sigma of two seeded probe vectors
sampled at the full 1p part plus 4096 fixed 2p1h positions.  Run from the
repository root (about half an hour of CPU):
    python tests/golden/make_golden.py canonical-200
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from synth import config_problem, normal01, uniform53  # noqa: E402
from oracle import restricted as R  # noqa: E402
from oracle.davidson import davidson  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))


def probes(dim, v, nsample=4096):
    """Seeded probe vectors and sample positions (same recipe in the GPU test)."""
    x = normal01(99, 7, 0, 2 * dim).reshape(2, dim)
    pos = v + np.unique((uniform53(99, 8, 0, 2 * nsample) * (dim - v)).astype(np.int64))[:nsample]
    return x, np.concatenate([np.arange(v), pos])


def canonical(name, nroots, tol=1e-8):
    t0 = time.time()
    pr = config_problem(name)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    dim = p.v + p.o * p.v * p.v
    x, idx = probes(dim, p.v)
    res = {"sample_index": idx}
    for order in (2, 3):
        sig = R.Sigma(p, order)
        res[f"m11_{order}"] = sig.M11
        res[f"sigma_probe{order}"] = sig(x)[:, idx]
        th, X, rn, it = davidson(sig, sig.diagonal(), nroots, tol=tol, max_sub=max(8 * nroots, 40))
        res[f"omega{order}"] = th
        res[f"resnorm{order}"] = rn
        print(name, "order", order, "roots", th, "iters", it, "resnorm", rn, f"{time.time() - t0:.0f}s", flush=True)
    np.savez_compressed(os.path.join(OUT, f"{name}.npz"), **res)


if __name__ == "__main__":
    name = sys.argv[1] if len(sys.argv) > 1 else "canonical-200"
    canonical(name, 4)
