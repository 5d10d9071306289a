"""Writes oracle reference values for the GPU parity tests.

Calls only the CPU oracle (``oracle/``) on inputs from ``synth``; nothing here
touches the CUDA path.  Run from the repository root:
    python tests/golden/make_golden.py canonical-200
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from synth import config_problem  # noqa: E402
from oracle import restricted as R  # noqa: E402
from oracle.davidson import davidson  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))


def canonical(name, nroots, tol=1e-8):
    t0 = time.time()
    pr = config_problem(name)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    res = {}
    for order in (2, 3):
        sig = R.Sigma(p, order)
        th, X, rn, it = davidson(sig, sig.diagonal(), nroots, tol=tol, max_sub=max(8 * nroots, 40))
        res[f"omega{order}"] = th
        res[f"resnorm{order}"] = rn
        res[f"m11_{order}"] = sig.M11
        # sigma of a fixed probe vector (first Ritz vector) for elementwise checks
        res[f"probe{order}"] = X[:, 0]
        res[f"sigma_probe{order}"] = sig(X[:, 0])
        print(name, "order", order, "roots", th, "iters", it, "resnorm", rn, f"{time.time() - t0:.0f}s", flush=True)
    np.savez_compressed(os.path.join(OUT, f"{name}.npz"), **res)


if __name__ == "__main__":
    name = sys.argv[1] if len(sys.argv) > 1 else "canonical-200"
    canonical(name, {"tiny": 4, "canonical-200": 4}[name])
