"""Counter-based synthetic problem generator (SplitMix64 -> Box-Muller).

Recipe (the same for every workload; sizes from the workload table below):

* occupied orbital energies: iid uniform on [-1.2, -0.4] Eh, sorted ascending;
* virtual orbital energies: geometric spacing from 0.02 to 20 Eh inclusive;
* density-fitting factor B[Q, p, q] over all n = o + v orbitals, symmetric in
  (p, q): the packed upper triangle (p <= q) holds iid N(0, 1) draws, the
  diagonal is multiplied by sqrt(2) (so B has the law of (G + G^T)/sqrt(2)
  for G iid N(0, 1)), and every auxiliary slice Q (0-based) is damped by
  exp(-Q / decay);
* a global scale s on B fixes the largest restricted first-order amplitude
  |(ia|jb) / (e_i + e_j - e_a - e_b)| to 0.05 (amplitudes scale as s^2).

The random numbers are SplitMix64 outputs (Steele, Lea and Flood, 2014) taken
as a counter-indexed sequence, turned into uniforms on (0, 1) from their top
53 bits and into normals by the Box-Muller transform.  Everything here is
input preparation: no EA-ADC term is evaluated.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM = np.uint64(0x632BE59BD9B4E019)

# name -> (o, v, naux, decay, seed)
CONFIGS = {
    "tiny": (5, 20, 60, 15.0, 1),          # 2020-dimensional secular matrix
    "canonical-200": (20, 200, 600, 150.0, 1),
    "fno-batch-400": (30, 400, 1200, 300.0, 1),
    "large-1250": (60, 1250, 3600, 900.0, 1),
    "learned-600": (40, 600, 1800, 450.0, 1),
}


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 sequence of (seed, stream)."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([seed], dtype=np.uint64) + np.uint64(stream) * _STREAM)[0]
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(key + idx * _GOLDEN)


def uniform53(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    z = splitmix64(seed, stream, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def normal01(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """count standard normals; draw k uses uniforms 2k and 2k+1 of the stream."""
    u = uniform53(seed, stream, 2 * start, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _max_amplitude(Bov: np.ndarray, eo: np.ndarray, ev: np.ndarray, block: int = 4096) -> float:
    """max |(ia|jb)| / |e_i + e_j - e_a - e_b| over all i, j, a, b (exact, blocked)."""
    naux, o, v = Bov.shape
    M = Bov.reshape(naux, o * v)
    dia = (eo[:, None] - ev[None, :]).reshape(-1)
    best = 0.0
    for s in range(0, o * v, block):
        e = min(o * v, s + block)
        G = M.T @ M[:, s:e]
        D = dia[:, None] + dia[None, s:e]
        best = max(best, float(np.max(np.abs(G / D))))
    return best


def make_problem(o: int, v: int, naux: int, decay: float, seed: int, tmax: float = 0.05):
    """Returns dict(eps_occ[o], eps_vir[v], B[naux, n, n]) in float64."""
    n = o + v
    eo = np.sort(-1.2 + 0.8 * uniform53(seed, 0, 0, o))
    ev = np.geomspace(0.02, 20.0, v) if v > 1 else np.array([0.02])
    iu = np.triu_indices(n)
    npk = iu[0].size
    B = np.empty((naux, n, n))
    for Q in range(naux):
        z = normal01(seed, 1, Q * npk, npk)
        z[iu[0] == iu[1]] *= np.sqrt(2.0)
        S = np.zeros((n, n))
        S[iu] = z
        S = S + np.triu(S, 1).T
        B[Q] = S * np.exp(-Q / decay)
    tm = _max_amplitude(B[:, :o, o:], eo, ev)
    B *= np.sqrt(tmax / tm)
    return {"eps_occ": eo, "eps_vir": ev, "B": B, "o": o, "v": v, "naux": naux}


def config_problem(name: str, seed: int | None = None):
    o, v, naux, decay, s0 = CONFIGS[name]
    return make_problem(o, v, naux, decay, s0 if seed is None else seed)
