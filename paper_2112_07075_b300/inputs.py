"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the oracle.

This module holds none of the hydrodynamics method's arithmetic: it only produces
vertex coordinates of structured box meshes (optionally jittered) and seeded random
arrays. Everything the method computes from these inputs (node positions, bases,
quadrature, operators) is implemented separately by each side.

Random numbers come from one counter-based generator defined here: the splitmix64
output finalizer (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to a key/counter combination, giving a 53-bit
uniform double per (seed, counter).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_KEY_MUL = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1), one per counter, from (seed, counter)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) * _KEY_MUL + (c + np.uint64(1)) * _GOLDEN
        z = _mix64(z)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform array in [lo, hi) of the given shape (C order counters)."""
    n = int(np.prod(shape)) if len(shape) else 1
    u = uniform01(seed, np.arange(n, dtype=np.uint64))
    return (lo + (hi - lo) * u).reshape(shape)


def box_vertices(dim: int, n: int, lo: float = 0.0, hi: float = 1.0,
                 jitter: float = 0.0, seed: int = 0) -> np.ndarray:
    """Vertices of an n^dim structured box mesh, shape [(n+1)^dim, dim].

    Vertex (i0, i1[, i2]) has flat index i0 + (n+1)*(i1 + (n+1)*i2) (first axis
    fastest). With jitter j > 0 every interior coordinate is moved by
    U(-j*h, j*h), h = (hi-lo)/n, drawn from uniform01(seed, 3*vertex + axis);
    boundary vertices keep their coordinate normal to the face they lie on, and
    also stay put along the face so the box keeps its straight faces.
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    if n < 1:
        raise ValueError("n must be >= 1")
    h = (hi - lo) / n
    g = lo + h * np.arange(n + 1, dtype=np.float64)
    g[-1] = hi
    if dim == 2:
        iy, ix = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
        idx = [ix.ravel(), iy.ravel()]
    else:
        iz, iy, ix = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
        idx = [ix.ravel(), iy.ravel(), iz.ravel()]
    V = np.stack([g[i] for i in idx], axis=1)
    if jitter > 0.0:
        nv = V.shape[0]
        interior = np.ones(nv, dtype=bool)
        for i in idx:
            interior &= (i > 0) & (i < n)
        ctr = (3 * np.arange(nv, dtype=np.uint64)[:, None] + np.arange(dim, dtype=np.uint64)[None, :])
        u = uniform01(seed, ctr.ravel()).reshape(nv, dim)
        V[interior] += (2.0 * u[interior] - 1.0) * jitter * h
    return np.ascontiguousarray(V)


def batch_problems(seed: int, count: int = 256, n_lo: int = 8, n_hi: int = 64):
    """Seeded list of independent 2D problems for the batching workload.

    Problem k gets order p = 1 + floor(4 u0) (uniform in 1..4), mesh size
    n = n_lo + floor((n_hi - n_lo + 1) u1) (uniform in [n_lo, n_hi]) and kind
    Taylor-Green for even k, Gresho for odd k (half each), with u0, u1 drawn
    from uniform01(seed, 2k) and uniform01(seed, 2k + 1).
    """
    u = uniform01(seed, np.arange(2 * count, dtype=np.uint64)).reshape(count, 2)
    out = []
    for k in range(count):
        p = 1 + min(3, int(4 * u[k, 0]))
        n = n_lo + min(n_hi - n_lo, int((n_hi - n_lo + 1) * u[k, 1]))
        kind = "taylor_green" if k % 2 == 0 else "gresho"
        lo, hi = (0.0, 1.0) if kind == "taylor_green" else (-0.5, 0.5)
        out.append(dict(order=p, n=n, kind=kind, lo=lo, hi=hi))
    return out
