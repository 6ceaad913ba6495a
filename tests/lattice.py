"""Small hand-built inputs for the oracle pins (lattices and clouds)."""
import math

import numpy as np

from paper_2104_00537_gb300 import cases


def lattice_case(n=11, dp=0.02, jitter=0.0, seed=1, **kw):
    """Cubic lattice of n^3 fluid particles at rest, rho = rho0, no gravity."""
    idx = np.arange(n)
    X, Y, Z = np.meshgrid(idx, idx, idx, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float64) * dp
    if jitter:
        pos += (2 * cases.uniform01(seed, pos.size) - 1).reshape(pos.shape) * jitter * dp
    kw.setdefault("gravity", (0.0, 0.0, 0.0))
    p = cases.default_params(dp, 0.4, (-3 * dp,) * 3, ((n + 3) * dp,) * 3, **kw)
    N = len(pos)
    return cases.Case("lattice", p, pos, np.zeros((N, 3)), np.full(N, p["rho0"]),
                      np.zeros(N, np.uint8), np.full(N, -1, np.int32), [], {"n": n})


def centre_index(n):
    """Index of the lattice point (n//2, n//2, n//2) in lattice_case order."""
    c = n // 2
    return (c * n + c) * n + c


def random_cloud(N=400, L=0.12, dp=0.02, seed=3, **kw):
    """Random fluid cloud (uniform in a cube of side L) with random v and rho."""
    u = cases.uniform01(seed, 7 * N).reshape(N, 7)
    pos = u[:, :3] * L
    kw.setdefault("gravity", (0.0, 0.0, 0.0))
    p = cases.default_params(dp, 0.4, (-0.05,) * 3, (L + 0.05,) * 3, **kw)
    vel = (u[:, 3:6] - 0.5) * 0.4
    rho = p["rho0"] * (1.0 + 0.01 * (u[:, 6] - 0.5))
    return cases.Case("cloud", p, pos, vel, rho, np.zeros(N, np.uint8),
                      np.full(N, -1, np.int32), [], {})
