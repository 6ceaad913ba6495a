"""Seeded synthetic SPH cases: particle lattices, walls, initial density.

This module only builds inputs.  It holds none of the interaction or
integration arithmetic; it is the one module that both the GPU path's tests
and the FP64 oracle's tests use, so that both sides start from identical
numbers.  Velocities and densities are rounded to float32 values (stored as
float64) because the GPU state keeps them in float32.

Geometry conventions (DualSPHysics paper, Sect. 2.6.1 and 6 workloads):
- a tank has two layers of dynamic-boundary particles on its bottom and side
  walls (open top); wall planes lie on the tank faces, the second layer one
  dp outward; the fluid lattice starts one dp inside each wall;
- h = sqrt(3) dp, rho0 = 1000, gamma = 7, alpha = 0.01, delta = 0.1,
  C_CFL = 0.2, eta^2 = 0.001 h^2, cs0 = 10 sqrt(g H) with H the still depth;
- fluid positions carry an i.i.d. uniform jitter in [-1e-4 dp, 1e-4 dp] per
  component drawn from a counter-based SplitMix64 stream (seeded);
- the initial density is hydrostatic: rho = rho0 (1 + rho0 g d / B)^(1/gamma)
  with B = cs0^2 rho0 / gamma and d the depth below the free surface.
"""
from dataclasses import dataclass, field
import math

import numpy as np

G = 9.81
GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of SplitMix64 started at `seed` (Steele et al. 2014)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Case:
    """One SPH case: constants + particle arrays in generator (id) order."""
    name: str
    params: dict
    pos: np.ndarray            # [n,3] float64
    vel: np.ndarray            # [n,3] float64 holding float32 values
    rho: np.ndarray            # [n] float64 holding float32 values
    ptype: np.ndarray          # [n] uint8: 0 fluid, 1 boundary
    group: np.ndarray          # [n] int32: motion index, -1 = none
    motions: list = field(default_factory=list)
    meta: dict = field(default_factory=dict)
    ghost: np.ndarray = None   # [n,3] r_G - r_B of boundary particles (mDBC), or None

    @property
    def n(self) -> int:
        return len(self.pos)

    @property
    def n_fluid(self) -> int:
        return int((self.ptype == 0).sum())


def default_params(dp: float, depth: float, domain_min, domain_max, **kw) -> dict:
    h = math.sqrt(3.0) * dp
    p = dict(dp=dp, h=h, rho0=1000.0, cs0=10.0 * math.sqrt(G * depth), gamma=7.0,
             alpha=0.01, delta=0.1, cfl=0.2, eta2=0.001 * h * h,
             gravity=(0.0, 0.0, -G), domain_min=tuple(float(x) for x in domain_min),
             domain_max=tuple(float(x) for x in domain_max), cell_mode=0, ddt_mode=1,
             clamp_boundary_rho=1, dt_fixed=0.0, dt_min=0.0, integrator=0, verlet_steps=40,
             visc_mode=0, nu0=1e-6, boundary_mode=0, mdbc_slip=0)
    p.update(kw)
    return p


def _grid_points(ix, iy, iz) -> np.ndarray:
    """Integer lattice points of the product of three index ranges."""
    X, Y, Z = np.meshgrid(np.asarray(ix), np.asarray(iy), np.asarray(iz), indexing="ij")
    # generator order: x fastest, then y, then z
    return np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                     Z.transpose(2, 1, 0).ravel()], axis=1)


def tank_walls(NX: int, NY: int, NZ: int, ix0: int = 0, layers: int = 2) -> np.ndarray:
    """Open-top tank walls in lattice units: planes at i = ix0, NX; j = 0, NY;
    k = 0, plus layers - 1 more layers outward (two by default; the mDBC
    cases use enough layers to fill the kernel support, ceil(2h/dp))."""
    r = lambda a, b: np.arange(a, b + 1)
    L = layers - 1
    bottom = _grid_points(r(ix0 - L, NX + L), r(-L, NY + L), r(-L, 0))
    xw = _grid_points(list(range(ix0 - L, ix0 + 1)) + list(range(NX, NX + L + 1)),
                      r(-L, NY + L), r(1, NZ))
    yw = _grid_points(r(ix0 + 1, NX - 1), list(range(-L, 1)) + list(range(NY, NY + L + 1)),
                      r(1, NZ))
    return np.concatenate([bottom, xw, yw], axis=0)


def wall_layers(dp: float, kw: dict) -> int:
    """Wall layers of a case: 2 for the dynamic boundary condition (Eq 36);
    for mDBC (Eq 38-39) enough to fill the support 2h behind the wall."""
    if kw.get("boundary_mode", 0) == 1:
        h = kw.get("h", math.sqrt(3.0) * dp)
        return int(math.ceil(2.0 * h / dp - 1e-9))
    return 2


def wall_ghosts(bound_lat, lo, hi) -> np.ndarray:
    """Ghost-node offsets r_G - r_B (lattice units) of boundary points for the
    modified dynamic boundary condition: the mirror image of each point in
    every wall plane it lies behind.  The fluid side is the box lo..hi of
    lattice indices (hi[k] None: open); a wall plane lies half a spacing
    outside it, between the inner wall layer and the first fluid layer."""
    b = np.asarray(bound_lat, np.float64)
    g = np.zeros_like(b)
    for k in range(3):
        below = b[:, k] < lo[k]
        g[below, k] = 2.0 * (lo[k] - 0.5 - b[below, k])
        if hi[k] is not None:
            above = b[:, k] > hi[k]
            g[above, k] = 2.0 * (hi[k] + 0.5 - b[above, k])
    return g


def hydrostatic_rho(depth_below_surface, rho0, cs0, gamma):
    """Initial condition: density whose Tait pressure equals rho0 g d."""
    B = cs0 * cs0 * rho0 / gamma
    d = np.maximum(np.asarray(depth_below_surface, np.float64), 0.0)
    return rho0 * (1.0 + rho0 * G * d / B) ** (1.0 / gamma)


def _assemble(name, params, fluid_lat, bound_lat, dp, seed, surface_z, footprint=None,
              bound_group=None, motions=(), origin=(0.0, 0.0, 0.0), meta=None,
              bound_ghost=None):
    nf, nb = len(fluid_lat), len(bound_lat)
    pos = np.concatenate([fluid_lat, bound_lat], axis=0).astype(np.float64) * dp
    pos += np.asarray(origin, np.float64)
    jit = (2.0 * uniform01(seed, 3 * nf) - 1.0) * (1e-4 * dp)
    pos[:nf] += jit.reshape(nf, 3)
    ptype = np.concatenate([np.zeros(nf, np.uint8), np.ones(nb, np.uint8)])
    rho0, cs0, gamma = params["rho0"], params["cs0"], params["gamma"]
    depth = surface_z - pos[:, 2]
    rho = hydrostatic_rho(depth, rho0, cs0, gamma)
    if footprint is not None:
        (x0, x1), (y0, y1) = footprint
        pad = 2.0 * params["h"]
        bx, by = pos[nf:, 0], pos[nf:, 1]
        near = (bx >= x0 - pad) & (bx <= x1 + pad) & (by >= y0 - pad) & (by <= y1 + pad)
        rho[nf:][~near] = rho0
    rho = rho.astype(np.float32).astype(np.float64)
    vel = np.zeros((nf + nb, 3))
    group = np.full(nf + nb, -1, np.int32)
    if bound_group is not None:
        group[nf:] = bound_group
        for gi, m in enumerate(motions):
            v0 = m["amp"] * m["omega"] * math.cos(m.get("phase", 0.0))
            sel = group == gi
            vel[sel] = np.asarray(m["axis"], np.float64) * v0
    vel = vel.astype(np.float32).astype(np.float64)
    ghost = np.zeros((nf + nb, 3))
    if bound_ghost is not None:
        ghost[nf:] = np.asarray(bound_ghost, np.float64) * dp
    return Case(name, params, pos, vel, rho, ptype, group, list(motions), dict(meta or {}),
                ghost)


def dam_break(dp: float = 0.02, seed: int = 0, column=(0.4, 0.4, 0.4),
              tank=(1.6, 0.67, 0.6), **kw) -> Case:
    """3-D dam break: fluid column in the x=0, y=0 corner of an open tank.

    dp = 0.02 gives 8,000 fluid + 20,062 boundary particles; dp = 0.004
    gives 1,000,000 fluid + 479,826 boundary particles."""
    NX, NY, NZ = (int(round(L / dp)) for L in tank)
    nfx, nfy, nfz = (int(round(L / dp)) for L in column)
    r = lambda a, b: np.arange(a, b + 1)
    fluid = _grid_points(r(1, nfx), r(1, nfy), r(1, nfz))
    nl = wall_layers(dp, kw)
    walls = tank_walls(NX, NY, NZ, layers=nl)
    surface = (nfz + 0.5) * dp
    depth = nfz * dp
    dmin = (-nl * dp, -nl * dp, -nl * dp)
    dmax = ((NX + nl) * dp, (NY + nl) * dp, 1.5 * NZ * dp)
    params = default_params(dp, depth, dmin, dmax, **kw)
    return _assemble("dam_break", params, fluid, walls, dp, seed, surface,
                     footprint=((0.0, (nfx + 1) * dp), (0.0, (nfy + 1) * dp)),
                     meta=dict(column=column, tank=(NX * dp, NY * dp, NZ * dp), seed=seed),
                     bound_ghost=wall_ghosts(walls, (1, 1, 1), (NX - 1, NY - 1, None)))


def still_tank(dp: float = 0.02, seed: int = 0, size=(0.2, 0.2), depth: float = 0.3,
               height: float = 0.4, **kw) -> Case:
    """Fluid at rest filling a small tank to `depth` (hydrostatic test)."""
    NX, NY = (int(round(L / dp)) for L in size)
    NZ = int(round(height / dp))
    nfz = int(round(depth / dp))
    r = lambda a, b: np.arange(a, b + 1)
    fluid = _grid_points(r(1, NX - 1), r(1, NY - 1), r(1, nfz))
    nl = wall_layers(dp, kw)
    walls = tank_walls(NX, NY, NZ, layers=nl)
    surface = (nfz + 0.5) * dp
    dmin = (-nl * dp, -nl * dp, -nl * dp)
    dmax = ((NX + nl) * dp, (NY + nl) * dp, (NZ + 2) * dp)
    params = default_params(dp, nfz * dp, dmin, dmax, **kw)
    return _assemble("still_tank", params, fluid, walls, dp, seed, surface,
                     meta=dict(surface=surface, seed=seed),
                     bound_ghost=wall_ghosts(walls, (1, 1, 1), (NX - 1, NY - 1, None)))


def wave_flume(dp: float = 0.008, seed: int = 0, length=25.0, width=1.0, height=1.2,
               depth=0.6, stroke=0.1, period=1.5, **kw) -> Case:
    """Wave flume with a piston wavemaker at x = 0 (imposed motion, Eq 37):
    X(t) = (stroke/2) sin(2 pi t / period).  dp = 0.008 gives ~29M fluid."""
    NX, NY, NZ = (int(round(L / dp)) for L in (length, width, height))
    nfz = int(round(depth / dp))
    back = int(math.ceil((0.5 * stroke + 4 * dp) / dp))  # walls extend behind the piston
    r = lambda a, b: np.arange(a, b + 1)
    fluid = _grid_points(r(1, NX - 1), r(1, NY - 1), r(1, nfz))
    nl = wall_layers(dp, kw)
    walls = tank_walls(NX, NY, NZ, ix0=-back, layers=nl)
    # the back wall of tank_walls sits at -back; drop it and add the piston
    keep = ~np.isin(walls[:, 0], np.arange(-back - nl + 1, -back + 1)) | (walls[:, 2] <= 0)
    walls = walls[keep]
    piston = _grid_points(np.arange(-nl + 1, 1), r(1, NY - 1), r(1, NZ))
    bound = np.concatenate([walls, piston], axis=0)
    bgroup = np.concatenate([np.full(len(walls), -1, np.int32), np.zeros(len(piston), np.int32)])
    surface = (nfz + 0.5) * dp
    dmin = (-(back + nl) * dp, -nl * dp, -nl * dp)
    dmax = ((NX + nl) * dp, (NY + nl) * dp, (NZ + 2) * dp)
    params = default_params(dp, nfz * dp, dmin, dmax, **kw)
    motions = [dict(axis=(1.0, 0.0, 0.0), amp=0.5 * stroke, omega=2 * math.pi / period,
                    phase=0.0)]
    ghost = np.concatenate([wall_ghosts(walls, (-back + 1, 1, 1), (NX - 1, NY - 1, None)),
                            wall_ghosts(piston, (1, 1, 1), (NX - 1, NY - 1, None))], axis=0)
    return _assemble("wave_flume", params, fluid, bound, dp, seed, surface,
                     bound_group=bgroup, motions=motions,
                     meta=dict(length=length, width=width, depth=depth, seed=seed),
                     bound_ghost=ghost)


def sloshing_tank(n_target: int, depth: float, amp: float, freq: float, seed: int = 0,
                  size=(1.0, 0.5, 0.6), **kw) -> Case:
    """Tank translated as a whole, x(t) = amp sin(2 pi freq t) (Eq 37), filled
    to `depth`; dp chosen so that the fluid has about n_target particles."""
    dp = (size[0] * size[1] * depth / n_target) ** (1.0 / 3.0)
    NX, NY, NZ = (int(round(L / dp)) for L in size)
    nfz = max(1, int(round(depth / dp)))
    r = lambda a, b: np.arange(a, b + 1)
    fluid = _grid_points(r(1, NX - 1), r(1, NY - 1), r(1, nfz))
    nl = wall_layers(dp, kw)
    walls = tank_walls(NX, NY, NZ, layers=nl)
    surface = (nfz + 0.5) * dp
    pad = amp / dp + nl + 1
    dmin = (-pad * dp, -nl * dp, -nl * dp)
    dmax = ((NX + pad) * dp, (NY + nl) * dp, (NZ + 2) * dp)
    params = default_params(dp, nfz * dp, dmin, dmax, **kw)
    motions = [dict(axis=(1.0, 0.0, 0.0), amp=amp, omega=2 * math.pi * freq, phase=0.0)]
    bgroup = np.zeros(len(walls), np.int32)
    return _assemble("sloshing_tank", params, fluid, walls, dp, seed, surface,
                     bound_group=bgroup, motions=motions,
                     meta=dict(depth=depth, amp=amp, freq=freq, seed=seed),
                     bound_ghost=wall_ghosts(walls, (1, 1, 1), (NX - 1, NY - 1, None)))


def batch_dam_breaks(n_cases: int = 256, seed: int = 0, n_min: int = 5000,
                     n_max: int = 200000, dp: float = 0.02, **kw) -> list:
    """Uneven dam breaks: fluid count log-uniform in [n_min, n_max], column
    width/height ratio U(0.5, 2), tank length U(3, 5) x width, tank width =
    column width, tank height 1.5 x column height, cs0 = 10 sqrt(g H)."""
    u = uniform01(seed ^ 0x5EED, 3 * n_cases).reshape(n_cases, 3)
    cases = []
    for i in range(n_cases):
        N = math.exp(math.log(n_min) + u[i, 0] * (math.log(n_max) - math.log(n_min)))
        ratio = 0.5 + 1.5 * u[i, 1]
        H = dp * (N / ratio ** 2) ** (1.0 / 3.0)
        w = ratio * H
        L = (3.0 + 2.0 * u[i, 2]) * w
        nw = max(2, int(round(w / dp)))
        nh = max(2, int(round(H / dp)))
        c = dam_break(dp, seed=seed + 1 + i, column=(nw * dp, nw * dp, nh * dp),
                      tank=(max(L, (nw + 2) * dp), (nw + 1) * dp, 1.5 * nh * dp), **kw)
        c.meta.update(index=i)
        cases.append(c)
    return cases


def free_particle(dp: float = 0.02, pos=(0.5, 0.5, 0.5), vel=(0.3, -0.2, 0.1), **kw) -> Case:
    """A single fluid particle without neighbours (free fall)."""
    params = default_params(dp, 0.4, (0.0, 0.0, -50.0), (1.0, 1.0, 1.0), **kw)
    p = np.array([pos], np.float64)
    v = np.array([vel], np.float32).astype(np.float64)
    rho = np.array([params["rho0"]])
    return Case("free_particle", params, p, v, rho, np.zeros(1, np.uint8),
                np.full(1, -1, np.int32), [], {})


def sloshing_trace(n_requests: int = 100, rate: float = 20.0, seed: int = 0,
                   n_min: int = 10000, n_max: int = 2000000, t_end: float = 1.0):
    """Seeded serving trace: Poisson arrivals (mean `rate` per second) of
    sloshing-tank cases, fill depth U(0.2, 0.4) m, excitation amplitude
    U(0.01, 0.05) m and frequency U(0.5, 1.5) Hz, fluid count log-uniform in
    [n_min, n_max].  Returns a list of (arrival_s, case, t_end)."""
    u = uniform01(seed ^ 0x7E5A, 5 * n_requests).reshape(n_requests, 5)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += -math.log(1.0 - u[i, 0]) / rate
        n = math.exp(math.log(n_min) + u[i, 1] * (math.log(n_max) - math.log(n_min)))
        depth = 0.2 + 0.2 * u[i, 2]
        amp = 0.01 + 0.04 * u[i, 3]
        freq = 0.5 + 1.0 * u[i, 4]
        c = sloshing_tank(int(n), depth, amp, freq, seed=seed + 1 + i)
        c.meta.update(request=i)
        out.append((t, c, t_end))
    return out
