"""ctypes wrapper of the FP64 CPU oracle (liboracle.so, built from sph_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg import this package.  The GPU product
path never imports it and shares no code with it.

The wrapper only marshals numpy arrays; all arithmetic is in sph_oracle.c.
A *case* is any object with the attributes produced by the seeded input
generators (``params`` dict, ``pos`` [n,3] float64, ``vel`` [n,3], ``rho`` [n],
``ptype`` [n] uint8, ``group`` [n] int32 and ``motions`` list of dicts).
"""
import contextlib
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrcParams(C.Structure):
    _fields_ = [("dp", C.c_double), ("h", C.c_double), ("rho0", C.c_double),
                ("cs0", C.c_double), ("gamma", C.c_double), ("alpha", C.c_double),
                ("delta", C.c_double), ("cfl", C.c_double), ("eta2", C.c_double),
                ("g", C.c_double * 3), ("dmin", C.c_double * 3),
                ("dmax", C.c_double * 3), ("dt_fixed", C.c_double),
                ("cell_mode", C.c_int32), ("ddt_mode", C.c_int32),
                ("clamp_boundary_rho", C.c_int32), ("visc_mode", C.c_int32),
                ("nu0", C.c_double), ("boundary_mode", C.c_int32), ("mdbc_slip", C.c_int32)]


class OrcMotion(C.Structure):
    _fields_ = [("axis", C.c_double * 3), ("amp", C.c_double),
                ("omega", C.c_double), ("phase", C.c_double)]


_D = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        _lib = load_library(_build.build())
    return _lib


@contextlib.contextmanager
def library(path):
    """Route every call of this module to another build of sph_oracle.c for
    the duration of the block.  The mutation tests compile a copy with one
    plausible mistake planted and check that a pin fails on it."""
    global _lib
    saved = _lib
    _lib = load_library(path)
    try:
        yield
    finally:
        _lib = saved


def load_library(path):
    """A build of the oracle at `path`, with the ctypes signatures of this
    module's calls."""
    L = C.CDLL(path)
    P = C.POINTER(OrcParams)
    L.orc_wendland_w.restype = C.c_double
    L.orc_wendland_w.argtypes = [C.c_double, C.c_double]
    L.orc_wendland_gradfac.restype = C.c_double
    L.orc_wendland_gradfac.argtypes = [C.c_double, C.c_double]
    L.orc_tait.restype = C.c_double
    L.orc_tait.argtypes = [P, C.c_double]
    L.orc_sps_tau.restype = C.c_int
    L.orc_sps_tau.argtypes = [P, C.c_int64, _D, _D, _D, _U8, C.c_void_p, _D]
    L.orc_rho_hydro.restype = C.c_double
    L.orc_rho_hydro.argtypes = [P, C.POINTER(C.c_double)]
    L.orc_grid.restype = C.c_int
    L.orc_grid.argtypes = [P, _D, C.POINTER(C.c_double), _I64, C.POINTER(C.c_int32)]
    L.orc_cells.restype = C.c_int
    L.orc_cells.argtypes = [P, C.c_int64, _D, _I64]
    L.orc_sort.restype = C.c_int64
    L.orc_sort.argtypes = [P, C.c_int64, _D, _U8, C.c_void_p, C.c_void_p, _I64]
    L.orc_pairs.restype = C.c_int64
    L.orc_pairs.argtypes = [P, C.c_int64, _D, C.c_void_p, C.c_int, _I64, _U64,
                            C.c_void_p, C.c_int64]
    L.orc_interact.restype = C.c_int64
    L.orc_interact.argtypes = [P, C.c_int64, _D, _D, _D, _U8, C.c_void_p, C.c_int,
                               _D, _D, _D]
    L.orc_interact_range.restype = C.c_int64
    L.orc_interact_range.argtypes = [P, C.c_int64, _D, _D, _D, _U8, C.c_void_p, C.c_int,
                                     C.c_int64, C.c_int64, _D, _D, _D]
    L.orc_dt.restype = C.c_double
    L.orc_dt.argtypes = [P, C.c_int64, _D, _D, _U8, C.c_void_p]
    L.orc_step.restype = C.c_int64
    L.orc_step.argtypes = [P, C.c_void_p, C.c_int32, C.c_int64, _D, _D, _D, _U8,
                           _I32, _U8, C.c_void_p, C.POINTER(C.c_double),
                           C.POINTER(C.c_double), C.c_int64, _D]
    L.orc_mdbc.restype = C.c_int
    L.orc_mdbc.argtypes = [P, C.c_void_p, C.c_int32, C.c_int64, _D, _D, _D, _U8, _I32,
                           C.c_void_p, _D, C.c_double, C.c_void_p]
    L.orc_step_verlet.restype = C.c_int64
    L.orc_step_verlet.argtypes = [P, C.c_void_p, C.c_int32, C.c_int64, _D, _D, _D, _D, _D,
                                  _U8, _I32, _U8, C.c_void_p, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32,
                                  C.c_int64, _D]
    L.orc_diag.restype = C.c_int
    L.orc_diag.argtypes = [P, C.c_int64, _D, _D, _U8, C.c_void_p, _D]
    return L


def make_params(p: dict) -> OrcParams:
    """Convert a case parameter dict into the oracle's parameter struct."""
    o = OrcParams()
    for k in ("dp", "h", "rho0", "cs0", "gamma", "alpha", "delta", "cfl", "eta2"):
        setattr(o, k, float(p[k]))
    o.g[:] = [float(x) for x in p["gravity"]]
    o.dmin[:] = [float(x) for x in p["domain_min"]]
    o.dmax[:] = [float(x) for x in p["domain_max"]]
    o.dt_fixed = float(p.get("dt_fixed", 0.0))
    o.cell_mode = int(p.get("cell_mode", 0))
    o.ddt_mode = int(p.get("ddt_mode", 1))
    o.clamp_boundary_rho = int(p.get("clamp_boundary_rho", 1))
    o.visc_mode = int(p.get("visc_mode", 0))
    o.nu0 = float(p.get("nu0", 1e-6))
    o.boundary_mode = int(p.get("boundary_mode", 0))
    o.mdbc_slip = int(p.get("mdbc_slip", 0))
    return o


def make_motions(motions):
    arr = (OrcMotion * max(1, len(motions)))()
    for i, m in enumerate(motions):
        arr[i].axis[:] = [float(x) for x in m["axis"]]
        arr[i].amp = float(m["amp"])
        arr[i].omega = float(m["omega"])
        arr[i].phase = float(m.get("phase", 0.0))
    return arr


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def wendland_w(r, h):
    return lib().orc_wendland_w(float(r), float(h))


def wendland_gradfac(r, h):
    return lib().orc_wendland_gradfac(float(r), float(h))


def tait(params: dict, rho):
    return lib().orc_tait(C.byref(make_params(params)), float(rho))


def sps_tau(params: dict, pos, vel, rho, ptype, out=None):
    """tau / rho of Eq 25 per particle: columns xx, yy, zz, xy, xz, yz."""
    pos = np.ascontiguousarray(pos, np.float64)
    vel = np.ascontiguousarray(vel, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    ptype = np.ascontiguousarray(ptype, np.uint8)
    out_ = None if out is None else np.ascontiguousarray(out, np.uint8)
    tau = np.zeros((len(ptype), 6))
    if lib().orc_sps_tau(C.byref(make_params(params)), len(ptype), pos, vel, rho, ptype,
                         _ptr(out_), tau) != 0:
        raise ValueError("oracle sps_tau failed")
    return tau


def mdbc(case, pos, vel, rho, t=0.0, out=None, with_dets=False):
    """Eq 38-39 boundary values on the given state: returns (rho, vel) with
    the boundary entries replaced (and the moment determinants if asked)."""
    pos = np.ascontiguousarray(pos, np.float64)
    vel = np.array(vel, np.float64, order="C")
    rho = np.array(rho, np.float64, order="C")
    ptype = np.ascontiguousarray(case.ptype, np.uint8)
    group = np.ascontiguousarray(case.group, np.int32)
    ghost = ghost_of(case)
    out_ = None if out is None else np.ascontiguousarray(out, np.uint8)
    dets = np.zeros(len(ptype))
    mot = make_motions(case.motions)
    if lib().orc_mdbc(C.byref(make_params(case.params)), C.cast(mot, C.c_void_p),
                      len(case.motions), len(ptype), pos, vel, rho, ptype, group, _ptr(out_),
                      ghost, float(t), dets.ctypes.data_as(C.c_void_p)) != 0:
        raise ValueError("oracle mdbc failed")
    return (rho, vel, dets) if with_dets else (rho, vel)


def ghost_of(case):
    g = getattr(case, "ghost", None)
    if g is None:
        g = np.zeros((len(case.pos), 3))
    return np.ascontiguousarray(g, np.float64)


def rho_hydro(params: dict, rab):
    """Hydrostatic density difference rho^H_ab of Eq 19-20 for r_ab."""
    r = (C.c_double * 3)(*[float(x) for x in rab])
    return lib().orc_rho_hydro(C.byref(make_params(params)), r)


def grid(params: dict):
    o = np.zeros(3)
    cs = C.c_double()
    nc = np.zeros(3, np.int64)
    m = C.c_int32()
    if lib().orc_grid(C.byref(make_params(params)), o, C.byref(cs), nc, C.byref(m)):
        raise ValueError("bad grid parameters")
    return o, cs.value, nc, m.value


def cells(params: dict, pos):
    pos = np.ascontiguousarray(pos, np.float64)
    out = np.zeros(len(pos), np.int64)
    lib().orc_cells(C.byref(make_params(params)), len(pos), pos, out)
    return out


def sort_order(params: dict, pos, ptype, out=None, prev_order=None):
    """Neighbour-list order (stable by (is_boundary, cell)); returns (order, n_inside)."""
    pos = np.ascontiguousarray(pos, np.float64)
    ptype = np.ascontiguousarray(ptype, np.uint8)
    n = len(pos)
    order = np.zeros(n, np.int64)
    out_ = None if out is None else np.ascontiguousarray(out, np.uint8)
    prev = None if prev_order is None else np.ascontiguousarray(prev_order, np.int64)
    inside = lib().orc_sort(C.byref(make_params(params)), n, pos, ptype,
                            _ptr(out_), _ptr(prev), order)
    return order, int(inside)


def pairs(params: dict, pos, use_cells=True, out=None, want_list=False):
    """Neighbour pairs: returns (total, count[n], hash[n], sorted pair list or None)."""
    pos = np.ascontiguousarray(pos, np.float64)
    n = len(pos)
    count = np.zeros(n, np.int64)
    hsh = np.zeros(n, np.uint64)
    out_ = None if out is None else np.ascontiguousarray(out, np.uint8)
    P = C.byref(make_params(params))
    total = lib().orc_pairs(P, n, pos, _ptr(out_), int(use_cells), count, hsh, None, 0)
    plist = None
    if want_list:
        plist = np.zeros((max(total, 1), 2), np.int64)
        lib().orc_pairs(P, n, pos, _ptr(out_), int(use_cells), count, hsh,
                        _ptr(plist), total)
        plist = plist[:total]
    return int(total), count, hsh, plist


def interact(params: dict, pos, vel, rho, ptype, out=None, use_cells=True):
    """One PI evaluation: returns (acc [n,3], drho [n], mumax [n], npairs)."""
    pos = np.ascontiguousarray(pos, np.float64)
    vel = np.ascontiguousarray(vel, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    ptype = np.ascontiguousarray(ptype, np.uint8)
    n = len(pos)
    acc = np.zeros((n, 3))
    drho = np.zeros(n)
    mu = np.zeros(n)
    out_ = None if out is None else np.ascontiguousarray(out, np.uint8)
    npairs = lib().orc_interact(C.byref(make_params(params)), n, pos, vel, rho, ptype,
                                _ptr(out_), int(use_cells), acc, drho, mu)
    if npairs < 0:
        raise ValueError("oracle interaction failed")
    return acc, drho, mu, int(npairs)


def interact_range(params: dict, pos, vel, rho, ptype, a0, a1):
    """PI for the particles a in [a0, a1) only: returns (acc, drho, mumax, npairs)."""
    pos = np.ascontiguousarray(pos, np.float64)
    vel = np.ascontiguousarray(vel, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    ptype = np.ascontiguousarray(ptype, np.uint8)
    n = len(pos)
    acc = np.zeros((n, 3))
    drho = np.zeros(n)
    mu = np.zeros(n)
    npairs = lib().orc_interact_range(C.byref(make_params(params)), n, pos, vel, rho, ptype,
                                      None, 1, int(a0), int(a1), acc, drho, mu)
    if npairs < 0:
        raise ValueError("oracle interaction failed")
    return acc, drho, mu, int(npairs)


def time_step(params: dict, acc, mumax, ptype, out=None):
    acc = np.ascontiguousarray(acc, np.float64)
    mumax = np.ascontiguousarray(mumax, np.float64)
    ptype = np.ascontiguousarray(ptype, np.uint8)
    out_ = None if out is None else np.ascontiguousarray(out, np.uint8)
    return lib().orc_dt(C.byref(make_params(params)), len(ptype), acc, mumax, ptype,
                        _ptr(out_))


class OracleState:
    """Mutable FP64 state of one case, advanced by Symplectic steps (Eq 33-34)
    or, when the case's params say integrator = 1, by Verlet steps (Eq 30-31,
    with an Eq 31 step every verlet_steps steps)."""

    def __init__(self, case):
        self.params = dict(case.params)
        self.pos = np.array(case.pos, np.float64, order="C")
        self.vel = np.array(case.vel, np.float64, order="C")
        self.rho = np.array(case.rho, np.float64, order="C")
        self.ptype = np.ascontiguousarray(case.ptype, np.uint8)
        self.group = np.ascontiguousarray(case.group, np.int32)
        self.out = np.zeros(len(self.pos), np.uint8)
        self.order = np.arange(len(self.pos), dtype=np.int64)
        self.motions = list(case.motions)
        self.t = C.c_double(0.0)
        self.last_dt = C.c_double(0.0)
        self.steps = 0
        self.pairs = 0
        self.verlet = int(self.params.get("integrator", 0)) == 1
        self.vel_prev = self.vel.copy()
        self.rho_prev = self.rho.copy()
        self.step_count = C.c_int64(0)
        self.ghost = ghost_of(case)

    def step(self, nsteps=1):
        L = lib()
        mot = make_motions(self.motions)
        if self.verlet:
            ns = int(self.params.get("verlet_steps", 40)) or 40
            npairs = L.orc_step_verlet(C.byref(make_params(self.params)),
                                       C.cast(mot, C.c_void_p), len(self.motions),
                                       len(self.pos), self.pos, self.vel, self.rho,
                                       self.vel_prev, self.rho_prev, self.ptype, self.group,
                                       self.out, self.order.ctypes.data_as(C.c_void_p),
                                       C.byref(self.t), C.byref(self.last_dt),
                                       C.byref(self.step_count), ns, int(nsteps), self.ghost)
            if npairs < 0:
                raise ValueError("oracle step failed")
            self.steps += nsteps
            self.pairs += npairs
            return npairs
        npairs = L.orc_step(C.byref(make_params(self.params)), C.cast(mot, C.c_void_p),
                            len(self.motions), len(self.pos), self.pos, self.vel,
                            self.rho, self.ptype, self.group, self.out,
                            self.order.ctypes.data_as(C.c_void_p), C.byref(self.t),
                            C.byref(self.last_dt), int(nsteps), self.ghost)
        if npairs < 0:
            raise ValueError("oracle step failed")
        self.steps += nsteps
        self.pairs += npairs
        return npairs

    def diag(self):
        res = np.zeros(7)
        lib().orc_diag(C.byref(make_params(self.params)), len(self.pos), self.pos,
                       self.vel, self.ptype, _ptr(self.out), res)
        return dict(mass=res[0], ke=res[1], momentum=res[2:5].copy(), front=res[5],
                    n_out=int(res[6]))

    def pressure(self):
        P = make_params(self.params)
        L = lib()
        return np.array([L.orc_tait(C.byref(P), float(r)) for r in self.rho])
