"""Thin ctypes binding of libsph.so (C ABI in include/sph.h).

Only argument marshalling lives here: every step of the SPH hot path runs in
the CUDA kernels of libsph.so.  PyTorch is used for device memory (the
caching allocator, through the library's allocator callback) and streams.
There is no CPU fallback: if the library cannot be loaded or no CUDA device
is present, the calls raise.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))

SPH_OK = 0
SORT_STATIC_MAX_KEYS = 524288  # SPH_SORT_STATIC_MAX_KEYS of include/sph.h
ERRORS = {-1: "SPH_ERR_ARG", -2: "SPH_ERR_OOM", -3: "SPH_ERR_CUDA", -4: "SPH_ERR_UNSTABLE",
          -5: "SPH_ERR_DOMAIN", -7: "SPH_ERR_BUSY", -8: "SPH_ERR_STATE"}


class SphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class D3(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double)]


class CaseParams(C.Structure):
    _fields_ = [("dp", C.c_double), ("h", C.c_double), ("rho0", C.c_double),
                ("cs0", C.c_double), ("gamma", C.c_double), ("alpha", C.c_double),
                ("delta", C.c_double), ("cfl", C.c_double), ("eta2", C.c_double),
                ("gravity", D3), ("domain_min", D3), ("domain_max", D3),
                ("dt_fixed", C.c_double), ("dt_min", C.c_double),
                ("cell_mode", C.c_int32), ("ddt_mode", C.c_int32),
                ("clamp_boundary_rho", C.c_int32), ("max_out", C.c_int32),
                ("integrator", C.c_int32), ("verlet_steps", C.c_int32),
                ("visc_mode", C.c_int32), ("boundary_mode", C.c_int32), ("nu0", C.c_double),
                ("mdbc_slip", C.c_int32), ("pad2_", C.c_int32)]


class Motion(C.Structure):
    _fields_ = [("axis", D3), ("amplitude", C.c_double), ("omega", C.c_double),
                ("phase", C.c_double)]


class Particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p), ("vel", C.c_void_p),
                ("rho", C.c_void_p), ("type", C.c_void_p), ("motion_group", C.c_void_p),
                ("motions", C.c_void_p), ("n_motions", C.c_int32), ("ghost", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("t", C.c_double), ("last_dt", C.c_double), ("step", C.c_int64),
                ("interactions", C.c_int64), ("interactions_fb", C.c_int64),
                ("interactions_bf", C.c_int64), ("mass", C.c_double),
                ("kinetic_energy", C.c_double), ("momentum", C.c_double * 3),
                ("front", C.c_double), ("n_out", C.c_int64), ("flags", C.c_int32),
                ("n_fluid", C.c_int32), ("n", C.c_int64)]


class Options(C.Structure):
    _fields_ = [("pi_block", C.c_int32), ("pi_variant", C.c_int32),
                ("use_graph", C.c_int32), ("timing", C.c_int32),
                ("list_skin", C.c_float), ("check_list", C.c_int32),
                ("pi_lanes", C.c_int32), ("pair_once", C.c_int32),
                ("wide_records", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsph.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libsph.so is missing (%s): build it with __graft_entry__.build()" % path)
    L = C.CDLL(path)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    sig = {
        "sph_last_error": (C.c_char_p, []),
        "sph_create": (C.c_int, [C.POINTER(CaseParams), C.POINTER(Particles), vp, ALLOC_FN,
                                 FREE_FN, vp, C.POINTER(vp)]),
        "sph_batch_create": (C.c_int, [C.POINTER(CaseParams), C.POINTER(Particles), i32, vp,
                                       ALLOC_FN, FREE_FN, vp, C.POINTER(vp)]),
        "sph_step": (C.c_int, [vp, i64]),
        "sph_get_state": (C.c_int, [vp, i32, vp, vp, vp, vp, dp, C.POINTER(i64), dp]),
        "sph_get_stats": (C.c_int, [vp, i32, C.POINTER(Stats)]),
        "sph_set_options": (C.c_int, [vp, C.POINTER(Options)]),
        "sph_get_timing": (C.c_int, [vp, dp, C.POINTER(i64), dp, C.POINTER(i64), i32]),
        "sph_list_info": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]),
        "sph_get_step_times": (C.c_int, [vp, vp, i64, C.POINTER(i64)]),
        "sph_get_raw": (C.c_int, [vp, i32, vp, C.POINTER(C.c_size_t)]),
        "sph_create_from_raw": (C.c_int, [C.POINTER(CaseParams), C.POINTER(Particles), vp,
                                          C.c_size_t, vp, ALLOC_FN, FREE_FN, vp,
                                          C.POINTER(vp)]),
        "sph_eval_forces": (C.c_int, [vp, i32, vp, vp, vp, dp, C.POINTER(i64)]),
        "sph_eval_step": (C.c_int, [vp, i32, i32, vp, vp, vp, vp, vp, vp, dp,
                                    C.POINTER(i64)]),
        "sph_eval_sps": (C.c_int, [vp, i32, vp]),
        "sph_eval_boundary": (C.c_int, [vp, i32, vp, vp]),
        "sph_get_order": (C.c_int, [vp, i32, vp, vp, C.POINTER(i64)]),
        "sph_pair_stats": (C.c_int, [vp, i32, vp, vp]),
        "sph_pool_create": (C.c_int, [i64, i64, i32, vp, ALLOC_FN, FREE_FN, vp, C.POINTER(vp)]),
        "sph_pool_admit": (C.c_int, [vp, C.POINTER(CaseParams), C.POINTER(Particles),
                                     C.c_double, C.POINTER(i32)]),
        "sph_pool_step": (C.c_int, [vp, i64, vp, C.POINTER(i32)]),
        "sph_pool_release": (C.c_int, [vp, i32]),
        "sph_pool_usage": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)]),
        "sph_destroy": (None, [vp]),
        "sph_probe_peaks": (C.c_int, [dp, dp, C.POINTER(i32), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def probe_peaks(stream=None):
    """Measured FP32 and FP64 FMA throughput (TFLOP/s) and SM count of the
    current device (the roofline denominators of the pair loop)."""
    f32, f64, sms = C.c_double(), C.c_double(), C.c_int32()
    check(load().sph_probe_peaks(C.byref(f32), C.byref(f64), C.byref(sms),
                                 _stream_handle(stream)))
    return dict(fp32_tflops=f32.value, fp64_tflops=f64.value, sms=sms.value)


def last_error() -> str:
    return load().sph_last_error().decode()


def check(rc):
    if rc != SPH_OK:
        raise SphError(rc, last_error())
    return rc


def make_params(p: dict) -> CaseParams:
    """C struct from a case parameter dict (see cases.default_params)."""
    c = CaseParams()
    for k in ("dp", "h", "rho0", "cs0", "gamma", "alpha", "delta", "cfl", "eta2"):
        setattr(c, k, float(p[k]))
    c.gravity = D3(*map(float, p["gravity"]))
    c.domain_min = D3(*map(float, p["domain_min"]))
    c.domain_max = D3(*map(float, p["domain_max"]))
    c.dt_fixed = float(p.get("dt_fixed", 0.0))
    c.dt_min = float(p.get("dt_min", 0.0))
    c.cell_mode = int(p.get("cell_mode", 0))
    c.ddt_mode = int(p.get("ddt_mode", 1))
    c.clamp_boundary_rho = int(p.get("clamp_boundary_rho", 1))
    c.max_out = int(p.get("max_out", -1))
    c.integrator = int(p.get("integrator", 0))
    c.verlet_steps = int(p.get("verlet_steps", 40))
    c.visc_mode = int(p.get("visc_mode", 0))
    c.nu0 = float(p.get("nu0", 1e-6))
    c.boundary_mode = int(p.get("boundary_mode", 0))
    c.mdbc_slip = int(p.get("mdbc_slip", 0))
    return c


def state_buffers(n, pinned=False):
    """Host arrays of n particles for Engine.get_state(out=...); pinned: in
    page-locked memory (kept alive by the returned dict's "_keep")."""
    out = dict(pos=np.zeros((n, 3), np.float64), vel=np.zeros((n, 3), np.float32),
               rho=np.zeros(n, np.float32), press=np.zeros(n, np.float32))
    if pinned:
        import torch
        keep = [torch.from_numpy(a).pin_memory() for a in out.values()]
        out = dict(zip(out.keys(), (t.numpy() for t in keep)))
        out["_keep"] = keep
    return out


class HostParticles:
    """Keeps the host arrays of one case alive while the C struct points at them."""

    def __init__(self, case, pinned=False):
        n = case.n
        self.pos = np.ascontiguousarray(case.pos, np.float64).reshape(n, 3)
        self.vel = np.ascontiguousarray(case.vel, np.float32).reshape(n, 3)
        self.rho = np.ascontiguousarray(case.rho, np.float32).reshape(n)
        self.type = np.ascontiguousarray(case.ptype, np.uint8).reshape(n)
        self.group = np.ascontiguousarray(case.group, np.int32).reshape(n)
        g = getattr(case, "ghost", None)
        self.ghost = None if g is None else np.ascontiguousarray(g, np.float32).reshape(n, 3)
        self.motions = (Motion * max(1, len(case.motions)))()
        for i, m in enumerate(case.motions):
            self.motions[i].axis = D3(*map(float, m["axis"]))
            self.motions[i].amplitude = float(m["amp"])
            self.motions[i].omega = float(m["omega"])
            self.motions[i].phase = float(m.get("phase", 0.0))
        if pinned:
            self._pin()
        self.struct = Particles(n, self.pos.ctypes.data, self.vel.ctypes.data,
                                self.rho.ctypes.data, self.type.ctypes.data,
                                self.group.ctypes.data, C.addressof(self.motions),
                                len(case.motions),
                                None if self.ghost is None else self.ghost.ctypes.data)

    def _pin(self):
        import torch
        self._pinned = []
        for name in ("pos", "vel", "rho", "type", "group") + (("ghost",) if self.ghost is not None
                                                               else ()):
            a = getattr(self, name)
            t = torch.from_numpy(a).pin_memory()
            self._pinned.append(t)
            setattr(self, name, t.numpy())


class TorchAllocator:
    """Device memory for the library from the PyTorch caching allocator."""

    def __init__(self, device=0):
        import torch
        self.torch = torch
        self.device = device
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, size, stream, ctx):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(size), self.device,
                                                           stream if stream else None)
        except Exception:  # out of memory: the library reports SPH_ERR_OOM
            return None

    def _free(self, ptr, size, stream, ctx):
        self.torch.cuda.caching_allocator_delete(ptr)


_NULL_ALLOC = ALLOC_FN()
_NULL_FREE = FREE_FN()


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class Engine:
    """One libsph engine: a case, a batch of cases or a serving pool."""

    def __init__(self, handle, keep):
        self.h = handle
        self._keep = keep
        self.lib = load()

    # ---- constructors
    @classmethod
    def create(cls, case, stream=None, torch_alloc=True, pinned=False, host=None):
        """host: a HostParticles of the case prepared beforehand (e.g. pinned)."""
        L = load()
        hp = host if host is not None else HostParticles(case, pinned=pinned)
        prm = make_params(case.params)
        al = TorchAllocator() if torch_alloc else None
        h = C.c_void_p()
        check(L.sph_create(C.byref(prm), C.byref(hp.struct), _stream_handle(stream),
                           al.alloc_cb if al else _NULL_ALLOC, al.free_cb if al else _NULL_FREE,
                           None, C.byref(h)))
        e = cls(h, [al])
        e.sizes = [case.n]
        return e

    @classmethod
    def batch(cls, cases, stream=None, torch_alloc=True):
        L = load()
        hps = [HostParticles(c) for c in cases]
        prms = (CaseParams * len(cases))(*[make_params(c.params) for c in cases])
        parts = (Particles * len(cases))(*[hp.struct for hp in hps])
        al = TorchAllocator() if torch_alloc else None
        h = C.c_void_p()
        check(L.sph_batch_create(prms, parts, len(cases), _stream_handle(stream),
                                 al.alloc_cb if al else _NULL_ALLOC,
                                 al.free_cb if al else _NULL_FREE, None, C.byref(h)))
        e = cls(h, [al])
        e.sizes = [c.n for c in cases]
        return e

    @classmethod
    def pool(cls, max_particles, max_cells, max_cases, stream=None, torch_alloc=True):
        L = load()
        al = TorchAllocator() if torch_alloc else None
        h = C.c_void_p()
        check(L.sph_pool_create(int(max_particles), int(max_cells), int(max_cases),
                                _stream_handle(stream), al.alloc_cb if al else _NULL_ALLOC,
                                al.free_cb if al else _NULL_FREE, None, C.byref(h)))
        e = cls(h, [al])
        e.sizes = {}
        return e

    @classmethod
    def from_raw(cls, case, raw: bytes, stream=None, torch_alloc=True):
        L = load()
        hp = HostParticles(case)
        prm = make_params(case.params)
        al = TorchAllocator() if torch_alloc else None
        buf = C.create_string_buffer(raw, len(raw))
        h = C.c_void_p()
        check(L.sph_create_from_raw(C.byref(prm), C.byref(hp.struct), buf, len(raw),
                                    _stream_handle(stream), al.alloc_cb if al else _NULL_ALLOC,
                                    al.free_cb if al else _NULL_FREE, None, C.byref(h)))
        e = cls(h, [al])
        e.sizes = [case.n]
        return e

    # ---- calls
    def step(self, nsteps=1):
        check(self.lib.sph_step(self.h, int(nsteps)))

    def set_options(self, pi_block=0, pi_variant=-1, use_graph=0, timing=0, list_skin=-1.0,
                    check_list=0, pi_lanes=0, pair_once=0, wide_records=0):
        """pi_variant -1 keeps the engine default (where the engine supports
        a neighbour list: kept across steps, 5; else the compacted loop, 0;
        4, one list per step, keeps batch and pool cases equal to their runs
        alone bit for bit); list_skin:
        variant 5's added skin as a fraction of 2h (< 0: the default, 0.04);
        check_list: brute-force check of every list evaluation (list_info);
        pi_lanes: threads per target of the list walk (0: the default);
        pair_once: evaluate each pair once (atomic sums, not bit-reproducible);
        wide_records: 32-bit list records at any size (else beyond 2^25 only)."""
        o = Options(pi_block, pi_variant, use_graph, timing, list_skin, check_list, pi_lanes,
                    pair_once, wide_records)
        check(self.lib.sph_set_options(self.h, C.byref(o)))

    def list_info(self):
        """Neighbour-list builds so far and, with check_list, the brute-force
        pair count and the number of targets whose list missed or added pairs."""
        b, p, bad = C.c_int64(), C.c_int64(), C.c_int64()
        check(self.lib.sph_list_info(self.h, C.byref(b), C.byref(p), C.byref(bad)))
        return dict(builds=b.value, check_pairs=p.value, check_bad=bad.value)

    def timing(self, reset=False):
        pm, ln, sm, kl = C.c_double(), C.c_int64(), C.c_double(), C.c_int64()
        check(self.lib.sph_get_timing(self.h, C.byref(pm), C.byref(ln), C.byref(sm), C.byref(kl),
                                      int(reset)))
        return dict(pi_ms=pm.value, pi_launches=ln.value, step_ms=sm.value,
                    kernel_launches=kl.value)

    def step_times(self):
        """Device time of each step timed since the last timing reset (ms)."""
        n = C.c_int64()
        check(self.lib.sph_get_step_times(self.h, None, 0, C.byref(n)))
        out = np.zeros(n.value, np.float32)
        check(self.lib.sph_get_step_times(self.h, out.ctypes.data_as(C.c_void_p), n.value,
                                          C.byref(n)))
        return out

    def _n(self, icase):
        return self.sizes[icase]

    def get_state(self, icase=0, out=None):
        """The case's state in the caller's order; out: arrays from
        state_buffers(n) to fill instead of new ones."""
        n = self._n(icase)
        if out is None:
            out = state_buffers(n)
        pos, vel, rho, press = out["pos"], out["vel"], out["rho"], out["press"]
        assert pos.shape == (n, 3) and rho.shape == (n,)
        t, st, dt = C.c_double(), C.c_int64(), C.c_double()
        check(self.lib.sph_get_state(self.h, icase, pos.ctypes.data, vel.ctypes.data,
                                     rho.ctypes.data, press.ctypes.data, C.byref(t),
                                     C.byref(st), C.byref(dt)))
        return dict(pos=pos, vel=vel, rho=rho, press=press, t=t.value, step=st.value,
                    last_dt=dt.value)

    def stats(self, icase=0):
        s = Stats()
        check(self.lib.sph_get_stats(self.h, icase, C.byref(s)))
        return dict(t=s.t, last_dt=s.last_dt, step=s.step, interactions=s.interactions,
                    interactions_fb=s.interactions_fb, interactions_bf=s.interactions_bf,
                    mass=s.mass, ke=s.kinetic_energy, momentum=list(s.momentum), front=s.front,
                    n_out=s.n_out, flags=s.flags, n_fluid=s.n_fluid, n=s.n)

    def eval_forces(self, icase=0):
        n = self._n(icase)
        acc = np.zeros((n, 3), np.float32)
        drho = np.zeros(n, np.float32)
        mu = np.zeros(n, np.float32)
        dt, pairs = C.c_double(), C.c_int64()
        check(self.lib.sph_eval_forces(self.h, icase, acc.ctypes.data, drho.ctypes.data,
                                       mu.ctypes.data, C.byref(dt), C.byref(pairs)))
        return dict(acc=acc, drho=drho, mumax=mu, dt=dt.value, pairs=pairs.value)

    def eval_step(self, stage=0, icase=0):
        """One evaluation of the next step through the step's own launches
        (stage 0: state n; 1: the half-step state of a list step), without
        advancing: the evaluated state and its results, original order."""
        n = self._n(icase)
        pos = np.zeros((n, 3), np.float64)
        vel = np.zeros((n, 3), np.float32)
        rho = np.zeros(n, np.float32)
        acc = np.zeros((n, 3), np.float32)
        drho = np.zeros(n, np.float32)
        mu = np.zeros(n, np.float32)
        dt, pairs = C.c_double(), C.c_int64()
        check(self.lib.sph_eval_step(self.h, icase, int(stage), pos.ctypes.data,
                                     vel.ctypes.data, rho.ctypes.data, acc.ctypes.data,
                                     drho.ctypes.data, mu.ctypes.data, C.byref(dt),
                                     C.byref(pairs)))
        return dict(pos=pos, vel=vel, rho=rho, acc=acc, drho=drho, mumax=mu, dt=dt.value,
                    pairs=pairs.value)

    def eval_sps(self, icase=0):
        """tau / rho of Eq 25 per particle (original order): xx, yy, zz, xy, xz, yz."""
        tau = np.zeros((self._n(icase), 6), np.float32)
        check(self.lib.sph_eval_sps(self.h, icase, tau.ctypes.data))
        return tau

    def eval_boundary(self, icase=0):
        """mDBC boundary values (Eq 38-39) on the current state: (vel [n,3], rho [n])."""
        n = self._n(icase)
        vel = np.zeros((n, 3), np.float32)
        rho = np.zeros(n, np.float32)
        check(self.lib.sph_eval_boundary(self.h, icase, vel.ctypes.data, rho.ctypes.data))
        return vel, rho

    def order(self, icase=0):
        n = self._n(icase)
        ids = np.zeros(n, np.int64)
        cells = np.zeros(n, np.int64)
        ni = C.c_int64()
        check(self.lib.sph_get_order(self.h, icase, ids.ctypes.data, cells.ctypes.data,
                                     C.byref(ni)))
        return ids, cells, ni.value

    def pair_stats(self, icase=0):
        n = self._n(icase)
        cnt = np.zeros(n, np.int64)
        hsh = np.zeros(n, np.uint64)
        check(self.lib.sph_pair_stats(self.h, icase, cnt.ctypes.data, hsh.ctypes.data))
        return cnt, hsh

    def get_raw(self, icase=0) -> bytes:
        nb = C.c_size_t()
        check(self.lib.sph_get_raw(self.h, icase, None, C.byref(nb)))
        buf = C.create_string_buffer(nb.value)
        check(self.lib.sph_get_raw(self.h, icase, buf, C.byref(nb)))
        return buf.raw[:nb.value]

    # ---- pool
    def admit(self, case, t_end):
        hp = HostParticles(case)
        prm = make_params(case.params)
        slot = C.c_int32()
        check(self.lib.sph_pool_admit(self.h, C.byref(prm), C.byref(hp.struct), float(t_end),
                                      C.byref(slot)))
        self.sizes[slot.value] = case.n
        return slot.value

    def try_admit(self, case, t_end):
        """Admit, or return None when the pool is busy (no slot or memory)."""
        try:
            return self.admit(case, t_end)
        except SphError as e:
            if e.code == -7:
                return None
            raise

    def pool_step(self, nsteps=1):
        fin = (C.c_int32 * 65536)()
        nf = C.c_int32()
        check(self.lib.sph_pool_step(self.h, int(nsteps), fin, C.byref(nf)))
        return [fin[i] for i in range(nf.value)]

    def release(self, slot):
        check(self.lib.sph_pool_release(self.h, int(slot)))
        self.sizes.pop(slot, None)

    def usage(self):
        p, c, k = C.c_int64(), C.c_int64(), C.c_int32()
        check(self.lib.sph_pool_usage(self.h, C.byref(p), C.byref(c), C.byref(k)))
        return dict(particles=p.value, cells=c.value, cases=k.value)

    def destroy(self):
        if self.h:
            self.lib.sph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
