"""ctypes wrapper of the FP64 CPU oracle (oracle/dg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline / reference arm.  The product package never imports
it, and it imports nothing from the product package.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class RefMesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("bc", ctypes.c_int)]


class RefEos(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("gamma", ctypes.c_double), ("h", ctypes.c_double)]


class RefPlanet(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("r_p", ctypes.c_double), ("eps", ctypes.c_double),
                ("omega_p", ctypes.c_double), ("phi0", ctypes.c_double), ("enabled", ctypes.c_int)]


class RefDisc(ctypes.Structure):
    _fields_ = [("ic", ctypes.c_int), ("star", ctypes.c_int), ("r_soft", ctypes.c_double),
                ("sigma_slope", ctypes.c_double), ("sigma_floor", ctypes.c_double),
                ("noise_amp", ctypes.c_double), ("seed", ctypes.c_ulonglong),
                ("rdamp_in", ctypes.c_double), ("rdamp_out", ctypes.c_double),
                ("cfl", ctypes.c_double), ("rk", ctypes.c_int), ("prec", ctypes.c_int),
                ("amp", ctypes.c_double), ("vx0", ctypes.c_double), ("vy0", ctypes.c_double),
                ("limiter", ctypes.c_int), ("tvb_m", ctypes.c_double), ("positivity", ctypes.c_int),
                ("ring_r", ctypes.c_double), ("ring_p", ctypes.c_double)]


_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        L.ref_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(RefMesh), ctypes.c_int,
                               ctypes.POINTER(RefEos), ctypes.POINTER(RefPlanet),
                               ctypes.POINTER(RefDisc)]
        L.ref_destroy.argtypes = [vp]
        L.ref_step.argtypes = [vp, ctypes.c_int]
        L.ref_step_dt.argtypes = [vp, ctypes.c_int, ctypes.c_double]
        L.ref_rhs.argtypes = [vp, _DP]
        L.ref_cfl_dt.argtypes = [vp, _DP]
        L.ref_damp.argtypes = [vp, ctypes.c_double]
        L.ref_torque.argtypes = [vp, _DP, _DP]
        L.ref_torque_now.argtypes = [vp, ctypes.c_double, _DP, _DP]
        L.ref_indicator.argtypes = [vp, ctypes.c_double, ctypes.c_void_p]
        L.ref_limit.argtypes = [vp]
        L.ref_limit_flags.argtypes = [vp, ctypes.c_void_p]
        L.ref_step_so.argtypes = [vp, ctypes.c_int]
        L.ref_fetch.argtypes = [vp, _DP]
        L.ref_set_state.argtypes = [vp, _DP, ctypes.c_double, ctypes.c_long]
        L.ref_get_time.argtypes = [vp, _DP, _DP, ctypes.POINTER(ctypes.c_long)]
        L.ref_nodal.argtypes = [vp, _DP]
        L.ref_ghosts.argtypes = [vp, _DP]
        L.ref_l1_wave.argtypes = [vp, ctypes.c_double, ctypes.c_int, _DP]
        L.ref_gauss_legendre.argtypes = [ctypes.c_int, _DP, _DP]
        L.ref_legendre.argtypes = [ctypes.c_int, ctypes.c_double, _DP, _DP]
        L.ref_splitmix64_uniform.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong, _DP]
        L.ref_rk_linear.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _DP, _DP]
        L.ref_nthreads.argtypes = []
        L.ref_set_threads.argtypes = [ctypes.c_int]
        L.ref_set_threads.restype = None
        _lib = L
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def gauss_legendre(m):
    x = np.zeros(m)
    w = np.zeros(m)
    _check(lib().ref_gauss_legendre(m, _ptr(x), _ptr(w)), "gauss_legendre")
    return x, w


def legendre(n, x):
    P = np.zeros(n + 1)
    dP = np.zeros(n + 1)
    _check(lib().ref_legendre(n, float(x), _ptr(P), _ptr(dP)), "legendre")
    return P, dP


def splitmix64_uniform(seed, counter):
    u = ctypes.c_double()
    lib().ref_splitmix64_uniform(seed, counter, ctypes.byref(u))
    return u.value


def rk_linear(rk, a, b, dt):
    re = ctypes.c_double()
    im = ctypes.c_double()
    _check(lib().ref_rk_linear(rk, a, b, dt, ctypes.byref(re), ctypes.byref(im)), "rk_linear")
    return complex(re.value, im.value)


def nthreads():
    return lib().ref_nthreads()


def set_threads(n):
    """Threads of the oracle's element loops (results are independent of it)."""
    lib().ref_set_threads(int(n))


def _fill(struct_cls, d):
    s = struct_cls()
    for name, _ in struct_cls._fields_:
        if name in d:
            setattr(s, name, d[name])
    return s


class Oracle:
    """One oracle problem instance; `cfg` is a dict with keys mesh/order/eos/planet/disc
    (the same parameter dicts the product binding takes)."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.mesh = _fill(RefMesh, cfg["mesh"])
        self.eos = _fill(RefEos, cfg["eos"])
        self.planet = _fill(RefPlanet, cfg["planet"])
        self.disc = _fill(RefDisc, cfg["disc"])
        self.order = int(cfg["order"])
        self.m = self.order + 1
        self.M = self.m * self.m
        self.nv = 4 if self.eos.kind == 1 else 3
        self.shape = (self.nv, self.M, self.mesh.ny, self.mesh.nx)
        h = ctypes.c_void_p()
        _check(lib().ref_init(ctypes.byref(h), ctypes.byref(self.mesh), self.order,
                              ctypes.byref(self.eos), ctypes.byref(self.planet),
                              ctypes.byref(self.disc)), "init")
        self.h = h

    def close(self):
        if self.h:
            lib().ref_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        _check(lib().ref_step(self.h, n), "step")

    def step_dt(self, n, dt):
        _check(lib().ref_step_dt(self.h, n, dt), "step_dt")

    def rhs(self):
        out = np.zeros(self.shape)
        _check(lib().ref_rhs(self.h, _ptr(out)), "rhs")
        return out

    def cfl_dt(self):
        d = ctypes.c_double()
        _check(lib().ref_cfl_dt(self.h, ctypes.byref(d)), "cfl_dt")
        return d.value

    def damp(self, dt):
        _check(lib().ref_damp(self.h, dt), "damp")

    def indicator(self, M):
        """TVB-minmod troubled-cell flags of the current state, uint8 [ny, nx]."""
        out = np.zeros((self.mesh.ny, self.mesh.nx), dtype=np.uint8)
        _check(lib().ref_indicator(self.h, M, out.ctypes.data_as(ctypes.c_void_p)), "indicator")
        return out

    def limit(self):
        _check(lib().ref_limit(self.h), "limit")

    def limit_flags(self, flags):
        f = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self.mesh.ny, self.mesh.nx)
        _check(lib().ref_limit_flags(self.h, f.ctypes.data_as(ctypes.c_void_p)), "limit_flags")

    def step_so(self, n=1):
        _check(lib().ref_step_so(self.h, n), "step_so")

    def torque(self):
        g = ctypes.c_double()
        a = ctypes.c_double()
        _check(lib().ref_torque(self.h, ctypes.byref(g), ctypes.byref(a)), "torque")
        return g.value, a.value

    def torque_now(self, t):
        g = ctypes.c_double()
        a = ctypes.c_double()
        _check(lib().ref_torque_now(self.h, t, ctypes.byref(g), ctypes.byref(a)), "torque_now")
        return g.value, a.value

    def fetch(self):
        out = np.zeros(self.shape)
        _check(lib().ref_fetch(self.h, _ptr(out)), "fetch")
        return out

    def set_state(self, coeffs, t=0.0, step=0):
        c = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(self.shape)
        _check(lib().ref_set_state(self.h, _ptr(c), t, step), "set_state")

    def get_time(self):
        t = ctypes.c_double()
        dt = ctypes.c_double()
        st = ctypes.c_long()
        _check(lib().ref_get_time(self.h, ctypes.byref(t), ctypes.byref(dt), ctypes.byref(st)),
               "get_time")
        return t.value, dt.value, st.value

    def nodal(self):
        out = np.zeros(self.shape)
        _check(lib().ref_nodal(self.h, _ptr(out)), "nodal")
        return out

    def ghosts(self):
        nx, ny = self.mesh.nx, self.mesh.ny
        n = self.nv * self.M
        out = np.zeros(n * (2 * ny + 2 * nx))
        _check(lib().ref_ghosts(self.h, _ptr(out)), "ghosts")
        a = n * ny
        return (out[:a].reshape(self.nv, self.M, ny), out[a:2 * a].reshape(self.nv, self.M, ny),
                out[2 * a:2 * a + n * nx].reshape(self.nv, self.M, nx),
                out[2 * a + n * nx:].reshape(self.nv, self.M, nx))

    def l1_wave(self, t, var=0):
        e = ctypes.c_double()
        _check(lib().ref_l1_wave(self.h, t, var, ctypes.byref(e)), "l1_wave")
        return e.value
