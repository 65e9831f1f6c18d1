"""ctypes binding of libdg (include/dg.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of libdg.so.  The functions keep the C names (dg_init, dg_step, dg_torque,
dg_fetch, ...); `Disc` bundles them around one handle.  Device memory comes
from PyTorch's caching allocator (one workspace tensor handed to
dg_init_ex) and work is issued on PyTorch's current CUDA stream, unless the
caller asks otherwise.  There is no CPU fallback: without the built library or
a CUDA device every call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

DG_OK = 0
DG_ERR_ARG = -1
DG_ERR_UNSUPPORTED = -2
DG_ERR_CUDA = -3
DG_ERR_NUMERIC = -4
DG_ERR_TIMEOUT = -5
DG_ERR_NOMEM = -6

EXPORTED = ["dg_init", "dg_init_ex", "dg_workspace_bytes", "dg_step", "dg_step_dt", "dg_sync",
            "dg_rhs", "dg_torque", "dg_torque_series", "dg_fetch", "dg_set_state", "dg_get_time",
            "dg_set_state_async", "dg_torque_async",
            "dg_conserved", "dg_set_stream", "dg_shape", "dg_destroy", "dg_last_error",
            "dg_set_timing", "dg_timing", "dg_conserved_static", "dg_batch_create",
            "dg_batch_config", "dg_batch_get_config", "dg_batch_tune", "dg_batch_step",
            "dg_batch_sync", "dg_batch_destroy", "dg_indicator", "dg_limit", "dg_limit_flags",
            "dg_last_flags", "dg_mlp_create", "dg_mlp_destroy", "dg_mlp_nparams", "dg_mlp_get_params",
            "dg_mlp_set_params", "dg_mlp_forward", "dg_mlp_grad", "dg_mlp_train_step", "dg_features",
            "dg_set_indicator", "dg_indicator_logits", "dg_selftest_wait", "dg_prec_tiles",
            "dg_set_delta_async", "dg_fetch_delta"]


class DgMesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("bc", ctypes.c_int)]


class DgEos(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("gamma", ctypes.c_double), ("h", ctypes.c_double)]


class DgPlanet(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("r_p", ctypes.c_double), ("eps", ctypes.c_double),
                ("omega_p", ctypes.c_double), ("phi0", ctypes.c_double), ("enabled", ctypes.c_int)]


class DgDisc(ctypes.Structure):
    _fields_ = [("ic", ctypes.c_int), ("star", ctypes.c_int), ("r_soft", ctypes.c_double),
                ("sigma_slope", ctypes.c_double), ("sigma_floor", ctypes.c_double),
                ("noise_amp", ctypes.c_double), ("seed", ctypes.c_ulonglong),
                ("rdamp_in", ctypes.c_double), ("rdamp_out", ctypes.c_double),
                ("cfl", ctypes.c_double), ("rk", ctypes.c_int), ("prec", ctypes.c_int),
                ("amp", ctypes.c_double), ("vx0", ctypes.c_double), ("vy0", ctypes.c_double),
                ("limiter", ctypes.c_int), ("tvb_m", ctypes.c_double), ("positivity", ctypes.c_int),
                ("ring_r", ctypes.c_double), ("ring_p", ctypes.c_double)]


_DP = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_lib = None


def lib_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libdg.so (building it in-tree with nvcc if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libdg.so is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        P = ctypes.POINTER
        L.dg_init.argtypes = [P(_VP), P(DgMesh), ctypes.c_int, P(DgEos), P(DgPlanet), P(DgDisc)]
        L.dg_init_ex.argtypes = [P(_VP), P(DgMesh), ctypes.c_int, P(DgEos), P(DgPlanet), P(DgDisc),
                                 _VP, ctypes.c_size_t, _VP]
        L.dg_workspace_bytes.argtypes = [P(DgMesh), ctypes.c_int, P(DgEos), P(DgDisc),
                                         P(ctypes.c_size_t)]
        L.dg_step.argtypes = [_VP, ctypes.c_int]
        L.dg_step_dt.argtypes = [_VP, ctypes.c_int, ctypes.c_double]
        L.dg_sync.argtypes = [_VP]
        L.dg_rhs.argtypes = [_VP, _DP]
        L.dg_torque.argtypes = [_VP, _DP]
        L.dg_torque_series.argtypes = [_VP, _DP, ctypes.c_int, P(ctypes.c_int)]
        L.dg_fetch.argtypes = [_VP, _DP]
        L.dg_set_state.argtypes = [_VP, _DP, ctypes.c_double, ctypes.c_long]
        L.dg_set_state_async.argtypes = [_VP, _DP, ctypes.c_double, ctypes.c_long]
        L.dg_torque_async.argtypes = [_VP, _DP]
        L.dg_get_time.argtypes = [_VP, _DP, _DP, P(ctypes.c_long)]
        L.dg_conserved.argtypes = [_VP, _DP]
        L.dg_set_stream.argtypes = [_VP, _VP]
        L.dg_shape.argtypes = [_VP, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                               P(ctypes.c_int)]
        L.dg_destroy.argtypes = [_VP]
        L.dg_set_timing.argtypes = [_VP, ctypes.c_int]
        L.dg_timing.argtypes = [_VP, _DP, P(ctypes.c_longlong)]
        L.dg_conserved_static.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_double, _VP, _VP]
        L.dg_last_error.argtypes = [_VP]
        L.dg_last_error.restype = ctypes.c_char_p
        L.dg_indicator.argtypes = [_VP, ctypes.c_double, _VP]
        L.dg_limit.argtypes = [_VP]
        L.dg_limit_flags.argtypes = [_VP, _VP]
        L.dg_last_flags.argtypes = [_VP, _VP]
        L.dg_mlp_create.argtypes = [P(_VP), ctypes.c_int, ctypes.c_ulonglong]
        L.dg_mlp_destroy.argtypes = [_VP]
        L.dg_mlp_nparams.argtypes = [_VP, P(ctypes.c_int)]
        L.dg_mlp_get_params.argtypes = [_VP, _VP]
        L.dg_mlp_set_params.argtypes = [_VP, _VP]
        L.dg_mlp_forward.argtypes = [_VP, _VP, ctypes.c_int, _VP, _VP]
        L.dg_mlp_grad.argtypes = [_VP, _VP, _VP, ctypes.c_int, ctypes.c_float, _VP, _DP, _VP]
        L.dg_mlp_train_step.argtypes = [_VP, _VP, _VP, ctypes.c_int, ctypes.c_float, ctypes.c_float, _DP, _VP]
        L.dg_features.argtypes = [_VP, _VP, ctypes.c_int, _VP]
        L.dg_set_indicator.argtypes = [_VP, _VP, ctypes.c_float]
        L.dg_indicator_logits.argtypes = [_VP, _VP, _VP]
        L.dg_batch_create.argtypes = [P(_VP), P(_VP), ctypes.c_int]
        L.dg_batch_config.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.dg_batch_get_config.argtypes = [_VP, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                                          P(ctypes.c_int)]
        L.dg_batch_tune.argtypes = [_VP, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
                                    P(ctypes.c_int), P(ctypes.c_int), _DP]
        L.dg_batch_step.argtypes = [_VP, ctypes.c_int]
        L.dg_batch_sync.argtypes = [_VP]
        L.dg_batch_destroy.argtypes = [_VP]
        L.dg_selftest_wait.argtypes = [ctypes.c_int, P(ctypes.c_int)]
        L.dg_prec_tiles.argtypes = [_VP, P(ctypes.c_longlong), P(ctypes.c_longlong), P(ctypes.c_longlong)]
        L.dg_set_delta_async.argtypes = [_VP, _VP, ctypes.c_double, ctypes.c_long]
        L.dg_fetch_delta.argtypes = [_VP, _VP]
        _lib = L
    return _lib


class DgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libdg error %d: %s" % (code, msg))
        self.code = code


def _check(rc, h=None):
    if rc != DG_OK:
        raise DgError(rc, (lib().dg_last_error(h) or b"").decode())
    return rc


def _fill(cls, d):
    s = cls()
    for name, _ in cls._fields_:
        if name in d:
            setattr(s, name, d[name])
    return s


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def structs(cfg):
    return (_fill(DgMesh, cfg["mesh"]), int(cfg["order"]), _fill(DgEos, cfg["eos"]),
            _fill(DgPlanet, cfg["planet"]), _fill(DgDisc, cfg["disc"]))


def dg_workspace_bytes(cfg):
    mesh, order, eos, _, disc = structs(cfg)
    n = ctypes.c_size_t()
    _check(lib().dg_workspace_bytes(ctypes.byref(mesh), order, ctypes.byref(eos), ctypes.byref(disc),
                                    ctypes.byref(n)))
    return n.value


class Disc:
    """One DG problem on the GPU (a dg_handle)."""

    def __init__(self, cfg, torch_memory=True, stream=None):
        L = lib()
        self.cfg = cfg
        mesh, order, eos, planet, disc = structs(cfg)
        self._structs = (mesh, eos, planet, disc)
        self.order = order
        self.nv = 4 if eos.kind == 1 else 3
        self.m = order + 1
        self.M = self.m * self.m
        self.nx, self.ny = mesh.nx, mesh.ny
        self.shape = (self.nv, self.M, self.ny, self.nx)
        h = _VP()
        self._ws = None
        if torch_memory:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: libdg has no CPU path")
            nbytes = dg_workspace_bytes(cfg)
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            _check(L.dg_init_ex(ctypes.byref(h), ctypes.byref(mesh), order, ctypes.byref(eos),
                                ctypes.byref(planet), ctypes.byref(disc),
                                ctypes.c_void_p(self._ws.data_ptr()), nbytes,
                                ctypes.c_void_p(stream or 0)))
        else:
            _check(L.dg_init(ctypes.byref(h), ctypes.byref(mesh), order, ctypes.byref(eos),
                             ctypes.byref(planet), ctypes.byref(disc)))
        self.h = h
        self._keep = []  # host arrays that queued asynchronous copies still read

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            lib().dg_destroy(self.h)
            self.h = None
        self._ws = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls ---------------------------------------------------------------
    def step(self, n=1):
        _check(lib().dg_step(self.h, n), self.h)

    def step_dt(self, n, dt):
        _check(lib().dg_step_dt(self.h, n, dt), self.h)

    def sync(self):
        _check(lib().dg_sync(self.h), self.h)
        self._keep = []

    def set_state_async(self, coeffs, t=0.0, step=0):
        """dg_set_state_async: `coeffs`, a C-contiguous float64 array of the
        state's shape in page-locked memory (e.g. a pinned torch tensor's
        .numpy()), is kept referenced until the next sync()."""
        if coeffs.size != int(np.prod(self.shape)):
            raise ValueError("set_state_async: the array must hold the full state")
        _check(lib().dg_set_state_async(self.h, _ptr(coeffs), t, step), self.h)
        self._keep.append(coeffs)

    def set_delta_async(self, delta, t=0.0, step=0):
        """dg_set_delta_async (precision form): `delta`, a C-contiguous float32
        array of the state's shape in page-locked memory, is kept referenced
        until the next sync()."""
        if not (delta.dtype == np.float32 and delta.flags["C_CONTIGUOUS"] and
                delta.size == int(np.prod(self.shape))):
            raise ValueError("set_delta_async: a C-contiguous float32 array of the state's shape")
        _check(lib().dg_set_delta_async(self.h, delta.ctypes.data_as(_VP), t, step), self.h)
        self._keep.append(delta)

    def fetch_delta(self, out=None):
        """dg_fetch_delta (precision form): delta = u - u_b as float32 values
        at the Gauss-Legendre nodes, index q*m + r along the mode axis."""
        if out is None:
            out = np.empty(self.shape, dtype=np.float32)
        _check(lib().dg_fetch_delta(self.h, out.ctypes.data_as(_VP)), self.h)
        return out

    def torque_async(self, out, index=0):
        """dg_torque_async into out[index] (a float64 array in page-locked
        memory), valid after the next sync()."""
        if not (out.dtype == np.float64 and out.flags["C_CONTIGUOUS"] and 0 <= index < out.size):
            raise ValueError("torque_async: a C-contiguous float64 array and an index inside it")
        _check(lib().dg_torque_async(self.h, ctypes.cast(out.ctypes.data + 8 * index, _DP)), self.h)
        self._keep.append(out)

    def rhs(self):
        out = np.empty(self.shape)
        _check(lib().dg_rhs(self.h, _ptr(out)), self.h)
        return out

    def torque(self):
        g = ctypes.c_double()
        _check(lib().dg_torque(self.h, ctypes.byref(g)), self.h)
        return g.value

    def torque_series(self, cap=65536):
        out = np.empty(cap)
        n = ctypes.c_int()
        _check(lib().dg_torque_series(self.h, _ptr(out), cap, ctypes.byref(n)), self.h)
        return out[:n.value].copy()

    def fetch(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        _check(lib().dg_fetch(self.h, _ptr(out)), self.h)
        return out

    def indicator(self, M):
        """TVB troubled-cell flags of the current state, uint8 [ny, nx]."""
        out = np.zeros((self.ny, self.nx), dtype=np.uint8)
        _check(lib().dg_indicator(self.h, M, out.ctypes.data_as(_VP)), self.h)
        return out

    def limit(self):
        _check(lib().dg_limit(self.h), self.h)

    def limit_flags(self, flags):
        f = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self.ny, self.nx)
        _check(lib().dg_limit_flags(self.h, f.ctypes.data_as(_VP)), self.h)

    def last_flags(self):
        out = np.zeros((self.ny, self.nx), dtype=np.uint8)
        _check(lib().dg_last_flags(self.h, out.ctypes.data_as(_VP)), self.h)
        return out

    def features(self, elems):
        """FP32 features [n, 5 nv M] (a torch CUDA tensor) of the elements
        `elems` (a torch int32 CUDA tensor of indices j*nx + i)."""
        import torch
        _device_tensor(elems, torch.int32, (elems.numel(),), "elems")
        nin = 5 * self.nv * self.M
        out = torch.empty((elems.numel(), nin), dtype=torch.float32, device=elems.device)
        _check(lib().dg_features(self.h, _VP(elems.data_ptr()), elems.numel(), _VP(out.data_ptr())), self.h)
        return out

    def set_indicator(self, net, threshold=0.0):
        _check(lib().dg_set_indicator(self.h, net.net if net is not None else None, threshold), self.h)

    def indicator_logits(self):
        z = np.zeros((self.ny, self.nx), dtype=np.float32)
        f = np.zeros((self.ny, self.nx), dtype=np.uint8)
        _check(lib().dg_indicator_logits(self.h, z.ctypes.data_as(_VP), f.ctypes.data_as(_VP)), self.h)
        return z, f

    def set_state(self, coeffs, t=0.0, step=0):
        c = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(self.shape)
        _check(lib().dg_set_state(self.h, _ptr(c), t, step), self.h)

    def get_time(self):
        t = ctypes.c_double()
        dt = ctypes.c_double()
        st = ctypes.c_long()
        _check(lib().dg_get_time(self.h, ctypes.byref(t), ctypes.byref(dt), ctypes.byref(st)),
               self.h)
        return t.value, dt.value, st.value

    def conserved(self):
        out = np.empty(self.nv)
        _check(lib().dg_conserved(self.h, _ptr(out)), self.h)
        return out

    def set_timing(self, enable=True):
        _check(lib().dg_set_timing(self.h, 1 if enable else 0), self.h)

    def timing(self):
        """(sum of stage-kernel milliseconds, number of stage launches) since the last call."""
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        _check(lib().dg_timing(self.h, ctypes.byref(ms), ctypes.byref(n)), self.h)
        return ms.value, n.value

    def prec_tiles(self):
        """Precision form: (tiles, tiles that keep R_b, tiles touching a damping zone)."""
        n, r, z = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().dg_prec_tiles(self.h, ctypes.byref(n), ctypes.byref(r), ctypes.byref(z)), self.h)
        return n.value, r.value, z.value

    def set_stream(self, stream):
        _check(lib().dg_set_stream(self.h, ctypes.c_void_p(stream or 0)), self.h)


# C-named entry points
def dg_init(cfg, **kw):
    return Disc(cfg, **kw)


def dg_step(d, n=1):
    d.step(n)


def dg_step_dt(d, n, dt):
    d.step_dt(n, dt)


def dg_torque(d):
    return d.torque()


def dg_torque_series(d, cap=65536):
    return d.torque_series(cap)


def dg_fetch(d, out=None):
    return d.fetch(out)


def dg_set_state(d, coeffs, t=0.0, step=0):
    d.set_state(coeffs, t, step)


def dg_get_time(d):
    return d.get_time()


def dg_conserved(d):
    return d.conserved()


def dg_rhs(d):
    return d.rhs()


def dg_sync(d):
    d.sync()


def dg_set_timing(d, enable=True):
    d.set_timing(enable)


def dg_timing(d):
    return d.timing()


def dg_conserved_static(coeffs, dx, dy, out, stream=None):
    """Allocation-free conserved sums of a canonical FP64 device tensor `coeffs`
    of shape (nv, nmodes, ny, nx) into the FP64 device tensor `out` (nv values,
    on the same device), enqueued on `stream` (default: PyTorch's current
    stream of that device).  The call is made with coeffs' device current.
    Raises DgError on a bad argument or a CUDA failure."""
    import torch
    nv, nmodes, ny, nx = coeffs.shape
    assert coeffs.dtype == torch.float64 and coeffs.is_cuda and coeffs.is_contiguous()
    assert out.dtype == torch.float64 and out.is_cuda and out.numel() >= nv
    assert out.device == coeffs.device, "coeffs and out on different devices"
    with torch.cuda.device(coeffs.device):
        if stream is None:
            stream = torch.cuda.current_stream(coeffs.device).cuda_stream
        rc = lib().dg_conserved_static(ctypes.c_void_p(coeffs.data_ptr()), nv, nmodes, nx, ny, dx, dy,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream or 0))
    if rc != DG_OK:
        raise DgError(rc, "dg_conserved_static")


def dg_destroy(d):
    d.close()


class Batch:
    """Several precision-form discs advanced together (a dg_batch).  The discs
    must outlive the batch; after batched steps each Disc is used as usual."""

    POLICIES = ("given", "costliest-first", "row-interleaved")

    def __init__(self, discs):
        L = lib()
        self.discs = list(discs)
        arr = (_VP * len(self.discs))(*[d.h for d in self.discs])
        b = _VP()
        _check(L.dg_batch_create(ctypes.byref(b), arr, len(self.discs)))
        self.b = b

    def config(self, policy=1, dynamic=1, ctas_per_sm=0, tiles_per_item=1):
        """dynamic: 0 one CTA per tile, 1 persistent CTAs in each stage launch,
        2 one persistent launch per step (flow schedule, work items of
        tiles_per_item tiles from a queue counter), 3 the same with the
        queue positions dealt round-robin over the CTAs."""
        _check(lib().dg_batch_config(self.b, policy, dynamic, ctas_per_sm, tiles_per_item))

    def get_config(self):
        p, d, c, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().dg_batch_get_config(self.b, ctypes.byref(p), ctypes.byref(d), ctypes.byref(c),
                                         ctypes.byref(t)))
        return {"policy": p.value, "dynamic": d.value, "ctas_per_sm": c.value, "tiles_per_item": t.value}

    def tune(self, steps=3):
        p, d, c, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_double()
        _check(lib().dg_batch_tune(self.b, steps, ctypes.byref(p), ctypes.byref(d), ctypes.byref(c),
                                   ctypes.byref(t), ctypes.byref(ms)))
        return {"policy": p.value, "dynamic": d.value, "ctas_per_sm": c.value, "tiles_per_item": t.value,
                "ms_per_step": ms.value}

    def step(self, n=1):
        _check(lib().dg_batch_step(self.b, n))

    def sync(self):
        _check(lib().dg_batch_sync(self.b))

    def close(self):
        if getattr(self, "b", None):
            lib().dg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _device_tensor(t, dtype, shape, name):
    """The kernels read a tensor through its data pointer alone: refuse one of
    another dtype, shape or device, or one that is not contiguous, before its
    pointer is passed on."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}, "
                         f"got {t.dtype} {tuple(t.shape)}")


class Mlp:
    """The learned troubled-cell indicator's network (a dg_mlp): training and
    inference run in libdg's kernels; batches are torch CUDA tensors."""

    def __init__(self, nin, seed=0):
        net = _VP()
        _check(lib().dg_mlp_create(ctypes.byref(net), nin, seed))
        self.net = net
        self.nin = nin
        n = ctypes.c_int()
        _check(lib().dg_mlp_nparams(net, ctypes.byref(n)))
        self.nparams = n.value

    @staticmethod
    def _stream():
        import torch
        return _VP(torch.cuda.current_stream().cuda_stream)

    def _check_batch(self, x, y):
        import torch
        _device_tensor(x, torch.float32, (x.shape[0], self.nin), "x")
        _device_tensor(y, torch.float32, (x.shape[0],), "y")

    def get_params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        _check(lib().dg_mlp_get_params(self.net, p.ctypes.data_as(_VP)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        _check(lib().dg_mlp_set_params(self.net, p.ctypes.data_as(_VP)))

    def forward(self, x):
        import torch
        _device_tensor(x, torch.float32, (x.shape[0], self.nin), "x")
        z = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        _check(lib().dg_mlp_forward(self.net, _VP(x.data_ptr()), x.shape[0], _VP(z.data_ptr()), self._stream()))
        return z

    def grad(self, x, y, pos_weight=1.0):
        self._check_batch(x, y)
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().dg_mlp_grad(self.net, _VP(x.data_ptr()), _VP(y.data_ptr()), x.shape[0], pos_weight,
                                 g.ctypes.data_as(_VP), ctypes.byref(loss), self._stream()))
        return g, loss.value

    def train_step(self, x, y, pos_weight=1.0, lr=1e-3):
        self._check_batch(x, y)
        loss = ctypes.c_double()
        _check(lib().dg_mlp_train_step(self.net, _VP(x.data_ptr()), _VP(y.data_ptr()), x.shape[0], pos_weight,
                                       lr, ctypes.byref(loss), self._stream()))
        return loss.value

    def close(self):
        if getattr(self, "net", None):
            lib().dg_mlp_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
