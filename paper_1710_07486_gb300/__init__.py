"""Python binding of libternelbm: the ternary free-energy entropic lattice
Boltzmann update of arXiv:1710.07486 on GB300 (sm_103a).

Argument marshalling only: every step of the update runs in the CUDA kernels
of ``libternelbm.so`` (C ABI in ``include/ternelbm.h``).  There is no CPU
fallback: if the library cannot be built or loaded, ``lib()`` raises.

PyTorch is optional and only used to hand device buffers and streams to the
library (``init_device``, ``fields_device``, ``set_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["Lattice", "lib", "coexistence", "temperature_for_ratio", "TelError",
           "D2Q9", "D3Q27", "FP64", "FP32_SHIFTED", "PERIODIC", "BOUNCEBACK",
           "FORCE_POTENTIAL", "FORCE_LATTICE", "GAMMA_CLOSED", "GAMMA_EXACT", "GAMMA_CLOSED_F64SUM"]

D2Q9, D3Q27 = 0, 1
FP64, FP32_SHIFTED = 0, 1
PERIODIC, BOUNCEBACK = 0, 1
FORCE_POTENTIAL, FORCE_LATTICE = 0, 1
GAMMA_CLOSED, GAMMA_EXACT, GAMMA_CLOSED_F64SUM = 0, 1, 2
EOS_CS, EOS_VDW, EOS_PR = 0, 1, 2
MOMENTS_CARRIED, MOMENTS_PULLED = 0, 1

TEL_OK, TEL_EINVAL, TEL_ENOMEM, TEL_ECUDA, TEL_EUNSTABLE, TEL_ESTATE = 0, -1, -2, -3, -4, -5
_NAMES = {-1: "TEL_EINVAL", -2: "TEL_ENOMEM", -3: "TEL_ECUDA", -4: "TEL_EUNSTABLE", -5: "TEL_ESTATE"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libternelbm.so")


class TelError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    """Mirror of ``tel_params``."""

    _fields_ = [(n, C.c_double) for n in (
        "a", "b", "R", "T", "lambda1", "lambda2", "lambda3", "kappa1", "kappa2",
        "kappa3", "chi", "nu", "Gamma", "tau_g", "rho_ref")] + [
        ("precision", C.c_int), ("force_form", C.c_int), ("bc", C.c_int * 3), ("eos", C.c_int),
        ("omega", C.c_double), ("gamma_mode", C.c_int), ("solid", C.c_void_p),
        ("wet_rho", C.c_double), ("wet_phi", C.c_double), ("moments", C.c_int)]


_lib = None
SYMBOLS = ("tel_create", "tel_destroy", "tel_last_error", "tel_set_stream", "tel_init",
           "tel_init_device", "tel_step", "tel_sync", "tel_gamma_fallbacks", "tel_fields", "tel_fields_device",
           "tel_get_state", "tel_set_state", "tel_info", "tel_coexistence",
           "tel_temperature_for_ratio", "tel_coexistence_eos", "tel_temperature_for_ratio_eos",
           "tel_fields_noalloc", "tel_batch_create",
           "tel_batch_destroy", "tel_batch_last_error", "tel_batch_set_stream", "tel_batch_init", "tel_batch_init_device", "tel_batch_step",
           "tel_batch_sync", "tel_batch_fields", "tel_batch_fields_device", "tel_batch_errors",
           "tel_batch_tune", "tel_batch_info")


def lib(build: bool = True):
    """Load libternelbm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        from . import build as _b
        _b.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libternelbm.so not found at {LIB_PATH}; run paper_1710_07486_gb300/build.py")
    L = C.CDLL(LIB_PATH)
    vp, d, i = C.c_void_p, C.c_double, C.c_int
    dp = C.POINTER(C.c_double)
    L.tel_create.argtypes = [i, i, i, i, C.POINTER(Params), C.POINTER(vp)]
    L.tel_destroy.argtypes = [vp]
    L.tel_destroy.restype = None
    L.tel_last_error.argtypes = [vp]
    L.tel_last_error.restype = C.c_char_p
    L.tel_set_stream.argtypes = [vp, vp]
    for name in ("tel_init", "tel_init_device"):
        getattr(L, name).argtypes = [vp, vp, vp, vp]
    L.tel_step.argtypes = [vp, i]
    L.tel_sync.argtypes = [vp]
    L.tel_gamma_fallbacks.argtypes = [vp, C.POINTER(C.c_ulonglong)]
    for name in ("tel_fields", "tel_fields_device"):
        getattr(L, name).argtypes = [vp, vp, vp, vp, vp]
    L.tel_get_state.argtypes = [vp, vp, vp]
    L.tel_set_state.argtypes = [vp, vp, vp]
    L.tel_info.argtypes = [vp, dp]
    L.tel_coexistence.argtypes = [d, d, d, d, dp]
    L.tel_temperature_for_ratio.argtypes = [d, d, d, d, dp]
    L.tel_coexistence_eos.argtypes = [i, d, d, d, d, d, dp]
    L.tel_temperature_for_ratio_eos.argtypes = [i, d, d, d, d, d, dp]
    L.tel_fields_noalloc.argtypes = [i, i, i, i, C.POINTER(Params), vp, vp, vp, vp, vp, vp, vp]
    L.tel_batch_create.argtypes = [i, vp, vp, vp, C.POINTER(vp)]
    L.tel_batch_destroy.argtypes = [vp]
    L.tel_batch_destroy.restype = None
    L.tel_batch_last_error.argtypes = [vp]
    L.tel_batch_last_error.restype = C.c_char_p
    L.tel_batch_set_stream.argtypes = [vp, vp]
    L.tel_batch_init.argtypes = [vp, i, vp, vp, vp]
    L.tel_batch_init_device.argtypes = [vp, i, vp, vp, vp]
    L.tel_batch_step.argtypes = [vp, i]
    L.tel_batch_sync.argtypes = [vp]
    L.tel_batch_fields.argtypes = [vp, i, vp, vp, vp, vp]
    L.tel_batch_fields_device.argtypes = [vp, i, vp, vp, vp, vp]
    L.tel_batch_errors.argtypes = [vp, vp]
    L.tel_batch_tune.argtypes = [vp, i, vp]
    L.tel_batch_info.argtypes = [vp, dp]
    for name in SYMBOLS:
        if name not in ("tel_destroy", "tel_last_error", "tel_batch_destroy", "tel_batch_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def coexistence(a, b, R, T, eos=0, omega=0.0):
    """(rho_g, rho_l, mu_coex, p_coex) of the common tangent; eos: EOS_CS
    (Eq. 4), EOS_VDW or EOS_PR (omega: acentric factor)."""
    out = (C.c_double * 4)()
    rc = lib().tel_coexistence_eos(int(eos), a, b, R, T, float(omega), out)
    if rc:
        raise TelError(rc, f"no liquid-gas coexistence at T={T}")
    return tuple(out)


def temperature_for_ratio(a, b, R, ratio, eos=0, omega=0.0):
    T = C.c_double()
    rc = lib().tel_temperature_for_ratio_eos(int(eos), a, b, R, float(omega), ratio, C.byref(T))
    if rc:
        raise TelError(rc, f"no temperature with density ratio {ratio}")
    return T.value


NOALLOC_MAX_NODES = 262144


def _params_struct(p):
    s = Params()
    for k in ("a", "b", "R", "T", "lambda1", "lambda2", "lambda3", "kappa1", "kappa2",
              "kappa3", "chi", "nu", "Gamma", "tau_g"):
        setattr(s, k, float(p[k]))
    s.rho_ref = float(p.get("rho_ref", 0.0))
    s.precision = int(p.get("precision", FP64))
    s.force_form = int(p.get("force_form", FORCE_LATTICE))
    bcs = tuple(p.get("bc", (0, 0, 0)))
    for k in range(3):
        s.bc[k] = int(bcs[k])
    s.eos = int(p.get("eos", EOS_CS))
    s.omega = float(p.get("omega", 0.0))
    s.gamma_mode = int(p.get("gamma_mode", GAMMA_CLOSED))
    s.wet_rho = float(p.get("wet_rho", 0.0))
    s.wet_phi = float(p.get("wet_phi", 0.0))
    s.moments = int(p.get("moments", MOMENTS_CARRIED))
    solid = p.get("solid")
    if solid is not None:
        # kept alive on the struct until the call that copies it returns
        s._solid = np.ascontiguousarray(solid, dtype=np.uint8).ravel()
        s.solid = s._solid.ctypes.data
    return s


def fields_noalloc(lattice, nx, ny, nz, params, f_state, g_state, with_p=True, stream=None):
    """Fields of a state held in the caller's own device buffers (torch
    tensors or raw device pointers), without any allocation by the library:
    for callers that keep the device's memory to themselves.  At most
    NOALLOC_MAX_NODES nodes.  Returns host numpy arrays like Lattice.fields."""
    D = 2 if lattice == D2Q9 else 3
    N = nx * ny * (1 if lattice == D2Q9 else nz)
    ptr = lambda t: C.c_void_p(t if isinstance(t, int) else t.data_ptr())
    rho, phi = np.empty(N), np.empty(N)
    u = np.empty((D, N))
    p = np.empty(N) if with_p else None
    raw = None
    if stream is not None:
        raw = getattr(stream, "cuda_stream", stream)
    s = _params_struct(params)
    rc = lib().tel_fields_noalloc(int(lattice), int(nx), int(ny), int(nz), C.byref(s), ptr(f_state),
                                  ptr(g_state), _ptr(rho), _ptr(phi), _ptr(u), _ptr(p),
                                  C.c_void_p(raw) if raw else None)
    if rc:
        raise TelError(rc, lib().tel_last_error(None).decode())
    return {"rho": rho, "phi": phi, "u": u, "p": p}


class Batch:
    """Many independent D2Q9 lattices (own sizes and parameters, one precision)
    advanced together: one persistent kernel launch per step.

    ``shapes``: list of (nx, ny); ``params``: one dict or a list of dicts, as
    for Lattice (bc along z is ignored).
    """

    def __init__(self, shapes, params):
        shapes = [(int(a), int(b)) for a, b in shapes]
        n = len(shapes)
        plist = params if isinstance(params, (list, tuple)) else [params] * n
        if len(plist) != n:
            raise ValueError("one parameter dict per case")
        P = (Params * n)(*[_params_struct(p) for p in plist])
        nx = (C.c_int * n)(*[a for a, _ in shapes])
        ny = (C.c_int * n)(*[b for _, b in shapes])
        self._L = lib()
        h = C.c_void_p()
        rc = self._L.tel_batch_create(n, nx, ny, P, C.byref(h))
        if rc:
            raise TelError(rc, self._L.tel_batch_last_error(None).decode())
        self._h = h
        self.shapes = shapes
        self.ncases = n

    def _check(self, rc):
        if rc:
            raise TelError(rc, self._L.tel_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.tel_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        """``stream``: a torch.cuda.Stream (not the default stream), a raw
        cudaStream_t int, or None for the batch's own stream."""
        raw = None
        if stream is not None:
            raw = getattr(stream, "cuda_stream", stream)
        self._check(self._L.tel_batch_set_stream(self._h, C.c_void_p(raw) if raw else None))

    def init(self, c, rho, phi, u):
        nx, ny = self.shapes[c]
        N = nx * ny
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (rho, phi, u)]
        if a[0].size != N or a[1].size != N or a[2].size != 2 * N:
            raise ValueError(f"case {c}: expected fields of {N}, {N} and {2 * N} values")
        self._check(self._L.tel_batch_init(self._h, int(c), _ptr(a[0]), _ptr(a[1]), _ptr(a[2])))

    def init_device(self, c, rho, phi, u):
        """Case c from device float64 tensors of N, N and 2N elements
        (asynchronous on the batch's stream)."""
        nx, ny = self.shapes[c]
        N = nx * ny
        for t, n in ((rho, N), (phi, N), (u, 2 * N)):
            if t.numel() != n or not t.is_contiguous() or str(t.dtype) != "torch.float64" or not t.is_cuda:
                raise ValueError("init_device wants contiguous CUDA float64 tensors")
        self._check(self._L.tel_batch_init_device(self._h, int(c), C.c_void_p(rho.data_ptr()),
                                                  C.c_void_p(phi.data_ptr()), C.c_void_p(u.data_ptr())))

    def step(self, n=1):
        self._check(self._L.tel_batch_step(self._h, int(n)))

    def sync(self):
        self._check(self._L.tel_batch_sync(self._h))

    def tune(self, steps_per_config=5):
        """Times every tile width / chunk length on real steps (which advance
        the state) and keeps the fastest.  Returns (tile width, chunk, steps)."""
        out = (C.c_int * 3)()
        self._check(self._L.tel_batch_tune(self._h, int(steps_per_config), out))
        return tuple(out)

    def info(self):
        out = (C.c_double * 6)()
        self._check(self._L.tel_batch_info(self._h, out))
        keys = ("ncases", "nodes", "tile_x", "chunk", "items", "ctas")
        return {k: int(v) for k, v in zip(keys, out)}

    def fields_device(self, c, rho=None, phi=None, u=None, p=None):
        """Case c's fields into device float64 tensors (asynchronous on the
        batch's stream)."""
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._check(self._L.tel_batch_fields_device(self._h, int(c), ptr(rho), ptr(phi), ptr(u), ptr(p)))

    def errors(self):
        """Per-case error words (0 = stable), cleared after reading."""
        out = (C.c_uint * self.ncases)()
        self._check(self._L.tel_batch_errors(self._h, out))
        return list(out)

    def fields(self, c, with_p=True):
        nx, ny = self.shapes[c]
        N = nx * ny
        rho, phi, u = np.empty(N), np.empty(N), np.empty((2, N))
        p = np.empty(N) if with_p else None
        self._check(self._L.tel_batch_fields(self._h, int(c), _ptr(rho), _ptr(phi), _ptr(u), _ptr(p)))
        return {"rho": rho, "phi": phi, "u": u, "p": p}


class Lattice:
    """One lattice state on the current CUDA device.

    ``params``: dict with a, b, R, T, lambda1..3, kappa1..3, chi, nu, Gamma,
    tau_g and optionally rho_ref, precision, force_form, bc.
    """

    def __init__(self, lattice, nx, ny, nz=1, params=None, bc=None, precision=None,
                 force_form=None):
        p = dict(params or {})
        if bc is not None:
            p["bc"] = bc
        if precision is not None:
            p["precision"] = precision
        if force_form is not None:
            p["force_form"] = force_form
        if p.get("solid") is not None and np.asarray(p["solid"]).size != nx * ny * nz:
            raise ValueError(f"solid mask: expected {nx * ny * nz} values")
        s = _params_struct(p)
        self._L = lib()
        h = C.c_void_p()
        rc = self._L.tel_create(int(lattice), int(nx), int(ny), int(nz), C.byref(s), C.byref(h))
        if rc:
            raise TelError(rc, self._L.tel_last_error(None).decode())
        self._h = h
        info = (C.c_double * 10)()
        self._L.tel_info(self._h, info)
        self.D, self.Q = int(info[0]), int(info[1])
        self.nx, self.ny, self.nz = int(info[2]), int(info[3]), int(info[4])
        self.N = int(info[5])
        self.rho_g, self.rho_l, self.mu_coex, self.p_coex = info[6], info[7], info[8], info[9]
        self.precision = s.precision
        self.lattice = int(lattice)

    # ------------------------------------------------------------------ utils
    def _check(self, rc):
        if rc:
            raise TelError(rc, self._L.tel_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.tel_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f64(self, a, n):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.size != n:
            raise ValueError(f"expected {n} values, got {a.size}")
        return a

    # --------------------------------------------------------------- host API
    def init(self, rho, phi, u):
        rho = self._f64(rho, self.N)
        phi = self._f64(phi, self.N)
        u = self._f64(u, self.D * self.N)
        self._check(self._L.tel_init(self._h, _ptr(rho), _ptr(phi), _ptr(u)))

    def step(self, n=1):
        self._check(self._L.tel_step(self._h, int(n)))

    def sync(self):
        self._check(self._L.tel_sync(self._h))

    def gamma_fallbacks(self):
        """Nodes whose exact stabiliser fell back to the closed form so far."""
        n = C.c_ulonglong()
        self._check(self._L.tel_gamma_fallbacks(self._h, C.byref(n)))
        return int(n.value)

    def fields(self, with_p=True):
        rho = np.empty(self.N)
        phi = np.empty(self.N)
        u = np.empty((self.D, self.N))
        p = np.empty(self.N) if with_p else None
        self._check(self._L.tel_fields(self._h, _ptr(rho), _ptr(phi), _ptr(u), _ptr(p)))
        return {"rho": rho, "phi": phi, "u": u, "p": p}

    def get_state(self):
        f = np.empty((self.Q, self.N))
        g = np.empty((self.Q, self.N))
        self._check(self._L.tel_get_state(self._h, _ptr(f), _ptr(g)))
        return f, g

    def set_state(self, f, g):
        f = self._f64(f, self.Q * self.N)
        g = self._f64(g, self.Q * self.N)
        self._check(self._L.tel_set_state(self._h, _ptr(f), _ptr(g)))

    # ------------------------------------------------------------- device API
    def set_stream(self, stream=None):
        """``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        raw = None
        if stream is not None:
            raw = getattr(stream, "cuda_stream", stream)
        self._check(self._L.tel_set_stream(self._h, C.c_void_p(raw) if raw else None))

    def init_device(self, rho, phi, u):
        """Device float64 tensors (torch) of N, N and D*N elements."""
        for t, n in ((rho, self.N), (phi, self.N), (u, self.D * self.N)):
            if t.numel() != n or not t.is_contiguous() or str(t.dtype) != "torch.float64" or not t.is_cuda:
                raise ValueError("init_device wants contiguous CUDA float64 tensors")
        self._check(self._L.tel_init_device(self._h, C.c_void_p(rho.data_ptr()),
                                            C.c_void_p(phi.data_ptr()), C.c_void_p(u.data_ptr())))

    def fields_device(self, rho=None, phi=None, u=None, p=None):
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._check(self._L.tel_fields_device(self._h, ptr(rho), ptr(phi), ptr(u), ptr(p)))
