"""Python handle on the FP64 CPU oracle (``orc.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow restatement of the
ternary free-energy entropic LBM update of arXiv:1710.07486 that the CUDA
library is checked against.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg import this module.  It never imports the
library package, and the library never imports it.

``build()`` compiles ``orc.c`` with the host C compiler into
``oracle/_build/liborc.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liborc.so")
OMP_LIB_PATH = os.path.join(BUILD_DIR, "liborc_omp.so")

D2Q9, D3Q27 = 0, 1
PERIODIC, BOUNCEBACK = 0, 1


class Params(C.Structure):
    """Mirror of ``orc_params`` (symbols follow Eqs. 2-4 and the text)."""

    _fields_ = [(n, C.c_double) for n in (
        "a", "b", "R", "T", "lambda1", "lambda2", "lambda3",
        "kappa1", "kappa2", "kappa3", "chi", "nu", "Gamma", "tau_g")] + [
        ("force_form", C.c_int), ("eos", C.c_int), ("omega", C.c_double), ("gamma_mode", C.c_int),
        ("solid", C.c_void_p), ("wet_rho", C.c_double), ("wet_phi", C.c_double)]


CS, VDW, PR = 0, 1, 2  # equations of state
GAMMA_CLOSED, GAMMA_EXACT = 0, 1  # stabiliser: closed form or exact root


class Eos(C.Structure):
    """Mirror of ``orc_eos``."""

    _fields_ = [("kind", C.c_int)] + [(n, C.c_double) for n in ("a", "b", "R", "T", "omega")]


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no fast-math) and return its path.
    ``openmp``: the timing copy of the same source with its loops over nodes
    spread over the host cores (``liborc_omp.so``); the tests use the plain,
    single-threaded build."""
    src = os.path.join(HERE, "orc.c")
    path = OMP_LIB_PATH if openmp else LIB_PATH
    if not force and os.path.exists(path) and \
            os.path.getmtime(path) >= max(os.path.getmtime(src),
                                          os.path.getmtime(os.path.join(HERE, "orc.h"))):
        return path
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared",
                           "-fno-fast-math", "-ffp-contract=off"] + (["-fopenmp"] if openmp else [])
                          + [src, "-o", tmp, "-lm"])
    os.replace(tmp, path)
    return path


_libs = {}


def lib(openmp: bool = False):
    """The oracle library: the plain single-threaded build, or (``openmp``)
    the timing copy that spreads the loops over nodes across the host cores."""
    if openmp not in _libs:
        L = C.CDLL(build(openmp=openmp))
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        d = C.c_double
        for name in ("orc_psi_tilde", "orc_dpsi_tilde", "orc_p_eos"):
            fn = getattr(L, name)
            fn.argtypes = [d, d, d, d, d]
            fn.restype = d
        L.orc_coexistence.argtypes = [d, d, d, d, dp]
        L.orc_coexistence.restype = C.c_int
        L.orc_critical_point.argtypes = [d, d, d, dp]
        L.orc_critical_point.restype = C.c_int
        L.orc_temperature_for_ratio.argtypes = [d, d, d, d, C.POINTER(d)]
        L.orc_temperature_for_ratio.restype = C.c_int
        for name in ("orc_eos_psi", "orc_eos_dpsi", "orc_eos_p"):
            fn = getattr(L, name)
            fn.argtypes = [C.POINTER(Eos), d]
            fn.restype = d
        L.orc_eos_coexistence.argtypes = [C.POINTER(Eos), dp]
        L.orc_eos_coexistence.restype = C.c_int
        L.orc_eos_critical_point.argtypes = [C.c_int, d, d, d, d, dp]
        L.orc_eos_critical_point.restype = C.c_int
        L.orc_eos_temperature_for_ratio.argtypes = [C.c_int, d, d, d, d, d, C.POINTER(d)]
        L.orc_eos_temperature_for_ratio.restype = C.c_int
        L.orc_pr_tc.argtypes = [d, d, d]
        L.orc_pr_tc.restype = d
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(Params), ip]
        L.orc_create.restype = C.c_void_p
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_destroy.restype = None
        L.orc_Q.argtypes = [C.c_void_p]
        L.orc_Q.restype = C.c_int
        L.orc_N.argtypes = [C.c_void_p]
        L.orc_N.restype = C.c_long
        L.orc_velocities.argtypes = [C.c_void_p, ip, dp]
        L.orc_velocities.restype = None
        L.orc_derived.argtypes = [C.c_void_p, dp]
        L.orc_derived.restype = None
        L.orc_f_bulk.argtypes = [C.c_void_p, d, d]
        L.orc_f_bulk.restype = d
        L.orc_feq.argtypes = [C.c_void_p, d, dp, dp]
        L.orc_feq.restype = None
        L.orc_collide_f.argtypes = [C.c_void_p, dp, dp, dp, C.c_void_p, C.POINTER(d)]
        L.orc_collide_f.restype = C.c_int
        L.orc_gamma_exact.argtypes = [C.c_void_p, dp, dp, dp, d, C.POINTER(d)]
        L.orc_gamma_exact.restype = C.c_int
        L.orc_gamma_fallbacks.argtypes = [C.c_void_p]
        L.orc_gamma_fallbacks.restype = C.c_long
        L.orc_geq.argtypes = [C.c_void_p, d, d, dp, dp]
        L.orc_geq.restype = None
        L.orc_collide_g.argtypes = [C.c_void_p, dp, d, d, dp, dp]
        L.orc_collide_g.restype = None
        for name in ("orc_stream", "orc_unstream", "orc_laplacian"):
            fn = getattr(L, name)
            fn.argtypes = [C.c_void_p, dp, dp]
            fn.restype = None
        L.orc_gradient.argtypes = [C.c_void_p, dp, dp]
        L.orc_gradient.restype = None
        L.orc_laplacian_wet.argtypes = [C.c_void_p, dp, C.c_double, dp]
        L.orc_laplacian_wet.restype = None
        L.orc_chem_pot.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.orc_chem_pot.restype = None
        L.orc_force.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        L.orc_force.restype = None
        L.orc_init.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        L.orc_init.restype = C.c_int
        L.orc_step.argtypes = [C.c_void_p, dp, dp, C.c_int]
        L.orc_step.restype = C.c_int
        L.orc_fields.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, C.c_void_p]
        L.orc_fields.restype = C.c_int
        _libs[openmp] = L
    return _libs[openmp]


def _f64(x, n=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


# ---------------------------------------------------------------- thermodynamics
def psi_tilde(a, b, R, T, rho):
    return lib().orc_psi_tilde(a, b, R, T, rho)


def dpsi_tilde(a, b, R, T, rho):
    return lib().orc_dpsi_tilde(a, b, R, T, rho)


def p_eos(a, b, R, T, rho):
    return lib().orc_p_eos(a, b, R, T, rho)


def coexistence(a, b, R, T):
    """(rho_g, rho_l, mu_coex, p_coex) of the common-tangent construction."""
    out = np.zeros(4)
    if lib().orc_coexistence(a, b, R, T, out) != 0:
        raise ValueError("no coexistence at this temperature")
    return tuple(float(v) for v in out)


def critical_point(a, b, R):
    out = np.zeros(2)
    if lib().orc_critical_point(a, b, R, out) != 0:
        raise ValueError("bad EOS constants")
    return float(out[0]), float(out[1])


def temperature_for_ratio(a, b, R, ratio):
    T = C.c_double()
    if lib().orc_temperature_for_ratio(a, b, R, ratio, C.byref(T)) != 0:
        raise ValueError("ratio out of range")
    return T.value


def _eos(kind, a, b, R, T, omega):
    return Eos(int(kind), float(a), float(b), float(R), float(T), float(omega))


def eos_psi(kind, a, b, R, T, rho, omega=0.0):
    return lib().orc_eos_psi(C.byref(_eos(kind, a, b, R, T, omega)), rho)


def eos_dpsi(kind, a, b, R, T, rho, omega=0.0):
    return lib().orc_eos_dpsi(C.byref(_eos(kind, a, b, R, T, omega)), rho)


def eos_p(kind, a, b, R, T, rho, omega=0.0):
    return lib().orc_eos_p(C.byref(_eos(kind, a, b, R, T, omega)), rho)


def eos_coexistence(kind, a, b, R, T, omega=0.0):
    out = np.zeros(4)
    if lib().orc_eos_coexistence(C.byref(_eos(kind, a, b, R, T, omega)), out) != 0:
        raise ValueError("no coexistence at this temperature")
    return tuple(float(v) for v in out)


def eos_critical_point(kind, a, b, R, omega=0.0):
    out = np.zeros(2)
    if lib().orc_eos_critical_point(int(kind), a, b, R, omega, out) != 0:
        raise ValueError("bad EOS constants")
    return float(out[0]), float(out[1])


def eos_temperature_for_ratio(kind, a, b, R, ratio, omega=0.0):
    T = C.c_double()
    if lib().orc_eos_temperature_for_ratio(int(kind), a, b, R, omega, ratio, C.byref(T)) != 0:
        raise ValueError("ratio out of range")
    return T.value


def pr_tc(a, b, R):
    return lib().orc_pr_tc(a, b, R)


# ---------------------------------------------------------------- lattice model
class Oracle:
    """One lattice (D2Q9 or D3Q27) with its parameters; state arrays are numpy
    float64 ``[Q, N]`` (post-collision populations)."""

    def __init__(self, lattice, nx, ny, nz, params: dict, bc=(0, 0, 0), openmp=False):
        self._L = lib(openmp)
        self.lattice = lattice
        self.nx, self.ny, self.nz = nx, ny, nz
        self.params = dict(params)
        ints = ("force_form", "eos", "omega", "gamma_mode", "solid", "wet_rho", "wet_phi")
        vals = {k: float(params[k]) for k, _ in Params._fields_ if k not in ints}
        solid = params.get("solid")
        self.solid = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).ravel()
        if self.solid is not None:
            assert self.solid.size == nx * ny * nz
        p = Params(force_form=int(params.get("force_form", 1)), eos=int(params.get("eos", CS)),
                   omega=float(params.get("omega", 0.0)),
                   gamma_mode=int(params.get("gamma_mode", GAMMA_CLOSED)),
                   solid=None if self.solid is None else self.solid.ctypes.data,
                   wet_rho=float(params.get("wet_rho", 0.0)), wet_phi=float(params.get("wet_phi", 0.0)), **vals)
        bca = np.asarray(bc, dtype=np.int32)
        self._h = self._L.orc_create(lattice, nx, ny, nz, C.byref(p), bca)
        if not self._h:
            raise ValueError("orc_create failed (bad lattice/size or no coexistence)")
        self.Q = self._L.orc_Q(self._h)
        self.N = self._L.orc_N(self._h)
        self.D = 2 if lattice == D2Q9 else 3
        c = np.zeros(27 * 3, dtype=np.int32)
        w = np.zeros(27)
        self._L.orc_velocities(self._h, c, w)
        self.c = c.reshape(27, 3)[: self.Q].copy()
        self.w = w[: self.Q].copy()
        der = np.zeros(6)
        self._L.orc_derived(self._h, der)
        (self.rho_g, self.rho_l, self.mu_coex, self.p_coex,
         self.tau, self.beta) = (float(v) for v in der)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    # single node
    def f_bulk(self, rho, phi):
        return self._L.orc_f_bulk(self._h, rho, phi)

    def feq(self, rho, u):
        out = np.zeros(self.Q)
        self._L.orc_feq(self._h, rho, _f64(np.resize(np.asarray(u, float), 3)), out)
        return out

    def collide_f(self, f, F):
        """Returns (f_post, delta_s, gamma)."""
        fo = np.zeros(self.Q)
        ds = np.zeros(self.Q)
        g = C.c_double()
        rc = self._L.orc_collide_f(self._h, _f64(f, self.Q),
                                 _f64(np.resize(np.asarray(F, float), 3)), fo,
                                 ds.ctypes.data_as(C.c_void_p), C.byref(g))
        if rc != 0:
            raise FloatingPointError(f"orc_collide_f rc={rc}")
        return fo, ds, g.value

    def gamma_exact(self, feq, ds, dh, gamma0):
        """(iterations or -1 on fallback, gamma) of the exact stabiliser."""
        g = C.c_double()
        it = self._L.orc_gamma_exact(self._h, _f64(feq, self.Q), _f64(ds, self.Q), _f64(dh, self.Q),
                                   float(gamma0), C.byref(g))
        return it, g.value

    def gamma_fallbacks(self):
        return int(self._L.orc_gamma_fallbacks(self._h))

    def geq(self, phi, mu_phi, u):
        out = np.zeros(self.Q)
        self._L.orc_geq(self._h, phi, mu_phi, _f64(np.resize(np.asarray(u, float), 3)), out)
        return out

    def collide_g(self, g, phi, mu_phi, u):
        out = np.zeros(self.Q)
        self._L.orc_collide_g(self._h, _f64(g, self.Q), phi, mu_phi,
                            _f64(np.resize(np.asarray(u, float), 3)), out)
        return out

    # lattice
    def stream(self, post):
        pre = np.zeros((self.Q, self.N))
        self._L.orc_stream(self._h, _f64(post, self.Q * self.N), pre)
        return pre

    def unstream(self, pre):
        post = np.zeros((self.Q, self.N))
        self._L.orc_unstream(self._h, _f64(pre, self.Q * self.N), post)
        return post

    def laplacian(self, psi, wet=None):
        """Isotropic Laplacian; with wet, the ghost rule of a density-like
        field with that wetting gradient (orc_laplacian_wet)."""
        out = np.zeros(self.N)
        if wet is None:
            self._L.orc_laplacian(self._h, _f64(psi, self.N), out)
        else:
            self._L.orc_laplacian_wet(self._h, _f64(psi, self.N), float(wet), out)
        return out

    def gradient(self, psi):
        out = np.zeros((3, self.N))
        self._L.orc_gradient(self._h, _f64(psi, self.N), out)
        return out

    def chem_pot(self, rho, phi):
        mr = np.zeros(self.N)
        mp = np.zeros(self.N)
        self._L.orc_chem_pot(self._h, _f64(rho, self.N), _f64(phi, self.N), mr, mp)
        return mr, mp

    def force(self, rho, phi, mu_rho, mu_phi):
        F = np.zeros((3, self.N))
        self._L.orc_force(self._h, _f64(rho, self.N), _f64(phi, self.N),
                        _f64(mu_rho, self.N), _f64(mu_phi, self.N), F)
        return F

    def init(self, rho, phi, u):
        f = np.zeros((self.Q, self.N))
        g = np.zeros((self.Q, self.N))
        rc = self._L.orc_init(self._h, _f64(rho, self.N), _f64(phi, self.N),
                            _f64(u, self.D * self.N), f, g)
        if rc != 0:
            raise FloatingPointError(f"orc_init rc={rc}")
        return f, g

    def step(self, f, g, nsteps=1):
        """Advance (f, g) in place; returns the status code (0 ok, -3 unstable)."""
        assert f.dtype == np.float64 and f.flags.c_contiguous
        assert g.dtype == np.float64 and g.flags.c_contiguous
        return self._L.orc_step(self._h, f, g, int(nsteps))

    def fields(self, f, g, with_p=True):
        rho = np.zeros(self.N)
        phi = np.zeros(self.N)
        u = np.zeros((self.D, self.N))
        p = np.zeros(self.N) if with_p else None
        rc = self._L.orc_fields(self._h, _f64(f, self.Q * self.N), _f64(g, self.Q * self.N),
                              rho, phi, u,
                              p.ctypes.data_as(C.c_void_p) if with_p else None)
        return {"rho": rho, "phi": phi, "u": u, "p": p, "rc": rc}
