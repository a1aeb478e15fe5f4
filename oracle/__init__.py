"""FP64 CPU oracle of the lattice-Boltzmann phase-field scheme (arXiv 1602.07483).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow restatement of the
paper's algorithm that the CUDA library is checked against.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the product path never does.  It shares no code with the CUDA library.

The C sources (``lbpf_oracle.c``, ``fd_oracle.c``) are compiled here with gcc,
``-O2 -ffp-contract=off`` and no fast-math, into ``_build/liblbpf_oracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["lbpf_oracle.c", "fd_oracle.c"]
_LIB = None
_LOCK = threading.Lock()


def lib_path(openmp: bool = True) -> str:
    return os.path.join(_HERE, "_build", "liblbpf_oracle%s.so" % ("_omp" if openmp else ""))


def build(openmp: bool = True, force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or older than its sources."""
    out = lib_path(openmp)
    srcs = [os.path.join(_HERE, s) for s in _SRCS] + [os.path.join(_HERE, "lbpf_oracle.h")]
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           "-o", tmp] + [os.path.join(_HERE, s) for s in _SRCS] + ["-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class Params(ctypes.Structure):
    _fields_ = [
        ("W0", ctypes.c_double), ("tau0", ctypes.c_double),
        ("D", ctypes.c_double), ("kappa", ctypes.c_double),
        ("lam", ctypes.c_double), ("Mc_inf", ctypes.c_double), ("k", ctypes.c_double),
        ("aniso", ctypes.c_int32), ("eps1", ctypes.c_double), ("eps2", ctypes.c_double),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("antitrapping", ctypes.c_int32), ("grad2_min", ctypes.c_double),
    ]


def make_params(**kw) -> Params:
    p = Params()
    d = dict(W0=1.0, tau0=1.0, D=2.0, kappa=1.0, lam=2.0 / 0.6267, Mc_inf=1.0, k=0.15,
             aniso=0, eps1=0.05, eps2=0.0, dx=0.8, dt=0.01, antitrapping=1, grad2_min=1e-12)
    if "lambda_" in kw:
        kw["lam"] = kw.pop("lambda_")
    d.update(kw)
    for key, v in d.items():
        setattr(p, key, v)
    return p


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def load(openmp: bool = True):
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        # a test may point the binding at another build of these sources
        path = os.environ.get("LBPF_ORACLE_LIB") or build(openmp)
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        L.ora_lattice.argtypes = [ctypes.c_int, _I, _D, _D, _D, _D, _I]
        L.ora_aniso.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]
        L.ora_aniso.restype = ctypes.c_double
        L.ora_geq.argtypes = [ctypes.c_int, ctypes.c_double, _D, ctypes.c_double, _D]
        L.ora_heq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, ctypes.c_double, _D]
        L.ora_create.argtypes = [ctypes.c_int] * 6 + [ctypes.POINTER(Params)]
        L.ora_create.restype = vp
        L.ora_destroy.argtypes = [vp]
        L.ora_init_seed.argtypes = [vp, ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double]
        L.ora_set_state.argtypes = [vp, _D, _D, _D, ctypes.c_double]
        L.ora_get_pops.argtypes = [vp, ctypes.c_int, _D]
        L.ora_get_fields.argtypes = [vp, _D, _D, _D]
        L.ora_get_usource.argtypes = [vp, _D]
        L.ora_step.argtypes = [vp, ctypes.c_int64]
        L.ora_sums.argtypes = [vp, _D]
        L.ora_tip.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.ora_tip.restype = ctypes.c_double
        L.ora_steps_done.argtypes = [vp]
        L.ora_steps_done.restype = ctypes.c_int64
        L.fd_create.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(Params)]
        L.fd_create.restype = vp
        L.fd_destroy.argtypes = [vp]
        L.fd_init_seed.argtypes = [vp, ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double]
        L.fd_step.argtypes = [vp, ctypes.c_int64]
        L.fd_get_fields.argtypes = [vp, _D, _D, _D]
        _LIB = L
        return L


def lattice(q: int):
    """Return (e[q,3] int, w, A, B, e2, opp) as typed from the paper's Tables 1-4 (2D lattices with e_z = 0)."""
    L = load()
    e = np.zeros((q, 3), np.int32)
    w, A, B = np.zeros(q), np.zeros(q), np.zeros(q)
    e2 = np.zeros(1)
    opp = np.zeros(q, np.int32)
    rc = L.ora_lattice(q, e.ctypes.data_as(_I), _ptr(w), _ptr(A), _ptr(B), _ptr(e2), opp.ctypes.data_as(_I))
    if rc:
        raise ValueError("bad lattice %d" % q)
    return e, w, A, B, float(e2[0]), opp


def aniso(kind: int, eps1: float, eps2: float, grad):
    L = load()
    g = np.ascontiguousarray(grad, dtype=np.float64)
    das = np.zeros(3)
    a = L.ora_aniso(kind, eps1, eps2, _ptr(g), _ptr(das))
    return a, das


def geq(q, phi, N, c):
    out = np.zeros(q)
    load().ora_geq(q, phi, _ptr(np.ascontiguousarray(N, np.float64)), c, _ptr(out))
    return out


def heq(q, U, qz, J, dt_dx):
    out = np.zeros(q)
    load().ora_heq(q, U, qz, _ptr(np.ascontiguousarray(J, np.float64)), dt_dx, _ptr(out))
    return out


class Sim:
    """One oracle simulation.  Fields are returned as [nz, ny, nx] arrays."""

    def __init__(self, shape, lattices=(15, 19, 0), params=None, **kw):
        self.nx, self.ny, self.nz = shape
        self.q_phi, self.q_u, self.q_theta = lattices
        self.params = params if params is not None else make_params(**kw)
        self._L = load()
        self._h = self._L.ora_create(self.nx, self.ny, self.nz, self.q_phi, self.q_u, self.q_theta,
                                     ctypes.byref(self.params))
        if not self._h:
            raise ValueError("ora_create failed")

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def close(self):
        if self._h:
            self._L.ora_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_seed(self, centres, radii, U0, theta0=0.0):
        c = np.ascontiguousarray(np.asarray(centres, np.float64).reshape(-1))
        r = np.ascontiguousarray(np.asarray(radii, np.float64).reshape(-1))
        self._L.ora_init_seed(self._h, len(r), _ptr(c), _ptr(r), U0, theta0)
        self.theta0 = theta0

    def set_state(self, g, h, f=None, theta0=0.0):
        g = np.ascontiguousarray(g, np.float64)
        h = np.ascontiguousarray(h, np.float64)
        fp = _ptr(np.ascontiguousarray(f, np.float64)) if f is not None else None
        self._L.ora_set_state(self._h, _ptr(g), _ptr(h), fp, theta0)

    def step(self, n=1):
        self._L.ora_step(self._h, n)

    def pops(self, field):
        q = (self.q_phi, self.q_u, self.q_theta)[field]
        out = np.zeros((q, self.nz, self.ny, self.nx))
        self._L.ora_get_pops(self._h, field, _ptr(out))
        return out

    def fields(self):
        shp = (self.nz, self.ny, self.nx)
        phi, U, th = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        self._L.ora_get_fields(self._h, _ptr(phi), _ptr(U), _ptr(th))
        return phi, U, th

    def usource(self):
        out = np.zeros((self.nz, self.ny, self.nx))
        self._L.ora_get_usource(self._h, _ptr(out))
        return out

    def sums(self):
        out = np.zeros(4)
        self._L.ora_sums(self._h, _ptr(out))
        return out

    def tip(self, c, axis=0):
        """Tip coordinate along +axis from node c and the tip radius (see ora_tip)."""
        rho = np.zeros(1)
        x = self._L.ora_tip(self._h, int(axis), int(c[0]), int(c[1]), int(c[2]), _ptr(rho))
        return x, float(rho[0])

    @property
    def steps_done(self):
        return self._L.ora_steps_done(self._h)


class FDSim:
    """Explicit finite-difference solve of the same PDEs (cross-check only)."""

    def __init__(self, shape, theta_evolves=False, params=None, **kw):
        self.nx, self.ny, self.nz = shape
        self.params = params if params is not None else make_params(**kw)
        self._L = load()
        self._h = self._L.fd_create(self.nx, self.ny, self.nz, int(theta_evolves), ctypes.byref(self.params))

    def close(self):
        if self._h:
            self._L.fd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_seed(self, centres, radii, U0, theta0=0.0):
        c = np.ascontiguousarray(np.asarray(centres, np.float64).reshape(-1))
        r = np.ascontiguousarray(np.asarray(radii, np.float64).reshape(-1))
        self._L.fd_init_seed(self._h, len(r), _ptr(c), _ptr(r), U0, theta0)

    def step(self, n=1):
        self._L.fd_step(self._h, n)

    def fields(self):
        shp = (self.nz, self.ny, self.nx)
        phi, U, th = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        self._L.fd_get_fields(self._h, _ptr(phi), _ptr(U), _ptr(th))
        return phi, U, th
