"""ctypes binding of the CUDA library (``include/lbpf.h``), argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
only converts Python arguments to the C structs and pointers of the ABI and
raises :class:`LbpfError` on a negative return code.  There is no CPU
fallback: :func:`load` raises when ``_lib/liblbpf.so`` is missing (build it
with ``python -m paper_1602_07483_gb300.build``) and :class:`Sim` raises
``LbpfError(LBPF_ECUDA)`` without a usable GPU.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbpf.so")

LBPF_OK, LBPF_EINVAL, LBPF_EUNSTABLE, LBPF_ENOMEM, LBPF_ENAN, LBPF_ETIMEOUT, LBPF_ECUDA = 0, -1, -2, -3, -4, -5, -6
STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
SCHEDULES = {"two_kernels": 0, "one_launch": 1}
LBPF_PHI, LBPF_U, LBPF_THETA = 1, 2, 4

_LIB = None
_LOCK = threading.Lock()


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class Lattice(ctypes.Structure):
    _fields_ = [("q_phi", ctypes.c_int32), ("q_u", ctypes.c_int32), ("q_theta", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [
        ("W0", ctypes.c_double), ("tau0", ctypes.c_double),
        ("D", ctypes.c_double), ("kappa", ctypes.c_double),
        ("lam", ctypes.c_double), ("Mc_inf", ctypes.c_double), ("k", ctypes.c_double),
        ("aniso", ctypes.c_int32), ("eps1", ctypes.c_double), ("eps2", ctypes.c_double),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("antitrapping", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("grad2_min", ctypes.c_double),
    ]


class LbpfError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = load().lbpf_strerror(code).decode() if _LIB is not None else str(code)
        super().__init__("%s: %s (%d)" % (what, msg, code))


_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


def load(path: str = LIB_PATH):
    """Load the library (raises OSError when it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if not os.path.exists(path):
            raise OSError("CUDA library not built: %s (run python -m paper_1602_07483_gb300.build)" % path)
        L = ctypes.CDLL(path)
        i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        sig = {
            "lbpf_create": ([ctypes.POINTER(Grid), ctypes.POINTER(Lattice), ctypes.POINTER(Params), _VP,
                             ctypes.POINTER(_VP)], ctypes.c_int),
            "lbpf_init_seed": ([_VP, i32, _D, _D, ctypes.c_double, ctypes.c_double], ctypes.c_int),
            "lbpf_set_state": ([_VP, _D, _D, _D, ctypes.c_double], ctypes.c_int),
            "lbpf_get_state": ([_VP, _D, _D, _D], ctypes.c_int),
            "lbpf_step": ([_VP, i64], ctypes.c_int),
            "lbpf_read_fields": ([_VP, u32, _D, _D, _D], ctypes.c_int),
            "lbpf_step_timed": ([_VP, i64, _D], ctypes.c_int),
            "lbpf_sums": ([_VP, _D], ctypes.c_int),
            "lbpf_tip": ([_VP, i32, _D, _D, _D], ctypes.c_int),
            "lbpf_steps_done": ([_VP], i64),
            "lbpf_save": ([_VP, ctypes.c_char_p], ctypes.c_int),
            "lbpf_load": ([_VP, ctypes.c_char_p], ctypes.c_int),
            "lbpf_set_tiling": ([_VP, i32, i32], ctypes.c_int),
            "lbpf_get_tiling": ([_VP, ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
            "lbpf_autotune": ([_VP, i32, _D], ctypes.c_int),
            "lbpf_set_schedule": ([_VP, i32], ctypes.c_int),
            "lbpf_set_wait_polls": ([_VP, i32], ctypes.c_int),
            "lbpf_get_schedule": ([_VP, ctypes.POINTER(i32)], ctypes.c_int),
            "lbpf_wait_probe": ([i32, i32, ctypes.POINTER(i32)], ctypes.c_int),
            "lbpf_destroy": ([_VP], ctypes.c_int),
            "lbpf_batch_create": ([i32, ctypes.POINTER(Grid), ctypes.POINTER(Lattice), ctypes.POINTER(Params), _VP,
                                   ctypes.POINTER(_VP)], ctypes.c_int),
            "lbpf_batch_member": ([_VP, i32, ctypes.POINTER(_VP)], ctypes.c_int),
            "lbpf_batch_from_sims": ([i32, ctypes.POINTER(_VP), _VP, ctypes.POINTER(_VP)], ctypes.c_int),
            "lbpf_batch_step": ([_VP, i64], ctypes.c_int),
            "lbpf_batch_set_tiling": ([_VP, i32, i32], ctypes.c_int),
            "lbpf_batch_get_tiling": ([_VP, ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
            "lbpf_batch_autotune": ([_VP, i32, _D], ctypes.c_int),
            "lbpf_batch_set_schedule": ([_VP, i32], ctypes.c_int),
            "lbpf_batch_get_schedule": ([_VP, ctypes.POINTER(i32)], ctypes.c_int),
            "lbpf_batch_destroy": ([_VP], ctypes.c_int),
            "lbpf_strerror": ([ctypes.c_int], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
        return L


def _check(rc, what):
    if rc != LBPF_OK:
        raise LbpfError(rc, what)


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def make_params(storage="f64", **kw) -> Params:
    p = Params()
    d = dict(W0=1.0, tau0=1.0, D=2.0, kappa=1.0, lam=2.0 / 0.6267, Mc_inf=1.0, k=0.15, aniso=0, eps1=0.05,
             eps2=0.0, dx=0.8, dt=0.05, antitrapping=1, grad2_min=1e-12)
    d.update(kw)
    for key, v in d.items():
        setattr(p, key, v)
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    return p


class Sim:
    """One simulation on the current CUDA device (see ``lbpf_create``)."""

    def __init__(self, shape, lattices=(19, 19, 0), storage="f64", stream=None, params=None, _handle=None, **kw):
        self._L = load()
        self.nx, self.ny, self.nz = (int(v) for v in shape)
        self.q = tuple(int(v) for v in lattices)
        self.params = params if params is not None else make_params(storage, **kw)
        self._owned = _handle is None
        if _handle is not None:  # a batch member: the batch owns the handle
            self._h = _handle
            return
        h = _VP()
        rc = self._L.lbpf_create(ctypes.byref(Grid(self.nx, self.ny, self.nz)), ctypes.byref(Lattice(*self.q)),
                                 ctypes.byref(self.params), _VP(stream) if stream else None, ctypes.byref(h))
        _check(rc, "lbpf_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def shape3(self):
        return (self.nz, self.ny, self.nx)

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                self._L.lbpf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_seed(self, centres, radii, U0, theta0=0.0):
        c = np.ascontiguousarray(np.asarray(centres, np.float64).reshape(-1))
        r = np.ascontiguousarray(np.asarray(radii, np.float64).reshape(-1))
        _check(self._L.lbpf_init_seed(self._h, len(r), _dptr(c), _dptr(r), U0, theta0), "lbpf_init_seed")

    def set_state(self, g, h, f=None, theta0=0.0):
        g = np.ascontiguousarray(g, np.float64)
        h = np.ascontiguousarray(h, np.float64)
        f = None if f is None else np.ascontiguousarray(f, np.float64)
        _check(self._L.lbpf_set_state(self._h, _dptr(g), _dptr(h), _dptr(f), theta0), "lbpf_set_state")

    def get_state(self):
        out = [np.zeros((q,) + self.shape3) if q else None for q in self.q]
        _check(self._L.lbpf_get_state(self._h, *[_dptr(a) for a in out]), "lbpf_get_state")
        return out

    def step(self, n=1):
        _check(self._L.lbpf_step(self._h, int(n)), "lbpf_step")

    def step_timed(self, n=1):
        """Run n steps with per-kernel CUDA events; return (ms_phi, ms_uth, ms_span) in total."""
        out = np.zeros(3)
        _check(self._L.lbpf_step_timed(self._h, int(n), _dptr(out)), "lbpf_step_timed")
        return tuple(out)

    def read_fields(self, mask=LBPF_PHI | LBPF_U | LBPF_THETA, out=None):
        if out is None:
            out = [np.empty(self.shape3) if mask & m else None for m in (LBPF_PHI, LBPF_U, LBPF_THETA)]
        _check(self._L.lbpf_read_fields(self._h, mask, *[_dptr(a) for a in out]), "lbpf_read_fields")
        return out

    def sums(self, check=True):
        out = np.zeros(4)
        rc = self._L.lbpf_sums(self._h, _dptr(out))
        if check:
            _check(rc, "lbpf_sums")
        return out

    def tip(self, centre, axis=0):
        """Tip coordinate along +axis from the node nearest `centre` and the tip radius."""
        c = (ctypes.c_double * 3)(*[float(v) for v in centre])
        x, rho = ctypes.c_double(), ctypes.c_double()
        _check(self._L.lbpf_tip(self._h, int(axis), c, ctypes.byref(x), ctypes.byref(rho)), "lbpf_tip")
        return x.value, rho.value

    @property
    def steps_done(self):
        return int(self._L.lbpf_steps_done(self._h))

    def save(self, path):
        _check(self._L.lbpf_save(self._h, os.fsencode(path)), "lbpf_save")

    def load_checkpoint(self, path):
        _check(self._L.lbpf_load(self._h, os.fsencode(path)), "lbpf_load")

    def set_tiling(self, by=0, zchunk=0):
        _check(self._L.lbpf_set_tiling(self._h, by, zchunk), "lbpf_set_tiling")

    def get_tiling(self):
        by, zc = ctypes.c_int32(), ctypes.c_int32()
        _check(self._L.lbpf_get_tiling(self._h, ctypes.byref(by), ctypes.byref(zc)), "lbpf_get_tiling")
        return by.value, zc.value

    def autotune(self, steps=4):
        ms = ctypes.c_double()
        _check(self._L.lbpf_autotune(self._h, steps, ctypes.byref(ms)), "lbpf_autotune")
        return ms.value

    def set_schedule(self, schedule):
        """``"two_kernels"`` or ``"one_launch"`` (``lbpf_set_schedule``)."""
        _check(self._L.lbpf_set_schedule(self._h, SCHEDULES[schedule]), "lbpf_set_schedule")

    def set_wait_polls(self, polls):
        """Bound of each one-launch wait (``lbpf_set_wait_polls``)."""
        _check(self._L.lbpf_set_wait_polls(self._h, int(polls)), "lbpf_set_wait_polls")

    @property
    def schedule(self):
        v = ctypes.c_int32()
        _check(self._L.lbpf_get_schedule(self._h, ctypes.byref(v)), "lbpf_get_schedule")
        return {c: n for n, c in SCHEDULES.items()}[v.value]


class Batch:
    """Several simulations advanced together (see ``lbpf_batch_create``).

    ``Batch(sims)`` batches existing :class:`Sim` handles (``lbpf_batch_from_sims``);
    ``Batch.create(...)`` lets the library create and own the members."""

    def __init__(self, sims, stream=None, _handle=None):
        self._L = load()
        self.sims = list(sims)
        if _handle is not None:
            self._h = _handle
            return
        arr = (_VP * len(self.sims))(*[s.handle for s in self.sims])
        h = _VP()
        _check(self._L.lbpf_batch_from_sims(len(self.sims), arr, _VP(stream) if stream else None, ctypes.byref(h)),
               "lbpf_batch_from_sims")
        self._h = h

    @classmethod
    def create(cls, shapes, lattices, params, stream=None):
        """n members from per-member shapes (nx, ny, nz), one lattice triple and per-member
        :class:`Params` (``lbpf_batch_create``); members are :class:`Sim` views of handles
        the batch owns."""
        L = load()
        n = len(shapes)
        grids = (Grid * n)(*[Grid(*[int(v) for v in s]) for s in shapes])
        lats = (Lattice * n)(*[Lattice(*[int(v) for v in lattices]) for _ in range(n)])
        pars = (Params * n)(*params)
        h = _VP()
        _check(L.lbpf_batch_create(n, grids, lats, pars, _VP(stream) if stream else None, ctypes.byref(h)),
               "lbpf_batch_create")
        sims = []
        for i in range(n):
            m = _VP()
            _check(L.lbpf_batch_member(h, i, ctypes.byref(m)), "lbpf_batch_member")
            sims.append(Sim(shapes[i], lattices, params=params[i], _handle=m))
        return cls(sims, _handle=h)

    def step(self, n=1):
        _check(self._L.lbpf_batch_step(self._h, int(n)), "lbpf_batch_step")

    def set_tiling(self, by=0, zchunk=0):
        _check(self._L.lbpf_batch_set_tiling(self._h, int(by), int(zchunk)), "lbpf_batch_set_tiling")

    def get_tiling(self):
        by, zc = ctypes.c_int32(), ctypes.c_int32()
        _check(self._L.lbpf_batch_get_tiling(self._h, ctypes.byref(by), ctypes.byref(zc)), "lbpf_batch_get_tiling")
        return by.value, zc.value

    def autotune(self, steps=12):
        """Fastest tiling kept, state unchanged (``lbpf_batch_autotune``); ms per step."""
        ms = ctypes.c_double()
        _check(self._L.lbpf_batch_autotune(self._h, int(steps), ctypes.byref(ms)), "lbpf_batch_autotune")
        return ms.value

    def set_schedule(self, schedule):
        """``"two_kernels"`` or ``"one_launch"`` (``lbpf_batch_set_schedule``)."""
        _check(self._L.lbpf_batch_set_schedule(self._h, SCHEDULES[schedule]), "lbpf_batch_set_schedule")

    @property
    def schedule(self):
        v = ctypes.c_int32()
        _check(self._L.lbpf_batch_get_schedule(self._h, ctypes.byref(v)), "lbpf_batch_get_schedule")
        return {c: n for n, c in SCHEDULES.items()}[v.value]

    def close(self):
        if getattr(self, "_h", None):
            for s in self.sims:
                if not s._owned:  # views of handles the batch destroys
                    s._h = None
            self._L.lbpf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wait_probe(flag_value, polls):
    """The step's bounded wait on its own (``lbpf_wait_probe``): True if it saw the flag."""
    seen = ctypes.c_int32()
    _check(load().lbpf_wait_probe(int(flag_value), int(polls), ctypes.byref(seen)), "lbpf_wait_probe")
    return bool(seen.value)


def batch_from_workloads(ws, storage=None, stream=None):
    """A library-owned batch (``lbpf_batch_create``) of the given workloads, each seeded."""
    b = Batch.create([w.grid for w in ws], ws[0].lattices,
                     [make_params(storage or w.storage, **w.params) for w in ws], stream=stream)
    for w, s in zip(ws, b.sims):
        s.init_seed(w.centres, w.radii, w.U0, w.theta0)
    return b


def sim_from_workload(w, storage=None, stream=None):
    """Create and seed a :class:`Sim` from a :class:`workloads.Workload`."""
    s = Sim(w.grid, w.lattices, storage=storage or w.storage, stream=stream, **w.params)
    s.init_seed(w.centres, w.radii, w.U0, w.theta0)
    return s
