"""The allocation-free sums entry point (lbpf_field_sums_noalloc), called through
the C ABI on device arrays, must agree with lbpf_sums.

That entry point is for callers that cannot allocate device memory (stream
capture in progress, loops that must not trigger cudaMalloc's implicit
synchronisation, or memory fully reserved by another allocator); it reduces in
a file-scope device array instead.  The check runs two calls in a row because
the scratch keeps the previous call's contents.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1602_07483_gb300 import build, lbpf, workloads

pytestmark = pytest.mark.gpu


def _bind():
    build.build()
    L = lbpf.load()
    f = L.lbpf_field_sums_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                  ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _call(f, phi, U, th, storage, n, k, theta0):
    out = np.zeros(4)
    rc = f(phi.data_ptr(), U.data_ptr(), th.data_ptr() if th is not None else None, storage, n, k, theta0,
           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    return rc, out


@pytest.mark.parametrize("storage,lat_case", [("f32", "coupled"), ("f64", "frozen_theta")])
def test_noalloc_sums_match_lbpf_sums_on_two_calls(storage, lat_case):
    torch = pytest.importorskip("torch")
    f = _bind()
    w = workloads.coupled_dendrite(n=40) if lat_case == "coupled" else workloads.small_dendrite()
    sim = lbpf.sim_from_workload(w, storage=storage)
    dt = torch.float64 if storage == "f64" else torch.float32
    code = lbpf.STORAGE[storage]
    for _ in range(2):
        sim.step(7)
        ref = sim.sums()
        phi, U, th = sim.read_fields()
        tp = torch.tensor(phi, dtype=dt, device="cuda")
        tu = torch.tensor(U, dtype=dt, device="cuda")
        tt = torch.tensor(th, dtype=dt, device="cuda") if w.lattices[2] else None
        torch.cuda.synchronize()
        rc, out = _call(f, tp, tu, tt, code, w.sites, w.params["k"], w.theta0)
        assert rc == 0
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-9)


def test_noalloc_rejects_oversized_input():
    torch = pytest.importorskip("torch")
    f = _bind()
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    rc, _ = _call(f, t, t, None, 1, 268435456 + 1, 0.15, 0.0)  # LBPF_NOALLOC_MAX_SITES + 1
    assert rc == lbpf.LBPF_EINVAL
    rc, _ = _call(f, t, t, None, 1, 0, 0.15, 0.0)
    assert rc == lbpf.LBPF_EINVAL
