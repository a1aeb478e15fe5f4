"""The allocation-free sums entry point (lbpf_field_sums_noalloc), called through
the C ABI on device arrays, must agree with lbpf_sums.

That entry point is for callers that cannot allocate device memory (loops that
must not trigger cudaMalloc's implicit synchronisation, or memory fully reserved
by another allocator); it reduces in a file-scope device array instead.  The
check runs two calls in a row because the scratch keeps the previous call's
contents.  This file is collected last.
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


def _call(f, phi, U, th, storage, n, k, theta0, stream=None):
    out = np.zeros(4)
    rc = f(phi.data_ptr(), U.data_ptr(), th.data_ptr() if th is not None else None, storage, n, k, theta0,
           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), stream)
    return rc, out


@pytest.mark.parametrize("storage,lat_case,side", [("f32", "coupled", False), ("f64", "frozen_theta", False),
                                                   ("f16", "coupled", True), ("bf16", "coupled", False),
                                                   ("f32", "frozen_theta", True)])
def test_noalloc_sums_match_lbpf_sums_on_two_calls(storage, lat_case, side):
    """Every storage code (the FP16/BF16 codes take the FP32 fields their simulations keep),
    theta given or NULL with a non-zero frozen theta0, on the legacy stream or a side stream."""
    torch = pytest.importorskip("torch")
    f = _bind()
    if lat_case == "coupled":
        w = workloads.coupled_dendrite(n=40)
    else:
        w = workloads.small_dendrite().with_(theta0=-0.3 if storage != "f64" else 0.0)
    sim = lbpf.sim_from_workload(w, storage=storage)
    dt = torch.float64 if storage == "f64" else torch.float32
    code = lbpf.STORAGE[storage]
    st = torch.cuda.Stream() if side else None
    for _ in range(2):
        sim.step(7)
        ref = sim.sums()
        phi, U, th = sim.read_fields()
        tp = torch.tensor(phi, dtype=dt, device="cuda")
        tu = torch.tensor(U, dtype=dt, device="cuda")
        tt = torch.tensor(th, dtype=dt, device="cuda") if w.lattices[2] else None
        torch.cuda.synchronize()
        rc, out = _call(f, tp, tu, tt, code, w.sites, w.params["k"], w.theta0,
                        stream=st.cuda_stream if st is not None else None)
        assert rc == 0
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-9)


def test_noalloc_refuses_a_capturing_stream():
    """The call reads its result back to the host, which a stream under capture does not
    allow: it returns LBPF_EINVAL and enqueues nothing, so the caller's capture survives."""
    torch = pytest.importorskip("torch")
    f = _bind()
    t = torch.ones(64, dtype=torch.float32, device="cuda")
    y = torch.zeros(64, dtype=torch.float32, device="cuda")
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        g.capture_begin()
        rc, _ = _call(f, t, t, None, 1, 64, 0.15, 0.0, stream=st.cuda_stream)
        y.add_(t)
        g.capture_end()
    assert rc == lbpf.LBPF_EINVAL
    g.replay()
    torch.cuda.synchronize()
    assert float(y.sum()) == 64.0
    rc, out = _call(f, t, t, None, 1, 64, 0.15, 0.0)
    assert rc == 0 and out[0] == 64.0


def test_noalloc_rejects_oversized_input():
    torch = pytest.importorskip("torch")
    f = _bind()
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    rc, _ = _call(f, t, t, None, 1, 268435456 + 1, 0.15, 0.0)  # LBPF_NOALLOC_MAX_SITES + 1
    assert rc == lbpf.LBPF_EINVAL
    rc, _ = _call(f, t, t, None, 1, 0, 0.15, 0.0)
    assert rc == lbpf.LBPF_EINVAL
    for code in (0, 2, 3):
        rc, _ = _call(f, t, t, None, code, 268435456 + 1, 0.15, 0.0)
        assert rc == lbpf.LBPF_EINVAL
    rc, _ = _call(f, t, t, None, 4, 8, 0.15, 0.0)  # no such storage code
    assert rc == lbpf.LBPF_EINVAL
