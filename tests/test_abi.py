"""Host-side checks of the CUDA library's C ABI that need no GPU: it builds for
sm_103a, loads, exports every entry point that include/lbpf.h declares, and
rejects invalid or unstable parameters before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1602_07483_gb300 import build, lbpf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbpf.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lbpf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbpf_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    # and nothing else with C linkage under that prefix
    out = os.popen("nm -D --defined-only %s" % lbpf.LIB_PATH).read()
    exported = sorted(set(re.findall(r" T (lbpf_[a-z_]+)", out)))
    assert exported == names


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.lbpf_strerror(code)
    assert b"unstable" in lib.lbpf_strerror(-2)


def _create(lattices=(19, 19, 0), grid=(8, 8, 8), **kw):
    h = ctypes.c_void_p()
    p = lbpf.make_params(**kw)
    rc = lbpf.load().lbpf_create(ctypes.byref(lbpf.Grid(*grid)), ctypes.byref(lbpf.Lattice(*lattices)),
                                 ctypes.byref(p), None, ctypes.byref(h))
    if rc == 0:
        lbpf.load().lbpf_destroy(h)
    return rc


def test_rejects_invalid_arguments(lib):
    assert _create(lattices=(9, 19, 0)) == lbpf.LBPF_EINVAL
    assert _create(lattices=(19, 19, 5)) == lbpf.LBPF_EINVAL
    assert _create(grid=(0, 8, 8)) == lbpf.LBPF_EINVAL
    assert _create(k=0.0) == lbpf.LBPF_EINVAL
    assert _create(dx=-1.0) == lbpf.LBPF_EINVAL
    assert _create(storage=7) == lbpf.LBPF_EINVAL
    assert _create(aniso=3) == lbpf.LBPF_EINVAL
    # 2D lattices: nz = 1 and no mixing with 3D lattices
    assert _create(lattices=(9, 5, 5), grid=(8, 8, 2), dx=0.4, dt=0.008) == lbpf.LBPF_EINVAL
    assert _create(lattices=(9, 5, 7), grid=(8, 8, 1), dx=0.4, dt=0.008) == lbpf.LBPF_EINVAL
    assert _create(lattices=(5, 9, 0), grid=(8, 8, 1), storage=7) == lbpf.LBPF_EINVAL


def test_rejects_unstable_nonlocal_collision(lib):
    """eps = 0.05, dx = 0.8, dt = 0.01: a_s^2 eta_phi falls below 1/2 along <111>."""
    assert _create(eps1=0.05, dt=0.01) == lbpf.LBPF_EUNSTABLE
    assert _create(eps1=0.07, dt=0.03) == lbpf.LBPF_EUNSTABLE


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES") is None and os.path.exists("/dev/nvidia0"),
                    reason="a GPU is present")
def test_no_gpu_fails_loudly(lib):
    """Without a CUDA device the library refuses to run (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    assert _create(eps1=0.05, dt=0.05) == lbpf.LBPF_ECUDA
    assert _create(lattices=(9, 5, 5), grid=(8, 8, 1), dx=0.4, dt=0.008) == lbpf.LBPF_ECUDA  # valid 2D set
    with pytest.raises(lbpf.LbpfError):
        lbpf.Sim((8, 8, 8))
