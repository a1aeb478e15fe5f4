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
        assert lib.lbpf_strerror(code) != b"unknown error"
    assert b"unstable" in lib.lbpf_strerror(-2)
    assert b"bounded wait" in lib.lbpf_strerror(-5)  # the one-launch step's waits
    assert lib.lbpf_strerror(-7) == b"unknown error"


def test_signatures_follow_the_boundary(lib):
    """The declarations of the calls the method's boundary lists: the tip takes an axis and a
    centre in lattice coordinates (doubles), and a batch is created from per-member grids,
    lattices and parameters, with a second constructor over existing handles."""
    src = open(os.path.join(ROOT, "include", "lbpf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    flat = " ".join(src.split())
    assert "int lbpf_tip(lbpf_sim* sim, int32_t axis, const double centre_lu[3], double* x_tip_lu, double* rho_lu);" in flat
    assert ("int lbpf_batch_create(int32_t n, const lbpf_grid* grids, const lbpf_lattice* lattices, "
            "const lbpf_params* params, void* cuda_stream, lbpf_batch** out);") in flat
    assert "int lbpf_batch_from_sims(int32_t n, lbpf_sim* const* sims, void* cuda_stream, lbpf_batch** out);" in flat
    assert "int lbpf_batch_member(const lbpf_batch* batch, int32_t i, lbpf_sim** out);" in flat
    assert "#define LBPF_ETIMEOUT (-5)" in src
    assert "int lbpf_set_schedule(lbpf_sim* sim, int32_t schedule);" in flat


def test_batch_and_tip_reject_bad_arguments_without_gpu(lib):
    """Argument checks that run before any device work."""
    out = ctypes.c_void_p()
    g = (lbpf.Grid * 2)(lbpf.Grid(8, 8, 8), lbpf.Grid(9, 8, 8))
    la = (lbpf.Lattice * 2)(lbpf.Lattice(19, 19, 0), lbpf.Lattice(15, 19, 0))  # lattices differ
    pa = (lbpf.Params * 2)(lbpf.make_params(storage="f32", dt=0.05), lbpf.make_params(storage="f32", dt=0.05))
    assert lib.lbpf_batch_create(2, g, la, pa, None, ctypes.byref(out)) == lbpf.LBPF_EINVAL
    assert lib.lbpf_batch_create(0, g, la, pa, None, ctypes.byref(out)) == lbpf.LBPF_EINVAL
    assert lib.lbpf_batch_from_sims(1, None, None, ctypes.byref(out)) == lbpf.LBPF_EINVAL
    c = (ctypes.c_double * 3)(1.0, 2.0, 3.0)
    x = ctypes.c_double()
    assert lib.lbpf_tip(None, 0, c, ctypes.byref(x), None) == lbpf.LBPF_EINVAL
    m = ctypes.c_void_p()
    assert lib.lbpf_batch_member(None, 0, ctypes.byref(m)) == lbpf.LBPF_EINVAL
    ms = ctypes.c_double()
    assert lib.lbpf_batch_autotune(None, 6, ctypes.byref(ms)) == lbpf.LBPF_EINVAL
    assert lib.lbpf_batch_get_tiling(None, None, None) == lbpf.LBPF_EINVAL
    assert lib.lbpf_set_schedule(None, 1) == lbpf.LBPF_EINVAL
    assert lib.lbpf_set_wait_polls(None, 10) == lbpf.LBPF_EINVAL
    assert lib.lbpf_batch_set_schedule(None, 0) == lbpf.LBPF_EINVAL
    v = ctypes.c_int32()
    assert lib.lbpf_get_schedule(None, ctypes.byref(v)) == lbpf.LBPF_EINVAL
    assert lib.lbpf_wait_probe(1, 0, ctypes.byref(v)) == lbpf.LBPF_EINVAL  # no GPU work for bad arguments


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


def test_grid_size_limit(lib):
    """The step kernels address populations with 32-bit element offsets, so 19 x n_sites
    must stay below 2^32: 608 x 608 x 612 sites (19 x 226,234,368 > 2^32) is refused before
    any device work, for every lattice (the limit counts the largest lattice); the largest
    grid that fits, 608 x 608 x 611, passes validation (without a GPU the call then fails
    on the device, not on the size)."""
    assert 19 * 608 * 608 * 612 >= 2 ** 32 > 19 * 608 * 608 * 611
    for lat in ((19, 19, 0), (7, 7, 0), (15, 19, 7)):
        assert _create(lattices=lat, grid=(608, 608, 612), dt=0.05) == lbpf.LBPF_EINVAL
    if not _gpu_present():  # (with a GPU this would allocate the whole grid; the GPU test does that)
        assert _create(grid=(608, 608, 611), dt=0.05) == lbpf.LBPF_ECUDA


def _gpu_present():
    import torch
    return torch.cuda.is_available()


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
