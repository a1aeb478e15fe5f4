"""GPU parity of the 2D scheme (D2Q5 / D2Q9 on an nz = 1 grid, Tables 3-4 of
Sec. 3.4) against the FP64 CPU oracle, and the paper's 2D benchmark (Sec. 4.1).

Tolerances as for the 3D path: FP64 <= 1e-12 relative after one step from an
identical state; FP32 phi L-infinity <= 1e-5 after 200 steps."""
import json
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1602_07483_gb300 import build, lbpf, workloads

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
REL_F64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbpf.load()


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def oracle_params(p):
    q = dict(p)
    q.pop("storage", None)
    return oracle.make_params(**q)


CASES_2D = [
    ((37, 29, 1), (9, 5, 5), dict(aniso=0, eps1=0.05, kappa=2.0, dx=0.4, dt=0.008)),
    ((33, 18, 1), (5, 9, 0), dict(aniso=0, eps1=0.03, dx=0.4, dt=0.008)),
    ((40, 21, 1), (9, 9, 9), dict(aniso=1, eps1=-0.02, eps2=0.015, kappa=1.5, dx=0.4, dt=0.008)),
    ((61, 9, 1), (5, 5, 5), dict(aniso=0, eps1=0.04, kappa=1.0, antitrapping=0, dx=0.4, dt=0.008)),
]


def noisy_state_2d(shape, lattices, params, seed):
    nx, ny, _ = shape
    ora = oracle.Sim(shape, lattices, params=oracle_params(params))
    ora.init_seed([[nx / 2 - 0.3, ny / 2 + 0.2, 0.0]], [min(nx, ny) / 4.0], -0.55, -0.2)
    ora.step(3)
    ng, nh, nf = workloads.population_noise(shape, lattices, seed=seed, amplitude=1e-3)
    f = ora.pops(2) + nf if lattices[2] else None
    return ora.pops(0) + ng, ora.pops(1) + nh, f


@pytest.mark.parametrize("tiling", [(0, 0), (6, 4), (4, 1)])
@pytest.mark.parametrize("case", range(len(CASES_2D)))
def test_one_step_f64_parity_2d(case, tiling):
    shape, lat, extra = CASES_2D[case]
    params = workloads.base_params(**extra)
    g, h, f = noisy_state_2d(shape, lat, params, seed=case)
    ora = oracle.Sim(shape, lat, params=oracle_params(params))
    ora.set_state(g, h, f, theta0=-0.2)
    gpu = lbpf.Sim(shape, lat, storage="f64", **params)
    if tiling != (0, 0):
        gpu.set_tiling(*tiling)
    gpu.set_state(g, h, f, theta0=-0.2)
    ora.step(1)
    gpu.step(1)
    for a, b in zip(gpu.read_fields(), ora.fields()):
        assert rel_err(a, b) <= REL_F64
    gg, hg, fg = gpu.get_state()
    assert rel_err(gg, ora.pops(0)) <= REL_F64
    assert rel_err(hg, ora.pops(1)) <= REL_F64
    if lat[2]:
        assert rel_err(fg, ora.pops(2)) <= REL_F64


def test_multistep_f64_2d_benchmark_setup():
    """The Sec. 4.1 set-up on a 96^2 quarter domain: 400 graph-replayed steps track the
    oracle, and the diagnostics (sums, tip, tip radius from the xy plane) agree."""
    w = workloads.pure_substance_2d(n=96)
    ora = oracle.Sim(w.grid, w.lattices, params=oracle_params(w.params))
    ora.init_seed(w.centres, w.radii, w.U0, w.theta0)
    gpu = lbpf.sim_from_workload(w, storage="f64")
    errs = []
    for _ in range(4):
        ora.step(100)
        gpu.step(100)
        errs.append(max(rel_err(a, b) for a, b in zip(gpu.read_fields(), ora.fields())))
    assert max(errs) < 1e-10, errs
    assert np.allclose(gpu.sums(), ora.sums(), rtol=1e-11, atol=1e-9)
    xg, rg = gpu.tip((0, 0, 0))
    xo, ro = ora.tip((0, 0, 0))
    assert xg > 10 and abs(xg - xo) < 1e-9
    assert rg == ro == -1.0  # rows below the mirror corner do not exist
    # along the paper's y axis (the kernel's z axis): the seed sits on the mirror corner, so
    # the x <-> y symmetry of the set-up gives the same tip, and the oracle agrees
    yg, _ = gpu.tip((0, 0, 0), axis=1)
    yo, _ = ora.tip((0, 0, 0), axis=1)
    assert abs(yg - yo) < 1e-9 and abs(yg - xg) < 1e-9
    with pytest.raises(lbpf.LbpfError):
        gpu.tip((0, 0, 0), axis=2)


def test_f32_2d_phi_linf_after_200_steps():
    w = workloads.pure_substance_2d(n=128)
    ref = lbpf.sim_from_workload(w, storage="f64")
    low = lbpf.sim_from_workload(w, storage="f32")
    ref.step(200)
    low.step(200)
    assert rel_err(low.read_fields()[0], ref.read_fields()[0]) <= 1e-5


def test_batch_2d_matches_single_bitwise():
    """Uneven 2D simulations stepped in one batched launch equal their one-by-one runs."""
    ws = [workloads.pure_substance_2d(n=n, storage="f32") for n in (64, 96, 130)]
    singles = [lbpf.sim_from_workload(w) for w in ws]
    members = [lbpf.sim_from_workload(w) for w in ws]
    batch = lbpf.Batch(members)
    for s in singles:
        s.step(14)
    batch.step(14)
    batch.close()
    for s, m in zip(singles, members):
        for x, y in zip(s.read_fields(), m.read_fields()):
            assert np.array_equal(x, y)


def test_checkpoint_2d_round_trip_bitwise():
    w = workloads.pure_substance_2d(n=70, storage="f32")
    a = lbpf.sim_from_workload(w)
    a.step(11)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck2d.lbpf")
        a.save(path)
        a.step(13)
        b = lbpf.Sim(w.grid, w.lattices, storage="f32", **w.params)
        b.load_checkpoint(path)
        assert b.steps_done == 11
        b.step(13)
    for x, y in zip(a.read_fields(), b.read_fields()):
        assert np.array_equal(x, y)


def test_rejects_mixed_or_thick_2d():
    p = workloads.base_params(dx=0.4, dt=0.008)
    with pytest.raises(lbpf.LbpfError):
        lbpf.Sim((16, 16, 2), (9, 5, 0), storage="f64", **p)
    with pytest.raises(lbpf.LbpfError):
        lbpf.Sim((16, 16, 1), (9, 19, 0), storage="f64", **p)


def _vp_history(storage):
    w = workloads.pure_substance_2d(n=500)
    s = lbpf.sim_from_workload(w, storage=storage)
    hist = []
    for k in range(w.tip_every, w.steps + 1, w.tip_every):
        s.step(w.tip_every)
        hist.append((k * w.params["dt"], s.tip((0, 0, 0))[0]))
    s.close()
    return w, dict((round(t, 6), x) for t, x in hist)


def _vp(w, hist, t, span=10.0):
    return (hist[round(t, 6)] - hist[round(t - span, 6)]) * w.params["dx"] / span * w.extra["d0"] / w.params["kappa"]


@pytest.fixture(scope="module")
def vp_f64():
    return _vp_history("f64")


def test_paper_2d_tip_velocity_f64(vp_f64):
    """Sec. 4.1, Delta = 0.55 on 500^2: the paper's LB code gives V_p = 0.01735 at t = 300
    (Karma & Rappel's phase-field value 0.0174).  The GPU FP64 run reproduces it within
    2 % and, where the oracle's own run of the benchmark is stored, matches that run."""
    w, hist = vp_f64
    vp = _vp(w, hist, 300.0)
    assert abs(vp / 0.01735 - 1) < 0.02, vp
    gold = os.path.join(HERE, "golden", "tip_velocity_2d_oracle.json")
    if os.path.exists(gold):
        with open(gold) as f:
            d = json.load(f)
        ora = dict((round(t, 6), x) for t, x in d["history_t_xtip"])
        for t in (50.0, 150.0, 300.0):
            assert abs(hist[round(t, 6)] - ora[round(t, 6)]) < 1e-6, t


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_paper_2d_tip_velocity_low_precision(vp_f64, storage):
    """FP32, FP16 and BF16 storage (FP32 arithmetic) over the 37,500 steps: V_p(300) within
    1 % of FP64.  At dt = 0.008 theta changes little per step near the interface, so the
    half-precision codecs hold the bound only because f is stored as its deviation from
    w_i theta^{n-1} of the storing node (a constant shift w_i theta0 gave FP16 -4.5 % and
    lost the tip in BF16)."""
    w, ref = vp_f64
    _, hist = _vp_history(storage)
    assert abs(_vp(w, hist, 300.0) / _vp(w, ref, 300.0) - 1) < 0.01
