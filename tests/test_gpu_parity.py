"""GPU parity of the CUDA library (through its C ABI) against the FP64 CPU oracle.

Tolerances (fixed by the accuracy targets of the method's GPU forms):
  - FP64 storage and arithmetic: max |gpu - oracle| / max(1, |oracle|) <= 1e-12
    after ONE step from an identical state;
  - FP32: phi L-infinity <= 1e-5 after 200 steps;
  - FP16 shifted/scaled storage with FP32 arithmetic: tip velocity within 1 % of FP64.
Integer-like outputs (step counters, tiling-independence, batch vs single,
checkpoint round trips) are compared bit for bit.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1602_07483_gb300 import build, lbpf, workloads

pytestmark = pytest.mark.gpu

REL_F64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbpf.load()


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def oracle_params(p: dict):
    q = dict(p)
    q.pop("storage", None)
    return oracle.make_params(**q)


def noisy_state(shape, lattices, params, seed=0, pre_steps=3, amp=1e-3, U0=-0.55, theta0=-0.2):
    """A developed oracle state (seed + a few steps) with seeded population noise."""
    nx, ny, nz = shape
    ora = oracle.Sim(shape, lattices, params=oracle_params(params))
    c = np.array([[nx / 2 - 0.3, ny / 2 + 0.2, nz / 2 - 0.1]])
    ora.init_seed(c, [min(nx, ny, nz) / 4.0], U0, theta0)
    ora.step(pre_steps)
    g, h = ora.pops(0), ora.pops(1)
    f = ora.pops(2) if lattices[2] else None
    ng, nh, nf = workloads.population_noise(shape, lattices, seed=seed, amplitude=amp)
    g = g + ng
    h = h + nh
    if f is not None:
        f = f + nf
    return g, h, f


CASES = [
    # (shape, lattices, extra params)
    ((33, 29, 23), (15, 19, 0), dict(aniso=0, eps1=0.05)),
    ((33, 29, 23), (19, 19, 7), dict(aniso=0, eps1=0.05, kappa=3.0)),
    ((31, 17, 20), (19, 19, 19), dict(aniso=1, eps1=-0.02, eps2=0.015, kappa=2.0, dt=0.02)),
    ((20, 33, 9), (7, 19, 0), dict(aniso=0, eps1=0.03)),
    ((17, 12, 31), (15, 15, 15), dict(aniso=0, eps1=0.04, kappa=1.5, antitrapping=0)),
    ((9, 40, 11), (7, 7, 7), dict(aniso=1, eps1=0.01, eps2=-0.01, kappa=1.0)),
]


@pytest.mark.parametrize("tiling", [(0, 0), (6, 4), (4, 1)])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_one_step_f64_parity(case, tiling):
    shape, lat, extra = CASES[case]
    params = workloads.base_params(**extra)
    g, h, f = noisy_state(shape, lat, params, seed=case)
    ora = oracle.Sim(shape, lat, params=oracle_params(params))
    ora.set_state(g, h, f, theta0=-0.2)
    gpu = lbpf.Sim(shape, lat, storage="f64", **params)
    if tiling != (0, 0):
        gpu.set_tiling(*tiling)
    gpu.set_state(g, h, f, theta0=-0.2)
    # the import itself is exact
    g2, h2, f2 = gpu.get_state()
    assert np.array_equal(g2, g) and np.array_equal(h2, h)
    ora.step(1)
    gpu.step(1)
    po, uo, to = ora.fields()
    pg, ug, tg = gpu.read_fields()
    assert rel_err(pg, po) <= REL_F64
    assert rel_err(ug, uo) <= REL_F64
    assert rel_err(tg, to) <= REL_F64
    go, ho = ora.pops(0), ora.pops(1)
    gg, hg, fg = gpu.get_state()
    assert rel_err(gg, go) <= REL_F64
    assert rel_err(hg, ho) <= REL_F64
    if lat[2]:
        assert rel_err(fg, ora.pops(2)) <= REL_F64


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (1, 17, 1), (40, 1, 3), (5, 5, 64)])
def test_degenerate_grids_f64(shape):
    params = workloads.base_params(eps1=0.02)
    lat = (19, 19, 7)
    g, h, f = noisy_state(shape, lat, params, seed=7, pre_steps=1)
    ora = oracle.Sim(shape, lat, params=oracle_params(params))
    ora.set_state(g, h, f, theta0=-0.2)
    gpu = lbpf.Sim(shape, lat, storage="f64", **params)
    gpu.set_state(g, h, f, theta0=-0.2)
    ora.step(3)
    gpu.step(3)
    for a, b in zip(gpu.read_fields(), ora.fields()):
        assert rel_err(a, b) <= 1e-12


def test_multistep_f64_drift_small_dendrite():
    """The 32^3 D3Q15/D3Q19 dendrite from the seed: GPU FP64 tracks the oracle over
    many graph-replayed steps (drift reported; rounding only)."""
    w = workloads.small_dendrite()
    ora = oracle.Sim(w.grid, w.lattices, params=oracle_params(w.params))
    ora.init_seed(w.centres, w.radii, w.U0, w.theta0)
    gpu = lbpf.sim_from_workload(w, storage="f64")
    errs = []
    for _ in range(4):
        ora.step(25)
        gpu.step(25)
        pg, ug, _ = gpu.read_fields()
        po, uo, _ = ora.fields()
        errs.append(max(rel_err(pg, po), rel_err(ug, uo)))
    assert max(errs) < 1e-10, errs
    # diagnostics agree with the oracle's
    assert np.allclose(gpu.sums(), ora.sums(), rtol=1e-11, atol=1e-9)
    c = [int(v) for v in w.centres[0]]
    xg, rg = gpu.tip(c)
    xo, ro = ora.tip(c)
    assert abs(xg - xo) < 1e-9 and abs(rg - ro) < 1e-7


def test_f32_phi_linf_after_200_steps():
    """FP32 storage and arithmetic: phi L-infinity <= 1e-5 against the FP64 oracle
    after 200 steps of the 32^3 dendrite."""
    w = workloads.small_dendrite()
    ora = oracle.Sim(w.grid, w.lattices, params=oracle_params(w.params))
    ora.init_seed(w.centres, w.radii, w.U0, w.theta0)
    gpu = lbpf.sim_from_workload(w, storage="f32")
    ora.step(200)
    gpu.step(200)
    pg, ug, _ = gpu.read_fields()
    po, uo, _ = ora.fields()
    assert np.max(np.abs(pg - po)) <= 1e-5
    assert np.max(np.abs(ug - uo)) <= 1e-4


def test_f32_coupled_heat_solute_200_steps():
    """Coupled heat + solute (D3Q19/D3Q19/D3Q7, Lewis number 50) at 48^3, FP32 vs oracle."""
    w = workloads.coupled_dendrite(n=48)
    ora = oracle.Sim(w.grid, w.lattices, params=oracle_params(w.params))
    ora.init_seed(w.centres, w.radii, w.U0, w.theta0)
    gpu = lbpf.sim_from_workload(w, storage="f32")
    ora.step(200)
    gpu.step(200)
    (pg, ug, tg), (po, uo, to) = gpu.read_fields(), ora.fields()
    assert np.max(np.abs(pg - po)) <= 1e-5
    assert np.max(np.abs(ug - uo)) <= 1e-4
    assert np.max(np.abs(tg - to)) <= 1e-5


def _tip_velocity(storage, n=128, lo=24, window=400):
    """Tip speed along +x of the coupled 3D dendrite, measured over `window` steps once
    the tip is `lo` cells ahead of the seed centre (well before it nears the wall)."""
    w = workloads.coupled_dendrite(n=n)
    s = lbpf.sim_from_workload(w, storage=storage)
    c = [int(v) for v in w.centres[0]]
    x0 = -1.0
    for _ in range(200):
        s.step(30)
        x0, _ = s.tip(c)
        if x0 - c[0] >= lo:
            break
    assert x0 - c[0] >= lo
    s.step(window)
    x1, rho = s.tip(c)
    assert x1 > x0 and x1 < n - 4
    return (x1 - x0) * w.params["dx"] / (window * w.params["dt"]), rho


@pytest.fixture(scope="module")
def tip_f64():
    return _tip_velocity("f64")


@pytest.mark.parametrize("storage", ["f16", "f32"])
def test_low_precision_storage_tip_velocity_within_1pct(storage, tip_f64):
    v64, r64 = tip_f64
    v, r = _tip_velocity(storage)
    assert abs(v / v64 - 1) < 0.01, (v, v64)


def test_bf16_storage_runs_and_stays_close(tip_f64):
    v64, _ = tip_f64
    v, _ = _tip_velocity("bf16")
    assert abs(v / v64 - 1) < 0.10, (v, v64)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_tiling_does_not_change_results(storage):
    """Bit-identical fields under another tiling (block rows and z-chunks), for each
    single-precision storage: halo nodes recompute their owners' collisions exactly."""
    w = workloads.coupled_dendrite(n=40)
    a = lbpf.sim_from_workload(w, storage=storage)
    b = lbpf.sim_from_workload(w, storage=storage)
    b.set_tiling(5, 3)
    a.step(13)
    b.step(13)
    for x, y in zip(a.read_fields(), b.read_fields()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("tiling", [(0, 0), (6, 16), (4, 8)])
def test_batch_matches_single_bitwise(tiling):
    """A batch (under its default tiling and two others set with lbpf_batch_set_tiling)
    advances each member exactly as the member would alone."""
    sims = workloads.batch_sweep(count=4, storage="f32")
    singles = [lbpf.sim_from_workload(w) for w in sims]
    members = [lbpf.sim_from_workload(w) for w in sims]
    batch = lbpf.Batch(members)
    if tiling != (0, 0):
        batch.step(3)
        batch.set_tiling(*tiling)
        batch.step(11)
    else:
        batch.step(14)
    for s in singles:
        s.step(14)
    batch.close()
    for s, m in zip(singles, members):
        assert m.steps_done == 14
        for x, y in zip(s.read_fields(), m.read_fields()):
            assert np.array_equal(x, y)


BATCH_MEMBERS = [
    # (shape, extra params, U0): uneven grids, anisotropy strengths, partition coefficients
    ((33, 29, 23), dict(eps1=0.03, k=0.15), -0.55),
    ((24, 31, 19), dict(eps1=0.05, k=0.1), -0.4),
    ((40, 17, 21), dict(eps1=0.02, k=0.3), -0.3),
    ((17, 22, 36), dict(eps1=0.04, k=0.15, antitrapping=0), -0.6),
]


def test_batch_members_match_oracle_f64():
    """A library-owned batch (lbpf_batch_create) of four uneven FP64 simulations, each
    started from its own noisy oracle state, tracks the oracle member by member: <= 1e-12
    after one step, <= 1e-10 after 50 (one launch per kernel phase covers all members)."""
    lat = (19, 19, 7)
    states, oras, params = [], [], []
    for m, (shape, extra, U0) in enumerate(BATCH_MEMBERS):
        p = workloads.base_params(kappa=2.0, **extra)
        g, h, f = noisy_state(shape, lat, p, seed=20 + m, U0=U0)
        o = oracle.Sim(shape, lat, params=oracle_params(p))
        o.set_state(g, h, f, theta0=-0.2)
        states.append((g, h, f))
        oras.append(o)
        params.append(lbpf.make_params("f64", **p))
    batch = lbpf.Batch.create([mb[0] for mb in BATCH_MEMBERS], lat, params)
    for s, (g, h, f) in zip(batch.sims, states):
        s.set_state(g, h, f, theta0=-0.2)
    for steps, tol in ((1, REL_F64), (49, 1e-10)):
        batch.step(steps)
        for s, o in zip(batch.sims, oras):
            o.step(steps)
            for a, b in zip(s.read_fields(), o.fields()):
                assert rel_err(a, b) <= tol, (s.nx, s.ny, s.nz, steps)
    assert all(s.steps_done == 50 for s in batch.sims)
    batch.close()


def test_batch_f16_matches_single_bitwise():
    """FP16 storage (the batched sweep's precision): a batch of uneven sweep members advances
    each member bit for bit as the member would alone, through the library-owned form."""
    ws = workloads.batch_sweep(count=3, storage="f16")
    singles = [lbpf.sim_from_workload(w) for w in ws]
    batch = lbpf.batch_from_workloads(ws)
    batch.step(9)
    for s in singles:
        s.step(9)
    for s, m in zip(singles, batch.sims):
        assert m.steps_done == 9
        for x, y in zip(s.read_fields(), m.read_fields()):
            assert np.array_equal(x, y)
    batch.close()


def test_batch_orders_member_streams():
    """Members on their own streams, the batch on another stream: a member read right after a
    batch step (batch still open) sees the finished step, and a member seeded on its own
    stream just before the step is seen by the batch."""
    import torch
    ws = workloads.batch_sweep(count=3, storage="f32")
    singles = [lbpf.sim_from_workload(w) for w in ws]
    members = [lbpf.Sim(w.grid, w.lattices, storage="f32", **w.params) for w in ws]
    side = torch.cuda.Stream()
    batch = lbpf.Batch(members, stream=side.cuda_stream)
    for w, m in zip(ws, members):
        m.init_seed(w.centres, w.radii, w.U0, w.theta0)   # enqueued on the member's stream
    for k in range(3):
        batch.step(5)
        for s in singles:
            s.step(5)
        for s, m in zip(singles, members):
            for x, y in zip(s.read_fields(), m.read_fields()):
                assert np.array_equal(x, y), k
    batch.close()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_tip_along_each_axis_matches_oracle(axis):
    """lbpf_tip along +x, +y, +z from a centre given in lattice coordinates (rounded to the
    nearest node) agrees with the oracle's tip and radius on a grown 3D seed."""
    w = workloads.coupled_dendrite(n=40)
    ora = oracle.Sim(w.grid, w.lattices, params=oracle_params(w.params))
    ora.init_seed(w.centres, w.radii, w.U0, w.theta0)
    gpu = lbpf.sim_from_workload(w, storage="f64")
    ora.step(60)
    gpu.step(60)
    c = [int(v) for v in w.centres[0]]
    xg, rg = gpu.tip([v + 0.3 for v in c], axis=axis)
    xo, ro = ora.tip(c, axis=axis)
    assert xo > c[axis] and ro > 0
    assert abs(xg - xo) < 1e-9 and abs(rg - ro) < 1e-7
    with pytest.raises(lbpf.LbpfError):
        gpu.tip([-3, 0, 0], axis=axis)
    with pytest.raises(lbpf.LbpfError):
        gpu.tip(c, axis=3)


def test_batch_set_tiling_rejects_bad_values():
    members = [lbpf.sim_from_workload(w) for w in workloads.batch_sweep(count=2, storage="f32")]
    batch = lbpf.Batch(members)
    with pytest.raises(lbpf.LbpfError):
        batch.set_tiling(3, 0)
    with pytest.raises(lbpf.LbpfError):
        batch.set_tiling(9, 0)
    batch.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_checkpoint_round_trip_bitwise(storage):
    """Save, run on, reload, run the same steps again: bit for bit in every storage type
    (FP16 populations go through FP64 in the file, where decoding and re-encoding with a
    power-of-two scale is exact)."""
    w = workloads.coupled_dendrite(n=24)
    a = lbpf.sim_from_workload(w, storage=storage)
    a.step(20)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.lbpf")
        a.save(path)
        a.step(20)
        b = lbpf.Sim(w.grid, w.lattices, storage=storage, **w.params)
        b.load_checkpoint(path)
        assert b.steps_done == 20
        b.step(20)
        assert b.steps_done == 40
    for x, y in zip(a.read_fields(), b.read_fields()):
        assert np.array_equal(x, y)


def test_autotune_keeps_state():
    w = workloads.coupled_dendrite(n=40)
    a = lbpf.sim_from_workload(w, storage="f32")
    b = lbpf.sim_from_workload(w, storage="f32")
    a.step(7)
    b.step(7)
    ms = a.autotune(steps=2)
    assert ms > 0
    assert a.steps_done == 7
    a.step(9)
    b.step(9)
    for x, y in zip(a.read_fields(), b.read_fields()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_autotune_keeps_state(storage):
    """lbpf_batch_autotune times every candidate tiling and restores each member: after it,
    from an unaligned step count (7, not a multiple of the 6-step graph period), the batch
    continues bit for bit like members that were never tuned, and the tiling it kept is
    one of the candidates."""
    ws = workloads.batch_sweep(count=3, storage=storage)
    singles = [lbpf.sim_from_workload(w) for w in ws]
    batch = lbpf.batch_from_workloads(ws)
    batch.step(7)
    ms = batch.autotune(steps=6)
    assert ms > 0
    by, zc = batch.get_tiling()
    assert by in (4, 6, 8) and zc in (0, 12, 16, 24)
    assert all(m.steps_done == 7 for m in batch.sims)
    batch.step(11)
    for s in singles:
        s.step(18)
    for s, m in zip(singles, batch.sims):
        for x, y in zip(s.read_fields(), m.read_fields()):
            assert np.array_equal(x, y)
    batch.close()


def test_nan_is_reported():
    shape, lat = (12, 12, 12), (19, 19, 0)
    params = workloads.base_params()
    g, h, _ = noisy_state(shape, lat, params)
    g[3, 5, 5, 5] = np.nan
    s = lbpf.Sim(shape, lat, storage="f32", **params)
    s.set_state(g, h)
    s.step(2)
    with pytest.raises(lbpf.LbpfError) as e:
        s.sums()
    assert e.value.code == lbpf.LBPF_ENAN


def test_enthalpy_invariant_on_gpu():
    w = workloads.coupled_dendrite(n=48)
    s = lbpf.sim_from_workload(w, storage="f64")
    a = s.sums()
    s.step(60)
    b = s.sums()
    assert abs((b[2] - 0.5 * b[0]) - (a[2] - 0.5 * a[0])) < 1e-9 * w.sites


# ------------------------------------------------------------ full size

def _sample_sites(n, centres, count, seed):
    rng = np.random.default_rng(seed)
    pts = [rng.integers(0, n, size=3) for _ in range(count // 2)]
    for c in centres:   # near the seeds' interfaces
        for _ in range(count // (2 * len(centres))):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            pts.append(np.clip(np.round(c + d * rng.uniform(4, 8)), 0, n - 1).astype(int))
    pts += [np.array([0, 0, 0]), np.array([n - 1, 3, n - 2]), np.array([n // 2, n - 1, 0])]
    return pts


def test_full_size_sampled_parity_kh512_f32():
    """The 512^3 D3Q19 x 3 FP32 workload in the launch configuration the benchmark
    times: one step from the seeds, sampled sites against oracle sub-box runs.  After
    one step a node depends on nodes within 4 lattice links, so an 11^3 box around the
    sample (clipped by the real walls) reproduces it exactly."""
    w = workloads.large_kh(512)
    gpu = lbpf.sim_from_workload(w, storage="f32")
    gpu.step(1)
    phi, U, th = gpu.read_fields()
    n = 512
    for p in _sample_sites(n, w.centres, 24, seed=3):
        lo = np.maximum(p - 5, 0)
        hi = np.minimum(p + 6, n)
        shape = tuple(int(v) for v in (hi - lo))
        ora = oracle.Sim(shape, w.lattices, params=oracle_params(w.params))
        ora.init_seed(w.centres - lo[None, :], w.radii, w.U0, w.theta0)
        ora.step(1)
        po, uo, to = ora.fields()
        q = tuple(int(v) for v in (p - lo))
        x, y, z = int(p[0]), int(p[1]), int(p[2])
        assert abs(phi[z, y, x] - po[q[2], q[1], q[0]]) < 2e-6
        assert abs(U[z, y, x] - uo[q[2], q[1], q[0]]) < 2e-6
        assert abs(th[z, y, x] - to[q[2], q[1], q[0]]) < 2e-6
    # a property that holds at any size: the enthalpy invariant
    a = gpu.sums()
    gpu.step(12)
    b = gpu.sums()
    assert abs((b[2] - 0.5 * b[0]) - (a[2] - 0.5 * a[0])) < 1e-6 * w.sites


def test_largest_grid_sampled_parity_f32():
    """The largest grid the kernels' 32-bit element offsets allow: 608 x 608 x 611 sites, so
    that 19 x n_sites is just below 2^32 (the next plane is refused, tests/test_abi.py).  FP32
    with the benchmark's lattices, recipe and 8-row launch configuration (about 116 GB on the
    device): one step from four seeds, sampled sites against oracle sub-box runs, among them
    the far corner, whose last D3Q19 population sits 2^32 - 3.5 M elements into its array."""
    grid = (608, 608, 611)
    assert 19 * grid[0] * grid[1] * grid[2] < 2 ** 32 <= 19 * grid[0] * grid[1] * (grid[2] + 1)
    w = workloads.large_kh(608)
    gpu = lbpf.Sim(grid, w.lattices, storage="f32", **w.params)
    gpu.init_seed(w.centres, w.radii, w.U0, w.theta0)
    assert gpu.get_tiling()[0] == 8
    gpu.step(1)
    phi, U, th = gpu.read_fields()
    gpu.close()
    hi_all = np.array(grid)
    pts = [np.minimum(p, hi_all - 1) for p in _sample_sites(608, w.centres, 16, seed=5)]
    pts += [np.array([607, 607, 610]), np.array([0, 607, 610]), np.array([607, 0, 305]), np.array([301, 402, 609])]
    for p in pts:
        lo = np.maximum(p - 5, 0)
        hi = np.minimum(p + 6, hi_all)
        shape = tuple(int(v) for v in (hi - lo))
        ora = oracle.Sim(shape, w.lattices, params=oracle_params(w.params))
        ora.init_seed(w.centres - lo[None, :], w.radii, w.U0, w.theta0)
        ora.step(1)
        po, uo, to = ora.fields()
        q = tuple(int(v) for v in (p - lo))
        x, y, z = int(p[0]), int(p[1]), int(p[2])
        assert abs(phi[z, y, x] - po[q[2], q[1], q[0]]) < 2e-6, tuple(p)
        assert abs(U[z, y, x] - uo[q[2], q[1], q[0]]) < 2e-6, tuple(p)
        assert abs(th[z, y, x] - to[q[2], q[1], q[0]]) < 2e-6, tuple(p)


def test_grid_anisotropy_sphere_matches_oracle():
    """The isotropic-sphere set-up of Sec. 4.1 (pure substance, theta on D3Q7) on 51^3 for
    400 steps, phi on D3Q7 and D3Q19: the GPU FP64 fields track the oracle's and give the
    same grid-anisotropy coefficient A_g."""
    from paper_1602_07483_gb300.experiments import radii_100_110
    for q in (7, 19):
        w = workloads.grid_anisotropy(q_phi=q, n=51, storage="f64")
        ora = oracle.Sim(w.grid, w.lattices, params=oracle_params(w.params))
        ora.init_seed(w.centres, w.radii, w.U0, w.theta0)
        gpu = lbpf.sim_from_workload(w)
        ora.step(400)
        gpu.step(400)
        pg, _, tg = gpu.read_fields()
        po, _, to = ora.fields()
        assert rel_err(pg, po) < 1e-10 and rel_err(tg, to) < 1e-10
        ag_g = radii_100_110(pg, 25)[2]
        ag_o = radii_100_110(po, 25)[2]
        assert abs(ag_g - ag_o) < 1e-8, (ag_g, ag_o)
