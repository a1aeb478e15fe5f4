"""Seeded synthetic workloads shaped like the paper's dendrite runs.

This module holds only input recipes: grid sizes, lattices, physical
parameters, seed placement and random draws.  It contains none of the method's
arithmetic, so both the CUDA library's callers and the CPU oracle's tests can
use it.

Sizes and parameters follow the paper's simulations (Sec. 4: diffuse spherical
nuclei in a uniformly supersaturated or undercooled melt, zero-flux walls).

Time step.  With the non-local phase-field collision (Eq. collision stage,
Sec. 3.4) a uniform perturbation relaxes with rate 1/(a_s^2 eta_phi).  The
scheme is stable only while a_s^2 eta_phi > 1/2 for every interface
orientation, which with W0 = tau0 = 1, dx = 0.8 and a cubic anisotropy
eps = 0.05 (a_s down to 1 - 5 eps / 3 along <111>) needs dt > 0.024.  The
workloads below therefore use dt = 0.05 wherever the standard anisotropy is
used; the two-harmonic anisotropy of Eq. (As_K41-K61) with eps = -0.02,
delta = 0.015 keeps a_s >= 0.988 and runs at dt = 0.01.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

A2 = 0.6267  # a_2 of Eq. (Kinetic-Coeff)


@dataclass
class Workload:
    name: str
    grid: tuple            # (nx, ny, nz)
    lattices: tuple        # (q_phi, q_u, q_theta); q_theta = 0 freezes theta at theta0
    params: dict           # physical parameters (keys of the C parameter struct)
    centres: np.ndarray    # (n, 3) lattice units
    radii: np.ndarray      # (n,) lattice units
    U0: float
    theta0: float
    steps: int
    storage: str = "f64"   # "f64" | "f32" | "f16" | "bf16"
    tip_every: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def sites(self) -> int:
        return int(self.grid[0]) * int(self.grid[1]) * int(self.grid[2])

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def base_params(**kw) -> dict:
    """Isothermal alloy parameters of the paper's supersaturation test (Sec. 4.2),
    with lambda = D / a_2 (zero kinetic coefficient at W0 = tau0 = 1)."""
    p = dict(W0=1.0, tau0=1.0, D=2.0, kappa=1.0, lam=2.0 / A2, Mc_inf=1.0, k=0.15,
             aniso=0, eps1=0.05, eps2=0.0, dx=0.8, dt=0.05, antitrapping=1, grad2_min=1e-12)
    p.update(kw)
    return p


def centred_seed(n: int, R: float):
    c = n // 2
    return np.array([[c, c, c]], np.float64), np.array([R], np.float64)


def small_dendrite() -> Workload:
    """32^3, D3Q15 phi / D3Q19 U, theta frozen at 0, one seed R0 = 5 at the centre."""
    c, r = centred_seed(32, 5.0)
    return Workload("dendrite32_q15q19_f64", (32, 32, 32), (15, 19, 0), base_params(), c, r,
                    U0=-0.55, theta0=0.0, steps=500)


def single_dendrite(q_phi: int = 19) -> Workload:
    """128^3, D3Q19 phi and U (or D3Q7 phi for the grid-anisotropy comparison)."""
    c, r = centred_seed(128, 8.0)
    return Workload("dendrite128_q%dq19_f64" % q_phi, (128, 128, 128), (q_phi, 19, 0), base_params(), c, r,
                    U0=-0.55, theta0=0.0, steps=5000, tip_every=100)


def coupled_dendrite(storage: str = "f64", n: int = 256) -> Workload:
    """256^3 coupled heat + solute: phi/U on D3Q19, theta on D3Q7, Lewis number 50."""
    c, r = centred_seed(n, 8.0)
    p = base_params(kappa=100.0)
    return Workload("coupled%d_q19q19q7_%s" % (n, storage), (n, n, n), (19, 19, 7), p, c, r,
                    U0=-0.55, theta0=-0.3, steps=8000, storage=storage, tip_every=100)


def four_seeds(n: int, R0: float = 6.0, min_dist: float = 80.0, seed: int = 7, count: int = 4):
    """Integer seed centres in [R0+8, n-1-R0-8]^3, pairwise at least min_dist apart,
    drawn with numpy's PCG64 default_rng(seed) by rejection."""
    rng = np.random.default_rng(seed)
    lo, hi = int(R0 + 8), int(n - 1 - R0 - 8)
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cannot place %d seeds" % count)
        c = rng.integers(lo, hi + 1, size=3)
        if all(np.linalg.norm(c - o) >= min_dist for o in out):
            out.append(c)
    return np.array(out, np.float64), np.full(count, R0, np.float64)


def large_kh(n: int = 512, storage: str = "f32") -> Workload:
    """512^3, D3Q19 for phi, U and theta, two-harmonic anisotropy (<110>-type),
    four seeds R0 = 6 placed by default_rng(7) at least 80 cells apart."""
    c, r = four_seeds(n, min_dist=80.0 if n >= 256 else max(8.0, n / 6))
    p = base_params(aniso=1, eps1=-0.02, eps2=0.015, kappa=100.0, dt=0.01)
    return Workload("kh%d_q19x3_%s" % (n, storage), (n, n, n), (19, 19, 19), p, c, r,
                    U0=-0.5, theta0=-0.3, steps=4000, storage=storage)


def dense_kh(n: int = 512, spacing: int = 64, R0: float = 20.0, storage: str = "f32") -> Workload:
    """A stress case of the 512^3 two-harmonic workload with interface at most sites:
    seeds of radius R0 on a cubic lattice of the given spacing (8^3 = 512 seeds at 512^3,
    the first at spacing/2).  The seed profile's tails keep |grad phi|^2 above the
    threshold of the undefined normal within about 12 cells of each surface, so the
    anisotropy and anti-trapping arithmetic runs at over half of the sites, which a run
    from four seeds reaches only after dendrite arms fill the box."""
    g = np.arange(spacing // 2, n, spacing, dtype=np.float64)
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    p = base_params(aniso=1, eps1=-0.02, eps2=0.015, kappa=100.0, dt=0.01)
    return Workload("dense%d_s%d_q19x3_%s" % (n, spacing, storage), (n, n, n), (19, 19, 19), p, c,
                    np.full(len(c), R0), U0=-0.5, theta0=-0.3, steps=4000, storage=storage)


def pure_substance_2d(n: int = 500, storage: str = "f64") -> Workload:
    """The 2D anisotropic benchmark of Sec. 4.1 (pure substance, Delta = 0.55):
    D2Q9 for phi, D2Q5 for theta, n^2 nodes (500^2 in the paper), dx = 0.4 W0,
    dt = 0.008 tau0, kappa = 4, lambda* = kappa/a_2 = 6.3826 (zero kinetic
    coefficient), eps_s = 0.05, a seed of radius 10 dx centred on the corner
    (-1/2, -1/2) between the two mirror walls (quarter domain).  No solute coupling
    (M c_inf = 0): U runs on D2Q5 but does not act on phi.  The paper quotes
    V_p = V d0/kappa = 0.01735 at t = 300 (37,500 steps), d0 = 0.1385."""
    p = dict(W0=1.0, tau0=1.0, D=1.0, kappa=4.0, lam=6.3826, Mc_inf=0.0, k=1.0, aniso=0, eps1=0.05, eps2=0.0,
             dx=0.4, dt=0.008, antitrapping=0, grad2_min=1e-12)
    return Workload("pure2d_%d_d2q9_d2q5_%s" % (n, storage), (n, n, 1), (9, 5, 5), p,
                    np.array([[-0.5, -0.5, 0.0]]), np.array([10.0]), U0=0.0, theta0=-0.55, steps=37500,
                    storage=storage, tip_every=625, extra={"d0": 0.1385, "vp_paper_t300": 0.01735})


def grid_anisotropy(q_phi: int = 19, n: int = 301, delta: float = 0.25, storage: str = "f32") -> Workload:
    """The isotropic-sphere test of Sec. 4.1 (grid anisotropy A_g): pure substance
    (M c_inf = 0), eps_s = 0, n^3 nodes (301^3 in the paper), dx = 0.01, dt = 1.5e-5,
    W0 = 0.01, tau0 = 1e-4, lambda = 10, kappa = 0.7, a centred seed of radius 8 l.u.,
    compared at t = 10^4 dt.  The paper does not state the undercooling; Delta = 0.25.
    The phase field runs on q_phi, theta on D3Q7 (U, uncoupled, on D3Q7)."""
    p = dict(W0=0.01, tau0=1e-4, D=1.0, kappa=0.7, lam=10.0, Mc_inf=0.0, k=1.0, aniso=0, eps1=0.0, eps2=0.0,
             dx=0.01, dt=1.5e-5, antitrapping=0, grad2_min=1e-12)
    c, r = centred_seed(n, 8.0)
    return Workload("iso%d_q%d_%s" % (n, q_phi, storage), (n, n, n), (q_phi, 7, 7), p, c, r, U0=0.0,
                    theta0=-delta, steps=10000, storage=storage,
                    extra={"Ag_paper_pct": {7: 3.095, 15: 0.073, 19: 0.116}[q_phi]})


BATCH_EDGES = (48, 64, 80, 96)
BATCH_K = (0.1, 0.15, 0.3)


def batch_sweep(count: int = 64, seed: int = 11, storage: str = "f16"):
    """Independent simulations for the batched sweep, drawn sim-major with
    default_rng(seed): edge from {48,64,80,96}, Delta ~ U[0.3,0.65],
    eps ~ U[0.01,0.07], k from {0.1,0.15,0.3}; one centred seed R0 = 5."""
    rng = np.random.default_rng(seed)
    sims = []
    for s in range(count):
        edge = int(rng.choice(BATCH_EDGES))
        delta = float(rng.uniform(0.3, 0.65))
        eps = float(rng.uniform(0.01, 0.07))
        k = float(rng.choice(BATCH_K))
        c, r = centred_seed(edge, 5.0)
        p = base_params(eps1=eps, k=k)
        sims.append(Workload("sweep%02d_e%d" % (s, edge), (edge, edge, edge), (19, 19, 0), p, c, r,
                             U0=-delta, theta0=0.0, steps=2000, storage=storage))
    return sims


def by_name(name: str) -> Workload:
    table = {
        "dendrite32": small_dendrite,
        "dendrite128": single_dendrite,
        "coupled256": coupled_dendrite,
        "kh512": large_kh,
        "pure2d": pure_substance_2d,
    }
    return table[name]()


def population_noise(shape, lattices, seed: int = 0, amplitude: float = 0.05):
    """Seeded uniform noise in [-amplitude, amplitude] for every population of the
    three fields, population-major [Q][nz][ny][nx] (None for a frozen theta).  Parity
    tests add it to a seeded state so that every term of the collision is exercised."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    qp, qu, qt = lattices
    ng = rng.uniform(-amplitude, amplitude, size=(qp, nz, ny, nx))
    nh = rng.uniform(-amplitude, amplitude, size=(qu, nz, ny, nx))
    nf = rng.uniform(-amplitude, amplitude, size=(qt, nz, ny, nx)) if qt else None
    return ng, nh, nf
