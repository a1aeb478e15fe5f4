"""Run the paper's 2D anisotropic pure-substance benchmark with the FP64 oracle and
write the tip-velocity history to tip_velocity_2d_oracle.json.

Benchmark of Sec. 4.1 ("Anisotropic case"): D2Q9 for the phase field, D2Q5 for the
temperature, 500^2 nodes, dx/W0 = 0.4, dt = 0.008, W0 = tau0 = 1, kappa = 4,
lambda* = kappa/a2 = 6.3826 (zero kinetic coefficient), d0 = 0.1385, eps_s = 0.05,
undercooling Delta = 0.55 (theta0 = -0.55), no solute coupling (M = 0), a diffuse
circle of radius 10 dx at the origin of a quarter domain (the halfway walls at
x = -1/2 and y = -1/2 are the symmetry lines).  The paper prints the dimensionless
tip velocity V_p = V d0 / kappa = 0.01735 at t = 300 for its LB code.

Calls only the oracle.  Takes about 45 minutes on 8 cores:
    python tests/golden/make_tip_velocity_2d.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

N, DX, DT, KAPPA, LAM, D0, T_END = 500, 0.4, 0.008, 4.0, 6.3826, 0.1385, 300.0


def run(n=N, t_end=T_END, every_time=5.0):
    p = oracle.make_params(W0=1.0, tau0=1.0, D=1.0, kappa=KAPPA, lam=LAM, Mc_inf=0.0, k=1.0, aniso=0,
                           eps1=0.05, eps2=0.0, dx=DX, dt=DT, antitrapping=0, grad2_min=1e-12)
    s = oracle.Sim((n, n, 1), (9, 5, 5), params=p)
    s.init_seed([[-0.5, -0.5, 0.0]], [10.0], U0=0.0, theta0=-0.55)
    every = int(round(every_time / DT))
    hist = []
    for k in range(every, int(round(t_end / DT)) + 1, every):
        s.step(every)
        x, _ = s.tip((0, 0, 0))
        hist.append((k * DT, x))
    return hist


def velocity_p(hist, t, span=10.0):
    """V_p = (dx * d x_tip / dt) d0 / kappa from a centred difference of the history."""
    d = dict((round(a, 6), b) for a, b in hist)
    ta, tb = round(t - span, 6), round(t, 6)
    return (d[tb] - d[ta]) * DX / (tb - ta) * D0 / KAPPA


if __name__ == "__main__":
    t0 = time.time()
    hist = run()
    out = {"citation": "Sec. 4.1, anisotropic pure-substance benchmark; paper value V_p(t=300) = 0.01735",
           "paper_vp_t300": 0.01735, "oracle_vp_t300": velocity_p(hist, 300.0),
           "oracle_vp_t100": velocity_p(hist, 100.0), "history_t_xtip": hist,
           "runtime_s": time.time() - t0}
    with open(os.path.join(HERE, "tip_velocity_2d_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["oracle_vp_t300"], out["paper_vp_t300"])
