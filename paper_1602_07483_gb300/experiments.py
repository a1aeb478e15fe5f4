"""Runs of the workloads that report accuracy and throughput per precision.

    python -m paper_1602_07483_gb300.experiments precision   # 256^3 coupled run, FP64/FP32/FP16
    python -m paper_1602_07483_gb300.experiments dendrite    # 128^3, tip every 100 steps, D3Q19 and D3Q7 phi
    python -m paper_1602_07483_gb300.experiments sweep       # 64 uneven simulations, batched FP16 vs one-by-one FP64
    python -m paper_1602_07483_gb300.experiments pure2d      # 2D benchmark of Sec. 4.1, V_p(t) per precision
    python -m paper_1602_07483_gb300.experiments anisotropy  # grid anisotropy A_g of a 301^3 sphere, D3Q7/15/19

Every number comes from the CUDA library through its C ABI; each run prints one
JSON object.  FP32/FP16 errors are measured against the FP64 GPU path, which the
test-suite pins to the CPU oracle step by step.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import build, lbpf, workloads


def _sync():
    try:
        import torch
        torch.cuda.synchronize()
    except Exception:
        pass


def _tip_series(sim, centre, steps, every, stop_margin=None, n=None):
    """Tip position every `every` steps; stops early once the tip is within
    `stop_margin` nodes of the +x wall (the tip line then no longer crosses phi = 0)."""
    xs = []
    done = 0
    while done < steps:
        k = min(every, steps - done)
        sim.step(k)
        done += k
        x, rho = sim.tip(centre)
        xs.append((done, x, rho))
        if stop_margin is not None and (x < 0 or x > n - 1 - stop_margin):
            break
    return xs


def _velocity(series, dx, dt, window, end_step=None):
    """Mean tip speed (physical units) over `window` steps ending at `end_step` (default:
    the last sample whose tip is inside the domain)."""
    valid = [r for r in series if r[1] >= 0]
    if not valid:
        return None, None
    end = valid[-1] if end_step is None else min(valid, key=lambda r: abs(r[0] - end_step))
    start = min(valid, key=lambda r: abs((end[0] - r[0]) - window))
    if end[0] == start[0]:
        return None, None
    return (end[1] - start[1]) * dx / ((end[0] - start[0]) * dt), (start[0], end[0])


def precision(n=256, steps=8000, every=50, linf_at=200, window=2000, storages=("f64", "f32", "f16", "bf16")):
    """The coupled heat + solute workload in several storage precisions.  The FP64 run
    stops once its tip nears the +x wall; the others then run exactly as many steps so
    that velocities and radii are compared over the same window."""
    w = workloads.coupled_dendrite(n=n)
    c = [int(v) for v in w.centres[0]]
    out = {"workload": w.name.replace("_f64", ""), "grid": n, "steps_requested": steps, "dt": w.params["dt"],
           "runs": {}}
    ref_fields = ref_v = ref_rho = None
    stop_at = steps
    win = None
    for st in storages:
        s = lbpf.sim_from_workload(w, storage=st)
        s.step(linf_at)
        f200 = s.read_fields()
        _sync()
        t0 = time.perf_counter()
        if st == "f64":
            series = [(linf_at + a, b, r) for a, b, r in _tip_series(s, c, steps - linf_at, every, 8, n)]
            stop_at = series[-1][0]
        else:
            series = [(linf_at + a, b, r) for a, b, r in _tip_series(s, c, stop_at - linf_at, every)]
        _sync()
        el = time.perf_counter() - t0
        if st == "f64":
            v, win = _velocity(series, w.params["dx"], w.params["dt"], window)
            end = win[1] if win else None
        else:
            v, _ = _velocity(series, w.params["dx"], w.params["dt"], window, end_step=win[1] if win else None)
        rho = dict((a, r) for a, _, r in series).get(win[1] if win else -1, -1.0)
        r = {"steps_run": series[-1][0], "GLUPS_incl_diagnostics": w.sites * (series[-1][0] - linf_at) / el / 1e9,
             "tip_velocity": v, "velocity_window_steps": win, "tip_radius_at_window_end": rho,
             "sums_final": s.sums(check=False).tolist()}
        if st == "f64":
            ref_fields, ref_v, ref_rho = f200, v, rho
        else:
            r["phi_linf_at_%d" % linf_at] = float(np.abs(f200[0] - ref_fields[0]).max())
            r["U_linf_at_%d" % linf_at] = float(np.abs(f200[1] - ref_fields[1]).max())
            r["theta_linf_at_%d" % linf_at] = float(np.abs(f200[2] - ref_fields[2]).max())
            if v is not None and ref_v:
                r["tip_velocity_rel_err"] = v / ref_v - 1
            if ref_rho and ref_rho > 0 and rho > 0:
                r["tip_radius_rel_err"] = rho / ref_rho - 1
        out["runs"][st] = r
        s.close()
        print(json.dumps({st: r}), file=sys.stderr, flush=True)
    return out


def dendrite(n=128, steps=5000, every=100):
    """The single 3D dendrite with D3Q19 and with D3Q7 for phi: tip position every
    `every` steps (until the tip nears the wall), tip speed over the last 1000 steps
    before that, in physical units and as V d0 / D."""
    out = {"grid": n, "steps_requested": steps, "runs": {}}
    for qphi in (19, 7):
        w = workloads.single_dendrite(q_phi=qphi).with_(grid=(n, n, n))
        c = [int(v) for v in w.centres[0]]
        s = lbpf.sim_from_workload(w, storage="f64")
        series = _tip_series(s, c, steps, every, 8, n)
        v, win = _velocity(series, w.params["dx"], w.params["dt"], 1000)
        d0 = 5 * np.sqrt(2) / 8 * w.params["W0"] / w.params["lam"]
        out["runs"]["phi_D3Q%d" % qphi] = {
            "tip_series": [(k, round(x, 4), round(r, 4)) for k, x, r in series],
            "tip_velocity": v, "velocity_window_steps": win,
            "tip_velocity_d0_over_D": (v * d0 / w.params["D"]) if v else None, "d0": d0,
        }
        s.close()
    return out


def pure2d(n=500, storages=("f64", "f32", "f16", "bf16")):
    """The 2D pure-substance benchmark of Sec. 4.1 (Delta = 0.55, D2Q9 phi, D2Q5 theta):
    tip position every 5 time units to t = 300 and V_p = V d0/kappa over the last 10
    time units, per storage precision, against the paper's V_p(300) = 0.01735."""
    w = workloads.pure_substance_2d(n=n)
    dt, dx, d0, kappa = w.params["dt"], w.params["dx"], w.extra["d0"], w.params["kappa"]
    out = {"workload": w.name.replace("_f64", ""), "grid": list(w.grid), "steps": w.steps,
           "vp_paper_t300": w.extra["vp_paper_t300"], "runs": {}}
    ref = None
    for st in storages:
        s = lbpf.sim_from_workload(w, storage=st)
        _sync()
        t0 = time.perf_counter()
        xs = []
        for k in range(w.tip_every, w.steps + 1, w.tip_every):
            s.step(w.tip_every)
            xs.append((k * dt, s.tip((0, 0, 0))[0]))
        _sync()
        el = time.perf_counter() - t0
        s.close()
        vp = {}
        for t in (100.0, 200.0, 300.0):
            d = dict((round(a, 6), b) for a, b in xs)
            vp[t] = (d[round(t, 6)] - d[round(t - 10.0, 6)]) * dx / 10.0 * d0 / kappa
        r = {"vp_t100": vp[100.0], "vp_t200": vp[200.0], "vp_t300": vp[300.0],
             "vp_t300_rel_to_paper": vp[300.0] / w.extra["vp_paper_t300"] - 1,
             "x_tip_t300": xs[-1][1], "GLUPS_incl_tip_every_625_steps": w.sites * w.steps / el / 1e9}
        if st == "f64":
            ref = vp[300.0]
        else:
            r["vp_t300_rel_to_f64"] = vp[300.0] / ref - 1
        out["runs"][st] = r
        print(json.dumps({st: r}), file=sys.stderr, flush=True)
    return out


def radii_100_110(phi, c):
    """Radii of the phi = 0 surface from the centre node c along (1,0,0) and (1,1,0):
    first crossing phi >= 0 > phi_next on the node line, linearly interpolated; the
    (1,1,0) distance is sqrt2 times the node-step index.  Returns (R100, R110, A_g %)
    with A_g = |R100 - R110| / (R100 + R110) x 100 (Sec. 4.1)."""
    def crossing(line):
        i = int(np.where((line[:-1] >= 0) & (line[1:] < 0))[0][0])
        return i + line[i] / (line[i] - line[i + 1])
    r100 = crossing(phi[c, c, c:])
    m = min(phi.shape[1], phi.shape[2]) - c
    r110 = np.sqrt(2.0) * crossing(np.array([phi[c, c + j, c + j] for j in range(m)]))
    return float(r100), float(r110), float(abs(r100 - r110) / (r100 + r110) * 100)


def anisotropy(n=301, storage="f32", steps=None):
    """Grid anisotropy A_g of an isotropic growing sphere (Sec. 4.1) for the phase field on
    D3Q7, D3Q15 and D3Q19, against the paper's 3.095 / 0.073 / 0.116 %."""
    out = {"grid": n, "storage": storage, "runs": {}}
    for q in (7, 15, 19):
        w = workloads.grid_anisotropy(q_phi=q, n=n, storage=storage)
        k = steps or w.steps
        s = lbpf.sim_from_workload(w)
        _sync()
        t0 = time.perf_counter()
        s.step(k)
        phi = s.read_fields(lbpf.LBPF_PHI)[0]
        el = time.perf_counter() - t0
        s.close()
        c = n // 2
        r100, r110, ag = radii_100_110(phi, c)
        out["runs"]["phi_D3Q%d" % q] = {"steps": k, "R100": r100, "R110": r110, "Ag_pct": ag,
                                        "Ag_paper_pct": w.extra["Ag_paper_pct"], "seconds": el}
        print(json.dumps({q: out["runs"]["phi_D3Q%d" % q]}), file=sys.stderr, flush=True)
    return out


def sweep(count=64, steps=2000, baseline_steps=200):
    """The batched sweep: `count` uneven FP16-storage simulations advanced together
    (tiling autotuned first), against the same simulations one by one in FP64."""
    sims = workloads.batch_sweep(count=count, storage="f16")
    sites = sum(w.sites for w in sims)
    members = [lbpf.sim_from_workload(w) for w in sims]
    batch = lbpf.Batch(members)
    batch.autotune(steps=24)  # fastest tiling kept, members restored to their seeds
    tiling = batch.get_tiling()
    batch.step(6)
    _sync()
    members[0].sums(check=False)
    t0 = time.perf_counter()
    batch.step(steps)
    members[0].sums(check=False)
    _sync()
    el = time.perf_counter() - t0
    nan = [i for i, m in enumerate(members) if not np.all(np.isfinite(m.sums(check=False)))]
    batch.close()
    for m in members:
        m.close()
    # one-by-one plain FP64 on the same simulations (fewer steps; a rate)
    t_one = 0.0
    for w in sims:
        s = lbpf.sim_from_workload(w, storage="f64")
        s.step(6)
        s.sums(check=False)
        t0 = time.perf_counter()
        s.step(baseline_steps)
        s.sums(check=False)
        t_one += time.perf_counter() - t0
        s.close()
    return {"sims": count, "sites": sites, "steps": steps, "batch_tiling": {"block_rows": tiling[0], "zchunk": tiling[1]},
            "batched_f16_GLUPS": sites * steps / el / 1e9,
            "one_by_one_f64_GLUPS": sites * baseline_steps / t_one / 1e9,
            "nonfinite_sims": nan}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["precision", "dendrite", "sweep", "pure2d", "anisotropy"])
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--steps", type=int, default=0)
    a = ap.parse_args()
    build.build()
    kw = {}
    if a.n:
        kw["n"] = a.n
    if a.steps:
        kw["steps"] = a.steps
    fn = {"precision": precision, "dendrite": dendrite, "sweep": sweep, "pure2d": pure2d,
          "anisotropy": anisotropy}[a.which]
    print(json.dumps(fn(**kw)))


if __name__ == "__main__":
    main()
