#!/usr/bin/env python
"""Benchmark: coupled phi/U/theta lattice-Boltzmann site-updates per second.

Workload: 512^3 nodes, D3Q19 for phi, U and theta, FP32 storage and arithmetic,
two-harmonic anisotropy (eps = -0.02, delta = 0.015), four seeds R0 = 6 placed by
default_rng(7) at least 80 cells apart, Delta = 0.5, theta0 = -0.3 (seeded,
synthetic; shaped like the paper's 3D dendrite runs).  One step = the phase-field
kernel plus the U/theta kernel (all populations read once and written once).

Own arm (default): N ranks each advance an independent replica (weak scaling).
`value` = sites x steps x ranks / max-over-ranks device time.  The JSON line also
carries the roofline of the dominant kernel (k_uth, 38 populations per site), the
FP64 oracle's throughput on a bounded sample (cpu_baseline), an end-to-end number
through the C ABI with host buffers, and the SM clocks seen during the timed region.

Reference arm (--impl reference): the FP64 CPU oracle on the host cores, on a
bounded sample of the same workload (there is no GPU reference implementation).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled phi/U/theta site-updates/s (GLUPS) and % HBM roofline, FP32/FP16 vs FP64"
UNIT = "GLUPS"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def job_rate(t_local, units_local, device="cuda"):
    """Whole-job throughput of N ranks that each advance their own replica (weak scaling):
    the units all ranks processed over the slowest rank's timed span.  Returns
    (units / second, slowest span in seconds, total units)."""
    import torch
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized() and \
            torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(u, op=torch.distributed.ReduceOp.SUM)
    t_max, units = float(t.item()), float(u.item())
    return units / t_max, t_max, units


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class OracleSample:
    """The FP64 oracle on a bounded sample of the workload: an edge^3 box with the same
    lattices and parameters and one seed.  rate() steps it until a time budget is used
    and returns site-updates/s."""

    def __init__(self, edge=64):
        import oracle
        from paper_1602_07483_gb300 import workloads
        w = workloads.large_kh(512)
        self.edge = edge
        self.sim = oracle.Sim((edge, edge, edge), w.lattices, params=oracle.make_params(**dict(w.params)))
        self.sim.init_seed([[edge / 2, edge / 2, edge / 2]], [6.0], w.U0, w.theta0)
        self.sim.step(1)

    def rate(self, budget_s):
        steps, t0 = 0, time.perf_counter()
        while True:
            self.sim.step(1)
            steps += 1
            el = time.perf_counter() - t0
            if el > budget_s or steps >= 400:
                return self.edge ** 3 * steps / el, steps, el


def oracle_rate(budget_s=12.0, edge=64, threads=None):
    """FP64 oracle site-updates/s on a bounded sample of the workload (see OracleSample), on all
    host cores in this process and on one thread in a child process."""
    rate, steps, el = OracleSample(edge).rate(budget_s)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    one = oracle_rate_one_thread(budget_s=max(2.0, budget_s / 2), edge=32)
    return rate / 1e9, {"value": rate / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                        "sample": "%d^3 box of the 512^3 D3Q19x3 workload (same parameters, one seed), "
                                  "%d steps in %.1f s, FP64, OpenMP over z" % (edge, steps, el),
                        "single_thread": one}


def oracle_rate_one_thread(budget_s=6.0, edge=32):
    """The same oracle sample on one host thread (OMP_NUM_THREADS=1 in a child process)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "r, n, el = bench.OracleSample(%d).rate(%r); print(json.dumps([r, n, el]))" % (ROOT, edge, budget_s))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        r, n, el = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # the CPU leg must not hide the GPU result
        return {"value": None, "cores": 1, "sample": "failed: %s" % e}
    return {"value": r / 1e9, "unit": UNIT, "cores": 1,
            "sample": "%d^3 box, %d steps in %.1f s, FP64, one thread" % (edge, n, el)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    vals = []
    t_all = time.perf_counter()
    # bounded samples of one 64^3 box: about 20 s of warm-up and 100 s of timed samples in all
    sample = OracleSample(64)
    for _ in range(args.warmup):
        sample.rate(max(0.1, min(2.0, 20.0 / max(1, args.warmup))))
    total_steps, total_s = 0, 0.0
    for _ in range(args.steps):
        r, n, el = sample.rate(max(0.2, min(12.0, 100.0 / max(1, args.steps))))
        vals.append(r / 1e9)
        total_steps += n
        total_s += el
    value = statistics.median(vals)
    cb = {"value": value, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
          "kind": "oracle",
          "sample": "64^3 box of the 512^3 D3Q19x3 workload (same parameters, one seed), FP64, OpenMP over z; "
                    "%d samples, %d oracle steps in %.1f s, median rate" % (args.steps, total_steps, total_s)}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 64 ** 3 / (value * 1e9) * 1e3,  # one step of the sampled 64^3 box, measured
        "implied_ms_per_step_512": 512 ** 3 / (value * 1e9) * 1e3,  # a 512^3 step at the sampled rate
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "kh512_q19x3 (bounded CPU sample: each step is one step of a 64^3 box of it)",
                   "grid": [512, 512, 512], "lattices": [19, 19, 19]},
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_all,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_own(args):
    import numpy as np
    import torch
    from paper_1602_07483_gb300 import build, lbpf, workloads

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    build.build()
    st = torch.cuda.Stream()  # a real stream: the library enqueues on it and events are recorded on it
    torch.cuda.set_stream(st)
    if args.workload == "pure2d":
        w = workloads.pure_substance_2d(n=args.n if args.n != 512 else 8192, storage=args.storage)
    else:
        w = workloads.large_kh(args.n, storage=args.storage)
    hbm, peak_src = measured_peaks()

    def barrier_sync():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    sim = lbpf.Sim(w.grid, w.lattices, storage=args.storage, stream=st.cuda_stream, **w.params)
    sim.init_seed(w.centres, w.radii, w.U0, w.theta0)
    sim.set_schedule(args.schedule)
    if args.autotune:
        sim.autotune(steps=2)
    by, zchunk = sim.get_tiling()
    sim.step(args.warmup)
    barrier_sync()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    # the K timed steps as up to five back-to-back runs, each timed with CUDA events; the
    # line's value covers all K steps, and the median of the runs is reported beside it
    nruns = 5 if args.steps >= 5 else 1
    split = [args.steps // nruns + (1 if r < args.steps % nruns else 0) for r in range(nruns)]
    ms_phi = ms_uth = ms_span = 0.0
    run_rates = []
    for k in split:
        a, b, c = sim.step_timed(k)
        ms_phi, ms_uth, ms_span = ms_phi + a, ms_uth + b, ms_span + c
        run_rates.append(w.sites * k / (c * 1e-3) / 1e9)
    barrier_sync()
    clk = clocks.stop()
    # the FP64 diagnostics reduction (lbpf_sums: four sums over all sites, read back to the host)
    sim.sums(check=False)
    t0 = time.perf_counter()
    for _ in range(10):
        sim.sums(check=False)
    sums_ms = (time.perf_counter() - t0) / 10 * 1e3
    developed = None
    if args.developed and rank == 0 and world == 1 and args.workload == "kh":
        # the same simulation after it has grown for `developed` steps from the seeds
        sim.step(max(0, args.developed - args.warmup - args.steps))
        dk = 50
        d_phi, d_uth, d_span = sim.step_timed(dk)
        developed = {"after_steps": sim.steps_done - dk, "steps": dk, "GLUPS": w.sites * dk / (d_span * 1e-3) / 1e9,
                     "phi_ms": d_phi / dk, "uth_ms": d_uth / dk,
                     "what": "the timed simulation advanced to step %d, then %d steps timed as above" % (
                         sim.steps_done - dk, dk)}
    sites = w.sites
    rate, t_max, _ = job_rate(ms_span / 1e3, sites * args.steps)
    value = rate / 1e9
    # roofline of the dominant kernel: algorithmic bytes = read + write of every population it owns
    q_phi, q_u, q_t = w.lattices
    s_bytes = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[args.storage]
    bytes_uth = 2 * s_bytes * (q_u + q_t) * sites
    bytes_phi = 2 * s_bytes * q_phi * sites
    uth_ms = ms_uth / args.steps
    phi_ms = ms_phi / args.steps
    dom = ("k_uth", bytes_uth, uth_ms) if ms_uth >= ms_phi else ("k_phi", bytes_phi, phi_ms)
    if args.schedule == "one_launch":  # one kernel per step: its time is the phase-field entry
        dom = ("k_step", bytes_uth + bytes_phi, phi_ms)
    achieved = dom[1] / (dom[2] * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            with open(tr_path) as f:
                tr = json.load(f)
            ent = tr.get(dom[0])
            if ent and ent.get("source_hash") == kernel_source_hash():
                traffic = ent["bytes_per_launch_full"]
        except Exception:
            traffic = None
    step_alg = 2 * s_bytes * (q_phi + q_u + q_t) * sites / (t_max / args.steps) / 1e9

    # end to end through the C ABI: seeds uploaded from host memory, each step followed by a
    # device->host read of the step's diagnostics (FP64 sums), final phi field read back to pinned memory
    e2e = None
    if rank == 0 or world > 1:
        ke = max(2, min(50, args.steps // 2))
        phi_host = torch.empty(tuple(reversed(w.grid)), dtype=torch.float64, pin_memory=True).numpy()
        barrier_sync()
        t0 = time.perf_counter()
        sim.init_seed(w.centres, w.radii, w.U0, w.theta0)
        for _ in range(ke):
            sim.step(1)
            sim.sums(check=False)
        sim.read_fields(lbpf.LBPF_PHI, out=[phi_host, None, None])
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e_rate, _, _ = job_rate(te, sites * ke)
        h2d = (w.centres.size + w.radii.size) * 8 / ke
        d2h = 32 + sites * 8 / ke
        e2e = {"value": e2e_rate / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": ke,
               "what": "lbpf_init_seed from host seeds, then per step lbpf_step(1) + lbpf_sums (D2H), "
                       "then lbpf_read_fields(phi) into pinned host memory"}
    sim.close()
    del sim
    torch.cuda.empty_cache()

    variants = {}
    if args.variants and rank == 0 and world == 1 and args.workload == "kh":
        variants = run_variants(args, st)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.workload == "kh":
        try:
            _, cpu = oracle_rate(budget_s=12.0, edge=64)
        except Exception as e:  # the CPU leg must not hide the GPU result
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": "failed: %s" % e}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.storage == "f64" else "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.grid),
                       "lattices": [q_phi, q_u, q_t], "storage": args.storage,
                       "anisotropy": ("K41+K61 eps=-0.02 delta=0.015" if args.workload == "kh"
                                      else "cubic eps=0.05 (2D, Sec. 4.1 benchmark)"),
                       "seeds": len(w.radii),
                       "l2": "inputs larger than L2 (%.1f GB of populations)" % (
                           2 * s_bytes * (q_phi + q_u + q_t) * sites / 1e9),
                       "tiling": {"block": [32, by], "zchunk": zchunk}, "schedule": args.schedule,
                       "parallelism": "replicas x%d" % world},
            "roofline": {"bound": "hbm", "kernel": dom[0], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
                         "alg_bytes_per_launch": dom[1], "ms_per_launch": dom[2],
                         "phi_kernel": ({"ms": phi_ms, "GBps": bytes_phi / (phi_ms * 1e-3) / 1e9}
                                        if args.schedule == "two_kernels" else None),
                         "uth_kernel": ({"ms": uth_ms, "GBps": bytes_uth / (uth_ms * 1e-3) / 1e9}
                                        if args.schedule == "two_kernels" else None),
                         "step_alg_GBps": step_alg, "step_frac": step_alg / hbm},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": (1 if args.schedule == "one_launch" else 2) * args.steps,
            "clocks": clk,
            "developed": developed,
            "sums_ms": sums_ms,
            "runs": {"steps": split, "GLUPS": run_rates, "median_GLUPS": sorted(run_rates)[len(run_rates) // 2]},
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("lbpf_dev.cuh",):
        with open(os.path.join(ROOT, "paper_1602_07483_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _timed(s, k):
    """Per-kernel and whole-step device times of k steps of a simulation (ms per step)."""
    ms_phi, ms_uth, span = s.step_timed(k)
    return ms_phi / k, ms_uth / k, span / k


def fp64_peak_gflops(st, n=8192, reps=5):
    """Measured FP64 arithmetic rate of this GPU: a cuBLAS DGEMM (2 n^3 flops), timed with
    CUDA events on the bench stream after one warm-up; the denominator of the FP64 form."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(st):
        c = a @ b
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            c = a @ b
        e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del a, b, c
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (ms * 1e-3) / 1e9


def run_variants(args, st):
    """The FP16-storage form at 512^3, the plain FP64 form at 256^3, the same 512^3 workload
    with interface at most sites, the 2D scheme in FP32 on 8192^2, and the batched FP16
    sweep of 64 uneven simulations against the same simulations one by one in FP64."""
    import torch
    from paper_1602_07483_gb300 import lbpf, workloads
    hbm, _ = measured_peaks()
    out = {}
    for name, w, storage, k in (("f16", workloads.large_kh(args.n), "f16", 10),
                                ("f64", workloads.large_kh(256), "f64", 6),
                                ("dense_interface_f32", workloads.dense_kh(args.n), "f32", 10)):
        s = lbpf.Sim(w.grid, w.lattices, storage=storage, stream=st.cuda_stream, **w.params)
        s.init_seed(w.centres, w.radii, w.U0, w.theta0)
        s.step(3)
        torch.cuda.synchronize()
        phi_ms, uth_ms, ms = _timed(s, k)
        sb = {"f16": 2, "f32": 4, "f64": 8}[storage]
        glups = w.sites / (ms * 1e-3) / 1e9
        alg = glups * 2 * sb * 57
        out[name] = {"grid": list(w.grid), "storage": storage, "GLUPS": glups, "ms_per_step": ms,
                     "phi_ms": phi_ms, "uth_ms": uth_ms, "alg_GBps": alg, "hbm_frac": alg / hbm}
        if name == "f64":
            out[name]["fp64_GFLOPs"] = glups * 687  # FP64 operations per site-update counted by ncu (halo included)
            peak = fp64_peak_gflops(st)
            out[name]["fp64_peak_GFLOPs"] = peak
            out[name]["fp64_frac"] = glups * 687 / peak
            out[name]["fp64_peak_source"] = "cuBLAS DGEMM 8192^3 through torch.matmul, CUDA events, this run"
        if name.startswith("dense"):
            out[name]["seeds"] = len(w.radii)
        s.close()
        del s
        torch.cuda.empty_cache()
    # the 2D scheme (Sec. 4.1 benchmark recipe, D2Q9 phi, D2Q5 U and theta) on a large plane
    w = workloads.pure_substance_2d(n=8192, storage="f32")
    s = lbpf.Sim(w.grid, w.lattices, storage="f32", stream=st.cuda_stream, **w.params)
    s.init_seed(w.centres, w.radii, w.U0, w.theta0)
    s.step(3)
    torch.cuda.synchronize()
    phi_ms, uth_ms, ms = _timed(s, 10)
    glups = w.sites / (ms * 1e-3) / 1e9
    alg = glups * 2 * 4 * sum(w.lattices)
    out["pure2d_f32"] = {"grid": [8192, 8192, 1], "lattices": list(w.lattices), "GLUPS": glups, "ms_per_step": ms,
                         "alg_GBps": alg, "hbm_frac": alg / hbm, "phi_ms": phi_ms, "uth_ms": uth_ms}
    s.close()
    del s
    torch.cuda.empty_cache()
    out["sweep_f16"] = run_sweep(st, hbm)
    return out


def run_sweep(st, hbm, steps=60, base_steps=12):
    """The batched parameter sweep: 64 simulations with edges from {48, 64, 80, 96}, Delta, eps
    and k drawn by default_rng(11), FP16 storage, advanced together by one library-owned batch
    (tiling autotuned, graph-replayed steps, CUDA events on the batch stream); then the same simulations one by one
    in plain FP64.  Algorithmic bytes: 2 x 2 B x 38 populations = 152 B per FP16 site-update."""
    import numpy as np
    import torch
    from paper_1602_07483_gb300 import lbpf, workloads
    ws = workloads.batch_sweep(count=64, storage="f16")
    sites = sum(w.sites for w in ws)
    b = lbpf.batch_from_workloads(ws, stream=st.cuda_stream)
    b.autotune(steps=12)  # keeps the fastest batch tiling; the members' state is restored
    tiling = b.get_tiling()
    b.step(6)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    b.step(steps)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    nonfinite = [i for i, m in enumerate(b.sims) if not np.all(np.isfinite(m.sums(check=False)))]
    b.close()
    del b
    glups = sites * steps / (ms * 1e-3) / 1e9
    t_one = 0.0
    for w in ws:
        s = lbpf.Sim(w.grid, w.lattices, storage="f64", stream=st.cuda_stream, **w.params)
        s.init_seed(w.centres, w.radii, w.U0, w.theta0)
        s.step(6)
        torch.cuda.synchronize()
        e0.record(st)
        s.step(base_steps)
        e1.record(st)
        e1.synchronize()
        t_one += e0.elapsed_time(e1)
        s.close()
    torch.cuda.empty_cache()
    base = sites * base_steps / (t_one * 1e-3) / 1e9
    return {"sims": len(ws), "sites": sites, "steps": steps, "storage": "f16",
            "tiling": {"block_rows": tiling[0], "zchunk": tiling[1]}, "GLUPS": glups,
            "alg_GBps": glups * 152, "hbm_frac": glups * 152 / hbm, "one_by_one_f64_GLUPS": base,
            "one_by_one_f64_steps": base_steps, "speedup": glups / base, "nonfinite_sims": nonfinite}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--n", type=int, default=512, help="grid edge (the workload is defined at 512)")
    ap.add_argument("--workload", default="kh", choices=["kh", "pure2d"],
                    help="kh: the 512^3 D3Q19x3 two-harmonic dendrites (the headline); pure2d: the 2D "
                         "Sec. 4.1 benchmark recipe on an n^2 plane (8192^2 unless --n is given)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "f64"],
                    help="population storage (the headline line is f32)")
    ap.add_argument("--autotune", type=int, default=0)
    ap.add_argument("--schedule", default="two_kernels", choices=["two_kernels", "one_launch"],
                    help="step schedule (lbpf_set_schedule): the two step kernels, or one persistent launch")
    ap.add_argument("--variants", type=int, default=1)
    ap.add_argument("--developed", type=int, default=2000,
                    help="also time the headline simulation after it has run this many steps (0: skip)")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_own(args)


if __name__ == "__main__":
    sys.exit(main())
