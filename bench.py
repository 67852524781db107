#!/usr/bin/env python
"""Throughput of the electrostatic PIC hot path on one B300 (or N replicas).

Metric: particle-steps per second of gather + Boris push + move + CIC deposit
(the fused particle pass plus the int64 -> rho conversion), with the per-cell
sort at its cadence, on the 2D two-stream workload: 512 x 512 nodes, dx = 1,
64 electrons per cell (16,777,216), beams at +-3 v_te with v_te = 1, dt = 0.1,
sort every 20 steps.  One step of the timed loop = one pass of those stages
over every particle; particle state (335 MB) is larger than L2, so no L2
flush is needed between steps.  The field solve (Jacobi-PCG + E, and the
spectral solve) is run and timed separately; the end-to-end number runs the
full cycle with the spectral solve (and, for a few steps, with the CG).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun each rank runs an independent replica (the single-instance
path does not shard): value = all ranks' particle-steps / max rank time.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on this host's cores.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "particle-steps/s (gather+push+deposit)"

# DRAM traffic (read + write bytes) of one k_particle_pass launch on the benchmark
# workload, from the ncu capture summarised in profiles/, with the hash of the
# kernel sources it was taken on: reported only while the sources are unchanged.
PASS_TRAFFIC = {
    "two_stream_2d 512x512 64ppc": {"bytes": 619777792, "sources": "88d899fd608d1caa"},
}
TRAFFIC_SOURCES = ("paper_2608_15249_b300/csrc/pic_particles.cu",
                   "paper_2608_15249_b300/csrc/pic_internal.cuh")


def _pass_traffic(key):
    import hashlib
    rec = PASS_TRAFFIC.get(key)
    if rec is None:
        return None
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest()[:16] == rec["sources"] else None
UNIT = "particle-steps/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6400.0, "fallback"


def _workload(args):
    if args.workload == "two_stream_2d":
        return workloads.two_stream_2d(n=(args.n, args.n), ppc=args.ppc, seed=2)
    if args.workload == "magnetized_3d":
        return workloads.magnetized_3d(n=(args.n,) * 3, ppc=args.ppc)
    if args.workload == "precision_3d":
        return workloads.precision_3d(n=(args.n,) * 3, ppc=args.ppc)
    raise SystemExit(f"unknown workload {args.workload}")


def _bytes_per_particle(ndim, nv, f64=False):
    if f64:  # FP64 plain form: ndim FP64 positions + nv FP64 velocities, read and written
        return 2 * (8 * ndim + 8 * nv)
    # cell (int32) + ndim FP32 offsets + nv FP32 velocities, read and written once
    return 2 * (4 + 4 * ndim + 4 * nv)


def _grid_bytes_per_node(ndim, f64=False):
    # E read (ndim FP32, or FP64) + the int64 accumulator written once
    return (8 if f64 else 4) * ndim + 8


def _spectral_bytes_per_node(ndim):
    """Algorithmic bytes per node of one spectral field solve: two transform solves
    (the solve and its refinement), each a pass per axis over the complex grid (the
    first reads the FP32 right-hand side, 4 + 8 B; the last writes the FP32
    potential, 8 + 4 B; the others 8 + 8 B; in 1D one real-to-real pass, 4 + 4 B),
    the refinement's last pass also reading the potential it adds to (4 B), the FP64
    residual (8 B charge accumulator + 4 B phi + 4 B out) and E = -grad phi (4 B + 4 B per
    axis)."""
    solve = 8 if ndim == 1 else 12 + 16 * (2 * ndim - 3) + 12
    return 2 * solve + 4 + 16 + 4 + 4 * ndim


NOMINAL_HBM_GBS = 7700.0  # B300 HBM3e nominal bandwidth, for the fraction beside the measured one


def _roofline(alg_bytes, ms, kernel, peak, peak_kind, traffic=None, **extra):
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
           "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": ms,
           "peak_kind": peak_kind,
           "frac_of_nominal": achieved / NOMINAL_HBM_GBS}
    out.update(extra)
    return out


def _timed(fn):
    t0 = time.perf_counter()
    out = fn()
    return out, time.perf_counter() - t0


class Clocks:
    """nvidia-smi sampled every 100 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:  # noqa: BLE001
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:  # noqa: BLE001
        return os.cpu_count() or 1


def _oracle_particle_steps(oracle, ndim, n, dx, dt, x, v, E, q, m, weight, E0, B0, steps):
    """`steps` of the oracle's gather + Boris push (with the kinetic-energy
    diagnostic) + move + deposit on x, v in place, in the field E (the timing does
    not depend on its values); returns the seconds."""
    t0 = time.perf_counter()
    for _ in range(steps):
        Ep = oracle.gather(ndim, n, dx, x, E)
        oracle.boris(ndim, v, Ep, E0, B0, q / m, dt)
        oracle.kinetic(v, m * weight)
        oracle.move(ndim, n, dx, x, v, dt)
        oracle.deposit(ndim, n, dx, x, q * weight)
    return time.perf_counter() - t0


def run_oracle_sample(w, sample_np, steps, warmup, threads=1):
    """The oracle's gather + push + move + deposit on `sample_np` particles of the
    workload (full grid, zero field: the field solve is not part of the metric),
    `warmup` untimed then `steps` timed steps, its particle loops on `threads`
    threads; returns (particle-steps/s, seconds)."""
    import oracle

    oracle.set_threads(threads)
    x = np.ascontiguousarray(w.x[:sample_np], dtype=np.float64)
    v = np.ascontiguousarray(w.v[:sample_np], dtype=np.float64)
    E = np.zeros(w.ndim * w.cells)
    args = (oracle, w.ndim, w.n, w.dx, w.dt, x, v, E, w.q, w.m, w.weight, w.E0, w.B0)
    _oracle_particle_steps(*args, warmup)
    dt = _oracle_particle_steps(*args, steps)
    oracle.set_threads(1)
    return sample_np * steps / dt, dt


def cpu_baseline(w, sample_np, steps, warmup=0):
    """The oracle on all host cores (the baseline) and on one thread, on the same
    bounded sample of the workload."""
    cores = host_cores()
    v1, s1 = run_oracle_sample(w, sample_np, steps, warmup, threads=1)
    vn, sn = (v1, s1) if cores == 1 else run_oracle_sample(w, sample_np, steps, warmup,
                                                           threads=cores)
    what = f"{sample_np} of {w.np_} particles on the full grid, {steps} steps of " \
           "gather+push+move+deposit"
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what} ({sn:.1f} s on {cores} threads)",
            "single_thread": {"value": v1, "cores": 1, "seconds": s1}}


def bench_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = _workload(args)
    sample = min(w.np_, args.ref_sample)
    cores = host_cores()
    val, secs = run_oracle_sample(w, sample, args.steps, args.warmup, threads=cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": _config(args, w),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} of {w.np_} particles on the full grid, "
                                   f"{args.steps} steps of gather+push+move+deposit "
                                   f"on {cores} threads"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(args, w):
    return {"workload": f"{w.name} {w.n[0]}x{w.n[1]}" + (f"x{w.n[2]}" if w.ndim == 3 else "")
            + f", {args.ppc} ppc, {w.np_} electrons, dt={w.dt}, sort every {w.sort_every}",
            "grid": list(w.n[: w.ndim]), "particles": w.np_, "ppc": args.ppc,
            "sort_every": w.sort_every, "parallelism": f"replicas x{args.gpus}",
            "storage": "FP64 plain" if args.precision == "f64" else "int32 cell + FP32 offset",
            "l2": "particle state larger than L2 (no flush)",
            "pusher": args.pusher if args.pusher == "boris"
            else f"higuera-cary, c = {args.c_light or 'infinite'}"}


def aggregate_replicas(ms, np_per_rank, steps, world, dist=None, device=None):
    """Max-over-ranks timed-region length and whole-job throughput of `world`
    independent replicas: (max ms, np_per_rank * steps * world / max seconds)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, np_per_rank * steps * world / (ms * 1e-3)


def _stage_timed(g, hot_step, k0, steps, stream, torch):
    """Runs steps k0 .. k0 + steps - 1 with the library's stage timing (CUDA events
    recorded around each stage on the handle's stream); returns the stage totals and the
    loop's ms per step."""
    torch.cuda.synchronize()
    g.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(k0, k0 + steps):
        hot_step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    stages = g.get_timing()
    g.set_timing(False)
    return stages, e0.elapsed_time(e1) / steps


def bench_ours(args):
    import torch

    import paper_2608_15249_b300 as pk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = _workload(args)
    f64 = args.precision == "f64"
    stream = torch.cuda.current_stream()
    extra = dict(precision=pk.AP_PIC_FP64_PLAIN) if f64 else {}
    if args.pusher == "hc":
        extra.update(pusher=pk.AP_PIC_PUSHER_HIGUERA_CARY, c_light=args.c_light)
    g = pk.from_workload(w, stream=stream.cuda_stream, cg_rtol=args.cg_rtol, **extra)
    g.load(w.x, w.v)
    sort_every = 0 if f64 else w.sort_every

    def hot_step(k):
        g.push_deposit()
        if sort_every and k % sort_every == 0:
            g.sort()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # the clock sampler starts first (it takes a moment to come up), so that the
    # warm-up steps, not an idle GPU, lead into the timed region
    with Clocks(local) as clk:
        for k in range(1, args.warmup + 1):
            hot_step(k)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = pk.kernel_launches()
        ev0.record(stream)
        for k in range(args.warmup + 1, args.warmup + args.steps + 1):
            hot_step(k)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = pk.kernel_launches() - launches0
    ms, value = aggregate_replicas(ev0.elapsed_time(ev1), w.np_, args.steps, world, dist,
                                   device="cuda")
    # the same steps again with CUDA events around every stage (the events add a few
    # microseconds per step, so the timed loop above runs without them): the pass's
    # launch durations for the roofline and the stage breakdown
    stages, ms_events = _stage_timed(g, hot_step, args.warmup + args.steps + 1, args.steps,
                                     stream, torch)

    # roofline of the dominant kernel (the fused particle pass)
    peak, peak_kind = _peaks()
    pd_ms, pd_n = stages["push_deposit"]
    avg_ms = pd_ms / max(pd_n, 1)
    alg_bytes = (w.np_ * _bytes_per_particle(w.ndim, w.nv, f64)
                 + w.cells * _grid_bytes_per_node(w.ndim, f64))
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    breakdown = {k: (v[0] / max(v[1], 1)) for k, v in stages.items() if v[1]}

    # field solve timed separately (the CG, and the spectral solve where the form has
    # it), then the end-to-end job through host buffers
    g.set_timing(True)
    g.solve_field()
    fs = g.get_timing()["field"]
    g.set_timing(False)
    g.close()
    field_ms = {"cg": fs[0] / max(fs[1], 1)}
    if not f64:
        gf = pk.from_workload(w, stream=stream.cuda_stream, solver=pk.AP_PIC_SOLVER_FFT)
        gf.load(w.x, w.v)
        gf.solve_field()
        gf.set_timing(True)
        for _ in range(10):
            gf.solve_field()
        ff = gf.get_timing()["field"]
        gf.set_timing(False)
        gf.close()
        field_ms["fft"] = ff[0] / max(ff[1], 1)
    rows = not (f64 or args.no_rows)
    spectral = bench_spectral(args, w, field_ms["fft"], peak, peak_kind) if rows else None
    hc = bench_hc(args, w, pk, torch, stream, peak, peak_kind) if rows else None
    collisions = None if (f64 or args.no_collisions) else bench_collisions(
        args, pk, torch, stream, peak, peak_kind)
    em = None if (f64 or args.no_em) else bench_em(args, pk, torch, stream, peak, peak_kind)
    em3 = None if (f64 or args.no_em) else bench_em3(args, pk, torch, stream, peak, peak_kind)
    cpml = None if (f64 or args.no_em) else bench_cpml(args, pk, torch, stream, peak, peak_kind)
    e2e = None
    if not args.no_e2e:
        solver = "cg" if f64 else args.e2e_solver
        e2e = run_e2e(args, w, pk, torch, stream, dict(extra, solver=_SOLVERS[solver]),
                      args.e2e_steps)
        e2e["solver"] = solver
        if solver != "cg":
            other = run_e2e(args, w, pk, torch, stream, extra, args.e2e_steps_cg)
            e2e["cg"] = {"value": other["value"], "steps": other["steps"],
                         "seconds": other["seconds"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, min(w.np_, args.cpu_sample), args.cpu_steps)

    # the other single-GPU configurations of the metric: the 3D magnetised plasma and
    # the batch of uneven instances (with its per-instance FP64 plain comparison)
    configs = None
    if rank == 0 and world == 1 and not args.no_configs and w.name == "two_stream_2d":
        configs = {"magnetized_3d": run_config_3d(args, pk, torch, stream),
                   "batch": run_batch(args, pk, torch, stream, embedded=True)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if f64 else "f32", "data": "synthetic", "config": _config(args, w),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": None if (f64 or args.pusher != "boris") else _pass_traffic(
                             f"{w.name} {'x'.join(str(k) for k in w.n[:w.ndim])} {args.ppc}ppc"),
                         "kernel": ("k_plain_pass" if f64 else "k_particle_pass")
                         + " (gather+Boris+move+deposit)",
                         "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms,
                         "peak_kind": peak_kind,
                         "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "launch_ms_from": "CUDA events around each pass, a second run of "
                                           "the same steps"},
            "stage_ms_per_call": breakdown,
            "ms_per_step_with_stage_events": ms_events,
            "field_solve_ms": field_ms,
            "spectral_solve": spectral,
            "higuera_cary": hc,
            "collisions": collisions,
            "electromagnetic": em,
            "electromagnetic_3d": em3,
            "cpml_fields": cpml,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "configs": configs,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_config_3d(args, pk, torch, stream):
    """The 3D magnetised configuration (128^3 nodes, 64 ppc, 134,217,728 electrons,
    Maxwellian v_te = 1, B0 = 2 z, dt = 0.05, sort every 20): particle-steps/s of
    push + deposit with the sort at its cadence (CUDA events), the pass's roofline
    from the stage timing, clocks during the timed region, and the oracle on a bounded
    sample of the same workload."""
    w = workloads.magnetized_3d(n=(args.n3d,) * 3, ppc=args.ppc3d)
    g = pk.from_workload(w, stream=stream.cuda_stream, solver=pk.AP_PIC_SOLVER_FFT)
    t0 = time.perf_counter()
    g.load(w.x, w.v)
    torch.cuda.synchronize()
    load_s = time.perf_counter() - t0

    def hot_step(k):
        g.push_deposit()
        if k % w.sort_every == 0:
            g.sort()

    warm, steps = args.warmup, max(args.steps, w.sort_every)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for k in range(1, warm + 1):
            hot_step(k)
        torch.cuda.synchronize()
        launches0 = pk.kernel_launches()
        ev0.record(stream)
        for k in range(warm + 1, warm + steps + 1):
            hot_step(k)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = pk.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    st, ms_events = _stage_timed(g, hot_step, warm + steps + 1, steps, stream, torch)
    g.close()
    peak, peak_kind = _peaks()
    pd_ms = st["push_deposit"][0] / max(st["push_deposit"][1], 1)
    alg = w.np_ * _bytes_per_particle(3, 3) + w.cells * _grid_bytes_per_node(3)
    out = {"metric": METRIC, "value": w.np_ * steps / (ms * 1e-3), "unit": UNIT,
           "steps": steps, "warmup": warm, "ms_per_step": ms / steps,
           "config": {"workload": f"magnetized_3d {args.n3d}^3, {args.ppc3d} ppc, {w.np_} "
                                  f"electrons, B0 = 2 z, dt = {w.dt}, sort every {w.sort_every}",
                      "particles": w.np_, "load_seconds": load_s,
                      "l2": "particle state larger than L2 (no flush)"},
           "stage_ms_per_call": {k: v[0] / max(v[1], 1) for k, v in st.items() if v[1]},
           "ms_per_step_with_stage_events": ms_events,
           "roofline": _roofline(alg, pd_ms, "k_particle_pass (gather+Boris+move+deposit), 3D",
                                 peak, peak_kind,
                                 launch_ms_from="CUDA events around each pass, a second run "
                                                "of the same steps"),
           "gpu_launches": int(launches), "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, min(w.np_, args.cpu_sample_3d), args.cpu_steps_3d)
    return out


_SOLVERS = {"cg": 0, "fft": 1}

# Null-collision Monte Carlo of the benchmark's size: a 2D3V Maxwellian (collisions
# need three velocity components) on the same grid and particle count, constant
# cross sections giving a candidate fraction of about 4 % per step.
MCC_BENCH = dict(density=1.0, sigma_el=0.05, sigma_exc=0.02, eps_exc=1.5, mass_ratio=1e-4,
                 vmax=6.0, seed=99)


def _energy(g):
    d = g.get_diag()
    return d["kinetic"] + d["field_energy"]


def bench_precision(args):
    """The precision study: the FP32 cell + offset form against the FP64 plain form
    on the GPU, both against the FP64 oracle, on the 3D Maxwellian with 1 % white
    per-cell density noise (Jacobi-PCG field solve in every case):
      - full size (n^3, 16 ppc): L-infinity rho and E differences FP32 vs FP64 after
        `--prec-steps` steps, and the energy drift of each over those steps (relative
        to the total energy after the first step);
      - energy drift over `--drift-steps` steps on a (n/2)^3 grid;
      - both forms against the oracle after 10 steps on a 32^3 grid."""
    import torch

    import oracle
    import paper_2608_15249_b300 as pk

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    out = {"metric": "precision study (FP32 cell+offset vs FP64 plain vs FP64 oracle)",
           "data": "synthetic", "unit": "relative L-infinity / relative energy drift"}

    def pair(w, steps, track_energy):
        forms = {}
        for name, over in (("f32", {}), ("f64", dict(precision=pk.AP_PIC_FP64_PLAIN))):
            g = pk.from_workload(w, stream=stream.cuda_stream, sort_every=20, **over)
            g.load(w.x, w.v)
            t0 = time.perf_counter()
            # total energy (time-centred kinetic + field) from the first step on: the
            # load's diagnostics carry no kinetic energy yet
            g.step(1)
            e0 = _energy(g)
            drift = 0.0
            for _ in range(steps - 1):
                g.step(1)
                if track_energy:
                    drift = max(drift, abs(_energy(g) - e0) / e0)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            if not track_energy:
                drift = abs(_energy(g) - e0) / e0
            forms[name] = {"rho": g.get_rho(), "E": g.get_E(), "drift": drift, "seconds": secs,
                           "handle": g}
        return forms

    def linf(a, b):
        return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))

    # full size, a few steps
    n = args.n
    w = workloads.precision_3d(n=(n, n, n), ppc=args.ppc)
    f = pair(w, args.prec_steps, True)
    bg = w.weight * w.np_ / float(np.prod(w.L[:3]))  # the ions: rho_e = rho - bg (q = -1)
    rho_e_scale = float(np.max(np.abs(f["f64"]["rho"] - bg)))
    out["full"] = {
        "workload": f"precision_3d {n}^3, {args.ppc} ppc, {w.np_} electrons, "
                    f"{args.prec_steps} steps, CG field solve",
        "rho_f32_vs_f64": float(np.max(np.abs(f["f32"]["rho"] - f["f64"]["rho"]))) / rho_e_scale,
        "E_f32_vs_f64": linf(f["f32"]["E"], f["f64"]["E"]),
        "energy_drift": {"f32": f["f32"]["drift"], "f64": f["f64"]["drift"]},
        "seconds": {"f32": f["f32"]["seconds"], "f64": f["f64"]["seconds"]}}
    for v in f.values():
        v["handle"].close()
    del w, f
    # long run, smaller grid
    nd = max(8, n // 2)
    w = workloads.precision_3d(n=(nd, nd, nd), ppc=args.ppc, seed=14)
    f = pair(w, args.drift_steps, True)
    out["drift"] = {
        "workload": f"precision_3d {nd}^3, {args.ppc} ppc, {w.np_} electrons, "
                    f"{args.drift_steps} steps, CG field solve",
        "energy_drift_max": {"f32": f["f32"]["drift"], "f64": f["f64"]["drift"]},
        "E_f32_vs_f64_at_end": linf(f["f32"]["E"], f["f64"]["E"]),
        "seconds": {"f32": f["f32"]["seconds"], "f64": f["f64"]["seconds"]}}
    for v in f.values():
        v["handle"].close()
    del w, f
    # against the oracle
    no = 32
    w = workloads.precision_3d(n=(no, no, no), ppc=args.ppc, seed=24)
    f = pair(w, 10, False)
    sim = oracle.Simulation(3, w.n, w.dx, w.dt, weight=w.weight, rtol=1e-12).load(w.x, w.v)
    sim.step(10)
    scale = float(np.max(np.abs(sim.rho_e)))
    out["oracle"] = {
        "workload": f"precision_3d {no}^3, {args.ppc} ppc, {w.np_} electrons, 10 steps",
        "rho": {k: float(np.max(np.abs(f[k]["rho"] - sim.rho))) / scale for k in ("f32", "f64")},
        "E": {k: linf(f[k]["E"], sim.E) for k in ("f32", "f64")}}
    for v in f.values():
        v["handle"].close()
    print(json.dumps(out), flush=True)


def bench_em(args, pk, torch, stream, peak, peak_kind, steps=20):
    """CUDA-event time of full electromagnetic steps (particles with the Esirkepov
    current, Yee field update, sort every 20 steps) on a 2D3V Maxwellian of the
    benchmark's size, c = 4 v_te (Courant number 0.57); the roofline of its particle
    kernels (k_em_tile, k_em_spread: gather E and B, Boris, move, Esirkepov current; 48 B of
    record read and written per particle, E and B read and the int64 current
    written, 48 B per node) from the stage timing of separate steps; and the
    oracle's step on a sample of the particles on the same grid."""
    import oracle

    w = workloads.maxwellian_box(2, (args.n, args.n), ppc=args.ppc, nv=3, dt=0.1, seed=7)
    g = pk.from_workload(w, stream=stream.cuda_stream, em=1, c_light=4.0, sort_every=20)
    g.load(w.x, w.v)
    g.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    g.set_timing(True)
    g.step(steps)
    st = g.get_timing()
    g.set_timing(False)
    g.close()
    push_ms = st["push_deposit"][0] / max(st["push_deposit"][1], 1)
    field_ms = st["field"][0] / max(st["field"][1], 1)
    out = {"ms_per_step": ms, "particles": w.np_, "particle_steps_per_s": w.np_ / (ms * 1e-3),
           "stage_ms": {"em_particles": push_ms, "yee_fields": field_ms},
           "roofline": _roofline(w.np_ * 48 + w.cells * 48, push_ms,
                                 "k_em_tile + k_em_spread (gather E, B + Boris + move + Esirkepov current)",
                                 peak, peak_kind),
           "workload": f"maxwellian 2D3V {args.n}x{args.n}, {args.ppc} ppc, c = 4, dt = 0.1, "
                       "full electromagnetic step"}
    if not args.no_row_oracles:
        sample = min(w.np_, 1 << 20)
        sim = oracle.EmSimulation(w.n, w.dx, w.dt, 4.0, weight=w.weight, rtol=1e-6)
        sim.load(w.x[:sample], w.v[:sample])
        _, secs = _timed(lambda: sim.step(2))
        out["oracle"] = {"kind": "oracle", "cores": 1, "particle_steps_per_s": sample * 2 / secs,
                         "sample": f"{sample} of {w.np_} particles on the full grid, 2 full "
                                   f"electromagnetic steps ({secs:.1f} s)"}
    return out


def bench_em3(args, pk, torch, stream, peak, peak_kind, n=128, ppc=8, steps=10, sort_every=5):
    """CUDA-event time of full 3D electromagnetic steps (periodic 3D Yee lattice,
    particles with the 3D Esirkepov current, sorted every 5 steps into the step's
    default 4 x 4 x 4 bricks: the cadence with the shortest full step, as the particle
    kernel's fixed deposit windows hold more particles soon after a sort) on a 3D
    Maxwellian of 16.8M electrons (128^3 x 8 ppc), c = 3 v_te, dt = 0.1 (Courant number 0.52); the
    roofline of its particle kernel (56 B of record read and written per particle; E
    and B read, the int64 current and charge written: 56 B per node); the oracle's
    EmSimulation3 step on a sample of the particles on the same grid."""
    import oracle

    w = workloads.maxwellian_box(3, (n, n, n), ppc=ppc, nv=3, dt=0.1, seed=9)
    g = pk.from_workload(w, stream=stream.cuda_stream, em=1, c_light=3.0, sort_every=sort_every)
    g.load(w.x, w.v)
    g.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    g.set_timing(True)
    g.step(steps)
    st = g.get_timing()
    g.set_timing(False)
    g.close()
    push_ms = st["push_deposit"][0] / max(st["push_deposit"][1], 1)
    field_ms = st["field"][0] / max(st["field"][1], 1)
    out = {"ms_per_step": ms, "particles": w.np_, "particle_steps_per_s": w.np_ / (ms * 1e-3),
           "stage_ms": {"em_particles": push_ms, "yee_fields": field_ms},
           "roofline": _roofline(w.np_ * 56 + w.cells * 56, push_ms,
                                 "k_em3_push (gather E, B + Boris + move + 3D Esirkepov current)",
                                 peak, peak_kind),
           "workload": f"maxwellian 3D {n}^3, {ppc} ppc, c = 3, dt = 0.1, sort every "
                       f"{sort_every}, full 3D electromagnetic step"}
    if not args.no_row_oracles:
        sample = min(w.np_, 1 << 18)
        sim = oracle.EmSimulation3(w.n, w.dx, w.dt, 3.0, weight=w.weight, rtol=1e-6)
        sim.load(w.x[:sample], w.v[:sample])
        _, secs = _timed(lambda: sim.step(1))
        out["oracle"] = {"kind": "oracle", "cores": 1, "particle_steps_per_s": sample / secs,
                         "sample": f"{sample} of {w.np_} particles on the full grid, 1 full 3D "
                                   f"electromagnetic step ({secs:.1f} s)"}
    return out


def bench_cpml(args, pk, torch, stream, peak, peak_kind, n=2048, npml=16, steps=50):
    """The field-only electromagnetic step on a non-periodic n x n grid with a
    convolutional PML of npml cells on every side (c = 1, dt = 0.5, a prescribed
    current at the centre): CUDA-event time per step and its roofline.  Algorithmic
    bytes per node: two B half steps (12 B E read, 24 B B read and written, each) and
    the E step (12 B B read, 24 B E read and written, the int64 current read and
    cleared, 24 B each, 12 B prescribed current read), 168 B; plus, in the layers, the eight psi
    arrays read and written (64 B).  Beside it, the oracle's CpmlField step on a
    512 x 512 grid."""
    import oracle

    cfg = pk.make_config(2, (n, n), dt=0.5, nv=3, em=1, c_light=1.0, em_boundary=1,
                         pml_cells=npml, sort_every=0, diag_every=1 << 20)
    g = pk.Pic(cfg).load(np.zeros((0, 2)), np.zeros((0, 3)))
    J = np.zeros((3, n * n))
    J[2, n // 2 + n * (n // 2)] = 1.0
    g.set_current(J)
    g.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    g.close()
    nodes = n * n
    layer_nodes = nodes - (n - 2 * npml) ** 2
    out = {"ms_per_step": ms, "nodes": nodes, "node_steps_per_s": nodes / (ms * 1e-3),
           "roofline": _roofline(nodes * 168 + layer_nodes * 64, ms,
                                 "CPML field step (k_cpml_b x 2, k_cpml_e with the current conversion)",
                                 peak, peak_kind),
           "workload": f"non-periodic {n}x{n} grid, {npml}-cell CPML, c = 1, dt = 0.5, "
                       "prescribed current, fields only"}
    if not args.no_row_oracles:
        m = 512
        f = oracle.CpmlField((m, m), (1.0, 1.0), 0.5, 1.0, npml)
        Jo = np.zeros((3, m * m))
        Jo[2, m // 2 + m * (m // 2)] = 1.0
        _, secs = _timed(lambda: f.step(Jo, nsteps=16))
        out["oracle"] = {"kind": "oracle", "cores": 1, "node_steps_per_s": m * m * 16 / secs,
                         "sample": f"{m}x{m} grid, 16 steps ({secs:.2f} s)"}
    return out


def bench_collisions(args, pk, torch, stream, peak, peak_kind):
    """CUDA-event time of the collision pass alone (ap_pic_collide) on 2D3V electrons.
    Repeated passes without a step draw the same numbers, so the counts reported are
    those of the first pass.  Algorithmic bytes: every particle's id (4 B), and for
    each candidate (a fraction P = 1 - exp(-nu' dt) of the particles) its id again
    and its velocity read and written (4 + 24 B).  Beside it, the oracle's pass on
    a sample of the same particles."""
    import oracle

    w = workloads.maxwellian_box(2, (args.n, args.n), ppc=args.ppc, nv=3, dt=0.1, seed=6)
    g = pk.from_workload(w, stream=stream.cuda_stream).set_collisions(**MCC_BENCH)
    g.load(w.x, w.v)
    g.collide()
    counts = g.get_diag()["mcc_counts"]
    for _ in range(3):
        g.collide()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        g.collide()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    g.close()
    P = 1.0 - np.exp(-MCC_BENCH["density"] * (MCC_BENCH["sigma_el"] + MCC_BENCH["sigma_exc"])
                     * MCC_BENCH["vmax"] * w.dt)
    out = {"ms_per_pass": ms, "particles": w.np_, "particle_steps_per_s": w.np_ / (ms * 1e-3),
           "collisions_first_pass": {"elastic": counts[0], "excitation": counts[1],
                                     "above_bound": counts[2]},
           "candidate_fraction": P,
           "roofline": _roofline(w.np_ * 4 + P * w.np_ * 28, ms, "k_mcc", peak, peak_kind),
           "workload": f"maxwellian 2D3V {args.n}x{args.n}, {args.ppc} ppc, "
                       + ", ".join(f"{k}={v}" for k, v in MCC_BENCH.items())}
    if not args.no_row_oracles:
        v = np.array(w.v, dtype=np.float64)
        ids = np.arange(w.np_, dtype=np.uint32)
        (_, secs) = _timed(lambda: [oracle.mcc(v, ids, k, MCC_BENCH, w.m, w.dt)
                                    for k in range(1, 5)])
        out["oracle"] = {"kind": "oracle", "cores": 1, "particle_steps_per_s": w.np_ * 4 / secs,
                         "sample": f"all {w.np_} particles, 4 passes ({secs:.1f} s)"}
    return out


def bench_spectral(args, w, fft_ms, peak, peak_kind):
    """Roofline of the spectral field solve (timed on the GPU beside the CG) and the
    oracle's field solve of the same grid (FP64 Jacobi-PCG to 1e-12, whose discrete
    potential the spectral solve reproduces) on the charge of a sample of the
    workload's particles."""
    import oracle

    out = {"ms_per_solve": fft_ms, "nodes": w.cells,
           "roofline": _roofline(w.cells * _spectral_bytes_per_node(w.ndim), fft_ms,
                                 "spectral solve (k_fft_axis per axis x 2 solves, k_residual64, "
                                 "k_efield)", peak, peak_kind,
                                 residency="the grid (a few MB) stays in L2")}
    if not args.no_row_oracles:
        sample = min(w.np_, 1 << 20)
        rho = oracle.deposit(w.ndim, w.n, w.dx, w.x[:sample], w.q * w.weight * w.np_ / sample)
        rho -= rho.mean()
        (_, it, _), secs = _timed(lambda: oracle.poisson(w.ndim, w.n, w.dx, rho, 1e-12))
        out["oracle"] = {"kind": "oracle", "cores": 1, "ms_per_solve": secs * 1e3,
                         "iterations": int(it),
                         "sample": f"one solve of the full grid, right-hand side from {sample} "
                                   "particles"}
    return out


def bench_hc(args, w, pk, torch, stream, peak, peak_kind, steps=100, c=4.0):
    """The particle pass with the Higuera-Cary pusher (c = 4 v_te) on the headline
    workload: stage-timed push_deposit (same algorithmic bytes as the Boris pass),
    and the oracle's Higuera-Cary gather + push + move + deposit on a sample."""
    import oracle

    g = pk.from_workload(w, stream=stream.cuda_stream, pusher=pk.AP_PIC_PUSHER_HIGUERA_CARY,
                         c_light=c)
    g.load(w.x, w.v)
    for _ in range(5):
        g.push_deposit()
    torch.cuda.synchronize()
    g.set_timing(True)
    for k in range(1, steps + 1):
        g.push_deposit()
        if w.sort_every and k % w.sort_every == 0:
            g.sort()
    st = g.get_timing()
    g.set_timing(False)
    g.close()
    ms = st["push_deposit"][0] / max(st["push_deposit"][1], 1)
    alg = w.np_ * _bytes_per_particle(w.ndim, w.nv) + w.cells * _grid_bytes_per_node(w.ndim)
    out = {"pass_ms": ms, "particle_steps_per_s": w.np_ / (ms * 1e-3), "c": c,
           "roofline": _roofline(alg, ms, "k_particle_pass, Higuera-Cary mode", peak, peak_kind)}
    if not args.no_row_oracles:
        sample = min(w.np_, 1 << 20)
        sim = oracle.Simulation(w.ndim, w.n, w.dx, w.dt, q=w.q, m=w.m, weight=w.weight, B0=w.B0,
                                E0=w.E0, rtol=1e-6, pusher="hc", c=c)
        sim.load(w.x[:sample], w.v[:sample])

        def run():
            for _ in range(8):
                sim.push()
                sim.move()
                oracle.deposit(w.ndim, w.n, w.dx, sim.x, w.q * w.weight)
        _, secs = _timed(run)
        out["oracle"] = {"kind": "oracle", "cores": 1, "particle_steps_per_s": sample * 8 / secs,
                         "sample": f"{sample} of {w.np_} particles on the full grid, 8 steps of "
                                   f"gather+push+move+deposit ({secs:.1f} s)"}
    return out


def run_e2e(args, w, pk, torch, stream, extra, steps):
    """Load from pinned host memory, run the full cycle (with field solves) for
    e2e_steps steps reading the diagnostics back every step, then read rho."""
    import ctypes

    xs = torch.from_numpy(np.ascontiguousarray(w.x)).pin_memory()
    vs = torch.from_numpy(np.ascontiguousarray(w.v)).pin_memory()
    g = pk.from_workload(w, stream=stream.cuda_stream, cg_rtol=args.cg_rtol, **extra)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.load_ptr(w.np_, xs.data_ptr(), vs.data_ptr())
    for _ in range(steps):
        g.step(1)
        g.get_diag()
    rho = g.get_rho()
    t1 = time.perf_counter()
    g.close()
    h2d = w.x.nbytes + w.v.nbytes
    d2h = ctypes.sizeof(pk.ap_pic_diag) + 4  # diagnostics (+ error word) each step
    return {"value": w.np_ * steps / (t1 - t0), "unit": UNIT,
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h + rho.nbytes / steps,
            "steps": steps, "seconds": t1 - t0,
            "what": "load from pinned host + full cycle (push, deposit, sort, field solve, E) per step "
                    "+ diagnostics read each step + final rho read"}


def _per_instance_rate(pk, torch, stream, ws, steps, **over):
    """Particle-steps/s of push_deposit run instance by instance (one handle each)
    over `ws`: total particle-steps / total CUDA-event time."""
    ps, secs = 0, 0.0
    for w in ws:
        g = pk.from_workload(w, stream=stream.cuda_stream, **over)
        g.load(w.x, w.v)
        for _ in range(3):
            g.push_deposit()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.push_deposit()
        e1.record(stream)
        torch.cuda.synchronize()
        secs += e0.elapsed_time(e1) * 1e-3
        ps += w.np_ * steps
        g.close()
    return ps / secs


def bench_batch(args):
    """The batched serving workload on its own line (see run_batch)."""
    import torch

    import paper_2608_15249_b300 as pk

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    line = run_batch(args, pk, torch, torch.cuda.current_stream())
    print(json.dumps(line), flush=True)


def run_batch(args, pk, torch, stream, embedded=False):
    """The batched serving workload: `--instances` independent periodic 1D/2D
    instances (n per axis log-uniform in [32, 1024], 1k-200k electrons log-uniform,
    Maxwellian with a 1 % random mode, dt = 0.1) advanced together.  The value is
    the batch's particle-steps/s of gather + push + move + deposit (the shared
    particle pass and the charge conversion of every instance, with the sort at the
    tuned cadence); the field solve, the full step, and the same metric run instance
    by instance (FP64 plain and FP32 forms) on an unbiased sample of the instances
    are reported beside it.  Embedded in the default line, the lockstep CG
    comparison is left out and the oracle runs on a bounded sample of instances."""
    ws = workloads.batch_instances(count=args.instances, seed=5)
    total = sum(w.np_ for w in ws)
    nodes = sum(w.cells for w in ws)
    bt = pk.batch_from_workloads(ws, stream=stream.cuda_stream,
                                 solver=_SOLVERS[args.batch_solver])
    t0 = time.perf_counter()
    bt.load([w.x for w in ws], [w.v for w in ws])
    torch.cuda.synchronize()
    load_s = time.perf_counter() - t0
    tuning = (bt.autotune(steps_per_trial=3) if not args.no_autotune
              else bt.get_tuning().as_dict())
    sort_every = tuning["sort_every"]

    def hot_step(k):
        bt.push_deposit()
        if sort_every and k % sort_every == 0:
            bt.sort()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for k in range(1, args.warmup + 1):
            hot_step(k)
        torch.cuda.synchronize()
        launches0 = pk.kernel_launches()
        ev0.record(stream)
        for k in range(args.warmup + 1, args.warmup + args.steps + 1):
            hot_step(k)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = pk.kernel_launches() - launches0
    value = total * args.steps / (ms * 1e-3)
    # push_deposit alone (no sort) for the roofline
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        bt.push_deposit()
    e1.record(stream)
    torch.cuda.synchronize()
    pd_ms = e0.elapsed_time(e1) / 10
    # per node: E read (4 B per axis), the int64 accumulator cleared and read back by
    # the conversion (16 B), the FP32 right-hand side written (4 B)
    alg_bytes = sum(w.np_ * _bytes_per_particle(w.ndim, 2)
                    + w.cells * (4 * w.ndim + 8 + 8 + 4) for w in ws)
    peak, peak_kind = _peaks()
    achieved = alg_bytes / (pd_ms * 1e-3) / 1e9
    # the field solve of every instance, and the full step
    e0.record(stream)
    for _ in range(args.solve_reps):
        bt.solve_field()
    e1.record(stream)
    torch.cuda.synchronize()
    solve_ms = {args.batch_solver: e0.elapsed_time(e1) / args.solve_reps}
    e0.record(stream)
    bt.step(args.full_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    full_ms = e0.elapsed_time(e1) / args.full_steps
    iters = [bt.get_diag(i)["cg_iters"] for i in range(len(ws))]
    bt.close()
    if args.batch_solver != "cg" and args.cg_solve_reps > 0 and not embedded:
        # the lockstep Jacobi-PCG of the same batch, for comparison
        bc = pk.batch_from_workloads(ws, stream=stream.cuda_stream)
        bc.load([w.x for w in ws], [w.v for w in ws])
        for _ in range(3):
            bc.push_deposit()
        e0.record(stream)
        for _ in range(args.cg_solve_reps):
            bc.solve_field()
        e1.record(stream)
        torch.cuda.synchronize()
        solve_ms["cg"] = e0.elapsed_time(e1) / args.cg_solve_reps
        iters = [bc.get_diag(i)["cg_iters"] for i in range(len(ws))]
        bc.close()
    # the same metric instance by instance, on every k-th instance
    sample = ws[:: args.plain_stride]
    f64_rate = _per_instance_rate(pk, torch, stream, sample, args.plain_steps,
                                  precision=pk.AP_PIC_FP64_PLAIN)
    f32_rate = _per_instance_rate(pk, torch, stream, sample, args.plain_steps)
    line = {
        "metric": METRIC + ", batched", "value": value,
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch of {len(ws)} periodic 1D/2D instances, "
                               f"{total} electrons, {nodes} nodes, sort every {sort_every}",
                   "instances": len(ws), "particles": total, "nodes": nodes,
                   "tuning": tuning, "solver": args.batch_solver, "load_seconds": load_s,
                   "l2": "particle state larger than L2 (no flush)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "batch push_deposit (k_particle_pass per dimension class "
                               "+ memset + k_b_convert)",
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": pd_ms,
                     "peak_kind": peak_kind,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS},
        "field_solve_ms": solve_ms,
        "full_step_ms": full_ms,
        "full_step_particle_steps_per_s": total / (full_ms * 1e-3),
        "cg_iters_last_solve": {"max": max(iters), "median": statistics.median(iters),
                                "what": "the CG refinement's correction solve"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "per_instance": {
            "sample": f"every {args.plain_stride}th instance ({len(sample)}), "
                      f"{args.plain_steps} push_deposit calls each",
            "fp64_plain": f64_rate, "fp32": f32_rate, "unit": UNIT,
            "batched_over_fp64_plain": value / f64_rate},
    }
    if not args.no_cpu_baseline:
        # the oracle on every k-th instance (the same sample), all host cores
        import oracle

        cores = host_cores()
        oracle.set_threads(cores)
        ps, secs = 0, 0.0
        for w in ws[:: args.plain_stride * 4]:
            x, v = w.x.copy(), w.v.copy()
            secs += _oracle_particle_steps(oracle, w.ndim, w.n, w.dx, w.dt, x, v,
                                           np.zeros(w.ndim * w.cells), w.q, w.m, w.weight,
                                           w.E0, w.B0, 2)
            ps += 2 * w.np_
        oracle.set_threads(1)
        line["cpu_baseline"] = {
            "value": ps / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"every {args.plain_stride * 4}th instance, 2 steps of "
                      f"gather+push+move+deposit each ({secs:.1f} s on {cores} threads)"}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="two_stream_2d")
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--ppc", type=int, default=64)
    ap.add_argument("--cg-rtol", type=float, default=0.0, help="0: the form's default")
    ap.add_argument("--precision", choices=["f32", "f64"], default="f32",
                    help="f32: cell + FP32 offset form (the product); f64: FP64 plain form")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--e2e-solver", choices=["cg", "fft"], default="fft")
    ap.add_argument("--pusher", choices=["boris", "hc"], default="boris",
                    help="hc: Higuera-Cary (velocities read as momenta per mass)")
    ap.add_argument("--c-light", type=float, default=0.0, help="with --pusher hc; 0: infinite")
    ap.add_argument("--e2e-steps-cg", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-collisions", action="store_true")
    ap.add_argument("--no-em", action="store_true")
    ap.add_argument("--no-rows", action="store_true",
                    help="skip the spectral-solve and Higuera-Cary rows")
    ap.add_argument("--no-row-oracles", action="store_true",
                    help="skip the oracle timings beside the spectral, HC, MCC and EM rows")
    ap.add_argument("--prec-steps", type=int, default=10, help="--workload precision_study")
    ap.add_argument("--drift-steps", type=int, default=1000, help="--workload precision_study")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1 << 22)
    ap.add_argument("--cpu-steps", type=int, default=24)
    ap.add_argument("--ref-sample", type=int, default=1 << 16)
    ap.add_argument("--instances", type=int, default=1024, help="--workload batch")
    ap.add_argument("--plain-stride", type=int, default=8, help="--workload batch")
    ap.add_argument("--plain-steps", type=int, default=10, help="--workload batch")
    ap.add_argument("--solve-reps", type=int, default=3, help="--workload batch")
    ap.add_argument("--full-steps", type=int, default=3, help="--workload batch")
    ap.add_argument("--no-autotune", action="store_true", help="--workload batch")
    ap.add_argument("--batch-solver", choices=["cg", "fft"], default="fft",
                    help="--workload batch")
    ap.add_argument("--cg-solve-reps", type=int, default=1, help="--workload batch")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave the 3D and batch configurations out of the default line")
    ap.add_argument("--n3d", type=int, default=128, help="3D configuration: nodes per axis")
    ap.add_argument("--ppc3d", type=int, default=64, help="3D configuration: electrons per cell")
    ap.add_argument("--cpu-sample-3d", type=int, default=1 << 21)
    ap.add_argument("--cpu-steps-3d", type=int, default=4)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        bench_reference(args)
    elif args.workload == "precision_study":
        bench_precision(args)
    elif args.workload == "batch":
        bench_batch(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
