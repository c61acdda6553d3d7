"""Benchmark of the PIC time step: particle-steps/s and HBM roofline fraction.

Workload (default): the frame-dragging tube of a P = 0.5 s, B = 1e12 G pulsar
(R_* = 10 km, R = R_* sqrt(R_* Omega / c), length 2 R_*, Nz = 65536, GR
rho_GJ at i = 0.5 rad) prefilled with 1e8 FP32 macro-electrons (seeded
synthetic state, stratified uniform heights in ID order, gamma from a
frame-dragging ramp with 1 % jitter), fields re-solved from Eq. 4 with that
charge. One step = injection, gather, push, deposit, removal and the field
leap-frog on the whole tube.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+deposit), % HBM roofline; batched/adjoint vs plain"
UNIT = "particle-steps/s"
BYTES_PER_PARTICLE = 16          # FP32 xi and u, read once and written once per step
CSRC = os.path.join(ROOT, "paper_1011_6330_gb300", "csrc")
KERNEL_SRC = {"gr1e8": ["push.cu", "device_common.cuh", "sclf_internal.h"],
              "large": ["push_fix32.cu", "device_common.cuh", "sclf_internal.h"]}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "push_kernel_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["gr1e8", "large", "batch"], default="gr1e8",
                    help="gr1e8: P = 0.5 s frame-dragging tube, Nz = 65536, FP32 particles "
                         "(default); large: P = 0.1 s, B = 3e12 G, Nz = 2^20, 2^30 "
                         "fixed-point particles")
    ap.add_argument("--particles", type=float, default=None)
    ap.add_argument("--order", choices=["descending", "shuffled"], default="descending")
    ap.add_argument("--accumulate", choices=["fixed64", "fp64"], default="fixed64")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(work, seconds, device="cpu"):
    """Whole-job throughput of independent per-rank runs: the work of all
    ranks over the slowest rank's time (returns work_total, seconds_max).
    Single process: the inputs unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(work), float(seconds)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(w.item()), float(t.item())


def rank_seed(rank, base=0):
    """Seed of a rank's independent tube (distinct per rank)."""
    return base + 1000003 * rank


def kernel_sha(workload):
    """Hash of the workload's particle-kernel sources (ties a traffic capture
    to them)."""
    h = hashlib.sha256()
    for p in KERNEL_SRC[workload]:
        with open(os.path.join(CSRC, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_tube(B, workloads, workload, n, acc, order, seed):
    """Create the workload's tube and fill it with its seeded synthetic state.
    Returns (tube, params, derived, sample_z, sample_u, stride): every
    stride-th particle of the state, for the CPU baseline."""
    from paper_1011_6330_gb300 import synth
    if workload == "large":
        kw = workloads.large_tube(n_particles=n)
    else:
        kw = workloads.gr_tube(n_particles=n, accumulate=acc)
    t = B.Tube(B.default_params(**kw))
    d = t.derived
    # frame-dragging ramp for the initial momenta: gamma_far = Lambda0^2 kappa cos i
    eta_scale = d["R_over_Rstar"]
    gfar = d["Lambda0"] ** 2 * d["kappa"] * math.cos(kw["incl_rad"])
    eta = lambda zz: 1.0 + zz * eta_scale
    stride = 100 if n <= 2 * 10 ** 8 else 1024
    if order == "descending" and n > 2 * 10 ** 8:
        zs, us = [], []
        for z, u in synth.prefilled_beam_chunks(n, d["L"] - d["dz"], gfar, seed=seed,
                                                chunk=1 << 26, eta_of_z=eta):
            t.add_particles(z, u)
            zs.append(z[::stride])
            us.append(u[::stride])
        return t, kw, d, np.concatenate(zs), np.concatenate(us), stride
    z, u = synth.prefilled_beam(n, d["L"] - d["dz"], gfar, seed=seed, order=order,
                                eta_of_z=eta)
    t.add_particles(z, u)
    return t, kw, d, z[::stride], u[::stride], stride


def cpu_baseline(zs, us, n_total, kw, d, seconds, stride):
    """The oracle as it stands on a bounded sample: every stride-th particle
    of the same prefilled state (macro charge times stride), the workload's
    particle precision with the fixed-point current, the full Nz grid;
    stepped for ~seconds."""
    import oracle as orc
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
    nz = kw["Nz"]
    zn = np.arange(nz + 1) * (d["L"] / nz)
    rho = orc.rho_gj_profile(orc.RHO_GR, zn, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"])
    prec = "fix32" if kw["precision"] == 2 else "f32"
    o = orc.Tube(nz, d["L"], d["dt"], rho, d["s"] * stride, precision=prec, accumulate="fixed")
    o.add_particles(zs, us)
    o.solve_fields()
    o.step()                                   # warm-up
    t0 = time.perf_counter()
    steps, psteps = 0, 0
    while time.perf_counter() - t0 < seconds:
        n = o.xi.size + o.injection_count()
        o.step()
        steps += 1
        psteps += n
    el = time.perf_counter() - t0
    return {"value": psteps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d of the %d particles (every %dth, macro charge x%d), Nz=%d, "
                      "%s particles + fixed-point current, %d steps in %.1f s"
                      % (zs.size, n_total, stride, stride, nz, prec, steps, el)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1011_6330_gb300 import synth
    import oracle as orc
    n = int(args.particles or 1e8)
    stride = 100
    cu = orc.code_units(1e12, 0.5, 1e6, 0.5, 1.4 * 1.98847e33)
    L = 2.0 / cu["theta_p"]
    nz = 65536
    dz = L / nz
    zn = np.arange(nz + 1) * dz
    rho = orc.rho_gj_profile(orc.RHO_GR, zn, cu["Lambda0"], 0.5, cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"])
    dt = orc.default_dt(dz, cu["Lambda0"])
    s = orc.macro_charge_for(rho[0], L, n)
    gfar = cu["Lambda0"] ** 2 * cu["kappa"] * math.cos(0.5)
    z, u = synth.prefilled_beam(n // stride, L - dz, gfar, seed=0, order=args.order,
                                eta_of_z=lambda zz: 1.0 + zz * cu["R_over_Rstar"])
    o = orc.Tube(nz, L, dt, rho, s * stride, precision="f32", accumulate="fixed")
    o.add_particles(z, u)
    o.solve_fields()
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    ps = 0
    for _ in range(args.steps):
        ps += o.xi.size + o.injection_count()
        o.step()
    el = time.perf_counter() - t0
    v = ps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "gr_tube_P0.5s_B1e12G_Nz65536_1e8_particles_fp32",
                   "sample": "every %dth particle (%d), macro charge x%d" % (stride, z.size, stride),
                   "l2": "inputs larger than L2 on the GPU arm"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d particles of the 1e8-particle state, Nz=%d, %d steps"
                                   % (z.size, nz, args.steps)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_batch(args):
    """The death-line batch: 256 seeded pulsar tubes (flat and frame-dragging,
    Nz 1024..16384, 1e5..2e6 FP32 particles each) stepped by batched launches;
    reported next to the plain form (the same tubes stepped one at a time)."""
    import torch
    from paper_1011_6330_gb300 import binding as B
    from paper_1011_6330_gb300 import synth, workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    kws = workloads.death_line_batch(seed=rank_seed(rank))
    params = [B.default_params(**kw) for kw in kws]
    batch = B.Batch(params)
    plain = [B.Tube(p) for p in params]
    states = []
    for i, kw in enumerate(kws):
        d = batch.tubes[i].derived
        gr = kw["rho_gj_mode"] == B.SCLF_RHO_GR
        gfar = (d["Lambda0"] ** 2 * d["kappa"] * math.cos(kw["incl_rad"]) if gr
                else math.sqrt(2.0) * d["Lambda0"])
        eta = (lambda zz, r=d["R_over_Rstar"]: 1.0 + zz * r) if gr else None
        z, u = synth.prefilled_beam(kw["target_particles"], d["L"] - d["dz"], gfar,
                                    seed=rank_seed(rank) + i, eta_of_z=eta)
        for t in (batch.tubes[i], plain[i]):
            t.add_particles(z, u)
            t.solve_fields()
        if i == 1:
            states.append((z, u))
    batch.run(args.warmup)
    torch.cuda.synchronize()
    n0 = sum(t.status()["n_particles"] for t in batch.tubes)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    batch.set_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    batch.run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    tm = batch.timing()
    batch.set_timing(False)
    el_s = e0.elapsed_time(e1) * 1e-3
    n1 = sum(t.status()["n_particles"] for t in batch.tubes)
    work, el_s = combine_ranks(0.5 * (n0 + n1) * args.steps, el_s, device="cuda")
    push_avg_ms = tm["push_ms"] / max(tm["n_steps"], 1)
    slots = tm["particle_slots"] / max(tm["n_steps"], 1)
    achieved = BYTES_PER_PARTICLE * slots / (push_avg_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    # the plain form: the same tubes, one tube at a time
    k_plain = min(args.steps, 128)
    for t in plain:
        t.run(args.warmup)
    torch.cuda.synchronize()
    p0 = time.perf_counter()
    for t in plain:
        t.run(k_plain)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - p0
    plain_value = 0.5 * (n0 + n1) * k_plain / plain_s
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle as orc
        kw = kws[1]
        z, u = states[0]
        d = plain[1].derived
        o = orc.Tube(kw["Nz"], d["L"], d["dt"], np.full(kw["Nz"] + 1, d["rho0"]), d["s"],
                     precision="f32", accumulate="fixed")
        o.add_particles(z, u)
        o.solve_fields()
        o.step()
        t0 = time.perf_counter()
        steps = psteps = 0
        while time.perf_counter() - t0 < args.cpu_seconds:
            psteps += o.xi.size + o.injection_count()
            o.step()
            steps += 1
        el = time.perf_counter() - t0
        cpu = {"value": psteps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "tube 1 of the batch (flat rho_GJ, Nz=%d, %d particles), %d steps in %.1f s"
                         % (kw["Nz"], z.size, steps, el)}
    line = {
        "metric": METRIC, "value": work / el_s, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "death_line_batch_256_tubes", "tubes": len(kws),
                   "particles_total": int(n1), "cells_total": int(sum(kw["Nz"] for kw in kws)),
                   "l2": "inputs larger than L2 (%.0f MB of particle state)" % (8e-6 * n1),
                   "parallelism": "independent batch per GPU" if ws > 1 else "one batch"},
        "plain_form": {"value": plain_value, "unit": UNIT, "steps": k_plain,
                       "how": "the same 256 tubes, each stepped alone (tube_run, graphs)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "batch_push_kernel",
                     "peak_source": peak_kind, "push_ms_avg": push_avg_ms,
                     "field_ms_avg": tm["field_ms"] / max(tm["n_steps"], 1),
                     "compact_ms_total": tm["compact_ms"],
                     "bytes_per_launch": BYTES_PER_PARTICLE * slots},
        "cpu_baseline": cpu, "e2e": None,
        "gpu_launches": int(2 * tm["n_steps"] + tm["n_compactions"] * len(kws)),
        "clocks": clk,
        "status": {"check": int(max(t.check() for t in batch.tubes))},
    }
    if rank == 0:
        print(json.dumps(line))
    batch.close()
    for t in plain:
        t.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1011_6330_gb300 import binding as B
    from paper_1011_6330_gb300 import workloads
    B.load()
    acc = B.SCLF_ACC_FIXED64 if args.accumulate == "fixed64" else B.SCLF_ACC_FP64
    large = args.workload == "large"
    n = int(args.particles or (2 ** 30 if large else 1e8))
    t, kw, d, zs, us, stride = build_tube(B, workloads, args.workload, n, acc, args.order,
                                          seed=rank_seed(rank))
    t.solve_fields()
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up
    t.run(args.warmup)
    torch.cuda.synchronize()
    st0 = t.status()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier()
    torch.cuda.synchronize()
    t.set_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t.run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    el_ms = e0.elapsed_time(e1)
    tm = t.timing()
    t.set_timing(False)
    st1 = t.status()
    psteps_local = 0.5 * (st0["n_particles"] + st1["n_particles"]) * args.steps
    psteps, el_s = combine_ranks(psteps_local, el_ms * 1e-3, device="cuda")
    el_ms = el_s * 1e3
    value = psteps / el_s

    # roofline of the dominant kernel (the particle kernel)
    push_avg_ms = tm["push_ms"] / max(tm["n_steps"], 1)
    slots_per_launch = tm["particle_slots"] / max(tm["n_steps"], 1)
    achieved = BYTES_PER_PARTICLE * slots_per_launch / (push_avg_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        ent = tr.get(args.workload, {})
        if ent.get("kernel_sha") == kernel_sha(args.workload) \
                and ent.get("accumulate", "fixed64") == args.accumulate \
                and ent.get("order", "descending") == args.order and ent.get("particles") == n:
            traffic = ent["bytes_per_launch"]
    gpu_launches = 2 * tm["n_steps"] + tm["n_compactions"]
    check = t.check()

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e and not large:
        xi_h, u_h, _ = t.save_particles()
        pin_x = torch.empty(xi_h.size, dtype=torch.float32, pin_memory=True)
        pin_u = torch.empty(u_h.size, dtype=torch.float32, pin_memory=True)
        pin_x.numpy()[:] = xi_h
        pin_u.numpy()[:] = u_h
        del xi_h, u_h
        out_x = torch.empty_like(pin_x, pin_memory=True)
        out_u = torch.empty_like(pin_u, pin_memory=True)
        import ctypes as C
        lib = B.load()
        nout = C.c_int64()
        ksteps = args.steps
        barrier()
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        lib.tube_load_particles(t.h, pin_x.numel(), C.c_void_p(pin_x.data_ptr()),
                                C.c_void_p(pin_u.data_ptr()), None)
        n_e2e = 0
        for _ in range(ksteps):
            st = t.status()                              # per-step D2H of the counters
            n_e2e += st["n_particles"] + st["pending_injection"]
            t.step()
        cap = out_x.numel()
        rc = lib.tube_save_particles(t.h, cap, C.byref(nout), C.c_void_p(out_x.data_ptr()),
                                     C.c_void_p(out_u.data_ptr()), None)
        torch.cuda.synchronize()
        el_e2e = time.perf_counter() - h0
        n_all, el_e2e = combine_ranks(n_e2e, el_e2e, device="cuda")
        state_bytes = 8 * pin_x.numel()
        e2e = {"value": n_all / el_e2e, "unit": UNIT,
               "h2d_bytes_per_step": state_bytes / ksteps,
               "d2h_bytes_per_step": (8 * min(cap, nout.value) + ksteps * 88) / ksteps,
               "path": "tube_load_particles(pinned) + K x (tube_status, tube_step) + "
                       "tube_save_particles(pinned)", "rc": int(rc)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(zs, us, n, kw, d, args.cpu_seconds, stride)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "fix32+f32" if large else "f32",
        "data": "synthetic",
        "config": {"workload": ("large_tube_P0.1s_B3e12G_Nz%d_%d_particles_fix32" % (kw["Nz"], n))
                   if large else "gr_tube_P0.5s_B1e12G_Nz65536_%g_particles_fp32" % n,
                   "rho_gj": "frame-dragging (Eq. 6-7), i = 0.5 rad",
                   "particles_per_gpu": n, "Nz": kw["Nz"], "Lambda0": d["Lambda0"],
                   "dt_R_over_c": d["dt"], "order": args.order,
                   "current_accumulator": args.accumulate,
                   "l2": "inputs larger than L2 (particle state %.0f MB per GPU)" % (8 * n / 1e6),
                   "parallelism": "independent tube per GPU" if ws > 1 else "single tube"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "push_fix32_kernel" if large else
                     ("push_kernel<float, fixed64>" if acc == B.SCLF_ACC_FIXED64
                      else "push_kernel<float, fp64>"),
                     "peak_source": peak_kind, "push_ms_avg": push_avg_ms,
                     "field_ms_avg": tm["field_ms"] / max(tm["n_steps"], 1),
                     "compact_ms_total": tm["compact_ms"],
                     "compaction_checks": tm["n_compactions"],
                     "bytes_per_launch": BYTES_PER_PARTICLE * slots_per_launch},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(gpu_launches),
        "clocks": clk,
        "status": {"check": int(check), "n_particles": st1["n_particles"],
                   "injected_per_step": (st1["total_injected"] - st0["total_injected"]) / args.steps,
                   "flags": st1["flags"]},
    }
    if rank == 0:
        print(json.dumps(line))
    t.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
