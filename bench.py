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
              "gr1e8_fix32": ["push_fix32.cu", "device_common.cuh", "sclf_internal.h"],
              "large": ["push_fix32.cu", "device_common.cuh", "sclf_internal.h"],
              "batch": ["push.cu", "device_common.cuh", "sclf_internal.h"],
              "batch_fix32": ["push_fix32.cu", "device_common.cuh", "sclf_internal.h"]}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "push_kernel_traffic.json")
# Per-kernel event timing inside the timed region samples every TIME_EVERY-th
# unit of work (a step launched on its own or a 64-step graph replay): each
# event-record node adds about 2 us to the run's pace, which the unsampled
# value would carry on every step.
TIME_EVERY = 4
TIMING_SAMPLE = ("CUDA events around the kernels of every %dth unit of work in the timed "
                 "region (one step or one 64-step graph replay)" % TIME_EVERY)


# tube_params.launch_overlap of every tube the run builds (0: the library's
# default, programmatic dependent launch of a step's kernels; -1: plain
# stream order)
LAUNCH_OVERLAP = [0]


def tube_params(B, **kw):
    kw.setdefault("launch_overlap", LAUNCH_OVERLAP[0])
    return B.default_params(**kw)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["gr1e8", "large", "batch", "adjoint", "dtube"],
                    default="gr1e8",
                    help="gr1e8: P = 0.5 s frame-dragging tube, Nz = 65536, FP32 particles "
                         "(default); large: P = 0.1 s, B = 3e12 G, Nz = 2^20, 2^30 "
                         "fixed-point particles; batch: 256 pulsar tubes; adjoint: "
                         "gradients of a 2000-step run of a P = 0.3 s tube, Nz = 16384, "
                         "1e6 FP32 particles; dtube: the gr1e8 tube cut into --domains "
                         "z-domains on one GPU")
    ap.add_argument("--particles", type=float, default=None)
    ap.add_argument("--domains", type=int, default=4,
                    help="dtube workload: equal z-ranges the gr1e8 tube is cut into")
    ap.add_argument("--nz", type=int, default=None,
                    help="gr1e8/large: grid cells (default 65536 / 2^20), e.g. for a smaller "
                         "profiling case with the same particles per cell")
    ap.add_argument("--order", choices=["descending", "shuffled"], default="descending")
    ap.add_argument("--accumulate", choices=["fixed64", "fp64"], default="fixed64")
    ap.add_argument("--precision", choices=["f32", "fix32"], default="fix32",
                    help="gr1e8: particle positions as 32-bit fixed point (SCLF_FIX32, "
                         "default) or as float32; momenta float32 either way")
    ap.add_argument("--batch-precision", choices=["fix32", "f32"], default="fix32",
                    help="batch workload: positions of the death-line tubes")
    ap.add_argument("--no-extras", action="store_true",
                    help="gr1e8: only the headline measurement (no precision comparison, "
                         "no other-precision or FP64-accumulator figures, no batched or "
                         "adjoint forms)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--sort-interval", type=int, default=0,
                    help="gr1e8/large: re-sort the slots by cell (tube_sort) once before the "
                         "run and every this many steps (0: never)")
    ap.add_argument("--push-stages", type=int, default=0,
                    help="gr1e8/large: shared-memory stages of the particle kernel's bulk-copy "
                         "ring (1: loads straight into registers; 0: the library's default)")
    ap.add_argument("--launch-overlap", choices=["on", "off"], default="on",
                    help="step kernels by programmatic dependent launch (on, the library's "
                         "default) or in plain stream order (off)")
    ap.add_argument("--no-kernel-timing", action="store_true",
                    help="adjoint workload: no event-record nodes (for ncu runs, where "
                         "each event node is very slow); no per-kernel times or roofline")
    args = ap.parse_args()
    LAUNCH_OVERLAP[0] = 1 if args.launch_overlap == "on" else -1
    return args


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


def gr_workload_name(n, nz=65536, precision="fix32"):
    """Name of the frame-dragging tube workload (both arms print the same)."""
    return "gr_tube_P0.5s_B1e12G_Nz%d_%g_particles_%s" % (
        nz, n, "fix32" if precision == "fix32" else "fp32")


def host_info():
    """CPU model and logical core count of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def barrier(ws):
    """Barrier over the ranks of a multi-GPU run (no-op on one GPU)."""
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


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


def build_tube(B, workloads, workload, n, acc, order, seed, sort_interval=0, nz=None,
               push_stages=0, precision="f32"):
    """Create the workload's tube and fill it with its seeded synthetic state.
    Returns (tube, params, derived, sample_z, sample_u, stride): every
    stride-th particle of the state, for the CPU baseline."""
    from paper_1011_6330_gb300 import synth
    if workload == "large":
        kw = workloads.large_tube(n_particles=n, **({"Nz": nz} if nz else {}))
    else:
        kw = workloads.gr_tube(n_particles=n, accumulate=acc,
                               precision=B.SCLF_FIX32 if precision == "fix32" else B.SCLF_FP32,
                               **({"Nz": nz} if nz else {}))
    kw["sort_interval"] = sort_interval
    kw["push_stages"] = push_stages
    t = B.Tube(tube_params(B, **kw))
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
    _STATE["last"] = (n, z, u)
    return t, kw, d, z[::stride], u[::stride], stride


_STATE = {}


def _sample(n, stride):
    """Every stride-th particle of the last n-particle state build_tube made."""
    m, z, u = _STATE.pop("last")
    assert m == n
    return z[::stride].copy(), u[::stride].copy()


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


def _allcore_worker(w, nw, names, shapes, z, u, nz, L, dt, rho0, s, prec, barrier):
    """One process of the all-core baseline: the oracle's gather, push and
    deposit on its share of the particles, every step, between barriers."""
    from multiprocessing import shared_memory
    import oracle as orc
    shm = [shared_memory.SharedMemory(name=n) for n in names]
    ez = np.ndarray(shapes[0], np.float64, buffer=shm[0].buf)
    acc_all = np.ndarray(shapes[1], np.int64, buffer=shm[1].buf)
    res = np.ndarray(shapes[2], np.int64, buffer=shm[2].buf)
    ctl = np.ndarray(shapes[3], np.int64, buffer=shm[3].buf)
    o = orc.Tube(nz, L, dt, np.full(nz + 1, rho0), s, precision=prec, accumulate="fixed")
    o.add_particles(z, u)
    xi, uu = o.xi, o.u
    fix = o.fix
    top = (nz << o.fb) if fix else nz
    while True:
        barrier.wait()                                   # fields and n_inj are ready
        if ctl[1]:
            break
        if w == 0 and ctl[0] > 0:                        # (a1) injection at the base
            xi = np.concatenate([xi, np.zeros(int(ctl[0]), xi.dtype)])
            uu = np.concatenate([uu, np.zeros(int(ctl[0]), uu.dtype)])
        if fix:
            ep = orc.gather_fix32(ez, xi, o.fb)
            xi1, u1, finite = orc.push_fix32(xi, uu, ep, dt, o.dz, o.fb)
            acc = orc.deposit_fix32(nz, xi[finite], xi1[finite], o.fb)
        else:
            ep = orc.gather(ez, xi, o.rt)
            xi1, u1 = orc.push(xi, uu, ep, dt, o.dz, o.rt)
            acc = orc.deposit_fractions(nz, xi, xi1, o.rt, "fixed")
            finite = np.isfinite(xi1) & np.isfinite(u1)
        alive = finite & (xi1 >= 0) & (xi1 < top)
        xi, uu = xi1[alive], u1[alive]
        acc_all[w] = acc
        w0 = orc.base_weight_fix32(xi, o.fb) if fix else orc.base_weight_fixed(xi, o.rt)
        res[w] = (xi.size, w0, 0)
        barrier.wait()                                   # this step's share is written
    for m in shm:
        m.close()


def cpu_baseline_allcore(zs, us, n_total, kw, d, seconds, stride, workers=None, nsteps=None):
    """The oracle's step on all host cores: the particle sample split over
    `workers` spawned processes (gather, push, deposit and removal of their
    share with the oracle's functions), the integer current sums added in a
    fixed order and the field leap-frog and injection count done by this
    process (the oracle's field_update and injection_count), in shared
    memory. Computes the same fields as the one-process oracle. Runs for
    ~seconds, or exactly nsteps timed steps when given."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import oracle as orc
    workers = workers or os.cpu_count() or 1
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
    nz, L, dt = kw["Nz"], d["L"], d["dt"]
    zn = np.arange(nz + 1) * (L / nz)
    rho = orc.rho_gj_profile(orc.RHO_GR, zn, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"])
    prec = "fix32" if kw["precision"] == 2 else "f32"
    s = d["s"] * stride
    o = orc.Tube(nz, L, dt, rho, s, precision=prec, accumulate="fixed")
    o.add_particles(zs, us)
    o.solve_fields()
    ez, er, b = o.ez, o.er, o.b
    w0 = o.w0
    shapes = [(nz,), (workers, nz), (workers, 3), (2,)]
    shm = [shared_memory.SharedMemory(create=True, size=int(np.prod(sh)) * 8) for sh in shapes]
    ez_s = np.ndarray(shapes[0], np.float64, buffer=shm[0].buf)
    acc_all = np.ndarray(shapes[1], np.int64, buffer=shm[1].buf)
    res = np.ndarray(shapes[2], np.int64, buffer=shm[2].buf)
    ctl = np.ndarray(shapes[3], np.int64, buffer=shm[3].buf)
    ctl[:] = 0
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers + 1)
    parts = np.array_split(np.arange(zs.size), workers)
    procs = [ctx.Process(target=_allcore_worker,
                         args=(w, workers, [m.name for m in shm], shapes, zs[parts[w]],
                               us[parts[w]], nz, L, dt, rho[0], s, prec, barrier))
             for w in range(workers)]
    for p in procs:
        p.start()
    try:
        def step():
            nonlocal ez, er, b, w0
            n_inj, _ = orc.injection_count(ez[0], w0, s, o.dz, rho[0])
            ctl[0] = n_inj
            ez_s[:] = ez
            barrier.wait()
            barrier.wait()
            acc = acc_all[0].copy()
            for w in range(1, workers):                  # fixed order (exact integers)
                acc += acc_all[w]
            w0 = int(res[:, 1].sum())
            live = int(res[:, 0].sum())
            j = orc.current_from(acc, s, dt, "fixed")
            ez, er, b = orc.field_update(ez, er, b, j, dt, o.dz)
            return live, n_inj
        n_prev, _ = step()                               # warm-up
        t0 = time.perf_counter()
        steps = psteps = 0
        while (time.perf_counter() - t0 < seconds) if nsteps is None else steps < nsteps:
            live, inj = step()
            psteps += n_prev + inj
            n_prev = live
            steps += 1
        el = time.perf_counter() - t0
        ctl[1] = 1
        barrier.wait()
    finally:
        for p in procs:
            p.join(timeout=30)
        for m in shm:
            m.close()
            m.unlink()
    return {"value": psteps / el, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": "%d of the %d particles (every %dth, macro charge x%d), Nz=%d, %s particles + "
                      "fixed-point current, %d steps in %.1f s; the oracle's particle step on "
                      "%d processes, integer current sums added in a fixed order, fields and "
                      "injection in the main process"
                      % (zs.size, n_total, stride, stride, nz, prec, steps, el, workers),
            "final_ez": ez}


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
    prec = "fix32" if args.precision == "fix32" else "f32"
    o = orc.Tube(nz, L, dt, rho, s * stride, precision=prec, accumulate="fixed")
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
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fix32+f32" if prec == "fix32" else "f32", "data": "synthetic",
        "config": {"workload": gr_workload_name(n, nz, args.precision),
                   "sample": "every %dth particle (%d), macro charge x%d" % (stride, z.size, stride),
                   "l2": "inputs larger than L2 on the GPU arm"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d particles of the 1e8-particle state, Nz=%d, %d steps"
                                   % (z.size, nz, args.steps), "host": host_info()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_batch(args, sub=False):
    """The death-line batch: 256 seeded pulsar tubes (flat and frame-dragging,
    Nz 1024..16384, 1e5..2e6 FP32 particles each) stepped by batched launches;
    reported next to the plain form (the same tubes stepped one at a time)."""
    import torch
    from paper_1011_6330_gb300 import binding as B
    from paper_1011_6330_gb300 import synth, workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1 and not sub:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    bprec = B.SCLF_FP32 if getattr(args, "batch_precision", "fix32") == "f32" else B.SCLF_FIX32
    fix = bprec == B.SCLF_FIX32
    kws = workloads.death_line_batch(seed=rank_seed(rank), precision=bprec)
    params = [tube_params(B, **kw) for kw in kws]
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
    # the project's autotuner picks the particle kernel's shape on this batch
    # (its tuning steps are ordinary steps of the run)
    chosen, tune_ms = batch.autotune(5)
    batch.run(args.warmup)
    torch.cuda.synchronize()
    n0 = sum(t.status()["n_particles"] for t in batch.tubes)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    batch.set_timing(TIME_EVERY)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    batch.run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    tm = batch.timing()
    batch.set_timing(False)
    el_s = e0.elapsed_time(e1) * 1e-3
    n1 = sum(t.status()["n_particles"] for t in batch.tubes)
    work, el_s = combine_ranks(0.5 * (n0 + n1) * args.steps, el_s, device="cuda")
    push_avg_ms = tm["push_ms"] / max(tm["n_steps"], 1)
    slots = tm["particle_slots"] / max(tm["steps_run"], 1)
    achieved = BYTES_PER_PARTICLE * slots / (push_avg_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as f:
            ent = json.load(f).get("batch_fix32" if fix else "batch", {})
        if ent.get("kernel_sha") == kernel_sha("batch_fix32" if fix else "batch") \
                and ent.get("tubes") == len(kws) \
                and ws == 1:
            traffic = ent["bytes_per_launch"]
    # end to end through the C ABI: every tube's particles from pinned host
    # memory, K batch steps each followed by the batch's counters read back
    # (batch_status), every tube's particles back into pinned host memory
    e2e = None
    if not args.no_e2e:
        import ctypes as C
        lib = B.load()
        saved = [t.save_particles()[:2] for t in batch.tubes]
        counts = [x.size for x, _ in saved]
        offs = np.concatenate([[0], np.cumsum(counts)])
        caps = [int(t.params.capacity) for t in batch.tubes]
        xdt = torch.int32 if fix else torch.float32      # raw positions: X (FIX32) or xi
        pin_x = torch.empty(int(offs[-1]), dtype=xdt, pin_memory=True)
        pin_u = torch.empty(int(offs[-1]), dtype=torch.float32, pin_memory=True)
        for i, (x, u) in enumerate(saved):
            pin_x.numpy()[offs[i]:offs[i + 1]] = x
            pin_u.numpy()[offs[i]:offs[i + 1]] = u
        del saved
        ocaps = np.concatenate([[0], np.cumsum(caps)])
        out_x = torch.empty(int(ocaps[-1]), dtype=xdt, pin_memory=True)
        out_u = torch.empty(int(ocaps[-1]), dtype=torch.float32, pin_memory=True)
        nout = C.c_int64()
        ksteps = args.steps
        barrier(ws)
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        for i, t in enumerate(batch.tubes):
            rc = lib.tube_load_particles(t.h, counts[i],
                                         C.c_void_p(pin_x.data_ptr() + 4 * int(offs[i])),
                                         C.c_void_p(pin_u.data_ptr() + 4 * int(offs[i])), None)
            if rc:
                raise RuntimeError("tube_load_particles: %d" % rc)
        n_e2e = 0
        for _ in range(ksteps):
            st = batch.status()                        # per-step D2H of every tube's counters
            n_e2e += sum(x["n_particles"] + x["pending_injection"] for x in st)
            batch.step()
        n_back = 0
        for i, t in enumerate(batch.tubes):
            rc = lib.tube_save_particles(t.h, caps[i], C.byref(nout),
                                         C.c_void_p(out_x.data_ptr() + 4 * int(ocaps[i])),
                                         C.c_void_p(out_u.data_ptr() + 4 * int(ocaps[i])), None)
            if rc:
                raise RuntimeError("tube_save_particles: %d" % rc)
            n_back += nout.value
        torch.cuda.synchronize()
        el_e2e = time.perf_counter() - h0
        n_all, el_e2e = combine_ranks(n_e2e, el_e2e, device="cuda")
        stats_bytes = C.sizeof(B.TubeStats) * len(kws)
        e2e = {"value": n_all / el_e2e, "unit": UNIT,
               "h2d_bytes_per_step": 8.0 * float(offs[-1]) / ksteps,
               "d2h_bytes_per_step": (8.0 * n_back + ksteps * stats_bytes) / ksteps,
               "path": "per tube tube_load_particles(pinned) + K x (batch_status, batch_step) + "
                       "per tube tube_save_particles(pinned)"}
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
                     precision="fix32" if fix else "f32", accumulate="fixed")
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
        "scaling": "weak", "vs_baseline": None, "dtype": "fix32+f32" if fix else "f32",
        "data": "synthetic",
        "config": {"workload": "death_line_batch_256_tubes" + ("_fix32" if fix else "_fp32"),
                   "tubes": len(kws),
                   "particles_total": int(n1), "cells_total": int(sum(kw["Nz"] for kw in kws)),
                   "l2": "inputs larger than L2 (%.0f MB of particle state)" % (8e-6 * n1),
                   "kernel_shape": ({"chosen": {"particles_per_thread": 8, "ctas_per_sm": 4,
                                                "runs_per_thread": "run cell and the next"},
                                     "autotune_push_ms": {"8x4 (FIX32)": float(tune_ms[0])}}
                                    if fix else
                                    {"chosen": {"particles_per_thread": B.Batch.VARIANTS[chosen][0],
                                                "ctas_per_sm": B.Batch.VARIANTS[chosen][1],
                                                "runs_per_thread": B.Batch.VARIANTS[chosen][2]},
                                     "autotune_push_ms": {"%dx%dx%d" % v: float(m) for v, m in
                                                          zip(B.Batch.VARIANTS, tune_ms)}}),
                   "parallelism": "independent batch per GPU" if ws > 1 else "one batch"},
        "plain_form": {"value": plain_value, "unit": UNIT, "steps": k_plain,
                       "how": "the same 256 tubes, each stepped alone (tube_run, graphs)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": ("batch_push_fix32_kernel" if fix else
                                "batch_push_const_kernel" if len(kws) <= 400
                                else "batch_push_kernel"),
                     "peak_source": peak_kind, "push_ms_avg": push_avg_ms,
                     "field_ms_avg": tm["field_ms"] / max(tm["n_steps"], 1),
                     "compact_ms_total": tm["compact_ms"],
                     "timed_steps": tm["n_steps"], "timing_sample": TIMING_SAMPLE,
                     "bytes_per_launch": BYTES_PER_PARTICLE * slots},
        "cpu_baseline": cpu, "e2e": e2e,
        # per step: descriptor refresh, particle and field kernels; one
        # compaction kernel per tube per check
        "gpu_launches": int(3 * tm["steps_run"] + tm["compactions_run"] * len(kws)),
        "clocks": clk,
        "status": {"check": int(max(t.check() for t in batch.tubes))},
    }
    if rank == 0 and not sub:
        print(json.dumps(line))
    batch.close()
    for t in plain:
        t.close()
    if sub:
        return line
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


ADJ_STEPS, ADJ_EVERY, ADJ_TIME_EVERY = 2000, 100, 5


def adjoint_state(B, kw, seed):
    """Seeded prefilled beam of the adjoint workload (as for gr1e8)."""
    from paper_1011_6330_gb300 import synth
    d = B.derive(tube_params(B, **kw))
    gfar = d["Lambda0"] ** 2 * d["kappa"] * math.cos(kw["incl_rad"])
    return synth.prefilled_beam(kw["target_particles"], d["L"] - d["dz"], gfar, seed=seed,
                                eta_of_z=lambda zz: 1.0 + zz * d["R_over_Rstar"])


def adjoint_cpu_baseline(kw, d, z, u, seconds, stride=100):
    """The oracle's FP64 adjoint as it stands (float32 forward, reverse in
    FP64) on every stride-th particle of the same state (macro charge times
    stride), the full Nz = 16384 grid, as many steps as fit in ~seconds."""
    import oracle as orc
    from oracle import adjoint as oadj
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"],
                        kw["R_cm"])
    nz = kw["Nz"]
    zn = np.arange(nz + 1) * (d["L"] / nz)
    rho = orc.rho_gj_profile(orc.RHO_GR, zn, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"])
    run = oadj.AdjointRun(nz, d["L"], d["dt"], rho, d["s"] * stride, z[::stride], u[::stride],
                          precision="f32", accumulate="fixed")
    t0 = time.perf_counter()
    run.gradient("gamma", 4)
    per_step = (time.perf_counter() - t0) / 4
    n = min(ADJ_STEPS, max(4, int(seconds / per_step)))
    t0 = time.perf_counter()
    _, _, _, inj, _ = run.gradient("gamma", n)
    el = time.perf_counter() - t0
    ps = n * z[::stride].size + sum((n - k) * c for k, c in enumerate(inj))
    return {"value": ps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "oracle adjoint (forward + reverse) of %d steps on %d of the %d particles "
                      "(every %dth, macro charge x%d), Nz=%d, in %.1f s"
                      % (n, z[::stride].size, z.size, stride, stride, nz, el)}


def run_adjoint(args, sub=False):
    """Gradients of the mean terminal gamma with respect to (B, P, R, w) for a
    2000-step run of the B = 1e12 G, P = 0.3 s frame-dragging tube (Nz =
    16384, 1e6 FP32 electrons), checkpointed every 100 steps: one timed
    evaluation is the forward run plus the backward sweep. Reported next to
    the plain forward run of the same tube."""
    import torch
    from paper_1011_6330_gb300 import binding as B
    from paper_1011_6330_gb300 import workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1 and not sub:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    kw = workloads.adjoint_tube()
    d = B.derive(tube_params(B, **kw))
    z, u = adjoint_state(B, kw, rank_seed(rank))
    a = B.Adjoint(tube_params(B, **kw), ADJ_STEPS, ADJ_EVERY)
    a.tube.add_particles(z, u)
    n_eval = max(1, args.steps // ADJ_STEPS)
    timed = not args.no_kernel_timing
    for _ in range(max(1, args.warmup // 4)):
        a.forward()
        a.backward(B.SCLF_OBJ_GAMMA)
    if timed:
        a.set_timing(1)                      # builds both timed instances of each graph
        a.forward()
        a.backward(B.SCLF_OBJ_GAMMA)
        # timed region: every TIME_EVERY-th segment replays a graph with event
        # nodes around each kernel (they cost 2-3 us each against ~10 us kernels)
        a.set_timing(ADJ_TIME_EVERY)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    tf = tb = 0.0
    for _ in range(n_eval):
        vals = a.forward()
        tf += a.timing()["forward_ms"]
        g_rho, g_s = a.backward(B.SCLF_OBJ_GAMMA)
        tb += a.timing()["backward_ms"]
    clk = clocks.stop()
    kt = a.kernel_times()
    a.set_timing(0)
    psteps = a.timing()["particle_steps"]
    a.forward()                              # the same pass without any event node
    untimed_f = a.timing()["forward_ms"]
    a.backward(B.SCLF_OBJ_GAMMA)
    untimed_b = a.timing()["backward_ms"]
    grad_gamma = a.param_gradient(g_rho, g_s)
    g_rho_e, g_s_e = a.backward(B.SCLF_OBJ_EZ)
    bwd_ez_ms = a.timing()["backward_ms"]
    grad_ez = a.param_gradient(g_rho_e, g_s_e)
    el_s = 1e-3 * (tf + tb)
    work, el_s = combine_ranks(psteps * n_eval, el_s, device="cuda")
    # the plain form: the same tube and particles stepped by tube_run (graphs,
    # no event nodes), timed by events around the whole run
    t = B.Tube(tube_params(B, **dict(kw, track_ids=0)))
    t.add_particles(z, u)
    t.solve_fields()
    t.run(2 * ADJ_EVERY)
    stream = torch.cuda.current_stream()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s0 = t.status()["n_particles"]
    p0.record(stream)
    t.run(ADJ_STEPS)
    p1.record(stream)
    torch.cuda.synchronize()
    s1 = t.status()["n_particles"]
    plain_value = 0.5 * (s0 + s1) * ADJ_STEPS / (1e-3 * p0.elapsed_time(p1))
    t.close()
    # the same gradient with the segment length left to the library: the whole
    # run is one segment when its snapshots fit, so the backward pass
    # replays nothing (one warm-up evaluation, then one timed without event nodes)
    a.close()
    a1 = B.Adjoint(tube_params(B, **kw), ADJ_STEPS, 0)
    a1.tube.add_particles(z, u)
    a1.forward()
    a1.backward(B.SCLF_OBJ_GAMMA)
    a1.forward()
    f1_ms = a1.timing()["forward_ms"]
    g1 = a1.param_gradient(*a1.backward(B.SCLF_OBJ_GAMMA))
    b1_ms = a1.timing()["backward_ms"]
    p1 = a1.timing()["particle_steps"]
    one_segment = {"checkpoint_every": a1.checkpoint_every, "forward_ms": f1_ms,
                   "backward_ms": b1_ms, "value": p1 / (1e-3 * (f1_ms + b1_ms)),
                   "grad_gamma_rel_diff": [float(abs(x - y) / abs(y))
                                           for x, y in zip(g1, grad_gamma)]}
    a1.close()
    # FP32 against FP64: the same run with FP64 particles
    a64 = B.Adjoint(tube_params(B, **dict(kw, precision=B.SCLF_FP64)), ADJ_STEPS, ADJ_EVERY)
    a64.tube.add_particles(z, u)
    v64 = a64.forward()
    g64 = [a64.param_gradient(*a64.backward(i)) for i in (B.SCLF_OBJ_GAMMA, B.SCLF_OBJ_EZ)]
    a64.close()
    err32 = {name: [float(abs(x - y) / abs(y)) for x, y in zip(g32, gg)]
             for name, g32, gg in (("gamma", grad_gamma, g64[0]), ("ez", grad_ez, g64[1]))}
    val_err32 = [float(abs(x - y) / abs(y)) for x, y in zip(vals, v64)]
    # the same run with 32-bit fixed-point positions (SCLF_FIX32): its speed
    # (one untimed-graph evaluation after one warm-up) and its error against FP64
    ax = B.Adjoint(tube_params(B, **dict(kw, precision=B.SCLF_FIX32)), ADJ_STEPS, ADJ_EVERY)
    ax.tube.add_particles(z, u)
    ax.forward()
    ax.backward(B.SCLF_OBJ_GAMMA)
    vx = ax.forward()
    fx_ms = ax.timing()["forward_ms"]
    gx = [ax.param_gradient(*ax.backward(B.SCLF_OBJ_GAMMA))]
    bx_ms = ax.timing()["backward_ms"]
    gx.append(ax.param_gradient(*ax.backward(B.SCLF_OBJ_EZ)))
    px = ax.timing()["particle_steps"]
    ax.close()
    fix32 = {"value": px / (1e-3 * (fx_ms + bx_ms)), "unit": UNIT, "forward_ms": fx_ms,
             "backward_ms": bx_ms, "values": list(vx),
             "vs_fp64_values_rel_err": [float(abs(x - y) / abs(y)) for x, y in zip(vx, v64)],
             "vs_fp64_grad_rel_err": {name: [float(abs(x - y) / abs(y)) for x, y in zip(g, gg)]
                                      for name, g, gg in (("gamma", gx[0], g64[0]),
                                                          ("ez", gx[1], g64[1]))}}
    # per kernel: the forward and recompute passes launch the same two kernels
    # algorithmic bytes per launch: particles 16 B (x, u in and out) forward,
    # 24 B (x, u in; lambda_x, lambda_u in and out) in reverse; grid kernels
    # 80 B per cell forward (J accumulator read and cleared, E_z, E_r, B in
    # and out, J and the float gather table out) and 76 B per cell in reverse
    slots = psteps / ADJ_STEPS
    nzc = kw["Nz"]
    if not timed:
        kt = {k: (0.0, 0) for k in B.Adjoint.KERNELS}
    kernels = {
        "push_kernel": (kt["forward_push"][0] + kt["recompute_push"][0],
                        kt["forward_push"][1] + kt["recompute_push"][1], 16 * slots),
        "field_kernel": (kt["forward_field"][0] + kt["recompute_field"][0],
                         kt["forward_field"][1] + kt["recompute_field"][1], 80 * nzc),
        "adj_push_kernel": (kt["reverse_push"][0], kt["reverse_push"][1], 24 * slots),
        "adj_field_kernel": (kt["reverse_field"][0], kt["reverse_field"][1], 76 * nzc),
    }
    nseg = ADJ_STEPS // ADJ_EVERY
    per_eval = {"push_kernel": 2 * ADJ_STEPS - ADJ_EVERY, "field_kernel": 2 * ADJ_STEPS - ADJ_EVERY,
                "adj_push_kernel": ADJ_STEPS, "adj_field_kernel": ADJ_STEPS}
    per_launch = {k: (ms / n if n else 0.0) for k, (ms, n, _) in kernels.items()}
    share = {k: per_launch[k] * per_eval[k] for k in kernels}
    roof = None
    if timed:
        dom = max(share, key=share.get)
        peak, peak_kind = measured_peaks()
        bpl = kernels[dom][2]
        achieved = bpl / (per_launch[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom,
                "peak_source": peak_kind, "bytes_per_launch": bpl,
                "timed_launches": kernels[dom][1],
                "note": "1e6 particles (8 MB per slot array) per launch: launch- and "
                        "latency-bound; event brackets add ~3 us to each timed launch"}
    # end to end through the public API: theta -> objectives, .backward()
    e2e = None
    if not args.no_e2e:
        spec, theta0 = B.adjoint_problem({k: v for k, v in kw.items() if k not in ("dt", "R_cm")},
                                         ADJ_STEPS, ADJ_EVERY, z, u)
        spec["params"].update(dt=kw["dt"], R_cm=kw["R_cm"], launch_overlap=LAUNCH_OVERLAP[0])
        reps = []
        for i in range(3):
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            th = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
            out = B.tube_objectives(th, spec)
            out[0].backward()
            g = th.grad.numpy().copy()
            torch.cuda.synchronize()
            if i > 0:
                reps.append(time.perf_counter() - w0)
        e2e = {"value": psteps / statistics.median(reps), "unit": UNIT,
               "h2d_bytes_per_step": int(z.nbytes + u.nbytes),
               "d2h_bytes_per_step": int(8 * (kw["Nz"] + 1) + 8 + 16 + 32),
               "how": "tube_objectives(theta).backward(): driver creation, host particles in, "
                      "forward, backward, gradient out; median of 2 after 1 warm-up",
               "grad_matches": bool(np.allclose(g, grad_gamma, rtol=1e-9, atol=0))}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = adjoint_cpu_baseline(kw, d, z, u, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": work / el_s, "unit": UNIT, "n_gpus": ws,
        "steps": n_eval * ADJ_STEPS, "warmup": args.warmup,
        "ms_per_step": 1e3 * el_s / (n_eval * ADJ_STEPS), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "adjoint_gr_tube_P0.3s_B1e12G_Nz16384_1e6_particles_fp32",
                   "run_steps": ADJ_STEPS, "checkpoint_every": ADJ_EVERY,
                   "gradient_evaluations": n_eval,
                   "objective": "mean terminal gamma; d/d(B, P, R, w)",
                   "l2": "each pass writes 16 MB per step of snapshots (1.6 GB per segment), "
                         "larger than L2",
                   "parallelism": "independent tube per GPU" if ws > 1 else "one tube"},
        "adjoint": {"forward_ms": tf / n_eval, "backward_ms": tb / n_eval,
                    "timed_segments": ("every %dth" % ADJ_TIME_EVERY) if timed else "none",
                    "untimed_forward_ms": untimed_f, "untimed_backward_ms": untimed_b,
                    "backward_ez_ms": bwd_ez_ms, "values": list(vals),
                    "grad_gamma_BPRw": [float(x) for x in grad_gamma],
                    "grad_ez_BPRw": [float(x) for x in grad_ez],
                    "fp64_values": list(v64), "fp32_vs_fp64_values_rel_err": val_err32,
                    "fp32_vs_fp64_grad_rel_err": err32, "fix32": fix32,
                    "kernels_ms_per_launch": per_launch,
                    "kernels_share_per_evaluation": ({k: v / sum(share.values())
                                                      for k, v in share.items()}
                                                     if timed else None)},
        "plain_form": {"value": plain_value, "unit": UNIT, "steps": ADJ_STEPS,
                       "how": "the same tube and particles stepped by tube_run (graphs), "
                              "CUDA events around the run",
                       "adjoint_over_plain": (work / el_s) / plain_value},
        "one_segment": dict(one_segment, adjoint_over_plain=one_segment["value"] / plain_value,
                            how="checkpoint_every = 0: the library keeps the whole run as "
                                "one segment (its snapshots fit), no recompute; untimed "
                                "graphs"),
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        # per evaluation: the graph kernels (forward, recompute without the
        # last segment, reverse), the gather table, objectives (2) and seed
        # launches and one gather table per recomputed segment
        "gpu_launches": int(n_eval * (sum(per_eval.values()) + 4 + nseg - 1)),
        "clocks": clk,
    }
    if rank == 0 and not sub:
        print(json.dumps(line))
    if sub:
        return line
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


PREC_N, PREC_STEPS, PREC_BINS = 500000, 2000, 64


def binned_profiles(z, u, ez, L, nb):
    """Mean gamma per height bin, E_z averaged over each bin's cells, and the
    particle count per bin."""
    edges = np.linspace(0.0, L, nb + 1)
    idx = np.clip(np.digitize(z, edges) - 1, 0, nb - 1)
    cnt = np.bincount(idx, minlength=nb)
    g = np.sqrt(1.0 + np.asarray(u, np.float64) ** 2)
    gm = np.bincount(idx, weights=g, minlength=nb) / np.maximum(cnt, 1)
    return gm, np.asarray(ez).reshape(nb, -1).mean(axis=1), cnt


def precision_vs_fp64(B, workloads, seed):
    """The headline tube's grid and time step with PREC_N particles of the
    same kind of seeded prefilled beam, PREC_STEPS steps with FIX32, float32
    and FP64 positions on the GPU; the 32-bit runs against the FP64 run
    (which the GPU tests hold to the FP64 oracle within 1e-12): binned gamma
    and E_z (PREC_BINS height bins), E_z cell by cell, particle count per bin."""
    from paper_1011_6330_gb300 import synth
    kw = workloads.gr_tube(n_particles=PREC_N, precision=B.SCLF_FP64,
                           accumulate=B.SCLF_ACC_FIXED64)
    d = B.derive(tube_params(B, **kw))
    L = d["L"]
    gfar = d["Lambda0"] ** 2 * d["kappa"] * math.cos(kw["incl_rad"])
    z, u = synth.prefilled_beam(PREC_N, L - d["dz"], gfar, seed=seed,
                                eta_of_z=lambda zz: 1.0 + zz * d["R_over_Rstar"])
    runs = {}
    for name, prec in (("fp64", B.SCLF_FP64), ("fix32", B.SCLF_FIX32), ("f32", B.SCLF_FP32)):
        t = B.Tube(tube_params(B, **dict(kw, precision=prec)))
        t.add_particles(z, u)
        t.solve_fields()
        t.run(PREC_STEPS)
        zz, uu, _ = t.read_particles()
        ez = t.read_fields(rho=False)["ez"]
        runs[name] = (binned_profiles(zz, uu, ez, L, PREC_BINS), ez)
        t.close()
    (g0, e0, c0), ez0 = runs["fp64"]
    occ = c0 > 0
    out = {"reference": "FP64 particle positions and momenta on the GPU",
           "particles": PREC_N, "steps": PREC_STEPS, "bins": PREC_BINS,
           "how": "max |x - x_fp64| / max |x_fp64| per quantity (gamma bins: per bin, "
                  "relative to the bin's FP64 mean)"}
    for name in ("fix32", "f32"):
        (g, e, c), ez = runs[name]
        out[name] = {"gamma_bins": float(np.max(np.abs(g[occ] - g0[occ]) / g0[occ])),
                     "ez_bins": float(np.max(np.abs(e - e0)) / np.max(np.abs(e0))),
                     "ez_cells": float(np.max(np.abs(ez - ez0)) / np.max(np.abs(ez0))),
                     "count_bins": float(np.max(np.abs(c - c0))) / float(np.max(c0))}
    return out


def batch_precision_vs_fp64(B, workloads, seed, n_sample=8, steps=2000):
    """E_z of sampled death-line tubes (spread over Nz and P) after `steps`
    steps with FIX32 and float32 positions against FP64 positions, each tube
    stepped alone from its seeded prefilled state (a batched tube computes
    the same bits as that tube alone)."""
    from paper_1011_6330_gb300 import synth
    kws = workloads.death_line_batch(seed=seed, precision=B.SCLF_FP64)
    order = sorted(range(len(kws)), key=lambda i: (kws[i]["Nz"], kws[i]["P_s"]))
    pick = [order[k] for k in np.linspace(0, len(order) - 1, n_sample).astype(int)]
    errs = {"fix32": [], "f32": []}
    for i in pick:
        kw = dict(kws[i], track_ids=0)
        ez = {}
        for name, prec in (("fp64", B.SCLF_FP64), ("fix32", B.SCLF_FIX32), ("f32", B.SCLF_FP32)):
            t = B.Tube(tube_params(B, **dict(kw, precision=prec)))
            d = t.derived
            gr = kw["rho_gj_mode"] == B.SCLF_RHO_GR
            gfar = (d["Lambda0"] ** 2 * d["kappa"] * math.cos(kw["incl_rad"]) if gr
                    else math.sqrt(2.0) * d["Lambda0"])
            eta = (lambda zz, r=d["R_over_Rstar"]: 1.0 + zz * r) if gr else None
            z, u = synth.prefilled_beam(kw["target_particles"], d["L"] - d["dz"], gfar,
                                        seed=seed + i, eta_of_z=eta)
            t.add_particles(z, u)
            t.solve_fields()
            t.run(steps)
            ez[name] = t.read_fields(rho=False)["ez"]
            t.close()
        for name in errs:
            errs[name].append(float(np.max(np.abs(ez[name] - ez["fp64"])) /
                                    np.max(np.abs(ez["fp64"]))))
    return {"reference": "the same tubes with FP64 positions and momenta on the GPU",
            "tubes": [{"index": i, "Nz": kws[i]["Nz"], "P_s": kws[i]["P_s"],
                       "B_G": kws[i]["B_G"]} for i in pick],
            "steps": steps, "how": "max_j |E_z - E_z,fp64| / max |E_z,fp64| per tube",
            "fix32_ez": errs["fix32"], "f32_ez": errs["f32"],
            "fix32_ez_median": float(np.median(errs["fix32"])),
            "f32_ez_median": float(np.median(errs["f32"]))}


def secondary_tube(B, workloads, n, precision, acc, order, seed, steps, warmup):
    """Push time and roofline of the headline tube with another particle
    precision or current accumulator (same seeded state)."""
    t, kw, d, _, _, _ = build_tube(B, workloads, "gr1e8", n, acc, order, seed,
                                   precision=precision)
    _STATE.pop("last", None)
    t.solve_fields()
    t.run(warmup)
    t.set_timing(True)
    t.run(steps)
    tm = t.timing()
    t.close()
    push_ms = tm["push_ms"] / max(tm["n_steps"], 1)
    slots = tm["particle_slots"] / max(tm["steps_run"], 1)
    peak, kind = measured_peaks()
    achieved = BYTES_PER_PARTICLE * slots / (push_ms * 1e-3) / 1e9
    return {"positions": precision, "current_accumulator": "fp64" if acc == B.SCLF_ACC_FP64
            else "fixed64", "steps": steps, "push_ms_avg": push_ms,
            "particle_steps_per_s_push": slots / (push_ms * 1e-3),
            "roofline": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": kind}}


def form_summary(line, headline_value):
    """The batched or adjoint form's figures next to its plain form."""
    pf = line["plain_form"]
    roof = line.get("roofline") or {}
    out = {"workload": line["config"]["workload"], "dtype": line["dtype"],
           "value": line["value"], "unit": line["unit"],
           "steps": line["steps"], "plain_value": pf["value"],
           "vs_plain": line["value"] / pf["value"], "plain_how": pf["how"],
           "vs_headline": line["value"] / headline_value,
           "roofline": {k: roof.get(k) for k in ("kernel", "achieved", "peak", "frac",
                                                  "push_ms_avg", "bytes_per_launch")},
           "clocks": line["clocks"]}
    if "adjoint" in line:
        a = line["adjoint"]
        out["forward_ms"], out["backward_ms"] = a["forward_ms"], a["backward_ms"]
        out["checkpoint_every"] = ADJ_EVERY
        out["one_segment"] = line["one_segment"]
        out["fp32_vs_fp64_grad_rel_err"] = a["fp32_vs_fp64_grad_rel_err"]
    return out


def sub_args(args, **kw):
    """A copy of the arguments for a form measured inside the default run."""
    d = dict(vars(args))
    d.update(no_e2e=True, no_cpu_baseline=True, no_kernel_timing=False)
    d.update(kw)
    return argparse.Namespace(**d)


def run_dtube(args):
    """One tube split into z-domains on one GPU, as virtual sub-domains of a
    multi-GPU run (dtube_*): the gr1e8 tube (FIX32 by default) cut into
    args.domains equal cell ranges, each with its own slots, stream and grid
    copy, stepped by dtube_run with the per-step exchanges (boundary current,
    crossing particles, B_phi / E_z halos); reported next to the same seeded
    tube stepped whole by tube_run. Both are timed by the wall clock around
    the run with the device synchronised on both sides (dtube_run launches on
    several streams)."""
    import torch
    from paper_1011_6330_gb300 import binding as B
    from paper_1011_6330_gb300 import workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    n = int(args.particles or 1e8)
    t, kw, d, _, _, _ = build_tube(B, workloads, "gr1e8", n, B.SCLF_ACC_FIXED64, args.order,
                                   seed=rank_seed(rank), nz=args.nz, precision=args.precision)
    _, z, u = _STATE.pop("last")

    def timed(obj):
        obj.run(args.warmup)
        torch.cuda.synchronize()
        s0 = obj.status()
        w0 = time.perf_counter()
        obj.run(args.steps)
        torch.cuda.synchronize()
        el = time.perf_counter() - w0
        s1 = obj.status()
        return 0.5 * (s0["n_particles"] + s1["n_particles"]) * args.steps / el, el, s1

    t.solve_fields()
    whole, el_whole, _ = timed(t)
    t.close()
    dtb = B.DTube(tube_params(B, **kw), n=args.domains)
    dtb.load_particles(z, u)
    del z, u
    dtb.solve_fields()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    value, el, st = timed(dtb)
    clk = clocks.stop()
    xs = dtb.exchange_stats()
    per = max(xs["steps"], 1)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fix32+f32" if args.precision == "fix32" else "f32", "data": "synthetic",
            "config": {"workload": gr_workload_name(n, kw["Nz"], args.precision)
                       + "_zdomains%d" % args.domains,
                       "domains": args.domains, "Nz": kw["Nz"], "particles_per_gpu": n,
                       "parallelism": "one tube in %d z-domains on one GPU" % args.domains,
                       "timing": "wall clock around dtube_run / tube_run, device "
                                 "synchronised on both sides"},
            "whole_tube": {"value": whole, "ms_per_step": 1e3 * el_whole / args.steps},
            "vs_whole": value / whole,
            "exchange_per_step": {"field_bytes": xs["field_bytes"] / per,
                                  "particles": xs["particles"] / per,
                                  "particle_bytes": xs["particle_bytes"] / per},
            "clocks": clk, "status": {"flags": st["flags"], "n_particles": st["n_particles"]}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "dtube":
        return run_dtube(args)
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
                                          seed=rank_seed(rank), sort_interval=args.sort_interval,
                                          nz=args.nz, push_stages=args.push_stages,
                                          precision=args.precision)
    t.solve_fields()
    sort_ms = None
    if args.sort_interval > 0:                       # a stable re-sort by cell up front
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        t.sort()
        sort_ms = 1e3 * (time.perf_counter() - w0)
    stream = torch.cuda.current_stream()

    # warm-up
    t.run(args.warmup)
    torch.cuda.synchronize()
    st0 = t.status()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier(ws)
    torch.cuda.synchronize()
    t.set_timing(TIME_EVERY)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t.run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
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
    slots_per_launch = tm["particle_slots"] / max(tm["steps_run"], 1)
    achieved = BYTES_PER_PARTICLE * slots_per_launch / (push_avg_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = None
    fix32 = large or args.precision == "fix32"
    tkey = args.workload + ("_fix32" if fix32 and not large else "")
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        ent = tr.get(tkey, {})
        if ent.get("kernel_sha") == kernel_sha(tkey) \
                and ent.get("accumulate", "fixed64") == args.accumulate \
                and ent.get("order", "descending") == args.order and ent.get("particles") == n:
            traffic = ent["bytes_per_launch"]
    gpu_launches = 2 * tm["steps_run"] + tm["compactions_run"]
    check = t.check()

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        xi_h, u_h, _ = t.save_particles()
        tdt = {np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64,
               np.dtype(np.int32): torch.int32}
        pin_x = torch.empty(xi_h.size, dtype=tdt[xi_h.dtype], pin_memory=True)
        pin_u = torch.empty(u_h.size, dtype=tdt[u_h.dtype], pin_memory=True)
        pin_x.numpy()[:] = xi_h
        pin_u.numpy()[:] = u_h
        del xi_h, u_h
        out_x = torch.empty_like(pin_x, pin_memory=True)
        out_u = torch.empty_like(pin_u, pin_memory=True)
        import ctypes as C
        lib = B.load()
        nout = C.c_int64()
        ksteps = args.steps
        barrier(ws)
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        lib.tube_load_particles(t.h, pin_x.numel(), C.c_void_p(pin_x.data_ptr()),
                                C.c_void_p(pin_u.data_ptr()), None)
        tickets = []
        for _ in range(ksteps):
            tickets.append(t.status_async())             # per-step D2H of the counters
            t.step()
        cap = out_x.numel()
        rc = lib.tube_save_particles(t.h, cap, C.byref(nout), C.c_void_p(out_x.data_ptr()),
                                     C.c_void_p(out_u.data_ptr()), None)
        n_e2e = 0
        for k in tickets:                                # every step's counters on the host
            st = t.status_collect(k)
            n_e2e += st["n_particles"] + st["pending_injection"]
        torch.cuda.synchronize()
        el_e2e = time.perf_counter() - h0
        n_all, el_e2e = combine_ranks(n_e2e, el_e2e, device="cuda")
        state_bytes = pin_x.numel() * pin_x.element_size() + pin_u.numel() * pin_u.element_size()
        e2e = {"value": n_all / el_e2e, "unit": UNIT,
               "h2d_bytes_per_step": state_bytes / ksteps,
               "d2h_bytes_per_step": (state_bytes * min(cap, nout.value) / max(cap, 1)
                                      + ksteps * 144) / ksteps,   # 144-byte counter block
               "path": "tube_load_particles(pinned) + K x (tube_status_async, tube_step) + "
                       "tube_save_particles(pinned) + K x tube_status_collect",
               "amortised_over_steps": ksteps,
               "note": "the whole particle state goes in and comes back once per K = %d "
                       "steps; per-step copies are the 144-byte counter block" % ksteps,
               "rc": int(rc)}

    cpu = None
    cpu_all = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(zs, us, n, kw, d, args.cpu_seconds, stride)
        cpu["host"] = host_info()
        if not large:
            cpu_all = cpu_baseline_allcore(*_sample(n, 10), n, kw, d, args.cpu_seconds, 10)
            cpu_all.pop("final_ez")
            cpu_all["host"] = cpu["host"]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "fix32+f32" if fix32 else "f32",
        "data": "synthetic",
        "config": {"workload": ("large_tube_P0.1s_B3e12G_Nz%d_%d_particles_fix32" % (kw["Nz"], n))
                   if large else gr_workload_name(n, kw["Nz"], args.precision),
                   "positions": ("32-bit fixed point, 2^-%d cell (SCLF_FIX32)"
                                 % (31 - int(math.ceil(math.log2(kw["Nz"]))))) if fix32
                   else "float32",
                   "rho_gj": "frame-dragging (Eq. 6-7), i = 0.5 rad",
                   "particles_per_gpu": n, "Nz": kw["Nz"], "Lambda0": d["Lambda0"],
                   "dt_R_over_c": d["dt"], "order": args.order,
                   "current_accumulator": args.accumulate,
                   "push_stages": args.push_stages or "default",
                   "launch_overlap": getattr(args, "launch_overlap", "on"),
                   "sort_by_cell": ({"interval_steps": args.sort_interval,
                                     "first_sort_ms_wall": sort_ms}
                                    if args.sort_interval > 0 else None),
                   "l2": "inputs larger than L2 (particle state %.0f MB per GPU)" % (8 * n / 1e6),
                   "parallelism": "independent tube per GPU" if ws > 1 else "single tube"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "push_fix32_kernel" if fix32 else
                     ("push_kernel<float, fixed64>" if acc == B.SCLF_ACC_FIXED64
                      else "push_kernel<float, fp64>"),
                     "peak_source": peak_kind, "push_ms_avg": push_avg_ms,
                     "field_ms_avg": tm["field_ms"] / max(tm["n_steps"], 1),
                     "compact_ms_total": tm["compact_ms"],
                     "compaction_checks": tm["compactions_run"],
                     "timed_steps": tm["n_steps"], "timing_sample": TIMING_SAMPLE,
                     "bytes_per_launch": BYTES_PER_PARTICLE * slots_per_launch},
        "cpu_baseline": cpu,
        "cpu_baseline_allcore": cpu_all,
        "e2e": e2e,
        "gpu_launches": int(gpu_launches),
        "clocks": clk,
        "status": {"check": int(check), "n_particles": st1["n_particles"],
                   "injected_per_step": (st1["total_injected"] - st0["total_injected"]) / args.steps,
                   "flags": st1["flags"]},
    }
    t.close()
    # the same workload in its other forms, measured after the headline (N = 1)
    if not args.no_extras and ws == 1 and not large:
        other = "f32" if fix32 else "fix32"
        line["precision_vs_fp64"] = precision_vs_fp64(B, workloads, rank_seed(rank))
        line["other_positions"] = secondary_tube(B, workloads, n, other, B.SCLF_ACC_FIXED64,
                                                 args.order, rank_seed(rank), 100, 5)
        line["fp64_accumulator"] = secondary_tube(B, workloads, n, "f32", B.SCLF_ACC_FP64,
                                                  args.order, rank_seed(rank), 50, 5)
        line["batched"] = form_summary(run_batch(sub_args(args, steps=64, warmup=5), sub=True),
                                       value)
        line["batched"]["precision_vs_fp64"] = batch_precision_vs_fp64(B, workloads,
                                                                       rank_seed(rank))
        line["adjoint"] = form_summary(run_adjoint(sub_args(args, steps=2000, warmup=4),
                                                   sub=True), value)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
