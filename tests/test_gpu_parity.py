"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Integers (injection counts, IDs, removal counts) must match exactly.
Floating point is compared norm-wise per field and per step,
max|x - x_ref| / max|x_ref|: <= 1e-12 for FP64 particles, <= 1e-5 for FP32
particles (against the oracle run in the same particle precision, so that
the floating-point decisions -- which cell, inside or outside -- are taken
in the same precision on both sides).
"""

import ctypes as C
import math

import numpy as np
import pytest

import oracle as orc
from paper_1011_6330_gb300 import binding as B
from paper_1011_6330_gb300 import synth, workloads

pytestmark = pytest.mark.gpu

TOL = {B.SCLF_FP64: 1e-12, B.SCLF_FP32: 1e-5}


def rel(a, b, floor=0.0):
    """max|a - b| / max(max|b|, floor): norm-wise relative error."""
    den = max(float(np.max(np.abs(b))) if np.size(b) else 0.0, floor)
    return float(np.max(np.abs(a - b))) / den if den > 0 else float(np.max(np.abs(a - b), initial=0.0))


def pair(gpu_lib, kw, oprec, oacc, capacity=None):
    t = B.Tube(B.default_params(**kw))
    d = t.derived
    rho = np.asarray(kw["rho_gj_user"]) if kw.get("rho_gj_mode") == B.SCLF_RHO_USER else None
    if rho is None:
        cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
        z = np.arange(kw["Nz"] + 1) * (kw["L_over_R"] / kw["Nz"])
        rho = orc.rho_gj_profile(orc.RHO_GR, z, cu["Lambda0"], kw["incl_rad"],
                                 cu["theta_star"], cu["R_over_Rstar"], cu["kappa"])
    o = orc.Tube(kw["Nz"], kw["L_over_R"], d["dt"], rho, d["s"], precision=oprec,
                 accumulate=oacc, capacity=capacity)
    return t, o


def compare(t, o, tol, what=""):
    st = t.status()
    assert st["step"] == o.step_count
    assert st["total_injected"] == o.total_injected, what
    assert st["last_injected"] == o.last_injected, what
    assert st["last_removed"] == o.last_removed, what
    assert st["n_particles"] == o.xi.size, what
    z, u, ids = t.read_particles()
    assert np.array_equal(ids, o.ids), what
    f = t.read_fields(rho=False)
    # E_r and B_phi share E_z's units; their scale is the field's scale
    scale = float(np.max(np.abs(o.ez)))
    errs = dict(ez=rel(f["ez"], o.ez), er=rel(f["er"], o.er, scale),
                b=rel(f["b"], o.b, scale), j=rel(f["j"], o.j))
    if z.size:
        errs["z"] = float(np.max(np.abs(z - o.z()))) / o.L
        g, go = np.sqrt(1 + u * u), o.gamma()
        errs["gamma"] = float(np.max(np.abs(g - go) / go))
    for k, v in errs.items():
        assert v <= tol, (what, k, v)
    return errs


# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [B.SCLF_FP64, B.SCLF_FP32])
def test_initial_fields_match_oracle(gpu_lib, prec):
    kw = workloads.flat_sclf_small(precision=prec)
    t, o = pair(gpu_lib, kw, "f64", "sum")
    f = t.read_fields()
    assert rel(f["ez"], o.ez) < 1e-12 and rel(f["er"], o.er) < 1e-12
    assert np.all(f["b"] == 0) and np.all(f["rho"] == 0)
    st = t.status()
    n, es = orc.injection_count(o.ez[0], 0, o.s, o.dz, o.rho_gj[0])
    assert st["pending_injection"] == n and abs(st["surface_field"] - es) < 1e-12 * abs(es)
    t.close()


def test_initial_fields_gr_profile_match_oracle(gpu_lib):
    kw = workloads.gr_tube(Nz=4096, n_particles=10 ** 5, P_s=0.3)
    t, o = pair(gpu_lib, kw, "f32", "fixed")
    f = t.read_fields(rho=False)
    assert rel(f["ez"], o.ez) < 1e-11 and rel(f["er"], o.er) < 1e-11
    assert t.status()["pending_injection"] == o.injection_count()
    t.close()


def test_fp64_tube_matches_oracle_every_step(gpu_lib):
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP64, accumulate=B.SCLF_ACC_FP64)
    t, o = pair(gpu_lib, kw, "f64", "sum")
    worst = {}
    for n in range(200):
        t.step()
        o.step()
        e = compare(t, o, TOL[B.SCLF_FP64], "step %d" % n)
        worst = {k: max(v, worst.get(k, 0.0)) for k, v in e.items()}
    assert o.xi.size > 3000
    print("fp64 worst", worst)
    t.close()


@pytest.mark.parametrize("acc,oacc", [(B.SCLF_ACC_FIXED64, "fixed"), (B.SCLF_ACC_FP64, "sum")])
def test_fp32_tube_matches_same_precision_oracle_every_step(gpu_lib, acc, oacc):
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=acc)
    t, o = pair(gpu_lib, kw, "f32", oacc)
    worst = {}
    for n in range(200):
        t.step()
        o.step()
        e = compare(t, o, TOL[B.SCLF_FP32], "step %d" % n)
        worst = {k: max(v, worst.get(k, 0.0)) for k, v in e.items()}
    print("fp32", oacc, "worst", worst)
    t.close()


def test_fp32_error_against_fp64_oracle_is_stated(gpu_lib):
    """FP32 particles against the FP64 definition: bounded, and reported."""
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64)
    t, o = pair(gpu_lib, kw, "f64", "sum")
    t.run(200)
    o.run(200)
    f = t.read_fields(rho=False)
    z, u, ids = t.read_particles()
    e_ez = rel(f["ez"], o.ez)
    common = min(ids.size, o.ids.size)
    print("fp32 vs fp64 oracle after 200 steps: Ez %.2e, injected %d vs %d"
          % (e_ez, t.status()["total_injected"], o.total_injected))
    assert e_ez < 1e-3
    assert abs(t.status()["total_injected"] - o.total_injected) <= 0.01 * o.total_injected
    assert common > 0
    t.close()


def test_ragged_tiles_compaction_schedule_and_graphs_do_not_change_results(gpu_lib):
    """Prefilled particles spanning several tiles with a ragged tail; the same
    run with forced compactions every 7 steps, with compaction checks every
    1000 steps, and with CUDA graphs, is bit-identical (fixed-point current),
    and matches the oracle."""
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64)
    z, u = synth.random_particles(4096 * 3 + 1234, kw["L_over_R"], seed=7, u_sigma=2.0)
    runs = []
    for ci, graphs, forced in ((3, 0, True), (1000, 0, False), (4, 1, False)):
        t, o = pair(gpu_lib, dict(kw, compact_interval=ci, use_graphs=graphs), "f32", "fixed")
        t.add_particles(z, u)
        o.add_particles(z, u)
        if forced:                       # compact every 7 steps whatever the holes
            for n in range(101):
                t.step()
                if n % 7 == 6:
                    t.compact()
                    st = t.status()
                    assert st["n_slots"] == st["n_particles"]
        else:
            t.run(101)
        o.run(101)
        compare(t, o, TOL[B.SCLF_FP32], "compact %d graphs %d" % (ci, graphs))
        runs.append((t.read_particles(), t.read_fields(rho=False)))
        t.close()
    (p0, f0) = runs[0]
    for (p1, f1) in runs[1:]:
        for a, b in zip(p0, p1):
            assert np.array_equal(a, b)
        for k in ("ez", "er", "b", "j"):
            assert np.array_equal(f0[k], f1[k])


def test_empty_tube_with_positive_rho_gj_stays_empty_and_stationary(gpu_lib):
    nz = 257
    kw = dict(workloads.flat_sclf_small(precision=B.SCLF_FP64), Nz=nz, dt=0.4 * 8.0 / nz,
              rho_gj_user=np.linspace(0.5, 1.5, nz + 1), macro_charge=-1e-3)
    t, o = pair(gpu_lib, kw, "f64", "sum")
    f0 = t.read_fields(rho=False)
    t.run(500)
    o.run(500)
    st = t.status()
    assert st["n_particles"] == 0 and st["total_injected"] == 0
    f = t.read_fields(rho=False)
    assert rel(f["ez"], f0["ez"]) < 1e-12 and np.max(np.abs(f["b"])) < 1e-12 * np.max(np.abs(f0["ez"]))
    compare(t, o, 1e-12)
    t.close()


def test_capacity_exhaustion_clips_injection_and_sets_the_flag(gpu_lib):
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64,
                                   capacity=100)
    t, o = pair(gpu_lib, kw, "f32", "fixed", capacity=100)
    t.step()
    o.step()
    st = t.status()
    assert st["total_injected"] == 100 == o.total_injected
    assert st["flags"] & B.FLAG_CAPACITY and o.capacity_hit
    assert t.check() == -4
    compare(t, o, TOL[B.SCLF_FP32])
    t.close()


def test_particles_leave_through_both_ends(gpu_lib):
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP64, accumulate=B.SCLF_ACC_FP64)
    t, o = pair(gpu_lib, kw, "f64", "sum")
    dz = kw["L_over_R"] / kw["Nz"]
    z = np.array([0.1 * dz, 0.5, 8.0 - 0.1 * dz, 3.0])
    u = np.array([-50.0, 0.0, 50.0, 1.0])
    t.add_particles(z, u)
    o.add_particles(z, u)
    t.step()
    o.step()
    assert o.last_removed >= 2
    compare(t, o, 1e-12)
    t.close()


def test_inject_call_save_load_and_invalid_input(gpu_lib):
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64)
    t, o = pair(gpu_lib, kw, "f32", "fixed")
    n = t.inject()
    assert n == o.inject() and n > 1000
    t.run(30)
    xi, u, ids = t.save_particles()
    st = t.status()
    t.load_particles(xi, u, ids)
    xi2, u2, ids2 = t.save_particles()
    assert np.array_equal(xi, xi2) and np.array_equal(u, u2) and np.array_equal(ids, ids2)
    assert t.status()["total_injected"] == int(ids.max()) + 1
    assert t.status()["pending_injection"] == st["pending_injection"]
    with pytest.raises(B.SclfError):
        t.load_particles(np.array([1.0], np.float32), np.array([np.inf], np.float32))
    assert t.status()["n_particles"] == 0       # a rejected load leaves no particles
    with pytest.raises(B.SclfError):
        t.load_particles(np.array([1.0, 1024.0], np.float32), np.zeros(2, np.float32))
    with pytest.raises(B.SclfError):
        t.add_particles([8.0], [0.0])        # z = L is outside the tube
    t.close()


def test_pipelined_status_matches_the_blocking_read(gpu_lib):
    """tube_status_async queues a copy of the counters without waiting;
    tube_status_collect returns exactly what tube_status read at that point,
    and rejects tickets not yet issued or already overwritten in the ring."""
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64)
    t = B.Tube(B.default_params(**kw))
    z, u = synth.prefilled_beam(5000, 7.9, 5.0, seed=3)
    t.add_particles(z, u)
    t.solve_fields()
    tickets, direct = [], []
    for _ in range(12):
        tickets.append(t.status_async())
        direct.append(t.status())
        t.step()
    for k, st in zip(tickets, direct):
        assert t.status_collect(k) == st
    for bad in (-1, tickets[-1] + 1):
        with pytest.raises(B.SclfError):
            t.status_collect(bad)
    last = [t.status_async() for _ in range(1024)][-1]
    with pytest.raises(B.SclfError):
        t.status_collect(tickets[0])              # overwritten in the 1024-entry ring
    assert t.status_collect(last) == t.status()
    t.close()


def test_save_with_holes_compacts_and_keeps_id_order(gpu_lib):
    """Saving a tube whose slots hold holes (particles that left) returns the
    live particles in ID order (a device-side compaction), the same as
    read_particles and the oracle; loading them back resumes identically."""
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64)
    kw["compact_interval"] = 100000                 # no compaction check during the run
    t, o = pair(gpu_lib, kw, "f32", "fixed")
    z, u = synth.prefilled_beam(30000, 8.0 - 8.0 / 1024, 5.0, seed=2)
    t.add_particles(z, u)
    o.add_particles(z, u)
    for _ in range(150):
        t.step()
        o.step()
    st = t.status()
    assert st["n_slots"] > st["n_particles"]         # holes are there
    xi, uu, ids = t.save_particles()
    assert np.array_equal(ids, o.ids) and np.array_equal(xi, o.xi) and np.array_equal(uu, o.u)
    assert t.status()["n_slots"] == t.status()["n_particles"]
    t2 = B.Tube(B.default_params(**kw))
    t2.load_particles(xi, uu, ids)
    t2.solve_fields()
    assert t2.status()["total_injected"] == int(ids.max()) + 1
    t.close()
    t2.close()


def _state_against_oracle(t, o, cells_per_unit, what=""):
    """A tube's state against the oracle's, both stepped from the same seeded
    synthetic state with their own Eq. 4 solves. The two initial solves
    agree to ~1e-12 (different tridiagonal solvers), so the float32 gather
    tables may differ in the last bit of a few entries: the counts must match
    exactly, the fields norm-wise, the particles to an ulp-level bound, and
    nearly all particles bit for bit."""
    st = t.status()
    assert st["step"] == o.step_count, what
    assert st["last_injected"] == o.last_injected, what
    assert st["last_removed"] == o.last_removed, what
    assert st["n_particles"] == o.xi.size, what
    assert st["pending_injection"] == o.injection_count(), what
    f = t.read_fields(rho=False)
    scale = float(np.max(np.abs(o.ez)))
    assert rel(f["ez"], o.ez) < 1e-9, what
    assert rel(f["er"], o.er, scale) < 1e-9 and rel(f["b"], o.b, scale) < 1e-9, what
    assert rel(f["j"], o.j) < 1e-6, what
    x, u, _ = t.save_particles()                      # slot order = ID order
    same = np.count_nonzero((x.astype(o.xi.dtype) == o.xi) & (u == o.u))
    dx = float(np.max(np.abs(x.astype(np.float64) - o.xi.astype(np.float64)), initial=0.0))
    du = float(np.max(np.abs(u.astype(np.float64) - o.u) / np.sqrt(1.0 + o.u.astype(np.float64) ** 2),
                      initial=0.0))
    print("%s: %d of %d particles bit for bit, max |dxi| %.3g cells, max |du|/gamma %.3g"
          % (what, same, x.size, dx / cells_per_unit, du))
    assert same >= 0.999 * x.size, what
    assert dx / cells_per_unit < 1e-2 and du < 1e-5, what


def _full_size_against_oracle(t, o, steps, cells_per_unit):
    """Step the tube and the oracle together and compare after every step."""
    f = t.read_fields(rho=False)
    assert rel(f["ez"], o.ez) < 1e-10
    assert rel(f["er"], o.er, float(np.max(np.abs(o.ez)))) < 1e-10
    for n in range(steps):
        t.step()
        o.step()
        _state_against_oracle(t, o, cells_per_unit, "step %d" % n)
    assert t.check() == 0


def test_full_size_gr_tube_against_oracle_on_all_particles(gpu_lib):
    """The benchmark's tube (frame-dragging rho_GJ, 1e8 FP32 particles, Nz =
    65536, fixed-point current) in the launch configuration the benchmark
    times, and the oracle, both from the same seeded synthetic state: three
    steps compared on every particle, the whole grid and every count."""
    kw = workloads.gr_tube()
    t = B.Tube(B.default_params(**kw))
    d = t.derived
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
    eta = lambda zz: 1.0 + zz * cu["R_over_Rstar"]
    gfar = cu["Lambda0"] ** 2 * cu["kappa"] * math.cos(kw["incl_rad"])
    z, u = synth.prefilled_beam(kw["target_particles"], d["L"] - d["dz"], gfar, seed=0,
                                eta_of_z=eta)
    t.add_particles(z, u)
    t.solve_fields()
    zn = np.arange(kw["Nz"] + 1) * d["dz"]
    rho = orc.rho_gj_profile(orc.RHO_GR, zn, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"])
    o = orc.Tube(kw["Nz"], d["L"], d["dt"], rho, d["s"], precision="f32", accumulate="fixed")
    o.add_particles(z, u)
    del z, u
    o.solve_fields()
    _full_size_against_oracle(t, o, 3, 1.0)
    t.close()


# ---------------------------------------------------------------------------
# SCLF_FIX32: 32-bit fixed-point positions
# ---------------------------------------------------------------------------

def test_fix32_tube_matches_oracle_every_step(gpu_lib):
    kw = workloads.flat_sclf_small(precision=B.SCLF_FIX32, accumulate=B.SCLF_ACC_FIXED64)
    t, o = pair(gpu_lib, kw, "fix32", "fixed")
    assert t.derived["pos_unit"] == 2.0 ** -o.fb
    worst = {}
    for n in range(200):
        t.step()
        o.step()
        e = compare(t, o, TOL[B.SCLF_FP32], "step %d" % n)
        worst = {k: max(v, worst.get(k, 0.0)) for k, v in e.items()}
    X, u, ids = t.save_particles()
    assert np.array_equal(X.astype(np.int64), o.xi) and np.array_equal(u, o.u)
    print("fix32 worst", worst)
    t.close()


def test_fix32_ragged_tiles_with_forced_compaction(gpu_lib):
    kw = workloads.flat_sclf_small(precision=B.SCLF_FIX32, accumulate=B.SCLF_ACC_FIXED64)
    z, u = synth.random_particles(2048 * 5 + 77, kw["L_over_R"], seed=8, u_sigma=2.0)
    t, o = pair(gpu_lib, dict(kw, compact_interval=5), "fix32", "fixed")
    t.add_particles(z, u)
    o.add_particles(z, u)
    for n in range(60):
        t.step()
        o.step()
        if n % 9 == 8:
            t.compact()
    compare(t, o, TOL[B.SCLF_FP32])
    X, uu, ids = t.save_particles()
    assert np.array_equal(X.astype(np.int64), o.xi) and np.array_equal(ids, o.ids)
    t.close()


@pytest.mark.parametrize("nz", [16, 17, 33])
def test_fix32_smallest_grids_match_oracle(gpu_lib, nz):
    """FIX32 tubes of the fewest cells allowed (16: 27 fractional bits, the
    most; 17: 26; 33: 25), particles in every cell, exits at both ends,
    holes left between compactions and injection every step, against the
    FIX32 oracle every step."""
    L = 8.0
    kw = dict(workloads.flat_sclf_small(precision=B.SCLF_FIX32, accumulate=B.SCLF_ACC_FIXED64,
                                        capacity=1 << 21),
              Nz=nz, dt=0.4 * L / nz, rho_gj_user=-np.ones(nz + 1), compact_interval=8)
    z, u = synth.random_particles(3000, L * (1 - 1e-3), seed=20 + nz, u_sigma=2.0)
    t, o = pair(gpu_lib, kw, "fix32", "fixed")
    assert t.derived["pos_unit"] == 2.0 ** -o.fb
    t.add_particles(z, u)
    o.add_particles(z, u)
    for n in range(60):
        t.step()
        o.step()
        compare(t, o, TOL[B.SCLF_FP32], "Nz %d step %d" % (nz, n))
    assert t.status()["flags"] == 0
    assert o.total_injected > 0 and o.last_removed >= 0
    X, uu, ids = t.save_particles()
    assert np.array_equal(X.astype(np.int64), o.xi) and np.array_equal(uu, o.u)
    t.close()


def test_large_fix32_tube_against_oracle_on_all_particles(gpu_lib):
    """The large tube's configuration (B = 3e12 G, P = 0.1 s, Nz = 2^20,
    fixed-point positions) with 2^27 particles, and the oracle, both from the
    same seeded synthetic state: two steps compared on every particle, the
    whole grid and every count."""
    n = 2 ** 27
    kw = workloads.large_tube(n_particles=n)
    t = B.Tube(B.default_params(**kw))
    d = t.derived
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
    eta = lambda zz: 1.0 + zz * cu["R_over_Rstar"]
    gfar = cu["Lambda0"] ** 2 * cu["kappa"] * math.cos(kw["incl_rad"])
    zn = np.arange(kw["Nz"] + 1) * d["dz"]
    rho = orc.rho_gj_profile(orc.RHO_GR, zn, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"])
    o = orc.Tube(kw["Nz"], d["L"], d["dt"], rho, d["s"], precision="fix32", accumulate="fixed")
    for z, u in synth.prefilled_beam_chunks(n, d["L"] - d["dz"], gfar, seed=5,
                                            chunk=1 << 25, eta_of_z=eta):
        t.add_particles(z, u)
        o.add_particles(z, u)
    t.solve_fields()
    o.solve_fields()
    _full_size_against_oracle(t, o, 2, float(2 ** orc.fix32_bits(kw["Nz"])))
    t.close()


def test_large_tube_full_size_step_against_streamed_oracle(gpu_lib):
    """The large tube at its benchmark size (2^30 fixed-point particles, Nz =
    2^20, the benchmark's seeded state and launch configuration): one step
    against the oracle streamed over 2^26-particle chunks -- the oracle's own
    initial fields from the summed cloud-in-cell charge, then every
    particle's gather, push and deposit, the removals, the injected
    electrons, the whole current grid, the field update and the next
    injection count."""
    n, chunk = 2 ** 30, 1 << 26
    kw = workloads.large_tube(n_particles=n)
    t = B.Tube(B.default_params(**kw))
    d = t.derived
    nz, dz, dt, s = kw["Nz"], d["dz"], d["dt"], d["s"]
    fb = orc.fix32_bits(nz)
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
    eta = lambda zz: 1.0 + zz * cu["R_over_Rstar"]
    gfar = cu["Lambda0"] ** 2 * cu["kappa"] * math.cos(kw["incl_rad"])
    rho_gj = orc.rho_gj_profile(orc.RHO_GR, np.arange(nz + 1) * dz, cu["Lambda0"],
                                kw["incl_rad"], cu["theta_star"], cu["R_over_Rstar"], cu["kappa"])
    o = orc.Tube(nz, d["L"], dt, rho_gj, s, precision="fix32", accumulate="fixed")
    rho, w0, pieces = np.zeros(nz + 1), 0, []
    for z, u in synth.prefilled_beam_chunks(n, d["L"] - dz, gfar, seed=0, chunk=chunk,
                                            eta_of_z=eta):
        t.add_particles(z, u)
        oc = orc.Tube(nz, d["L"], dt, rho_gj, s, precision="fix32", accumulate="fixed")
        oc.add_particles(z, u)
        rho += oc.rho_nodes()
        w0 += oc.w0
        pieces.append((oc.xi.astype(np.int32), oc.u))
        del z, u, oc
    t.solve_fields()
    o.solve_fields(rho)
    f0 = t.read_fields(rho=False)
    assert rel(f0["ez"], o.ez) < 1e-10
    n_inj, _ = orc.injection_count(o.ez[0], w0, s, dz, rho_gj[0])
    assert t.status()["pending_injection"] == n_inj
    t.step()
    st = t.status()
    f1 = t.read_fields(rho=False)
    Xg, ug, _ = t.save_particles()                    # slot order = ID order
    pieces.append((np.zeros(n_inj, np.int32), np.zeros(n_inj, np.float32)))
    acc = np.zeros(nz, np.int64)
    off = removed = same = w1 = 0
    dx = du = 0.0
    for X, u in pieces:
        X = X.astype(np.int64)
        e = orc.gather_fix32(o.ez, X, fb)
        X1, u1, ok = orc.push_fix32(X, u, e, dt, dz, fb)
        acc += orc.deposit_fix32(nz, X[ok], X1[ok], fb)
        alive = ok & (X1 >= 0) & (X1 < (nz << fb))
        X1, u1 = X1[alive], u1[alive]
        k = X1.size
        removed += X.size - k
        gx, gu = Xg[off:off + k].astype(np.int64), ug[off:off + k]
        assert gx.size == k
        same += int(np.count_nonzero((gx == X1) & (gu == u1)))
        if k:
            dx = max(dx, float(np.max(np.abs(gx - X1))) * 2.0 ** -fb)
            du = max(du, float(np.max(np.abs(gu.astype(np.float64) - u1)
                                      / np.sqrt(1.0 + u1.astype(np.float64) ** 2))))
        w1 += orc.base_weight_fix32(X1, fb)
        off += k
    print("2^30 step: %d of %d particles bit for bit, max |dxi| %.3g cells, max |du|/gamma %.3g"
          % (same, off, dx, du))
    assert off == Xg.size == st["n_particles"]
    assert st["last_injected"] == n_inj and st["last_removed"] == removed
    assert same >= 0.999 * off and dx < 1e-2 and du < 1e-5
    j = orc.current_from(acc, s, dt, "fixed")
    ez, er, b = orc.field_update(o.ez, o.er, o.b, j, dt, dz)
    scale = float(np.max(np.abs(ez)))
    assert rel(f1["j"], j) < 1e-6
    assert rel(f1["ez"], ez) < 1e-9 and rel(f1["er"], er, scale) < 1e-9
    assert rel(f1["b"], b, scale) < 1e-9
    n_next, _ = orc.injection_count(ez[0], w1, s, dz, rho_gj[0])
    assert st["pending_injection"] == n_next
    assert t.check() == 0
    t.close()


# ---------------------------------------------------------------------------
# Batches of independent tubes
# ---------------------------------------------------------------------------

def _small_batch_params(precision=B.SCLF_FP32):
    """Five uneven tubes: flat and frame-dragging, Nz from 64 to 4096."""
    specs = [(1e12, 0.5, 0.5, 64, 3000), (3e11, 1.3, 0.0, 200, 9000),
             (2e12, 0.2, 0.5, 1024, 20000), (5e12, 2.0, 0.0, 333, 1000),
             (1e11, 0.05, 0.5, 4096, 12000)]
    out = []
    for i, (Bg, P, incl, nz, n) in enumerate(specs):
        kw = workloads.gr_tube(B_G=Bg, P_s=P, incl=incl, Nz=nz, n_particles=n,
                               capacity=n + 4096, track_ids=1, precision=precision)
        kw["rho_gj_mode"] = B.SCLF_RHO_GR if incl > 0 else B.SCLF_RHO_FLAT
        kw["compact_interval"] = 7
        out.append(kw)
    return out


def _fill(t, kw, seed):
    d = t.derived
    gfar = 3.0 * d["Lambda0"]
    z, u = synth.prefilled_beam(kw["target_particles"], d["L"] - d["dz"], gfar, seed=seed)
    t.add_particles(z, u)
    t.solve_fields()


@pytest.mark.parametrize("prec", [B.SCLF_FP32, B.SCLF_FIX32])
def test_batched_tubes_equal_tubes_stepped_alone_and_the_oracle(gpu_lib, prec):
    """A batch of five uneven tubes equals the same tubes stepped alone bit
    for bit, and two of them match the same-precision oracle step by step;
    with FIX32 positions (fractional bits 19 to 25 from the tubes' Nz) the
    batch has one kernel shape."""
    kws = _small_batch_params(prec)
    batch = B.Batch([B.default_params(**kw) for kw in kws])
    alone = [B.Tube(B.default_params(**kw)) for kw in kws]
    for i, kw in enumerate(kws):
        _fill(batch.tubes[i], kw, seed=i)
        _fill(alone[i], kw, seed=i)
    with pytest.raises(B.SclfError) as e:
        batch.tubes[0].step()
    assert e.value.code == -7                   # a batch member is stepped by its batch
    if prec == B.SCLF_FIX32:
        with pytest.raises(B.SclfError):
            batch.set_variant(1)
        chosen, ms = batch.autotune(2)
        assert chosen == 0 and ms[0] > 0 and all(m == -1.0 for m in ms[1:])
    else:
        batch.autotune(2)
    n_tune = 4 if prec == B.SCLF_FIX32 else 4 * 6
    batch.run(40)
    batch.step()
    batch.run(25)
    for t in alone:
        t.run(66 + n_tune)
    gathered = batch.status()                   # one gather for the whole batch
    assert len(gathered) == len(kws)
    for i in range(len(kws)):
        a, b = batch.tubes[i], alone[i]
        sa, sb = a.status(), b.status()
        assert gathered[i] == sa, i
        for k in ("step", "n_particles", "total_injected", "last_injected", "last_removed",
                  "pending_injection", "flags"):
            assert sa[k] == sb[k], (i, k)
        pa, pb = a.read_particles(), b.read_particles()
        for x, y in zip(pa, pb):
            assert np.array_equal(x, y), i
        fa, fb = a.read_fields(rho=False), b.read_fields(rho=False)
        for k in ("ez", "er", "b", "j"):
            assert np.array_equal(fa[k], fb[k]), (i, k)
    # and two of the tubes against the oracle, step by step
    batch2 = B.Batch([B.default_params(**kws[0]), B.default_params(**kws[3])])
    oracles = []
    for t, kw, seed in zip(batch2.tubes, (kws[0], kws[3]), (0, 3)):
        cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
        zn = np.arange(kw["Nz"] + 1) * (kw["L_over_R"] / kw["Nz"])
        mode = orc.RHO_GR if kw["rho_gj_mode"] == B.SCLF_RHO_GR else orc.RHO_FLAT
        rho = orc.rho_gj_profile(mode, zn, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                                 cu["R_over_Rstar"], cu["kappa"])
        d = t.derived
        o = orc.Tube(kw["Nz"], kw["L_over_R"], d["dt"], rho, d["s"],
                     precision="fix32" if prec == B.SCLF_FIX32 else "f32", accumulate="fixed")
        z, u = synth.prefilled_beam(kw["target_particles"], d["L"] - d["dz"], 3.0 * d["Lambda0"],
                                    seed=seed)
        t.add_particles(z, u)
        t.solve_fields()
        o.add_particles(z, u)
        o.solve_fields()
        oracles.append(o)
    for n in range(30):
        batch2.step()
        for t, o in zip(batch2.tubes, oracles):
            o.step()
            compare(t, o, TOL[B.SCLF_FP32], "batch step %d" % n)
    batch.close()
    batch2.close()
    for t in alone:
        t.close()


def _binned_profiles(z, u, ez, L, nb=32):
    """Mean gamma per height bin, E_z averaged over each bin's cells, and the
    particle count per bin."""
    edges = np.linspace(0.0, L, nb + 1)
    idx = np.clip(np.digitize(z, edges) - 1, 0, nb - 1)
    cnt = np.bincount(idx, minlength=nb)
    g = np.sqrt(1.0 + np.asarray(u, np.float64) ** 2)
    gm = np.bincount(idx, weights=g, minlength=nb) / np.maximum(cnt, 1)
    return gm, np.asarray(ez).reshape(nb, -1).mean(axis=1), cnt


def test_long_run_profiles_against_the_fp64_oracle(gpu_lib):
    """Config 1 (flat SCLF tube, empty start) for its full 2000 steps, with
    FP64 and with FP32 particles, against the FP64 oracle: the binned gamma(z)
    and E_z(z) profiles, the particle count per bin, and the first step where
    the injection counts part. Observed: FP64 never parts, profiles within
    ~1e-11 and E_z within 4e-10; FP32 parts at step 1161 with binned gamma
    6.7e-6, binned E_z 1.4e-5 and E_z 1.8e-4 -- the float32 oracle mirror's
    own figures, as it is bit-identical to the GPU run."""
    nsteps = 2000
    kw64 = workloads.flat_sclf_small(precision=B.SCLF_FP64, accumulate=B.SCLF_ACC_FIXED64)
    L, nz = kw64["L_over_R"], kw64["Nz"]
    d = B.derive(B.default_params(**kw64))
    o = orc.Tube(nz, L, d["dt"], -np.ones(nz + 1), d["s"], precision="f64", accumulate="fixed")
    inj_o = []
    for _ in range(nsteps):
        o.step()
        inj_o.append(o.last_injected)
    go, eo, co = _binned_profiles(o.z(), o.u, o.ez, L)
    occ = co > 0
    # (gamma bins, binned E_z, full E_z, per-bin count) bounds per precision
    tol = {B.SCLF_FP64: (1e-8, 1e-8, 1e-7, 0), B.SCLF_FP32: (1e-4, 1e-3, 1e-2, 0.01)}
    for prec in (B.SCLF_FP64, B.SCLF_FP32):
        t = B.Tube(B.default_params(**workloads.flat_sclf_small(
            precision=prec, accumulate=B.SCLF_ACC_FIXED64)))
        inj = []
        for _ in range(nsteps):
            t.step()
            inj.append(t.status()["last_injected"])
        z, u, _ = t.read_particles()
        f = t.read_fields(rho=False)
        g, e, c = _binned_profiles(z, u, f["ez"], L)
        part = np.nonzero(np.array(inj) != np.array(inj_o))[0]
        eg = float(np.max(np.abs(g[occ] - go[occ]) / go[occ]))
        ee = float(np.max(np.abs(e - eo)) / np.max(np.abs(eo)))
        ef = rel(f["ez"], o.ez)
        ec = float(np.max(np.abs(c - co))) / float(np.max(co))
        print("precision %d: injections part at step %s; gamma bins %.2g, E_z bins %.2g, "
              "E_z %.2g, counts %.2g" % (prec, part[0] if part.size else None, eg, ee, ef, ec))
        tg, te, tf, tc = tol[prec]
        assert eg <= tg and ee <= te and ef <= tf and ec <= tc
        assert np.array_equal(c > 0, occ)
        t.close()


def test_frame_dragging_grid_precision_against_the_fp64_oracle(gpu_lib):
    """The 1e8-particle frame-dragging tube's grid and time step (B = 1e12 G,
    P = 0.5 s, Nz = 65536, length 2 R_*) with 5e5 particles of the same
    seeded prefilled beam, 2000 steps, with FP64, float32 and 32-bit
    fixed-point (FIX32) positions, against the FP64 oracle: binned gamma(z)
    and E_z(z) (64 bins), E_z cell by cell and the particle count per bin.
    FP64 agrees to rounding. Float32 positions have a spacing of 2^-8 cell in
    the upper half of the tube, where an electron at v ~ c moves 0.0093 cell
    per step: the steps round to 0.0078 and the current there is ~16 % low;
    observed E_z error ~17 %. FIX32 (2^-15-cell spacing) has none of this:
    observed binned gamma 5e-5, binned E_z 7e-4, E_z 5e-3."""
    n, nsteps, nb = 500000, 2000, 64
    kw = workloads.gr_tube(n_particles=n, precision=B.SCLF_FP64,
                           accumulate=B.SCLF_ACC_FIXED64, track_ids=1)
    d = B.derive(B.default_params(**kw))
    L, nz = d["L"], kw["Nz"]
    gfar = d["Lambda0"] ** 2 * d["kappa"] * math.cos(kw["incl_rad"])
    z, u = synth.prefilled_beam(n, L - d["dz"], gfar, seed=0,
                                eta_of_z=lambda zz: 1.0 + zz * d["R_over_Rstar"])
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
    zn = np.arange(nz + 1) * (L / nz)
    rho = orc.rho_gj_profile(orc.RHO_GR, zn, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"])
    o = orc.Tube(nz, L, d["dt"], rho, d["s"], precision="f64", accumulate="fixed")
    o.add_particles(z, u)
    o.solve_fields()
    for _ in range(nsteps):
        o.step()
    go, eo, co = _binned_profiles(o.z(), o.u, o.ez, L, nb)
    occ = co > 0
    errs = {}
    for prec in (B.SCLF_FP64, B.SCLF_FP32, B.SCLF_FIX32):
        t = B.Tube(B.default_params(**dict(kw, precision=prec)))
        t.add_particles(z, u)
        t.solve_fields()
        t.run(nsteps)
        zz, uu, _ = t.read_particles()
        f = t.read_fields(rho=False)
        g, e, c = _binned_profiles(zz, uu, f["ez"], L, nb)
        errs[prec] = (float(np.max(np.abs(g[occ] - go[occ]) / go[occ])),
                      float(np.max(np.abs(e - eo)) / np.max(np.abs(eo))), rel(f["ez"], o.ez),
                      float(np.max(np.abs(c - co))) / float(np.max(co)))
        assert t.status()["total_injected"] == o.total_injected
        print("precision %d against the FP64 oracle: gamma bins %.2g, E_z bins %.2g, E_z %.2g, "
              "counts %.2g" % ((prec,) + errs[prec]))
        t.close()
    assert max(errs[B.SCLF_FP64][:3]) < 1e-10 and errs[B.SCLF_FP64][3] == 0
    eg, eb, ef, ec = errs[B.SCLF_FIX32]
    assert eg < 2e-4 and eb < 3e-3 and ef < 2e-2 and ec < 1e-3
    # the float32 bias is real and FIX32 removes it
    assert errs[B.SCLF_FP32][1] > 0.05 and errs[B.SCLF_FP32][1] > 20 * eb


@pytest.mark.parametrize("variant,alpha,tables", [(B.SCLF_GR_BOTH, 0, False),
                                                  (B.SCLF_GR_COS, 1, True)])
def test_eq6_variant_tube_matches_oracle(gpu_lib, variant, alpha, tables):
    """A frame-dragging tube built with an Eq. 6 variant (Omega -> Omega - omega
    on both terms; redshift alpha with f, H tables): initial fields, injection
    counts and 50 FP64 steps with a prefilled beam against the oracle."""
    kw = workloads.gr_tube(B_G=1e12, P_s=0.3, Nz=2048, n_particles=20000,
                           precision=B.SCLF_FP64, accumulate=B.SCLF_ACC_FIXED64, track_ids=1)
    nz, L = kw["Nz"], kw["L_over_R"]
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
    z = np.arange(nz + 1) * (L / nz)
    eta = 1.0 + z * cu["R_over_Rstar"]
    f = 1.0 + 0.2 * (1.0 - 1.0 / eta) if tables else None
    H = 1.0 - 0.1 * (1.0 - 1.0 / eta) if tables else None
    t = B.Tube(B.default_params(**kw, gr_variant=variant, gr_alpha=alpha, gr_f=f, gr_H=H))
    d = t.derived
    rho = orc.rho_gj_profile(orc.RHO_GR, z, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"],
                             variant="both" if variant == B.SCLF_GR_BOTH else "cos", f=f, H=H,
                             rg_over_Rstar=cu["rg_over_Rstar"] if alpha else None)
    o = orc.Tube(nz, L, d["dt"], rho, d["s"], precision="f64", accumulate="fixed")
    fl = t.read_fields(rho=False)
    assert rel(fl["ez"], o.ez) < 1e-11 and rel(fl["er"], o.er) < 1e-11
    zp, up = synth.prefilled_beam(20000, L - L / nz, 1e3, seed=4)
    t.add_particles(zp, up)
    t.solve_fields()
    o.add_particles(zp, up)
    o.solve_fields()
    for n in range(50):
        t.step()
        o.step()
        compare(t, o, TOL[B.SCLF_FP64], "variant step %d" % n)
    assert o.xi.size >= 19000
    t.close()


def _batch_state(batch):
    out = []
    for t in batch.tubes:
        st = t.status()
        out.append((st["step"], st["n_particles"], st["total_injected"], st["pending_injection"],
                    t.read_particles(), t.read_fields(rho=False)))
    return out


def _same_state(sa, sb):
    for a, b in zip(sa, sb):
        assert a[:4] == b[:4]
        for x, y in zip(a[4], b[4]):
            assert np.array_equal(x, y)
        for k in ("ez", "er", "b", "j"):
            assert np.array_equal(a[5][k], b[5][k]), k


@pytest.mark.parametrize("prec", [B.SCLF_FIX32, B.SCLF_FP32])
def test_full_size_batch_against_oracle_on_sampled_tubes(gpu_lib, prec):
    """The 256-tube death-line batch at its benchmark size and launch
    configuration (seeded states, autotuned particle-kernel shape; the
    tuning steps are ordinary steps): after the tuning steps and one more,
    five sampled tubes (flat and frame-dragging, the smallest and largest
    grids) against the oracle run from the same seeded states, with FIX32
    (the benchmark's) and float32 positions."""
    kws = workloads.death_line_batch(precision=prec)
    batch = B.Batch([B.default_params(**kw) for kw in kws])
    nzs = [kw["Nz"] for kw in kws]
    sample = sorted({0, 1, int(np.argmin(nzs)), int(np.argmax(nzs)), len(kws) - 1})
    states = {}
    for i, kw in enumerate(kws):
        t = batch.tubes[i]
        d = t.derived
        gr = kw["rho_gj_mode"] == B.SCLF_RHO_GR
        gfar = (d["Lambda0"] ** 2 * d["kappa"] * math.cos(kw["incl_rad"]) if gr
                else math.sqrt(2.0) * d["Lambda0"])
        eta = (lambda zz, r=d["R_over_Rstar"]: 1.0 + zz * r) if gr else None
        z, u = synth.prefilled_beam(kw["target_particles"], d["L"] - d["dz"], gfar, seed=i,
                                    eta_of_z=eta)
        t.add_particles(z, u)
        t.solve_fields()
        if i in sample:
            states[i] = (z, u)
    chosen, ms = batch.autotune(1)
    batch.step()
    nsteps = batch.tubes[0].status()["step"]
    shapes = 1 if prec == B.SCLF_FIX32 else len(B.Batch.VARIANTS)
    assert nsteps == shapes * 3 + 1
    for i in sample:
        kw, t = kws[i], batch.tubes[i]
        d = t.derived
        cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
        mode = orc.RHO_GR if kw["rho_gj_mode"] == B.SCLF_RHO_GR else orc.RHO_FLAT
        rho = orc.rho_gj_profile(mode, np.arange(kw["Nz"] + 1) * d["dz"], cu["Lambda0"],
                                 kw["incl_rad"], cu["theta_star"], cu["R_over_Rstar"], cu["kappa"])
        fix = prec == B.SCLF_FIX32
        o = orc.Tube(kw["Nz"], d["L"], d["dt"], rho, d["s"], precision="fix32" if fix else "f32",
                     accumulate="fixed")
        o.add_particles(*states[i])
        o.solve_fields()
        o.run(nsteps)
        _state_against_oracle(t, o, 2.0 ** orc.fix32_bits(kw["Nz"]) if fix else 1.0,
                              "tube %d (Nz %d, shape %s)" % (i, kw["Nz"], B.Batch.VARIANTS[chosen]))
    assert max(t.check() for t in batch.tubes) == 0
    batch.close()


def test_large_batch_descriptor_kernel_equals_parameter_table_kernel(gpu_lib):
    """Batches of more tubes than the particle kernel's parameter table holds
    read every tube's constants from the device descriptors instead: a
    401-tube batch advances its first five tubes bit for bit as a five-tube
    batch does."""
    small = _small_batch_params()
    kws = [small[i % len(small)] for i in range(401)]
    big = B.Batch([B.default_params(**kw) for kw in kws])
    few = B.Batch([B.default_params(**kw) for kw in small])
    for i, kw in enumerate(small):
        _fill(big.tubes[i], kw, seed=30 + i)
        _fill(few.tubes[i], kw, seed=30 + i)
    for v in (0, 3):                              # one and two runs per thread
        big.set_variant(v)
        few.set_variant(v)
        big.run(35)
        few.run(35)
    sb, sf = big.status(), few.status()
    for i in range(len(small)):
        assert sb[i] == sf[i], i
        pa, pb = big.tubes[i].read_particles(), few.tubes[i].read_particles()
        for x, y in zip(pa, pb):
            assert np.array_equal(x, y), i
        fa, fb = big.tubes[i].read_fields(rho=False), few.tubes[i].read_fields(rho=False)
        for k in ("ez", "er", "b", "j"):
            assert np.array_equal(fa[k], fb[k]), (i, k)
    big.close()
    few.close()


def test_batch_members_survive_a_save_and_load_round_trip(gpu_lib):
    """Saving every tube of a batch to host memory and loading it back (the
    end-to-end path: tube_save_particles, tube_load_particles on batch
    members) changes nothing the batch computes afterwards: fields bit for
    bit, live particles in slot order, injection counts."""
    kws = _small_batch_params()
    a = B.Batch([B.default_params(**kw) for kw in kws])
    b = B.Batch([B.default_params(**kw) for kw in kws])
    for bb in (a, b):
        for i, kw in enumerate(kws):
            _fill(bb.tubes[i], kw, seed=10 + i)
        bb.run(20)
    for t in a.tubes:
        xi, u, _ = t.save_particles()
        t.load_particles(xi, u)
    a.run(75)
    b.run(75)
    sa, sb = a.status(), b.status()
    for i in range(len(kws)):
        for k in ("step", "n_particles", "last_injected", "last_removed", "pending_injection",
                  "surface_field", "flags"):
            assert sa[i][k] == sb[i][k], (i, k)
        pa, pb = a.tubes[i].read_particles(), b.tubes[i].read_particles()
        for x, y in zip(pa[:2], pb[:2]):
            assert np.array_equal(x, y), i
        fa, fb = a.tubes[i].read_fields(rho=False), b.tubes[i].read_fields(rho=False)
        for k in ("ez", "er", "b", "j"):
            assert np.array_equal(fa[k], fb[k]), (i, k)
    a.close()
    b.close()


def test_batch_kernel_shapes_agree_bit_for_bit_and_autotune_keeps_one(gpu_lib):
    """Every shape of the batched particle kernel (particles per thread, CTAs
    per SM) advances a batch to the same state bit for bit; the autotuner
    keeps one of them and the tuned batch equals an untuned one stepped as
    many times."""
    kws = _small_batch_params()
    batches = []
    for v in range(len(B.Batch.VARIANTS)):
        b = B.Batch([B.default_params(**kw) for kw in kws])
        for i, kw in enumerate(kws):
            _fill(b.tubes[i], kw, seed=i)
        b.set_variant(v)
        b.run(70)                      # one 64-step graph (with a compaction check) and single steps
        batches.append(b)
    ref = _batch_state(batches[0])
    for b in batches[1:]:
        _same_state(_batch_state(b), ref)
    tuned, plain = batches[0], batches[1]
    chosen, ms = tuned.autotune(3)
    assert 0 <= chosen < len(B.Batch.VARIANTS) and np.all(ms > 0) and ms[chosen] == ms.min()
    plain.run(len(B.Batch.VARIANTS) * 5)
    tuned.run(10)
    plain.run(10)
    _same_state(_batch_state(tuned), _batch_state(plain))
    for b in batches:
        b.close()


@pytest.mark.parametrize("prec", [B.SCLF_FP32, B.SCLF_FP64, B.SCLF_FIX32])
def test_push_stages_change_no_result(gpu_lib, prec):
    """The particle kernel with its slots loaded straight into registers
    (push_stages 1) and streamed through a ring of 2, 3 or 4 shared-memory
    stages by bulk asynchronous copies gives the same run bit for bit. The
    tube holds enough tiles that every CTA refills its ring several times,
    with a ragged tail and injection every step; no wait gives up. (The
    fields start from the empty tube's: the Eq. 4 solve with the particles'
    charge sums FP64 atomics, whose order is not fixed.)"""
    kw = workloads.flat_sclf_small(precision=prec, accumulate=B.SCLF_ACC_FIXED64,
                                   capacity=1 << 23)
    z, u = synth.random_particles(6 * 10 ** 6 + 1234, kw["L_over_R"], seed=11, u_sigma=2.0)
    ref = None
    for stages in (1, 2, 3, 4):
        t = B.Tube(B.default_params(**kw, push_stages=stages))
        t.add_particles(z, u)
        t.run(12)
        st = t.status()
        assert st["flags"] == 0, (stages, st["flags"])
        got = (st, t.read_particles(), t.read_fields(rho=False))
        t.close()
        if ref is None:
            ref = got
            continue
        for k in ("n_particles", "n_slots", "total_injected", "last_removed",
                  "pending_injection"):
            assert got[0][k] == ref[0][k], (stages, k)
        for a, b in zip(got[1], ref[1]):
            assert np.array_equal(a, b), stages
        for k in ("ez", "er", "b", "j"):
            assert np.array_equal(got[2][k], ref[2][k]), (stages, k)


def _run_state(t):
    st = t.status()
    return st, t.read_particles(), t.read_fields(rho=False)


def _same_run_state(a, b, what):
    for k in ("step", "n_particles", "n_slots", "total_injected", "last_removed",
              "pending_injection", "flags"):
        assert a[0][k] == b[0][k], (what, k)
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y), what
    for k in ("ez", "er", "b", "j"):
        assert np.array_equal(a[2][k], b[2][k]), (what, k)


@pytest.mark.parametrize("prec", [B.SCLF_FP32, B.SCLF_FP64, B.SCLF_FIX32])
def test_launch_overlap_changes_no_result(gpu_lib, prec):
    """The step kernels launched with programmatic dependent launch (each
    scheduled while the one before it finishes, waiting for it on the device
    before its first memory access) give the same run bit for bit as plain
    stream order: stepped one call at a time, in captured graphs with their
    compaction checks, and in the timed graphs, whose event nodes sit between
    the kernels. Injection every step, removals at both ends, a ragged last
    tile."""
    kw = workloads.flat_sclf_small(precision=prec, accumulate=B.SCLF_ACC_FIXED64,
                                   capacity=1 << 22)
    z, u = synth.random_particles(2 * 10 ** 6 + 77, kw["L_over_R"], seed=12, u_sigma=2.0)
    got = {}
    for ov in (-1, 1):
        t = B.Tube(B.default_params(**kw, launch_overlap=ov))
        t.add_particles(z, u)
        for _ in range(5):
            t.step()
        t.run(130)
        t.set_timing(True)
        t.run(64)
        t.set_timing(False)
        got[ov] = _run_state(t)
        assert got[ov][0]["flags"] == 0, ov
        assert got[ov][0]["last_removed"] > 0, ov
        t.close()
    _same_run_state(got[-1], got[1], prec)


@pytest.mark.parametrize("prec", [B.SCLF_FIX32, B.SCLF_FP32])
def test_batch_launch_overlap_changes_no_result(gpu_lib, prec):
    """A batch's refresh, particle and field kernels by programmatic dependent
    launch equal the same batch in plain stream order, bit for bit, over
    graph chunks and single steps."""
    kws = _small_batch_params(prec)
    states = {}
    for ov in (-1, 1):
        batch = B.Batch([B.default_params(**kw, launch_overlap=ov) for kw in kws])
        for i, kw in enumerate(kws):
            _fill(batch.tubes[i], kw, seed=i)
        batch.run(70)
        batch.step()
        states[ov] = _batch_state(batch)
        batch.close()
    _same_state(states[-1], states[1])


def test_sampled_timing_counts_the_run_and_keeps_its_results(gpu_lib):
    """tube_set_timing(3) times every third unit of work (a step launched on
    its own, or a 64-step graph replay); steps_run and compactions_run count
    every step and compaction check, and the run equals an untimed one bit
    for bit. batch_set_timing(2) times every second step and lets the others
    replay the graph. The counts follow from the schedules (graph replays
    start at an even step right after a compaction check)."""
    kw = workloads.flat_sclf_small(precision=B.SCLF_FIX32, accumulate=B.SCLF_ACC_FIXED64,
                                   capacity=1 << 21)
    z, u = synth.random_particles(5 * 10 ** 5 + 3, kw["L_over_R"], seed=13, u_sigma=2.0)
    a, b = (B.Tube(B.default_params(**kw)) for _ in range(2))
    for t in (a, b):
        t.add_particles(z, u)
        t.run(10)
    a.set_timing(3)
    a.run(300)              # 54 single steps, 3 graph replays, 54 single steps
    tm = a.timing()
    a.set_timing(0)
    b.run(300)
    _same_run_state(_run_state(a), _run_state(b), "sampled timing")
    assert tm["steps_run"] == 300 and tm["compactions_run"] == 4
    assert tm["n_steps"] == 18 + 64 + 18 and tm["n_compactions"] == 2
    assert tm["push_ms"] > 0 and tm["field_ms"] > 0
    n = a.status()["n_slots"]
    assert 0.8 * 300 * n < tm["particle_slots"] < 1.25 * 300 * n
    a.close()
    b.close()

    kws = _small_batch_params(B.SCLF_FIX32)
    ba, bb = (B.Batch([B.default_params(**kw) for kw in kws]) for _ in range(2))
    for batch in (ba, bb):
        for i, kw in enumerate(kws):
            _fill(batch.tubes[i], kw, seed=i)
        batch.run(10)
    # compaction checks every 7 steps, graph replays of 8: the 10 warm-up
    # steps are a replay and 2 single steps; then 5 single steps (units 0-4,
    # a check after the last), one more to reach an even step (unit 5), 6
    # (units 6-11, a check), 17 replays (units 12-147) and 2 single steps
    # (units 148-149); every second unit is timed
    ba.set_timing(2)
    ba.run(150)
    tb = ba.timing()
    ba.set_timing(0)
    bb.run(150)
    _same_state(_batch_state(ba), _batch_state(bb))
    assert tb["steps_run"] == 150 and tb["compactions_run"] == 2 + 17
    assert tb["n_steps"] == 3 + 3 + 1 and tb["n_compactions"] == 2
    ba.close()
    bb.close()


@pytest.mark.parametrize("prec", [B.SCLF_FP32, B.SCLF_FIX32])
def test_sort_by_cell_changes_no_result(gpu_lib, prec):
    """A shuffled beam stepped with a stable re-sort by cell every 10 steps
    (tube_run's sort_interval) gives the same fields bit for bit and the same
    particles (compared by ID) as without; right after tube_sort the slots are
    in cell order and the holes are gone."""
    kw = workloads.flat_sclf_small(precision=prec, accumulate=B.SCLF_ACC_FIXED64)
    a = B.Tube(B.default_params(**kw))
    b = B.Tube(B.default_params(**kw, sort_interval=10))
    z, u = synth.prefilled_beam(40000, 8.0 - 8.0 / 1024, 5.0, seed=6, order="shuffled")
    for t in (a, b):
        t.add_particles(z, u)
        t.solve_fields()
        t.run(95)
    sa, sb = a.status(), b.status()
    for k in ("n_particles", "total_injected", "pending_injection", "last_removed", "flags"):
        assert sa[k] == sb[k], k
    fa, fb = a.read_fields(rho=False), b.read_fields(rho=False)
    for k in ("ez", "er", "b", "j"):
        assert np.array_equal(fa[k], fb[k]), k
    za, ua, ia = a.read_particles()
    zb, ub, ib = b.read_particles()
    oa, ob = np.argsort(ia), np.argsort(ib)
    assert np.array_equal(ia[oa], ib[ob])
    assert np.array_equal(za[oa], zb[ob]) and np.array_equal(ua[oa], ub[ob])
    assert sb["n_slots"] < sb["n_particles"] + 40000      # holes were dropped on the way
    b.sort()
    xs, _, ids = b.save_particles()
    cells = np.floor(xs.astype(np.float64) * b.derived["pos_unit"])
    assert np.all(np.diff(cells) >= 0) and b.status()["n_slots"] == b.status()["n_particles"]
    assert np.array_equal(np.sort(ids), np.sort(ia))
    a.close()
    b.close()


def _same_run(whole, dt, what):
    """Fields bit for bit, particles bit for bit by ID, and the counters."""
    sw, sd = whole.status(), dt.status()
    for k in ("step", "n_particles", "total_injected", "last_injected", "pending_injection",
              "flags"):
        assert sw[k] == sd[k], (what, k, sw[k], sd[k])
    fw = whole.read_fields(rho=False)
    fd = dt.read_fields()
    for k in ("ez", "er", "b", "j"):
        assert np.array_equal(fw[k], fd[k]), (what, k)
    zw, uw, iw = whole.read_particles()
    o = np.argsort(iw, kind="stable")
    zd, ud, idd = dt.read_particles()
    assert np.array_equal(iw[o], idd), what
    assert np.array_equal(zw[o], zd) and np.array_equal(uw[o], ud), what


@pytest.mark.parametrize("prec,cuts", [(B.SCLF_FP64, [0, 100, 333, 1024]),
                                       (B.SCLF_FP32, [0, 100, 333, 700, 1024]),
                                       (B.SCLF_FIX32, [0, 2, 512, 1022, 1024])])
def test_decomposed_flat_tube_equals_the_whole_tube(gpu_lib, prec, cuts):
    """Config 1 (flat tube, empty start, injection) split into 3 or 4 z-ranges
    (sub-domains with their own slots, streams and grid copies, exchanging
    the boundary current, B_phi and E_z halos and the crossing particles each
    step) gives the same fields bit for bit, the same particles by ID and the
    same counters as the whole tube, checked every 150 steps up to 600 while
    the electron front passes the cuts (FIX32 also with 2-cell sub-domains at
    both ends)."""
    kw = workloads.flat_sclf_small(precision=prec, accumulate=B.SCLF_ACC_FIXED64)
    whole = B.Tube(B.default_params(**kw))
    dt = B.DTube(B.default_params(**kw), cuts=cuts)
    for n in range(4):
        whole.run(150)
        dt.run(150)
        _same_run(whole, dt, "step %d" % (150 * (n + 1)))
    ex = dt.exchange_stats()
    ts = 8 if prec == B.SCLF_FP64 else 4
    assert ex["steps"] == 600
    assert ex["field_bytes"] == 600 * (len(cuts) - 2) * (16 + 16 + 2 * ts)
    assert ex["particles"] > 0
    assert ex["particle_bytes"] == ex["particles"] * (2 * ts + 8)
    whole.close()
    dt.close()


@pytest.mark.parametrize("prec", [B.SCLF_FIX32, B.SCLF_FP32])
def test_decomposed_frame_dragging_tube_equals_the_whole_tube(gpu_lib, prec):
    """The 1e8-particle tube's grid (Nz = 65536) prefilled with 5e5 particles,
    fields from Eq. 4 with their charge, split into 4 uneven sub-domains:
    300 steps give the same fields, particles and counters as the whole tube
    (at ~8 particles per cell moving 0.0093 cell per step, about one particle
    crosses a cut every 14 steps: ~60 hand-overs in all)."""
    n = 500000
    kw = workloads.gr_tube(n_particles=n, precision=prec, accumulate=B.SCLF_ACC_FIXED64,
                           track_ids=1)
    whole = B.Tube(B.default_params(**kw))
    d = whole.derived
    gfar = d["Lambda0"] ** 2 * d["kappa"] * math.cos(kw["incl_rad"])
    z, u = synth.prefilled_beam(n, d["L"] - d["dz"], gfar, seed=4,
                                eta_of_z=lambda zz: 1.0 + zz * d["R_over_Rstar"])
    whole.add_particles(z, u)
    whole.solve_fields()
    f0 = whole.read_fields(rho=False)
    dt = B.DTube(B.default_params(**kw), cuts=[0, 9000, 30001, 47000, 65536])
    dt.load_particles(z, u)
    dt.set_fields(f0["ez"], f0["er"], f0["b"])
    _same_run(whole, dt, "start")
    for k in range(3):
        whole.run(100)
        dt.run(100)
        _same_run(whole, dt, "step %d" % (100 * (k + 1)))
    assert dt.exchange_stats()["particles"] > 30
    whole.close()
    dt.close()


@pytest.mark.parametrize("n", [1, 16])
def test_decomposed_tube_with_one_and_sixteen_equal_subdomains(gpu_lib, n):
    """The degenerate split (one sub-domain: no exchange) and 16 equal
    sub-domains of 64 cells on config 1 with a prefilled random beam equal the
    whole tube bit for bit after 300 steps; loading particles into a tube
    that has stepped is refused; the decomposed Eq. 4 solve (density summed
    over the sub-domains) agrees with the whole tube's to rounding."""
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64)
    z, u = synth.random_particles(30000, kw["L_over_R"] * 0.999, seed=21, u_sigma=3.0)
    whole = B.Tube(B.default_params(**kw))
    whole.add_particles(z, u)
    whole.solve_fields()
    f0 = whole.read_fields(rho=False)
    dt = B.DTube(B.default_params(**kw), n=n)
    dt.load_particles(z, u)
    dt.solve_fields()
    fs = dt.read_fields()
    assert rel(fs["ez"], f0["ez"]) < 1e-12 and rel(fs["er"], f0["er"]) < 1e-12
    dt.set_fields(f0["ez"], f0["er"], f0["b"])
    whole.run(300)
    dt.run(300)
    _same_run(whole, dt, "%d sub-domains" % n)
    ex = dt.exchange_stats()
    assert ex["field_bytes"] == 300 * (n - 1) * (16 + 16 + 8)
    assert (ex["particles"] > 0) == (n > 1)
    with pytest.raises(B.SclfError) as e:
        dt.load_particles(z[:10], u[:10])
    assert e.value.code == -7
    whole.close()
    dt.close()


def test_diagnostics_match_the_oracle(gpu_lib):
    """tube_diagnostics (gamma max and mean, kinetic and field energy, Gauss
    residual) against the same quantities from the oracle's state after 150
    FP64 steps of the flat SCLF tube (to 1e-10: the two FP64 runs start from
    Eq. 4 solutions that differ in the last bits -- a Thomas sweep and LAPACK's
    banded solver -- and 150 steps amplify that to ~1e-11); the Gauss residual
    stays at rounding level (charge conservation of the step)."""
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP64, accumulate=B.SCLF_ACC_FIXED64)
    t, o = pair(gpu_lib, kw, "f64", "fixed")
    for _ in range(150):
        t.step()
        o.step()
    dg = t.diagnostics()
    g = o.gamma()
    assert dg["n_particles"] == o.xi.size
    assert abs(dg["gamma_max"] - g.max()) <= 1e-10 * g.max()
    assert abs(dg["gamma_mean"] - g.mean()) <= 1e-10 * g.mean()
    assert abs(dg["kinetic"] - abs(o.s) * np.sum(g - 1.0)) <= 1e-10 * abs(o.s) * np.sum(g - 1.0)
    w = np.ones(o.nz + 1)
    w[0] = w[-1] = 0.5
    fe = (np.sum(o.ez ** 2 + o.b ** 2) * o.dz + np.sum(w * o.er ** 2) * o.dz) / (8 * math.pi)
    assert abs(dg["field_energy"] - fe) <= 1e-10 * fe
    res = o.gauss_residual()
    assert dg["gauss_max"] <= 1e-9 * dg["gauss_scale"]
    assert abs(dg["gauss_max"] - np.max(np.abs(res))) <= 1e-9 * dg["gauss_scale"]
    t.close()


def test_bounds_checked_build_flags_nothing_and_changes_nothing(gpu_lib, tmp_path):
    """The bounds-checked build (every data-dependent index in the particle,
    batch and adjoint kernels tested before the access) runs the edge-heavy
    cases of tests/checked_worker.py -- particles on cell and tube
    boundaries, at rest and at gamma ~ 1e7 in both directions, compaction,
    re-sorts, both batch run shapes, the float32 and fixed-point adjoint --
    without setting SCLF_FLAG_BOUNDS, and gives the results the normal build
    gives: counts, IDs and flags exactly, floating-point results norm-wise
    to 1e-6 (the charge density behind each prefilled tube's initial Eq. 4
    solve and the adjoint's lambda_E are summed by FP64 atomics, whose order
    differs between any two runs)."""
    import os
    import subprocess
    import sys
    if not os.path.exists(B.LIB_CHECKED_PATH):
        from paper_1011_6330_gb300 import build
        build.build(checked=True)
    worker = os.path.join(os.path.dirname(os.path.abspath(__file__)), "checked_worker.py")
    res = {}
    for name, lib in (("plain", B.LIB_PATH), ("checked", B.LIB_CHECKED_PATH)):
        out = tmp_path / (name + ".npz")
        r = subprocess.run([sys.executable, worker, str(out)], capture_output=True, text=True,
                           env=dict(os.environ, SCLF_TUBE_LIB=lib), timeout=900)
        assert r.returncode == 0, r.stderr[-3000:]
        res[name] = np.load(out)
    plain, checked = res["plain"], res["checked"]
    assert "bounds-checked" in str(checked["version"])
    assert "bounds-checked" not in str(plain["version"])
    assert set(plain.files) == set(checked.files)
    n_flags = n_same = 0
    for k in plain.files:
        if k == "version":
            continue
        if k.endswith("_flags"):
            n_flags += 1
            assert int(checked[k][0]) & B.FLAG_BOUNDS == 0, k
        if k.endswith(("_ids", "_counts", "_flags")):
            assert np.array_equal(plain[k], checked[k]), k
        else:
            a, c = plain[k].astype(np.float64), checked[k].astype(np.float64)
            assert a.shape == c.shape and rel(c, a) < 1e-6, k
        n_same += int(np.array_equal(plain[k], checked[k]))
    print("%d of %d results bit for bit" % (n_same, len(plain.files) - 1))
    assert n_flags == 9


def test_bounded_wait_gives_up_and_the_context_stays_usable(gpu_lib):
    """The compaction look-back's wait is bounded: with the first tile's state
    withheld (a flag nothing sets) the second tile gives up, the device reports
    SCLF_ETIMEOUT through the sticky flags, and the CUDA context keeps
    working -- a fresh tube then steps exactly like the oracle."""
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64)
    t = B.Tube(B.default_params(**kw))
    assert t.lib.tube_selftest_wait_timeout(t.h) == -1      # one tile: nothing to wait for
    z, u = synth.prefilled_beam(10000, 7.9, 5.0, seed=8)
    t.add_particles(z, u)
    assert t.lib.tube_selftest_wait_timeout(t.h) == -6      # SCLF_ETIMEOUT
    assert t.status()["flags"] & B.FLAG_TIMEOUT
    assert t.check() == -6
    t.close()
    t2, o = pair(gpu_lib, kw, "f32", "fixed")
    for n in range(20):
        t2.step()
        o.step()
        compare(t2, o, TOL[B.SCLF_FP32], "after the timeout, step %d" % n)
    assert t2.check() == 0
    t2.close()


def test_velocity_routine_equals_ieee_sequence_on_every_float32(gpu_lib):
    """The particle kernels' float32 velocity u / sqrt(1 + u^2) (Newton step
    on the hardware reciprocal square root, Markstein's FMA division) equals
    the correctly rounded sequence RN(u / RN(sqrt(RN(1 + RN(u u))))) bit for
    bit on all 2^32 float32 inputs, so the float32 results stay those of the
    float32 oracle."""
    n = C.c_uint64()
    first = C.c_uint32()
    assert gpu_lib.tube_selftest_velocity(0, 1 << 32, C.byref(n), C.byref(first)) == 0
    assert n.value == 0, (n.value, hex(first.value))
