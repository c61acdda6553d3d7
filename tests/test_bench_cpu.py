"""The benchmark's reference arm (the oracle on the host cores) runs without a
GPU: its JSON line carries the contract's keys, the GPU arm's metric, unit and
workload name, and a cpu_baseline describing the run."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--particles", "2e6"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["workload"] == bench.gr_workload_name(2e6)
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert cb["host"]["nproc"] >= 1 and d["dtype"] == "fix32+f32"
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_all_core_baseline_computes_the_one_process_oracle_fields():
    """The all-core CPU baseline (the oracle's particle step split over
    spawned processes, integer current sums added in a fixed order) gives the
    one-process oracle's E_z bit for bit after the same steps."""
    sys.path.insert(0, ROOT)
    import math
    import numpy as np
    import bench
    import oracle as orc
    from paper_1011_6330_gb300 import binding as B
    from paper_1011_6330_gb300 import synth, workloads
    n, nsteps = 20000, 12
    kw = workloads.gr_tube(n_particles=n, Nz=512, precision=B.SCLF_FIX32)
    d = B.derive(B.default_params(**kw))
    gfar = d["Lambda0"] ** 2 * d["kappa"] * math.cos(kw["incl_rad"])
    z, u = synth.prefilled_beam(n, d["L"] - d["dz"], gfar, seed=3,
                                eta_of_z=lambda zz: 1.0 + zz * d["R_over_Rstar"])
    res = bench.cpu_baseline_allcore(z, u, n, kw, d, 0.0, 1, workers=3, nsteps=nsteps)
    assert res["cores"] == 3 and res["value"] > 0
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
    zn = np.arange(kw["Nz"] + 1) * (d["L"] / kw["Nz"])
    rho = orc.rho_gj_profile(orc.RHO_GR, zn, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"])
    o = orc.Tube(kw["Nz"], d["L"], d["dt"], rho, d["s"], precision="fix32", accumulate="fixed")
    o.add_particles(z, u)
    o.solve_fields()
    o.run(nsteps + 1)                                  # the baseline's warm-up step too
    assert np.array_equal(res["final_ez"], o.ez)
