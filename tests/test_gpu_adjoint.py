"""GPU discrete adjoint (adjoint_* of the C ABI) against the oracle's FP64
adjoint, against central differences of the GPU's own forward run, and
through the torch.autograd wrapper.

Events (injections per step, removals per step) must match the oracle
exactly. Gradients are compared norm-wise, max|g - g_ref| / max|g_ref|:
<= 1e-9 with FP64 particles (same trajectory to rounding, sums in another
order), <= 1e-6 with FP32 particles (the oracle reverses the same float32
trajectory in FP64; the GPU keeps the particle adjoints in float32).
"""

import math

import numpy as np
import pytest

import oracle as orc
from oracle import adjoint as oadj
from paper_1011_6330_gb300 import binding as B
from paper_1011_6330_gb300 import synth, workloads

pytestmark = pytest.mark.gpu

TOL = {B.SCLF_FP64: 1e-9, B.SCLF_FP32: 1e-6, B.SCLF_FIX32: 1e-6}
OPREC = {B.SCLF_FP64: "f64", B.SCLF_FP32: "f32", B.SCLF_FIX32: "fix32"}
M_STAR = 1.4 * orc.M_SUN


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / float(np.max(np.abs(b)))


def flat_problem(prec, n=20000, nsteps=60, K=10):
    kw = workloads.flat_sclf_small(precision=prec, accumulate=B.SCLF_ACC_FIXED64)
    L, nz = kw["L_over_R"], kw["Nz"]
    z, u = synth.prefilled_beam(n, 0.9 * L, 5.0, seed=7)
    return kw, z, u, nsteps, K


def gr_problem(prec, n=50000, nsteps=100, K=10, Nz=1024):
    kw = workloads.gr_tube(B_G=1e12, P_s=0.3, Nz=Nz, n_particles=n, precision=prec,
                           accumulate=B.SCLF_ACC_FIXED64)
    d = B.derive(B.default_params(**kw))
    kw.update(dt=d["dt"], R_cm=d["R_cm"])
    L = kw["L_over_R"]
    z, u = synth.prefilled_beam(n, L - L / Nz, 1e3, seed=9)
    return kw, z, u, nsteps, K


def gpu_run(kw, z, u, nsteps, K, injections=None):
    a = B.Adjoint(B.default_params(**kw), nsteps, K)
    if z is not None and len(z):
        a.tube.add_particles(z, u)
    if injections is not None:
        a.set_injections(injections)
    vals = a.forward()
    return a, vals


def oracle_run(kw, z, u, prec):
    d = B.derive(B.default_params(**kw))
    nz, L = kw["Nz"], kw["L_over_R"]
    if kw.get("rho_gj_mode") == B.SCLF_RHO_USER:
        rho = np.asarray(kw["rho_gj_user"], np.float64)
    else:
        cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"],
                            kw.get("R_cm", 0.0))
        zz = np.arange(nz + 1) * (L / nz)
        rho = orc.rho_gj_profile(kw["rho_gj_mode"], zz, cu["Lambda0"], kw["incl_rad"],
                                 cu["theta_star"], cu["R_over_Rstar"], cu["kappa"])
    return oadj.AdjointRun(nz, L, d["dt"], rho, d["s"], z, u, precision=OPREC[prec],
                           accumulate="fixed")


@pytest.mark.parametrize("prec", [B.SCLF_FP64, B.SCLF_FP32, B.SCLF_FIX32])
def test_adjoint_matches_oracle_flat_tube(gpu_lib, prec):
    """Flat SCLF tube (Nz = 1024, rho_GJ = -1), 2e4 prefilled electrons plus
    injection, 60 steps in 6 checkpointed segments; FP64, FP32 and 32-bit
    fixed-point particles."""
    kw, z, u, nsteps, K = flat_problem(prec)
    a, vals = gpu_run(kw, z, u, nsteps, K)
    run = oracle_run(kw, z, u, prec)
    ev = a.events()
    for i, which in enumerate(("gamma", "ez")):
        v, d_rho, d_s, inj, rem = run.gradient(which, nsteps)
        assert np.array_equal(ev["injected"], inj)
        assert np.array_equal(ev["removed"], [len(r) for r in rem])
        assert abs(vals[i] - v) <= 1e-12 * abs(v) + (1e-6 * abs(v) if prec != B.SCLF_FP64 and i == 1 else 0)
        g_rho, g_s = a.backward(i)
        e_rho, e_s = rel(g_rho, d_rho), abs(g_s - d_s) / abs(d_s)
        print(which, "prec", prec, "d_rho err", e_rho, "d_s err", e_s)
        assert e_rho <= TOL[prec] and e_s <= TOL[prec]
    assert sum(ev["injected"]) > 0 and sum(ev["removed"]) > 0
    a.close()


def test_adjoint_matches_oracle_gr_tube_fp64(gpu_lib):
    """Frame-dragging tube of a B = 1e12 G, P = 0.3 s pulsar at Nz = 1024
    with 5e4 electrons, 100 steps in 10 segments: gradients with respect to
    rho_GJ, s and (B, P, R, w) against the oracle's FP64 adjoint (whose
    rho_GJ Jacobian is analytic; the library's is a central difference)."""
    kw, z, u, nsteps, K = gr_problem(B.SCLF_FP64)
    a, vals = gpu_run(kw, z, u, nsteps, K)
    d = B.derive(B.default_params(**kw))
    for i, which in enumerate(("gamma", "ez")):
        v, grad, run, inj, rem = oadj.parameter_gradient(
            which, orc.RHO_GR, kw["B_G"], kw["P_s"], kw["R_cm"], kw["Rstar_cm"], kw["incl_rad"],
            kw["mass_g"], kw["Nz"], kw["L_over_R"], d["dt"], d["s"], nsteps, z, u,
            precision="f64", accumulate="fixed")
        assert np.array_equal(a.events()["injected"], inj)
        assert abs(vals[i] - v) <= 1e-12 * abs(v)
        g_rho, g_s = a.backward(i)
        pg = a.param_gradient(g_rho, g_s)
        errs = np.abs(pg - grad) / np.abs(grad)
        print(which, "grad", pg, "oracle", grad, "err", errs)
        assert np.all(errs <= 1e-7)
    a.close()


def test_adjoint_matches_central_differences_gpu(gpu_lib):
    """d(mean gamma, ||E_z||)/d(B, P, R, w) from the GPU adjoint against
    central differences (relative step 1e-4) of the GPU forward run, with
    the injection counts of the base run replayed and the removals checked
    to be the same (FP64 particles, GR tube at Nz = 1024, 5e4 electrons)."""
    kw, z, u, nsteps, K = gr_problem(B.SCLF_FP64)
    a, vals = gpu_run(kw, z, u, nsteps, K)
    ev = a.events()
    grads = []
    for i in range(2):
        g_rho, g_s = a.backward(i)
        grads.append(a.param_gradient(g_rho, g_s))
    s_ref = B.derive(B.default_params(**kw))["s"]
    theta = [kw["B_G"], kw["P_s"], kw["R_cm"], 1.0]
    for k in range(4):
        fv = []
        for sg in (1.0, -1.0):
            th = list(theta)
            th[k] *= 1.0 + sg * 1e-4
            kk = dict(kw, B_G=th[0], P_s=th[1], R_cm=th[2], macro_charge=th[3] * s_ref)
            b, v = gpu_run(kk, z, u, nsteps, K, injections=ev["injected"])
            assert np.array_equal(b.events()["removed"], ev["removed"])
            fv.append(v)
            b.close()
        for i in range(2):
            fd = (fv[0][i] - fv[1][i]) / (2e-4 * theta[k])
            err = abs(grads[i][k] - fd) / abs(fd)
            print("obj", i, "param", k, grads[i][k], fd, err)
            assert err <= 1e-5
    a.close()


def test_charge_free_run_obeys_euler_identity_gpu(gpu_lib):
    """No particles, no injection: ||E_z|| is homogeneous of degree one in
    rho_GJ, so sum_j rho_j d||E_z||/drho_j = ||E_z||."""
    nz, L = 1024, 8.0
    zz = np.arange(nz + 1) * (L / nz)
    rho = -1.0 - 0.3 * np.sin(zz)
    kw = dict(L_over_R=L, Nz=nz, dt=0.4 * L / nz, rho_gj_mode=B.SCLF_RHO_USER,
              rho_gj_user=rho, target_particles=50000, capacity=1 << 14,
              precision=B.SCLF_FP64, accumulate=B.SCLF_ACC_FIXED64)
    a, vals = gpu_run(kw, None, None, 40, 10, injections=np.zeros(40, np.int64))
    g_rho, g_s = a.backward(B.SCLF_OBJ_EZ)
    assert g_s == 0.0
    assert abs(float(np.dot(rho, g_rho)) - vals[1]) <= 1e-10 * vals[1]
    a.close()


def test_autograd_function_gives_the_adjoint_gradient(gpu_lib):
    """tube_objectives(theta).backward() equals the direct adjoint calls, at
    an injection weight w != 1 (d/dw = d_s s_ref comes from the C ABI), and a
    second backward through a retained graph gives the same gradient again."""
    import torch
    kw, z, u, nsteps, K = gr_problem(B.SCLF_FP32, n=20000, nsteps=40)
    base = {k: v for k, v in kw.items() if k not in ("dt", "R_cm")}
    spec, theta0 = B.adjoint_problem(base, nsteps, K, z, u)
    theta0 = theta0.copy()
    theta0[3] = 1.25
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    out = B.tube_objectives(theta, spec)
    loss = out[0] + 2.0 * out[1] / float(out[1].detach())
    loss.backward(retain_graph=True)
    g1 = theta.grad.numpy().copy()
    loss.backward()                                   # the same recorded run again
    g2 = theta.grad.numpy() - g1
    a, vals = gpu_run(dict(kw, macro_charge=1.25 * spec["s_ref"]), z, u, nsteps, K)
    assert np.allclose(out.detach().numpy(), vals, rtol=1e-12, atol=0)
    want = np.zeros(4)
    for i, w in enumerate((1.0, 2.0 / vals[1])):
        g_rho, g_s = a.backward(i)
        pg = a.param_gradient(g_rho, g_s, spec["s_ref"])
        assert pg[3] == g_s * spec["s_ref"]
        want += w * pg
    assert np.allclose(g1, want, rtol=1e-12, atol=0)
    assert np.allclose(g2, want, rtol=1e-12, atol=0)
    a.close()


def test_adjoint_rejects_unsupported_states(gpu_lib):
    kw, z, u, nsteps, K = flat_problem(B.SCLF_FP32, n=100, nsteps=10, K=10)
    a = B.Adjoint(B.default_params(**kw), nsteps, K)
    with pytest.raises(B.SclfError) as e:
        a.backward(0)
    assert e.value.code == -7                      # SCLF_ESTATE before a forward pass
    with pytest.raises(B.SclfError):
        a.tube.step()                              # the driver steps its tube
    a.close()


def test_timed_passes_count_kernels_and_keep_the_gradient(gpu_lib):
    """Timing mode replays graphs with event-record nodes: the launch counts
    are those of the checkpoint schedule (the last segment is not
    recomputed) and the gradient is unchanged."""
    kw, z, u, nsteps, K = flat_problem(B.SCLF_FP32, n=5000, nsteps=40, K=10)
    a, _ = gpu_run(kw, z, u, nsteps, K)
    g0, s0 = a.backward(B.SCLF_OBJ_GAMMA)
    a.set_timing(1)
    a.forward()
    g1, s1 = a.backward(B.SCLF_OBJ_GAMMA)
    kt = a.kernel_times()
    assert kt["forward_push"][1] == nsteps and kt["forward_field"][1] == nsteps
    assert kt["recompute_push"][1] == nsteps - K and kt["reverse_push"][1] == nsteps
    assert all(ms > 0.0 for ms, n in kt.values())
    assert rel(g1, g0) <= 1e-12 and abs(s1 - s0) <= 1e-12 * abs(s0)
    a.set_timing(2)                          # segments 0 and 2 of each kind
    a.forward()
    a.backward(B.SCLF_OBJ_GAMMA)
    kt = a.kernel_times()
    assert kt["forward_push"][1] == 2 * K and kt["reverse_push"][1] == 2 * K
    assert kt["recompute_push"][1] == 2 * K      # 3 recomputed segments: 1st and 3rd
    a.close()


def test_fix32_gradient_against_fp64_is_stated(gpu_lib):
    """Frame-dragging tube of config 4 at Nz = 1024 with 5e4 electrons, 100
    steps: the FP32 and 32-bit fixed-point gradients against the FP64 one
    (printed; the fixed-point positions must be at least as close)."""
    errs = {}
    grads = {}
    for prec in (B.SCLF_FP64, B.SCLF_FP32, B.SCLF_FIX32):
        kw, z, u, nsteps, K = gr_problem(prec)
        a, vals = gpu_run(kw, z, u, nsteps, K)
        grads[prec] = [a.param_gradient(*a.backward(i)) for i in range(2)]
        a.close()
    for prec in (B.SCLF_FP32, B.SCLF_FIX32):
        errs[prec] = max(float(np.max(np.abs(g - r) / np.abs(r)))
                         for g, r in zip(grads[prec], grads[B.SCLF_FP64]))
    print("max rel gradient error vs FP64: fp32 %.3e fix32 %.3e" % (errs[B.SCLF_FP32],
                                                                  errs[B.SCLF_FIX32]))
    assert errs[B.SCLF_FIX32] <= max(errs[B.SCLF_FP32], 1e-6)


@pytest.mark.parametrize("prec", [B.SCLF_FP64, B.SCLF_FP32])
def test_weighted_ez_profile_gradient_matches_oracle(gpu_lib, prec):
    """The projection sum_j w_j E_z,j of the final E_z profile (random
    weights) on the flat tube: GPU gradient against the oracle's adjoint."""
    kw, z, u, nsteps, K = flat_problem(prec)
    a, _ = gpu_run(kw, z, u, nsteps, K)
    w = np.random.default_rng(3).standard_normal(kw["Nz"])
    with pytest.raises(B.SclfError) as e:
        a.backward(B.SCLF_OBJ_EZ_WEIGHTED)            # no weights yet
    assert e.value.code == -7
    a.set_weights(w)
    g_rho, g_s = a.backward(B.SCLF_OBJ_EZ_WEIGHTED)
    run = oracle_run(kw, z, u, prec)
    v, d_rho, d_s, _, _ = run.gradient("ez_weighted", nsteps, weights=w)
    ez = a.tube.read_fields(rho=False)["ez"]
    scale = float(np.sum(np.abs(w) * np.abs(ez)))
    assert abs(float(np.dot(w, ez)) - v) <= (1e-12 if prec == B.SCLF_FP64 else 1e-6) * scale
    assert rel(g_rho, d_rho) <= TOL[prec] and abs(g_s - d_s) <= TOL[prec] * abs(d_s)
    a.close()


@pytest.mark.parametrize("prec", [B.SCLF_FP32, B.SCLF_FIX32])
def test_launch_overlap_gives_the_same_gradient(gpu_lib, prec):
    """The forward, recompute and reverse kernels by programmatic dependent
    launch give the same values bit for bit as plain stream order, and the
    same (rho_GJ, s) gradients to the order of the FP64 atomic grid sums."""
    kw, z, u, nsteps, K = flat_problem(prec)
    plain, vp = gpu_run(dict(kw, launch_overlap=-1), z, u, nsteps, K)
    over, vo = gpu_run(dict(kw, launch_overlap=1), z, u, nsteps, K)
    assert np.array_equal(vp, vo)
    for obj in (B.SCLF_OBJ_GAMMA, B.SCLF_OBJ_EZ):
        gp, sp = plain.backward(obj)
        go, so = over.backward(obj)
        assert rel(go, gp) < 1e-12 and abs(so - sp) <= 1e-12 * abs(sp), obj
    plain.close()
    over.close()


@pytest.mark.parametrize("prec", [B.SCLF_FP32, B.SCLF_FIX32])
def test_one_segment_chosen_by_the_library_gives_the_same_gradient(gpu_lib, prec):
    """checkpoint_every = 0: the library keeps the whole run as one segment
    when its snapshots fit (here they do), so the backward pass replays
    nothing; the values equal those of the run checkpointed every 10 steps
    bit for bit (the recompute reproduces the trajectory exactly) and the
    (rho_GJ, s) gradients to the order of the FP64 atomic grid sums."""
    kw, z, u, nsteps, K = flat_problem(prec)
    a10, v10 = gpu_run(kw, z, u, nsteps, K)
    a1, v1 = gpu_run(kw, z, u, nsteps, 0)
    assert a10.checkpoint_every == K and a1.checkpoint_every == nsteps
    assert np.array_equal(v10, v1)
    for obj in (B.SCLF_OBJ_GAMMA, B.SCLF_OBJ_EZ):
        g10, s10 = a10.backward(obj)
        g1, s1 = a1.backward(obj)
        assert rel(g1, g10) < 1e-12 and abs(s1 - s10) <= 1e-12 * abs(s10), obj
    a10.close()
    a1.close()
