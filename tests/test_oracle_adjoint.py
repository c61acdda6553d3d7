"""Pins of the oracle's FP64 discrete adjoint (oracle/adjoint.py).

The adjoint is checked against things other than itself: the exact
transposes of the linear steps (dot-product identities with the oracle's own
forward functions), the homogeneity of a charge-free run (Euler's identity),
central finite differences of the oracle's forward run with the injection
counts replayed (rel. step 1e-4), and central differences of the
closed-form rho_GJ profile for the parameter Jacobian. A dropped term, a
wrong sign or a transposed index in any reverse step fails one of them.
"""

import math

import numpy as np
import pytest

import oracle as orc
from oracle import adjoint as adj
from paper_1011_6330_gb300 import synth

M_STAR = 1.4 * orc.M_SUN


def test_field_update_adjoint_is_the_transpose():
    """<F(x), y> = <x, F^T(y)> for the (E_z, E_r, B, J) -> (E_z, E_r, B)
    leap-frog of Eq. 3, which is linear."""
    rng = np.random.default_rng(11)
    for nz in (2, 3, 37):
        dz, dt = 0.1, 0.03
        x = [rng.standard_normal(nz), rng.standard_normal(nz + 1),
             rng.standard_normal(nz), rng.standard_normal(nz)]
        y = [rng.standard_normal(nz), rng.standard_normal(nz + 1), rng.standard_normal(nz)]
        fx = orc.field_update(x[0], x[1], x[2], x[3], dt, dz)
        fty = adj.field_update_adjoint(y[0], y[1], y[2], dt, dz)
        lhs = sum(float(np.dot(a, b)) for a, b in zip(fx, y))
        rhs = sum(float(np.dot(a, b)) for a, b in zip(fty, x))
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0)


def test_poisson_adjoint_is_the_transpose():
    """<phi(src), l> = <src, phi^T(l)> for the Eq. 4 solve of the oracle."""
    rng = np.random.default_rng(12)
    for nz in (2, 5, 64):
        dz = 8.0 / nz
        src = rng.standard_normal(nz + 1)
        lphi = rng.standard_normal(nz + 1)
        lhs = float(np.dot(orc.poisson_potential(src, dz), lphi))
        rhs = float(np.dot(src, adj.poisson_adjoint(lphi, dz)))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)
        assert adj.poisson_adjoint(lphi, dz)[0] == 0.0


def test_charge_free_run_obeys_euler_identity():
    """With no particles and no injection the run is linear in rho_GJ, so
    ||E_z|| is homogeneous of degree one: sum_j rho_j d/drho_j = ||E_z||."""
    nz, L = 128, 8.0
    dz = L / nz
    z = np.arange(nz + 1) * dz
    rho = -1.0 - 0.3 * np.sin(z)
    run = adj.AdjointRun(nz, L, 0.4 * dz, rho, -1e-3)
    value, d_rho, d_s, inj, _ = run.gradient("ez", 50, injections=[0] * 50)
    assert sum(inj) == 0 and d_s == 0.0
    assert abs(float(np.dot(rho, d_rho)) - value) <= 1e-10 * value


def flat_case(nsteps=10):
    nz, L = 64, 8.0
    dz = L / nz
    s = orc.macro_charge_for(1.0, L, 2000)
    z0, u0 = synth.prefilled_beam(600, 0.8 * L, 3.0, seed=3)
    return adj.AdjointRun(nz, L, 0.4 * dz, -np.ones(nz + 1), s, z0, u0,
                          precision="f64", accumulate="sum"), nsteps


def central_difference(run, which, nsteps, inj, rem, rho=None, s=None, d_rho=None,
                       d_s=0.0, rel=1e-4):
    """(f(+h) - f(-h)) / 2h along (d_rho, d_s), injections replayed; checks
    that both perturbed runs remove the same particles as the base run."""
    rho = run.rho_gj if rho is None else rho
    s = run.s if s is None else s
    vals = []
    for sg in (1.0, -1.0):
        r = rho + sg * rel * (0.0 if d_rho is None else d_rho)
        t, _, rem2, _ = run.forward(nsteps, rho_gj=r, s=s + sg * rel * d_s, injections=inj)
        assert all(np.array_equal(a, b) for a, b in zip(rem, rem2))
        vals.append(adj.objective_value(which, t.u, t.ez, run.dz))
    return (vals[0] - vals[1]) / (2.0 * rel)


@pytest.mark.parametrize("which", ["gamma", "ez"])
def test_gradient_matches_central_differences(which):
    """d/drho_GJ along a random direction and d/ds against central
    differences of the oracle run (FP64, injections replayed)."""
    run, n = flat_case()
    value, d_rho, d_s, inj, rem = run.gradient(which, n)
    assert sum(inj) > 0                       # injection happens in the run
    d = np.random.default_rng(5).standard_normal(run.nz + 1)
    fd = central_difference(run, which, n, inj, rem, d_rho=d)
    assert abs(float(np.dot(d_rho, d)) - fd) <= 1e-6 * abs(fd)
    fds = central_difference(run, which, n, inj, rem, d_s=run.s) / run.s
    assert abs(d_s - fds) <= 1e-6 * abs(fds)


def test_parameter_jacobian_matches_closed_form_differences():
    """d rho_GJ / d(B, P, R) of the analytic chain against central
    differences of code_units + rho_gj_profile (R held independent)."""
    for mode, incl in ((orc.RHO_GR, 0.5), (orc.RHO_FLAT, 0.3)):
        B, P, Rs = 1e12, 0.3, 1e6
        cu = orc.code_units(B, P, Rs, incl, M_STAR)
        R = cu["R_cm"]
        z = np.linspace(0.0, 2.0 / cu["theta_p"], 33)
        jac = adj.rho_gj_parameter_jacobian(mode, z, B, P, R, Rs, incl, M_STAR)

        def rho_of(b, p, r):
            c = orc.code_units(b, p, Rs, incl, M_STAR, r)
            return orc.rho_gj_profile(mode, z, c["Lambda0"], incl, c["theta_star"],
                                      c["R_over_Rstar"], c["kappa"])
        for k, key in enumerate("BPR"):
            base = (B, P, R)[k]
            hp, hm = [B, P, R], [B, P, R]
            hp[k] += 1e-6 * base
            hm[k] -= 1e-6 * base
            fd = (rho_of(*hp) - rho_of(*hm)) / (2e-6 * base)
            assert np.max(np.abs(fd - jac[key])) <= 1e-7 * np.max(np.abs(fd))


@pytest.mark.parametrize("which", ["gamma", "ez"])
def test_pulsar_parameter_gradient_matches_central_differences(which):
    """Gradient with respect to (B, P, R, w) of a frame-dragging tube of a
    B = 1e12 G, P = 0.3 s pulsar against central differences with relative
    step 1e-4, injections replayed, grid (L, Nz, dt) fixed."""
    mode, B, P, Rs, incl = orc.RHO_GR, 1e12, 0.3, 1e6, 0.5
    cu = orc.code_units(B, P, Rs, incl, M_STAR)
    R = cu["R_cm"]
    nz, L = 64, 2.0 / cu["theta_p"]
    dz = L / nz
    z = np.arange(nz + 1) * dz
    dt = orc.default_dt(dz, cu["Lambda0"])
    rho0 = orc.rho_gj_profile(mode, 0.0, cu["Lambda0"], incl, cu["theta_star"],
                              cu["R_over_Rstar"], cu["kappa"])
    s = orc.macro_charge_for(abs(float(rho0)), L, 3000)
    z0, u0 = synth.prefilled_beam(1500, L - dz, 1e3, seed=5)
    n = 20
    value, grad, run, inj, rem = adj.parameter_gradient(
        which, mode, B, P, R, Rs, incl, M_STAR, nz, L, dt, s, n, z0, u0, accumulate="sum")
    assert sum(inj) > 0
    theta = [B, P, R, 1.0]
    for k in range(4):
        vals = []
        for sg in (1.0, -1.0):
            th = list(theta)
            th[k] *= 1.0 + sg * 1e-4
            c = orc.code_units(th[0], th[1], Rs, incl, M_STAR, th[2])
            r = orc.rho_gj_profile(mode, z, c["Lambda0"], incl, c["theta_star"],
                                   c["R_over_Rstar"], c["kappa"])
            t, _, rem2, _ = run.forward(n, rho_gj=r, s=s * th[3], injections=inj)
            assert all(np.array_equal(a, b) for a, b in zip(rem, rem2))
            vals.append(adj.objective_value(which, t.u, t.ez, dz))
        fd = (vals[0] - vals[1]) / (2e-4 * theta[k])
        assert abs(grad[k] - fd) <= 1e-6 * abs(fd), (k, grad[k], fd)


def test_float32_trajectory_gradient_is_close_to_float64():
    """The adjoint of the float32 run (reverse sweep in FP64) stays close to
    that of the FP64 run on a short run where the trajectories agree to
    float32 rounding."""
    run, n = flat_case()
    v64, g64, s64, inj, _ = run.gradient("gamma", n)
    run32 = adj.AdjointRun(run.nz, run.L, run.dt, run.rho_gj, run.s, run.z0, run.u0,
                           precision="f32", accumulate="sum")
    v32, g32, s32, _, _ = run32.gradient("gamma", n, injections=inj)
    assert abs(v32 - v64) <= 1e-6 * v64
    assert np.max(np.abs(g32 - g64)) <= 1e-3 * np.max(np.abs(g64))
    assert abs(s32 - s64) <= 1e-3 * abs(s64)


def test_fix32_trajectory_gradient_is_close_to_float64():
    """The adjoint of the 32-bit fixed-point run (displacement rounding
    differentiated as the identity, reverse sweep in FP64) stays close to the
    FP64 run's on a short run."""
    run, n = flat_case()
    v64, g64, s64, inj, _ = run.gradient("gamma", n)
    runx = adj.AdjointRun(run.nz, run.L, run.dt, run.rho_gj, run.s, run.z0, run.u0,
                          precision="fix32", accumulate="fixed")
    vx, gx, sx, _, _ = runx.gradient("gamma", n, injections=inj)
    assert abs(vx - v64) <= 1e-7 * v64
    assert np.max(np.abs(gx - g64)) <= 1e-5 * np.max(np.abs(g64))
    assert abs(sx - s64) <= 1e-5 * abs(s64)


def test_weighted_ez_gradient_matches_central_differences():
    """The projection sum_j w_j E_z,j of the final E_z profile (random
    weights): gradient along a random rho_GJ direction and in s against
    central differences; with no particles and no injection it is linear in
    rho_GJ, so its gradient dotted with rho_GJ is the value itself."""
    run, n = flat_case()
    w = np.random.default_rng(9).standard_normal(run.nz)
    value, d_rho, d_s, inj, rem = run.gradient("ez_weighted", n, weights=w)
    d = np.random.default_rng(10).standard_normal(run.nz + 1)
    vals = []
    for sg in (1.0, -1.0):
        t, _, rem2, _ = run.forward(n, rho_gj=run.rho_gj + sg * 1e-4 * d, injections=inj)
        assert all(np.array_equal(a, b) for a, b in zip(rem, rem2))
        vals.append(float(np.dot(w, t.ez)))
    fd = (vals[0] - vals[1]) / 2e-4
    assert abs(float(np.dot(d_rho, d)) - fd) <= 1e-6 * abs(fd)
    empty = adj.AdjointRun(run.nz, run.L, run.dt, run.rho_gj * 1.3, run.s)
    v0, g0, s0, _, _ = empty.gradient("ez_weighted", 30, injections=[0] * 30, weights=w)
    assert abs(float(np.dot(g0, empty.rho_gj)) - v0) <= 1e-10 * abs(v0)
