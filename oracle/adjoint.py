"""FP64 discrete adjoint of the oracle tube -- test infrastructure only.

Only ``tests/`` and ``bench.py``'s CPU legs import this module; the GPU
library never calls it.

The differentiated map. N steps of :class:`oracle.sclf_oracle.Tube` (Sec. 2,
Figure A) from particles given at t = 0, with fields that solve Eq. 4 for
the tube's charge at t = 0 (:meth:`Tube.solve_fields`). Its inputs are

  * rho_GJ at the nodes -- it enters through the t = 0 fields of Eq. 4 (the
    Ampere-form update of Eq. 3 never reads it again);
  * the macro-particle charge s -- it enters the current J = (s/dt) sum F
    (Sec. 2 deposit) and the charge of the prefilled particles in Eq. 4.

Held fixed (the frozen events): the number of electrons injected at each
step (an integer, piecewise constant in the inputs), the grid (L, Nz, dt in
code units) and the rounding of the particle precision (the adjoint
differentiates the real-number formulas at the computed trajectory). Which
particles leave the tube follows from the trajectory; a finite-difference
check is valid only where the perturbed runs remove the same particles,
which :meth:`AdjointRun.forward` reports.

The gather and the deposit are piecewise linear in the positions; their
derivative is taken inside the pieces: dF_j(x)/dx = 1 for j <= x < j + 1
(F_j(x) = clamp(x - j, 0, 1)), and dE_p/dx = E_{m+1/2} - E_{m-1/2}.

Objectives at the end of the run:
  'gamma': mean over the live particles of gamma = sqrt(1 + u^2)
  'ez'   : ||E_z||_2 = sqrt(sum_j E_z,j^2 dz)
  'ez_weighted': sum_j w_j E_z,j for given cell weights w (any projection of
           the E_z profile; unit weights give one cell's sensitivity)
"""

from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_banded

from . import sclf_oracle as so

OBJECTIVES = ("gamma", "ez", "ez_weighted")


# ---------------------------------------------------------------------------
# Transposes of the linear pieces
# ---------------------------------------------------------------------------

def field_update_adjoint(lez1, ler1, lb1, dt, dz):
    """Transpose of :func:`oracle.sclf_oracle.field_update` (Eq. 3 leap-frog,
    R = 1), which is linear in (E_z, E_r, B, J): the adjoints of the new
    (E_z, E_r, B) give those of the old ones and of J."""
    cdt = dt / dz
    nz = lez1.size
    lez1 = np.array(lez1, np.float64)
    ler1 = np.array(ler1, np.float64)
    lb1 = np.asarray(lb1, np.float64)
    # B' = B - cdt (E_r'_{j+1} - E_r'_j) - dt E_z'_j
    lb = lb1.copy()
    ler1[1:] -= cdt * lb1
    ler1[:-1] += cdt * lb1
    lez1 -= dt * lb1
    # E_r'_k = E_r,k - cdt (B_k - B_{k-1}) for k = 1..Nz with the ghost
    # B_Nz := B_{Nz-1}; E_r'_0 = E_r,0
    ler = ler1.copy()
    k = np.arange(1, nz + 1)
    np.add.at(lb, np.minimum(k, nz - 1), -cdt * ler1[1:])
    np.add.at(lb, k - 1, cdt * ler1[1:])
    # E_z' = E_z + dt B - 4 pi dt J
    lez = lez1
    lb += dt * lez1
    lj = -4.0 * math.pi * dt * lez1
    return lez, ler, lb, lj


def poisson_adjoint(lphi, dz):
    """Transpose of :func:`oracle.sclf_oracle.poisson_potential` (Eq. 4 on
    the nodes, phi_0 = 0, ghost phi_{Nz+1} = phi_{Nz-1}), a linear map from
    the source at nodes 0..Nz to phi at nodes 0..Nz: returns the adjoint of
    the source. Node 0 of the source does not enter (phi_0 = 0)."""
    lphi = np.asarray(lphi, np.float64)
    nz = lphi.size - 1
    n = nz
    # banded transpose of the tridiagonal system: the sub- and
    # super-diagonals swap, so the ghost entry 2 of the last row moves to
    # the super-diagonal of the last column
    abt = np.zeros((3, n))
    abt[0, 1:] = 1.0
    abt[0, n - 1] = 2.0
    abt[1, :] = -(2.0 + dz * dz)
    abt[2, :-1] = 1.0
    lsrc = np.zeros(nz + 1)
    lsrc[1:] = 4.0 * math.pi * dz * dz * solve_banded((1, 1), abt, lphi[1:])
    return lsrc


def initial_fields_adjoint(lez0, ler0, dz):
    """Adjoint of the source of Eq. 4 from those of the t = 0 fields
    E_z = -(phi_{j+1} - phi_j)/dz, E_r = phi (B = 0 carries none)."""
    lphi = np.array(ler0, np.float64)
    lphi[1:] -= lez0 / dz
    lphi[:-1] += lez0 / dz
    return poisson_adjoint(lphi, dz)


# ---------------------------------------------------------------------------
# Objectives
# ---------------------------------------------------------------------------

def objective_value(which, u, ez, dz, weights=None):
    if which == "ez_weighted":
        return float(np.dot(np.asarray(weights, np.float64), np.asarray(ez, np.float64)))
    if which == "gamma":
        u = np.asarray(u, np.float64)
        return float(np.mean(np.sqrt(1.0 + u * u))) if u.size else 0.0
    if which == "ez":
        ez = np.asarray(ez, np.float64)
        return float(math.sqrt(np.sum(ez * ez) * dz))
    raise ValueError(which)


# ---------------------------------------------------------------------------
# A recorded run and its adjoint
# ---------------------------------------------------------------------------

class AdjointRun:
    """A tube configuration (grid, rho_GJ, s, particles at t = 0, particle
    precision, current accumulation) whose N-step run can be replayed and
    differentiated."""

    def __init__(self, nz, L, dt, rho_gj, s, z0=None, u0=None, precision="f64",
                 accumulate="fixed"):
        if precision not in ("f64", "f32", "fix32"):
            raise ValueError(precision)
        if precision == "fix32" and accumulate != "fixed":
            raise ValueError("'fix32' positions deposit exact fixed-point fractions")
        self.nz, self.L, self.dt = int(nz), float(L), float(dt)
        self.dz = self.L / self.nz
        self.rho_gj = np.asarray(rho_gj, np.float64).copy()
        self.s = float(s)
        self.z0 = np.zeros(0) if z0 is None else np.asarray(z0, np.float64)
        self.u0 = np.zeros(0) if u0 is None else np.asarray(u0, np.float64)
        self.precision = precision
        self.accumulate = accumulate

    def make_tube(self, rho_gj=None, s=None):
        """The oracle tube at t = 0: particles added, fields from Eq. 4."""
        t = so.Tube(self.nz, self.L, self.dt,
                    self.rho_gj if rho_gj is None else rho_gj,
                    self.s if s is None else s,
                    precision=self.precision, accumulate=self.accumulate)
        if self.z0.size:
            t.add_particles(self.z0, self.u0)
        t.solve_fields()
        return t

    def forward(self, nsteps, rho_gj=None, s=None, injections=None, keep=False):
        """Run nsteps. injections=None lets the tube choose N_inj (Sec. 2
        rule); a sequence replays those counts. Returns (tube, injected per
        step, IDs removed per step, states) where states (keep=True) holds
        per step [xi, u before injection, E_z used by the gather, J, N_inj]."""
        t = self.make_tube(rho_gj, s)
        inj_log, rem_log, states = [], [], []
        for n in range(int(nsteps)):
            if injections is not None:
                k = int(injections[n])
                t.injection_count = lambda k=k: k          # replayed count
            if keep:
                states.append([t.xi.copy(), t.u.copy(), t.ez.copy()])
            ids_pre, tot0 = t.ids.copy(), t.total_injected
            t.step()
            inj = t.last_injected
            all_ids = np.concatenate([ids_pre, tot0 + np.arange(inj, dtype=np.int64)])
            inj_log.append(inj)
            rem_log.append(np.setdiff1d(all_ids, t.ids))
            if keep:
                states[-1] += [t.j.copy(), inj]
        return t, inj_log, rem_log, states

    def gradient(self, which, nsteps, injections=None, weights=None):
        """Objective and its gradient with respect to rho_GJ (nodes 0..Nz)
        and s, by the discrete adjoint of the recorded run ('ez_weighted'
        takes the cell weights). Returns (value, d_rho_gj, d_s, injected per
        step, removed IDs per step)."""
        if which not in OBJECTIVES:
            raise ValueError(which)
        t, inj_log, rem_log, states = self.forward(nsteps, injections=injections, keep=True)
        rt = t.rt
        nz, dz, dt, s = self.nz, self.dz, self.dt, self.s
        dt_r = float(rt(dt))                 # the constants the push used
        cfl_r = float(rt(dt / dz))
        u_end = t.u.astype(np.float64)
        value = objective_value(which, u_end, t.ez, dz, weights)

        lez = np.zeros(nz)
        ler = np.zeros(nz + 1)
        lb = np.zeros(nz)
        lx = np.zeros(u_end.size)
        if which == "gamma":
            lu = u_end / np.sqrt(1.0 + u_end * u_end) / max(u_end.size, 1)
        elif which == "ez":
            lu = np.zeros(u_end.size)
            lez = t.ez * dz / value if value > 0.0 else np.zeros(nz)
        else:
            lu = np.zeros(u_end.size)
            lez = np.array(weights, np.float64)
        sum_lj_j = 0.0

        fix = self.precision == "fix32"
        fb = t.fb
        scale = 2.0 ** -fb if fix else 1.0           # cells per stored position unit
        for n in reversed(range(int(nsteps))):
            xi_pre, u_pre, ez, jn, ninj = states[n]
            x0r = np.concatenate([xi_pre, np.zeros(ninj, xi_pre.dtype)])
            u0r = np.concatenate([u_pre, np.zeros(ninj, u_pre.dtype)])
            # the step's forward values, recomputed as the tube computed them
            if fix:
                ep = so.gather_fix32(ez, x0r, fb)
                x1r, u1r, finite = so.push_fix32(x0r, u0r, ep, dt, dz, fb)
                alive = finite & (x1r >= 0) & (x1r < (nz << fb))
                h = x0r + (1 << (fb - 1))
                m = h >> fb
                f = ((h & ((1 << fb) - 1)).astype(np.float32)
                     * np.float32(2.0 ** -fb)).astype(np.float64)
            else:
                ep = so.gather(ez, x0r, rt)
                x1r, u1r = so.push(x0r, u0r, ep, dt, dz, rt)
                finite = np.isfinite(x1r) & np.isfinite(u1r)
                alive = finite & (x1r >= 0) & (x1r < nz)
                hh = x0r + rt(0.5)
                mf = np.floor(hh)
                f = (hh - mf).astype(np.float64)
                m = mf.astype(np.int64)
            lx1 = np.zeros(x0r.size)
            lu1 = np.zeros(x0r.size)
            lx1[alive] = lx
            lu1[alive] = lu
            # (a6) Eq. 3, transposed
            lez, ler, lb, lj = field_update_adjoint(lez, ler, lb, dt, dz)
            sum_lj_j += float(np.dot(lj, jn))
            lS = (s / dt) * lj                       # adjoint of the fraction sums
            # (a4) deposit: J_j = (s/dt) sum_p [F_j(x1) - F_j(x0)], positions in cells
            x0 = x0r.astype(np.float64) * scale
            x1 = np.where(alive, x1r, 0).astype(np.float64) * scale
            c0 = np.floor(x0).astype(np.int64)
            c1 = np.floor(x1).astype(np.int64)
            lx1 = lx1 + np.where(alive, lS[np.clip(c1, 0, nz - 1)], 0.0)
            lx0 = np.where(finite, lx1 - lS[np.clip(c0, 0, nz - 1)], 0.0)
            # (a3) Eq. 1: u1 = u0 - E_p dt, x1 = x0 + (u1 / gamma1) dt/dz (the
            # rounding of the displacement to the position grid as the identity)
            u1 = np.where(finite, u1r, 0).astype(np.float64)
            g1 = np.sqrt(1.0 + u1 * u1)
            lu0 = np.where(finite, lu1 + lx1 * cfl_r / g1 ** 3, 0.0)
            lep = -dt_r * lu0
            # (a2) gather: E_p = (1 - f) E_{m-1/2} + f E_{m+1/2}, f = x + 1/2 - m
            ia = np.clip(m - 1, 0, nz - 1)
            ib = np.clip(m, 0, nz - 1)
            e = np.asarray(ez, np.float64).astype(rt).astype(np.float64)
            np.add.at(lez, ia, (1.0 - f) * lep)
            np.add.at(lez, ib, f * lep)
            lx0 = lx0 + lep * (e[ib] - e[ia])
            # injected electrons start at fixed (0, 0): their adjoint ends here
            lx = lx0[:xi_pre.size]
            lu = lu0[:xi_pre.size]

        # t = 0: fields from Eq. 4 with source rho_GJ - rho_particles(s)
        d_rho = initial_fields_adjoint(lez, ler, dz)
        cells0 = (np.asarray(states[0][0], np.float64) * scale if nsteps
                  else t.cells())
        rho_p = so.rho_nodes(cells0, s, dz, nz)
        d_s = sum_lj_j / s - float(np.dot(d_rho, rho_p)) / s
        return value, d_rho, d_s, inj_log, rem_log


# ---------------------------------------------------------------------------
# Pulsar parameters (B, P, R, injection weight)
# ---------------------------------------------------------------------------

def rho_gj_parameter_jacobian(mode, z, B_G, P_s, R_cm, Rstar_cm, incl, mass_g):
    """d rho_GJ / d(B, P, R) at the node heights z (code units, held fixed)
    for the profiles of :func:`oracle.sclf_oracle.rho_gj_profile`, with R an
    independent coordinate (not R_* theta_p(P)).

    rho = -(Lambda0^2 / 4 pi) G(eta, theta_*), Lambda0^2 proportional to
    Omega B R^2 (Sec. 3: omega_p^2 = 4 pi n0 e^2 / m, n0 = Omega B / 2 pi c e),
    theta_* = 0.67 sqrt(Omega R_* / c), eta = 1 + z R / R_*, Omega = 2 pi / P:
      d/dB = rho / B
      d/dP = -rho / P - (Lambda0^2/4 pi) dG/dtheta_* dtheta_*/dP,
             dtheta_*/dP = -theta_* / (2 P)
      d/dR = 2 rho / R - (Lambda0^2/4 pi) dG/deta z / R_*
    with G = cos i + 3/2 sqrt(eta) theta_* sin i (flat) or
    (1 - kappa / eta^3) cos i + 3/2 sqrt(eta) theta_* sin i (frame dragging).
    Returns a dict of arrays keyed 'B', 'P', 'R'."""
    cu = so.code_units(B_G, P_s, Rstar_cm, incl, mass_g, R_cm)
    z = np.asarray(z, np.float64)
    lam2 = cu["Lambda0"] ** 2
    eta = 1.0 + z * cu["R_over_Rstar"]
    th = cu["theta_star"]
    rho = so.rho_gj_profile(mode, z, cu["Lambda0"], incl, th, cu["R_over_Rstar"], cu["kappa"])
    dG_dth = 1.5 * np.sqrt(eta) * math.sin(incl)
    dG_deta = 0.75 * th * math.sin(incl) / np.sqrt(eta)
    if mode == so.RHO_GR:
        dG_deta = dG_deta + 3.0 * cu["kappa"] * math.cos(incl) / eta ** 4
    pref = -lam2 / (4.0 * math.pi)
    return {
        "B": rho / B_G,
        "P": -rho / P_s + pref * dG_dth * (-th / (2.0 * P_s)),
        "R": 2.0 * rho / cu["R_cm"] + pref * dG_deta * z / Rstar_cm,
    }


def parameter_gradient(which, mode, B_G, P_s, R_cm, Rstar_cm, incl, mass_g, nz, L, dt,
                       s, nsteps, z0=None, u0=None, precision="f64",
                       accumulate="fixed", injections=None):
    """Objective and its gradient with respect to (B, P, R, w) at a fixed
    grid, where rho_GJ comes from (B, P, R) as in
    :func:`oracle.sclf_oracle.rho_gj_profile` and the macro charge is w s
    (w = 1 at the point of evaluation). Returns (value, grad[4], run,
    injected per step, removed IDs per step)."""
    z = np.arange(nz + 1) * (L / nz)
    cu = so.code_units(B_G, P_s, Rstar_cm, incl, mass_g, R_cm)
    rho = so.rho_gj_profile(mode, z, cu["Lambda0"], incl, cu["theta_star"],
                            cu["R_over_Rstar"], cu["kappa"])
    run = AdjointRun(nz, L, dt, rho, s, z0, u0, precision, accumulate)
    value, d_rho, d_s, inj, rem = run.gradient(which, nsteps, injections)
    jac = rho_gj_parameter_jacobian(mode, z, B_G, P_s, R_cm, Rstar_cm, incl, mass_g)
    grad = np.array([np.dot(d_rho, jac["B"]), np.dot(d_rho, jac["P"]),
                     np.dot(d_rho, jac["R"]), d_s * s])
    return value, grad, run, inj, rem
