"""Plain CPU oracle of the paper's 1D particle-in-cell time step.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (CPU baseline and reference arm) may import this module; the
CUDA library and its binding never do, and this module imports nothing
from them.

Source: Y. Barzilay, "Full simulation of the open field lines above pulsar's
polar cap - Part I" (arXiv:1011.6330).

One time step, in the order of Sec. 2 and Figure A:
  (a1) electrons are injected at the base while rho_GJ there is not
       compensated (Sec. 2; "free ejection", Abstract);
  (a2) E_z is weighted (interpolated) to each particle, cloud-in-cell
       (Sec. 2, PIC as in Birdsall & Langdon);
  (a3) each particle is pushed with Eq. 1, F = q E_z = d(gamma m v)/dt,
       v = dz/dt;
  (a4) the current is deposited from all particles (Sec. 2, Figure A);
  (a5) particles leaving the tube are removed (Sec. 3: electrons may
       return to the star);
  (a6) Eq. 3 (Maxwell with d/dr -> 1/R) is advanced by leap-frog (Sec. 2).
Set-up (a7): Eq. 4 with phi = 0 at the base and phi' = 0 at the top, empty
tube, B_phi = 0 (Sec. 2). Profiles: flat rho_GJ Eq. 5, frame-dragging
rho_GJ Eq. 6 with omega from Eq. 7.

Units (Sec. 3): c = 1, lengths in R (so R = 1 and d/dr -> 1/R is a factor
1), time in R/c, electron q/m = -1, charge density in units where
omega_p^2 = 4 pi |rho| |q/m|, hence |rho_GJ| = Lambda^2 / (4 pi) with
Lambda = omega_p R / c.

Discretisation (the paper only says "leap-frog" and "PIC"; these are the
readings this oracle fixes):
  * Nz uniform cells of width dz = L / Nz. Nodes j = 0..Nz carry phi,
    rho, rho_GJ and E_r; cell centres j + 1/2 (index j = 0..Nz-1) carry
    E_z, B_phi and J (a 1D Yee layout). E_z, E_r, rho, z live at integer
    steps n; u = gamma*beta, J and B_phi at half steps.
  * A particle's position is kept in cell units, xi = z / dz.
  * Gather: m = floor(xi + 1/2), f = xi + 1/2 - m,
    E_p = (1 - f) E_{m-1/2} + f E_{m+1/2}, the two end half-cells clamped.
  * Deposit: with F_j(xi) = clamp(xi - j, 0, 1), a particle moving from
    xi to xi' adds s/dt * (F_j(xi') - F_j(xi)) to J_{j+1/2}. This is
    charge conserving against cloud-in-cell rho at the nodes, so Gauss's
    law is kept exactly on the interior nodes.
  * Injection ("as long as rho_GJ at the base is not compensated", Sec. 2):
    the surface field E_s follows from Gauss's law over the half cell
    [0, dz/2] at the base, E_s = E_{1/2} - 4 pi s W_0 + 2 pi dz rho_GJ,0,
    with W_0 = sum of the cloud-in-cell weights (1 - xi) of the particles
    in the base cell. While E_s < 0 pulls electrons off the surface,
    N_inj = max(0, round-half-even(-E_s / (4 pi |s|))) electrons are added
    at xi = 0 with u = 0 (each lifts E_s by 4 pi |s|) and pushed in the
    same step. W_0 is summed in 2^-32 fixed point so the count is an exact
    function of the positions.
  * Removal: xi' >= Nz (top) or xi' < 0 (back into the star).
  * Field top boundary: ghost B_{Nz+1/2} = B_{Nz-1/2} (phi' = 0 at the top);
    E_r at node 0 is 0 (phi = 0 on the conducting surface).

Modes of :class:`Tube`:
  precision  'f64' (default), 'f32' or 'fix32'. In 'f32' the particle
             arithmetic (xi, u, weights, current fractions) is IEEE float32
             with one rounding per operation and no fused multiply-add,
             gathering from a float32 copy of E_z. In 'fix32' positions are
             integers X = xi * 2^fb (fb = 31 - ceil(log2 Nz) fractional bits,
             uniform resolution along the tube), u and the push are float32 as
             in 'f32', the displacement is rounded to the 2^-fb grid and the
             current fractions are exact integers. All grids stay FP64.
  accumulate 'sum': the per-cell sum of current fractions in FP64, in
             particle order; 'fixed': each F_j(xi) is rounded to a multiple
             of 2^-32 before the difference F_j(xi') - F_j(xi) is taken, and
             the sum is exact in int64, so it does not depend on the order
             of the particles and a particle's moved charge telescopes
             exactly.
  deposit    'fast': evaluates F_j only for the <= 2 cells a particle can
             touch; 'brute': evaluates it for every (particle, cell) pair.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_banded

# cgs constants (CODATA values).
C_LIGHT = 2.99792458e10      # cm/s
E_CHARGE = 4.80320471e-10    # esu
M_ELECTRON = 9.1093837015e-28  # g
G_NEWTON = 6.67430e-8        # cm^3 g^-1 s^-2
M_SUN = 1.98847e33           # g

FIXED_SCALE = 2.0 ** 32      # quantum of the 'fixed' current accumulator

RHO_FLAT, RHO_GR, RHO_USER = 0, 1, 2


# ---------------------------------------------------------------------------
# Units and profiles (Sec. 3 normalisation; Eq. 5, 6, 7)
# ---------------------------------------------------------------------------

def code_units(B_G, P_s, Rstar_cm, incl_rad, mass_g, R_cm=0.0):
    """Code-unit parameters of a pulsar tube (Sec. 3 and Eq. 5-7).

    Omega = 2 pi / P; polar-cap angle theta_p = sqrt(Omega R_* / c) (Sec. 3);
    tube radius R = R_* theta_p unless given; the aligned surface density
    n_0 = Omega B / (2 pi c e) (Sec. 3 gives n_GJ = n_0 cos i); the plasma
    frequency omega_p0 = sqrt(4 pi n_0 e^2 / m) (Sec. 3) and
    Lambda_0 = omega_p0 R / c. Frame dragging: r_g = 2 G M / c^2 and
    kappa = (2/5) r_g / R_* (Eq. 7); theta_* = 0.67 theta_p (Eq. 5 text).
    """
    omega = 2.0 * math.pi / P_s
    theta_p = math.sqrt(omega * Rstar_cm / C_LIGHT)
    R = R_cm if R_cm > 0.0 else Rstar_cm * theta_p
    n0 = omega * B_G / (2.0 * math.pi * C_LIGHT * E_CHARGE)
    omega_p0 = math.sqrt(4.0 * math.pi * n0 * E_CHARGE * E_CHARGE / M_ELECTRON)
    lam0 = omega_p0 * R / C_LIGHT
    rg = 2.0 * G_NEWTON * mass_g / (C_LIGHT * C_LIGHT)
    kappa = 0.4 * rg / Rstar_cm
    return dict(Omega=omega, theta_p=theta_p, R_cm=R, n0=n0,
                omega_p0=omega_p0, Lambda0=lam0, rg_over_Rstar=rg / Rstar_cm,
                kappa=kappa, theta_star=0.67 * theta_p,
                R_over_Rstar=R / Rstar_cm, incl=incl_rad)


def rho_gj_profile(mode, z, Lambda0, incl, theta_star, R_over_Rstar, kappa,
                   variant="cos", f=None, H=None, rg_over_Rstar=None):
    """rho_GJ at heights z (in R), code units.

    Flat space, Eq. 5 with the (R_*/r)^3 factor dropped (constant-radius
    tube, text after Eq. 5), phi = 0 (so cos(phi) = 1):
        rho = -(Lambda0^2 / 4 pi) [cos i + 3/2 sqrt(eta) theta_* sin i]
    Frame dragging, Eq. 6 with omega / Omega = kappa / eta^3 (Eq. 7) and the
    (R_*/r)^3 factor dropped as in the flat case:
        rho = -(Lambda0^2 / 4 pi) (f / f(1)) / alpha
              [(1 - kappa/eta^3) cos i + 3/2 sqrt(eta) (H / f^(1/2)) theta_* sin i]
    with f, H the curved-space factors at the given heights (f = H = 1 when
    None: the paper gives them only by reference; f(1), the base value, is
    f's first entry, so z must start at the base) and alpha = (1 - r_g/r)^(1/2)
    when rg_over_Rstar is given (else alpha = 1). variant='both' applies
    Omega -> Omega - omega to Eq. 6's prefactor instead, so the factor
    (1 - kappa/eta^3) multiplies both terms. eta = r / R_* = 1 + z R / R_*.
    The unit of density is the aligned surface value, so Lambda0^2 / 4 pi =
    Omega B / (2 pi c) in code units.
    """
    z = np.asarray(z, dtype=np.float64)
    eta = 1.0 + z * R_over_Rstar
    if mode == RHO_FLAT:
        bracket = math.cos(incl) + 1.5 * np.sqrt(eta) * theta_star * math.sin(incl)
    elif mode == RHO_GR:
        fz = np.ones_like(eta) if f is None else np.asarray(f, np.float64)
        hz = np.ones_like(eta) if H is None else np.asarray(H, np.float64)
        f1 = 1.0 if f is None else float(np.asarray(f, np.float64).ravel()[0])
        sin_term = 1.5 * np.sqrt(eta) * (hz / np.sqrt(fz)) * theta_star * math.sin(incl)
        drag = 1.0 - kappa / eta ** 3
        if variant == "cos":
            bracket = drag * math.cos(incl) + sin_term
        elif variant == "both":
            bracket = drag * (math.cos(incl) + sin_term)
        else:
            raise ValueError("variant must be 'cos' or 'both'")
        alpha = 1.0 if rg_over_Rstar is None else np.sqrt(1.0 - rg_over_Rstar / eta)
        bracket = (fz / f1) / alpha * bracket
    else:
        raise ValueError("mode must be RHO_FLAT or RHO_GR")
    return -(Lambda0 ** 2 / (4.0 * math.pi)) * bracket


def poisson_potential(rho_gj, dz):
    """phi at nodes 0..Nz from Eq. 4 with an empty tube (rho = 0).

    d^2phi/dz^2 - phi / R^2 = 4 pi rho_GJ (R = 1), phi(0) = 0 and
    phi'(L) = 0 (Sec. 2 boundary conditions). Second-order differences on
    the nodes; the top condition is a ghost node phi_{Nz+1} = phi_{Nz-1}.
    Unknowns phi_1..phi_Nz, a tridiagonal system solved by LAPACK.
    """
    rho_gj = np.asarray(rho_gj, dtype=np.float64)
    nz = rho_gj.size - 1
    n = nz
    ab = np.zeros((3, n))
    ab[0, 1:] = 1.0                     # super-diagonal (phi_{j+1})
    ab[1, :] = -(2.0 + dz * dz)         # diagonal
    ab[2, :-1] = 1.0                    # sub-diagonal (phi_{j-1})
    ab[2, n - 2] = 2.0                  # row Nz: ghost phi_{Nz+1} = phi_{Nz-1}
    rhs = 4.0 * math.pi * dz * dz * rho_gj[1:]
    phi = np.zeros(nz + 1)
    phi[1:] = solve_banded((1, 1), ab, rhs)
    return phi


def initial_fields(rho_gj, dz):
    """E_z (cells), E_r (nodes), B_phi (cells) at t = 0 (Sec. 2).

    E_z = -dphi/dz at the cell centres; E_r = -dphi/dr -> phi / R with
    phi = 0 on the conducting wall (d/dr -> 1/R, Sec. 2), at the nodes;
    B_phi = 0 because the tube starts empty (text after Eq. 4).
    """
    phi = poisson_potential(rho_gj, dz)
    ez = -(phi[1:] - phi[:-1]) / dz
    er = phi.copy()
    b = np.zeros(ez.size)
    return ez, er, b, phi


def default_dt(dz, Lambda0):
    """Time step when none is given: min(0.4 dz, 0.2 / Lambda0) (in R/c).

    The paper gives no dt rule; this keeps the light-crossing time of a
    cell and the plasma period resolved.
    """
    return min(0.4 * dz, 0.2 / Lambda0)


def macro_charge_for(rho0, L, target_particles):
    """Macro-particle charge s < 0 that fills the tube with rho_GJ(0)."""
    return -abs(rho0) * L / float(target_particles)


def base_weight_fixed(xi, rt):
    """W_0 of the base cell in 2^-32 units: sum over 0 <= xi < 1 of
    round-half-even((1 - xi) * 2^32), with 1 - xi in the particle precision."""
    xi = np.asarray(xi, rt)
    w = rt(1.0) - xi[(xi >= rt(0.0)) & (xi < rt(1.0))]
    return int(np.rint(w.astype(np.float64) * FIXED_SCALE).astype(np.int64).sum())


def injection_count(ez_half, w0_fixed, s, dz, rho0):
    """N_inj from the surface field (Sec. 2 injection rule, Gauss's law
    over the base half cell, Eq. 2 with E_r = 0 on the conducting base):

        E_s = E_{1/2} - 4 pi s W_0 + 2 pi dz rho_GJ,0
        N_inj = max(0, round-half-even(-E_s / (4 pi |s|)))
    """
    four_pi_s = 4.0 * math.pi * s
    two_pi_dz_rho0 = 2.0 * math.pi * dz * rho0
    sheet = 4.0 * math.pi * abs(s)
    es = ez_half - four_pi_s * (w0_fixed * (1.0 / FIXED_SCALE)) + two_pi_dz_rho0
    return max(0, int(np.rint(-es / sheet))), es


# ---------------------------------------------------------------------------
# The pieces of one step, as plain functions of their inputs
# ---------------------------------------------------------------------------

def gather(ez, xi, rt):
    """(a2) Cloud-in-cell weight of E_z (cells, FP64) at positions xi.

    E_z is first rounded to the particle precision rt; then
    m = floor(xi + 1/2), f = xi + 1/2 - m and
    E_p = (1 - f) E_{m-1/2} + f E_{m+1/2}, clamping E_{-1/2} := E_{1/2}
    and E_{Nz+1/2} := E_{Nz-1/2}.
    """
    nz = ez.size
    e = np.asarray(ez, np.float64).astype(rt)
    h = xi + rt(0.5)
    mf = np.floor(h)
    f = h - mf
    m = mf.astype(np.int64)
    ia = np.clip(m - 1, 0, nz - 1)
    ib = np.clip(m, 0, nz - 1)
    return (rt(1.0) - f) * e[ia] + f * e[ib]


def push(xi, u, ep, dt, dz, rt):
    """(a3) Eq. 1 with q/m = -1 and c = 1, leap-frog:
    u^{n+1/2} = u^{n-1/2} - E_p dt, gamma = sqrt(1 + u^2),
    xi^{n+1} = xi^n + (u / gamma) (dt / dz). Returns (xi', u')."""
    u1 = u - ep * rt(dt)
    gam = np.sqrt(rt(1.0) + u1 * u1)
    xi1 = xi + (u1 / gam) * rt(dt / dz)
    return xi1, u1


def fractions(xi0, xi1, j, rt):
    """F_j(xi1) - F_j(xi0) with F_j(x) = clamp(x - j, 0, 1)."""
    jj = np.asarray(j).astype(rt)
    one, zero = rt(1.0), rt(0.0)
    return (np.minimum(np.maximum(xi1 - jj, zero), one)
            - np.minimum(np.maximum(xi0 - jj, zero), one))


def quantized_fraction(x, j, rt):
    """F_j(x) = clamp(x - j, 0, 1) in the particle precision, rounded
    half-even to a multiple of 2^-32 and returned in 2^-32 units (int64)."""
    jj = np.asarray(j).astype(rt)
    f = np.minimum(np.maximum(x - jj, rt(0.0)), rt(1.0))
    return np.rint(f.astype(np.float64) * FIXED_SCALE).astype(np.int64)


def fixed_fractions(xi0, xi1, j, rt):
    """F_j(xi1) - F_j(xi0) with each F quantised to 2^-32 first
    (:func:`quantized_fraction`); int64 in 2^-32 units. The differences of a
    particle's quantised F telescope, so the charge it moves is conserved
    exactly in integers."""
    return quantized_fraction(xi1, j, rt) - quantized_fraction(xi0, j, rt)


def fix32_bits(nz):
    """Fractional bits of the 'fix32' position: the largest fb with
    Nz * 2^fb <= 2^31 (a sign bit stays free)."""
    return 31 - int(math.ceil(math.log2(nz)))


def gather_fix32(ez, X, fb):
    """(a2) on fixed-point positions X = xi 2^fb: h = X + 2^(fb-1),
    m = h >> fb, f = float32((h mod 2^fb) 2^-fb), then as :func:`gather`."""
    nz = ez.size
    e = np.asarray(ez, np.float64).astype(np.float32)
    X = np.asarray(X, np.int64)
    h = X + (1 << (fb - 1))
    m = h >> fb
    f = (h & ((1 << fb) - 1)).astype(np.float32) * np.float32(2.0 ** -fb)
    ia = np.clip(m - 1, 0, nz - 1)
    ib = np.clip(m, 0, nz - 1)
    return (np.float32(1.0) - f) * e[ia] + f * e[ib]


def push_fix32(X, u, ep, dt, dz, fb):
    """(a3) in 'fix32': the float32 push of :func:`push`, then the
    displacement d = (u'/gamma)(dt/dz) rounded half-even to the 2^-fb grid.
    Returns (X', u', finite) with finite = isfinite(d); X' is meaningful
    only where finite."""
    f32 = np.float32
    u1 = u - ep * f32(dt)
    gam = np.sqrt(f32(1.0) + u1 * u1)
    d = (u1 / gam) * f32(dt / dz)
    finite = np.isfinite(d)
    inc = np.rint(np.where(finite, d, f32(0.0)).astype(np.float64) * 2.0 ** fb)
    return np.asarray(X, np.int64) + inc.astype(np.int64), u1, finite


def fix32_fractions(X0, X1, j, fb):
    """F_j(X1) - F_j(X0) in 2^-32 units, exact: F_j(X) =
    clamp(X - j 2^fb, 0, 2^fb) 2^(32 - fb)."""
    one = np.int64(1) << fb
    jj = np.asarray(j, np.int64) << fb
    f1 = np.minimum(np.maximum(np.asarray(X1, np.int64) - jj, 0), one)
    f0 = np.minimum(np.maximum(np.asarray(X0, np.int64) - jj, 0), one)
    return (f1 - f0) << (32 - fb)


def deposit_fix32(nz, X0, X1, fb, brute=False):
    """(a4) in 'fix32' (int64 sums in 2^-32 units); cells floor(X0 / 2^fb)
    and floor(X1 / 2^fb), or all cells with brute=True."""
    X0 = np.asarray(X0, np.int64)
    X1 = np.asarray(X1, np.int64)
    if brute:
        j = np.arange(nz, dtype=np.int64)
        cells = np.broadcast_to(j[None, :], (X0.size, nz)).ravel()
        fr = fix32_fractions(X0[:, None], X1[:, None], j[None, :], fb).ravel()
        return accumulate(nz, cells, fr, "fixed")
    c0 = X0 >> fb
    c1 = X1 >> fb
    cross = c1 != c0
    cells = np.concatenate([c0, c1[cross]])
    x0 = np.concatenate([X0, X0[cross]])
    x1 = np.concatenate([X1, X1[cross]])
    inside = (cells >= 0) & (cells < nz)
    fr = fix32_fractions(x0[inside], x1[inside], cells[inside], fb)
    return accumulate(nz, cells[inside], fr, "fixed")


def base_weight_fix32(X, fb):
    """W_0 in 2^-32 units for fixed-point positions: sum over the base cell
    of (2^fb - X) 2^(32 - fb)."""
    X = np.asarray(X, np.int64)
    X = X[(X >= 0) & (X < (1 << fb))]
    return int((((1 << fb) - X) << (32 - fb)).sum())


def accumulate(nz, cells, frac, mode):
    """Per-cell sum of fractions: FP64 in the given order ('sum'), or the
    exact int64 sum of 2^-32-unit terms ('fixed', frac already int64)."""
    if mode == "fixed":
        acc = np.zeros(nz, np.int64)
        np.add.at(acc, cells, np.asarray(frac, np.int64))
        return acc
    acc = np.zeros(nz, np.float64)
    np.add.at(acc, cells, np.asarray(frac, np.float64))
    return acc


def deposit_fractions(nz, xi0, xi1, rt, mode="sum", brute=False):
    """(a4) Sum over particles of F_j(xi1) - F_j(xi0) for every cell j.

    The fast form visits the cells floor(xi0) and floor(xi1) only (a
    particle moves less than one cell per step, so F_j changes nowhere
    else); brute=True visits every (particle, cell) pair. Cells outside
    [0, Nz) are dropped: that current leaves the tube.
    """
    xi0 = np.asarray(xi0, rt)
    xi1 = np.asarray(xi1, rt)
    frac_of = fixed_fractions if mode == "fixed" else fractions
    if brute:
        j = np.arange(nz, dtype=np.int64)
        cells = np.broadcast_to(j[None, :], (xi0.size, nz)).ravel()
        fr = frac_of(xi0[:, None], xi1[:, None], j[None, :], rt).ravel()
        return accumulate(nz, cells, fr, mode)
    c0 = np.floor(xi0).astype(np.int64)
    c1 = np.floor(xi1).astype(np.int64)
    cross = c1 != c0
    cells = np.concatenate([c0, c1[cross]])
    x0 = np.concatenate([xi0, xi0[cross]])
    x1 = np.concatenate([xi1, xi1[cross]])
    inside = (cells >= 0) & (cells < nz)
    fr = frac_of(x0[inside], x1[inside], cells[inside], rt)
    return accumulate(nz, cells[inside], fr, mode)


def current_from(acc, s, dt, mode="sum"):
    """J^{n+1/2}_{j+1/2} = (s / dt) * (sum of fractions), FP64."""
    if mode == "fixed":
        ssum = np.asarray(acc).astype(np.float64) * (1.0 / FIXED_SCALE)
    else:
        ssum = np.asarray(acc, np.float64)
    return (s / dt) * ssum


def field_update(ez, er, b, j, dt, dz):
    """(a6) Leap-frog of Eq. 3 with R = 1 and c = 1 (FP64).

    E_z^{n+1} = E_z^n + dt B^{n+1/2} - 4 pi dt J^{n+1/2}          (cells)
    E_r^{n+1}_j = E_r^n_j - (dt/dz)(B_{j+1/2} - B_{j-1/2})         (nodes 1..Nz)
    B^{n+3/2} = B^{n+1/2} - (dt/dz)(E_r,j+1 - E_r,j) - dt E_z^{n+1} (cells)
    E_r at node 0 stays 0 (phi = 0 on the conducting base); the top node
    uses the ghost B_{Nz+1/2} = B_{Nz-1/2} (phi' = 0 at the top).
    Returns new (ez, er, b).
    """
    cdt = dt / dz
    fourpi_dt = 4.0 * math.pi * dt
    ez1 = ez + dt * b - fourpi_dt * j
    bext = np.concatenate([b, b[-1:]])
    er1 = er.copy()
    er1[1:] = er[1:] - cdt * (bext[1:] - bext[:-1])
    b1 = b - cdt * (er1[1:] - er1[:-1]) - dt * ez1
    return ez1, er1, b1


def rho_nodes(xi, s, dz, nz):
    """Cloud-in-cell charge density at nodes 0..Nz (FP64):
    rho_j = sum_p s max(0, 1 - |xi_p - j|) / dz."""
    xi = np.asarray(xi, np.float64)
    rho = np.zeros(nz + 1)
    if xi.size:
        j = np.floor(xi).astype(np.int64)
        w = xi - j
        np.add.at(rho, j, s * (1.0 - w) / dz)
        np.add.at(rho, np.minimum(j + 1, nz), s * w / dz)
    return rho


# ---------------------------------------------------------------------------
# The tube
# ---------------------------------------------------------------------------

class Tube:
    """State and time step of one tube (Sec. 2, Figure A).

    Particles are kept in ID order: injection appends, removal keeps the
    order of the survivors. IDs count every particle ever added.
    """

    def __init__(self, nz, L, dt, rho_gj, s, *, capacity=None,
                 precision="f64", accumulate="sum", deposit="fast"):
        if precision not in ("f64", "f32", "fix32"):
            raise ValueError(precision)
        if precision == "fix32" and accumulate != "fixed":
            raise ValueError("'fix32' positions deposit exact fixed-point fractions")
        if accumulate not in ("sum", "fixed"):
            raise ValueError(accumulate)
        if deposit not in ("fast", "brute"):
            raise ValueError(deposit)
        self.nz = int(nz)
        self.L = float(L)
        self.dz = self.L / self.nz
        self.dt = float(dt)
        if not (0.0 < self.dt < self.dz):
            raise ValueError("need 0 < dt < dz (c = 1)")
        self.rho_gj = np.asarray(rho_gj, dtype=np.float64).copy()
        if self.rho_gj.size != self.nz + 1:
            raise ValueError("rho_gj needs Nz + 1 node values")
        self.s = float(s)
        if not self.s < 0.0:
            raise ValueError("macro charge s must be negative (electrons)")
        self.capacity = capacity
        self.precision = precision
        self.accumulate = accumulate
        self.brute = deposit == "brute"
        self.rt = np.float64 if precision == "f64" else np.float32
        self.fix = precision == "fix32"
        self.fb = fix32_bits(self.nz) if self.fix else 0

        self.ez, self.er, self.b, self.phi0 = initial_fields(self.rho_gj, self.dz)
        self.j = np.zeros(self.nz)          # J^{n+1/2} of the last step
        self.xi = np.zeros(0, np.int64 if self.fix else self.rt)   # X in 'fix32'
        self.u = np.zeros(0, self.rt)
        self.ids = np.zeros(0, np.int64)
        self.w0 = 0                         # W_0 in 2^-32 units
        self.surface_field = 0.0
        self.total_injected = 0
        self.step_count = 0
        self.capacity_hit = False
        self.nonfinite = False
        self.last_injected = 0
        self.last_removed = 0

    # -- particles ---------------------------------------------------------
    def add_particles(self, z, u):
        """Append particles at heights z (in R) with u = gamma beta;
        xi = z / dz is computed in FP64 and rounded to the precision."""
        z = np.asarray(z, np.float64)
        if self.fix:
            xi = np.rint(z / self.dz * 2.0 ** self.fb).astype(np.int64)
        else:
            xi = (z / self.dz).astype(self.rt)
        uu = np.asarray(u, np.float64).astype(self.rt)
        n = xi.size
        self.xi = np.concatenate([self.xi, xi])
        self.u = np.concatenate([self.u, uu])
        self.ids = np.concatenate(
            [self.ids, self.total_injected + np.arange(n, dtype=np.int64)])
        self.total_injected += n
        self.w0 = self._base_weight()

    def _base_weight(self):
        if self.fix:
            return base_weight_fix32(self.xi, self.fb)
        return base_weight_fixed(self.xi, self.rt)

    def solve_fields(self, rho=None):
        """Eq. 4 with the tube's current charge: phi'' - phi = -4 pi (rho - rho_GJ)
        with rho the cloud-in-cell density of the particles at the nodes,
        phi(0) = 0, phi'(L) = 0; E_z = -phi', E_r = phi, B_phi = 0 (the
        Sec. 2 initialisation applied to a prefilled tube). `rho` replaces
        the tube's own density, for a state held outside the tube (e.g. the
        sum of rho_nodes over chunks of a very large one)."""
        if rho is None:
            rho = self.rho_nodes()
        rho = np.asarray(rho, np.float64)
        phi = poisson_potential(self.rho_gj - rho, self.dz)
        self.ez = -(phi[1:] - phi[:-1]) / self.dz
        self.er = phi.copy()
        self.b = np.zeros(self.nz)

    def injection_count(self):
        """N_inj for the current state (see :func:`injection_count`)."""
        n, es = injection_count(self.ez[0], self.w0, self.s, self.dz,
                                self.rho_gj[0])
        self.surface_field = es
        return n

    def inject(self):
        """(a1) Append N_inj electrons at z = 0 with u = 0."""
        n_inj = self.injection_count()
        if self.capacity is not None and self.xi.size + n_inj > self.capacity:
            n_inj = max(0, self.capacity - self.xi.size)
            self.capacity_hit = True
        self.xi = np.concatenate([self.xi, np.zeros(n_inj, self.xi.dtype)])
        self.u = np.concatenate([self.u, np.zeros(n_inj, self.rt)])
        self.ids = np.concatenate(
            [self.ids, self.total_injected + np.arange(n_inj, dtype=np.int64)])
        self.total_injected += n_inj
        self.last_injected = n_inj
        self.w0 += n_inj * int(FIXED_SCALE)      # each new particle has W_0 = 1
        return n_inj

    # -- one step --------------------------------------------------------------
    def step(self):
        """(a1)-(a6) once, in the order of Figure A."""
        rt = self.rt
        self.inject()                                              # (a1)
        xi0, u0 = self.xi, self.u
        if self.fix:
            fb = self.fb
            ep = gather_fix32(self.ez, xi0, fb)                    # (a2)
            xi1, u1, finite = push_fix32(xi0, u0, ep, self.dt, self.dz, fb)   # (a3)
            if not np.all(finite):
                self.nonfinite = True
            acc = deposit_fix32(self.nz, xi0[finite], xi1[finite], fb,         # (a4)
                                self.brute)
            self.j = current_from(acc, self.s, self.dt, "fixed")
            alive = finite & (xi1 >= 0) & (xi1 < (self.nz << fb))  # (a5)
            self.last_removed = int(xi1.size - np.count_nonzero(alive))
        else:
            ep = gather(self.ez, xi0, rt)                          # (a2)
            xi1, u1 = push(xi0, u0, ep, self.dt, self.dz, rt)      # (a3)
            acc = deposit_fractions(self.nz, xi0, xi1, rt,         # (a4)
                                    self.accumulate, self.brute)
            self.j = current_from(acc, self.s, self.dt, self.accumulate)
            finite = np.isfinite(xi1) & np.isfinite(u1)
            if not np.all(finite):
                self.nonfinite = True
            alive = finite & (xi1 >= 0) & (xi1 < rt(self.nz))      # (a5)
            self.last_removed = int(xi1.size - np.count_nonzero(alive))
        self.xi, self.u, self.ids = xi1[alive], u1[alive], self.ids[alive]
        self.w0 = self._base_weight()
        self.ez, self.er, self.b = field_update(                   # (a6)
            self.ez, self.er, self.b, self.j, self.dt, self.dz)
        self.step_count += 1

    def run(self, nsteps):
        for _ in range(int(nsteps)):
            self.step()

    # -- diagnostics -----------------------------------------------------------
    def cells(self):
        """Particle positions in cell units (FP64)."""
        if self.fix:
            return self.xi.astype(np.float64) * 2.0 ** -self.fb
        return self.xi.astype(np.float64)

    def z(self):
        """Particle heights in R (FP64)."""
        return self.cells() * self.dz

    def gamma(self):
        u = self.u.astype(np.float64)
        return np.sqrt(1.0 + u * u)

    def rho_nodes(self):
        return rho_nodes(self.cells(), self.s, self.dz, self.nz)

    def gauss_residual(self):
        """G_j = (E_{j+1/2} - E_{j-1/2})/dz + E_r,j - 4 pi (rho_j - rho_GJ,j)
        on the interior nodes 1..Nz-1 (Eq. 2 with d/dr -> 1/R, R = 1)."""
        rho = self.rho_nodes()
        return ((self.ez[1:] - self.ez[:-1]) / self.dz + self.er[1:-1]
                - 4.0 * math.pi * (rho[1:-1] - self.rho_gj[1:-1]))
