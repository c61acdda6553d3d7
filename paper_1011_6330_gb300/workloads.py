"""Named tube configurations used by the tests and the benchmark.

Each returns keyword arguments for ``binding.default_params``.
"""

from __future__ import annotations

import math

import numpy as np

from . import binding as B

M_SUN = 1.98847e33


def flat_sclf_small(precision=B.SCLF_FP64, accumulate=B.SCLF_ACC_FP64, capacity=1 << 17):
    """Flat-space SCLF tube: R = 1, L = 8 R, Nz = 1024, rho_GJ = -1 in code
    units (Lambda = sqrt(4 pi)), dt = 0.4 dz, macro charge giving 5e4
    particles for a tube full of rho_GJ."""
    nz, L = 1024, 8.0
    dz = L / nz
    return dict(L_over_R=L, Nz=nz, dt=0.4 * dz, rho_gj_mode=B.SCLF_RHO_USER,
                rho_gj_user=-np.ones(nz + 1), target_particles=50000,
                capacity=capacity, precision=precision, accumulate=accumulate,
                track_ids=1)


def gr_tube(B_G=1e12, P_s=0.5, Rstar_cm=1e6, incl=0.5, Nz=65536, n_particles=10 ** 8,
            capacity=None, precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64,
            track_ids=0):
    """Frame-dragging tube of a pulsar: R = R_* sqrt(R_* Omega / c), length
    2 R_*, GR rho_GJ (Eq. 6-7) at inclination incl, dt from the default
    rule, macro charge so that n_particles carry rho_GJ(0) over the tube."""
    omega = 2.0 * math.pi / P_s
    theta_p = math.sqrt(omega * Rstar_cm / 2.99792458e10)
    L = 2.0 / theta_p                          # 2 R_* in units of R = R_* theta_p
    if capacity is None:
        capacity = int(n_particles * 1.02) + (1 << 20)
    return dict(B_G=B_G, P_s=P_s, Rstar_cm=Rstar_cm, incl_rad=incl, mass_g=1.4 * M_SUN,
                R_cm=0.0, L_over_R=L, Nz=Nz, dt=0.0, rho_gj_mode=B.SCLF_RHO_GR,
                target_particles=n_particles, capacity=capacity, precision=precision,
                accumulate=accumulate, track_ids=track_ids)


def large_tube(n_particles=2 ** 30, Nz=2 ** 20, capacity=None, track_ids=0):
    """Large single frame-dragging tube: B = 3e12 G, P = 0.1 s, R_* = 10 km,
    length 2 R_*, Nz = 2^20, GR rho_GJ at i = 0.5, 2^30 particles with
    32-bit fixed-point positions (SCLF_FIX32) and float32 momenta -- 8 bytes
    per particle, uniform 2^-11-cell position resolution."""
    return gr_tube(B_G=3e12, P_s=0.1, Rstar_cm=1e6, incl=0.5, Nz=Nz,
                   n_particles=n_particles, capacity=capacity,
                   precision=B.SCLF_FIX32, accumulate=B.SCLF_ACC_FIXED64,
                   track_ids=track_ids)


def adjoint_tube(n_particles=10 ** 6, Nz=16384, precision=B.SCLF_FP32):
    """Frame-dragging tube of a B = 1e12 G, P = 0.3 s pulsar (R_* = 10 km,
    length 2 R_*, GR rho_GJ at i = 0.5) with Nz = 16384 and 1e6 FP32
    macro-electrons, for gradients of a 2000-step run checkpointed every
    100 steps. dt and R are fixed explicitly (their derived values) so that
    perturbing (B, P, R) leaves the grid alone."""
    kw = gr_tube(B_G=1e12, P_s=0.3, Nz=Nz, n_particles=n_particles, precision=precision,
                 accumulate=B.SCLF_ACC_FIXED64)
    d = B.derive(B.default_params(**kw))
    kw.update(dt=d["dt"], R_cm=d["R_cm"])
    return kw


def death_line_batch(n_tubes=256, seed=0, nz_min=1024, nz_max=16384, n_min=10 ** 5,
                     n_max=2 * 10 ** 6, precision=B.SCLF_FIX32):
    """Batch of independent pulsar tubes for death-line / pair-front sweeps:
    P log-uniform in [0.03, 3] s, B log-uniform in [1e11, 1e13] G (seeded),
    frame-dragging rho_GJ (i = 0.5) for even tubes and flat (i = 0) for odd
    ones, tube length 2 R_*; Nz grows with the tube length (in R) from
    nz_min to nz_max (log scale, multiple of 64) and the particle count with
    Nz from n_min to n_max. Positions are 32-bit fixed point by default
    (with float32 positions these tubes' E_z is 7-45 % off FP64 after 2000
    steps: the per-step displacement, 1e-4 to 7e-3 cell, is comparable to the
    float32 spacing of the upper cells). Returns a list of keyword dicts."""
    rng = np.random.default_rng(seed)
    P = 10.0 ** rng.uniform(math.log10(0.03), math.log10(3.0), n_tubes)
    Bf = 10.0 ** rng.uniform(11.0, 13.0, n_tubes)
    c = 2.99792458e10
    L = [2.0 / math.sqrt(2.0 * math.pi / p * 1e6 / c) for p in P]
    lmin, lmax = 2.0 / math.sqrt(2.0 * math.pi / 0.03 * 1e6 / c), 2.0 / math.sqrt(2.0 * math.pi / 3.0 * 1e6 / c)
    out = []
    for i in range(n_tubes):
        frac = (math.log(L[i]) - math.log(lmin)) / (math.log(lmax) - math.log(lmin))
        nz = int(round(nz_min * (nz_max / nz_min) ** frac / 64.0)) * 64
        nz = min(max(nz, nz_min), nz_max)
        npart = int(n_min * (n_max / n_min) ** ((math.log(nz) - math.log(nz_min)) /
                                                (math.log(nz_max) - math.log(nz_min))))
        gr = i % 2 == 0
        kw = gr_tube(B_G=float(Bf[i]), P_s=float(P[i]), incl=0.5 if gr else 0.0, Nz=nz,
                     n_particles=npart, capacity=int(npart * 1.05) + 8192, precision=precision)
        kw["rho_gj_mode"] = B.SCLF_RHO_GR if gr else B.SCLF_RHO_FLAT
        kw["compact_interval"] = 64
        out.append(kw)
    return out
