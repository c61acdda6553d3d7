"""Seeded synthetic inputs (shared by the tests, the benchmark and users).

Holds no arithmetic of the simulation method: it only draws particle
positions and momenta from stated distributions, with numpy's PCG64
generator seeded by the caller.
"""

from __future__ import annotations

import numpy as np


def stratified_heights(n, L, seed, order="descending"):
    """n heights in [0, L): one uniform draw in each of n equal strata.

    order='descending' lists them from the top of the tube down (the order
    in which a beam injected at the base carries its oldest electrons
    first); 'shuffled' permutes them with the same generator.
    """
    rng = np.random.default_rng(seed)
    k = np.arange(n, dtype=np.float64)
    z = L * (1.0 - (k + rng.random(n)) / n)          # strictly inside (0, L]
    z = np.minimum(z, np.nextafter(L, 0.0))
    if order == "shuffled":
        z = z[rng.permutation(n)]
    elif order != "descending":
        raise ValueError(order)
    return z


def gamma_ramp(z, gamma_far, scale=1.0, eta_of_z=None):
    """A smooth acceleration profile used to fill a tube before a run:
    gamma(z) = 1 + gamma_far * g(z) * (1 - exp(-z / scale)), where
    g = 1 - eta^-3 when eta_of_z is given (frame-dragging shape) else 1."""
    z = np.asarray(z, dtype=np.float64)
    shape = 1.0 - np.exp(-z / scale)
    if eta_of_z is not None:
        eta = eta_of_z(z)
        shape = shape * (1.0 - eta ** -3)
    return 1.0 + gamma_far * shape


def prefilled_beam(n, L, gamma_far, seed, order="descending", jitter=0.01,
                   eta_of_z=None):
    """(z, u) of n electrons spread uniformly over [0, L) (pass the filled
    height, e.g. the tube length less one cell, so that no height rounds to
    the top of the tube in float32) with
    u = sqrt(gamma^2 - 1), gamma from :func:`gamma_ramp` with a relative
    Gaussian jitter (clipped at gamma >= 1)."""
    z = stratified_heights(n, L, seed, order)
    rng = np.random.default_rng(seed + 1)
    g = gamma_ramp(z, gamma_far, eta_of_z=eta_of_z)
    g = np.maximum(g * (1.0 + jitter * rng.standard_normal(n)), 1.0)
    u = np.sqrt(g * g - 1.0)
    return z, u


def random_particles(n, L, seed, u_sigma=0.5):
    """n particles uniform in [0, L) with Gaussian u (both directions)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(0.0, L, n)
    u = rng.normal(0.0, u_sigma, n)
    return z, u


def prefilled_beam_chunks(n, L, gamma_far, seed, chunk=1 << 24, jitter=0.01,
                          eta_of_z=None):
    """The state of :func:`prefilled_beam` (descending stratified heights,
    ramp momenta with jitter) generated in chunks of `chunk` particles so
    that large tubes fit in host memory; chunk c draws from
    default_rng([seed, c]). Yields (z, u) in ID order."""
    for c, k0 in enumerate(range(0, n, chunk)):
        m = min(chunk, n - k0)
        rng = np.random.default_rng([seed, c])
        k = np.arange(k0, k0 + m, dtype=np.float64)
        z = L * (1.0 - (k + rng.random(m)) / n)
        z = np.minimum(z, np.nextafter(L, 0.0))
        g = gamma_ramp(z, gamma_far, eta_of_z=eta_of_z)
        g = np.maximum(g * (1.0 + jitter * rng.standard_normal(m)), 1.0)
        yield z, np.sqrt(g * g - 1.0)
