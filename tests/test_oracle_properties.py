"""Property tests of the oracle's deposit (CPU; skipped where hypothesis is
not installed): on random small states the two-cell deposit equals the
all-pairs sum exactly, each particle's fixed-point fractions telescope to the
change of its quantised position, and the current and the cloud-in-cell
charge satisfy discrete continuity (Sec. 2's charge-conserving weighting)."""

import numpy as np
import pytest

import oracle as orc

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings


def _state(nz, seed, n, reach):
    """n particles in [0, nz) moved by at most `reach` cells (some leave)."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.0, nz, n)
    x0[: n // 8] = np.floor(x0[: n // 8])                # some exactly on nodes
    x1 = x0 + rng.uniform(-reach, reach, n)
    return x0, x1


@settings(max_examples=60, deadline=None)
@given(nz=st.integers(2, 40), seed=st.integers(0, 2 ** 31), n=st.integers(1, 200),
       prec=st.sampled_from([np.float64, np.float32]))
def test_two_cell_deposit_equals_all_pairs(nz, seed, n, prec):
    x0, x1 = _state(nz, seed, n, 0.999)
    x0, x1 = x0.astype(prec), x1.astype(prec)
    fast = orc.deposit_fractions(nz, x0, x1, prec, "fixed")
    brute = orc.deposit_fractions(nz, x0, x1, prec, "fixed", brute=True)
    assert np.array_equal(fast, brute)


@settings(max_examples=60, deadline=None)
@given(nz=st.integers(2, 40), seed=st.integers(0, 2 ** 31), n=st.integers(1, 200))
def test_fixed_point_fractions_telescope_per_particle(nz, seed, n):
    """Sum over all cells of a particle's quantised F_j differences equals
    Q(x1) - Q(x0), Q(x) = sum_j q(clamp(x - j)) -- the integer charge it
    moved, whatever the cells in between."""
    x0, x1 = _state(nz, seed, n, 0.999)
    j = np.arange(nz)
    for a, b in zip(x0, x1):
        moved = int(np.sum(orc.fixed_fractions(np.full(nz, a), np.full(nz, b), j, np.float64)))
        qa = int(np.sum(orc.quantized_fraction(np.full(nz, a), j, np.float64)))
        qb = int(np.sum(orc.quantized_fraction(np.full(nz, b), j, np.float64)))
        assert moved == qb - qa


@settings(max_examples=40, deadline=None)
@given(nz=st.integers(4, 40), seed=st.integers(0, 2 ** 31), n=st.integers(1, 300))
def test_current_and_charge_satisfy_discrete_continuity(nz, seed, n):
    """(rho^{n+1}_j - rho^n_j) dz + dt (J_{j+1/2} - J_{j-1/2}) = 0 on the
    interior nodes for particles that stay inside the tube (FP64, exact
    fractions)."""
    x0, x1 = _state(nz, seed, n, 0.4)
    inside = (x1 >= 0.0) & (x1 < nz)
    x0, x1 = x0[inside], x1[inside]
    s, dt, dz = -1e-3, 0.01, 0.05
    acc = orc.deposit_fractions(nz, x0, x1, np.float64, "sum")
    jc = orc.current_from(acc, s, dt, "sum")
    r0, r1 = orc.rho_nodes(x0, s, dz, nz), orc.rho_nodes(x1, s, dz, nz)
    res = (r1[1:-1] - r0[1:-1]) * dz + dt * (jc[1:] - jc[:-1])
    scale = max(float(np.max(np.abs(r0))) * dz, 1e-300)
    assert np.max(np.abs(res)) <= 1e-12 * scale * max(n, 1)
