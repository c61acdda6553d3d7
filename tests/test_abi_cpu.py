"""The C ABI library on a machine without a GPU: it builds, loads, exports
every function include/sclf_tube.h declares, and its host-only calls
(parameter defaults, unit derivation, workspace sizing) behave."""

import math
import os

import numpy as np
import pytest

import oracle as orc
from paper_1011_6330_gb300 import binding as B
from paper_1011_6330_gb300 import workloads


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        from paper_1011_6330_gb300 import build
        build.build()
    return B.load()


def test_every_declared_function_is_exported(lib):
    names = B.header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.SIGNATURES), set(names) ^ set(B.SIGNATURES)


def test_version_and_error_strings(lib):
    assert b"sm_103a" in lib.tube_version()
    assert b"bounds-checked" not in lib.tube_version()
    for code in range(0, -9, -1):
        assert lib.tube_strerror(code) and lib.tube_strerror(code) != b"unknown error"
    assert lib.tube_strerror(-99) == b"unknown error"


def test_bounds_checked_build_exports_the_same_calls(lib):
    """libsclf_tube_checked.so (-DSCLF_CHECKED) exports every declared call
    and says what it is."""
    import ctypes
    if not os.path.exists(B.LIB_CHECKED_PATH):
        from paper_1011_6330_gb300 import build
        build.build(checked=True)
    chk = ctypes.CDLL(B.LIB_CHECKED_PATH)
    for n in B.header_functions():
        assert hasattr(chk, n), n
    chk.tube_version.restype = ctypes.c_char_p
    assert b"bounds-checked" in chk.tube_version()


def test_defaults_are_the_standard_pulsar(lib):
    p = B.default_params()
    assert (p.B_G, p.P_s, p.Rstar_cm) == (1e12, 1.0, 1e6)
    d = B.derive(p)
    cu = orc.code_units(1e12, 1.0, 1e6, 0.0, 1.4 * orc.M_SUN)
    # two independent restatements of the Sec. 3 / Eq. 7 formulas
    for k in ("theta_p", "R_cm", "n0", "omega_p0", "Lambda0", "kappa", "theta_star"):
        assert abs(d[k] / cu[k] - 1.0) < 1e-12, k
    assert d["rho0"] == pytest.approx(-cu["Lambda0"] ** 2 / (4 * math.pi), rel=1e-13)
    assert d["dt"] == pytest.approx(min(0.4 * d["dz"], 0.2 / d["Lambda0"]), rel=0)


def test_gr_workload_units(lib):
    p = B.default_params(**workloads.gr_tube())
    d = B.derive(p)
    cu = orc.code_units(1e12, 0.5, 1e6, 0.5, 1.4 * orc.M_SUN)
    assert abs(d["Lambda0"] / cu["Lambda0"] - 1) < 1e-12
    assert abs(d["L"] - 2.0 / cu["theta_p"]) < 1e-9          # 2 R_*
    z0 = orc.rho_gj_profile(orc.RHO_GR, 0.0, cu["Lambda0"], 0.5, cu["theta_star"],
                            cu["R_over_Rstar"], cu["kappa"])
    assert abs(d["rho0"] / z0 - 1) < 1e-13
    assert d["s"] == pytest.approx(-abs(z0) * d["L"] / 1e8, rel=1e-13)
    assert 0 < d["dt"] < d["dz"]
    # the oracle's own dt rule and macro charge give the numbers the parity
    # tests hand to both sides
    L_o = 2.0 / cu["theta_p"]
    assert d["dt"] == pytest.approx(orc.default_dt(L_o / 65536, cu["Lambda0"]), rel=1e-12)
    assert d["s"] == pytest.approx(orc.macro_charge_for(z0, L_o, 10 ** 8), rel=1e-12)
    kw1 = workloads.flat_sclf_small()
    d1 = B.derive(B.default_params(**kw1))
    assert d1["dt"] == pytest.approx(0.4 * 8.0 / 1024, rel=1e-15)
    assert d1["s"] == pytest.approx(orc.macro_charge_for(-1.0, 8.0, 50000), rel=1e-12)


def test_invalid_parameters_are_rejected(lib):
    kw = workloads.flat_sclf_small()
    for bad in (dict(dt=kw["L_over_R"] / kw["Nz"]),       # c dt = dz
                dict(Nz=1), dict(capacity=-1), dict(precision=7),
                dict(accumulate=3), dict(rho_gj_mode=9), dict(L_over_R=0.0),
                dict(push_stages=-1), dict(push_stages=5),
                dict(launch_overlap=-2), dict(launch_overlap=2)):
        p = B.default_params(**{**kw, **bad})
        with pytest.raises(B.SclfError) as e:
            B.derive(p)
        assert e.value.code == -1
    p = B.default_params(**{**kw, "macro_charge": 0.5})
    with pytest.raises(B.SclfError):
        B.derive(p)


def test_workspace_grows_with_capacity_and_grid(lib):
    a = B.workspace_bytes(B.default_params(**workloads.flat_sclf_small(capacity=1 << 16)))
    b = B.workspace_bytes(B.default_params(**workloads.flat_sclf_small(capacity=1 << 18)))
    assert b - a >= 3 * (1 << 16) * 8 * 2          # xi, u (FP64) + ids
    g = B.workspace_bytes(B.default_params(**workloads.gr_tube()))
    assert g >= 2 * 4 * 10 ** 8                     # FP32 xi and u of 1e8 slots
    assert g < 2 * 4 * 10 ** 8 * 1.1 + 64 * 2 ** 20


def test_adjoint_create_validates_before_touching_the_device():
    """adjoint_create rejects FP64 atomics (the recompute must reproduce the
    run bit for bit), bad checkpoint intervals and odd run lengths with
    SCLF_EINVAL before any CUDA call (checkpoint_every = 0 asks the library
    to choose)."""
    import ctypes as C
    lib = B.load()
    h = C.c_void_p()
    for kw, n, k in ((dict(precision=B.SCLF_FP64, accumulate=B.SCLF_ACC_FP64), 100, 10),
                     (dict(accumulate=B.SCLF_ACC_FP64), 100, 10),
                     (dict(), 100, 7), (dict(), 100, -2), (dict(), 105, 10), (dict(), 0, 10),
                     (dict(), 101, 0)):
        p = B.default_params(**kw)
        assert lib.adjoint_create(C.byref(p), n, k, None, C.byref(h)) == -1
    assert lib.adjoint_backward(None, 0, None, None) == -1
    assert lib.adjoint_forward(None, None) == -1


@pytest.mark.parametrize("variant,alpha,tables", [
    (B.SCLF_GR_COS, 0, False), (B.SCLF_GR_BOTH, 0, False),
    (B.SCLF_GR_COS, 1, False), (B.SCLF_GR_BOTH, 1, True), (B.SCLF_GR_COS, 0, True)])
def test_host_rho_gj_profile_matches_oracle_eq6_variants(variant, alpha, tables):
    """The library's host rho_GJ builder (Eq. 6 variants: Omega -> Omega - omega
    on the cos term or on both, redshift alpha, f and H tables) against the
    oracle's profile at every node."""
    kw = workloads.gr_tube(B_G=1e12, P_s=0.3, Nz=2048, n_particles=10 ** 5)
    nz, L = kw["Nz"], kw["L_over_R"]
    cu = orc.code_units(kw["B_G"], kw["P_s"], kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
    z = np.arange(nz + 1) * (L / nz)
    eta = 1.0 + z * cu["R_over_Rstar"]
    f = 1.0 + 0.2 * (1.0 - 1.0 / eta) if tables else None
    H = 1.0 - 0.1 * (1.0 - 1.0 / eta) if tables else None
    rho = B.rho_gj_profile(B.default_params(**kw, gr_variant=variant, gr_alpha=alpha, gr_f=f, gr_H=H))
    ref = orc.rho_gj_profile(orc.RHO_GR, z, cu["Lambda0"], kw["incl_rad"], cu["theta_star"],
                             cu["R_over_Rstar"], cu["kappa"],
                             variant="both" if variant == B.SCLF_GR_BOTH else "cos", f=f, H=H,
                             rg_over_Rstar=cu["rg_over_Rstar"] if alpha else None)
    assert np.max(np.abs(rho - ref)) <= 1e-13 * np.max(np.abs(ref))
    d = B.derive(B.default_params(**kw, gr_variant=variant, gr_alpha=alpha, gr_f=f, gr_H=H))
    assert abs(d["rho0"] - ref[0]) <= 1e-13 * abs(ref[0])


def test_eq6_parameters_are_validated():
    import ctypes as C
    lib = B.load()
    kw = workloads.gr_tube(Nz=64, n_particles=1000)
    d = B.TubeDerived()
    for bad in (dict(gr_variant=2), dict(gr_alpha=3), dict(gr_f=np.zeros(65)),
                dict(gr_H=np.full(65, np.nan))):
        p = B.default_params(**kw, **bad)
        assert lib.tube_derive(C.byref(p), C.byref(d)) == -1, bad


@pytest.mark.parametrize("mode,variant,alpha,tables,override", [
    (B.SCLF_RHO_FLAT, B.SCLF_GR_COS, 0, False, 0.0),
    (B.SCLF_RHO_GR, B.SCLF_GR_COS, 0, False, 0.0),
    (B.SCLF_RHO_GR, B.SCLF_GR_BOTH, 1, True, 0.0),
    (B.SCLF_RHO_GR, B.SCLF_GR_COS, 1, False, 0.0),
    (B.SCLF_RHO_GR, B.SCLF_GR_COS, 0, True, 3.0e4)])
def test_rho_gj_param_gradient_is_the_derivative_of_the_host_profile(
        lib, mode, variant, alpha, tables, override):
    """tube_rho_gj_param_gradient (the analytic chain from rho_GJ to B, P, R
    the adjoint uses) against central differences of the library's own host
    profile (tube_rho_gj_profile) at fixed R, for the flat profile and the
    Eq. 6 variants; with Lambda0 overridden only theta_* and eta move; and for
    the default frame-dragging profile against the oracle's analytic
    Jacobian."""
    kw = workloads.gr_tube(B_G=1e12, P_s=0.3, Nz=1024, n_particles=10 ** 5)
    kw.update(rho_gj_mode=mode, lambda_override=override)
    d0 = B.derive(B.default_params(**kw))
    kw.update(R_cm=d0["R_cm"], dt=d0["dt"], macro_charge=d0["s"])
    nz, L = kw["Nz"], kw["L_over_R"]
    z = np.arange(nz + 1) * (L / nz)
    eta = 1.0 + z * d0["R_over_Rstar"]
    if tables:
        kw.update(gr_f=1.0 + 0.2 * (1.0 - 1.0 / eta), gr_H=1.0 - 0.1 * (1.0 - 1.0 / eta))
    kw.update(gr_variant=variant, gr_alpha=alpha)
    rng = np.random.default_rng(7)
    w = rng.normal(size=nz + 1)
    g = B.rho_gj_param_gradient(B.default_params(**kw), w)
    for k, name in enumerate(("B_G", "P_s", "R_cm")):
        h = 1e-5 * kw[name]
        rp = B.rho_gj_profile(B.default_params(**{**kw, name: kw[name] + h}))
        rm = B.rho_gj_profile(B.default_params(**{**kw, name: kw[name] - h}))
        fd = float(w @ (rp - rm)) / (2.0 * h)
        assert abs(g[k] - fd) <= 1e-7 * max(abs(fd), 1e-30) + 1e-12 * abs(g).max(), (name, g[k], fd)
    if override:
        assert g[0] == 0.0
    if mode == B.SCLF_RHO_GR and variant == B.SCLF_GR_COS and not alpha and not tables:
        from oracle import adjoint as oadj
        jac = oadj.rho_gj_parameter_jacobian(orc.RHO_GR, z, kw["B_G"], kw["P_s"], kw["R_cm"],
                                              kw["Rstar_cm"], kw["incl_rad"], kw["mass_g"])
        for k, key in enumerate("BPR"):
            assert g[k] == pytest.approx(float(w @ jac[key]), rel=1e-11)


def test_rho_gj_param_gradient_of_a_user_profile_is_zero(lib):
    kw = workloads.flat_sclf_small()
    g = B.rho_gj_param_gradient(B.default_params(**kw), np.ones(kw["Nz"] + 1))
    assert np.array_equal(g, np.zeros(3))


def test_velocity_selftest_validates_its_range_without_a_device(lib):
    import ctypes as C
    n, first = C.c_uint64(7), C.c_uint32(7)
    assert lib.tube_selftest_velocity(1, 1 << 32, C.byref(n), C.byref(first)) == -1
    assert lib.tube_selftest_velocity(0, 1, None, C.byref(first)) == -1
    assert lib.tube_selftest_velocity(5, 0, C.byref(n), C.byref(first)) == 0
    assert n.value == 0 and first.value == 0xffffffff


def test_decomposed_tube_validates_before_touching_the_device(lib):
    """dtube_create rejects bad sub-domain counts, cuts that do not cover
    [0, Nz) in ranges of at least 2 cells, and the FP64-atomic current, with
    SCLF_EINVAL before any CUDA call."""
    import ctypes as C
    kw = workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64)
    p = B.default_params(**kw)
    out = C.c_void_p()
    for n in (0, 65):
        assert lib.dtube_create(C.byref(p), n, None, C.byref(out)) == -1
    for cuts in ([1, 512, 1024], [0, 512, 1000], [0, 1, 1024], [0, 600, 500, 1024],
                 [0, 1023, 1024]):
        c = np.array(cuts, dtype=np.int64)
        assert lib.dtube_create(C.byref(p), len(cuts) - 1, c.ctypes.data_as(B._pi64),
                                C.byref(out)) == -1, cuts
    p64 = B.default_params(**dict(kw, accumulate=B.SCLF_ACC_FP64))
    assert lib.dtube_create(C.byref(p64), 2, None, C.byref(out)) == -1
    assert not out.value
