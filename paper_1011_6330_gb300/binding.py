"""Thin Python binding of the sclf_tube C ABI (include/sclf_tube.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library. PyTorch provides the device workspace (its caching allocator) and
the stream (``torch.cuda.current_stream()``). Loading fails loudly when the
in-tree library has not been built; there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB_PATH = os.path.join(PKG, "libsclf_tube.so")
# The bounds-checked build of the same library (tests load it in a separate
# process through SCLF_TUBE_LIB).
LIB_CHECKED_PATH = os.path.join(PKG, "libsclf_tube_checked.so")
HEADER = os.path.join(ROOT, "include", "sclf_tube.h")

SCLF_RHO_FLAT, SCLF_RHO_GR, SCLF_RHO_USER = 0, 1, 2
SCLF_GR_COS, SCLF_GR_BOTH = 0, 1
SCLF_FP32, SCLF_FP64, SCLF_FIX32 = 0, 1, 2
SCLF_ACC_FIXED64, SCLF_ACC_FP64 = 0, 1
FLAG_CAPACITY, FLAG_NONFINITE, FLAG_TIMEOUT, FLAG_BOUNDS = 1, 2, 4, 8
SCLF_OBJ_GAMMA, SCLF_OBJ_EZ, SCLF_OBJ_EZ_WEIGHTED = 0, 1, 2


class TubeParams(C.Structure):
    _fields_ = [
        ("B_G", C.c_double), ("P_s", C.c_double), ("Rstar_cm", C.c_double),
        ("incl_rad", C.c_double), ("mass_g", C.c_double), ("R_cm", C.c_double),
        ("L_over_R", C.c_double), ("Nz", C.c_int64), ("dt", C.c_double),
        ("rho_gj_mode", C.c_int32), ("precision", C.c_int32),
        ("rho_gj_user", C.POINTER(C.c_double)),
        ("lambda_override", C.c_double), ("macro_charge", C.c_double),
        ("target_particles", C.c_int64), ("capacity", C.c_int64),
        ("accumulate", C.c_int32), ("track_ids", C.c_int32),
        ("compact_interval", C.c_int32), ("use_graphs", C.c_int32),
        ("gr_variant", C.c_int32), ("gr_alpha", C.c_int32),
        ("gr_f", C.POINTER(C.c_double)), ("gr_H", C.POINTER(C.c_double)),
        ("sort_interval", C.c_int32), ("push_stages", C.c_int32),
        ("launch_overlap", C.c_int32),
    ]


class TubeDerived(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "Omega", "theta_p", "R_cm", "n0", "omega_p0", "Lambda0", "kappa",
        "theta_star", "R_over_Rstar", "L", "dz", "dt", "s", "rho0", "pos_unit")]


class TubeStats(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("n_particles", C.c_int64), ("n_slots", C.c_int64),
        ("total_injected", C.c_int64), ("last_injected", C.c_int64),
        ("last_removed", C.c_int64), ("pending_injection", C.c_int64),
        ("surface_field", C.c_double), ("flags", C.c_uint32), ("reserved", C.c_uint32),
    ]


class TubeDiag(C.Structure):
    _fields_ = [("n_particles", C.c_int64)] + [(n, C.c_double) for n in (
        "gamma_max", "gamma_mean", "kinetic", "field_energy", "gauss_max", "gauss_scale")]


class TubeTiming(C.Structure):
    _fields_ = [
        ("push_ms", C.c_double), ("field_ms", C.c_double), ("compact_ms", C.c_double),
        ("n_steps", C.c_int64), ("n_compactions", C.c_int64),
        ("particle_slots", C.c_int64), ("steps_run", C.c_int64),
        ("compactions_run", C.c_int64),
    ]


_vp, _i64, _i32 = C.c_void_p, C.c_int64, C.c_int
_pd = C.POINTER(C.c_double)
_pi64 = C.POINTER(C.c_int64)

SIGNATURES = {
    "tube_params_default": (_i32, [C.POINTER(TubeParams)]),
    "tube_derive": (_i32, [C.POINTER(TubeParams), C.POINTER(TubeDerived)]),
    "tube_workspace_bytes": (_i32, [C.POINTER(TubeParams), _pi64]),
    "tube_rho_gj_profile": (_i32, [C.POINTER(TubeParams), _pd]),
    "tube_create": (_i32, [C.POINTER(TubeParams), _vp, _i64, _vp, C.POINTER(_vp)]),
    "tube_destroy": (_i32, [_vp]),
    "tube_get_derived": (_i32, [_vp, C.POINTER(TubeDerived)]),
    "tube_inject": (_i32, [_vp, _pi64]),
    "tube_add_particles": (_i32, [_vp, _i64, _pd, _pd]),
    "tube_step": (_i32, [_vp]),
    "tube_run": (_i32, [_vp, _i64]),
    "tube_read_fields": (_i32, [_vp, _pd, _pd, _pd, _pd, _pd]),
    "tube_read_particles": (_i32, [_vp, _i64, _pi64, _pd, _pd, _pi64]),
    "tube_save_particles": (_i32, [_vp, _i64, _pi64, _vp, _vp, _pi64]),
    "tube_load_particles": (_i32, [_vp, _i64, _vp, _vp, _pi64]),
    "tube_solve_fields": (_i32, [_vp]),
    "tube_status": (_i32, [_vp, C.POINTER(TubeStats)]),
    "tube_status_async": (_i32, [_vp, C.POINTER(_i64)]),
    "tube_status_collect": (_i32, [_vp, _i64, C.POINTER(TubeStats)]),
    "tube_check": (_i32, [_vp]),
    "tube_diagnostics": (_i32, [_vp, C.POINTER(TubeDiag)]),
    "tube_compact": (_i32, [_vp]),
    "tube_sort": (_i32, [_vp]),
    "tube_selftest_wait_timeout": (_i32, [_vp]),
    "tube_selftest_velocity": (_i32, [C.c_uint32, C.c_uint64, C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint32)]),
    "tube_set_timing": (_i32, [_vp, _i32]),
    "tube_get_timing": (_i32, [_vp, C.POINTER(TubeTiming)]),
    "dtube_create": (_i32, [C.POINTER(TubeParams), C.c_int32, _pi64, C.POINTER(_vp)]),
    "dtube_destroy": (_i32, [_vp]),
    "dtube_domains": (_i32, [_vp, C.POINTER(C.c_int32)]),
    "dtube_domain": (_i32, [_vp, C.c_int32, C.POINTER(_vp), _pi64, _pi64]),
    "dtube_load_particles": (_i32, [_vp, _i64, _pd, _pd]),
    "dtube_set_fields": (_i32, [_vp, _pd, _pd, _pd]),
    "dtube_solve_fields": (_i32, [_vp]),
    "dtube_step": (_i32, [_vp]),
    "dtube_run": (_i32, [_vp, _i64]),
    "dtube_status": (_i32, [_vp, C.POINTER(TubeStats)]),
    "dtube_read_fields": (_i32, [_vp, _pd, _pd, _pd, _pd]),
    "dtube_exchange_stats": (_i32, [_vp, _pi64, _pi64, _pi64, _pi64]),
    "batch_create": (_i32, [C.c_int32, C.POINTER(TubeParams), _vp, C.POINTER(_vp)]),
    "batch_destroy": (_i32, [_vp]),
    "batch_size": (_i32, [_vp, C.POINTER(C.c_int32)]),
    "batch_tube": (_i32, [_vp, C.c_int32, C.POINTER(_vp)]),
    "batch_status": (_i32, [_vp, C.c_int32, C.POINTER(TubeStats)]),
    "batch_step": (_i32, [_vp]),
    "batch_run": (_i32, [_vp, _i64]),
    "batch_set_timing": (_i32, [_vp, _i32]),
    "batch_get_timing": (_i32, [_vp, C.POINTER(TubeTiming)]),
    "batch_set_variant": (_i32, [_vp, C.c_int32]),
    "batch_autotune": (_i32, [_vp, C.c_int32, _pd, C.POINTER(C.c_int32)]),
    "adjoint_create": (_i32, [C.POINTER(TubeParams), _i64, C.c_int32, _vp, C.POINTER(_vp)]),
    "adjoint_destroy": (_i32, [_vp]),
    "adjoint_checkpoint_every": (_i32, [_vp, C.POINTER(C.c_int32)]),
    "adjoint_tube": (_i32, [_vp, C.POINTER(_vp)]),
    "adjoint_set_injections": (_i32, [_vp, _pi64]),
    "adjoint_forward": (_i32, [_vp, _pd]),
    "adjoint_set_weights": (_i32, [_vp, _pd]),
    "adjoint_events": (_i32, [_vp, _pi64, _pi64, _pi64]),
    "adjoint_backward": (_i32, [_vp, C.c_int32, _pd, _pd]),
    "adjoint_param_gradient": (_i32, [_vp, _pd, C.c_double, C.c_double, _pd]),
    "tube_rho_gj_param_gradient": (_i32, [C.POINTER(TubeParams), _pd, _pd]),
    "adjoint_timing": (_i32, [_vp, _pd, _pd, _pi64]),
    "adjoint_set_timing": (_i32, [_vp, _i32]),
    "adjoint_kernel_times": (_i32, [_vp, _pd, _pi64]),
    "tube_push_deposit_static": (_i32, [_vp, _vp, _i64, _vp, C.c_int32, C.c_double,
                                         C.c_double, C.c_double, _vp, _vp, _vp, _vp]),
    "tube_strerror": (C.c_char_p, [_i32]),
    "tube_version": (C.c_char_p, []),
}

_LIB = None


class SclfError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = _LIB.tube_strerror(code).decode() if _LIB is not None else str(code)
        super().__init__("%s failed: %s (%d)" % (what, msg, code))


def load(path=None):
    """Load the in-tree library (built by ``paper_1011_6330_gb300.build``):
    libsclf_tube.so, or the file SCLF_TUBE_LIB names (e.g. the
    bounds-checked build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if path is None:
        path = os.environ.get("SCLF_TUBE_LIB", LIB_PATH)
    if not os.path.exists(path):
        raise RuntimeError(
            "sclf_tube library not built (%s missing); run "
            "`python -m paper_1011_6330_gb300.build` or __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(rc, what):
    if rc != 0:
        raise SclfError(rc, what)


def _dptr(a):
    return a.ctypes.data_as(_pd) if a is not None else None


_ARRAY_PARAMS = ("rho_gj_user", "gr_f", "gr_H")


def default_params(**kw):
    """tube_params_default() with keyword overrides (rho_gj_user, gr_f, gr_H:
    arrays of Nz+1 node values, or None)."""
    lib = load()
    p = TubeParams()
    _check(lib.tube_params_default(C.byref(p)), "tube_params_default")
    keep = []
    for k, v in kw.items():
        if k in _ARRAY_PARAMS:
            if v is None:
                setattr(p, k, None)
                continue
            a = np.ascontiguousarray(v, dtype=np.float64)
            keep.append(a)
            setattr(p, k, a.ctypes.data_as(_pd))
        else:
            setattr(p, k, v)
    p._keep = keep      # keep the arrays alive with the struct
    return p


def derive(params):
    lib = load()
    d = TubeDerived()
    _check(lib.tube_derive(C.byref(params), C.byref(d)), "tube_derive")
    return {n: getattr(d, n) for n, _ in TubeDerived._fields_}


def rho_gj_profile(params):
    """rho_GJ at the Nz+1 nodes as the library builds it (host only)."""
    lib = load()
    rho = np.empty(int(params.Nz) + 1)
    _check(lib.tube_rho_gj_profile(C.byref(params), _dptr(rho)), "tube_rho_gj_profile")
    return rho


def rho_gj_param_gradient(params, d_rho):
    """sum_j d_rho[j] d rho_GJ,j / d(B_G, P_s, R_cm) on the tube's fixed grid
    (host only)."""
    d_rho = np.ascontiguousarray(d_rho, dtype=np.float64)
    g = np.empty(3)
    _check(load().tube_rho_gj_param_gradient(C.byref(params), _dptr(d_rho), _dptr(g)),
           "tube_rho_gj_param_gradient")
    return g


def workspace_bytes(params):
    lib = load()
    b = C.c_int64()
    _check(lib.tube_workspace_bytes(C.byref(params), C.byref(b)), "tube_workspace_bytes")
    return b.value


class Tube:
    """One tube on the current CUDA device and stream."""

    def __init__(self, params, stream=None, torch_workspace=True):
        import torch
        self.lib = load()
        self.params = params
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        nbytes = workspace_bytes(params)
        self._ws = None
        ws_ptr = None
        if torch_workspace:
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            ws_ptr = (base + 255) // 256 * 256
        h = C.c_void_p()
        _check(self.lib.tube_create(C.byref(params), ws_ptr, nbytes,
                                    C.c_void_p(stream.cuda_stream), C.byref(h)),
               "tube_create")
        self.h = h
        d = TubeDerived()
        _check(self.lib.tube_get_derived(self.h, C.byref(d)), "tube_get_derived")
        self.derived = {n: getattr(d, n) for n, _ in TubeDerived._fields_}
        self.nz = int(params.Nz)
        self.fp64 = params.precision == SCLF_FP64
        self.fix32 = params.precision == SCLF_FIX32

    def close(self):
        if getattr(self, "h", None):
            self.lib.tube_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- steps -----------------------------------------------------------
    def step(self):
        _check(self.lib.tube_step(self.h), "tube_step")

    def run(self, n):
        _check(self.lib.tube_run(self.h, int(n)), "tube_run")

    def inject(self):
        n = C.c_int64()
        _check(self.lib.tube_inject(self.h, C.byref(n)), "tube_inject")
        return n.value

    def compact(self):
        _check(self.lib.tube_compact(self.h), "tube_compact")

    def sort(self):
        """Re-sort the slots by cell (stable), dropping holes."""
        _check(self.lib.tube_sort(self.h), "tube_sort")

    # -- particles -------------------------------------------------------
    def add_particles(self, z, u):
        z = np.ascontiguousarray(z, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert z.shape == u.shape
        _check(self.lib.tube_add_particles(self.h, z.size, _dptr(z), _dptr(u)),
               "tube_add_particles")

    def read_particles(self):
        n = C.c_int64()
        _check(self.lib.tube_read_particles(self.h, 0, C.byref(n), None, None, None),
               "tube_read_particles")
        cap = n.value
        z = np.empty(cap)
        u = np.empty(cap)
        ids = np.empty(cap, np.int64)
        _check(self.lib.tube_read_particles(self.h, cap, C.byref(n), _dptr(z), _dptr(u),
                                            ids.ctypes.data_as(_pi64)), "tube_read_particles")
        return z[:n.value], u[:n.value], ids[:n.value]

    def save_particles(self):
        n = C.c_int64()
        _check(self.lib.tube_save_particles(self.h, 0, C.byref(n), None, None, None),
               "tube_save_particles")
        dt = np.float64 if self.fp64 else np.float32
        xi = np.empty(n.value, np.int32 if self.fix32 else dt)
        u = np.empty(n.value, dt)
        ids = np.empty(n.value, np.int64)
        _check(self.lib.tube_save_particles(self.h, n.value, C.byref(n), xi.ctypes.data,
                                            u.ctypes.data, ids.ctypes.data_as(_pi64)),
               "tube_save_particles")
        return xi, u, ids

    def load_particles(self, xi, u, ids=None):
        dt = np.float64 if self.fp64 else np.float32
        xi = np.ascontiguousarray(xi, dtype=np.int32 if self.fix32 else dt)
        u = np.ascontiguousarray(u, dtype=dt)
        idp = None
        if ids is not None:
            ids = np.ascontiguousarray(ids, dtype=np.int64)
            idp = ids.ctypes.data_as(_pi64)
        _check(self.lib.tube_load_particles(self.h, xi.size, xi.ctypes.data, u.ctypes.data, idp),
               "tube_load_particles")

    # -- fields and counters ---------------------------------------------
    def read_fields(self, rho=True):
        nz = self.nz
        ez, er, b, j = np.empty(nz), np.empty(nz + 1), np.empty(nz), np.empty(nz)
        r = np.empty(nz + 1) if rho else None
        _check(self.lib.tube_read_fields(self.h, _dptr(ez), _dptr(er), _dptr(b), _dptr(j),
                                         _dptr(r)), "tube_read_fields")
        out = {"ez": ez, "er": er, "b": b, "j": j}
        if rho:
            out["rho"] = r
        return out

    def solve_fields(self):
        _check(self.lib.tube_solve_fields(self.h), "tube_solve_fields")

    def status(self):
        s = TubeStats()
        _check(self.lib.tube_status(self.h, C.byref(s)), "tube_status")
        return {n: getattr(s, n) for n, _ in TubeStats._fields_}

    def status_async(self):
        """Queue a copy of the counters (pipelined, no wait); returns a ticket
        for status_collect."""
        k = C.c_int64()
        _check(self.lib.tube_status_async(self.h, C.byref(k)), "tube_status_async")
        return k.value

    def status_collect(self, ticket):
        s = TubeStats()
        _check(self.lib.tube_status_collect(self.h, int(ticket), C.byref(s)), "tube_status_collect")
        return {n: getattr(s, n) for n, _ in TubeStats._fields_}

    def check(self):
        return self.lib.tube_check(self.h)

    def diagnostics(self):
        d = TubeDiag()
        _check(self.lib.tube_diagnostics(self.h, C.byref(d)), "tube_diagnostics")
        return {n: getattr(d, n) for n, _ in TubeDiag._fields_}

    def set_timing(self, enable):
        """True or 1: time every step; n > 1: every n-th unit of work (a
        single step or a graph replay); False or 0: off."""
        _check(self.lib.tube_set_timing(self.h, int(enable)), "tube_set_timing")

    def timing(self):
        t = TubeTiming()
        _check(self.lib.tube_get_timing(self.h, C.byref(t)), "tube_get_timing")
        return {n: getattr(t, n) for n, _ in TubeTiming._fields_}


class _TubeView(Tube):
    """A tube that belongs to a batch (no workspace of its own)."""

    def __init__(self, lib, handle, params):
        self.lib = lib
        self.params = params
        self._ws = None
        self.h = handle
        d = TubeDerived()
        _check(self.lib.tube_get_derived(self.h, C.byref(d)), "tube_get_derived")
        self.derived = {n: getattr(d, n) for n, _ in TubeDerived._fields_}
        self.nz = int(params.Nz)
        self.fp64 = params.precision == SCLF_FP64
        self.fix32 = params.precision == SCLF_FIX32

    def close(self):           # the batch owns it
        self.h = None


class DTube:
    """One tube split into z-ranges of cells (sub-domains), each with its
    own slots, stream and grid copy, stepped with the per-step exchanges a
    multi-GPU run makes (include/sclf_tube.h, dtube_*). n sub-domains of
    near-equal size, or the cell boundaries `cuts` (n + 1 values)."""

    def __init__(self, params, n=2, cuts=None):
        self.lib = load()
        self.params = params
        self.h = _vp()
        c = None
        if cuts is not None:
            cuts = np.ascontiguousarray(cuts, dtype=np.int64)
            n = cuts.size - 1
            c = cuts.ctypes.data_as(_pi64)
        _check(self.lib.dtube_create(C.byref(params), int(n), c, C.byref(self.h)),
               "dtube_create")
        self.nz = int(params.Nz)
        self.n = int(n)

    def close(self):
        if self.h:
            _check(self.lib.dtube_destroy(self.h), "dtube_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def domain(self, i):
        """(tube, lo, hi): sub-domain i's tube (for reading) and its cells."""
        t, lo, hi = _vp(), C.c_int64(), C.c_int64()
        _check(self.lib.dtube_domain(self.h, int(i), C.byref(t), C.byref(lo), C.byref(hi)),
               "dtube_domain")
        return _TubeView(self.lib, t, self.params), lo.value, hi.value

    def load_particles(self, z, u):
        z = np.ascontiguousarray(z, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        _check(self.lib.dtube_load_particles(self.h, z.size, _dptr(z), _dptr(u)),
               "dtube_load_particles")

    def set_fields(self, ez, er, b=None):
        ez = np.ascontiguousarray(ez, dtype=np.float64)
        er = np.ascontiguousarray(er, dtype=np.float64)
        b = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
        _check(self.lib.dtube_set_fields(self.h, _dptr(ez), _dptr(er), _dptr(b)),
               "dtube_set_fields")

    def solve_fields(self):
        _check(self.lib.dtube_solve_fields(self.h), "dtube_solve_fields")

    def step(self):
        _check(self.lib.dtube_step(self.h), "dtube_step")

    def run(self, nsteps):
        _check(self.lib.dtube_run(self.h, int(nsteps)), "dtube_run")

    def status(self):
        s = TubeStats()
        _check(self.lib.dtube_status(self.h, C.byref(s)), "dtube_status")
        return {n: getattr(s, n) for n, _ in TubeStats._fields_}

    def read_fields(self):
        nz = self.nz
        f = {"ez": np.empty(nz), "er": np.empty(nz + 1), "b": np.empty(nz), "j": np.empty(nz)}
        _check(self.lib.dtube_read_fields(self.h, _dptr(f["ez"]), _dptr(f["er"]),
                                          _dptr(f["b"]), _dptr(f["j"])), "dtube_read_fields")
        return f

    def read_particles(self):
        """All sub-domains' live particles (z, u, ids), in ID order."""
        parts = [self.domain(i)[0].read_particles() for i in range(self.n)]
        z = np.concatenate([p[0] for p in parts])
        u = np.concatenate([p[1] for p in parts])
        ids = np.concatenate([p[2] for p in parts])
        o = np.argsort(ids, kind="stable")
        return z[o], u[o], ids[o]

    def exchange_stats(self):
        v = [C.c_int64() for _ in range(4)]
        _check(self.lib.dtube_exchange_stats(self.h, *[C.byref(x) for x in v]),
               "dtube_exchange_stats")
        return dict(zip(("steps", "field_bytes", "particles", "particle_bytes"),
                        (x.value for x in v)))


class Batch:
    """Independent tubes stepped together by batched launches."""

    def __init__(self, params_list, stream=None):
        import torch
        self.lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        n = len(params_list)
        arr = (TubeParams * n)()
        for i, p in enumerate(params_list):
            arr[i] = p
        self._params = list(params_list)      # keep user profiles alive
        h = C.c_void_p()
        _check(self.lib.batch_create(n, arr, C.c_void_p(stream.cuda_stream), C.byref(h)),
               "batch_create")
        self.h = h
        self.tubes = []
        for i in range(n):
            th = C.c_void_p()
            _check(self.lib.batch_tube(self.h, i, C.byref(th)), "batch_tube")
            self.tubes.append(_TubeView(self.lib, th, params_list[i]))

    def step(self):
        _check(self.lib.batch_step(self.h), "batch_step")

    def status(self):
        """Every tube's counters from one gather and one copy: a list of
        dicts with the fields of Tube.status()."""
        n = len(self.tubes)
        arr = (TubeStats * n)()
        _check(self.lib.batch_status(self.h, n, arr), "batch_status")
        return [{f: getattr(arr[i], f) for f, _ in TubeStats._fields_} for i in range(n)]

    def run(self, n):
        _check(self.lib.batch_run(self.h, int(n)), "batch_run")

    def set_timing(self, enable):
        """True or 1: time every step; n > 1: every n-th step; 0: off."""
        _check(self.lib.batch_set_timing(self.h, int(enable)), "batch_set_timing")

    def timing(self):
        t = TubeTiming()
        _check(self.lib.batch_get_timing(self.h, C.byref(t)), "batch_get_timing")
        return {n: getattr(t, n) for n, _ in TubeTiming._fields_}

    # (particles per thread, CTAs per SM, per-thread current runs)
    VARIANTS = ((8, 4, 1), (8, 3, 1), (4, 4, 1), (8, 4, 2), (8, 3, 2), (16, 2, 2))

    def set_variant(self, v):
        _check(self.lib.batch_set_variant(self.h, int(v)), "batch_set_variant")

    def autotune(self, steps):
        """Time every particle-kernel shape for `steps` steps (the batch
        advances) and keep the fastest; returns (chosen, ms per shape)."""
        ms = np.empty(len(self.VARIANTS))
        ch = C.c_int32()
        _check(self.lib.batch_autotune(self.h, int(steps), _dptr(ms), C.byref(ch)),
               "batch_autotune")
        return ch.value, ms

    def close(self):
        if getattr(self, "h", None):
            for t in self.tubes:
                t.h = None
            self.lib.batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adjoint:
    """Discrete adjoint of an nsteps-step run of one tube, checkpointed every
    checkpoint_every steps (adjoint_* in include/sclf_tube.h)."""

    def __init__(self, params, nsteps, checkpoint_every, stream=None):
        import torch
        self.lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        self.params = params
        self.nsteps = int(nsteps)
        h = C.c_void_p()
        _check(self.lib.adjoint_create(C.byref(params), self.nsteps, int(checkpoint_every),
                                       C.c_void_p(stream.cuda_stream), C.byref(h)),
               "adjoint_create")
        self.h = h
        k = C.c_int32()
        _check(self.lib.adjoint_checkpoint_every(self.h, C.byref(k)), "adjoint_checkpoint_every")
        self.checkpoint_every = k.value           # the library's choice for checkpoint_every=0
        th = C.c_void_p()
        _check(self.lib.adjoint_tube(self.h, C.byref(th)), "adjoint_tube")
        self.tube = _TubeView(self.lib, th, params)
        self.nz = int(params.Nz)

    def set_injections(self, n_inj=None):
        if n_inj is None:
            _check(self.lib.adjoint_set_injections(self.h, None), "adjoint_set_injections")
            return
        a = np.ascontiguousarray(n_inj, dtype=np.int64)
        assert a.size == self.nsteps
        _check(self.lib.adjoint_set_injections(self.h, a.ctypes.data_as(_pi64)),
               "adjoint_set_injections")

    def set_weights(self, w):
        """Cell weights of the SCLF_OBJ_EZ_WEIGHTED objective sum_j w_j E_z,j."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        assert w.size == self.nz
        _check(self.lib.adjoint_set_weights(self.h, _dptr(w)), "adjoint_set_weights")

    def forward(self):
        """(mean terminal gamma, ||E_z||_2) of the run."""
        v = np.empty(2)
        _check(self.lib.adjoint_forward(self.h, _dptr(v)), "adjoint_forward")
        return float(v[0]), float(v[1])

    def events(self):
        inj, rem, slots = (np.empty(self.nsteps, np.int64) for _ in range(3))
        _check(self.lib.adjoint_events(self.h, inj.ctypes.data_as(_pi64),
                                       rem.ctypes.data_as(_pi64), slots.ctypes.data_as(_pi64)),
               "adjoint_events")
        return {"injected": inj, "removed": rem, "slots": slots}

    def backward(self, objective):
        """(d objective / d rho_GJ at the nodes, d objective / d s)."""
        d_rho = np.empty(self.nz + 1)
        d_s = C.c_double()
        _check(self.lib.adjoint_backward(self.h, int(objective), _dptr(d_rho), C.byref(d_s)),
               "adjoint_backward")
        return d_rho, d_s.value

    def param_gradient(self, d_rho, d_s, s_ref=0.0):
        """d objective / d(B_G, P_s, R_cm, w) with macro charge s = w s_ref
        (s_ref = 0: the tube's own s, w = 1)."""
        d_rho = np.ascontiguousarray(d_rho, dtype=np.float64)
        g = np.empty(4)
        _check(self.lib.adjoint_param_gradient(self.h, _dptr(d_rho), float(d_s), float(s_ref),
                                               _dptr(g)),
               "adjoint_param_gradient")
        return g

    def timing(self):
        f, b = C.c_double(), C.c_double()
        n = C.c_int64()
        _check(self.lib.adjoint_timing(self.h, C.byref(f), C.byref(b), C.byref(n)),
               "adjoint_timing")
        return {"forward_ms": f.value, "backward_ms": b.value, "particle_steps": n.value}

    KERNELS = ("forward_push", "forward_field", "recompute_push", "recompute_field",
               "reverse_field", "reverse_push")

    def set_timing(self, every):
        """Time every every-th segment of each kind (0 or False: off)."""
        _check(self.lib.adjoint_set_timing(self.h, int(every)), "adjoint_set_timing")

    def kernel_times(self):
        ms = np.empty(6)
        n = np.empty(6, np.int64)
        _check(self.lib.adjoint_kernel_times(self.h, _dptr(ms), n.ctypes.data_as(_pi64)),
               "adjoint_kernel_times")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KERNELS)}

    def close(self):
        if getattr(self, "h", None):
            self.tube.h = None
            self.lib.adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adjoint_problem(params_kw, nsteps, checkpoint_every, z=None, u=None, injections=None):
    """Fix a run for differentiation in theta = (B_G, P_s, R_cm, w): the
    grid (L, Nz), dt and the base macro charge s_ref are taken from
    params_kw's derived values and held, R becomes an explicit parameter.
    Returns (spec, theta0) for :class:`TubeObjectives`."""
    d = derive(default_params(**params_kw))
    kw = dict(params_kw)
    kw.update(dt=d["dt"], R_cm=d["R_cm"])
    spec = {"params": kw, "s_ref": d["s"], "nsteps": int(nsteps),
            "checkpoint_every": int(checkpoint_every),
            "z": None if z is None else np.asarray(z, np.float64),
            "u": None if u is None else np.asarray(u, np.float64),
            "injections": injections}
    theta0 = np.array([params_kw.get("B_G", 1e12), params_kw.get("P_s", 1.0), d["R_cm"], 1.0])
    return spec, theta0


def _adjoint_at(spec, theta):
    kw = dict(spec["params"])
    kw.update(B_G=float(theta[0]), P_s=float(theta[1]), R_cm=float(theta[2]),
              macro_charge=float(theta[3]) * spec["s_ref"])
    a = Adjoint(default_params(**kw), spec["nsteps"], spec["checkpoint_every"])
    if spec["z"] is not None and spec["z"].size:
        a.tube.add_particles(spec["z"], spec["u"])
    if spec["injections"] is not None:
        a.set_injections(spec["injections"])
    return a


def _objectives_function():
    import torch

    class TubeObjectives(torch.autograd.Function):
        """theta = (B_G, P_s, R_cm, w) -> (mean terminal gamma, ||E_z||_2) of
        the run that :func:`adjoint_problem` fixed, differentiated by the
        library's discrete adjoint (float64 CPU tensors in and out)."""

        @staticmethod
        def forward(ctx, theta, spec):
            th = theta.detach().cpu().double().numpy()
            a = _adjoint_at(spec, th)
            # the driver (and its checkpoints) lives as long as ctx, so a
            # second backward (retain_graph) sweeps the same recorded run
            ctx.adj, ctx.spec, ctx.theta = a, spec, th
            return torch.tensor(a.forward(), dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            a, spec = ctx.adj, ctx.spec
            g = grad_out.detach().cpu().double().numpy()
            grad = np.zeros(4)
            for obj in (SCLF_OBJ_GAMMA, SCLF_OBJ_EZ):
                if g[obj] != 0.0:
                    d_rho, d_s = a.backward(obj)
                    grad += g[obj] * a.param_gradient(d_rho, d_s, spec["s_ref"])
            return torch.tensor(grad, dtype=torch.float64), None

    return TubeObjectives


_TUBE_OBJECTIVES = None


def tube_objectives(theta, spec):
    """Differentiable (mean terminal gamma, ||E_z||_2) as a function of the
    float64 tensor theta = (B_G, P_s, R_cm, w)."""
    global _TUBE_OBJECTIVES
    if _TUBE_OBJECTIVES is None:
        _TUBE_OBJECTIVES = _objectives_function()
    return _TUBE_OBJECTIVES.apply(theta, spec)


def header_functions(path=HEADER):
    """Names of the functions include/sclf_tube.h declares."""
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:tube|dtube|batch|adjoint)_[a-z_]+)\s*\(", text)))
