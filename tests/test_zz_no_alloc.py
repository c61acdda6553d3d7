"""The allocation-free entry point against the tube step it mirrors.

tube_push_deposit_static is for callers that cannot call cudaMalloc: an
application whose allocator already owns the device's memory, a plug-in host
that forbids allocation at run time, or a latency-critical loop that cannot
take cudaMalloc's device-wide synchronisation. It keeps its scratch in one
fixed device array of the library. Here, after a first call on the device
(which loads the library's module), two calls in a row go through the C ABI
on the same state as the existing tube step (tube_step): positions, momenta,
removal counts and the current must equal the tube step's bit for bit (the
two run the same float32 operations and the same exact 2^-32 integer sums),
and they are also checked against the float32 oracle stepped from the same
seeded particles. Free device memory (cudaMemGetInfo) and torch's allocated
bytes must not change across either call, and the second call shows that the
shared scratch is cleared between calls.
"""

import ctypes as C

import numpy as np
import pytest

from paper_1011_6330_gb300 import binding as B
from paper_1011_6330_gb300 import synth, workloads
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-5          # FP32 particles against the oracle, norm-wise relative


def rel(a, b):
    den = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / den if den > 0 else float(np.max(np.abs(a - b)))


def _call(lib, xi_d, u_d, ez_d, nz, d, j_d, nrem_d, flags_d, stream):
    return lib.tube_push_deposit_static(
        C.c_void_p(xi_d.data_ptr()), C.c_void_p(u_d.data_ptr()), xi_d.numel(),
        C.c_void_p(ez_d.data_ptr()), nz, d["dt"], d["dz"], d["s"],
        C.c_void_p(j_d.data_ptr()), C.c_void_p(nrem_d.data_ptr()),
        C.c_void_p(flags_d.data_ptr()), stream)


def test_static_pass_matches_the_tube_step_on_two_calls(gpu_lib):
    import torch

    nz, L = 1024, 8.0
    rho = np.full(nz + 1, 1.0)
    kw = dict(workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64),
              rho_gj_user=rho, macro_charge=-1e-4, compact_interval=1000)
    t = B.Tube(B.default_params(**kw))
    d = t.derived
    z, u = synth.random_particles(20000 + 77, L, seed=11, u_sigma=3.0)
    t.add_particles(z, u)
    t.solve_fields()
    assert t.status()["pending_injection"] == 0      # the tube step injects nothing here
    o = oracle.Tube(nz, L, d["dt"], rho, d["s"], precision="f32", accumulate="fixed")
    o.add_particles(z, u)
    o.solve_fields()

    xi0, u0, _ = t.save_particles()
    dev = torch.device("cuda")
    xi_d = torch.from_numpy(xi0.copy()).to(dev)
    u_d = torch.from_numpy(u0.copy()).to(dev)
    ez_d = torch.empty(nz, dtype=torch.float64, device=dev)
    j_d = torch.empty(nz, dtype=torch.float64, device=dev)
    nrem_d = torch.zeros(1, dtype=torch.int64, device=dev)
    flags_d = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = gpu_lib

    # the first call on this device loads the module; it runs on a copy
    xw, uw = xi_d.clone(), u_d.clone()
    ez_d.zero_()
    assert _call(lib, xw, uw, ez_d, nz, d, j_d, nrem_d, flags_d, stream) == 0
    torch.cuda.synchronize()
    del xw, uw

    for call in range(2):
        ez = t.read_fields(rho=False)["ez"]             # E_z^n the step gathers from
        ez_d.copy_(torch.from_numpy(ez))
        j_d.fill_(float("nan"))
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        rc = _call(lib, xi_d, u_d, ez_d, nz, d, j_d, nrem_d, flags_d, stream)
        assert rc == 0, lib.tube_strerror(rc)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, call       # nothing allocated
        assert torch.cuda.memory_allocated() == alloc0, call
        t.step()                                          # the existing entry point
        st = t.status()
        assert st["last_injected"] == 0
        f = t.read_fields(rho=False)
        xs, us, _ = t.save_particles()                    # live particles in order
        xi_s = xi_d.cpu().numpy()
        u_s = u_d.cpu().numpy()
        live = xi_s >= 0
        assert int(nrem_d.item()) == st["last_removed"], call
        assert int(flags_d.item()) == 0, call
        assert np.count_nonzero(live) == xs.size, call
        assert np.array_equal(j_d.cpu().numpy(), f["j"]), call
        assert np.array_equal(xi_s[live], xs), call
        assert np.array_equal(u_s[live], us), call
        # the float32 oracle, from its own Eq. 4 solve and field update
        assert o.injection_count() == 0
        o.step()
        assert o.last_removed == st["last_removed"], call
        assert o.xi.size == xs.size, call
        assert rel(j_d.cpu().numpy(), o.j) <= TOL, call
        assert rel(xi_s[live].astype(np.float64), o.xi.astype(np.float64)) <= TOL, call
        assert rel(u_s[live].astype(np.float64), o.u.astype(np.float64)) <= TOL, call
    assert t.status()["step"] == 2 and st["last_removed"] > 0
    t.close()


def test_static_pass_flags_a_non_finite_push(gpu_lib):
    """A particle whose momentum is infinite leaves a hole, is counted in
    n_removed and sets SCLF_FLAG_NONFINITE; the others are pushed."""
    import torch
    nz = 64
    dz = 8.0 / nz
    dev = torch.device("cuda")
    xi = torch.tensor([10.5, 20.25, 30.75, 40.0], dtype=torch.float32, device=dev)
    u = torch.tensor([1.0, float("inf"), -2.0, 0.5], dtype=torch.float32, device=dev)
    ez = torch.zeros(nz, dtype=torch.float64, device=dev)
    j = torch.empty(nz, dtype=torch.float64, device=dev)
    nrem = torch.zeros(1, dtype=torch.int64, device=dev)
    flags = torch.full((1,), 0x10, dtype=torch.int32, device=dev)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _call(gpu_lib, xi, u, ez, nz, {"dt": 0.4 * dz, "dz": dz, "s": -1e-3}, j, nrem, flags,
               stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(nrem.item()) == 1
    assert int(flags.item()) == 0x10 | B.FLAG_NONFINITE
    x = xi.cpu().numpy()
    assert x[1] == -1.0 and np.all(x[[0, 2, 3]] >= 0)


def test_static_pass_rejects_a_grid_beyond_its_fixed_scratch(gpu_lib):
    import torch
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    big = B.load().tube_push_deposit_static
    nz = 65536 + 1
    ez = torch.zeros(nz, dtype=torch.float64, device="cuda")
    j = torch.zeros(nz, dtype=torch.float64, device="cuda")
    rc = big(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), 4, C.c_void_p(ez.data_ptr()),
             nz, 1e-3, 1e-2, -1e-3, C.c_void_p(j.data_ptr()), None, None, None)
    assert rc == -1                                     # SCLF_EINVAL
