"""The allocation-free entry point against the tube step it mirrors.

tube_push_deposit_static is for callers that cannot call cudaMalloc: an
application whose allocator already owns the device's memory, a plug-in host
that forbids allocation at run time, or a latency-critical loop that cannot
take cudaMalloc's device-wide synchronisation. It keeps its scratch in one
fixed device array of the library. Here two calls in a row go through the C
ABI and are checked against the existing tube step (tube_step) on the same
state, within the FP32 parity tolerance used by the other GPU tests; the
second call also shows that the shared scratch is cleared between calls.
"""

import ctypes as C

import numpy as np
import pytest

from paper_1011_6330_gb300 import binding as B
from paper_1011_6330_gb300 import synth, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5          # FP32 particles, norm-wise relative (as in test_gpu_parity)


def rel(a, b):
    den = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / den if den > 0 else float(np.max(np.abs(a - b)))


def test_static_pass_matches_the_tube_step_on_two_calls(gpu_lib):
    import torch

    nz, L = 1024, 8.0
    kw = dict(workloads.flat_sclf_small(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64),
              rho_gj_user=np.full(nz + 1, 1.0), macro_charge=-1e-4, compact_interval=1000)
    t = B.Tube(B.default_params(**kw))
    d = t.derived
    z, u = synth.random_particles(20000 + 77, L, seed=11, u_sigma=3.0)
    t.add_particles(z, u)
    t.solve_fields()
    assert t.status()["pending_injection"] == 0      # the tube step injects nothing here

    xi0, u0, _ = t.save_particles()
    dev = torch.device("cuda")
    xi_d = torch.from_numpy(xi0.copy()).to(dev)
    u_d = torch.from_numpy(u0.copy()).to(dev)
    ez_d = torch.empty(nz, dtype=torch.float64, device=dev)
    j_d = torch.empty(nz, dtype=torch.float64, device=dev)
    nrem_d = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = gpu_lib

    for call in range(2):
        ez = t.read_fields(rho=False)["ez"]             # E_z^n the step gathers from
        ez_d.copy_(torch.from_numpy(ez))
        rc = lib.tube_push_deposit_static(
            C.c_void_p(xi_d.data_ptr()), C.c_void_p(u_d.data_ptr()), xi_d.numel(),
            C.c_void_p(ez_d.data_ptr()), nz, d["dt"], d["dz"], d["s"],
            C.c_void_p(j_d.data_ptr()), C.c_void_p(nrem_d.data_ptr()), stream)
        assert rc == 0, lib.tube_strerror(rc)
        t.step()                                          # the existing entry point
        st = t.status()
        assert st["last_injected"] == 0
        f = t.read_fields(rho=False)
        xs, us, _ = t.save_particles()                    # live particles in order
        torch.cuda.synchronize()
        xi_s = xi_d.cpu().numpy()
        u_s = u_d.cpu().numpy()
        live = xi_s >= 0
        assert int(nrem_d.item()) == st["last_removed"], call
        assert np.count_nonzero(live) == xs.size, call
        assert rel(j_d.cpu().numpy(), f["j"]) <= TOL, call
        assert rel(xi_s[live].astype(np.float64), xs.astype(np.float64)) <= TOL, call
        assert rel(u_s[live].astype(np.float64), us.astype(np.float64)) <= TOL, call
    assert t.status()["step"] == 2
    t.close()


def test_static_pass_rejects_a_grid_beyond_its_fixed_scratch(gpu_lib):
    import torch
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    big = B.load().tube_push_deposit_static
    nz = 65536 + 1
    ez = torch.zeros(nz, dtype=torch.float64, device="cuda")
    j = torch.zeros(nz, dtype=torch.float64, device="cuda")
    rc = big(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), 4, C.c_void_p(ez.data_ptr()),
             nz, 1e-3, 1e-2, -1e-3, C.c_void_p(j.data_ptr()), None, None)
    assert rc == -1
