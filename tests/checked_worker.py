"""Edge-heavy runs through whichever build of the library SCLF_TUBE_LIB names.

Usage: python tests/checked_worker.py OUT.npz

Particles sit on the cell and tube boundaries (xi = 0, just below 1, on
nodes, just below Nz), move fast in both directions or rest, and the runs
cover every particle kernel: FP64, FP32 (both accumulators), SCLF_FIX32,
compaction, re-sorts, a batch in both run shapes and the adjoint in float32
and fixed point. Every result is saved to OUT.npz, together with each
tube's status flags. test_gpu_parity runs it once with the normal and once
with the bounds-checked build and compares.
"""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1011_6330_gb300 import binding as B  # noqa: E402
from paper_1011_6330_gb300 import synth, workloads  # noqa: E402


def edge_particles(nz, L, n_random, seed):
    """Boundary positions and extreme momenta, then a random beam."""
    dz = L / nz
    top = nz * (1.0 - 1e-6)
    xi = [0.0, 1e-7, 0.5, 1.0 - 1e-7, 1.0, 2.0, nz / 2.0, nz - 1.0, nz - 1.0 + 1e-4, top]
    us = [0.0, 1e-3, -1e-3, 1e3, -1e3, 1e7, -1e7, 3.0, -3.0, 0.0]
    xi_e = np.repeat(np.array(xi), len(us))
    u_e = np.tile(np.array(us), len(xi))
    z_r, u_r = synth.prefilled_beam(n_random, L - dz, 20.0, seed=seed, order="shuffled")
    u_r = u_r * np.where(np.arange(n_random) % 3 == 0, -1.0, 1.0)
    return np.concatenate([xi_e * dz, z_r]), np.concatenate([u_e, u_r])


def tube_case(out, name, kw, steps, seed, sort_every=0):
    t = B.Tube(B.default_params(**kw))
    z, u = edge_particles(kw["Nz"], kw["L_over_R"], 20000, seed)
    t.add_particles(z, u)
    t.solve_fields()
    for n in range(steps):
        t.step()
        if n % 17 == 16:
            t.compact()
        if sort_every and n % sort_every == sort_every - 1:
            t.sort()
    f = t.read_fields(rho=False)
    x, uu, ids = t.save_particles()
    st = t.status()
    for k in ("ez", "er", "b", "j"):
        out["%s_%s" % (name, k)] = f[k]
    out[name + "_x"], out[name + "_u"], out[name + "_ids"] = x, uu, ids
    out[name + "_counts"] = np.array([st["step"], st["n_particles"], st["total_injected"],
                                      st["pending_injection"]], np.int64)
    out[name + "_flags"] = np.array([st["flags"]], np.int64)
    t.close()


def main(path):
    B.load()
    out = {}
    flat = workloads.flat_sclf_small
    tube_case(out, "fp64", flat(precision=B.SCLF_FP64, accumulate=B.SCLF_ACC_FIXED64), 120, 1)
    tube_case(out, "fp32", flat(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FIXED64), 120, 2,
              sort_every=25)
    tube_case(out, "fp32acc", flat(precision=B.SCLF_FP32, accumulate=B.SCLF_ACC_FP64), 120, 3)
    tube_case(out, "fix32", flat(precision=B.SCLF_FIX32, accumulate=B.SCLF_ACC_FIXED64), 120, 4,
              sort_every=40)
    # a batch of uneven tubes in the one-run and two-run shapes
    specs = [(1e12, 0.5, 0.5, 64, 3000), (3e11, 1.3, 0.0, 200, 9000), (2e12, 0.2, 0.5, 1024, 20000)]
    kws = []
    for Bg, P, incl, nz, n in specs:
        kw = workloads.gr_tube(B_G=Bg, P_s=P, incl=incl, Nz=nz, n_particles=n,
                               capacity=n + 8192, track_ids=1)
        kw["rho_gj_mode"] = B.SCLF_RHO_GR if incl > 0 else B.SCLF_RHO_FLAT
        kw["compact_interval"] = 7
        kws.append(kw)
    b = B.Batch([B.default_params(**kw) for kw in kws])
    for i, kw in enumerate(kws):
        z, u = edge_particles(kw["Nz"], kw["L_over_R"], kw["target_particles"], 10 + i)
        b.tubes[i].add_particles(z, u)
        b.tubes[i].solve_fields()
    for v in (0, 3):
        b.set_variant(v)
        b.run(30)
    for i, st in enumerate(b.status()):
        x, uu, ids = b.tubes[i].save_particles()
        f = b.tubes[i].read_fields(rho=False)
        out["batch%d_x" % i], out["batch%d_u" % i] = x, uu
        out["batch%d_ez" % i], out["batch%d_j" % i] = f["ez"], f["j"]
        out["batch%d_flags" % i] = np.array([st["flags"]], np.int64)
    b.close()
    # the adjoint in float32 and fixed point
    for prec, name in ((B.SCLF_FP32, "adj32"), (B.SCLF_FIX32, "adjfix")):
        kw = flat(precision=prec, accumulate=B.SCLF_ACC_FIXED64)
        a = B.Adjoint(B.default_params(**kw), 40, 10)
        z, u = edge_particles(kw["Nz"], kw["L_over_R"], 20000, 20 + prec)
        a.tube.add_particles(z, u)
        out[name + "_values"] = np.asarray(a.forward(), np.float64)
        for obj in (B.SCLF_OBJ_GAMMA, B.SCLF_OBJ_EZ):
            d_rho, d_s = a.backward(obj)
            out["%s_drho%d" % (name, obj)] = np.asarray(d_rho)
            out["%s_ds%d" % (name, obj)] = np.array([d_s])
        out[name + "_flags"] = np.array([a.tube.status()["flags"]], np.int64)
        a.close()
    out["version"] = np.array(B.load().tube_version().decode())
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
