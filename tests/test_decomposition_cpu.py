"""The z-domain decomposition of one tube as gloo ranks on the CPU, with the
oracle's step pieces doing the work: each rank owns a contiguous range of
cells and the particles in it, keeps its own copy of the grids, and per step
exchanges exactly what the GPU's decomposed tube (dtube_*) exchanges:

  after the deposit:    the current its particles put in the neighbour's
                        boundary cell (exact integer sums);
  after the particles:  the particles that left its cells for a neighbour's;
  after the fields:     B_phi and E_z of its boundary cells (the neighbour's
                        halo for the next field update and gather).

E_r at a shared node is computed on both sides. Only rank 0 (the base)
injects. The run must equal the whole tube stepped by the oracle, bit for bit
(fields on the owned cells, particles by ID, injection totals): Sec. 2's
field equations (Eq. 3) and the cloud-in-cell gather couple a cell only to
its neighbours, and a particle moves less than a cell per step."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _flat_tube(prec):
    import oracle as orc
    nz, L = 256, 2.0
    dz = L / nz
    return orc.Tube(nz, L, 0.4 * dz, -np.ones(nz + 1), -2e-4, precision=prec, accumulate="fixed")


def _prefill(tube, seed):
    from paper_1011_6330_gb300 import synth
    z, u = synth.random_particles(3000, tube.L * (1 - 1.0 / tube.nz), seed=seed, u_sigma=3.0)
    tube.add_particles(z, u)
    tube.solve_fields()


def _send(dist, arr, dst):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(arr))
    dist.send(torch.tensor([t.numel()], dtype=torch.int64), dst)
    if t.numel():
        dist.send(t, dst)


def _recv(dist, dtype, src):
    import torch
    n = torch.zeros(1, dtype=torch.int64)
    dist.recv(n, src)
    buf = torch.zeros(int(n.item()), dtype=dtype)
    if buf.numel():
        dist.recv(buf, src)
    return buf.numpy()


def _rank(rank, world, port, prec, cuts, nsteps, out):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc
    t = _flat_tube(prec)                     # this rank's grid copy and parameters
    _prefill(t, seed=5)
    nz, dz, dt, s, rt = t.nz, t.dz, t.dt, t.s, t.rt
    lo, hi = cuts[rank], cuts[rank + 1]
    fix = t.fix
    unit = (1 << t.fb) if fix else 1         # positions per cell
    cell = (lambda x: x >> t.fb) if fix else (lambda x: np.floor(x).astype(np.int64))
    mine = (t.xi >= 0) & (cell(t.xi) >= lo) & (cell(t.xi) < hi)
    xi, u, ids = t.xi[mine], t.u[mine], t.ids[mine]
    ez, er, b = t.ez.copy(), t.er.copy(), t.b.copy()
    total_injected = t.total_injected
    w0 = t.w0 if rank == 0 else 0
    sent = 0
    pos_dt = torch.int64 if fix else (torch.float64 if rt == np.float64 else torch.float32)
    mom_dt = torch.float64 if rt == np.float64 else torch.float32
    for _ in range(nsteps):
        # (a1) injection at the base (rank 0)
        if rank == 0:
            n_inj, _ = orc.injection_count(ez[0], w0, s, dz, t.rho_gj[0])
            xi = np.concatenate([xi, np.zeros(n_inj, xi.dtype)])
            u = np.concatenate([u, np.zeros(n_inj, rt)])
            ids = np.concatenate([ids, total_injected + np.arange(n_inj, dtype=np.int64)])
            total_injected += n_inj
        # (a2)-(a4) on this rank's particles
        if fix:
            ep = orc.gather_fix32(ez, xi, t.fb)
            xi1, u1, finite = orc.push_fix32(xi, u, ep, dt, dz, t.fb)
            acc = orc.deposit_fix32(nz, xi[finite], xi1[finite], t.fb)
        else:
            ep = orc.gather(ez, xi, rt)
            xi1, u1 = orc.push(xi, u, ep, dt, dz, rt)
            acc = orc.deposit_fractions(nz, xi, xi1, rt, "fixed")
            finite = np.isfinite(xi1) & np.isfinite(u1)
        acc = np.asarray(acc, np.int64)
        # exchange: current deposited in the neighbours' boundary cells
        if rank + 1 < world:
            _send(dist, acc[hi:hi + 1], rank + 1)
            acc[hi - 1] += _recv(dist, torch.int64, rank + 1)[0]
        if rank > 0:
            got = _recv(dist, torch.int64, rank - 1)[0]
            _send(dist, acc[lo - 1:lo], rank - 1)
            acc[lo] += got
        j = orc.current_from(acc, s, dt, "fixed")
        # (a5) removal at the ends; hand-off of the particles leaving [lo, hi)
        inside = finite & (xi1 >= 0) & (xi1 < nz * unit)
        c1 = np.where(inside, cell(np.where(inside, xi1, 0)), -1)
        keep = inside & (c1 >= lo) & (c1 < hi)
        down, up = inside & (c1 < lo), inside & (c1 >= hi)
        outgoing = [(nb, (xi1[m], u1[m], ids[m])) for nb, m in ((rank - 1, down), (rank + 1, up))
                    if 0 <= nb < world]
        arrived = []
        for nb, arrs in outgoing:            # the lower rank sends first on each boundary
            sent += int(arrs[0].size)
            if nb > rank:
                for a in arrs:
                    _send(dist, a, nb)
                arrived.append([_recv(dist, dtp, nb) for dtp in (pos_dt, mom_dt, torch.int64)])
            else:
                arrived.append([_recv(dist, dtp, nb) for dtp in (pos_dt, mom_dt, torch.int64)])
                for a in arrs:
                    _send(dist, a, nb)
        xi = np.concatenate([xi1[keep]] + [a[0].astype(xi1.dtype) for a in arrived])
        u = np.concatenate([u1[keep]] + [a[1].astype(u1.dtype) for a in arrived])
        ids = np.concatenate([ids[keep]] + [a[2] for a in arrived])
        if rank == 0:
            w0 = orc.base_weight_fix32(xi, t.fb) if fix else orc.base_weight_fixed(xi, rt)
        # (a6) fields on this rank's copy, then the boundary halos
        ez, er, b = orc.field_update(ez, er, b, j, dt, dz)
        if rank + 1 < world:
            _send(dist, np.array([b[hi - 1], ez[hi - 1]]), rank + 1)
            b[hi], ez[hi] = _recv(dist, torch.float64, rank + 1)
        if rank > 0:
            got = _recv(dist, torch.float64, rank - 1)
            _send(dist, np.array([b[lo], ez[lo]]), rank - 1)
            b[lo - 1], ez[lo - 1] = got
    hi_node = hi + 1 if rank + 1 == world else hi
    out[rank] = dict(ez=ez[lo:hi], er=er[lo:hi_node], b=b[lo:hi], xi=xi, u=u, ids=ids,
                     total_injected=total_injected, sent=sent)
    dist.destroy_process_group()


@pytest.mark.parametrize("prec,cuts", [("f64", [0, 97, 256]), ("f32", [0, 2, 130, 256]),
                                       ("fix32", [0, 128, 254, 256])])
def test_decomposed_oracle_ranks_equal_the_whole_tube(prec, cuts):
    world = len(cuts) - 1
    nsteps = 120
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), prec, cuts, nsteps, out),
                       nprocs=world, start_method="spawn", join=True)
    whole = _flat_tube(prec)
    _prefill(whole, seed=5)
    for _ in range(nsteps):
        whole.step()
    res = [out[r] for r in range(world)]
    for k in ("ez", "er", "b"):
        got = np.concatenate([r[k] for r in res])
        assert np.array_equal(got, getattr(whole, k)), k
    ids = np.concatenate([r["ids"] for r in res])
    o = np.argsort(ids)
    assert np.array_equal(ids[o], whole.ids)
    assert np.array_equal(np.concatenate([r["xi"] for r in res])[o], whole.xi)
    assert np.array_equal(np.concatenate([r["u"] for r in res])[o], whole.u)
    assert res[0]["total_injected"] == whole.total_injected
    assert sum(r["sent"] for r in res) > 0              # particles crossed the cuts
