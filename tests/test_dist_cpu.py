"""The partitioned Poisson solve on CPU ranks: the slab plan's bookkeeping,
and Jacobi-PCG over 2, 3 and 4 gloo ranks - the library's partitioned driver
(ax_cg_solve_part, host code) with oracle-backed rank-local work as its ops
table - against the single-domain oracle PCG."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2506_20994_gb300 import dist as adist
from paper_2506_20994_gb300 import synth


@pytest.mark.parametrize("dims,lx,world", [((2, 3, 4), 4, 2), ((2, 2, 5), 3, 3),
                                           ((3, 2, 3), 5, 3), ((2, 2, 2), 4, 1)])
def test_slab_plan_covers_the_box(dims, lx, world):
    nx, ny, nz = dims
    plans = [adist.SlabPlan(nx, ny, nz, lx, world, r) for r in range(world)]
    assert plans[0].e0 == 0 and plans[-1].e1 == nx * ny * nz
    for a, b in zip(plans, plans[1:]):
        assert a.e1 == b.e0 and a.z1 == b.z0
    # slab ids + offsets reproduce the whole box's numbering
    whole = oracle.numbering(nx, ny, nz, lx).reshape(-1, lx ** 3)
    for p in plans:
        assert np.array_equal(p.glob.reshape(-1, lx ** 3) + p.offset, whole[p.e0:p.e1])
    # copies summed over ranks = the whole box's multiplicity
    mult = oracle.multiplicity(whole).reshape(-1, lx ** 3)
    counts = np.zeros(int(whole.max()) + 1)
    for p in plans:
        np.add.at(counts, p.glob + p.offset, 1.0)
    assert np.array_equal(counts[whole], mult)
    # shared planes: what one side sends lands on the node the other side owns
    for p in plans:
        for nb, base in p.neighbours:
            q = plans[nb]
            sent = p.glob[p.send_idx[nb]] + p.offset
            back = dict(q.neighbours)[p.rank]
            recv = np.empty(q.plane, dtype=np.int64)
            recv[q.recv_pos[p.rank]] = q.glob[q.recv_idx[p.rank]] + q.offset
            assert np.array_equal(sent, recv)
            assert np.array_equal(np.sort(p.glob[p.send_idx[nb]]), base + np.arange(p.plane))
            assert back in (0, q.nzl * (lx - 1) * q.plane)
    with pytest.raises(ValueError):
        adist.SlabPlan(nx, ny, nz, lx, nz + 1, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, dims, lx, outdir):
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from _dist_ops import OracleSlabOps
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny, nz = dims
        v = synth.box_vertices(nx, ny, nz, seed=3)
        h1 = synth.uniform((nx * ny * nz, lx, lx, lx), seed=4, lo=0.5, hi=2.0)
        plan = adist.SlabPlan(nx, ny, nz, lx, world, rank)
        ops = OracleSlabOps(plan, v, h1)
        comm = adist.TorchComm("cpu")
        adist.setup(ops, plan, comm)
        b = ops.rhs_partial(oracle.poisson_rhs_f)
        adist.halo_sum(ops, plan, comm, b)
        x, it, rel = adist.pcg(ops, plan, comm, b, tol=1e-8)
        np.savez(os.path.join(outdir, f"r{rank}.npz"), x=x.numpy(), it=it, rel=rel,
                 b=b.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dims,lx", [(2, (2, 2, 4), 4), (3, (2, 3, 3), 3), (4, (2, 2, 4), 3)])
def test_partitioned_pcg_matches_single_domain(world, dims, lx, tmp_path):
    import paper_2506_20994_gb300 as ax
    ax.build()  # the driver is library code; its ranks load libaxhelm.so
    mp.spawn(_rank_main, args=(world, _free_port(), dims, lx, str(tmp_path)), nprocs=world,
             join=True)
    nx, ny, nz = dims
    v = synth.box_vertices(nx, ny, nz, seed=3)
    h1 = synth.uniform((nx * ny * nz, lx, lx, lx), seed=4, lo=0.5, hi=2.0)
    P = oracle.Problem(v, lx, h1=h1, f=oracle.poisson_rhs_f)
    x_ref, it_ref, _ = oracle.pcg(P, P.b, tol=1e-8)
    parts = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    x = np.concatenate([p["x"].reshape(-1, lx ** 3) for p in parts])
    b = np.concatenate([p["b"].reshape(-1, lx ** 3) for p in parts])
    # the assembled right-hand side is the single-domain one
    np.testing.assert_allclose(b, P.b.reshape(-1, lx ** 3), rtol=0,
                               atol=1e-14 * np.abs(P.b).max())
    its = {int(p["it"]) for p in parts}
    assert len(its) == 1 and abs(its.pop() - it_ref) <= 1
    assert all(float(p["rel"]) <= 1e-8 for p in parts)
    err = np.linalg.norm(x - x_ref.reshape(-1, lx ** 3)) / np.linalg.norm(x_ref)
    assert err <= 1e-9
    # copies of a node on two ranks hold the same bits
    g = oracle.numbering(nx, ny, nz, lx).reshape(-1, lx ** 3)
    first = {}
    for val, node in zip(x.ravel(), g.ravel()):
        assert first.setdefault(node, val) == val
