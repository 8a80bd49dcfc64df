"""The z-slab decomposition's rank plumbing on CPU ranks (gloo, world sizes 2
and 3): the partition of the planes, the halo planes of each part, and the
point-to-point halo exchange of paper_1605_06015_gb300.slabs, with the FP64
oracle stepping each part (halo planes included, their own update discarded
by the next exchange).  The parts' own planes, gathered, equal the oracle's
run of the undivided grid bitwise: every node sees the same neighbours and
weights."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1605_06015_gb300 import slabs
from paper_1605_06015_gb300 import workloads as wl


def _geometry():
    mask, fib = wl.random_geometry(19, 13, 17, seed=31, tissue_frac=0.8)
    return mask, fib


def _initial(model, mask):
    import oracle
    rest = oracle.rest_state(model)
    S = len(rest)
    st = np.empty((S,) + mask.shape)
    for v in range(S):
        st[v] = rest[v]
    if model == oracle.BARKLEY:
        st[0, :, :4, :5] = 1.0
    else:
        st[0, :, :4, :5] = 20.0
    return st


def _rank_main(rank, world, port, model, n_steps, out_q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mask, fib = _geometry()
        nz = mask.shape[0]
        a, b, lo, hi = slabs.local_bounds(nz, world, rank)
        st = np.ascontiguousarray(_initial(model, mask)[:, a:b])
        g = oracle.Grid(mask.shape[2], mask.shape[1], b - a, 0.3, mask[a:b], fib[a:b], 1.0, 0.25)
        sim = oracle.Sim(g, model, state=st)
        plane = lambda z: torch.from_numpy(sim.state[0, z])  # a view: received values land in the state
        for _ in range(n_steps):
            slabs.exchange(dist, rank, world,
                           plane(lo) if lo else None, plane(b - a - 1 - hi) if hi else None,
                           plane(0) if lo else None, plane(b - a - 1) if hi else None)
            sim.step(0.005, 1)
        own = np.ascontiguousarray(sim.state[:, lo:b - a - hi])
        act = np.ascontiguousarray(sim.act[lo:b - a - hi])
        out_q.put((rank, own, act))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("world,model_name", [(2, "BARKLEY"), (3, "BR")])
def test_slab_ranks_reproduce_the_undivided_grid_bitwise(world, model_name):
    import oracle
    model = getattr(oracle, model_name)
    n_steps = 25
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, model, n_steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, own, act = q.get(timeout=300)
        res[r] = (own, act)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mask, fib = _geometry()
    g = oracle.Grid(mask.shape[2], mask.shape[1], mask.shape[0], 0.3, mask, fib, 1.0, 0.25)
    sim = oracle.Sim(g, model, state=_initial(model, mask))
    sim.step(0.005, n_steps)
    got = np.concatenate([res[r][0] for r in range(world)], axis=1)
    got_act = np.concatenate([res[r][1] for r in range(world)], axis=0)
    tis = mask != 0
    assert np.array_equal(got[:, tis], sim.state[:, tis])
    assert np.array_equal(got_act, sim.act)
    # the wave crossed at least one cut
    z_cut = slabs.slab_bounds(mask.shape[0], world, 0)[1]
    assert np.any(sim.state[0, z_cut][tis[z_cut]] != sim.state[0, -1][tis[-1]][0])


def test_partition_covers_every_plane_once():
    for nz in (3, 7, 64, 65):
        for parts in range(1, min(nz, 9) + 1):
            seen = []
            for i in range(parts):
                z0, z1 = slabs.slab_bounds(nz, parts, i)
                a, b, lo, hi = slabs.local_bounds(nz, parts, i)
                assert z1 > z0 and a == z0 - lo and b == z1 + hi and 0 <= a and b <= nz
                assert lo == (i > 0) and hi == (i < parts - 1)
                seen.extend(range(z0, z1))
            assert seen == list(range(nz))
    with pytest.raises(ValueError):
        slabs.slab_bounds(3, 4, 0)
