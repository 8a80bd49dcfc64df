"""Batched stepping of many independent grids (one graph-captured launch per
kernel type and step) against stepping each grid alone and against the FP64
oracle."""
import numpy as np
import pytest

import oracle
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx as b
    return b


def _members():
    """Uneven sizes, three kernel types, parameter sweeps, two time steps."""
    rng = np.random.default_rng(11)
    ws = []
    for nx, ny in ((70, 33), (130, 64), (64, 129), (200, 17)):
        k = rng.uniform(0.8, 1.2, size=4)
        ws.append(wl.fhn_sheet(nx, ny, seed=int(rng.integers(1 << 30)), D=k[0], eps=0.3 * k[1], beta=0.71 * k[2],
                               gamma=0.5 * k[3]))
    for nx, ny, nz in ((64, 40, 20), (100, 30, 12)):
        k = rng.uniform(0.8, 1.2, size=4)
        srng = np.random.default_rng(int(rng.integers(1 << 30)))
        reg = wl.point_stimuli(nx, ny, nz, srng, count=2)
        D = k[0]
        ws.append(wl.Workload("blk", nx, ny, nz, 0.3, 0.005, wl.BARKLEY, [0.75 * k[1], 0.02 * k[2], 0.02 * k[3]],
                              D, D, ic_region=reg, ic_value=1.0, theta=0.5))
    mask, fib = wl.random_geometry(45, 26, 9, 5, tissue_frac=0.7)
    ws.append(wl.Workload("zfk", 45, 26, 9, 0.5, 0.01, wl.ZFK, [0.13], 1.0, 0.3, mask=mask, fibres=fib,
                          ic_fields={0: rng.random((9, 26, 45))}, theta=0.5))
    return ws


def _grid(bbx, w, st0):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_fibres(w.fibres, w.D_par, w.D_perp if w.fibres is not None else w.D_par)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    G.set_timestep(w.dt)
    G.write_all(st0)
    return G


def test_batch_matches_individual_steps_bitwise_and_the_oracle(bbx):
    ws = _members()
    st0 = [w.initial_state(oracle.rest_state(w.model, w.params)).astype(np.float32) for w in ws]
    n = 40
    solo = []
    for w, s0 in zip(ws, st0):
        G = _grid(bbx, w, s0)
        G.step(w.dt, n)
        solo.append((G.read_all(), G.read_activation(), G.step_total()))
    grids = [_grid(bbx, w, s0) for w, s0 in zip(ws, st0)]
    B = bbx.Batch(grids)
    assert B.info()["n_groups"] == 3
    B.step(n)  # graph-captured chunks
    B.sync()
    for i, (w, G) in enumerate(zip(ws, grids)):
        st, act, tot = solo[i]
        assert np.array_equal(G.read_all(), st), w.name
        assert np.array_equal(G.read_activation(), act), w.name
        assert G.step_total() == pytest.approx(tot, rel=1e-12, abs=1e-12)
        t, k = G.get_time()
        assert k == n and t == pytest.approx(n * w.dt, rel=1e-12)
        og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
        osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0[i].astype(np.float64))
        osim.step(w.dt, n)
        tis = og.psi
        err = np.abs(st[0][tis] - osim.state[0][tis]).max() / np.abs(osim.state[0][tis]).max()
        assert err <= 1e-4, (w.name, err)


def test_batch_odd_step_counts_autotune_and_member_changes(bbx):
    ws = _members()[:5]
    st0 = [w.initial_state(oracle.rest_state(w.model, w.params)).astype(np.float32) for w in ws]
    grids = [_grid(bbx, w, s0) for w, s0 in zip(ws, st0)]
    B = bbx.Batch(grids)
    B.autotune()  # leaves no trace
    for G, s0 in zip(grids, st0):
        assert np.array_equal(G.read_all(), s0) and G.get_time()[1] == 0
    B.step(1)
    B.step(19)    # one graph of 16 and 3 direct launches
    grids[0].set_threshold(0.1)  # a member change rebuilds the batch
    B.step(5)
    B.sync()
    # the solo references use the tile height the autotuner gave each member's
    # kernel group (the rounding of a few operations differs between heights)
    keys = []
    for w in ws:
        k = (w.model, w.mask is not None, w.fibres is not None, w.nz == 1)
        if k not in keys:
            keys.append(k)
    tys = B.info()["tile_y"]
    ref = [_grid(bbx, w, s0) for w, s0 in zip(ws, st0)]
    ref[0].set_threshold(0.1)
    for R, w in zip(ref, ws):
        R.set_tiling(tys[keys.index((w.model, w.mask is not None, w.fibres is not None, w.nz == 1))],
                     16 if w.nz > 1 else 1)
    for G, R, w in zip(grids, ref, ws):
        R.step(w.dt, 25)
        assert np.array_equal(G.read_all(), R.read_all())
        assert G.get_time()[1] == 25


def test_batch_argument_errors(bbx):
    w = wl.fhn_sheet(64, 40)
    G = bbx.Grid(w.nx, w.ny, 1, w.h)
    with pytest.raises(bbx.BbxError):
        bbx.Batch([G])  # no model
    G.set_ionic_model(bbx.BBX_FHN)
    with pytest.raises(bbx.BbxError):
        bbx.Batch([G])  # no time step yet
    G.set_timestep(0.01)
    with pytest.raises(bbx.BbxError):
        bbx.Batch([G, G])  # duplicate member
    B = bbx.Batch([G])
    B.step(3)
    B.sync()
    assert G.get_time()[1] == 3


def test_grid_without_tissue_in_a_batch_advances_time_and_totals(bbx):
    # a member whose mask holds no tissue has no pieces: its time and step
    # count still advance every batch step (the last CTA finishes it), and
    # the grids with pieces are finished by the CTA that completes them, with
    # totals equal to the grid stepped alone
    ws = _members()[:3]
    st0 = [w.initial_state(oracle.rest_state(w.model, w.params)).astype(np.float32) for w in ws]
    empty = wl.Workload("void", 40, 20, 6, 0.3, 0.005, wl.BARKLEY, [0.75, 0.02, 0.02], 1.0, 1.0,
                        mask=np.zeros((6, 20, 40), np.uint8), theta=0.5)
    e0 = empty.initial_state(oracle.rest_state(empty.model, empty.params)).astype(np.float32)
    n = 20
    solo_tot = []
    for w, s0 in zip(ws, st0):
        G = _grid(bbx, w, s0)
        G.step(w.dt, n)
        solo_tot.append(G.step_total())
    grids = [_grid(bbx, w, s0) for w, s0 in zip(ws, st0)] + [_grid(bbx, empty, e0)]
    B = bbx.Batch(grids)
    B.step(n)
    B.sync()
    t, steps = grids[-1].get_time()
    assert steps == n and abs(t - n * empty.dt) < 1e-12
    for G, ref in zip(grids[:-1], solo_tot):
        assert G.get_time()[1] == n
        assert abs(G.step_total() - ref) <= 1e-12 * max(1.0, abs(ref))
    B.step(n)  # again: the per-grid piece counts were left at zero
    B.sync()
    assert grids[-1].get_time()[1] == 2 * n
    assert all(G.get_time()[1] == 2 * n for G in grids)
