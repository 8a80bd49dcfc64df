"""z-slab decomposition on one GPU (section "Domain partitioning"): a grid cut
into 2 and 4 slabs, each a bbx grid with halo planes, halo planes refreshed
by bbx_halo_exchange before every step.  The slabs' own planes equal the
undivided grid stepped on the GPU at the same tile shape bitwise (every node
computes the same arithmetic from the same neighbours), and the FP64 oracle
on the undivided grid within the parity bars; the slabs' tissue sums add up
to the whole grid's."""
import numpy as np
import pytest

import oracle
from paper_1605_06015_gb300 import slabs
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx
    return torch, bbx


def _workload(kind):
    if kind == "barkley_masked":
        mask, fib = wl.random_geometry(96, 40, 30, seed=41, tissue_frac=0.85)
        w = wl.barkley_slab(96, 40, 30)
        w.mask, w.fibres = mask, fib
        return w
    if kind == "barkley_slab":
        return wl.barkley_slab(130, 50, 26)
    return wl.br_shell(64)


def _grid(bbx, w, a=0, b=None, lo=0, hi=0):
    b = w.nz if b is None else b
    G = bbx.Grid(w.nx, w.ny, b - a, w.h, None if w.mask is None else w.mask[a:b])
    G.set_fibres(None if w.fibres is None else w.fibres[a:b], w.D_par, w.D_perp)
    G.set_tiling(14, 8)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    if lo or hi:
        G.set_halo_planes(lo, hi)
    return G


@pytest.mark.parametrize("kind,parts", [("barkley_masked", 2), ("barkley_masked", 4), ("barkley_slab", 3),
                                        ("br_shell", 4)])
def test_slabs_on_one_device_equal_the_undivided_grid(env, kind, parts):
    torch, bbx = env
    w = _workload(kind)
    n = 100
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    whole = _grid(bbx, w)
    whole.write_all(st0)
    whole.step(w.dt, n)
    ref = whole.read_all()
    ref_act = whole.read_activation()
    ref_total = whole.step_total()
    parts_g, bounds = [], []
    for i in range(parts):
        a, b, lo, hi = slabs.local_bounds(w.nz, parts, i)
        G = _grid(bbx, w, a, b, lo, hi)
        G.write_all(np.ascontiguousarray(st0[:, a:b]))
        parts_g.append(G)
        bounds.append((a, b, lo, hi))
        assert G.get_info()["n_tissue"] == int(
            np.count_nonzero(w.mask[a + lo:b - hi]) if w.mask is not None else w.nx * w.ny * (b - a - lo - hi))
    slabs.step_on_one_device(parts_g, w.dt, n)
    got = np.concatenate([G.read_all()[:, lo:(b - a) - hi] for G, (a, b, lo, hi) in zip(parts_g, bounds)], axis=1)
    got_act = np.concatenate([G.read_activation()[lo:(b - a) - hi] for G, (a, b, lo, hi) in zip(parts_g, bounds)])
    tis = np.ones(w.shape, bool) if w.mask is None else w.mask != 0
    assert np.array_equal(got[:, tis], ref[:, tis])
    assert np.array_equal(got_act, ref_act)
    tot = sum(G.step_total() for G in parts_g)
    assert tot == pytest.approx(ref_total, rel=1e-10)
    assert sum(G.total(0) for G in parts_g) == pytest.approx(whole.total(0), rel=1e-10)
    # and the oracle on the undivided grid
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
    osim.step(w.dt, n)
    e = np.abs(got[0][tis] - osim.state[0][tis]).max() / np.abs(osim.state[0][tis]).max()
    assert e <= 1e-4, e
    ao, ag = osim.act.astype(np.int64), got_act.astype(np.int64)
    ao[ao == oracle.INT32_MAX] = n + 1
    ag[ag == oracle.INT32_MAX] = n + 1
    assert np.abs(ao - ag)[tis].max() <= 1
    if w.model != oracle.BR:
        assert (ao[tis] <= n).sum() > 0  # a wave crossed (the BR shell's stays near its ball in 100 steps)
    for G in parts_g:
        G.close()
    whole.close()


def test_slab_grid_planes_are_views_of_the_bound_buffers(env):
    # The rank path: each part's state in torch buffers bound to its grid, the
    # halo planes exchanged as tensor views (here by plain copies on one
    # device, where ranks would send and receive them).
    torch, bbx = env
    w = wl.barkley_slab(70, 30, 20)
    n = 60
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    whole = _grid(bbx, w)
    whole.write_all(st0)
    whole.step(w.dt, n)
    ref = whole.read_all()
    P = [slabs.SlabGrid(w, 2, i) for i in range(2)]
    for p in P:
        p.G.set_tiling(14, 8)
        p.write_global_state(st0)
    for _ in range(n):
        lo_send, lo_recv = P[1]._view(0, 0), P[1]._view(0, 1)
        hi_send, hi_recv = P[0]._view(1, 0), P[0]._view(1, 1)
        lo_recv.copy_(hi_send)
        hi_recv.copy_(lo_send)
        for p in P:
            p.G.step(w.dt, 1)
    got = np.concatenate([p.own(p.G.read_all()) for p in P], axis=1)
    assert np.array_equal(got, ref)
    for p in P:
        p.close()
    whole.close()


def test_halo_api_errors(env):
    torch, bbx = env
    w = wl.barkley_slab(40, 20, 6)
    G = _grid(bbx, w)
    with pytest.raises(bbx.BbxError):
        bbx.bbx_halo_plane(G.g, 0, 1)  # no halo plane yet
    with pytest.raises(bbx.BbxError):
        G.set_halo_planes(2, 0)
    G.set_halo_planes(1, 1)
    assert G.get_info()["n_tissue"] == 40 * 20 * 4
    H = _grid(bbx, w)
    with pytest.raises(bbx.BbxError):
        bbx.bbx_halo_exchange(G.g, H.g)  # H has no halo plane below
    G.close()
    H.close()
