"""W-tilde sums that vanish are not loaded (bbx_set_wsum_elision).

The W-tilde part of the weights of Eq. (W) differences the diffusion tensor
across a node.  For fibres in the x-y plane turning with z only (the
rotational anisotropy of the slab workloads) and for uniform fibres, every
such sum is exactly zero.  A single-grid step then runs a kernel variant
without the sums (plain kernels of unmasked grids) or skips their copies and
uses zeros (masked grids, the general variants).  The result must be bitwise
the one with the sums loaded, and stay within the oracle bars."""
import numpy as np
import pytest

import oracle
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

V_TOL = 1e-4


@pytest.fixture(scope="module")
def bbx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx as b
    return b


def _uniform_fibres(nx, ny, nz, f=(1.0, 0.5, 0.25)):
    fib = np.empty((nz, ny, nx, 3), dtype=np.float32)
    fib[...] = np.asarray(f, dtype=np.float32)
    return fib


def _grid(bbx, w, fibres, elide, ty=None, setup=None):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_wsum_elision(elide)
    G.set_fibres(fibres, w.D_par, w.D_perp)
    if ty is not None:
        G.set_tiling(ty, 16)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    if setup is not None:
        setup(G)
    return G


def _run(bbx, w, fibres, elide, n_steps, ty=None, setup=None):
    G = _grid(bbx, w, fibres, elide, ty, setup)
    rest = [float(G.read_state(v).reshape(-1)[0]) for v in range(G.get_info()["nvars"])]
    G.write_all(w.initial_state(rest).astype(np.float32))
    G.step(w.dt, n_steps)
    return G, G.read_all(), G.read_activation(), G.step_total(), G.get_info()["wsum_skipped"]


def _barkley(nx, ny, nz, mask=None):
    w = wl.barkley_slab(nx, ny, nz)
    w.mask = mask
    return w


def _tabulated(G):
    G.set_tabulation(True)


def _lie(G):
    G.set_scheme(1)


# The plain kernels of unmasked grids have a variant without the sums; masked
# grids and the general variants (Lie scheme, RK4, tabulation) keep the sums
# in the stage ring and skip only their copies.
CASES = [
    # name, workload, fibres, steps, tile rows, extra set-up
    ("rotational slab, 7-row tiles", lambda: _barkley(100, 37, 19), "rot", 60, 7, None),
    ("rotational slab, 14-row tiles", lambda: _barkley(100, 37, 19), "rot", 60, 14, None),
    ("rotational slab, 28-row tiles", lambda: _barkley(130, 61, 11), "rot", 60, 28, None),
    ("rotational slab, Lie scheme", lambda: _barkley(100, 37, 19), "rot", 60, 14, _lie),
    ("masked block, uniform fibres", lambda: _barkley(
        70, 45, 20, wl.random_geometry(70, 45, 20, seed=7, tissue_frac=0.8, aniso=False)[0]), "uni", 40, None,
     None),
    ("sheet, uniform oblique fibres", lambda: wl.fhn_sheet(150, 70), "uni2d", 80, None, None),
    ("Beeler-Reuter slab, rotational", lambda: wl.br_slab(96, 40, 12), "rot", 40, None, None),
    ("Beeler-Reuter slab, tabulated", lambda: wl.br_slab(96, 40, 12), "rot", 40, 7, _tabulated),
]


def _fibres(w, kind):
    if kind == "rot":
        return wl.rotational_fibres(w.nx, w.ny, w.nz)
    if kind == "uni2d":
        return _uniform_fibres(w.nx, w.ny, w.nz, (0.6, 0.8, 0.0))
    return _uniform_fibres(w.nx, w.ny, w.nz)


@pytest.mark.parametrize("name,make,kind,n_steps,ty,setup", CASES, ids=[c[0] for c in CASES])
def test_skipped_sums_give_the_loaded_result_bitwise(bbx, name, make, kind, n_steps, ty, setup):
    w = make()
    if kind == "uni2d":
        w.D_par, w.D_perp = 1.0, 0.3
    fib = _fibres(w, kind)
    on = _run(bbx, w, fib, True, n_steps, ty, setup)
    off = _run(bbx, w, fib, False, n_steps, ty, setup)
    assert on[4] == 1 and off[4] == 0
    assert np.array_equal(on[1].view(np.uint32), off[1].view(np.uint32))
    assert np.array_equal(on[2], off[2])
    assert on[3] == off[3]


def test_sums_that_do_not_vanish_are_loaded(bbx):
    # smooth fibres with a z component: the sums are nonzero, nothing is skipped
    w = _barkley(64, 30, 12)
    fib = wl.smooth_fibres(w.nx, w.ny, w.nz, w.h)
    G = _grid(bbx, w, fib, True)
    assert G.get_info()["wsum_skipped"] == 0
    # isotropic grids have no sums at all
    G2 = _grid(bbx, w, None, True)
    assert G2.get_info()["wsum_skipped"] == 0
    # a field with one rotated fibre somewhere: nonzero sums around it
    fib = wl.rotational_fibres(w.nx, w.ny, w.nz)
    fib[5, 10, 20] = np.array([0.0, 0.6, 0.8], dtype=np.float32)
    G3 = _grid(bbx, w, fib, True)
    assert G3.get_info()["wsum_skipped"] == 0
    # and back to the rotational field: skipped again
    G3.set_fibres(wl.rotational_fibres(w.nx, w.ny, w.nz), w.D_par, w.D_perp)
    assert G3.get_info()["wsum_skipped"] == 1


def test_skipped_sums_against_the_oracle(bbx):
    # the rotational slab with the sums skipped, 100 steps, against the FP64 oracle
    w = _barkley(100, 37, 19)
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
    osim.step(w.dt, 100)
    G = _grid(bbx, w, w.fibres, True)
    assert G.get_info()["wsum_skipped"] == 1
    G.write_all(st0)
    G.step(w.dt, 100)
    V = G.read_state(0).astype(np.float64)
    ref = osim.state[0]
    assert np.abs(V - ref).max() / np.abs(ref).max() <= V_TOL
