"""GPU parity of Beeler-Reuter with tabulated Rush-Larsen coefficients
(bbx_set_tabulation: A(V), B(V) of Eq. RLcoeff and the V factors of I_x1 and
I_K1 from a table of V, interpolated linearly) against the FP64 oracle, which
evaluates them per node; and against the library's per-node kernel."""
import numpy as np
import pytest

import oracle
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

V_TOL = 1e-4
OTHER_TOL = 1e-3


@pytest.fixture(scope="module")
def bbx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx as b
    return b


def _rel_linf(got, ref, sel):
    scale = max(np.abs(ref[sel]).max(), 1e-30)
    return np.abs(got[sel] - ref[sel]).max() / scale


def _grid(bbx, w, ty=None, tz=None, tab=True):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_fibres(w.fibres, w.D_par, w.D_perp)
    if ty is not None:
        G.set_tiling(ty, tz)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    G.set_tabulation(tab)
    return G


def _pair(bbx, w, n_steps, ty=None, tz=None):
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
    G = _grid(bbx, w, ty, tz)
    G.write_all(st0)
    osim.step(w.dt, n_steps)
    G.step(w.dt, n_steps)
    return osim, G, st0


def _check(osim, G):
    tis = osim.grid.psi
    got = G.read_all()
    e = [_rel_linf(got[v], osim.state[v], tis) for v in range(osim.S)]
    assert e[0] <= V_TOL, e
    assert max(e[1:]) <= OTHER_TOL, e
    return got


@pytest.mark.parametrize("ty,tz", [(7, 4), (14, 8)])
def test_tabulated_slab_against_the_oracle_and_the_per_node_kernel(bbx, ty, tz):
    w = wl.br_slab(72, 20, 10)
    osim, G, st0 = _pair(bbx, w, 100, ty, tz)
    got = _check(osim, G)
    assert osim.state[0].max() > 0.0
    H = _grid(bbx, w, ty, tz, tab=False)
    H.write_all(st0)
    H.step(w.dt, 100)
    ref = H.read_all()
    assert not np.array_equal(got, ref)  # the table is in use
    assert _rel_linf(got[0], ref[0], osim.grid.psi) < 1e-4


def test_tabulated_masked_shell_against_the_oracle(bbx):
    osim, G, _ = _pair(bbx, wl.br_shell(48), 100, 7, 4)
    _check(osim, G)


def test_tabulated_time_step_change(bbx):
    w = wl.br_slab(60, 16, 6)
    osim, G, _ = _pair(bbx, w, 40)
    osim.step(0.01, 40)
    G.step(0.01, 40)
    _check(osim, G)


def test_tabulated_activation_times_within_one_step(bbx):
    w = wl.br_slab(64, 12, 4)
    osim, G, _ = _pair(bbx, w, 1500)
    fired = osim.act != oracle.INT32_MAX
    act_g = G.read_activation()
    assert fired.sum() > 0.5 * fired.size
    assert np.array_equal(fired, act_g != bbx.BBX_ACT_NONE)
    assert np.abs(act_g[fired].astype(np.int64) - osim.act[fired]).max() <= 1


def test_tabulation_is_for_beeler_reuter_only(bbx):
    w = wl.fhn_sheet(40, 20)
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h)
    G.set_ionic_model(w.model, w.params)
    with pytest.raises(bbx.BbxError) as e:
        G.set_tabulation(True)
    assert e.value.code == bbx.BBX_ERR_UNSUPPORTED
