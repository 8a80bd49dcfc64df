"""GPU parity of the multivariate matrix Rush-Larsen model (BBX_BR_FCA:
Beeler-Reuter whose slow inward current is inactivated by a two-gate channel,
a voltage gate and a calcium gate, with a small direct transition between
them) against the FP64 oracle.  Both sides split the channel's generator
A(V, Ca) into the voltage gate's part, the calcium gate's part and the
remainder; the library takes the voltage gate's coefficients from its V-table
and the calcium gate's step in closed form, the oracle evaluates everything
per node with no table.  With the parameter onfly both sides apply the
exponential of the whole generator instead (the library by the Taylor series
of its action, the oracle by a scaled and squared matrix series)."""
import numpy as np
import pytest

import oracle
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

V_TOL = 1e-4      # relative L-infinity on V after 100 steps
OTHER_TOL = 1e-3  # Ca and the scalar gates, relative to their largest value
# the four channel probabilities, absolute: several of them stay near 0 over
# a run (relative bars would measure FP32 rounding of their pair totals, 6e-8
# a step); the cases below with a large eps make the remainder's effect on
# them (~1e-4 over 100 steps) far larger than this bar
Q_TOL = 1e-5
STRONG = [4.0, 0.003, 50.0, 0.09, 5e-6, 2.0, 2.0]  # eps = 2


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


def _grid(bbx, w, ty=None, tz=None, params=None):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_fibres(w.fibres, w.D_par, w.D_perp) if w.fibres is not None else G.set_fibres(None, w.D_par, w.D_par)
    if ty is not None:
        G.set_tiling(ty, tz)
    G.set_ionic_model(w.model, w.params if params is None else params)
    G.set_threshold(w.theta)
    return G


def _pair(bbx, w, n_steps, ty=None, tz=None, dt=None, params=None):
    par = w.params if params is None else params
    rest = oracle.rest_state(w.model, par)
    st0 = w.initial_state(rest).astype(np.float32)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=par, theta=w.theta, state=st0.astype(np.float64))
    G = _grid(bbx, w, ty, tz, params)
    G.write_all(st0)
    osim.step(dt or w.dt, n_steps)
    G.step(dt or w.dt, n_steps)
    return osim, G


def _check(osim, G):
    tis = osim.grid.psi
    got = G.read_all()
    e = [_rel_linf(got[v], osim.state[v], tis) for v in range(7)]
    q = [float(np.abs(got[v][tis] - osim.state[v][tis]).max()) for v in range(7, 11)]
    assert e[0] <= V_TOL, (e, q)
    assert max(e[1:]) <= OTHER_TOL, (e, q)
    assert max(q) <= Q_TOL, (e, q)
    return got


@pytest.mark.parametrize("ty,tz,par", [(7, 4, None), (14, 8, None), (7, 4, STRONG)])
def test_calcium_gated_slab_100_steps_against_the_oracle(bbx, ty, tz, par):
    w = wl.br_fca_slab(72, 20, 10)
    osim, G = _pair(bbx, w, 100, ty, tz, params=par)
    got = _check(osim, G)
    assert osim.state[0].max() > 0.0  # the upstroke is inside the run
    tis = osim.grid.psi
    assert np.abs(got[7:].sum(axis=0)[tis] - 1.0).max() < 1e-5  # probability conserved
    # the calcium gate has moved: Q2 + Q3 (c open) is not uniform any more
    c_open = (osim.state[9] + osim.state[10])[tis]
    assert c_open.max() - c_open.min() > 1e-3
    if par is STRONG:
        # the remainder moves more probability than the bar: a run without it
        # (eps = 0) is farther from the oracle than Q_TOL
        o0 = oracle.Sim(osim.grid, w.model, par=par[:6] + [0.0], theta=w.theta,
                        state=w.initial_state(oracle.rest_state(w.model, par)).astype(np.float32).astype(np.float64))
        o0.step(w.dt, 100)
        assert np.abs(o0.state[7:] - osim.state[7:]).max() > 5 * Q_TOL


@pytest.mark.parametrize("masked,eps", [(False, 0.05), (True, 0.05), (False, 2.0)])
def test_onfly_exponential_against_the_oracle(bbx, masked, eps):
    # onfly = 1: the channel by exp(dt A(V, Ca)) of the whole generator at
    # run time (the oracle's matrix exponential per node), 100 steps
    par = [4.0, 0.003, 50.0, 0.09, 5e-6, 2.0, eps, 1.0]
    if masked:
        w = wl.br_shell(48)
        w.model = wl.BR_FCA
    else:
        w = wl.br_fca_slab(72, 20, 10)
    osim, G = _pair(bbx, w, 100, 7, 4, params=par)
    got = _check(osim, G)
    tis = osim.grid.psi
    assert np.abs(got[7:].sum(axis=0)[tis] - 1.0).max() < 1e-5
    if not masked:
        # and it differs from the split step by the splitting error only
        osp, _ = _pair(bbx, w, 100, 7, 4, params=par[:7])
        d = np.abs(osp.state[7:] - osim.state[7:]).max()
        assert 0.0 < d < 1e-3


def test_calcium_gated_masked_shell_against_the_oracle(bbx):
    w = wl.br_shell(48)
    w.model = wl.BR_FCA
    osim, G = _pair(bbx, w, 60, 7, 4)
    _check(osim, G)


def test_calcium_gated_sheet_and_time_step_change(bbx):
    # a 2D sheet (planar kernel), and a new dt half way (the table is rebuilt)
    w = wl.br_fca_slab(90, 40, 1)
    osim, G = _pair(bbx, w, 40, 14, 1)
    osim.step(0.01, 40)
    G.step(0.01, 40)
    _check(osim, G)


def test_calcium_gate_time_constant_change_rebuilds_the_table(bbx):
    # a second model setting with another tau_c and eps on the same grid at
    # the same dt: the table's calcium constant follows the parameters
    w = wl.br_fca_slab(64, 14, 4)
    G = _grid(bbx, w, 7, 4)
    G.step(w.dt, 3)
    par = [4.0, 0.003, 50.0, 0.09, 5e-6, 10.0, 0.2]
    rest = oracle.rest_state(w.model, par)
    st0 = w.initial_state(rest).astype(np.float32)
    G.set_ionic_model(w.model, par)
    G.set_threshold(w.theta)
    G.write_all(st0)
    G.step(w.dt, 100)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=par, theta=w.theta, state=st0.astype(np.float64))
    osim.step(w.dt, 100)
    _check(osim, G)


def test_calcium_gated_activation_times_within_one_step(bbx):
    w = wl.br_fca_slab(64, 12, 4)
    osim, G = _pair(bbx, w, 1500)  # 30 ms: the wave crosses the slab
    act_o = osim.act
    act_g = G.read_activation()
    fired = act_o != oracle.INT32_MAX
    assert fired.sum() > 0.5 * fired.size
    assert np.array_equal(fired, act_g != bbx.BBX_ACT_NONE)
    assert np.abs(act_g[fired].astype(np.int64) - act_o[fired]).max() <= 1


def test_with_the_calcium_gate_held_open_it_is_the_scalar_br_kernel(bbx):
    # Kc huge: c_inf = 1, no remainder; with Q0 = Q1 = 0 the channel is the
    # scalar f gate (Q3 = f): V follows the library's Beeler-Reuter kernel
    wb = wl.br_slab(64, 24, 8)
    wf = wl.br_fca_slab(64, 24, 8)
    Gb = _grid(bbx, wb, 7, 8)
    Gf = _grid(bbx, wf, 7, 8, params=[4.0, 0.003, 50.0, 0.09, 1e20, 2.0, 0.05])
    rb = [float(Gb.read_state(v).reshape(-1)[0]) for v in range(8)]
    sb = wb.initial_state(rb).astype(np.float32)
    sf = np.zeros((11,) + wf.shape, np.float32)
    sf[:7] = sb[:7]
    sf[9] = 1.0 - sb[7]
    sf[10] = sb[7]
    Gb.write_all(sb)
    Gf.write_all(sf)
    Gb.step(wb.dt, 150)
    Gf.step(wf.dt, 150)
    b = Gb.read_all()
    f = Gf.read_all()
    assert b[0].max() > 0.0
    assert np.abs(f[0] - b[0]).max() / np.abs(b[0]).max() < 1e-4
    assert np.abs(f[10] - b[7]).max() < 1e-4
    assert np.abs(f[7:9]).max() < 1e-6


def test_calcium_gated_rest_state_and_refusals(bbx):
    w = wl.br_fca_slab(40, 8, 2)
    G = _grid(bbx, w)
    rest = np.array([float(G.read_state(v).reshape(-1)[0]) for v in range(11)])
    ro = oracle.rest_state(w.model, w.params)
    assert abs(rest[0] - ro[0]) < 0.05
    assert np.abs(rest[2:] - ro[2:]).max() < 2e-3
    assert abs(rest[1] - ro[1]) < 0.01 * ro[1]
    assert abs(rest[7:].sum() - 1.0) < 1e-5
    for call, arg in ((G.set_scheme, bbx.BBX_SCHEME_LIE), (G.set_solver, bbx.BBX_SOLVER_RK4),
                      (G.set_gate_storage, bbx.BBX_GATES_UNORM16), (G.set_tabulation, True)):
        with pytest.raises(bbx.BbxError) as e:
            call(arg)
        assert e.value.code == bbx.BBX_ERR_UNSUPPORTED
    G.step(w.dt, 50)  # the rest state stays put
    got = G.read_all()
    assert np.abs(got[0] - rest[0]).max() < 1e-3
    assert np.abs(got[7:] - rest[7:, None, None, None]).max() < 1e-5


def test_calcium_gated_grid_in_a_batch_matches_the_grid_stepped_alone(bbx):
    w = wl.br_fca_slab(64, 14, 4)
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    A = _grid(bbx, w, 7, 4)
    A.set_timestep(w.dt)
    A.write_all(st0)
    A.step(w.dt, 30)
    solo = A.read_all()
    B = _grid(bbx, w, 7, 4)
    B.set_timestep(w.dt)
    B.write_all(st0)
    F = _grid(bbx, wl.fhn_sheet(80, 40))
    F.set_timestep(0.01)
    batch = bbx.Batch([B, F])
    ty = batch.info()["tile_y"]
    batch.step(30)
    batch.sync()
    got = B.read_all()
    if 7 in ty and len(set(ty)) == len(ty):
        assert np.array_equal(got, solo)
    tis = np.ones(w.shape, bool)
    assert _rel_linf(got[0], solo[0], tis) < 1e-5
