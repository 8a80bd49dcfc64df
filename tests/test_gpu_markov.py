"""GPU parity of the matrix Rush-Larsen model (BBX_BR_MRL: Beeler-Reuter with
the sodium activation in its Markov form, the chain advanced by a tabulated
T(V) = exp(dt A(V))) against the FP64 oracle, which computes T per node with
no table; and against the library's own scalar Beeler-Reuter kernel, which
the Markov form reproduces exactly in exact arithmetic."""
from math import comb

import numpy as np
import pytest

import oracle
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

V_TOL = 1e-4      # relative L-infinity on V after 100 steps
OTHER_TOL = 1e-3  # other state variables


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


def _grid(bbx, w, ty=None, tz=None):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_fibres(w.fibres, w.D_par, w.D_perp) if w.fibres is not None else G.set_fibres(None, w.D_par, w.D_par)
    if ty is not None:
        G.set_tiling(ty, tz)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    return G


def _pair(bbx, w, n_steps, ty=None, tz=None, dt=None):
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
    G = _grid(bbx, w, ty, tz)
    G.write_all(st0)
    osim.step(dt or w.dt, n_steps)
    G.step(dt or w.dt, n_steps)
    return osim, G


def _check(osim, G):
    tis = osim.grid.psi
    got = G.read_all()
    e = [_rel_linf(got[v], osim.state[v], tis) for v in range(osim.S)]
    assert e[0] <= V_TOL, e
    assert max(e[1:]) <= OTHER_TOL, e
    return got


@pytest.mark.parametrize("ty,tz", [(7, 4), (14, 8)])
def test_markov_slab_100_steps_against_the_oracle(bbx, ty, tz):
    w = wl.br_mrl_slab(72, 20, 10)
    osim, G = _pair(bbx, w, 100, ty, tz)
    got = _check(osim, G)
    assert osim.state[0].max() > 0.0  # the upstroke is inside the run
    tis = osim.grid.psi
    assert np.abs(got[7:].sum(axis=0)[tis] - 1.0).max() < 1e-5  # probability conserved


def test_markov_masked_shell_against_the_oracle(bbx):
    w = wl.br_shell(48)
    w.model = wl.BR_MRL
    osim, G = _pair(bbx, w, 60, 7, 4)
    _check(osim, G)


def test_markov_sheet_and_time_step_change(bbx):
    # a 2D sheet (planar kernel), and a new dt half way (the table is rebuilt)
    w = wl.br_mrl_slab(90, 40, 1)
    osim, G = _pair(bbx, w, 40, 14, 1)
    osim.step(0.01, 40)
    G.step(0.01, 40)
    _check(osim, G)


def test_markov_activation_times_within_one_step(bbx):
    w = wl.br_mrl_slab(64, 12, 4)
    osim, G = _pair(bbx, w, 1500)  # 30 ms: the wave crosses the slab
    act_o = osim.act
    act_g = G.read_activation()
    fired = act_o != oracle.INT32_MAX
    assert fired.sum() > 0.5 * fired.size
    assert np.array_equal(fired, act_g != bbx.BBX_ACT_NONE)
    assert np.abs(act_g[fired].astype(np.int64) - act_o[fired]).max() <= 1


def test_markov_form_reproduces_the_scalar_br_kernel(bbx):
    # same slab, scalar m gate (BBX_BR) and Markov chain (BBX_BR_MRL) from the
    # binomial distribution of the same m: V agrees to the table's
    # interpolation and float rounding, P3 tracks m^3
    wb = wl.br_slab(64, 24, 8)
    wm = wl.br_mrl_slab(64, 24, 8)
    Gb = _grid(bbx, wb, 7, 8)
    Gm = _grid(bbx, wm, 7, 8)
    rb = [float(Gb.read_state(v).reshape(-1)[0]) for v in range(8)]
    sb = wb.initial_state(rb).astype(np.float32)
    m = sb[3].astype(np.float64)
    sm = np.empty((11,) + wm.shape, np.float32)
    for dst, src in zip(range(7), (0, 1, 2, 4, 5, 6, 7)):
        sm[dst] = sb[src]
    for k in range(4):
        sm[7 + k] = comb(3, k) * m ** k * (1 - m) ** (3 - k)
    Gb.write_all(sb)
    Gm.write_all(sm)
    Gb.step(wb.dt, 150)
    Gm.step(wm.dt, 150)
    b = Gb.read_all()
    mm = Gm.read_all()
    assert b[0].max() > 0.0
    assert np.abs(mm[0] - b[0]).max() / np.abs(b[0]).max() < 1e-4
    assert np.abs(mm[10] - b[3].astype(np.float64) ** 3).max() < 1e-4


def test_markov_rest_state_and_refusals(bbx):
    # the library's rest state: its Beeler-Reuter rest state with the chain
    # at the binomial distribution of m
    w = wl.br_mrl_slab(40, 8, 2)
    G = _grid(bbx, w)
    rest = np.array([float(G.read_state(v).reshape(-1)[0]) for v in range(11)])
    Gb = _grid(bbx, wl.br_slab(40, 8, 2))
    rb = np.array([float(Gb.read_state(v).reshape(-1)[0]) for v in range(8)])
    assert np.array_equal(rest[:7], rb[[0, 1, 2, 4, 5, 6, 7]])
    m = float(rb[3])
    assert np.allclose(rest[7:], [(1 - m) ** 3, 3 * m * (1 - m) ** 2, 3 * m * m * (1 - m), m ** 3], rtol=1e-6, atol=0)
    with pytest.raises(bbx.BbxError) as e:
        G.set_scheme(bbx.BBX_SCHEME_LIE)
    assert e.value.code == bbx.BBX_ERR_UNSUPPORTED
    with pytest.raises(bbx.BbxError) as e:
        G.set_solver(bbx.BBX_SOLVER_RK4)
    assert e.value.code == bbx.BBX_ERR_UNSUPPORTED
    G.step(w.dt, 5)  # still steps
    assert np.isfinite(G.read_all()).all()


def test_markov_grid_in_a_batch_matches_the_grid_stepped_alone(bbx):
    w = wl.br_mrl_slab(64, 14, 4)
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
