"""Resident multi-step mode for small sheets (bbx_set_resident): a cluster of
CTAs keeps the sheet in distributed shared memory for many steps.  Checked
against the FP64 oracle (state, activation, totals, time) and against the
tiled kernel stepped one step per call."""
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


def _grid(bbx, w, st, resident=True):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_fibres(w.fibres, w.D_par, w.D_perp)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    G.write_all(st)
    if resident:
        G.set_resident(True)
    return G


def _oracle(w, st, n, stim=None):
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    sim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st.astype(np.float64))
    if stim is not None:
        sim.set_stimulus(*stim)
    sim.step(w.dt, n)
    return sim


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("shape", [(200, 200), (131, 37), (64, 300)])
def test_resident_fhn_sheet_matches_the_oracle(bbx, shape):
    w = wl.fhn_sheet(*shape)
    st = w.initial_state(oracle.rest_state(w.model, w.params)).astype(np.float32)
    G = _grid(bbx, w, st)
    G.step(w.dt, 100)
    sim = _oracle(w, st, 100)
    got = G.read_all()
    assert _rel(got[0], sim.state[0]) <= 1e-4 and _rel(got[1], sim.state[1]) <= 1e-3
    assert G.step_total() == pytest.approx(float(sim.state[0].sum()), rel=1e-5)
    t, n = G.get_time()
    assert n == 100 and t == pytest.approx(100 * w.dt, rel=1e-12)


def test_resident_activation_over_the_full_run(bbx):
    w = wl.fhn_sheet()
    st = w.initial_state(oracle.rest_state(w.model, w.params)).astype(np.float32)
    G = _grid(bbx, w, st)
    G.step(w.dt, w.n_steps)
    sim = _oracle(w, st, w.n_steps)
    ag = G.read_activation().astype(np.int64)
    ao = sim.act.astype(np.int64)
    big = w.n_steps + 1
    ag[ag == oracle.INT32_MAX] = big
    ao[ao == oracle.INT32_MAX] = big
    assert np.abs(ag - ao).max() <= 1 and np.count_nonzero(ao < big) > 1000


def test_resident_and_tiled_agree_and_mix(bbx):
    w = wl.fhn_sheet(150, 120)
    st = w.initial_state(oracle.rest_state(w.model, w.params)).astype(np.float32)
    R = _grid(bbx, w, st)
    T = _grid(bbx, w, st, resident=False)
    for n in (3, 1, 7, 2, 1, 6):  # odd counts exercise the buffer parity; n = 1 takes the tiled kernel
        R.step(w.dt, n)
    for _ in range(20):
        T.step(w.dt, 1)
    a, b = R.read_all(), T.read_all()
    assert _rel(a[0], b[0]) <= 2e-6 and _rel(a[1], b[1]) <= 2e-6
    assert R.get_time()[1] == T.get_time()[1] == 20


def test_resident_stimulus_window_barkley_sheet(bbx):
    nx, ny = 96, 80
    w = wl.Workload("bk2d", nx, ny, 1, 0.3, 0.005, wl.BARKLEY, [0.75, 0.02, 0.02], 1.0, 1.0, theta=0.5)
    st = np.zeros((2, 1, ny, nx), np.float32)
    reg = np.zeros((1, ny, nx), np.uint8)
    reg[0, 30:40, 10:20] = 1
    stim = (reg, 40.0, 0.02, 0.2)
    G = _grid(bbx, w, st)
    G.set_stimulus(*stim)
    G.step(w.dt, 300)
    sim = _oracle(w, st, 300, stim)
    got = G.read_all()
    assert _rel(got[0], sim.state[0]) <= 1e-4
    ag = G.read_activation().astype(np.int64)
    ao = sim.act.astype(np.int64)
    ag[ag == oracle.INT32_MAX] = 10 ** 6
    ao[ao == oracle.INT32_MAX] = 10 ** 6
    assert np.abs(ag - ao).max() <= 1 and np.count_nonzero(ao < 10 ** 6) > 50


def test_resident_refused_where_it_does_not_apply(bbx):
    w = wl.fhn_sheet(40, 30)
    st = w.initial_state(oracle.rest_state(w.model, w.params)).astype(np.float32)
    G = _grid(bbx, w, st, resident=False)
    G.set_resident(True)
    G.set_resident(False)
    mask = np.ones((1, 30, 40), np.uint8)
    mask[0, 0, 0] = 0
    M = bbx.Grid(40, 30, 1, 0.5, mask)
    M.set_ionic_model(bbx.BBX_FHN, None)
    with pytest.raises(bbx.BbxError):
        M.set_resident(True)
    s = wl.barkley_slab(32, 16, 8)
    S3 = bbx.Grid(s.nx, s.ny, s.nz, s.h, None)
    S3.set_ionic_model(bbx.BBX_BARKLEY, None)
    with pytest.raises(bbx.BbxError):
        S3.set_resident(True)
    big = bbx.Grid(2048, 2048, 1, 0.5, None)
    big.set_ionic_model(bbx.BBX_FHN, None)
    with pytest.raises(bbx.BbxError):
        big.set_resident(True)
