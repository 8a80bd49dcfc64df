"""Pins of the oracle's Lie operator-splitting mode (section "Operator
splitting"): a diffusion substep on its own, then the kinetics step from the
half-step voltage with no diffusion term."""
import numpy as np
import scipy.ndimage

import oracle
from paper_1605_06015_gb300 import workloads as wl


def _sim(w, split, state):
    g = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    return oracle.Sim(g, w.model, par=w.params, theta=w.theta, state=state, split=split)


def test_one_fhn_step_is_the_printed_split_scheme():
    # the section's example: u_{n+1/2} = u_n + dt L u_n, then the FitzHugh-Nagumo
    # kinetics (cubic, reading c1) from (u_{n+1/2}, v_n); L by the textbook
    # 5-point Laplacian with no-flux edges
    w = wl.fhn_sheet(23, 17)
    st = w.initial_state(oracle.rest_state(oracle.FHN, w.params))
    sim = _sim(w, True, st)
    sim.step(w.dt, 1)
    eps, bet, gam = w.params
    u, v = st[0, 0], st[1, 0]
    lap = scipy.ndimage.laplace(u, mode="nearest") * (w.D_par / w.h ** 2)
    uh = u + w.dt * lap
    u1 = uh + w.dt * ((uh - uh ** 3 / 3.0 - v) / eps)
    v1 = v + w.dt * eps * (uh + bet - gam * v)
    assert np.allclose(sim.state[0, 0], u1, rtol=0, atol=1e-13)
    assert np.allclose(sim.state[1, 0], v1, rtol=0, atol=1e-13)


def test_pure_diffusion_split_equals_unsplit_bitwise():
    w = wl.barkley_slab(19, 13, 7)
    rng = np.random.default_rng(3)
    st = rng.random((1,) + w.shape)
    a = _sim(wl.Workload("d", w.nx, w.ny, w.nz, w.h, w.dt, oracle.DIFFUSION, [], w.D_par, w.D_perp,
                         fibres=w.fibres), False, st)
    b = _sim(wl.Workload("d", w.nx, w.ny, w.nz, w.h, w.dt, oracle.DIFFUSION, [], w.D_par, w.D_perp,
                         fibres=w.fibres), True, st)
    a.step(w.dt, 20)
    b.step(w.dt, 20)
    assert np.array_equal(a.state, b.state)


def test_homogeneous_tissue_split_equals_unsplit_bitwise():
    # L = 0 exactly on a uniform state: both schemes are the single-cell ODE
    w = wl.br_slab(9, 7, 5)
    y0 = oracle.rest_state(oracle.BR)
    y0[0] += 15.0
    st = np.empty((8,) + w.shape)
    for v in range(8):
        st[v] = y0[v]
    a, b = _sim(w, False, st), _sim(w, True, st)
    a.step(w.dt, 200)
    b.step(w.dt, 200)
    assert np.array_equal(a.state, b.state)


def test_split_differs_from_unsplit_at_first_order_in_dt():
    w = wl.fhn_sheet(24, 24)
    st = w.initial_state(oracle.rest_state(oracle.FHN, w.params))
    T = 0.4
    d = []
    for dt in (0.01, 0.005):
        n = int(round(T / dt))
        a, b = _sim(w, False, st), _sim(w, True, st)
        a.step(dt, n)
        b.step(dt, n)
        d.append(np.abs(a.state - b.state).max())
    ratio = d[0] / d[1]
    assert 1.7 < ratio < 2.3, (d, ratio)
