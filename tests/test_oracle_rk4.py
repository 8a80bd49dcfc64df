"""Pins of the oracle's classical fourth-order Runge-Kutta kinetics step (the
rk4 solver of section "Explicit solvers"): fourth-order convergence against
an independent high-accuracy ODE solve, exactness for a constant source,
grid = single cell for homogeneous tissue, and the source entering the
voltage equation only."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
from paper_1605_06015_gb300 import workloads as wl

FHN_PAR = [0.3, 0.71, 0.5]
BARKLEY_PAR = [0.75, 0.02, 0.02]


def _fhn(t, y, I):
    eps, bet, gam = FHN_PAR
    return [(y[0] - y[0] ** 3 / 3 - y[1]) / eps + I, eps * (y[0] + bet - gam * y[1])]


def _barkley(t, y, I):
    a, b, eps = BARKLEY_PAR
    return [y[0] * (1 - y[0]) * (y[0] - (y[1] + b) / a) / eps + I, y[0] - y[1]]


@pytest.mark.parametrize("model,par,f,y0,T,dts", [
    (oracle.FHN, FHN_PAR, _fhn, [1.2, -0.4], 1.0, (0.02, 0.01)),
    (oracle.BARKLEY, BARKLEY_PAR, _barkley, [0.6, 0.1], 0.1, (0.004, 0.002)),
])
def test_fourth_order_against_an_independent_solve(model, par, f, y0, T, dts):
    I = 0.37  # a frozen diffusion term plus stimulus
    ref = solve_ivp(f, (0.0, T), y0, args=(I,), method="DOP853", rtol=1e-13, atol=1e-15).y[:, -1]
    err = []
    for dt in dts:
        y = np.array(y0, dtype=float)
        for _ in range(int(round(T / dt))):
            y = oracle.cell_update_rk4(model, y, L=0.3, Istim=0.07, dt=dt, par=par)
        err.append(np.abs(y - ref).max())
    ratio = err[0] / err[1]
    assert 13.0 < ratio < 19.0, (err, ratio)
    # forward Euler on the same problem is only first order
    eu = []
    for dt in dts:
        y = np.array(y0, dtype=float)
        for _ in range(int(round(T / dt))):
            y = oracle.cell_update(model, y, L=0.3, Istim=0.07, dt=dt, par=par)
        eu.append(np.abs(y - ref).max())
    assert 1.6 < eu[0] / eu[1] < 2.4 and err[1] < 1e-3 * eu[1]


def test_constant_source_is_integrated_exactly():
    y = oracle.cell_update_rk4(oracle.DIFFUSION, np.array([0.25]), L=1.5, Istim=-0.5, dt=0.125)
    assert y[0] == 0.25 + 0.125 * 1.0


def test_grid_rk4_on_homogeneous_tissue_is_the_single_cell_step():
    w = wl.barkley_slab(9, 7, 5)
    y0 = np.array([0.55, 0.12])
    st = np.empty((2,) + w.shape)
    st[0], st[1] = y0[0], y0[1]
    g = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    sim = oracle.Sim(g, oracle.BARKLEY, par=BARKLEY_PAR, state=st, rk4=True)
    sim.step(w.dt, 30)
    y = y0.copy()
    for _ in range(30):
        y = oracle.cell_update_rk4(oracle.BARKLEY, y, dt=w.dt, par=BARKLEY_PAR)
    assert np.array_equal(sim.state[0], np.full(w.shape, y[0]))
    assert np.array_equal(sim.state[1], np.full(w.shape, y[1]))


def test_rk4_is_refused_for_the_rush_larsen_model():
    w = wl.br_slab(6, 5, 4)
    g = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    sim = oracle.Sim(g, oracle.BR, rk4=True)
    with pytest.raises(RuntimeError):
        sim.step(w.dt, 1)
