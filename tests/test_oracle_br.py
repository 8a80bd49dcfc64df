"""Pins of the oracle's Beeler-Reuter (1977) arithmetic: the rate table of
orc_br_rates and the currents of br_currents_m3.

The BeatBox paper names the model (section "Cell models", the ionic format)
but prints neither its equations nor its constants, so nothing here compares
with a number the paper prints.  Each test checks a property that follows
from the physics and physiology the 1977 model was built to reproduce, not
from the constant table itself:

  - rate constants are positive and finite at every voltage;
  - activation gates (x1, m, d) open with depolarisation and inactivation
    gates (h, j, f) close, each saturating at the ends of the physiological
    range, with half-points in the classical windows of the currents they
    gate (fast sodium activation and inactivation, slow inward calcium
    current, time-dependent outward potassium current);
  - the kinetic hierarchy of the Hodgkin-Huxley type formulation: sodium
    activation is the fastest gate everywhere, faster than sodium
    inactivation (h), which is faster than its slow reactivation (j);
    calcium activation (d) is faster than calcium inactivation (f); the
    outward current's gate x1 is slower than h, j and d everywhere;
  - reversal potentials: the sodium current vanishes at E_Na, the slow
    inward current at E_s(Ca) with the ln(Ca) slope RT/(2F) of a divalent
    ion, the potassium currents near the potassium equilibrium potential of
    ventricular muscle; the background potassium current I_K1 rectifies
    inwardly (its slope conductance near reversal is many times its
    plateau-range slope);
  - calcium balance: with no slow inward current Ca relaxes to 1e-7 M, an
    inward current raises it;
  - the whole cell: a stable resting potential, a threshold between a
    decaying and a propagating depolarisation, an overshoot, a plateau, and
    repolarisation within the action potential durations of ventricular
    muscle.

The mutation check in the design doc lists which single-constant transcription
slips of the table these tests catch.
"""
import numpy as np
import pytest

import oracle

GATES = ["x1", "m", "h", "j", "d", "f"]
ACTIVATION = ["x1", "m", "d"]
INACTIVATION = ["h", "j", "f"]
VGRID = np.linspace(-100.0, 40.0, 1401)  # 0.1 mV


def _rates(vs):
    A = np.empty((len(vs), 6))
    B = np.empty((len(vs), 6))
    for i, v in enumerate(vs):
        A[i], B[i] = oracle.br_rates(v)
    return A, B


@pytest.fixture(scope="module")
def kinetics():
    A, B = _rates(VGRID)
    yinf = A / (A + B)
    tau = 1.0 / (A + B)
    return A, B, yinf, tau


def _g(name):
    return GATES.index(name)


def test_rates_positive_and_finite_everywhere():
    vs = np.linspace(-120.0, 80.0, 4001)  # includes the removable points -47 and -23
    A, B = _rates(vs)
    assert np.all(np.isfinite(A)) and np.all(np.isfinite(B))
    assert np.all(A > 0) and np.all(B > 0)


def test_steady_states_open_or_close_with_depolarisation(kinetics):
    _, _, yinf, _ = kinetics
    for n in ACTIVATION:
        y = yinf[:, _g(n)]
        assert np.all(np.diff(y) >= -1e-15), n
        assert y[0] < 0.05 and y[-1] > 0.95, (n, y[0], y[-1])
    for n in INACTIVATION:
        y = yinf[:, _g(n)]
        assert np.all(np.diff(y) <= 1e-15), n
        assert y[0] > 0.95 and y[-1] < 0.05, (n, y[0], y[-1])


def _half_point(y):
    i = int(np.argmin(np.abs(y - 0.5)))
    return VGRID[i]


def test_half_activation_voltages_in_their_classical_windows(kinetics):
    _, _, yinf, _ = kinetics
    v = {n: _half_point(yinf[:, _g(n)]) for n in GATES}
    assert -60.0 <= v["m"] <= -35.0, v    # fast sodium activation
    assert -85.0 <= v["h"] <= -60.0, v    # sodium inactivation
    assert -85.0 <= v["j"] <= -60.0, v    # slow sodium reactivation
    assert -40.0 <= v["d"] <= -10.0, v    # slow inward (calcium) activation
    assert -40.0 <= v["f"] <= -10.0, v    # its inactivation
    assert -40.0 <= v["x1"] <= 0.0, v     # time-dependent outward current
    # the sodium window: inactivation half-point well below activation
    assert v["h"] < v["m"] - 10.0 and v["j"] < v["m"] - 10.0, v


def test_kinetic_hierarchy_of_the_gates(kinetics):
    _, _, _, tau = kinetics
    t = {n: tau[:, _g(n)] for n in GATES}
    for other in ("x1", "h", "j", "d", "f"):
        assert np.all(t["m"] < t[other]), other
    assert np.all(t["h"] < t["j"])
    assert np.all(t["d"] < t["f"])
    for other in ("h", "j", "d"):
        assert np.all(t[other] < t["x1"]), other
    # magnitudes: sub-millisecond sodium activation, millisecond sodium
    # inactivation, tens of ms for the slow inward current's gates, hundreds
    # of ms for x1
    assert t["m"].max() < 1.0
    assert 1.0 < t["h"].max() < 50.0
    assert 5.0 < t["d"].max() < 100.0
    assert t["f"].max() > 100.0 and t["x1"].max() > 100.0


def test_time_constants_are_largest_near_the_half_points(kinetics):
    # For a gate with one rate rising and the other falling with V, tau =
    # 1/(alpha+beta) peaks where alpha ~ beta, i.e. near y_inf = 1/2.
    A, B, yinf, tau = kinetics
    for n in ("x1", "m", "h", "j", "d"):
        g = _g(n)
        vmax = VGRID[int(np.argmax(tau[:, g]))]
        assert abs(vmax - _half_point(yinf[:, g])) < 6.0, (n, vmax)


PAR_NO_BACKGROUND = [4.0, 0.0, 50.0, 0.09]  # gNa, gNaC = 0, ENa, gs


def _I(v, x1=0.0, m=0.0, h=0.0, j=0.0, d=0.0, f=0.0, ca=1e-7, par=PAR_NO_BACKGROUND):
    y = np.array([v, ca, x1, m, h, j, d, f])
    return oracle.br_currents(y, par)  # I_ion, I_s, dCa/dt


def I_K1(v):
    return _I(v)[0]  # every gate closed, no background sodium conductance


def I_x1_per_gate(v):
    return _I(v, x1=1.0)[0] - _I(v)[0]


def test_sodium_current_reverses_at_ENa():
    rng = np.random.default_rng(3)
    for ena in (50.0, 40.0, 65.0):
        par = [4.0, 0.003, ena, 0.09]
        for _ in range(5):
            m, h, j = rng.random(3)
            on = _I(ena, m=m, h=h, j=j, par=par)[0]
            off = _I(ena, par=par)[0]
            assert abs(on - off) < 1e-12  # I_Na = 0 at V = ENa
        # inward below ENa, proportional to the conductance g m^3 h j
        g1 = _I(ena - 30.0, m=1, h=1, j=1, par=par)[0] - _I(ena - 30.0, par=par)[0]
        assert g1 == pytest.approx(-4.0 * 30.0, rel=1e-12)


def test_slow_inward_current_reverses_at_the_calcium_potential():
    # E_s = E0 - k ln[Ca]: I_s vanishes there for any Ca, and k is the
    # divalent Nernst slope RT/(2F) at a temperature of the preparation.
    R, F = 8.314462618, 96485.33212
    es = {}
    for ca in (1e-7, 3e-7, 1e-6):
        vs = np.linspace(0.0, 250.0, 2501)
        Is = np.array([_I(v, d=1.0, f=1.0, ca=ca)[1] for v in vs])
        k = int(np.nonzero(np.diff(np.sign(Is)))[0][0])
        es[ca] = vs[k] - Is[k] * (vs[k + 1] - vs[k]) / (Is[k + 1] - Is[k])
        assert abs(_I(es[ca], d=1.0, f=1.0, ca=ca)[1]) < 1e-9
    slope = (es[1e-7] - es[1e-6]) / np.log(10.0)  # mV per e-fold of Ca
    T = slope * 1e-3 * 2 * F / R
    assert 290.0 < T < 315.0, T
    assert 100.0 < es[1e-7] < 150.0  # strongly positive at resting calcium


def test_potassium_currents_reverse_near_EK_and_IK1_rectifies_inwardly():
    vs = np.linspace(-110.0, 40.0, 1501)
    ik1 = np.array([I_K1(v) for v in vs])
    ix1 = np.array([I_x1_per_gate(v) for v in vs])
    for cur in (ik1, ix1):
        up = np.nonzero((cur[:-1] < 0) & (cur[1:] >= 0))[0]
        down = np.nonzero((cur[:-1] >= 0) & (cur[1:] < 0))[0]
        assert up.size == 1 and down.size == 0  # one reversal, inward below it
        assert -95.0 < vs[up[0]] < -70.0, vs[up[0]]
    # outward above reversal up to +40 mV, inward below
    assert np.all(ik1[vs > -80] > 0) and np.all(ik1[vs < -95] < 0)
    # inward rectification: large slope conductance near reversal, small on
    # the plateau
    g_rev = (I_K1(-85.0) - I_K1(-95.0)) / 10.0
    g_plat = abs(I_K1(-20.0) - I_K1(-50.0)) / 30.0
    assert g_rev > 10.0 * g_plat, (g_rev, g_plat)
    assert np.all(np.diff(ix1) > 0)  # x1 current: monotone, no rectification hump


def test_calcium_relaxes_to_its_resting_level():
    for ca in (5e-8, 1e-7, 4e-7):
        d = _I(-84.0, ca=ca)[2]  # d = f = 0: no slow inward current
        assert d == pytest.approx(0.07 * (1e-7 - ca), rel=1e-12, abs=1e-22)
    # an inward slow current (I_s < 0) raises Ca
    I, Is, dca = _I(0.0, d=1.0, f=1.0, ca=1e-7)
    assert Is < 0 and dca > 0


def _ap(y, dt=0.01, T=600.0):
    n = int(round(T / dt))
    V = np.empty(n)
    for i in range(n):
        y = oracle.cell_update(oracle.BR, y, dt=dt)
        V[i] = y[0]
    return np.arange(1, n + 1) * dt, V, y


def test_whole_cell_threshold_action_potential_and_repolarisation():
    rest = oracle.rest_state(oracle.BR)
    assert -86.0 < rest[0] < -83.0
    # the rest state is a fixed point of the step
    assert np.allclose(oracle.cell_update(oracle.BR, rest, dt=0.01), rest, rtol=0, atol=1e-9)
    # subthreshold depolarisation decays back
    y = rest.copy(); y[0] = -70.0
    t, V, _ = _ap(y, T=50.0)
    assert V.max() < -69.0 and abs(V[-1] - rest[0]) < 2.0
    # suprathreshold: overshoot, plateau, repolarisation
    y = rest.copy(); y[0] = -40.0
    t, V, yend = _ap(y)
    assert 20.0 < V.max() < 60.0
    tpk = t[int(np.argmax(V))]
    assert tpk < 10.0
    amp = V.max() - rest[0]
    apd90 = t[np.nonzero((t > tpk) & (V < rest[0] + 0.1 * amp))[0][0]] - tpk
    assert 200.0 < apd90 < 400.0, apd90
    plateau = V[(t > 50.0) & (t < 150.0)]
    assert plateau.min() > -40.0 and plateau.max() < 20.0
    assert abs(yend[0] - rest[0]) < 1.5  # back to rest by 600 ms
