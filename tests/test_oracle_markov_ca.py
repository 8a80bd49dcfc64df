"""Pins of the multivariate matrix Rush-Larsen scheme in the oracle (section
"Exponential solvers": a generator A(V, Ca) written as a sum of univariate
matrices plus a small multivariate remainder, integrated by Lie splitting, each
univariate subsystem by its exact step and the remainder by forward Euler).

The model (BR_FCA) gives the slow inward current of Beeler-Reuter a two-gate
inactivation channel: the voltage gate f of the 1977 model and a calcium gate
c (closed -> open at c_inf / tau_c, open -> closed at (1 - c_inf) / tau_c,
c_inf = 1 / (1 + Ca / Kc)); the four channel states q = f + 2 c; the remainder
is a direct (f open, c closed) -> (f closed, c open) transition at eps
alpha_f (1 - c_inf).

What fixes the oracle here without reference to itself: two independent gates
have the Kronecker-sum generator and the Kronecker-product transition matrix;
the exact step is the matrix exponential (scipy's expm, a different
algorithm); Lie splitting is first order globally, second order per step; a
stochastic matrix keeps probability; with the calcium gate held open the
model is the 1977 Beeler-Reuter model."""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle

VS = [-90.0, -84.0, -60.0, -40.0, -20.0, 0.0, 30.0]
CAS = [1e-7, 5e-7, 2e-6, 1e-5]
KC, TAUC, EPS = oracle.FCA_DEFAULTS[4:7]


def _gate(a, b):
    """Generator of one two-state gate over (closed, open)."""
    return np.array([[-a, b], [a, -b]])


def _rates(V, Ca, Kc=KC, tauc=TAUC):
    al, be = oracle.br_rates(V)
    ci = 1.0 / (1.0 + Ca / Kc)
    return al[5], be[5], ci / tauc, (1.0 - ci) / tauc, ci


def test_generator_is_the_kronecker_sum_of_the_gates_plus_the_remainder():
    I2 = np.eye(2)
    for V in VS:
        for Ca in CAS:
            af, bf, ac, bc, ci = _rates(V, Ca)
            # state index q = f + 2 c: c is the major index, f the minor one
            ref = np.kron(I2, _gate(af, bf)) + np.kron(_gate(ac, bc), I2)
            r = EPS * af * (1.0 - ci)
            ref[2, 1] += r
            ref[1, 1] -= r
            A = oracle.fca_generator(V, Ca)
            assert np.allclose(A, ref, rtol=1e-14, atol=1e-18)
            assert np.all(A - np.diag(np.diag(A)) >= 0.0)
            assert np.allclose(A.sum(axis=0), 0.0, atol=1e-14 * np.abs(A).max())


def test_exact_step_is_the_matrix_exponential():
    rng = np.random.default_rng(3)
    for V in VS:
        for Ca in CAS:
            for dt in (0.01, 0.1, 1.0, 20.0):
                u = rng.dirichlet(np.ones(4))
                ref = expm(dt * oracle.fca_generator(V, Ca)) @ u
                assert np.allclose(oracle.fca_exact_step(V, Ca, dt, u), ref, rtol=0, atol=1e-13)


def test_without_remainder_the_split_step_is_exact():
    # eps = 0: A = A_f (+) A_c, whose two terms commute, so the Lie split
    # exp(dt A_c) exp(dt A_f) is exp(dt A) itself
    par = list(oracle.FCA_DEFAULTS)
    par[6] = 0.0
    rng = np.random.default_rng(4)
    for V in VS:
        for Ca in CAS:
            for dt in (0.02, 0.5, 5.0):
                u = rng.dirichlet(np.ones(4))
                ref = expm(dt * oracle.fca_generator(V, Ca, par)) @ u
                got = oracle.fca_split_step(V, Ca, dt, u, par)
                assert np.allclose(got, ref, rtol=0, atol=2e-15), (V, Ca, dt)


def test_independent_gates_stay_a_product_of_scalar_rush_larsen_steps():
    # eps = 0 and u = (1-f, f) x (1-c, c): each gate by Eq. (RL) on its own
    par = list(oracle.FCA_DEFAULTS)
    par[6] = 0.0
    for V in VS:
        for Ca in CAS:
            af, bf, ac, bc, ci = _rates(V, Ca)
            f, c, dt = 0.3, 0.8, 0.05
            un = oracle.fca_split_step(V, Ca, dt, np.kron([1 - c, c], [1 - f, f]), par)
            fn = af / (af + bf) + (f - af / (af + bf)) * np.exp(-(af + bf) * dt)
            cn = ci + (c - ci) * np.exp(-dt / TAUC)
            assert np.allclose(un, np.kron([1 - cn, cn], [1 - fn, fn]), rtol=0, atol=1e-15)


def test_split_error_is_second_order_per_step():
    rng = np.random.default_rng(5)
    u = rng.dirichlet(np.ones(4))
    for V, Ca in [(-20.0, 2e-6), (0.0, 1e-5), (-60.0, 5e-7)]:
        errs = []
        for dt in (0.2, 0.1, 0.05, 0.025):
            errs.append(np.abs(oracle.fca_split_step(V, Ca, dt, u) - oracle.fca_exact_step(V, Ca, dt, u)).max())
        ratios = np.array(errs[:-1]) / np.array(errs[1:])
        assert np.all((ratios > 3.6) & (ratios < 4.4)), (V, Ca, ratios)
    # and the splitting error scales with the remainder
    def err(eps):
        par = list(oracle.FCA_DEFAULTS)
        par[6] = eps
        return np.abs(oracle.fca_split_step(-20.0, 2e-6, 0.1, u, par)
                      - oracle.fca_exact_step(-20.0, 2e-6, 0.1, u, par)).max()
    assert err(0.005) < 0.2 * err(0.05)


def test_split_step_keeps_probability():
    rng = np.random.default_rng(6)
    for V in VS:
        for Ca in CAS:
            for dt in (0.01, 0.1, 1.0):
                u = rng.dirichlet(np.ones(4))
                un = oracle.fca_split_step(V, Ca, dt, u)
                assert abs(un.sum() - 1.0) < 1e-15 * 8
                assert np.all(un >= 0.0)


def test_global_error_of_the_split_scheme_is_first_order():
    # a voltage-clamp protocol with Ca(t) given: the split scheme against the
    # exact exponential integrator over 20 ms
    def Vt(t):
        return -84.0 + 100.0 * (t > 2.0) * np.exp(-(t - 2.0) / 30.0)

    def Cat(t):
        return 1e-7 + 3e-6 * (t > 2.0) * (1 - np.exp(-(t - 2.0) / 5.0))

    def run(step, dt, T=20.0):
        u = np.array([0.0, 1.0, 0.0, 0.0])
        for n in range(int(round(T / dt))):
            u = step(Vt(n * dt), Cat(n * dt), dt, u)
        return u

    e = [np.abs(run(oracle.fca_split_step, dt) - run(oracle.fca_exact_step, dt)).max() for dt in (0.1, 0.05, 0.025)]
    r = np.array(e[:-1]) / np.array(e[1:])
    assert np.all((r > 1.7) & (r < 2.3)), r


def _cell(model, y, n, dt=0.01, par=None):
    V = np.empty(n)
    for i in range(n):
        y = oracle.cell_update(model, y, dt=dt, par=par)
        V[i] = y[0]
    return V, y


def test_with_the_calcium_gate_held_open_the_model_is_beeler_reuter():
    # Kc huge: c_inf = 1, the remainder vanishes, a channel started with c
    # open stays so, Q3 = f and I_s is the 1977 current
    par = list(oracle.FCA_DEFAULTS)
    par[4] = 1e300
    rb = oracle.rest_state(oracle.BR)
    y = np.zeros(11)
    y[:7] = rb[:7]
    f = rb[7]
    y[7:] = [0.0, 0.0, 1.0 - f, f]
    y[0] = -40.0
    yb = rb.copy()
    yb[0] = -40.0
    Vf, yf = _cell(oracle.BR_FCA, y, 30000, par=par)
    Vb, yb = _cell(oracle.BR, yb, 30000)
    assert np.max(np.abs(Vf - Vb)) < 1e-8 * 100
    assert abs(yf[10] - yb[7]) < 1e-10 and yf[7] == 0.0 and yf[8] == 0.0


def test_rest_state_and_calcium_dependent_inactivation():
    r = oracle.rest_state(oracle.BR_FCA)
    assert -86.0 < r[0] < -83.0
    assert abs(r[7:].sum() - 1.0) < 1e-10 and np.all(r[7:] >= 0)
    assert np.allclose(oracle.cell_update(oracle.BR_FCA, r, dt=0.01), r, rtol=0, atol=1e-9)
    # raising Ca closes the calcium gate: the steady open probability of
    # the channel (null vector of A) falls with Ca
    def p_open(Ca):
        w, v = np.linalg.eig(oracle.fca_generator(0.0, Ca))
        s = np.real(v[:, np.argmin(np.abs(w))])
        return (s / s.sum())[3]
    p = [p_open(Ca) for Ca in (1e-7, 1e-6, 1e-5, 1e-4)]
    assert all(a > b for a, b in zip(p, p[1:]))
    # the action potential: a plateau shorter than Beeler-Reuter's
    def apd(model):
        rs = oracle.rest_state(model)
        y = rs.copy(); y[0] = -40.0
        V, _ = _cell(model, y, 40000, dt=0.01)
        t = np.arange(1, V.size + 1) * 0.01
        tpk = t[np.argmax(V)]
        amp = V.max() - rs[0]
        assert 20.0 < V.max() < 60.0
        return t[np.nonzero((t > tpk) & (V < rs[0] + 0.1 * amp))[0][0]] - tpk
    a_br, a_fca = apd(oracle.BR), apd(oracle.BR_FCA)
    assert 100.0 < a_fca < 0.8 * a_br, (a_fca, a_br)


def test_rk4_is_refused_and_lie_splitting_runs():
    g = oracle.Grid(6, 5, 1, 0.25)
    s = oracle.Sim(g, oracle.BR_FCA, rk4=True)
    with pytest.raises(Exception):
        s.step(0.02, 1)
    s = oracle.Sim(g, oracle.BR_FCA, split=True)
    s.step(0.02, 3)
    assert np.all(np.isfinite(s.state))


def test_onfly_cell_update_takes_the_exponential_of_the_whole_generator():
    # parameter onfly = 1: the channel's step in the cell update is
    # exp(dt A(V_n, Ca_n)) u_n (scipy's expm); the other variables are those
    # of the split cell update
    par_s = list(oracle.FCA_DEFAULTS)
    par_x = list(oracle.FCA_DEFAULTS)
    par_x[7] = 1.0
    rng = np.random.default_rng(7)
    r = oracle.rest_state(oracle.BR_FCA)
    for V, Ca in [(-84.0, 1.6e-7), (-20.0, 2e-6), (10.0, 8e-6)]:
        y = r.copy()
        y[0], y[1] = V, Ca
        y[7:] = rng.dirichlet(np.ones(4))
        for dt in (0.02, 0.5):
            ys = oracle.cell_update(oracle.BR_FCA, y, dt=dt, par=par_s)
            yx = oracle.cell_update(oracle.BR_FCA, y, dt=dt, par=par_x)
            ref = expm(dt * oracle.fca_generator(V, Ca)) @ y[7:]
            assert np.allclose(yx[7:], ref, rtol=0, atol=1e-13)
            assert np.array_equal(yx[:7], ys[:7])
            assert 0.0 < np.abs(yx[7:] - ys[7:]).max() < 0.05 * dt * dt
