"""Pins of the matrix Rush-Larsen scheme in the oracle (section "Exponential
solvers": du/dt = A(V) u, u_{n+1} = exp(dt A(V_n)) u_n) on the Markov form of
the Beeler-Reuter sodium activation: a chain over the number k = 0..3 of open
activation subunits, k -> k+1 at (3-k) alpha_m and k -> k-1 at k beta_m.

Three independent two-state subunits evolve exactly like this chain, so for
V held fixed the chain's transition matrix has a closed form in the scalar
Rush-Larsen coefficients of one subunit (Eq. RL, RLcoeff): a subunit open at
the start is open after dt with probability a + b, a closed one with
probability b.  That closed form, the generator's definition, probability
conservation, the semigroup law and the equivalence with the scalar scheme
for m^3 pin the oracle's matrix exponential without reference to itself."""
from math import comb

import numpy as np
import pytest

import oracle

VS = [-90.0, -84.0, -60.0, -47.0, -40.0, -20.0, 0.0, 30.0]
DTS = [0.005, 0.02, 0.1, 0.5]


def _subunit_rl(V, dt):
    al, be = oracle.br_rates(V)
    a, b = al[1], be[1]
    A = np.exp(-(a + b) * dt)
    B = a / (a + b) * (1.0 - A)
    return A, B


def _closed_form(V, dt):
    """T[j, i] = P(j open after dt | i open before) for independent subunits."""
    A, B = _subunit_rl(V, dt)
    q11, q01 = A + B, B  # open -> open, closed -> open
    T = np.zeros((4, 4))
    for i in range(4):
        for j in range(4):
            s = 0.0
            for a in range(0, min(i, j) + 1):  # a of the i open subunits stay open
                c = j - a  # opened from the 3 - i closed ones
                if c > 3 - i:
                    continue
                s += (comb(i, a) * q11 ** a * (1 - q11) ** (i - a)
                      * comb(3 - i, c) * q01 ** c * (1 - q01) ** (3 - i - c))
            T[j, i] = s
    return T


def test_generator_is_the_birth_death_chain_of_three_subunits():
    for V in VS:
        al, be = oracle.br_rates(V)
        a, b = al[1], be[1]
        A = oracle.mrl_generator(V)
        ref = np.array([[-3 * a, b, 0, 0],
                        [3 * a, -(2 * a + b), 2 * b, 0],
                        [0, 2 * a, -(a + 2 * b), 3 * b],
                        [0, 0, a, -3 * b]])
        assert np.allclose(A, ref, rtol=1e-15, atol=0)
        assert np.allclose(A.sum(axis=0), 0.0, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("dt", DTS)
def test_transition_matrix_equals_the_independent_subunit_closed_form(dt):
    for V in VS:
        T = oracle.mrl_transition(V, dt)
        ref = _closed_form(V, dt)
        # rounding grows with the squarings (up to 2^9 at V = -90 mV, dt = 0.5 ms)
        assert np.abs(T - ref).max() < 2e-13, (V, dt, np.abs(T - ref).max())


def test_probability_is_conserved_and_entries_are_probabilities():
    for V in VS:
        for dt in DTS:
            T = oracle.mrl_transition(V, dt)
            assert np.allclose(T.sum(axis=0), 1.0, atol=1e-14)
            assert T.min() >= -1e-15 and T.max() <= 1.0 + 1e-15


def test_semigroup_and_small_step_limit():
    for V in VS:
        T1 = oracle.mrl_transition(V, 0.05)
        T2 = oracle.mrl_transition(V, 0.1)
        assert np.abs(T1 @ T1 - T2).max() < 1e-14
        A = oracle.mrl_generator(V)
        errs = []
        for dt in (1e-3, 5e-4):
            errs.append(np.abs((oracle.mrl_transition(V, dt) - np.eye(4)) / dt - A).max())
        # first-order remainder dt/2 A^2: halving dt halves the error
        assert errs[1] < 0.55 * errs[0] + 1e-12, (V, errs)


def test_binomial_states_stay_binomial_of_the_scalar_rush_larsen_gate():
    # a binomial distribution of one subunit probability m maps to the
    # binomial distribution of the scalar scheme's a m + b
    for V in VS:
        for dt in DTS:
            A, B = _subunit_rl(V, dt)
            for m in (0.0, 1e-3, 0.2, 0.7, 1.0):
                u = np.array([comb(3, k) * m ** k * (1 - m) ** (3 - k) for k in range(4)])
                m1 = A * m + B
                ref = np.array([comb(3, k) * m1 ** k * (1 - m1) ** (3 - k) for k in range(4)])
                assert np.abs(oracle.mrl_transition(V, dt) @ u - ref).max() < 2e-13


def test_markov_model_run_reproduces_the_scalar_beeler_reuter_run():
    # the whole-grid step: BR with m^3 from the chain equals BR with the
    # scalar m gate, node by node, through an upstroke
    nz, ny, nx = 3, 6, 20
    g = oracle.Grid(nx, ny, nz, 0.2, None, None, 0.1, 0.1)
    rs = oracle.rest_state(oracle.BR)
    st = np.empty((8, nz, ny, nx))
    for v in range(8):
        st[v] = rs[v]
    st[0][:, :, :4] = 10.0  # depolarised edge starts a wave
    m = st[3]
    stm = np.empty((11, nz, ny, nx))
    for dst, src in zip(range(7), (0, 1, 2, 4, 5, 6, 7)):
        stm[dst] = st[src]
    for k in range(4):
        stm[7 + k] = comb(3, k) * m ** k * (1 - m) ** (3 - k)
    a = oracle.Sim(g, oracle.BR, state=st)
    b = oracle.Sim(g, oracle.BR_MRL, state=stm)
    a.step(0.02, 150)
    b.step(0.02, 150)
    assert a.state[0].max() > 0.0  # the upstroke happened
    assert np.abs(b.state[0] - a.state[0]).max() < 1e-9
    for dst, src in zip(range(1, 7), (1, 2, 4, 5, 6, 7)):
        assert np.abs(b.state[dst] - a.state[src]).max() < 1e-11
    assert np.abs(b.state[10] - a.state[3] ** 3).max() < 1e-12
    assert np.abs(b.state[7:].sum(axis=0) - 1.0).max() < 1e-12  # 150 steps of rounding
    assert np.array_equal(a.act, b.act)


def test_markov_rest_state_is_the_binomial_of_the_br_rest_gate():
    r = oracle.rest_state(oracle.BR)
    rm = oracle.rest_state(oracle.BR_MRL)
    m = r[3]
    assert np.allclose(rm[:7], r[[0, 1, 2, 4, 5, 6, 7]], rtol=0, atol=0)
    assert np.allclose(rm[7:], [(1 - m) ** 3, 3 * m * (1 - m) ** 2, 3 * m * m * (1 - m), m ** 3], rtol=1e-15, atol=0)
