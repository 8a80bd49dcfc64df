"""The oracle's threaded node loops (used to time the oracle on all host
cores and for long parity runs) give bit-identical results to the serial
loops: each node's update is computed by the same arithmetic whatever
thread runs it."""
import numpy as np

import oracle
from paper_1605_06015_gb300 import workloads as wl


def _run(threads, model, mask, fib, st, n, stim=None):
    nz, ny, nx = mask.shape
    oracle.set_threads(threads)
    try:
        g = oracle.Grid(nx, ny, nz, 0.2, mask, fib, 0.1, 0.025)
        sim = oracle.Sim(g, model, state=st)
        if stim is not None:
            sim.set_stimulus(stim, amp=40.0, t_on=0.0, t_off=0.5)
        sim.step(0.02, n)
        return sim.state.copy(), sim.act.copy(), sim.t.value, sim.n.value
    finally:
        oracle.set_threads(1)


def test_threaded_oracle_is_bitwise_serial():
    mask, fib = wl.random_geometry(23, 17, 9, seed=11, tissue_frac=0.85)
    rest = oracle.rest_state(oracle.BR)
    st = np.empty((8,) + mask.shape)
    for v in range(8):
        st[v] = rest[v]
    st[0, :, :, :4] = 20.0  # a depolarised face launches a wave
    stim = np.zeros(mask.shape, np.uint8); stim[:, :3, -3:] = 1
    a = _run(1, oracle.BR, mask, fib, st, 40, stim)
    for th in (2, 5, 8):
        b = _run(th, oracle.BR, mask, fib, st, 40, stim)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert a[2] == b[2] and a[3] == b[3]
    assert oracle.set_threads(1) == 1
