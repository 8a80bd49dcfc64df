"""FP64 CPU oracle for the BeatBox monodomain explicit step (arXiv:1605.06015).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library; the C source ``bbx_oracle.c`` follows the paper passage
by passage (each function names its equation).

Parity status per function (see ``bbx_oracle.c`` for the passages):
  tensor, weights, L, FHN, Barkley, ZFK, Euler, Rush-Larsen, activation,
  total, active bricks: pinned by the tests in ``tests/test_oracle_*.py``.
  output.py (byte quantisation, colour map, phase singularities): pinned by
  tests/test_oracle_output.py.
  Matrix Rush-Larsen (transition matrix of the Markov form of the BR sodium
  activation, the BR_MRL model): pinned by tests/test_oracle_markov.py.
  Multivariate matrix Rush-Larsen (the two-gate calcium-dependent
  inactivation channel of BR_FCA, split into its univariate subsystems):
  pinned by tests/test_oracle_markov_ca.py.
  Beeler-Reuter rates and currents: the paper does not print them
  (transcribed from Beeler & Reuter 1977); pinned by physics and physiology
  in tests/test_oracle_br.py (directions, windows, hierarchy, reversal
  potentials, the whole-cell action potential), which catch gross slips of
  one constant but not a small change: PARITY PARTIAL for the exact values
  of the constants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbx_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

FHN, BARKLEY, BR, ZFK, DIFFUSION, BR_MRL, BR_FCA = 1, 2, 3, 4, 5, 6, 7
NVARS = {FHN: 2, BARKLEY: 2, BR: 8, ZFK: 1, DIFFUSION: 1, BR_MRL: 11, BR_FCA: 11}
# default parameters of BR_FCA: gNa, gNaC, ENa, gs, Kc (mol/L), tau_c (ms), eps,
# onfly (1: the channel by the unsplit exponential instead of the split step)
FCA_DEFAULTS = (4.0, 0.003, 50.0, 0.09, 5e-6, 2.0, 0.05, 0.0)
MAXS = 11
INT32_MAX = np.iinfo(np.int32).max


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE double: no fast-math, no FMA
    contraction; OpenMP for the optional threaded node loops).  Returns the
    library path."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double),
                ("psi", ctypes.c_void_p), ("fib", ctypes.c_void_p),
                ("Dpar", ctypes.c_double), ("Dperp", ctypes.c_double)]


class RunCfg(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("par", ctypes.c_void_p), ("npar", ctypes.c_int),
                ("stim", ctypes.c_void_p), ("amp", ctypes.c_double), ("t_on", ctypes.c_double),
                ("t_off", ctypes.c_double), ("theta", ctypes.c_double), ("split", ctypes.c_int),
                ("rk4", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        L.orc_cell_weights.argtypes = [P, I, I, I, P]
        L.orc_apply_L.argtypes = [P, P, P]
        L.orc_diffusion_tensor.argtypes = [P, I, I, I, P]
        L.orc_diffusion_tensor.restype = I
        L.orc_check_fibres.argtypes = [P]
        L.orc_check_fibres.restype = I
        L.orc_rest_state.argtypes = [I, P, I, P]
        L.orc_rest_state.restype = I
        L.orc_cell_update.argtypes = [I, P, I, P, D, D, D, P]
        L.orc_cell_update_rk4.argtypes = [I, P, I, P, D, D, D, P]
        L.orc_cell_update_rk4.restype = I
        L.orc_br_rates.argtypes = [D, P, P]
        L.orc_br_currents.argtypes = [P, P, P]
        L.orc_mrl_generator.argtypes = [D, P]
        L.orc_mrl_transition.argtypes = [D, D, P]
        L.orc_fca_generator.argtypes = [P, I, D, D, P]
        L.orc_fca_split_step.argtypes = [P, I, D, D, D, P, P]
        L.orc_fca_exact_step.argtypes = [P, I, D, D, D, P, P]
        L.orc_run.argtypes = [P, P, P, D, I, P, P, P]
        L.orc_run.restype = I
        L.orc_set_threads.argtypes = [I]
        L.orc_set_threads.restype = I
        L.orc_step_cells.argtypes = [P, P, P, D, D, P, I, P]
        L.orc_step_cells.restype = I
        L.orc_total.argtypes = [P, P]
        L.orc_total.restype = D
        L.orc_active_bricks.argtypes = [P, I, I, I, P, ctypes.c_longlong]
        L.orc_active_bricks.restype = ctypes.c_longlong
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Threads for the whole-grid loops of Sim.step (1 = serial, the
    default).  Results are bit-identical for any count.  Returns the count in
    use."""
    return lib().orc_set_threads(int(n))


def _ptr(a):
    return None if a is None else a.ctypes.data


class Grid:
    """Geometry (shape, spacing, tissue indicator psi, fibres, D_par, D_perp)
    as the oracle sees it.  Arrays are kept alive by this object.  mask and
    fibres use the dense layout [nz][ny][nx] (fibres [nz][ny][nx][3])."""

    def __init__(self, nx, ny, nz, h, mask=None, fibres=None, D_par=1.0, D_perp=None):
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self.fibres = None if fibres is None else np.ascontiguousarray(fibres, dtype=np.float32).reshape(-1)
        if self.mask is not None:
            assert self.mask.size == self.N
        if self.fibres is not None:
            assert self.fibres.size == 3 * self.N
        self.g = Geom(nx, ny, nz, float(h), _ptr(self.mask), _ptr(self.fibres), float(D_par),
                      float(D_par if D_perp is None else D_perp))

    @property
    def psi(self):
        if self.mask is None:
            return np.ones(self.shape, dtype=bool)
        return self.mask.reshape(self.shape) != 0

    def weights(self, x, y, z):
        W = np.zeros(27)
        lib().orc_cell_weights(ctypes.byref(self.g), x, y, z, W.ctypes.data)
        return W.reshape(3, 3, 3)  # [qz+1][qy+1][qx+1]

    def tensor(self, x, y, z):
        D = np.zeros(9)
        rc = lib().orc_diffusion_tensor(ctypes.byref(self.g), x, y, z, D.ctypes.data)
        return rc, D.reshape(3, 3)

    def check_fibres(self):
        return lib().orc_check_fibres(ctypes.byref(self.g))

    def apply_L(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        assert u.size == self.N
        out = np.zeros(self.N)
        lib().orc_apply_L(ctypes.byref(self.g), u.ctypes.data, out.ctypes.data)
        return out.reshape(self.shape)

    def total(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        return lib().orc_total(ctypes.byref(self.g), u.ctypes.data)

    def active_bricks(self, tx, ty, tz):
        nb = (-(-self.shape[2] // tx)) * (-(-self.shape[1] // ty)) * (-(-self.shape[0] // tz))
        out = np.zeros(max(nb, 1), dtype=np.int32)
        cnt = lib().orc_active_bricks(ctypes.byref(self.g), tx, ty, tz, out.ctypes.data, nb)
        assert cnt >= 0
        return out[:cnt].copy()


def rest_state(model, par=None):
    par = np.zeros(0) if par is None else np.ascontiguousarray(par, dtype=np.float64)
    y = np.zeros(MAXS)
    rc = lib().orc_rest_state(model, _ptr(par) if par.size else None, par.size, y.ctypes.data)
    assert rc == 0
    return y[:NVARS[model]].copy()


def cell_update(model, y, L=0.0, Istim=0.0, dt=0.01, par=None):
    par = np.zeros(0) if par is None else np.ascontiguousarray(par, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    yn = np.zeros(MAXS)
    lib().orc_cell_update(model, _ptr(par) if par.size else None, par.size, y.ctypes.data,
                          float(L), float(Istim), float(dt), yn.ctypes.data)
    return yn[:NVARS[model]].copy()


def cell_update_rk4(model, y, L=0.0, Istim=0.0, dt=0.01, par=None):
    """One classical RK4 step of a single node (rhs models)."""
    par = np.zeros(0) if par is None else np.ascontiguousarray(par, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    yn = np.zeros(MAXS)
    rc = lib().orc_cell_update_rk4(model, _ptr(par) if par.size else None, par.size, y.ctypes.data,
                                   float(L), float(Istim), float(dt), yn.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle orc_cell_update_rk4 failed: %d" % rc)
    return yn[:NVARS[model]].copy()


def br_rates(V):
    a = np.zeros(6); b = np.zeros(6)
    lib().orc_br_rates(float(V), a.ctypes.data, b.ctypes.data)
    return a, b


def mrl_generator(V):
    """Transition-rate matrix A(V) of the Markov form of the BR sodium
    activation (4 x 4, A[i, j] = rate from state j into state i)."""
    A = np.zeros(16)
    lib().orc_mrl_generator(float(V), A.ctypes.data)
    return A.reshape(4, 4)


def mrl_transition(V, dt):
    """T = exp(dt A(V)), the matrix Rush-Larsen step of the chain."""
    T = np.zeros(16)
    lib().orc_mrl_transition(float(V), float(dt), T.ctypes.data)
    return T.reshape(4, 4)


def _fca_par(par):
    p = np.array(FCA_DEFAULTS if par is None else par, dtype=np.float64)
    return p, len(p)


def fca_generator(V, Ca, par=None):
    """Generator A(V, Ca) of the two-gate slow-inward inactivation channel
    of BR_FCA (4 x 4, state q = f + 2 c, A[i, j] = rate from j into i)."""
    p, n = _fca_par(par)
    A = np.zeros(16)
    lib().orc_fca_generator(p.ctypes.data, n, float(V), float(Ca), A.ctypes.data)
    return A.reshape(4, 4)


def fca_split_step(V, Ca, dt, u, par=None):
    """The multivariate matrix Rush-Larsen step of the channel: the exact
    step of the voltage gate, then of the calcium gate, then Euler for the
    remainder."""
    p, n = _fca_par(par)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_fca_split_step(p.ctypes.data, n, float(V), float(Ca), float(dt), u.ctypes.data, out.ctypes.data)
    return out


def fca_exact_step(V, Ca, dt, u, par=None):
    """exp(dt A(V, Ca)) u, the unsplit matrix Rush-Larsen step."""
    p, n = _fca_par(par)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_fca_exact_step(p.ctypes.data, n, float(V), float(Ca), float(dt), u.ctypes.data, out.ctypes.data)
    return out


def br_currents(y, par=None):
    p = np.array([4.0, 0.003, 50.0, 0.09] if par is None else par, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_br_currents(p.ctypes.data, y.ctypes.data, out.ctypes.data)
    return out


class Sim:
    """Whole-grid stepping on the oracle: state is float64 [nvars][nz][ny][nx]."""

    def __init__(self, grid: Grid, model, par=None, theta=None, state=None, split=False, rk4=False):
        """split: Lie operator splitting (a diffusion substep, then the
        kinetics step) instead of the unsplit step.  rk4: the kinetics step by
        the classical fourth-order Runge-Kutta scheme instead of forward Euler
        (models given by a right-hand side)."""
        self.grid = grid
        self.split = bool(split)
        self.rk4 = bool(rk4)
        self.model = model
        self.S = NVARS[model]
        self.par = np.zeros(0) if par is None else np.ascontiguousarray(par, dtype=np.float64)
        if theta is None:
            theta = {FHN: 0.0, BARKLEY: 0.5, BR: -40.0, ZFK: 0.5, DIFFUSION: 0.5, BR_MRL: -40.0,
                     BR_FCA: -40.0}[model]
        self.theta = float(theta)
        if state is None:
            rs = rest_state(model, self.par if self.par.size else None)
            state = np.empty((self.S,) + grid.shape)
            for v in range(self.S):
                state[v] = rs[v]
        self.state = np.ascontiguousarray(state, dtype=np.float64).reshape((self.S,) + grid.shape).copy()
        self.act = np.full(grid.shape, INT32_MAX, dtype=np.int32)
        self.t = ctypes.c_double(0.0)
        self.n = ctypes.c_longlong(0)
        self.stim = None
        self.amp = 0.0
        self.t_on = 0.0
        self.t_off = 0.0

    def set_stimulus(self, region, amp, t_on, t_off):
        self.stim = np.ascontiguousarray(region, dtype=np.uint8).reshape(-1)
        self.amp, self.t_on, self.t_off = float(amp), float(t_on), float(t_off)

    def _cfg(self):
        return RunCfg(self.model, _ptr(self.par) if self.par.size else None, self.par.size,
                      _ptr(self.stim), self.amp, self.t_on, self.t_off, self.theta, int(self.split),
                      int(self.rk4))

    def step(self, dt, n_steps=1):
        cfg = self._cfg()
        rc = lib().orc_run(ctypes.byref(self.grid.g), ctypes.byref(cfg), self.state.ctypes.data,
                           float(dt), int(n_steps), ctypes.byref(self.t), ctypes.byref(self.n),
                           self.act.ctypes.data)
        if rc != 0:
            raise RuntimeError(f"oracle orc_run failed: {rc}")

    def step_cells(self, dt, cells):
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((cells.size, self.S))
        cfg = self._cfg()
        rc = lib().orc_step_cells(ctypes.byref(self.grid.g), ctypes.byref(cfg), self.state.ctypes.data,
                                  float(dt), self.t.value, cells.ctypes.data, cells.size, out.ctypes.data)
        if rc != 0:
            raise RuntimeError(f"oracle orc_step_cells failed: {rc}")
        return out
