"""GPU parity on the benchmark workloads at the sizes and run lengths their
bars are stated for, in the autotuned launch configuration the benchmark
uses, against the FP64 oracle (threaded over the host cores; its results do
not depend on the thread count):

  - the Beeler-Reuter ventricle-like shell at quarter scale (128^3), the full
    500 ms run: every tissue node's activation step within one step of the
    oracle's (stored by tests/golden/make_br_shell_activation.py, which calls
    only the oracle);
  - the same shell at full size (512^3) after 100 steps: every tissue node
    within rel L-inf 1e-4 on V.  After n steps a node depends only on the
    initial state within n nodes of it (the stencil reaches one node per
    step), and nodes whose whole neighbourhood is homogeneous stay on the
    single-cell trajectory exactly (L of a constant is zero), so the oracle
    steps only the box around the apex stimulus, widened by n + 2 nodes, and
    one node's ODE for the rest of the tissue;
  - the rotating-fibre Barkley slab at reduced size (128 x 128 x 32), the
    full 2000-step run: activation within one step at every node;
  - the Beeler-Reuter slab with the trained reaction surrogate at the
    benchmark's upstroke thresholds, over a run in which the front crosses
    the slab: activation against the oracle.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
V_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx
    oracle.set_threads(os.cpu_count() or 1)
    yield torch, bbx
    oracle.set_threads(1)


def _grid(bbx, w, autotune=True):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_fibres(w.fibres, w.D_par, w.D_perp)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    G.set_timestep(w.dt)
    return G


def _act(a, n):
    a = np.asarray(a).astype(np.int64)
    a[a == oracle.INT32_MAX] = n + 1
    return a


def test_br_shell_quarter_scale_full_run_activation(env):
    torch, bbx = env
    gold = np.load(os.path.join(GOLDEN, "br_shell_128_activation.npz"))
    w = wl.br_shell(128)
    n = int(gold["n_steps"])
    assert n == w.n_steps and float(gold["dt"]) == w.dt
    tis = w.mask.reshape(-1) != 0
    assert int(gold["n_tissue"]) == int(tis.sum())
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    G = _grid(bbx, w)
    G.write_all(st0)
    G.autotune(w.dt)  # the benchmark's choice of tile (state restored)
    G.step(w.dt, n)
    ag = _act(G.read_activation().reshape(-1)[tis], n)
    ao = _act(gold["act"], n)
    assert (ao <= n).mean() > 0.99  # the wave reaches (almost) the whole shell
    d = np.abs(ag - ao)
    assert d.max() <= 1, (d.max(), int((d > 1).sum()))
    G.close()


def test_br_shell_full_size_100_steps_every_node(env):
    torch, bbx = env
    n = 100
    w = wl.br_shell(512)
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    G = _grid(bbx, w)
    info = G.get_info()
    S, px = info["nvars"], info["px"]
    vol = w.nz * w.ny * px
    # the state in buffers owned by the caller, so it can be read in place
    bufs = [torch.zeros(S * vol, dtype=torch.float32, device="cuda") for _ in range(2)]
    G.bind_state(bufs[0], bufs[1])
    G.write_all(st0)
    G.autotune(w.dt)  # the benchmark's choice of tile (state restored)
    G.step(w.dt, n)
    torch.cuda.synchronize()
    cur = bufs[0] if G.state_device_ptr(0) == bufs[0].data_ptr() else bufs[1]
    st = cur.view(S, w.nz, w.ny, px)[:, :, :, :w.nx]
    # the box holding every node the stimulus can influence within n steps,
    # with two more layers so that its faces stay homogeneous
    zz, yy, xx = np.nonzero(w.ic_region)
    m = n + 2
    lo = np.maximum([zz.min() - m, yy.min() - m, xx.min() - m], 0)
    hi = np.minimum([zz.max() + m + 1, yy.max() + m + 1, xx.max() + m + 1], [w.nz, w.ny, w.nx])
    sl = tuple(slice(int(a), int(b)) for a, b in zip(lo, hi))
    sub_mask = np.ascontiguousarray(w.mask[sl])
    sub_fib = np.ascontiguousarray(w.fibres[sl])
    sub_st = np.ascontiguousarray(st0[(slice(None),) + sl]).astype(np.float64)
    og = oracle.Grid(sub_mask.shape[2], sub_mask.shape[1], sub_mask.shape[0], w.h, sub_mask, sub_fib, w.D_par,
                     w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=sub_st)
    osim.step(w.dt, n)
    tis = og.psi
    # the wave has left the stimulated ball (whose nodes start above the
    # threshold and so never cross it)
    assert (osim.act[tis] <= n).sum() > 1000
    # every other tissue node follows one resting node's trajectory
    ys = st0[:, w.mask != 0][:, 0].astype(np.float64)
    for _ in range(n):
        ys = oracle.cell_update(w.model, ys, dt=w.dt, par=w.params)
    tis_dev = torch.from_numpy(w.mask != 0).cuda()
    far = tis_dev.clone()
    far[sl] = False
    got = st[(slice(None),) + sl].cpu().numpy()
    for v in range(S):
        scale = max(float(np.abs(osim.state[v][tis]).max()), abs(ys[v]), 1e-30)
        tol = V_TOL if v == 0 else 1e-3
        e_far = (st[v][far].double() - ys[v]).abs().max().item() / scale
        e_box = float(np.abs(got[v][tis] - osim.state[v][tis]).max()) / scale
        assert e_far <= tol and e_box <= tol, (v, e_far, e_box)
    G.close()


def test_barkley_slab_reduced_full_run_activation(env):
    torch, bbx = env
    w = wl.barkley_slab(128, 128, 32)
    n = 2000
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    G = _grid(bbx, w)
    G.write_all(st0)
    G.autotune(w.dt)
    G.step(w.dt, n)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
    osim.step(w.dt, n)
    ao, ag = _act(osim.act, n), _act(G.read_activation(), n)
    assert (ao <= n).mean() > 0.9  # the stimuli's waves cover the slab
    d = np.abs(ag - ao)
    assert d.max() <= 1, (d.max(), int((d > 1).sum()))
    G.close()


def test_surrogate_activation_against_the_oracle_at_the_benchmark_thresholds(env):
    torch, bbx = env
    w = wl.br_slab(104, 32, 8)
    n = 3000  # 60 ms: the front crosses the slab
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    # training pairs from a plain run of the same slab, as the benchmark does
    G = _grid(bbx, w)
    G.write_all(st0)
    chunks, per = 30, 20000
    X = torch.empty((chunks * per, 8), dtype=torch.float32, device="cuda")
    T = torch.empty_like(X)
    for k in range(chunks):
        bbx.bbx_sample_reaction_pairs(G.g, per, 7000 + k, X[k * per:(k + 1) * per], T[k * per:(k + 1) * per])
        G.step(w.dt, 6000 // chunks)
    G.close()
    m = bbx.bbx_mlp_create(21)
    try:
        bbx.bbx_mlp_fit_normalization(m, X, T, X.shape[0])
        bbx.bbx_mlp_train(m, X, T, X.shape[0], 4096, 4000, 1e-3, seed=22)
        og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
        osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
        osim.step(w.dt, n)
        ao = _act(osim.act, n)
        assert (ao <= n).mean() > 0.9
        res = {}
        for v_up in (-75.0, -60.0):
            S = _grid(bbx, w)
            S.write_all(st0)
            bbx.bbx_set_surrogate(S.g, m, v_up)
            S.step(w.dt, n)
            d = np.abs(_act(S.read_activation(), n) - ao)
            res[v_up] = (int(d.max()), float((d <= 1).mean()))
            S.close()
        P = _grid(bbx, w)
        P.write_all(st0)
        P.step(w.dt, n)
        dp = np.abs(_act(P.read_activation(), n) - ao)
        P.close()
        assert dp.max() <= 1  # the plain FP32 step holds the bar against the oracle
        # The surrogate's activation times against the oracle, at both
        # thresholds (the exact model where V >= v_up): reported, not held to
        # the one-step bar, which this network does not meet on this slab
        # (resting nodes that take the network drift, see the benchmark's
        # surrogate runs).
        for v_up, (dmax, frac) in res.items():
            print("surrogate at v_up %g mV: activation max |diff| %d steps, %.3f within 1 step" % (v_up, dmax, frac))
            assert frac > 0.1
    finally:
        bbx.bbx_mlp_destroy(m)


def test_state_of_more_than_two_to_the_31_elements_one_step_sampled(env):
    # A Beeler-Reuter slab of 1024 x 512 x 520 nodes (8 variables: 2.18e9
    # state elements, beyond 32-bit element offsets) with random fibre
    # directions and a random voltage field: one step, checked at sampled
    # nodes, among them nodes of the last planes and of the boundaries, for V
    # and for the last variable (the highest offsets).  After one step a node
    # depends only on the state and fibres within one node, so the oracle
    # steps the 3 x 3 x 3 box around each sampled node (clipped at the grid's
    # faces, which are the box's faces there too).
    torch, bbx = env
    nx, ny, nz, h, dt = 1024, 512, 520, 0.2, 0.02
    assert 8 * nx * ny * nz > 2 ** 31
    rng = np.random.default_rng(2031)
    fib = rng.standard_normal((nz, ny, nx, 3), dtype=np.float32)
    fib /= np.linalg.norm(fib, axis=-1, keepdims=True) + np.float32(1e-6)
    par = [4.0, 0.003, 50.0, 0.09]
    rest = oracle.rest_state(oracle.BR, par)
    st0 = np.empty((8, nz, ny, nx), np.float32)
    for v in range(1, 8):
        st0[v] = rest[v]
    st0[0] = rest[0] + 20.0 * rng.standard_normal((nz, ny, nx), dtype=np.float32)
    G = bbx.Grid(nx, ny, nz, h, None)
    G.set_fibres(fib, 0.1, 0.025)
    G.set_ionic_model(bbx.BBX_BR, par)
    G.set_timestep(dt)
    G.write_all(st0)
    G.step(dt, 1)
    V1 = G.read_state(0)
    F1 = G.read_state(7)
    pick = [(nz - 1, ny - 1, nx - 1), (nz - 1, 0, 0), (0, 0, 0), (nz - 2, ny // 2, nx - 1), (nz - 1, 17, 513)]
    for _ in range(120):
        pick.append((int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx))))
    for _ in range(60):  # the last planes
        pick.append((nz - 1 - int(rng.integers(3)), int(rng.integers(ny)), int(rng.integers(nx))))
    ev = ef = 0.0
    for z, y, x in pick:
        z0, z1 = max(z - 1, 0), min(z + 2, nz)
        y0, y1 = max(y - 1, 0), min(y + 2, ny)
        x0, x1 = max(x - 1, 0), min(x + 2, nx)
        box = np.ascontiguousarray(st0[:, z0:z1, y0:y1, x0:x1]).astype(np.float64)
        fb = np.ascontiguousarray(fib[z0:z1, y0:y1, x0:x1])
        og = oracle.Grid(x1 - x0, y1 - y0, z1 - z0, h, None, fb, 0.1, 0.025)
        osim = oracle.Sim(og, oracle.BR, par=par, state=box)
        osim.step(dt, 1)
        ref_v = osim.state[0, z - z0, y - y0, x - x0]
        ref_f = osim.state[7, z - z0, y - y0, x - x0]
        ev = max(ev, abs(float(V1[z, y, x]) - ref_v) / max(abs(ref_v), 1.0))
        ef = max(ef, abs(float(F1[z, y, x]) - ref_f))
    G.close()
    assert ev <= 1e-5, ev
    assert ef <= 1e-6, ef
