"""The reaction surrogate inside the step kernel (Beeler-Reuter): tensor-core
inference against an FP64 forward pass with the same BF16 roundings, exact
fallback outside the envelope or above the upstroke threshold, and the
trained network's activation-time map against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx
    return torch, bbx


def _bf16(a):
    """Round float64 values to bfloat16 (round to nearest, ties to even)."""
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _random_states(shape, seed):
    """Physiological Beeler-Reuter states, independent per node."""
    rng = np.random.default_rng(seed)
    st = np.empty((8,) + shape)
    st[0] = rng.uniform(-88, 30, shape)
    st[1] = 10 ** rng.uniform(-7, -5.5, shape)
    for v in range(2, 8):
        st[v] = rng.uniform(0.0, 1.0, shape)
    return st


def _norm_for(st):
    x = st.reshape(8, -1).T
    n = np.zeros(48)
    n[0:8] = x.mean(0)
    n[8:16] = x.std(0)
    n[16:24] = np.array([1e-2, 1e-9, 1e-4, 1e-3, 1e-3, 1e-3, 1e-5, 1e-4]) * 0.1
    n[24:32] = np.array([1e-2, 1e-9, 1e-4, 1e-3, 1e-3, 1e-3, 1e-5, 1e-4])
    n[32:40] = x.min(0) - 1.0
    n[40:48] = x.max(0) + 1.0
    return n.astype(np.float32)


def _grid(bbx, w, st, tile=(14, 4)):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_fibres(w.fibres, w.D_par, w.D_perp)
    G.set_tiling(*tile)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    G.set_timestep(w.dt)
    G.write_all(st.astype(np.float32))
    return G


def test_fused_inference_matches_bf16_forward_pass(env):
    torch, bbx = env
    w = wl.br_slab(70, 20, 5)
    st = _random_states(w.shape, 5).astype(np.float32).astype(np.float64)
    norm = _norm_for(st)
    p = mlp.init_params(17)
    vec = mlp.pack(p).astype(np.float32)
    m = bbx.bbx_mlp_create(1)
    G = _grid(bbx, w, st)
    try:
        bbx.bbx_mlp_set_params(m, vec)
        bbx.bbx_mlp_set_normalization(m, norm)
        bbx.bbx_set_surrogate(G.g, m, 1e9)  # the network everywhere inside the envelope
        G.step(w.dt, 1)
        got = G.read_all().reshape(8, -1).T.astype(np.float64)
    finally:
        bbx.bbx_mlp_destroy(m)
    # FP64 reference with the kernel's roundings: BF16 weights, inputs and
    # hidden activations; biases and accumulation in (at least) float
    q = mlp.unpack(vec.astype(np.float64))
    x = st.reshape(8, -1).T
    xb = _bf16((x - norm[0:8]) / norm[8:16])
    h1 = _bf16(np.maximum(xb @ _bf16(q["W1"]).T + q["b1"], 0.0))
    h2 = _bf16(np.maximum(h1 @ _bf16(q["W2"]).T + q["b2"], 0.0))
    y = h2 @ _bf16(q["W3"]).T + q["b3"]
    d = y * norm[24:32] + norm[16:24]
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    L = og.apply_L(st[0]).reshape(-1)
    ref = x + d
    ref[:, 0] += w.dt * L
    # a hidden unit may round to the neighbouring BF16 value when float and
    # double accumulation straddle a rounding boundary: allow a few BF16 ulps
    # of the output scale
    tol = 3e-2 * norm[24:32] + 1e-3 * np.abs(d) + 1e-6 * np.abs(x)
    bad = np.abs(got - ref) > tol
    assert bad.mean() < 1e-3, (bad.sum(), np.abs(got - ref).max(0))


def test_fallback_is_the_exact_model_bitwise(env):
    torch, bbx = env
    w = wl.br_slab(72, 20, 6)
    rest = oracle.rest_state(oracle.BR)
    st = w.initial_state(rest)
    m = bbx.bbx_mlp_create(3)
    try:
        bbx.bbx_mlp_set_normalization(m, _norm_for(_random_states(w.shape, 6)))
        A = _grid(bbx, w, st)
        B = _grid(bbx, w, st)
        bbx.bbx_set_surrogate(B.g, m, -1e9)  # upstroke threshold below every V: never the network
        A.step(w.dt, 60)
        B.step(w.dt, 60)
        assert np.array_equal(A.read_all(), B.read_all())
        assert np.array_equal(A.read_activation(), B.read_activation())
        # an envelope that excludes every state: the exact model again
        nrm = _norm_for(_random_states(w.shape, 6))
        nrm[32:40] = 1e9
        nrm[40:48] = 2e9
        bbx.bbx_mlp_set_normalization(m, nrm)
        C = _grid(bbx, w, st)
        bbx.bbx_set_surrogate(C.g, m, 1e9)
        C.step(w.dt, 60)
        assert np.array_equal(A.read_all(), C.read_all())
        bbx.bbx_set_surrogate(C.g, None)
    finally:
        bbx.bbx_mlp_destroy(m)


def _train_on_trajectories(torch, bbx, w, st0, n_per, every, steps, seed):
    """Sample (state, reaction increment) pairs along a plain run and train."""
    G = _grid(bbx, w, st0)
    chunks = []
    for k in range(steps // every):
        x = torch.empty((n_per, 8), dtype=torch.float32, device="cuda")
        t = torch.empty((n_per, 8), dtype=torch.float32, device="cuda")
        bbx.bbx_sample_reaction_pairs(G.g, n_per, seed + k, x, t)
        chunks.append((x, t))
        G.step(w.dt, every)
    X = torch.cat([c[0] for c in chunks])
    T = torch.cat([c[1] for c in chunks])
    m = bbx.bbx_mlp_create(seed)
    bbx.bbx_mlp_fit_normalization(m, X, T, X.shape[0])
    l0 = bbx.bbx_mlp_train(m, X, T, X.shape[0], 2048, 1, 1e-3, seed=seed + 1)
    l1 = bbx.bbx_mlp_train(m, X, T, X.shape[0], 2048, 4000, 1e-3, seed=seed + 2)
    return m, l0, l1


def test_trained_surrogate_keeps_activation_times_within_one_step(env):
    torch, bbx = env
    w = wl.br_slab(128, 24, 6)
    rest = oracle.rest_state(oracle.BR)
    st0 = w.initial_state(rest)
    n = 1500  # 30 ms: the front crosses the slab
    m, l0, l1 = _train_on_trajectories(torch, bbx, w, st0, 2000, 10, 3000, 1234)
    try:
        assert l1 < 0.05 * l0, (l0, l1)
        S = _grid(bbx, w, st0)
        bbx.bbx_set_surrogate(S.g, m, -60.0)
        S.step(w.dt, n)
        P = _grid(bbx, w, st0)
        P.step(w.dt, n)
        og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
        osim = oracle.Sim(og, oracle.BR, theta=w.theta, state=st0.astype(np.float32).astype(np.float64))
        osim.step(w.dt, n)

        def act(a):
            a = a.astype(np.int64)
            a[a == oracle.INT32_MAX] = n + 1
            return a
        ao, ap, asu = act(osim.act), act(P.read_activation()), act(S.read_activation())
        assert (ao <= n).mean() > 0.3  # the front crossed a good part of the slab
        assert np.abs(ap - ao).max() <= 1
        assert np.abs(asu - ao).max() <= 1, np.abs(asu - ao).max()
        # and an untrained network of the same shape does not hold that bar
        u = bbx.bbx_mlp_create(99)
        try:
            bbx.bbx_mlp_set_normalization(u, bbx.bbx_mlp_get_normalization(m))
            U = _grid(bbx, w, st0)
            bbx.bbx_set_surrogate(U.g, u, -60.0)
            U.step(w.dt, n)
            try:
                au = act(U.read_activation())
                assert np.abs(au - ao).max() > 1
            except bbx.BbxError:
                pass  # diverged: non-finite V
        finally:
            bbx.bbx_mlp_destroy(u)
    finally:
        bbx.bbx_mlp_destroy(m)
