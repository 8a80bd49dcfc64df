"""Pins of the FP64 surrogate reference (oracle/mlp.py): gradients against
central finite differences, the first Adam step's closed form, and training
of the output layer against the least-squares solution."""
import numpy as np

from oracle import mlp


def _data(seed, B=37):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, 8)), rng.normal(size=(B, 8))


def test_gradients_match_central_finite_differences():
    p = mlp.init_params(1)
    x, t = _data(2)
    g = mlp.grads(p, x, t)
    rng = np.random.default_rng(3)
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            h = 1e-6
            flat[idx] = old + h; lp = mlp.loss(p, x, t)
            flat[idx] = old - h; lm = mlp.loss(p, x, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (k, idx, fd, an)


def test_zero_weights_output_is_the_last_bias_and_pack_roundtrip():
    p = mlp.init_params(4)
    for k in p:
        p[k][...] = 0.0
    p["b3"][:] = np.arange(8.0)
    y, _ = mlp.forward(p, np.ones((3, 8)))
    assert np.array_equal(y, np.tile(np.arange(8.0), (3, 1)))
    q = mlp.init_params(5)
    vec = mlp.pack(q)
    assert vec.size == 8 * 64 + 64 + 64 * 64 + 64 + 64 * 8 + 8
    r = mlp.unpack(vec)
    assert all(np.array_equal(q[k], r[k]) for k in q)


def test_first_adam_step_moves_each_parameter_by_lr_times_sign():
    p = mlp.init_params(6)
    x, t = _data(7)
    g = mlp.grads(p, x, t)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    before = {k: a.copy() for k, a in p.items()}
    mlp.adam_step(p, g, m, v, step=1, lr=1e-3, eps=1e-12)
    for k in p:
        nz = np.abs(g[k]) > 1e-9
        assert np.allclose((p[k] - before[k])[nz], -1e-3 * np.sign(g[k][nz]), rtol=1e-6)


def test_training_the_output_layer_reaches_least_squares():
    p = mlp.init_params(8)
    x, _ = _data(9, B=200)
    _, (_, _, h2) = mlp.forward(p, x)
    rng = np.random.default_rng(10)
    t = rng.normal(size=(200, 8))
    A = np.hstack([h2, np.ones((200, 1))])
    sol, *_ = np.linalg.lstsq(A, t, rcond=None)
    best = np.mean((A @ sol - t) ** 2)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    for s in range(1, 3001):
        g = mlp.grads(p, x, t)
        for k in ("W1", "b1", "W2", "b2"):
            g[k][...] = 0.0  # only the output layer trains: a linear least-squares problem
        mlp.adam_step(p, g, m, v, step=s, lr=3e-2)
    assert mlp.loss(p, x, t) <= best * (1 + 1e-3)
