"""Pins of the oracle's diffusion operator (section "Monodomain diffusion and
boundary conditions", Eq. (Lu), Eq. (sigma) and the weight definitions) against
facts that do not come from the oracle itself: exact discrete identities,
textbook special cases, an independent NumPy assembly, symmetry of the
problem, and consistency with the continuous operator."""
import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from paper_1605_06015_gb300 import workloads as wl


def _rand_u(shape, seed):
    return np.random.default_rng(seed).normal(size=shape)


def _oblique(shape, f=(0.6, -0.3, 0.74)):
    fib = np.zeros(shape + (3,), dtype=np.float32)
    fib[...] = np.array(f, dtype=np.float32)
    return fib


def test_constants_are_in_the_kernel_exactly():
    # Difference form of W0 = -sum W_q: L(const) = 0 exactly, any geometry.
    mask, fib = wl.random_geometry(7, 6, 5, seed=3)
    g = oracle.Grid(7, 6, 5, 0.3, mask, fib, 1.0, 0.25)
    Lu = g.apply_L(np.full(g.shape, -84.57))
    assert np.all(Lu == 0.0)


def test_centre_weight_is_minus_sum():
    mask, fib = wl.random_geometry(5, 5, 5, seed=4)
    g = oracle.Grid(5, 5, 5, 0.2, mask, fib, 0.1, 0.025)
    for (z, y, x) in zip(*np.nonzero(mask)):
        W = g.weights(int(x), int(y), int(z))
        assert abs(W[1, 1, 1] + (W.sum() - W[1, 1, 1])) < 1e-12 * np.abs(W).sum()
        assert W[0, 0, 0] == 0 and W[2, 2, 2] == 0 and W[0, 2, 0] == 0  # corners


def test_isotropic_2d_is_textbook_5_point_laplacian():
    # Full rectangle, isotropic: no-flux by mirroring u_p into outside nodes is
    # the 'nearest' boundary mode of the textbook 5-point Laplacian.
    nx, ny, h = 13, 9, 0.5
    g = oracle.Grid(nx, ny, 1, h, D_par=1.0)
    u = _rand_u((1, ny, nx), 1)
    ref = ndi.laplace(u[0], mode="nearest") / h ** 2
    assert np.allclose(g.apply_L(u)[0], ref, rtol=0, atol=1e-12)


def test_isotropic_3d_is_textbook_7_point_laplacian():
    nx, ny, nz, h, D = 7, 6, 5, 0.3, 1.7
    g = oracle.Grid(nx, ny, nz, h, D_par=D)
    u = _rand_u((nz, ny, nx), 2)
    ref = D * ndi.laplace(u, mode="nearest") / h ** 2
    assert np.allclose(g.apply_L(u), ref, rtol=0, atol=1e-11)


def test_conservation_uniform_D_masked():
    # W^p_q = psi_{p+q} c_q with c_q = c_{-q} for uniform D, so the tissue sum
    # of L u vanishes for every u (no-flux boundaries conserve total V).
    mask, _ = wl.random_geometry(9, 8, 7, seed=5, tissue_frac=0.6)
    fib = _oblique((7, 8, 9))
    g = oracle.Grid(9, 8, 7, 0.25, mask, fib, 1.0, 0.25)
    u = _rand_u((7, 8, 9), 6)
    Lu = g.apply_L(u)
    assert abs((Lu * (mask != 0)).sum()) < 1e-12 * np.abs(Lu).sum()


def test_second_moment_grows_by_exactly_2Dk():
    # For uniform D: sum_q W_q q = 0 and sum_q W_q q_j q_k h^2 = 2 D_jk, so one
    # forward Euler diffusion step keeps the mean and adds 2 D k (times mass)
    # to the second-moment tensor.  Gaussian far from the boundary.
    n, h, k = 24, 0.5, 0.01
    fib = _oblique((n, n, n))
    f = fib[0, 0, 0].astype(np.float64); f /= np.linalg.norm(f)
    Dpar, Dperp = 1.0, 0.25
    D = Dperp * np.eye(3) + (Dpar - Dperp) * np.outer(f, f)
    g = oracle.Grid(n, n, n, h, None, fib, Dpar, Dperp)
    z, y, x = np.meshgrid(*(np.arange(n) * h,) * 3, indexing="ij")
    c = (n - 1) * h / 2
    u = np.exp(-((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) / 1.0)  # tails ~1e-16 at the boundary
    u1 = u + k * g.apply_L(u)
    X = [x - c, y - c, z - c]
    m0, m1 = u.sum(), u1.sum()
    assert abs(m1 - m0) < 1e-12 * m0
    for j in range(3):
        assert abs((u1 * X[j]).sum() - (u * X[j]).sum()) < 1e-10 * m0
        for kk in range(3):
            grow = ((u1 - u) * X[j] * X[kk]).sum() / m0
            assert abs(grow - 2 * D[j, kk] * k) < 1e-9 * k, (j, kk, grow, 2 * D[j, kk] * k)


def test_transpose_and_mirror_invariance_nonuniform_fibres():
    nx, ny, nz = 8, 8, 5
    mask, fib = wl.random_geometry(nx, ny, nz, seed=7, tissue_frac=0.75)
    u = _rand_u((nz, ny, nx), 8)
    g = oracle.Grid(nx, ny, nz, 0.3, mask, fib, 1.0, 0.3)
    Lu = g.apply_L(u)
    # x <-> y transpose with (f_x, f_y) swapped
    mt = np.ascontiguousarray(mask.transpose(0, 2, 1))
    ft = np.ascontiguousarray(fib.transpose(0, 2, 1, 3)[..., [1, 0, 2]])
    gt = oracle.Grid(ny, nx, nz, 0.3, mt, ft, 1.0, 0.3)
    Lt = gt.apply_L(np.ascontiguousarray(u.transpose(0, 2, 1)))
    assert np.allclose(Lt, Lu.transpose(0, 2, 1), rtol=0, atol=1e-11)
    # mirror x -> -x with f_x -> -f_x
    mm = np.ascontiguousarray(mask[:, :, ::-1])
    fm = np.ascontiguousarray(fib[:, :, ::-1, :] * np.array([-1, 1, 1], dtype=np.float32))
    gm = oracle.Grid(nx, ny, nz, 0.3, mm, fm, 1.0, 0.3)
    Lm = gm.apply_L(np.ascontiguousarray(u[:, :, ::-1]))
    assert np.allclose(Lm, Lu[:, :, ::-1], rtol=0, atol=1e-11)


def test_fibre_sign_is_irrelevant_bitwise():
    mask, fib = wl.random_geometry(6, 7, 4, seed=9)
    u = _rand_u((4, 7, 6), 10)
    a = oracle.Grid(6, 7, 4, 0.3, mask, fib, 1.0, 0.3).apply_L(u)
    b = oracle.Grid(6, 7, 4, 0.3, mask, -fib, 1.0, 0.3).apply_L(u)
    assert np.array_equal(a, b)


def _numpy_weights(mask, fib, h, Dpar, Dperp):
    """Independent assembly of W^p_q straight from the paper's case analysis,
    as a dense operator matrix.  Out-of-array and void neighbours have psi=0;
    D at a void p +- q_j is replaced by D^p."""
    nz, ny, nx = mask.shape
    N = mask.size
    f = fib.astype(np.float64)
    f = f / np.linalg.norm(f, axis=-1, keepdims=True)
    Dall = Dperp * np.eye(3)[None, None, None] + (Dpar - Dperp) * f[..., :, None] * f[..., None, :]

    def psi(z, y, x):
        return 1.0 if (0 <= x < nx and 0 <= y < ny and 0 <= z < nz and mask[z, y, x]) else 0.0

    A = np.zeros((N, N))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not mask[z, y, x]:
                    continue
                p = np.array([x, y, z])
                Dp = Dall[z, y, x]
                S = np.zeros(3)
                for j in range(3):
                    for s in (+1, -1):
                        c = p.copy(); c[j] += s
                        Dn = Dall[c[2], c[1], c[0]] if psi(c[2], c[1], c[0]) else Dp
                        S += s * Dn[j]
                i = x + nx * (y + ny * z)
                for qz in (-1, 0, 1):
                    for qy in (-1, 0, 1):
                        for qx in (-1, 0, 1):
                            q = np.array([qx, qy, qz])
                            nnz = np.count_nonzero(q)
                            if nnz == 0 or nnz == 3:
                                continue
                            t = p + q
                            ps = psi(t[2], t[1], t[0])
                            if nnz == 1:
                                kk = int(np.nonzero(q)[0][0])
                                m = p - q
                                w = ps * Dp[kk, kk] / h ** 2 + q[kk] * ps * psi(m[2], m[1], m[0]) * S[kk] / (4 * h ** 2)
                            else:
                                j, kk = np.nonzero(q)[0]
                                w = (1 if q[j] == q[kk] else -1) * ps * Dp[j, kk] / (2 * h ** 2)
                            if w != 0:
                                jn = t[0] + nx * (t[1] + ny * t[2])
                                A[i, jn] += w
                                A[i, i] -= w
    return A


@pytest.mark.parametrize("shape,seed", [((4, 5, 6), 11), ((5, 5, 5), 12), ((1, 6, 6), 13), ((3, 4, 2), 14)])
def test_independent_numpy_assembly(shape, seed):
    nz, ny, nx = shape
    mask, fib = wl.random_geometry(nx, ny, nz, seed=seed, tissue_frac=0.7)
    h, Dpar, Dperp = 0.37, 1.3, 0.2
    A = _numpy_weights(mask, fib, h, Dpar, Dperp)
    u = _rand_u(shape, seed + 100)
    ref = (A @ u.reshape(-1)).reshape(shape)
    got = oracle.Grid(nx, ny, nz, h, mask, fib, Dpar, Dperp).apply_L(u)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_consistency_with_continuous_operator_second_order():
    """For smooth D(r) and u(r), (L u)_p approaches d_j(D_jk d_k u) at interior
    nodes with O(h^2) error: the error ratio between h and h/2 is about 4.  A
    wrong sign or index in Wtilde or in the edge weights leaves an O(1) error."""
    sympy = pytest.importorskip("sympy")
    X = sympy.symbols("x y z")
    kx, ky, kz = 0.7, 0.5, 0.3
    th = 0.6 * sympy.sin(kx * X[0]) + 0.4 * sympy.cos(ky * X[1]) + 0.3 * X[2] * kz
    ph = 0.5 * sympy.cos(kz * X[2] + 0.3 * X[0])
    f = [sympy.cos(th) * sympy.cos(ph), sympy.sin(th) * sympy.cos(ph), sympy.sin(ph)]
    Dpar, Dperp = 1.0, 0.2
    Dm = [[Dperp * (j == k) + (Dpar - Dperp) * f[j] * f[k] for k in range(3)] for j in range(3)]
    u = sympy.sin(0.9 * X[0] + 0.2) * sympy.cos(0.7 * X[1] - 0.4) * sympy.exp(0.3 * X[2])
    Lu = sum(sympy.diff(Dm[j][k] * sympy.diff(u, X[k]), X[j]) for j in range(3) for k in range(3))
    Lf = sympy.lambdify(X, Lu, "numpy")
    uf = sympy.lambdify(X, u, "numpy")
    errs = []
    for h in (0.2, 0.1):
        n = int(round(2.4 / h)) + 1
        z, y, x = np.meshgrid(*(np.arange(n) * h,) * 3, indexing="ij")
        fib = wl.smooth_fibres(n, n, n, h, kx, ky, kz).astype(np.float64)
        g = oracle.Grid(n, n, n, h, None, fib.astype(np.float32), Dpar, Dperp)
        num = g.apply_L(uf(x, y, z))
        ex = Lf(x, y, z)
        # centre region (1.0 units wide), away from the no-flux boundary
        c = n // 2
        r = int(round(0.5 / h))
        sl = (slice(c - r, c + r + 1),) * 3
        errs.append(np.abs(num[sl] - ex[sl]).max())
    ratio = errs[0] / errs[1]
    assert errs[1] < 0.05 and 3.0 < ratio < 5.0, (errs, ratio)


def test_zero_fibre_at_tissue_is_an_error_and_void_fibres_ignored():
    mask = np.ones((2, 3, 3), np.uint8)
    fib = _oblique((2, 3, 3))
    fib[1, 1, 1] = 0
    assert oracle.Grid(3, 3, 2, 0.3, mask, fib, 1, 0.2).check_fibres() == -3
    mask[1, 1, 1] = 0
    assert oracle.Grid(3, 3, 2, 0.3, mask, fib, 1, 0.2).check_fibres() == 0


def test_rotational_fibres_have_no_first_order_term():
    # Fibres in the x-y plane whose angle depends on z only: D_xz = D_yz = 0,
    # D_zz = D_perp and D_xx, D_yy, D_xy vary with z alone, so every
    # divergence sum_j d_j D_jk vanishes and the W-tilde part of the weights
    # (the only part of the face weights that is odd in q) is zero: opposite
    # face weights are equal, and L of the linear field u = z is exactly 0 on
    # every plane with two z neighbours.  A field with out-of-plane, varying
    # fibres breaks both.
    nx, ny, nz, h = 9, 7, 8, 0.3
    u = np.broadcast_to(np.arange(nz, dtype=np.float64)[:, None, None], (nz, ny, nx)).copy()
    g = oracle.Grid(nx, ny, nz, h, None, wl.rotational_fibres(nx, ny, nz), 1.0, 0.25)
    assert np.all(g.apply_L(u)[1:-1] == 0.0)
    for (z, y, x) in [(1, 1, 1), (3, 0, 4), (nz - 2, ny - 1, nx - 1), (4, 3, 0)]:
        W = g.weights(x, y, z)
        assert W[1, 1, 0] == W[1, 1, 2] or x in (0, nx - 1)
        assert W[1, 0, 1] == W[1, 2, 1] or y in (0, ny - 1)
        assert W[0, 1, 1] == W[2, 1, 1]
    gs = oracle.Grid(nx, ny, nz, h, None, wl.smooth_fibres(nx, ny, nz, h), 1.0, 0.25)
    assert np.abs(gs.apply_L(u)[1:-1]).max() > 1e-3
    W = gs.weights(4, 3, 4)
    assert max(abs(W[1, 1, 0] - W[1, 1, 2]), abs(W[1, 0, 1] - W[1, 2, 1]), abs(W[0, 1, 1] - W[2, 1, 1])) > 1e-6


def test_uniform_fibres_on_a_masked_grid_have_no_first_order_term():
    # With a void neighbour's tensor replaced by the node's own (the reading of
    # the W-tilde sums at void and out-of-array neighbours), uniform fibres
    # give vanishing sums everywhere, also beside the mask's holes: each face
    # weight is exactly psi of that neighbour times D_kk / h^2, with no odd part.
    nx, ny, nz, h = 7, 6, 5, 0.3
    mask = wl.random_geometry(nx, ny, nz, seed=11, tissue_frac=0.7, aniso=False)[0]
    g = oracle.Grid(nx, ny, nz, h, mask, _oblique((nz, ny, nx)), 1.0, 0.25)
    faces = {0: ((1, 1, 2), (1, 1, 0)), 1: ((1, 2, 1), (1, 0, 1)), 2: ((2, 1, 1), (0, 1, 1))}
    checked = 0
    for (z, y, x) in zip(*np.nonzero(mask)):
        x, y, z = int(x), int(y), int(z)
        W = g.weights(x, y, z)
        rc, D = g.tensor(x, y, z)
        assert rc == 0
        for k, (ip, im) in faces.items():
            for idx, d in ((ip, 1), (im, -1)):
                c = [x, y, z]
                c[k] += d
                inside = 0 <= c[0] < nx and 0 <= c[1] < ny and 0 <= c[2] < nz
                psi = 1.0 if inside and mask[c[2], c[1], c[0]] else 0.0
                assert abs(W[idx] - psi * D[k, k] / h ** 2) <= 1e-12 * D[k, k] / h ** 2
                checked += 1
    assert checked > 100
