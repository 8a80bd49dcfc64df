"""Pins of the output arithmetic in oracle/output.py: the byte quantisation
(end points, midpoint, clamping, the half-step error bound), the sample
script's colour map, and phase singularities at the closed-form zeros of
linear and polynomial fields."""
import numpy as np

from oracle import output


def test_quantisation_end_points_midpoint_clamping_and_error_bound():
    lo, hi = -85.0, 40.0
    assert output.quantise(lo, lo, hi) == 0
    assert output.quantise(hi, lo, hi) == 255
    assert output.quantise(0.5 * (lo + hi), lo, hi) == 128  # 127.5 rounds up
    assert output.quantise(lo - 10, lo, hi) == 0 and output.quantise(hi + 10, lo, hi) == 255
    v = np.random.default_rng(1).uniform(lo, hi, 10000)
    q = output.quantise(v, lo, hi).astype(np.float64)
    t = (v - lo) / (hi - lo)
    assert np.abs(q / 255.0 - t).max() <= 0.5 / 255.0 + 1e-6
    assert np.all(np.diff(q[np.argsort(v)]) >= 0)  # monotone


def test_paintgl_colour_map_of_the_sample_script():
    layers, lo, hi = output.paintgl_ranges()
    st = np.zeros((2, 1, 1, 3))
    st[0, 0, 0] = [1.0, 0.0, 0.5]
    st[1, 0, 0] = [0.8, 0.0, 0.4]
    f = output.ppm_frame(st, None, layers, lo, hi)
    assert f[0, 0, 0].tolist() == [255, 255, 0]
    assert f[0, 0, 1].tolist() == [0, 0, 0]
    assert f[0, 0, 2].tolist() == [128, 128, 0]


def test_void_nodes_are_black():
    st = np.ones((1, 2, 3, 4))
    mask = np.ones((2, 3, 4), np.uint8)
    mask[1, 2, 3] = 0
    f = output.ppm_frame(st, mask, (0, 0, -1), (0, 0, 0), (1, 1, 1))
    assert f[1, 2, 3].tolist() == [0, 0, 0] and f[0, 0, 0].tolist() == [255, 255, 0]


def test_linear_fields_give_their_exact_intersection_in_every_plane():
    # a = cos(phi) x + sin(phi) y - c1, b = -sin(phi) x + cos(phi) y - c2:
    # straight isolines (linear interpolation is exact), meeting at one point
    nz, ny, nx = 3, 20, 24
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = 0.37
    x0, y0 = 11.3, 7.8
    a = np.cos(phi) * (x - x0) + np.sin(phi) * (y - y0)
    b = -np.sin(phi) * (x - x0) + np.cos(phi) * (y - y0)
    pts = output.phase_singularities(a, b, 0.0, 0.0)
    assert pts.shape == (3, 3)
    assert np.allclose(pts[:, 0], x0, atol=1e-12) and np.allclose(pts[:, 1], y0, atol=1e-12)
    assert sorted(pts[:, 2].tolist()) == [0.0, 1.0, 2.0]


def test_zeros_of_a_polynomial_field_are_found_and_nothing_else():
    # a + i b = (w - w1)(w - w2)(w - w3) / s^3 with w = x + i y: three
    # phase singularities at the zeros, located to second order in h
    nx = ny = 60
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    w = x + 1j * y
    zeros = [14.3 + 17.6j, 41.7 + 22.2j, 28.4 + 45.1j]
    f = np.ones_like(w)
    for z0 in zeros:
        f = f * (w - z0) / 20.0
    pts = output.phase_singularities(f.real[None], f.imag[None], 0.0, 0.0)
    assert len(pts) == 3
    for z0 in zeros:
        d = np.hypot(pts[:, 0] - z0.real, pts[:, 1] - z0.imag).min()
        assert d < 0.05, (z0, d)


def test_cells_with_a_void_corner_are_skipped():
    nz, ny, nx = 1, 10, 10
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    a = (x - 4.5)[None].astype(float)
    b = (y - 4.5)[None].astype(float)
    assert len(output.phase_singularities(a, b, 0, 0)) == 1
    mask = np.ones((nz, ny, nx), np.uint8)
    mask[0, 5, 5] = 0
    assert len(output.phase_singularities(a, b, 0, 0, mask)) == 0
