"""Output arithmetic of the paper's monitoring devices, for the headless output
kernels: the 1-byte quantisation of three grid layers (``ppmout``, section
"Input and output": each value discretized to the 0..255 scale between a
lower and an upper bound), the ``k_paintgl`` colour map of the appendix's
sample script (red = u, green = v / 0.8, blue = 0), and phase singularities
in z cross-sections (``singz``, same section: intersections of the isolines
of two fields, located inside a grid cell by linear interpolation of the
isoline pieces).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain NumPy and Python
loops.  Readings where the paper is silent:
  * quantisation: t = (v - lo) / (hi - lo) clamped to [0, 1], code =
    floor(255 t + 0.5), evaluated in float32 (the precision of the state
    being quantised) with one rounding per operation;
  * void nodes and channels without a layer give 0;
  * an isoline crosses a cell edge where f - f* is > 0 at one end and not at
    the other; a cell holds a piece of the isoline only if exactly two of its
    edges are crossed (saddle cells with four crossings are skipped); the
    singularity is the intersection of the two pieces when it lies on both
    (parameters in [0, 1]); cells with a void corner are skipped.
"""
from __future__ import annotations

import numpy as np


def quantise(v, lo, hi):
    """Byte codes of values v between lo and hi (float32 arithmetic)."""
    v = np.asarray(v, dtype=np.float32)
    lo32, hi32 = np.float32(lo), np.float32(hi)
    t = (v - lo32) / (hi32 - lo32)
    t = np.minimum(np.maximum(t, np.float32(0.0)), np.float32(1.0))
    return np.floor(t * np.float32(255.0) + np.float32(0.5)).astype(np.uint8)


def ppm_frame(state, mask, layers, lo, hi):
    """RGB bytes [nz][ny][nx][3] of the given layers (index, or -1 for a dark
    channel) of state [S][nz][ny][nx]; void nodes are black."""
    state = np.asarray(state, dtype=np.float32)
    out = np.zeros(state.shape[1:] + (3,), dtype=np.uint8)
    for c in range(3):
        if layers[c] >= 0:
            out[..., c] = quantise(state[layers[c]], lo[c], hi[c])
    if mask is not None:
        out[np.asarray(mask) == 0] = 0
    return out


def paintgl_ranges():
    """The sample script's colour map as quantisation ranges: red = u over
    [0, 1], green = v / 0.8, i.e. v over [0, 0.8], blue dark."""
    return (0, 1, -1), (0.0, 0.0, 0.0), (1.0, 0.8, 1.0)


def _crossings(g, corners):
    pts = []
    for i in range(4):
        j = (i + 1) % 4
        if (g[i] > 0) != (g[j] > 0):
            s = g[i] / (g[i] - g[j])
            pts.append(corners[i] + s * (corners[j] - corners[i]))
    return pts


def phase_singularities(a, b, iso_a, iso_b, mask=None, with_params=False):
    """Intersections of the isolines a = iso_a and b = iso_b in every z
    cross-section of the fields a, b [nz][ny][nx] (float64 arithmetic on the
    given values).  Returns an array of (x, y, z) rows in cell order, and with
    with_params also the segment parameters (alpha, beta) of each point."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nz, ny, nx = a.shape
    tis = np.ones(a.shape, bool) if mask is None else np.asarray(mask) != 0
    corners = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    off = [(0, 0), (1, 0), (1, 1), (0, 1)]
    out, par = [], []
    for z in range(nz):
        for y in range(ny - 1):
            for x in range(nx - 1):
                if not all(tis[z, y + dy, x + dx] for dx, dy in off):
                    continue
                ga = np.array([a[z, y + dy, x + dx] - iso_a for dx, dy in off])
                gb = np.array([b[z, y + dy, x + dx] - iso_b for dx, dy in off])
                pa = _crossings(ga, corners)
                pb = _crossings(gb, corners)
                if len(pa) != 2 or len(pb) != 2:
                    continue
                d1, d2 = pa[1] - pa[0], pb[1] - pb[0]
                det = d1[0] * (-d2[1]) - d1[1] * (-d2[0])
                if det == 0.0:
                    continue
                r = pb[0] - pa[0]
                al = (r[0] * (-d2[1]) - r[1] * (-d2[0])) / det
                be = (d1[0] * r[1] - d1[1] * r[0]) / det
                if 0.0 <= al <= 1.0 and 0.0 <= be <= 1.0:
                    p = pa[0] + al * d1
                    out.append((x + p[0], y + p[1], float(z)))
                    par.append((al, be))
    pts = np.array(out, dtype=np.float64).reshape(-1, 3)
    if with_params:
        return pts, np.array(par, dtype=np.float64).reshape(-1, 2)
    return pts
