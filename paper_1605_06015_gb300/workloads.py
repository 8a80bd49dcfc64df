"""Seeded synthetic inputs shaped like the paper's workloads.

This module serves both the CUDA path and the FP64 oracle.  It holds only
input generation (geometry, fibre fields, initial-condition patterns, random
parameter sweeps) and none of the method's arithmetic: no diffusion tensor,
no stencil weights, no cell model, no rest state.  Everything is NumPy with
``default_rng(seed)``; the default seed of workload i is 16050601 + i.

Layouts are dense with x fastest: scalar fields ``[nz][ny][nx]``, fibres
``[nz][ny][nx][3]`` float32.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED0 = 16050601

FHN, BARKLEY, BR, ZFK, BR_MRL, BR_FCA = 1, 2, 3, 4, 6, 7


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    dt: float
    model: int
    params: list
    D_par: float
    D_perp: float
    mask: np.ndarray | None = None       # uint8 [nz][ny][nx] or None (all tissue)
    fibres: np.ndarray | None = None     # float32 [nz][ny][nx][3] or None (isotropic)
    # initial condition: dict var -> full field, or patterns applied on top of rest
    ic_fields: dict = field(default_factory=dict)   # var -> float array [nz][ny][nx]
    ic_region: np.ndarray | None = None  # bool [nz][ny][nx]: var 0 set to ic_value there
    ic_value: float = 0.0
    n_steps: int = 0
    theta: float = 0.0

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_cells(self):
        return self.nx * self.ny * self.nz

    def n_active(self):
        return self.n_cells if self.mask is None else int(np.count_nonzero(self.mask))

    def initial_state(self, rest):
        """Full initial state [S][nz][ny][nx] float64 built from a rest state
        vector supplied by the caller (the oracle's or the library's)."""
        S = len(rest)
        st = np.empty((S,) + self.shape, dtype=np.float64)
        for v in range(S):
            st[v] = rest[v]
        for v, f in self.ic_fields.items():
            st[v] = f
        if self.ic_region is not None:
            st[0][self.ic_region] = self.ic_value
        return st


# ---------------------------------------------------------------------------
# 1: 2D FitzHugh-Nagumo sheet, cross-field initial condition
# ---------------------------------------------------------------------------

def fhn_sheet(nx=200, ny=200, seed=SEED0 + 0, h=0.5, dt=0.01, D=1.0,
              eps=0.3, beta=0.71, gamma=0.5, noise=1e-3, n_steps=1000):
    """Cross-field IC: u = +1.7 for x-index < nx/2 else -1.7; v = +0.7 for
    y-index < ny/2 else -0.7; plus U(-noise, noise) on both (u first)."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    u = np.where(x < nx // 2, 1.7, -1.7) * np.ones((1, ny, nx))
    v = np.where(y < ny // 2, 0.7, -0.7) * np.ones((1, ny, nx))
    u = u + rng.uniform(-noise, noise, size=u.shape)
    v = v + rng.uniform(-noise, noise, size=v.shape)
    return Workload("fhn2d_%dx%d" % (nx, ny), nx, ny, 1, h, dt, FHN, [eps, beta, gamma], D, D,
                    ic_fields={0: u, 1: v}, n_steps=n_steps, theta=0.0)


# ---------------------------------------------------------------------------
# 2: 3D Barkley slab with rotational anisotropy
# ---------------------------------------------------------------------------

def rotational_fibres(nx, ny, nz, total_deg=120.0):
    """Fibre angle theta(z) = total_deg * z / (nz-1) in the x-y plane."""
    th = np.deg2rad(total_deg) * (np.arange(nz) / max(nz - 1, 1))
    f = np.zeros((nz, ny, nx, 3), dtype=np.float32)
    f[..., 0] = np.cos(th)[:, None, None]
    f[..., 1] = np.sin(th)[:, None, None]
    return f


def point_stimuli(nx, ny, nz, rng, count=8, radius=3.0):
    """Boolean field of `count` balls of the given radius (cells) with
    uniformly drawn centres."""
    reg = np.zeros((nz, ny, nx), dtype=bool)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for _ in range(count):
        cx, cy, cz = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz)
        reg |= (xx - cx) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2 <= radius * radius
    return reg


def barkley_slab(nx=256, ny=256, nz=64, seed=SEED0 + 1, h=0.3, dt=0.005, a=0.75, b=0.02,
                 eps=0.02, D_par=1.0, D_perp=0.25, n_steps=2000):
    rng = np.random.default_rng(seed)
    reg = point_stimuli(nx, ny, nz, rng)
    return Workload("barkley3d_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, h, dt, BARKLEY, [a, b, eps],
                    D_par, D_perp, fibres=rotational_fibres(nx, ny, nz), ic_region=reg, ic_value=1.0,
                    n_steps=n_steps, theta=0.5)


# ---------------------------------------------------------------------------
# 3: ventricle-like thick ellipsoidal shell, helical fibres, Beeler-Reuter
# ---------------------------------------------------------------------------

def shell_geometry(n=512, outer=(200, 200, 240), wall=40):
    """Mask and helical fibres of an ellipsoidal shell centred in an n^3 box.
    Semi-axes scale with n/512.  Fibre angle goes linearly from -60 deg
    (inner surface) to +60 deg (outer surface) in the local tangent plane,
    measured from the circumferential direction."""
    s = n / 512.0
    ao = np.array(outer, dtype=np.float64) * s
    ai = ao - wall * s
    c = (n - 1) / 2.0
    mask = np.zeros((n, n, n), dtype=np.uint8)
    fib = np.zeros((n, n, n, 3), dtype=np.float32)
    x = np.arange(n, dtype=np.float64) - c
    X, Y = np.meshgrid(x, x, indexing="xy")  # [y][x]
    for zi in range(n):
        Z = np.full_like(X, zi - c)
        ro = (X / ao[0]) ** 2 + (Y / ao[1]) ** 2 + (Z / ao[2]) ** 2
        ri = (X / ai[0]) ** 2 + (Y / ai[1]) ** 2 + (Z / ai[2]) ** 2
        m = (ro <= 1.0) & (ri > 1.0)
        if not m.any():
            continue
        mask[zi][m] = 1
        px, py, pz = X[m], Y[m], Z[m]
        # wall depth d in [0,1]: the member of the ellipsoid family with
        # semi-axes ai + d (ao - ai) through the point, by bisection.
        lo = np.zeros(px.shape); hi = np.ones(px.shape)
        for _ in range(40):
            mid = 0.5 * (lo + hi)
            ax = ai[:, None] + mid[None, :] * (ao - ai)[:, None]
            r = (px / ax[0]) ** 2 + (py / ax[1]) ** 2 + (pz / ax[2]) ** 2
            inside = r <= 1.0
            hi = np.where(inside, mid, hi)
            lo = np.where(inside, lo, mid)
        d = 0.5 * (lo + hi)
        ax = ai[:, None] + d[None, :] * (ao - ai)[:, None]
        nrm = np.stack([px / ax[0] ** 2, py / ax[1] ** 2, pz / ax[2] ** 2], axis=1)
        nrm /= np.maximum(np.linalg.norm(nrm, axis=1, keepdims=True), 1e-30)
        circ = np.cross(np.array([0.0, 0.0, 1.0])[None, :], nrm)
        cn = np.linalg.norm(circ, axis=1, keepdims=True)
        circ = np.where(cn > 1e-6, circ / np.maximum(cn, 1e-30), np.array([1.0, 0.0, 0.0])[None, :])
        longi = np.cross(nrm, circ)
        alpha = np.deg2rad(-60.0 + 120.0 * d)[:, None]
        f = np.cos(alpha) * circ + np.sin(alpha) * longi
        fib[zi][m] = f.astype(np.float32)
    return mask, fib, ao, c


def br_shell(n=512, seed=SEED0 + 2, h=0.2, dt=0.02, D_par=0.1, D_perp=0.025, t_end=500.0):
    """Apex stimulus: V = +20 mV at t = 0 in a ball of radius 10 (scaled)
    around the outer surface's -z pole; every other variable at rest."""
    mask, fib, ao, c = shell_geometry(n)
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    apex = np.array([c, c, c - ao[2]])
    r = 10.0 * n / 512.0
    reg = ((xx - apex[0]) ** 2 + (yy - apex[1]) ** 2 + (zz - apex[2]) ** 2 <= r * r) & (mask != 0)
    return Workload("br_shell_%d" % n, n, n, n, h, dt, BR, [4.0, 0.003, 50.0, 0.09], D_par, D_perp,
                    mask=mask, fibres=fib, ic_region=reg, ic_value=20.0,
                    n_steps=int(round(t_end / dt)), theta=-40.0)


def br_slab(nx=256, ny=256, nz=64, seed=SEED0 + 3, h=0.2, dt=0.02, D_par=0.1, D_perp=0.025,
            n_steps=100):
    """The slab of workload 2 with Beeler-Reuter physics; V = +20 mV in the
    x < 4 face layer at t = 0."""
    reg = np.zeros((nz, ny, nx), dtype=bool)
    reg[:, :, :4] = True
    return Workload("br_slab_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, h, dt, BR, [4.0, 0.003, 50.0, 0.09],
                    D_par, D_perp, fibres=rotational_fibres(nx, ny, nz), ic_region=reg, ic_value=20.0,
                    n_steps=n_steps, theta=-40.0)


def br_mrl_slab(nx=256, ny=256, nz=64, **kw):
    """br_slab with the sodium activation in its Markov form (BR_MRL, matrix
    Rush-Larsen); same geometry, fibres, physics and initial condition."""
    w = br_slab(nx, ny, nz, **kw)
    w.name = "br_mrl_slab_%dx%dx%d" % (nx, ny, nz)
    w.model = BR_MRL
    return w


def br_fca_slab(nx=256, ny=256, nz=64, onfly=False, **kw):
    """br_slab with the slow inward current's inactivation as a two-gate
    channel (voltage gate f, calcium gate c; BR_FCA, the multivariate chain
    split into univariate parts, or with onfly its whole generator's
    exponential at run time); same geometry, fibres and initial condition,
    default channel parameters."""
    w = br_slab(nx, ny, nz, **kw)
    w.name = "br_fca_slab_%dx%dx%d%s" % (nx, ny, nz, "_onfly" if onfly else "")
    w.model = BR_FCA
    if onfly:
        w.params = [4.0, 0.003, 50.0, 0.09, 5e-6, 2.0, 0.05, 1.0]
    return w


# ---------------------------------------------------------------------------
# 5: batch of independent tissues
# ---------------------------------------------------------------------------

def tissue_batch(seed=SEED0 + 4, n2d=192, n3d=64, side2d=(64, 512), side3d=(64, 128), sweep=0.2,
                 n_steps=1000):
    """n2d FHN sheets with sides drawn uniformly in side2d and n3d Barkley
    blocks with sides drawn uniformly in side3d; D and model parameters each
    scaled by a factor drawn uniformly in [1-sweep, 1+sweep]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n2d):
        nx, ny = (int(v) for v in rng.integers(side2d[0], side2d[1] + 1, size=2))
        k = rng.uniform(1 - sweep, 1 + sweep, size=4)
        w = fhn_sheet(nx, ny, seed=seed * 1000 + i, D=1.0 * k[0], eps=0.3 * k[1], beta=0.71 * k[2],
                      gamma=0.5 * k[3], n_steps=n_steps)
        out.append(w)
    for i in range(n3d):
        nx, ny, nz = (int(v) for v in rng.integers(side3d[0], side3d[1] + 1, size=3))
        k = rng.uniform(1 - sweep, 1 + sweep, size=4)
        srng = np.random.default_rng(seed * 1000 + n2d + i)
        reg = point_stimuli(nx, ny, nz, srng, count=2)
        D = 1.0 * k[0]
        out.append(Workload("barkley_block_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, 0.3, 0.005, BARKLEY,
                            [0.75 * k[1], 0.02 * k[2], 0.02 * k[3]], D, D, ic_region=reg,
                            ic_value=1.0, n_steps=n_steps, theta=0.5))
    return out


# ---------------------------------------------------------------------------
# small random geometries for tests
# ---------------------------------------------------------------------------

def random_geometry(nx, ny, nz, seed, tissue_frac=0.7, aniso=True):
    """Random mask (tissue with probability tissue_frac) and random non-unit
    fibre vectors (normal components, re-drawn where the norm is tiny)."""
    rng = np.random.default_rng(seed)
    mask = (rng.random((nz, ny, nx)) < tissue_frac).astype(np.uint8)
    fib = None
    if aniso:
        fib = rng.normal(size=(nz, ny, nx, 3)).astype(np.float32)
        small = np.linalg.norm(fib, axis=-1) < 0.1
        fib[small] = np.array([1.0, 0.5, 0.25], dtype=np.float32)
    return mask, fib


def smooth_fibres(nx, ny, nz, h, kx=0.7, ky=0.5, kz=0.3):
    """A smooth, non-uniform unit fibre field f(r) on a grid of spacing h
    (angles are smooth functions of position)."""
    z, y, x = np.meshgrid(np.arange(nz) * h, np.arange(ny) * h, np.arange(nx) * h, indexing="ij")
    th = 0.6 * np.sin(kx * x) + 0.4 * np.cos(ky * y) + 0.3 * z * kz
    ph = 0.5 * np.cos(kz * z + 0.3 * x)
    f = np.stack([np.cos(th) * np.cos(ph), np.sin(th) * np.cos(ph), np.sin(ph)], axis=-1)
    return f.astype(np.float32)
