"""Headless output kernels through the C ABI against oracle/output.py: the
byte frame bit-exact (the quantisation is decided in float32 on both sides),
phase singularities as point sets (order is free; a point may be missing on
one side only where its position on an isoline piece is within rounding of
the piece's end)."""
import numpy as np
import pytest

import oracle
from oracle import output
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx
    return torch, bbx


def _grid(bbx, w, st):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_fibres(w.fibres, w.D_par, w.D_perp if w.fibres is not None else w.D_par)
    G.set_ionic_model(w.model, w.params)
    G.write_all(st.astype(np.float32))
    return G


def _frame(torch, bbx, G, w, layers, lo, hi):
    out = torch.empty(3 * w.n_cells, dtype=torch.uint8, device="cuda")
    G.ppm_frame(layers, lo, hi, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(w.shape + (3,))


def _oracle_state(w, n_steps):
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    sim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0)
    sim.step(w.dt, n_steps)
    return sim.state.astype(np.float32)


def test_ppm_frame_is_bit_exact(env):
    torch, bbx = env
    w = wl.br_slab(70, 20, 6)
    st = _oracle_state(w, 40)  # a front with every variable away from rest
    G = _grid(bbx, w, st)
    layers, lo, hi = (0, 2, 7), (-90.0, 0.0, 0.0), (40.0, 1.0, 1.0)
    got = _frame(torch, bbx, G, w, layers, lo, hi)
    ref = output.ppm_frame(st, w.mask, layers, lo, hi)
    assert np.array_equal(got, ref)
    # two calls in a row give the same frame; a dark channel stays dark
    got2 = _frame(torch, bbx, G, w, (1, -1, 0), (0.0, 0.0, -90.0), (1e-6, 1.0, 40.0))
    assert np.array_equal(got2, output.ppm_frame(st, w.mask, (1, -1, 0), (0.0, 0.0, -90.0), (1e-6, 1.0, 40.0)))
    assert not got2[..., 1].any()


def test_ppm_frame_masked_shell_and_sheet_colour_map(env):
    torch, bbx = env
    w = wl.br_shell(48)
    st = _oracle_state(w, 20)
    G = _grid(bbx, w, st)
    got = _frame(torch, bbx, G, w, (0, 3, 4), (-90.0, 0.0, 0.0), (40.0, 1.0, 1.0))
    assert np.array_equal(got, output.ppm_frame(st, w.mask, (0, 3, 4), (-90.0, 0.0, 0.0), (40.0, 1.0, 1.0)))
    assert not got[w.mask == 0].any()
    s = wl.fhn_sheet(64, 48)
    st = _oracle_state(s, 50)
    G = _grid(bbx, s, st)
    layers, lo, hi = output.paintgl_ranges()
    assert np.array_equal(_frame(torch, bbx, G, s, layers, lo, hi), output.ppm_frame(st, None, layers, lo, hi))


def _match(gpu, ref, ref_par, tol=2e-4, edge=1e-3):
    """Every GPU point has an oracle point within tol and vice versa, except
    oracle points on the edge of their isoline pieces."""
    def near(p, q):
        if len(q) == 0:
            return np.zeros(len(p), bool)
        d = np.abs(p[:, None, :] - q[None, :, :]).max(axis=2)
        return d.min(axis=1) <= tol
    ok_ref = near(ref, gpu)
    borderline = (np.minimum(ref_par, 1.0 - ref_par) < edge).any(axis=1) if len(ref) else np.zeros(0, bool)
    assert np.all(ok_ref | borderline), (np.count_nonzero(~ok_ref), len(ref))
    assert np.all(near(gpu, ref)), (len(gpu), len(ref))


def _singz(torch, bbx, G, a, ia, b, ib, max_points=4096):
    xyz = torch.empty(3 * max_points, dtype=torch.float32, device="cuda")
    n = G.phase_singularities(a, ia, b, ib, xyz, max_points)
    return n, xyz[:3 * min(n, max_points)].cpu().numpy().reshape(-1, 3).astype(np.float64)


def test_phase_singularities_of_polynomial_fields(env):
    torch, bbx = env
    w = wl.barkley_slab(72, 60, 3)
    z, y, x = np.meshgrid(np.arange(w.nz), np.arange(w.ny), np.arange(w.nx), indexing="ij")
    wc = x + 1j * y
    f = np.ones_like(wc)
    for k, z0 in enumerate([14.3 + 17.6j, 51.7 + 22.2j, 28.4 + 45.1j, 60.2 + 50.9j]):
        f = f * (wc - z0 - 0.7 * z) / 20.0
    st = np.stack([f.real, f.imag]).astype(np.float32)
    G = _grid(bbx, w, st)
    n, got = _singz(torch, bbx, G, 0, 0.0, 1, 0.0)
    ref, par = output.phase_singularities(st[0], st[1], 0.0, 0.0, with_params=True)
    assert n == len(got) and abs(n - len(ref)) <= 1 and len(ref) == 12
    _match(got, ref, par)


def test_phase_singularities_of_a_simulated_spiral_and_truncation(env):
    torch, bbx = env
    w = wl.fhn_sheet(200, 200)
    st = _oracle_state(w, 600)  # the cross-field initial condition curls into a spiral
    G = _grid(bbx, w, st)
    iso_u, iso_v = 0.0, 0.0
    n, got = _singz(torch, bbx, G, 0, iso_u, 1, iso_v)
    ref, par = output.phase_singularities(st[0], st[1], iso_u, iso_v, with_params=True)
    assert n >= 1 and abs(n - len(ref)) <= 1
    _match(got, ref, par)
    # a call with room for fewer points reports the full count and fills what fits
    n2, few = _singz(torch, bbx, G, 0, iso_u, 1, iso_v, max_points=max(n - 1, 0))
    assert n2 == n and len(few) == max(n - 1, 0)
    # masked cells are skipped
    m = np.ones(w.shape, np.uint8)
    m[:, :, : w.nx // 2] = 0
    wm = wl.Workload("fhn_half", w.nx, w.ny, w.nz, w.h, w.dt, w.model, w.params, w.D_par, w.D_perp, mask=m,
                     theta=w.theta)
    Gm = _grid(bbx, wm, st)
    nm, gm = _singz(torch, bbx, Gm, 0, iso_u, 1, iso_v)
    refm, parm = output.phase_singularities(st[0], st[1], iso_u, iso_v, mask=m, with_params=True)
    assert abs(nm - len(refm)) <= 1
    _match(gm, refm, parm)
