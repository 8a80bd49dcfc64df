"""GPU parity: the CUDA step (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Bars: relative L-infinity of V <= 1e-4 after 100 steps,
activation steps within 1 step over a full run, integer outputs bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

V_TOL = 1e-4      # relative L-infinity on V after 100 steps
OTHER_TOL = 1e-3  # other state variables (reported, looser)


@pytest.fixture(scope="module")
def bbx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx as b
    return b


def _rel_linf(got, ref, sel):
    scale = max(np.abs(ref[sel]).max(), 1e-30)
    return np.abs(got[sel] - ref[sel]).max() / scale


def _gpu_grid(bbx, w, ty=None, tz=None):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    if w.fibres is not None:
        G.set_fibres(w.fibres, w.D_par, w.D_perp)
    else:
        G.set_fibres(None, w.D_par, w.D_par)
    if ty is not None:
        G.set_tiling(ty, tz)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    return G


def _pair(bbx, w, n_steps, ty=None, tz=None, stim=None):
    """Run n_steps on both sides from the same float32-rounded initial state."""
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
    G = _gpu_grid(bbx, w, ty, tz)
    G.write_all(st0)
    if stim is not None:
        osim.set_stimulus(*stim)
        G.set_stimulus(*stim)
    osim.step(w.dt, n_steps)
    G.step(w.dt, n_steps)
    return osim, G


def _check_state(osim, G, w):
    tis = osim.grid.psi
    got = G.read_all()
    e = [_rel_linf(got[v], osim.state[v], tis) for v in range(osim.S)]
    assert e[0] <= V_TOL, e
    for v in range(1, osim.S):
        assert e[v] <= OTHER_TOL, (v, e)
    # void nodes are never touched
    if w.mask is not None:
        void = ~tis
        assert np.array_equal(got[:, void], osim.state[:, void].astype(np.float32))
    return e


def _check_activation(osim, G, n_steps):
    ag = G.read_activation().astype(np.int64)
    ao = osim.act.astype(np.int64)
    big = n_steps + 1
    ag[ag == oracle.INT32_MAX] = big
    ao[ao == oracle.INT32_MAX] = big
    tis = osim.grid.psi
    d = np.abs(ag - ao)[tis]
    assert d.max() <= 1, (d.max(), np.count_nonzero(d > 1))
    return int(np.count_nonzero(ao[tis] < big))


def test_fhn2d_config1_100_steps(bbx):
    w = wl.fhn_sheet()
    osim, G = _pair(bbx, w, 100)
    _check_state(osim, G, w)


def test_fhn2d_config1_activation_full_run(bbx):
    w = wl.fhn_sheet()
    osim, G = _pair(bbx, w, w.n_steps)
    n_act = _check_activation(osim, G, w.n_steps)
    assert n_act > 1000  # the cross-field IC makes a wave that activates tissue


@pytest.mark.parametrize("shape,ty,tz", [((96, 40, 24), 14, 16), ((67, 45, 13), 7, 5), ((130, 33, 9), 28, 4),
                                         ((64, 16, 40), 14, 40)])
def test_barkley3d_rotating_fibres_100_steps(bbx, shape, ty, tz):
    nx, ny, nz = shape
    w = wl.barkley_slab(nx, ny, nz)
    osim, G = _pair(bbx, w, 100, ty, tz)
    _check_state(osim, G, w)
    _check_activation(osim, G, 100)


def test_br_slab_100_steps(bbx):
    w = wl.br_slab(72, 20, 10)
    osim, G = _pair(bbx, w, 100, 14, 5)
    _check_state(osim, G, w)


@pytest.mark.parametrize("ty,tz", [(14, 8), (7, 4)])
def test_br_shell_masked_100_steps_and_bricks(bbx, ty, tz):
    w = wl.br_shell(64)
    osim, G = _pair(bbx, w, 100, ty, tz)
    _check_state(osim, G, w)
    _check_activation(osim, G, 100)
    og = osim.grid
    for ty, tz in ((14, 8), (7, 3), (14, 64)):
        G.set_tiling(ty, tz)
        assert np.array_equal(G.read_active_bricks(), og.active_bricks(64, ty, min(tz, w.nz)))


@pytest.mark.parametrize("seed,shape,aniso", [(1, (37, 29, 11), True), (2, (70, 9, 6), True), (3, (23, 41, 1), True),
                                              (4, (65, 17, 7), False)])
def test_random_masks_and_fibres_zfk(bbx, seed, shape, aniso):
    nx, ny, nz = shape
    mask, fib = wl.random_geometry(nx, ny, nz, seed, tissue_frac=0.6, aniso=aniso)
    rng = np.random.default_rng(seed + 50)
    w = wl.Workload("zfk_rand", nx, ny, nz, 0.5, 0.01, wl.ZFK, [0.13], 1.0, 0.3 if aniso else 1.0, mask=mask,
                    fibres=fib, ic_fields={0: rng.random((nz, ny, nx))}, theta=0.5)
    osim, G = _pair(bbx, w, 60, 7, 4)
    _check_state(osim, G, w)
    for ty, tz in ((28, 2), (7, 5), (14, 64)):
        G.set_tiling(ty, tz)
        assert np.array_equal(G.read_active_bricks(), osim.grid.active_bricks(64, ty, min(tz, w.nz)))


def test_isotropic_2d_fhn_ragged_sheet(bbx):
    w = wl.fhn_sheet(131, 77)
    osim, G = _pair(bbx, w, 100, 28, 1)
    _check_state(osim, G, w)


@pytest.mark.parametrize("shape,ty,masked", [((150, 90), 7, False), ((150, 90), 14, False), ((131, 61), 28, False),
                                             ((64, 200), 14, False), ((97, 83), 14, True)])
def test_anisotropic_sheet_tiles_march_along_y(bbx, shape, ty, masked):
    """Sheets (nz = 1) with smooth fibres that leave the plane (f_z != 0, so the
    z terms must vanish): several tiles per piece, a ragged last tile, and a
    masked sheet whose interior bit counts in-plane neighbours only."""
    nx, ny = shape
    rng = np.random.default_rng(nx + 1000 * ty)
    fib = wl.smooth_fibres(nx, ny, 1, 0.5)
    mask = (rng.random((1, ny, nx)) < 0.8).astype(np.uint8) if masked else None
    if masked:
        mask[:, ny // 3:ny // 3 + 20, nx // 4:nx // 4 + 30] = 1  # an all-tissue block: interior nodes
    w = wl.Workload("zfk_sheet", nx, ny, 1, 0.5, 0.01, wl.ZFK, [0.13], 1.0, 0.3, mask=mask, fibres=fib,
                    ic_fields={0: rng.random((1, ny, nx))}, theta=0.5)
    osim, G = _pair(bbx, w, 60, ty, 1)
    _check_state(osim, G, w)


@pytest.mark.parametrize("name", ["fhn", "barkley", "br"])
def test_lie_splitting_matches_the_oracle(bbx, name):
    """bbx_set_scheme(BBX_SCHEME_LIE): the diffusion substep, then the
    kinetics step from the half-step voltage (section "Operator splitting"),
    against the oracle's split mode."""
    w = {"fhn": lambda: wl.fhn_sheet(90, 70), "barkley": lambda: wl.barkley_slab(70, 30, 12),
         "br": lambda: wl.br_slab(72, 20, 8)}[name]()
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64), split=True)
    G = _gpu_grid(bbx, w)
    G.set_scheme(bbx.BBX_SCHEME_LIE)
    G.write_all(st0)
    osim.step(w.dt, 100)
    G.step(w.dt, 100)
    _check_state(osim, G, w)
    _check_activation(osim, G, 100)
    # and the unsplit oracle is measurably different (the mode is not ignored)
    ou = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
    ou.step(w.dt, 100)
    got = G.read_all()[0]
    assert _rel_linf(got, ou.state[0], og.psi) > 10 * _rel_linf(got, osim.state[0], og.psi)


def test_lie_splitting_of_pure_diffusion_is_the_unsplit_step(bbx):
    w = wl.barkley_slab(40, 24, 10)
    rng = np.random.default_rng(8)
    st0 = rng.random((1,) + w.shape).astype(np.float32)
    out = []
    for scheme in (bbx.BBX_SCHEME_UNSPLIT, bbx.BBX_SCHEME_LIE):
        G = bbx.Grid(w.nx, w.ny, w.nz, w.h, None)
        G.set_fibres(w.fibres, w.D_par, w.D_perp)
        G.set_ionic_model(bbx.BBX_DIFFUSION, None)
        G.set_scheme(scheme)
        G.write_all(st0)
        G.step(w.dt, 50)
        out.append(G.read_all())
    assert np.abs(out[0] - out[1]).max() <= 2e-7 * np.abs(out[0]).max()
    with pytest.raises(bbx.BbxError):
        G.set_scheme(7)


@pytest.mark.parametrize("name,split", [("fhn", False), ("barkley", False), ("zfk", False), ("barkley", True)])
def test_rk4_kinetics_matches_the_oracle(bbx, name, split):
    """bbx_set_solver(BBX_SOLVER_RK4): one classical RK4 step of the kinetics
    per time step (diffusion term frozen, or the Lie scheme), against the
    oracle's RK4 mode; and Euler is measurably different."""
    if name == "zfk":
        nx, ny, nz = 50, 30, 9
        rng = np.random.default_rng(4)
        w = wl.Workload("zfk", nx, ny, nz, 0.5, 0.02, wl.ZFK, [0.13], 1.0, 0.3, fibres=wl.smooth_fibres(nx, ny, nz, 0.5),
                        ic_fields={0: rng.random((nz, ny, nx))}, theta=0.5)
    else:
        w = {"fhn": lambda: wl.fhn_sheet(90, 70), "barkley": lambda: wl.barkley_slab(70, 30, 12)}[name]()
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64), split=split, rk4=True)
    G = _gpu_grid(bbx, w)
    G.set_solver(bbx.BBX_SOLVER_RK4)
    if split:
        G.set_scheme(bbx.BBX_SCHEME_LIE)
    G.write_all(st0)
    osim.step(w.dt, 100)
    G.step(w.dt, 100)
    _check_state(osim, G, w)
    _check_activation(osim, G, 100)
    oe = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64), split=split)
    oe.step(w.dt, 100)
    got = G.read_all()[0]
    assert _rel_linf(got, oe.state[0], og.psi) > 10 * _rel_linf(got, osim.state[0], og.psi)


def test_rk4_refused_for_beeler_reuter(bbx):
    w = wl.br_slab(20, 10, 4)
    G = _gpu_grid(bbx, w)
    with pytest.raises(bbx.BbxError):
        G.set_solver(bbx.BBX_SOLVER_RK4)


def test_stimulus_current(bbx):
    w = wl.fhn_sheet(70, 50)
    w.ic_fields = {}
    reg = np.zeros(w.shape, np.uint8)
    reg[0, 20:30, 10:20] = 1
    osim, G = _pair(bbx, w, 100, stim=(reg, 1.5, 0.2, 0.6))
    _check_state(osim, G, w)


def test_totals_fused_and_standalone(bbx):
    w = wl.br_shell(48)
    osim, G = _pair(bbx, w, 20, 14, 8)
    g = osim.grid
    for v in range(osim.S):
        got = G.total(v)
        ref = g.total(G.read_state(v).astype(np.float64))
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-300)
    ref0 = g.total(G.read_state(0).astype(np.float64))
    assert G.step_total() == pytest.approx(ref0, rel=1e-12)



def test_step_total_across_retiling_batches_and_autotune(bbx):
    # A single-grid step leaves its total as per-piece partials, summed when
    # asked for: it must survive a new tile shape (which replaces the
    # partials), follow batch steps of the same grid, and be restored by the
    # autotuner together with the state.
    w = wl.barkley_slab(70, 40, 10)
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    G = _gpu_grid(bbx, w, 14, 4)
    G.write_all(st0)

    def sum_now():
        return og.total(G.read_state(0).astype(np.float64))

    G.step(w.dt, 3)
    t3 = sum_now()
    G.set_tiling(7, 8)
    assert G.step_total() == pytest.approx(t3, rel=1e-12)
    G.step(w.dt, 2)
    assert G.step_total() == pytest.approx(sum_now(), rel=1e-12)
    H = _gpu_grid(bbx, wl.fhn_sheet(50, 30))
    H.set_timestep(0.01)
    B = bbx.Batch([G, H])
    B.step(2)
    B.sync()
    assert G.step_total() == pytest.approx(sum_now(), rel=1e-12)
    G.step(w.dt, 1)
    t_before = G.step_total()
    assert t_before == pytest.approx(sum_now(), rel=1e-12)
    G.step(w.dt, 1)
    t_now = sum_now()
    G.autotune(w.dt)
    assert G.step_total() == pytest.approx(t_now, rel=1e-12)
    assert sum_now() == t_now


def test_non_finite_state_is_reported(bbx):
    w = wl.fhn_sheet(64, 32)
    G = _gpu_grid(bbx, w)
    st = np.zeros((2, 1, 32, 64), np.float32)
    st[0, 0, 10, 20] = 3e38  # the cubic overflows: inf, then nan
    G.write_all(st)
    G.step(w.dt, 2)
    with pytest.raises(bbx.BbxError) as e:
        G.step_total()
    assert e.value.code == bbx.BBX_ERR_NAN
    G.clear_device_error()


def test_conservation_uniform_fibres_masked_diffusion(bbx):
    mask, _ = wl.random_geometry(70, 30, 12, 9, tissue_frac=0.8, aniso=False)
    fib = np.zeros((12, 30, 70, 3), np.float32)
    fib[...] = np.array([0.6, -0.3, 0.74], np.float32)
    rng = np.random.default_rng(3)
    u0 = rng.random((12, 30, 70)).astype(np.float32)
    G = bbx.Grid(70, 30, 12, 0.5, mask)
    G.set_fibres(fib, 1.0, 0.25)
    G.set_ionic_model(bbx.BBX_DIFFUSION)
    G.write_state(0, u0)
    T0 = G.total(0)
    G.step(0.02, 300)
    T1 = G.total(0)
    u1 = G.read_state(0)
    tis = mask != 0
    # no-flux boundaries conserve the tissue total; FP32 round-off only
    assert abs(T1 - T0) <= 1e-5 * np.abs(u0[tis]).sum()
    assert u1[tis].std() < 0.5 * u0[tis].std()  # and it did diffuse


def test_homogeneous_tissue_stays_homogeneous_bitwise(bbx):
    mask, fib = wl.random_geometry(50, 20, 9, 11, tissue_frac=0.7)
    G = bbx.Grid(50, 20, 9, 0.3, mask)
    G.set_fibres(fib, 1.0, 0.2)
    G.set_ionic_model(bbx.BBX_BARKLEY)
    G.write_state(0, np.full((9, 20, 50), 0.9, np.float32))
    G.write_state(1, np.full((9, 20, 50), 0.1, np.float32))
    G.step(0.005, 150)
    u = G.read_state(0)[mask != 0]
    assert np.all(u == u[0])


def test_edge_cases(bbx):
    # single node, isotropic and anisotropic
    for fib in (None, np.array([[[[0.0, 0.0, 2.0]]]], np.float32)):
        G = bbx.Grid(1, 1, 1, 0.3)
        G.set_fibres(fib, 1.0, 0.5)
        G.set_ionic_model(bbx.BBX_FHN)
        G.write_state(0, np.array([[[1.7]]], np.float32))
        G.step(0.01, 10)
        y = np.array([1.7, oracle.rest_state(oracle.FHN)[1]], np.float32).astype(np.float64)
        for _ in range(10):
            y = oracle.cell_update(oracle.FHN, y, dt=0.01)
        assert abs(G.read_state(0)[0, 0, 0] - y[0]) < 1e-5
    # no tissue at all: stepping is a no-op
    G = bbx.Grid(40, 10, 3, 0.3, np.zeros((3, 10, 40), np.uint8))
    G.set_ionic_model(bbx.BBX_BARKLEY)
    G.step(0.005, 5)
    assert G.step_total() == 0.0 and G.get_info()["n_bricks"] == 0
    # isolated tissue nodes behave as single cells
    m = np.zeros((5, 6, 7), np.uint8)
    m[0, 0, 0] = m[2, 3, 4] = m[4, 5, 6] = 1
    G = bbx.Grid(7, 6, 5, 0.3, m)
    G.set_fibres(np.ones((5, 6, 7, 3), np.float32), 1.0, 0.1)
    G.set_ionic_model(bbx.BBX_BARKLEY)
    G.write_state(0, np.full((5, 6, 7), 0.9, np.float32))
    G.step(0.005, 50)
    u = G.read_state(0)[m != 0]
    assert np.all(u == u[0])
    # one-node-thick 3D sheet (nz = 1 plane inside a 3-plane box)
    m = np.zeros((3, 20, 70), np.uint8)
    m[1] = 1
    w = wl.Workload("sheet", 70, 20, 3, 0.4, 0.01, wl.ZFK, [0.13], 1.0, 0.3, mask=m,
                    fibres=wl.rotational_fibres(70, 20, 3),
                    ic_fields={0: np.random.default_rng(0).random((3, 20, 70))}, theta=0.5)
    osim, G = _pair(bbx, w, 50, 7, 2)
    _check_state(osim, G, w)


def test_errors_are_reported(bbx):
    G = bbx.Grid(16, 8, 4, 0.3)
    with pytest.raises(bbx.BbxError) as e:
        G.step(0.01, 1)
    assert e.value.code == bbx.BBX_ERR_STATE
    G.set_ionic_model(bbx.BBX_FHN)
    with pytest.raises(bbx.BbxError) as e:
        G.step(1.0, 1)
    assert e.value.code == bbx.BBX_ERR_UNSTABLE
    # parameters the kernels divide by are refused, and the grid keeps its model
    for model, par in ((bbx.BBX_FHN, [0.0]), (bbx.BBX_BARKLEY, [0.75, 0.02, 0.0]),
                       (bbx.BBX_BR_FCA, [4.0, 0.003, 50.0, 0.09, 5e-6, 0.0]),
                       (bbx.BBX_BR_FCA, [4.0, 0.003, 50.0, 0.09, -1.0])):
        with pytest.raises(bbx.BbxError) as e:
            G.set_ionic_model(model, par)
        assert e.value.code == bbx.BBX_ERR_ARG
    assert G.get_info()["model"] == bbx.BBX_FHN
    fib = np.ones((4, 8, 16, 3), np.float32)
    fib[1, 2, 3] = 0
    with pytest.raises(bbx.BbxError) as e:
        G.set_fibres(fib, 1.0, 0.2)
    assert e.value.code == bbx.BBX_ERR_FIBRE
    assert G.get_info()["anisotropic"] == 0
    # a tile shape whose stage ring does not fit shared memory is refused and
    # the grid keeps working with its previous shape
    H = bbx.Grid(64, 64, 8, 0.2, np.ones((8, 64, 64), np.uint8))
    H.set_fibres(np.ones((8, 64, 64, 3), np.float32), 0.1, 0.025)
    H.set_ionic_model(bbx.BBX_BR)
    with pytest.raises(bbx.BbxError) as e:
        H.set_tiling(28, 8)
    assert e.value.code == bbx.BBX_ERR_UNSUPPORTED
    H.step(0.02, 2)
    assert np.isfinite(H.read_state(0)).all()


def test_bounded_wait_reports_timeout_and_recovers(bbx):
    # Fault injection on the host side of the protocol: one CTA waits for
    # bytes no copy delivers; its bounded wait runs out and the step records
    # a timeout instead of hanging.  The context stays usable.
    w = wl.barkley_slab(64, 32, 16)
    G = _gpu_grid(bbx, w, 14, 8)
    G.debug_poison_first_load(1)
    G.step(w.dt, 1)
    with pytest.raises(bbx.BbxError) as e:
        G.read_state(0)
    assert e.value.code == bbx.BBX_ERR_TIMEOUT
    G.debug_poison_first_load(0)
    G.clear_device_error()
    osim, G2 = _pair(bbx, w, 20, 14, 8)
    _check_state(osim, G2, w)


def test_checkpoint_resume_is_bit_identical(bbx):
    w = wl.barkley_slab(80, 24, 12)
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    A = _gpu_grid(bbx, w, 14, 4)
    A.write_all(st0)
    A.step(w.dt, 60)
    mid, act, (t, n) = A.read_all(), A.read_activation(), A.get_time()
    A.step(w.dt, 60)
    B = _gpu_grid(bbx, w, 14, 4)
    B.write_all(mid)
    B.write_activation(act)
    B.set_time(t, n)
    B.step(w.dt, 60)
    assert np.array_equal(A.read_all(), B.read_all())
    assert np.array_equal(A.read_activation(), B.read_activation())


def test_bound_torch_buffers(bbx):
    import torch
    w = wl.barkley_slab(64, 20, 6)
    G = _gpu_grid(bbx, w, 14, 6)
    info = G.get_info()
    n = info["nvars"] * info["nz"] * info["ny"] * info["px"]
    a = torch.zeros(n, dtype=torch.float32, device="cuda")
    b = torch.zeros(n, dtype=torch.float32, device="cuda")
    G.bind_state(a, b)
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    G.write_all(st0)
    G.step(w.dt, 3)
    torch.cuda.synchronize()
    cur = a if G.state_device_ptr(0) == a.data_ptr() else b
    u = cur.view(info["nvars"], info["nz"], info["ny"], info["px"])[0, :, :, :info["nx"]].cpu().numpy()
    assert np.array_equal(u, G.read_state(0))


def test_full_size_slab_one_step_sampled(bbx):
    """The 256x256x64 rotating-fibre Barkley slab at full size, in the
    autotuned launch configuration the benchmark uses: one step from the
    seeded initial state, checked node by node at sampled nodes."""
    w = wl.barkley_slab()
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    G = _gpu_grid(bbx, w)
    G.write_all(st0)
    G.autotune(w.dt)
    G.step(w.dt, 1)
    got = G.read_all()
    rng = np.random.default_rng(77)
    reg = w.ic_region
    edge = np.zeros_like(reg)
    edge[:, :, 1:] |= reg[:, :, 1:] != reg[:, :, :-1]
    edge[:, 1:, :] |= reg[:, 1:, :] != reg[:, :-1, :]
    edge[1:, :, :] |= reg[1:, :, :] != reg[:-1, :, :]
    cand = np.flatnonzero(edge)
    cells = np.concatenate([rng.choice(cand, min(1500, cand.size), replace=False), rng.integers(0, w.n_cells, 500)])
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
    ref = osim.step_cells(w.dt, cells)
    flat = got.reshape(got.shape[0], -1)
    for v in range(2):
        e = np.abs(flat[v, cells] - ref[:, v]).max() / max(np.abs(ref[:, v]).max(), 1e-30)
        assert e <= 1e-5, (v, e)


def test_host_parity_mirror_through_every_stepping_path(bbx):
    # Single-grid launches of unmasked 3D grids issue their first copies from
    # the parity the host expects; any disagreement with the device would be
    # reported (BBX_ERR_STATE) by the next synchronising call.  Step one grid
    # through every path that moves the parity and compare with a grid that
    # only steps alone.
    w = wl.barkley_slab(70, 30, 10)
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    G = _gpu_grid(bbx, w, 14, 4)
    H = _gpu_grid(bbx, w, 14, 4)
    for X in (G, H):
        X.set_timestep(w.dt)
        X.write_all(st0)
    F = _gpu_grid(bbx, wl.fhn_sheet(40, 20))
    F.set_timestep(0.01)
    G.step(w.dt, 3)
    B = bbx.Batch([G, F])
    B.step(3)
    B.sync()
    G.step(w.dt, 2)
    t, n = G.get_time()
    G.set_time(t, n)
    G.step(w.dt, 1)
    G.read_state(0)
    G.step(w.dt, 1)
    H.step(w.dt, 10)
    got, ref = G.read_all(), H.read_all()
    assert G.get_time()[1] == H.get_time()[1] == 10
    assert _rel_linf(got[0], ref[0], np.ones(w.shape, bool)) < 1e-5
    G.autotune(w.dt)  # leaves the state as it was
    G.step(w.dt, 3)
    H.step(w.dt, 3)
    assert _rel_linf(G.read_all()[0], H.read_all()[0], np.ones(w.shape, bool)) < 1e-5


@pytest.mark.parametrize("nx,masked", [(64, False), (64, True), (70, False)])
def test_exchange_state_is_read_all_then_write_all(bbx, nx, masked):
    # bbx_exchange_state returns the current state while taking a new one
    # (overlapping copies on two streams; one after the other for padded rows)
    w = wl.barkley_slab(nx, 24, 8)
    if masked:
        w.mask, w.fibres = wl.random_geometry(nx, 24, 8, seed=9, tissue_frac=0.8)
    rest = oracle.rest_state(w.model, w.params)
    s0 = w.initial_state(rest).astype(np.float32)
    s1 = (s0 + np.float32(0.01) * np.random.default_rng(3).random(s0.shape, dtype=np.float32)).astype(np.float32)
    G = _gpu_grid(bbx, w, 14, 4)
    H = _gpu_grid(bbx, w, 14, 4)
    G.write_all(s0)
    out = np.empty_like(s0)
    G.exchange_state(s1, out)
    assert np.array_equal(out, s0)
    assert np.array_equal(G.read_all(), s1)
    H.write_all(s1)
    G.step(w.dt, 3)
    H.step(w.dt, 3)
    ref = H.read_all()
    assert np.array_equal(G.read_all(), ref)
    out2 = np.empty_like(s0)
    G.exchange_state(s0, out2)
    assert np.array_equal(out2, ref)
    G.step(w.dt, 2)
    H.write_all(s0)
    H.step(w.dt, 2)
    assert np.array_equal(G.read_all(), H.read_all())


@pytest.mark.parametrize("masked", [False, True])
def test_asynchronous_exchange_pipeline_matches_the_synchronous_one(bbx, masked):
    # a pipeline of exchange-then-step with new inputs every step: the
    # asynchronous exchange (stages on the device, copies on their own
    # streams, no wait until the end) gives every step's output bitwise as the
    # synchronous exchange does; then the state is read back as usual
    import torch
    w = wl.barkley_slab(64, 24, 8)
    if masked:
        w.mask, w.fibres = wl.random_geometry(64, 24, 8, seed=9, tissue_frac=0.8)
    rest = oracle.rest_state(w.model, w.params)
    s0 = w.initial_state(rest).astype(np.float32)
    rng = np.random.default_rng(5)
    ins = [(s0 + np.float32(0.01) * rng.random(s0.shape, dtype=np.float32)).astype(np.float32) for _ in range(5)]
    A = _gpu_grid(bbx, w, 14, 4)
    B = _gpu_grid(bbx, w, 14, 4)
    A.write_all(s0)
    B.write_all(s0)
    pin_in = [torch.from_numpy(x).pin_memory() for x in ins]
    pin_out = [torch.empty(s0.shape, dtype=torch.float32).pin_memory() for _ in ins]
    ref_out = [np.empty_like(s0) for _ in ins]
    for k in range(len(ins)):
        A.exchange_state_async(pin_in[k], pin_out[k])
        A.step(w.dt, 2)
        B.exchange_state(ins[k], ref_out[k])
        B.step(w.dt, 2)
    A.exchange_wait()
    for k in range(len(ins)):
        assert np.array_equal(pin_out[k].numpy(), ref_out[k]), k
    assert np.array_equal(A.read_all(), B.read_all())
    # the same host buffers reused every step (the pattern of a streaming loop)
    for k in range(3):
        A.exchange_state_async(pin_in[k], pin_out[0])
        A.step(w.dt, 1)
        B.exchange_state(ins[k], ref_out[0])
        B.step(w.dt, 1)
    A.exchange_wait()
    assert np.array_equal(pin_out[0].numpy(), ref_out[0])
    assert np.array_equal(A.read_all(), B.read_all())
    # a synchronous exchange after an asynchronous one waits for it first
    prev = A.read_all()
    out = np.empty_like(s0)
    A.exchange_state_async(pin_in[0], pin_out[1])
    A.exchange_state(ins[1], out)
    assert np.array_equal(pin_out[1].numpy(), prev)
    assert np.array_equal(out, ins[0])
    assert np.array_equal(A.read_all(), ins[1])


def test_asynchronous_exchange_refusals(bbx):
    import torch
    w = wl.barkley_slab(70, 24, 8)  # padded rows
    G = _gpu_grid(bbx, w, 14, 4)
    S = 2
    a = torch.zeros((S,) + w.shape, dtype=torch.float32).pin_memory()
    b = torch.zeros((S,) + w.shape, dtype=torch.float32).pin_memory()
    with pytest.raises(bbx.BbxError) as e:
        G.exchange_state_async(a, b)
    assert e.value.code == bbx.BBX_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        G.exchange_state_async(a.double(), b)
    G.exchange_wait()  # nothing pending: returns at once
