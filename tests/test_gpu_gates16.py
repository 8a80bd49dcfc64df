"""Beeler-Reuter gates stored in 16 bits (bbx_set_gate_storage): the step's
arithmetic is the FP32 kernel's, rounded when the gates are stored; with the
16-bit fixed-point encoding the step keeps the parity bars against the FP64
oracle (rel L-inf V <= 1e-4 after 100 steps, activation within one step
over the full quarter-scale shell run); the settings that have no 16-bit
kernel are refused."""
import os

import numpy as np
import pytest

import oracle
from paper_1605_06015_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx
    oracle.set_threads(os.cpu_count() or 1)
    yield torch, bbx
    oracle.set_threads(1)


def _grid(bbx, w, gates, tile=(14, 4)):
    G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask)
    G.set_fibres(w.fibres, w.D_par, w.D_perp)
    G.set_tiling(*tile)
    G.set_ionic_model(w.model, w.params)
    G.set_threshold(w.theta)
    if gates:
        G.set_gate_storage(gates)
    return G


def _q16(y, gates, bbx):
    """Host rounding of float32 gate values to the 16-bit encoding and back."""
    y = np.asarray(y, np.float32)
    if gates == bbx.BBX_GATES_FP16:
        return y.astype(np.float16).astype(np.float32)
    u = np.rint(np.clip(y, 0, 1).astype(np.float32) * np.float32(65535.0))
    return (u.astype(np.float32) * np.float32(1.0 / 65535.0)).astype(np.float32)


@pytest.mark.parametrize("gates", [1, 2])
def test_16bit_step_is_the_fp32_step_rounded(env, gates):
    torch, bbx = env
    w = wl.br_slab(72, 20, 10)
    rest = oracle.rest_state(w.model, w.params)
    st = w.initial_state(rest).astype(np.float32)
    # a state with a front in it, gates exactly representable in 16 bits
    A = _grid(bbx, w, 0)
    A.write_all(st)
    A.step(w.dt, 40)
    st = A.read_all()
    st[2:] = _q16(st[2:], gates, bbx)
    A.write_all(st)
    B = _grid(bbx, w, gates)
    B.write_all(st)
    assert np.array_equal(B.read_all(), st)  # storage round trip
    A.step(w.dt, 1)
    B.step(w.dt, 1)
    a, b = A.read_all(), B.read_all()
    assert np.array_equal(a[:2], b[:2])  # V, Ca: same FP32 arithmetic
    assert np.array_equal(_q16(a[2:], gates, bbx), b[2:])  # gates: FP32 results, rounded when stored
    assert A.step_total() == pytest.approx(B.step_total(), rel=1e-12)
    A.close()
    B.close()


@pytest.mark.parametrize("kind", ["slab", "shell"])
def test_unorm16_gates_100_steps_against_the_oracle(env, kind):
    torch, bbx = env
    if kind == "slab":
        w, tile = wl.br_slab(72, 20, 10), (14, 5)
    else:
        w, tile = wl.br_shell(64), (7, 4)
    n = 100
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    G = _grid(bbx, w, bbx.BBX_GATES_UNORM16, tile)
    G.write_all(st0)
    G.step(w.dt, n)
    og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    osim = oracle.Sim(og, w.model, par=w.params, theta=w.theta, state=st0.astype(np.float64))
    osim.step(w.dt, n)
    got = G.read_all()
    tis = og.psi
    # V within the parity bar.  Each stored gate is rounded to the nearest of
    # 65536 levels every step and the Rush-Larsen map y -> A y + B (0 < A <= 1)
    # does not grow an error, so after n steps a gate is off by at most n half
    # steps (slow gates such as x1 move by fewer than a few levels per step).
    # Ca follows I_s = g_s d f (V - E_s), with the resting d (3e-3) stored in
    # steps of 5e-3 of its value: within 1e-2 of the largest Ca.
    for v in range(8):
        err = np.abs(got[v][tis] - osim.state[v][tis]).max()
        if v >= 2:
            assert err <= n * 0.5 / 65535 + 1e-6, (v, err)
            continue
        e = err / max(np.abs(osim.state[v][tis]).max(), 1e-30)
        assert e <= (1e-4 if v == 0 else 1e-2), (v, e)
    ag, ao = G.read_activation().astype(np.int64), osim.act.astype(np.int64)
    ag[ag == oracle.INT32_MAX] = n + 1
    ao[ao == oracle.INT32_MAX] = n + 1
    assert np.abs(ag - ao)[tis].max() <= 1
    G.close()


@pytest.mark.parametrize("mode", ["tab", "lie"])
def test_unorm16_gates_with_tabulation_or_lie_scheme(env, mode):
    # the 16-bit variants of the general kernels: against the FP32 kernel in
    # the same mode (the oracle comparison of those modes is in
    # test_gpu_tabulation.py and test_gpu_parity.py)
    torch, bbx = env
    w = wl.br_slab(72, 20, 10)
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    out = []
    for gates in (0, bbx.BBX_GATES_UNORM16):
        G = _grid(bbx, w, 0, (14, 5))
        if mode == "tab":
            G.set_tabulation(1)
        else:
            G.set_scheme(bbx.BBX_SCHEME_LIE)
        if gates:
            G.set_gate_storage(gates)
        G.write_all(st0)
        G.step(w.dt, 100)
        out.append(G.read_all())
        G.close()
    e = np.abs(out[0][0] - out[1][0]).max() / np.abs(out[0][0]).max()
    assert e <= 1e-4, e


def test_unorm16_gates_quarter_shell_full_run_activation(env):
    torch, bbx = env
    gold = np.load(os.path.join(GOLDEN, "br_shell_128_activation.npz"))
    w = wl.br_shell(128)
    n = int(gold["n_steps"])
    tis = w.mask.reshape(-1) != 0
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32)
    G = _grid(bbx, w, bbx.BBX_GATES_UNORM16, (7, 4))
    G.write_all(st0)
    G.step(w.dt, n)
    ag = G.read_activation().reshape(-1)[tis].astype(np.int64)
    ao = gold["act"].astype(np.int64)
    ag[ag == oracle.INT32_MAX] = n + 1
    ao[ao == oracle.INT32_MAX] = n + 1
    d = np.abs(ag - ao)
    assert d.max() <= 1, (d.max(), int((d > 1).sum()))
    G.close()


def test_gate_storage_settings(env):
    torch, bbx = env
    w = wl.br_slab(64, 14, 6)
    G = _grid(bbx, w, 0, (14, 4))
    st = G.read_all()
    G.set_gate_storage(bbx.BBX_GATES_UNORM16)
    assert G.get_info()["tile_y"] == 14
    with pytest.raises(bbx.BbxError):
        G.set_tiling(28, 4)  # 28-row tiles have no 16-bit kernel
    assert G.get_info()["tile_y"] == 14
    frame = torch.empty(3 * w.nx * w.ny * w.nz, dtype=torch.uint8, device="cuda")
    for call in (lambda: G.total(3), lambda: G.ppm_frame([2, -1, -1], [0, 0, 0], [1, 1, 1], frame)):
        with pytest.raises(bbx.BbxError) as e:
            call()
        assert e.value.code == bbx.BBX_ERR_UNSUPPORTED
    assert G.total(0) == pytest.approx(float(st[0].astype(np.float64).sum()), rel=1e-12)
    back = G.read_all()
    assert np.array_equal(back[:2], st[:2]) and np.abs(back[2:] - st[2:]).max() <= 0.5 / 65535 + 1e-7
    G.set_gate_storage(bbx.BBX_GATES_FP32)  # and back: the 16-bit values, now in 32 bits
    assert np.array_equal(G.read_all(), back)
    F = _grid(bbx, wl.fhn_sheet(64, 32), 0, (14, 1))
    with pytest.raises(bbx.BbxError) as e:
        F.set_gate_storage(bbx.BBX_GATES_FP16)
    assert e.value.code == bbx.BBX_ERR_UNSUPPORTED
    G.close()
    F.close()
