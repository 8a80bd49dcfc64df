"""Thin ctypes binding of the C ABI in include/bbx.h (libbbx.so).

Every function keeps the C name and only marshals arguments: NumPy arrays (or
PyTorch CPU tensors, e.g. pinned buffers) become host pointers, status codes
become ``BbxError``.  All computation happens in the CUDA library; there is no
fallback.  Importing this module fails loudly if libbbx.so has not been built
(``__graft_entry__.build()`` or ``python paper_1605_06015_gb300/build.py``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbbx.so")

BBX_OK = 0
BBX_ERR_ARG = -1
BBX_ERR_CUDA = -2
BBX_ERR_FIBRE = -3
BBX_ERR_UNSTABLE = -4
BBX_ERR_NAN = -5
BBX_ERR_TIMEOUT = -6
BBX_ERR_STATE = -7
BBX_ERR_NOMEM = -8
BBX_ERR_UNSUPPORTED = -9

BBX_FHN, BBX_BARKLEY, BBX_BR, BBX_ZFK, BBX_DIFFUSION, BBX_BR_MRL, BBX_BR_FCA = 1, 2, 3, 4, 5, 6, 7
NVARS = {BBX_FHN: 2, BBX_BARKLEY: 2, BBX_BR: 8, BBX_ZFK: 1, BBX_DIFFUSION: 1, BBX_BR_MRL: 11, BBX_BR_FCA: 11}
BBX_ACT_NONE = 2147483647
BBX_SCHEME_UNSPLIT, BBX_SCHEME_LIE = 0, 1
BBX_SOLVER_EULER, BBX_SOLVER_RK4 = 0, 1
BBX_GATES_FP32, BBX_GATES_FP16, BBX_GATES_UNORM16 = 0, 1, 2


class BbxError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, bbx_status_string(code), code))


class Info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("px", ctypes.c_int),
                ("nvars", ctypes.c_int), ("model", ctypes.c_int), ("masked", ctypes.c_int),
                ("anisotropic", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("tile_z", ctypes.c_int), ("n_bricks", ctypes.c_longlong), ("n_tissue", ctypes.c_longlong),
                ("step", ctypes.c_longlong), ("t", ctypes.c_double), ("wsum_skipped", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libbbx.so is not built (%s): run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, Z, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_longlong
    sig = {
        "bbx_create_grid": [ctypes.POINTER(P), I, I, I, D, P, P],
        "bbx_set_fibres": [P, P, D, D],
        "bbx_set_ionic_model": [P, I, P, I],
        "bbx_write_state": [P, I, P, Z],
        "bbx_write_all": [P, P, Z],
        "bbx_read_all": [P, P, Z],
        "bbx_exchange_state": [P, P, P, Z],
        "bbx_exchange_state_async": [P, P, P, Z],
        "bbx_exchange_wait": [P],
        "bbx_debug_cover_chunks": [P, I, I, I, I, I, I, P, I, P],
        "bbx_debug_plan_first_pieces": [P, I, I, P, I, P],
        "bbx_bind_state": [P, P, P, Z],
        "bbx_set_stimulus": [P, P, D, D, D],
        "bbx_set_threshold": [P, D],
        "bbx_step": [P, D, I],
        "bbx_read_state": [P, I, P, Z],
        "bbx_read_activation": [P, P, Z],
        "bbx_write_activation": [P, P, Z],
        "bbx_total": [P, I, ctypes.POINTER(D)],
        "bbx_step_total": [P, ctypes.POINTER(D)],
        "bbx_get_time": [P, ctypes.POINTER(D), ctypes.POINTER(LL)],
        "bbx_set_time": [P, D, LL],
        "bbx_get_info": [P, ctypes.POINTER(Info)],
        "bbx_read_active_bricks": [P, P, Z, ctypes.POINTER(LL)],
        "bbx_set_tiling": [P, I, I],
        "bbx_autotune": [P, D, ctypes.POINTER(D)],
        "bbx_state_device_ptr": [P, I, ctypes.POINTER(P)],
        "bbx_debug_poison_first_load": [P, I],
        "bbx_clear_device_error": [P],
        "bbx_set_timestep": [P, D],
        "bbx_set_scheme": [P, I],
        "bbx_set_solver": [P, I],
        "bbx_set_resident": [P, I],
        "bbx_set_tabulation": [P, I],
        "bbx_set_wsum_elision": [P, I],
        "bbx_ppm_frame": [P, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D), P],
        "bbx_phase_singularities": [P, I, D, I, D, P, I, ctypes.POINTER(I)],
        "bbx_batch_create": [ctypes.POINTER(P), ctypes.POINTER(P), I],
        "bbx_batch_step": [P, I],
        "bbx_batch_sync": [P],
        "bbx_batch_autotune": [P, ctypes.POINTER(D)],
        "bbx_batch_info": [P, ctypes.POINTER(I), ctypes.POINTER(I), I],
        "bbx_debug_expm1": [P, P, P, I, P],
        "bbx_set_gate_storage": [P, I],
        "bbx_set_halo_planes": [P, I, I],
        "bbx_halo_exchange": [P, P],
        "bbx_halo_plane": [P, I, I, ctypes.POINTER(P), ctypes.POINTER(Z)],
        "bbx_total_noalloc": [P, P, I, I, I, I, P, P],
        "bbx_mlp_create": [ctypes.POINTER(P), ctypes.c_ulonglong, P],
        "bbx_mlp_set_params": [P, P, Z],
        "bbx_mlp_get_params": [P, P, Z],
        "bbx_mlp_set_normalization": [P, P, Z],
        "bbx_mlp_get_normalization": [P, P, Z],
        "bbx_mlp_fit_normalization": [P, P, P, LL],
        "bbx_mlp_gradients": [P, P, P, I, P, Z, ctypes.POINTER(D)],
        "bbx_mlp_train": [P, P, P, LL, I, I, D, ctypes.c_ulonglong, ctypes.POINTER(D)],
        "bbx_sample_reaction_pairs": [P, LL, ctypes.c_ulonglong, P, P],
        "bbx_set_surrogate": [P, P, D],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = I
    L.bbx_destroy_grid.argtypes = [P]
    L.bbx_destroy_grid.restype = None
    L.bbx_batch_destroy.argtypes = [P]
    L.bbx_batch_destroy.restype = None
    L.bbx_mlp_destroy.argtypes = [P]
    L.bbx_mlp_destroy.restype = None
    L.bbx_status_string.argtypes = [I]
    L.bbx_status_string.restype = ctypes.c_char_p
    return L


_lib = _load()


def lib():
    return _lib


def _check(rc, where):
    if rc != BBX_OK:
        raise BbxError(rc, where)


def _hostptr(a, dtype, n):
    """Host pointer of a contiguous NumPy array or CPU torch tensor of n
    elements of dtype; returns (pointer, keep-alive object)."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if a.is_cuda or not a.is_contiguous() or a.numel() != n:
            raise ValueError("expected a contiguous CPU tensor of %d elements" % n)
        if a.element_size() != np.dtype(dtype).itemsize:
            raise ValueError("dtype mismatch")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype).reshape(-1)
    if arr.size != n:
        raise ValueError("expected %d elements, got %d" % (n, arr.size))
    return arr.ctypes.data, arr


def _stream_handle(stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def bbx_status_string(code):
    return _lib.bbx_status_string(int(code)).decode()


_shapes = {}  # grid handle -> (n, (nz, ny, nx)), filled at creation


def bbx_create_grid(nx, ny, nz, h, mask=None, stream=None):
    g = ctypes.c_void_p()
    n = nx * ny * nz
    mp, keep = _hostptr(None if mask is None else (np.asarray(mask) != 0), np.uint8, n)
    _check(_lib.bbx_create_grid(ctypes.byref(g), int(nx), int(ny), int(nz), float(h), mp,
                                _stream_handle(stream)), "bbx_create_grid")
    _shapes[g.value] = (n, (nz, ny, nx))
    return g


def bbx_destroy_grid(g):
    _shapes.pop(getattr(g, "value", g), None)
    _lib.bbx_destroy_grid(g)


def bbx_get_info(g):
    inf = Info()
    _check(_lib.bbx_get_info(g, ctypes.byref(inf)), "bbx_get_info")
    return {f: getattr(inf, f) for f, _ in Info._fields_}


def _ncell(g):
    key = getattr(g, "value", g)
    if key in _shapes:
        return _shapes[key]
    i = bbx_get_info(g)
    return i["nx"] * i["ny"] * i["nz"], (i["nz"], i["ny"], i["nx"])


def bbx_set_fibres(g, fibres, D_par, D_perp):
    n, _ = _ncell(g)
    fp, keep = _hostptr(fibres, np.float32, 3 * n)
    _check(_lib.bbx_set_fibres(g, fp, float(D_par), float(D_perp)), "bbx_set_fibres")


def bbx_set_ionic_model(g, model, params=None):
    p = np.zeros(0) if params is None else np.ascontiguousarray(params, dtype=np.float64)
    _check(_lib.bbx_set_ionic_model(g, int(model), p.ctypes.data if p.size else None, p.size),
           "bbx_set_ionic_model")


def bbx_write_state(g, var, values):
    n, _ = _ncell(g)
    vp, keep = _hostptr(values, np.float32, n)
    _check(_lib.bbx_write_state(g, int(var), vp, n), "bbx_write_state")


def bbx_write_all(g, state):
    """All variables at once: state [nvars][nz][ny][nx] float32 (NumPy or a
    CPU torch tensor, pinned or not)."""
    n, _ = _ncell(g)
    S = bbx_get_info(g)["nvars"]
    vp, keep = _hostptr(state, np.float32, S * n)
    _check(_lib.bbx_write_all(g, vp, S * n), "bbx_write_all")


def bbx_read_all(g, out=None):
    """All variables at once into out [nvars][nz][ny][nx] float32 (new
    NumPy array if None)."""
    n, shape = _ncell(g)
    S = bbx_get_info(g)["nvars"]
    if out is None:
        out = np.empty((S,) + tuple(shape), dtype=np.float32)
    op, keep = _hostptr(out, np.float32, S * n)
    if isinstance(keep, np.ndarray) and keep is not out and not np.shares_memory(keep, out):
        raise ValueError("out must be a contiguous float32 array")
    _check(_lib.bbx_read_all(g, op, S * n), "bbx_read_all")
    return out


def bbx_exchange_state(g, state_in, out):
    """out <- the current state, state_in -> the new state, both
    [nvars][nz][ny][nx] float32, the copies overlapping (pinned CPU tensors or
    arrays)."""
    n, _ = _ncell(g)
    S = bbx_get_info(g)["nvars"]
    ip, keep_in = _hostptr(state_in, np.float32, S * n)
    op, keep_out = _hostptr(out, np.float32, S * n)
    if isinstance(keep_out, np.ndarray) and keep_out is not out and not np.shares_memory(keep_out, out):
        raise ValueError("out must be a contiguous float32 array")
    _check(_lib.bbx_exchange_state(g, ip, op, S * n), "bbx_exchange_state")
    return out


def _pinned_ptr(a):
    """(host pointer, elements) of a contiguous float32 buffer that the caller
    keeps alive (a pinned CPU tensor or a NumPy array); no copies."""
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if a.is_cuda or not a.is_contiguous() or a.element_size() != 4 or a.is_floating_point() is False:
            raise ValueError("expected a contiguous float32 CPU tensor")
        return a.data_ptr(), a.numel()
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
        raise ValueError("expected a contiguous float32 array")
    return a.ctypes.data, a.size


def bbx_exchange_state_async(g, state_in, out):
    """Enqueue out <- the current state and state_in -> the new state without
    waiting; both must be contiguous float32 buffers of nvars x nz x ny x nx
    elements (pinned CPU tensors for the copies to overlap) that stay alive
    and untouched until bbx_exchange_wait.  Makes no synchronising call (the
    library checks the element count against the grid)."""
    ip, ni = _pinned_ptr(state_in)
    op, no = _pinned_ptr(out)
    if ni != no:
        raise ValueError("state_in and out differ in size")
    _check(_lib.bbx_exchange_state_async(g, ip, op, ni), "bbx_exchange_state_async")
    return out


def bbx_exchange_wait(g):
    """Wait for the grid's asynchronous exchanges to finish with their host buffers."""
    _check(_lib.bbx_exchange_wait(g), "bbx_exchange_wait")


def bbx_debug_cover_chunks(flags, ty, zb, nz):
    """Host-only hook: the pieces (x0, y0, z0, z1) a masked 3D grid is cut
    into, from its chunk flags [nbz][nby][ncx] (no GPU needed)."""
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    nbz, nby, ncx = f.shape
    cap = nbz * nby * ncx + 1
    out = np.zeros(4 * cap, np.int32)
    cnt = ctypes.c_int(0)
    _check(_lib.bbx_debug_cover_chunks(f.ctypes.data, ncx, nby, nbz, int(ty), int(zb), int(nz), out.ctypes.data,
                                       cap, ctypes.byref(cnt)), "bbx_debug_cover_chunks")
    return out[: 4 * cnt.value].reshape(-1, 4)


def bbx_debug_plan_first_pieces(segs, ctas):
    """Host-only hook: the first piece of each CTA when the segments
    (x0, y0, z0, z1) are shared among ctas CTAs; returns (pieces, CTAs used)."""
    s = np.ascontiguousarray(np.asarray(segs, dtype=np.int32).reshape(-1))
    out = np.zeros(4 * int(ctas), np.int32)
    used = ctypes.c_int(0)
    _check(_lib.bbx_debug_plan_first_pieces(s.ctypes.data, s.size // 4, int(ctas), out.ctypes.data, int(ctas),
                                            ctypes.byref(used)), "bbx_debug_plan_first_pieces")
    return out[: 4 * used.value].reshape(-1, 4), used.value


def bbx_bind_state(g, dev_a, dev_b, nbytes=None):
    """dev_a, dev_b: CUDA torch tensors (or raw device pointers with nbytes)."""
    if hasattr(dev_a, "data_ptr"):
        nbytes = min(dev_a.numel() * dev_a.element_size(), dev_b.numel() * dev_b.element_size())
        dev_a, dev_b = dev_a.data_ptr(), dev_b.data_ptr()
    _check(_lib.bbx_bind_state(g, dev_a, dev_b, int(nbytes)), "bbx_bind_state")


def bbx_set_stimulus(g, region, amp, t_on, t_off):
    n, _ = _ncell(g)
    rp, keep = _hostptr(None if region is None else (np.asarray(region) != 0), np.uint8, n)
    _check(_lib.bbx_set_stimulus(g, rp, float(amp), float(t_on), float(t_off)), "bbx_set_stimulus")


def bbx_set_threshold(g, theta):
    _check(_lib.bbx_set_threshold(g, float(theta)), "bbx_set_threshold")


def bbx_step(g, dt, n_steps=1):
    _check(_lib.bbx_step(g, float(dt), int(n_steps)), "bbx_step")


def bbx_read_state(g, var, out=None):
    n, shape = _ncell(g)
    if out is None:
        out = np.empty(shape, dtype=np.float32)
    op, keep = _hostptr(out, np.float32, n)
    if isinstance(keep, np.ndarray) and keep is not out and not np.shares_memory(keep, out):
        raise ValueError("out must be a contiguous float32 array")
    _check(_lib.bbx_read_state(g, int(var), op, n), "bbx_read_state")
    return out


def bbx_read_activation(g, out=None):
    n, shape = _ncell(g)
    if out is None:
        out = np.empty(shape, dtype=np.int32)
    _check(_lib.bbx_read_activation(g, out.ctypes.data, n), "bbx_read_activation")
    return out


def bbx_write_activation(g, act):
    n, _ = _ncell(g)
    ap, keep = _hostptr(act, np.int32, n)
    _check(_lib.bbx_write_activation(g, ap, n), "bbx_write_activation")


def bbx_total(g, var=0):
    out = ctypes.c_double()
    _check(_lib.bbx_total(g, int(var), ctypes.byref(out)), "bbx_total")
    return out.value


def bbx_ppm_frame(g, layers, lo, hi, out_dev):
    """out_dev: a device uint8 tensor of 3*nx*ny*nz bytes (filled on the grid's stream)."""
    ly = (ctypes.c_int * 3)(*[int(v) for v in layers])
    l3 = (ctypes.c_double * 3)(*[float(v) for v in lo])
    h3 = (ctypes.c_double * 3)(*[float(v) for v in hi])
    _check(_lib.bbx_ppm_frame(g, ly, l3, h3, _devptr(out_dev)), "bbx_ppm_frame")


def bbx_phase_singularities(g, var_a, iso_a, var_b, iso_b, xyz_dev, max_points):
    """Fills xyz_dev (a device float32 tensor of 3*max_points) and returns the
    number of points found."""
    n = ctypes.c_int()
    _check(_lib.bbx_phase_singularities(g, int(var_a), float(iso_a), int(var_b), float(iso_b), _devptr(xyz_dev),
                                        int(max_points), ctypes.byref(n)), "bbx_phase_singularities")
    return n.value


def bbx_step_total(g):
    out = ctypes.c_double()
    _check(_lib.bbx_step_total(g, ctypes.byref(out)), "bbx_step_total")
    return out.value


def bbx_get_time(g):
    t, n = ctypes.c_double(), ctypes.c_longlong()
    _check(_lib.bbx_get_time(g, ctypes.byref(t), ctypes.byref(n)), "bbx_get_time")
    return t.value, n.value


def bbx_set_time(g, t, step):
    _check(_lib.bbx_set_time(g, float(t), int(step)), "bbx_set_time")


def bbx_read_active_bricks(g):
    cnt = ctypes.c_longlong()
    rc = _lib.bbx_read_active_bricks(g, None, 0, ctypes.byref(cnt))
    if rc not in (BBX_OK, BBX_ERR_ARG):
        _check(rc, "bbx_read_active_bricks")
    out = np.zeros(max(cnt.value, 1), dtype=np.int32)
    _check(_lib.bbx_read_active_bricks(g, out.ctypes.data, out.size, ctypes.byref(cnt)),
           "bbx_read_active_bricks")
    return out[:cnt.value].copy()


def bbx_set_tiling(g, tile_y, tile_z):
    _check(_lib.bbx_set_tiling(g, int(tile_y), int(tile_z)), "bbx_set_tiling")


def bbx_autotune(g, dt):
    ms = ctypes.c_double()
    _check(_lib.bbx_autotune(g, float(dt), ctypes.byref(ms)), "bbx_autotune")
    return ms.value


def bbx_state_device_ptr(g, var):
    p = ctypes.c_void_p()
    _check(_lib.bbx_state_device_ptr(g, int(var), ctypes.byref(p)), "bbx_state_device_ptr")
    return p.value


def bbx_debug_poison_first_load(g, on):
    _check(_lib.bbx_debug_poison_first_load(g, int(bool(on))), "bbx_debug_poison_first_load")


def bbx_clear_device_error(g):
    _check(_lib.bbx_clear_device_error(g), "bbx_clear_device_error")


def bbx_set_scheme(g, scheme):
    _check(_lib.bbx_set_scheme(g, int(scheme)), "bbx_set_scheme")


def bbx_set_solver(g, solver):
    _check(_lib.bbx_set_solver(g, int(solver)), "bbx_set_solver")


def bbx_set_tabulation(g, on=True):
    _check(_lib.bbx_set_tabulation(g, int(bool(on))), "bbx_set_tabulation")


def bbx_set_wsum_elision(g, on=True):
    _check(_lib.bbx_set_wsum_elision(g, int(bool(on))), "bbx_set_wsum_elision")


def bbx_set_resident(g, on=True):
    _check(_lib.bbx_set_resident(g, int(bool(on))), "bbx_set_resident")


def bbx_set_timestep(g, dt):
    _check(_lib.bbx_set_timestep(g, float(dt)), "bbx_set_timestep")


def bbx_batch_create(grids):
    """grids: sequence of grid handles (or Grid objects)."""
    hs = [getattr(x, "g", x) for x in grids]
    arr = (ctypes.c_void_p * len(hs))(*[h.value if hasattr(h, "value") else h for h in hs])
    b = ctypes.c_void_p()
    _check(_lib.bbx_batch_create(ctypes.byref(b), arr, len(hs)), "bbx_batch_create")
    return b


def bbx_batch_step(b, n_steps=1):
    _check(_lib.bbx_batch_step(b, int(n_steps)), "bbx_batch_step")


def bbx_batch_sync(b):
    _check(_lib.bbx_batch_sync(b), "bbx_batch_sync")


def bbx_batch_autotune(b):
    ms = ctypes.c_double()
    _check(_lib.bbx_batch_autotune(b, ctypes.byref(ms)), "bbx_batch_autotune")
    return ms.value


def bbx_batch_info(b):
    n = ctypes.c_int()
    tys = (ctypes.c_int * 64)()
    _check(_lib.bbx_batch_info(b, ctypes.byref(n), tys, 64), "bbx_batch_info")
    return {"n_groups": n.value, "tile_y": list(tys[:min(n.value, 64)])}


def bbx_batch_destroy(b):
    _lib.bbx_batch_destroy(b)


def bbx_debug_expm1(x_dev, out_dev, ref_dev, stream=None):
    """The kernels' e^x - 1 and CUDA's expm1f of device tensors (test hook)."""
    _check(_lib.bbx_debug_expm1(_devptr(x_dev), _devptr(out_dev), _devptr(ref_dev), int(x_dev.numel()),
                                _stream_handle(stream)), "bbx_debug_expm1")


def bbx_set_gate_storage(g, mode):
    _check(_lib.bbx_set_gate_storage(g, int(mode)), "bbx_set_gate_storage")


def bbx_set_halo_planes(g, lo, hi):
    _check(_lib.bbx_set_halo_planes(g, int(lo), int(hi)), "bbx_set_halo_planes")


def bbx_halo_exchange(lower, upper):
    _check(_lib.bbx_halo_exchange(lower, upper), "bbx_halo_exchange")


def bbx_halo_plane(g, side, halo):
    """(device address, bytes) of one V plane of the buffer the next step reads."""
    p = ctypes.c_void_p()
    n = ctypes.c_size_t()
    _check(_lib.bbx_halo_plane(g, int(side), int(halo), ctypes.byref(p), ctypes.byref(n)), "bbx_halo_plane")
    return p.value, n.value


def bbx_total_noalloc(field_dev, mask_dev, nx, ny, nz, pitch, out_dev, stream=None):
    """Device pointers in, one double written to out_dev on the stream; the
    library allocates nothing (see include/bbx.h)."""
    _check(_lib.bbx_total_noalloc(field_dev, mask_dev, int(nx), int(ny), int(nz), int(pitch), out_dev,
                                  _stream_handle(stream)), "bbx_total_noalloc")


MLP_PARAMS = 8 * 64 + 64 + 64 * 64 + 64 + 64 * 8 + 8
MLP_NORM = 48


def _devptr(t):
    return t.data_ptr() if hasattr(t, "data_ptr") else t


def bbx_mlp_create(seed=1, stream=None):
    m = ctypes.c_void_p()
    _check(_lib.bbx_mlp_create(ctypes.byref(m), int(seed), _stream_handle(stream)), "bbx_mlp_create")
    return m


def bbx_mlp_destroy(m):
    _lib.bbx_mlp_destroy(m)


def bbx_mlp_set_params(m, params):
    p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
    _check(_lib.bbx_mlp_set_params(m, p.ctypes.data, p.size), "bbx_mlp_set_params")


def bbx_mlp_get_params(m):
    p = np.empty(MLP_PARAMS, dtype=np.float32)
    _check(_lib.bbx_mlp_get_params(m, p.ctypes.data, p.size), "bbx_mlp_get_params")
    return p


def bbx_mlp_set_normalization(m, norm):
    p = np.ascontiguousarray(norm, dtype=np.float32).reshape(-1)
    _check(_lib.bbx_mlp_set_normalization(m, p.ctypes.data, p.size), "bbx_mlp_set_normalization")


def bbx_mlp_get_normalization(m):
    p = np.empty(MLP_NORM, dtype=np.float32)
    _check(_lib.bbx_mlp_get_normalization(m, p.ctypes.data, p.size), "bbx_mlp_get_normalization")
    return p


def bbx_mlp_fit_normalization(m, x_dev, t_dev, n):
    _check(_lib.bbx_mlp_fit_normalization(m, _devptr(x_dev), _devptr(t_dev), int(n)), "bbx_mlp_fit_normalization")


def bbx_mlp_gradients(m, x_dev, t_dev, batch):
    g = np.empty(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _check(_lib.bbx_mlp_gradients(m, _devptr(x_dev), _devptr(t_dev), int(batch), g.ctypes.data, g.size,
                                  ctypes.byref(loss)), "bbx_mlp_gradients")
    return g, loss.value


def bbx_mlp_train(m, x_dev, t_dev, n, batch, steps, lr, seed=1):
    loss = ctypes.c_double()
    _check(_lib.bbx_mlp_train(m, _devptr(x_dev), _devptr(t_dev), int(n), int(batch), int(steps), float(lr),
                              int(seed), ctypes.byref(loss)), "bbx_mlp_train")
    return loss.value


def bbx_set_surrogate(g, m, v_upstroke=-60.0):
    _check(_lib.bbx_set_surrogate(g, m, float(v_upstroke)), "bbx_set_surrogate")


def bbx_sample_reaction_pairs(g, n, seed, x_dev, t_dev):
    _check(_lib.bbx_sample_reaction_pairs(g, int(n), int(seed), _devptr(x_dev), _devptr(t_dev)),
           "bbx_sample_reaction_pairs")


class Batch:
    """Owner of a batch handle; keeps its member Grid objects alive."""

    def __init__(self, grids):
        self.grids = list(grids)
        self.b = bbx_batch_create(self.grids)

    def step(self, n_steps=1):
        bbx_batch_step(self.b, n_steps)

    def sync(self):
        bbx_batch_sync(self.b)

    def autotune(self):
        return bbx_batch_autotune(self.b)

    def info(self):
        return bbx_batch_info(self.b)

    def close(self):
        if self.b:
            bbx_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    """Convenience owner of a grid handle (destroyed with the object)."""

    def __init__(self, nx, ny, nz, h, mask=None, stream=None):
        self.shape = (nz, ny, nx)
        self.h = h
        self.g = bbx_create_grid(nx, ny, nz, h, mask, stream)

    def close(self):
        if self.g:
            bbx_destroy_grid(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __getattr__(self, name):
        fn = globals().get("bbx_" + name)
        if fn is None or not callable(fn):
            raise AttributeError(name)
        return lambda *a, **k: fn(self.g, *a, **k)

    def read_all(self, out=None):
        return bbx_read_all(self.g, out)

    def write_all(self, state):
        bbx_write_all(self.g, state)
