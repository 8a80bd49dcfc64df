"""z-slab decomposition of one grid (section "Domain partitioning").

The paper's parallel layer cuts the grid into subdomains, one per process,
each surrounded by exchange buffers one node deep that are refreshed from
the neighbours before every step (figure domdec).  Only the transmembrane
voltage diffuses, so only its layer is exchanged.  Here the cut is along z:
part i owns the global planes [z0, z1) and keeps one halo plane below and
above wherever it has a neighbour part; its bbx grid holds those planes with
their mask and fibres (bbx_set_halo_planes), and before each step the halo
planes receive the neighbours' boundary planes of V:

  - on one device, between the grids themselves (bbx_halo_exchange);
  - across ranks, by point-to-point sends and receives of torch.distributed
    (NCCL on GPUs), straight into the halo plane: the state lives in torch
    buffers bound to the grid, so a plane is a view of one of them.

The arithmetic of every node is the same as in the undivided grid (the
stencil reads the same neighbours, the halo planes carry the same values),
so the parts' own planes reproduce the undivided grid's step.
"""
from __future__ import annotations


def slab_bounds(nz: int, parts: int, i: int):
    """Global planes [z0, z1) owned by part i of `parts` (sizes differ by at
    most one plane)."""
    if not (0 <= i < parts) or parts > nz:
        raise ValueError("part %d of %d for %d planes" % (i, parts, nz))
    return i * nz // parts, (i + 1) * nz // parts


def local_bounds(nz: int, parts: int, i: int):
    """(a, b, lo, hi): part i's grid holds the global planes [a, b); lo, hi
    (0 or 1) are its halo planes below and above."""
    z0, z1 = slab_bounds(nz, parts, i)
    lo = 1 if i > 0 else 0
    hi = 1 if i < parts - 1 else 0
    return z0 - lo, z1 + hi, lo, hi


def exchange(dist, rank: int, world: int, send_lo, send_hi, recv_lo, recv_hi):
    """One halo exchange between ranks holding consecutive slabs: rank r sends
    its lowest own plane to r - 1 and its highest to r + 1, and receives their
    boundary planes into its halo planes (tensors; the ones without a
    neighbour may be None)."""
    reqs = []
    if rank > 0:
        reqs.append(dist.isend(send_lo, rank - 1))
        reqs.append(dist.irecv(recv_lo, rank - 1))
    if rank < world - 1:
        reqs.append(dist.isend(send_hi, rank + 1))
        reqs.append(dist.irecv(recv_hi, rank + 1))
    for r in reqs:
        r.wait()


class SlabGrid:
    """Part i of a grid cut into `parts` z-slabs: a bbx grid of the part's
    planes and halo planes, its state in two torch buffers bound to it.

    w: the global workload (shape, spacing, mask, fibres, model); the part
    takes its planes of the mask and fibres."""

    def __init__(self, w, parts: int, i: int, stream=None, device=None):
        import torch
        from . import bbx
        self.w, self.parts, self.i = w, parts, i
        self.a, self.b, self.lo, self.hi = local_bounds(w.nz, parts, i)
        self.nz = self.b - self.a
        mask = None if w.mask is None else w.mask[self.a:self.b]
        G = bbx.Grid(w.nx, w.ny, self.nz, w.h, mask, stream=stream)
        G.set_fibres(None if w.fibres is None else w.fibres[self.a:self.b], w.D_par,
                     w.D_perp if w.fibres is not None else w.D_par)
        G.set_ionic_model(w.model, w.params)
        G.set_threshold(w.theta)
        G.set_halo_planes(self.lo, self.hi)
        info = G.get_info()
        self.S, self.px = info["nvars"], info["px"]
        self.plane = self.px * w.ny
        n = self.S * self.plane * self.nz
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.bufs = [torch.zeros(n, dtype=torch.float32, device=dev) for _ in range(2)]
        G.bind_state(self.bufs[0], self.bufs[1])
        self.G = G

    def write_global_state(self, st):
        """Write this part's planes (halo planes included) of a global state
        [S][nz][ny][nx]."""
        import numpy as np
        self.G.write_all(np.ascontiguousarray(st[:, self.a:self.b]))

    def own(self, local):
        """The part's own planes of a local array [..., nz_local, ny, nx]."""
        return local[..., self.lo:self.nz - self.hi, :, :]

    def _view(self, side, halo):
        from . import bbx
        ptr, nbytes = bbx.bbx_halo_plane(self.G.g, side, halo)
        for buf in self.bufs:
            off = ptr - buf.data_ptr()
            if 0 <= off < buf.numel() * 4:
                return buf[off // 4: off // 4 + nbytes // 4]
        raise RuntimeError("halo plane outside the bound buffers")

    def exchange(self, dist, rank: int, world: int):
        """Halo exchange with the ranks holding the neighbouring parts."""
        send_lo = self._view(0, 0) if self.lo else None
        recv_lo = self._view(0, 1) if self.lo else None
        send_hi = self._view(1, 0) if self.hi else None
        recv_hi = self._view(1, 1) if self.hi else None
        exchange(dist, rank, world, send_lo, send_hi, recv_lo, recv_hi)

    def close(self):
        self.G.close()


def step_on_one_device(grids, dt: float, n_steps: int):
    """n_steps steps of the parts of one grid held on one device (bbx grids
    in z order, consecutive ones sharing a face): each step refreshes every
    halo plane, then steps every part."""
    from . import bbx
    for _ in range(n_steps):
        for lower, upper in zip(grids[:-1], grids[1:]):
            bbx.bbx_halo_exchange(lower.g, upper.g)
        for g in grids:
            g.step(dt, 1)
