"""Host scheduling logic of the library, checked without a GPU through its
host-only test hooks: how a masked 3D grid is cut into pieces (every tissue
chunk in exactly one piece, origins on the 16-byte rule of the mask copy,
z-runs merged), and how column-planes are shared among CTAs (equal shares in
segment order, and the first piece of each CTA given by the closed form the
step kernel uses to issue its first copies before reading the plan)."""
import numpy as np
import pytest

from paper_1605_06015_gb300 import bbx

KTILE, KCHUNK = 64, 16


def _cover(flags, ty, zb, nz):
    return bbx.bbx_debug_cover_chunks(flags, ty, zb, nz)


def _first_pieces(segs, ctas):
    return bbx.bbx_debug_plan_first_pieces(segs, ctas)


@pytest.mark.parametrize("seed", range(6))
def test_every_tissue_chunk_is_in_exactly_one_piece(seed):
    rng = np.random.default_rng(seed)
    ty, zb = int(rng.choice([7, 14])), int(rng.choice([2, 4, 8]))
    nbz, nby, ncx = 7, 5, int(rng.integers(5, 23))
    nz = nbz * zb - int(rng.integers(0, zb))  # a cut last band
    flags = rng.random((nbz, nby, ncx)) < rng.uniform(0.1, 0.6)
    pieces = _cover(flags, ty, zb, nz)
    covered = np.zeros((nbz, nby, ncx), np.int32)
    for x0, y0, z0, z1 in pieces:
        assert x0 % KCHUNK == 0 and y0 % ty == 0 and z0 % zb == 0  # 16-byte rule of the mask copy
        assert 0 <= z0 < z1 <= nz and (z1 % zb == 0 or z1 == nz)
        by, c0 = y0 // ty, x0 // KCHUNK
        assert flags[z0 // zb, by, c0]  # a piece starts at a tissue chunk
        for bz in range(z0 // zb, (z1 - 1) // zb + 1):
            covered[bz, by, c0:c0 + KTILE // KCHUNK] += 1
    assert np.all(covered[flags] == 1)  # every tissue chunk exactly once
    assert covered.max() <= 1  # pieces never overlap


def test_consecutive_bands_with_one_origin_merge_into_one_run():
    flags = np.zeros((6, 1, 8), bool)
    flags[0:4, 0, 3] = True   # one wall crossing a 64-column boundary: one piece at chunk 3 ...
    flags[0:4, 0, 5] = True
    flags[5, 0, 0] = True     # ... and a separate band
    pieces = _cover(flags, 7, 4, 24)
    assert pieces.tolist() == [[0, 0, 20, 24], [48, 0, 0, 16]]


@pytest.mark.parametrize("ncols,nz,ctas", [(76, 64, 304), (296, 64, 304), (10, 7, 304), (40, 256, 152),
                                           (3, 5, 4), (5, 1000, 7)])
def test_first_piece_of_each_cta_has_the_kernels_closed_form(ncols, nz, ctas):
    # unmasked 3D grid: whole columns of nz planes in order (x fastest)
    nbx, ty = 4, 14
    segs = [((c % nbx) * KTILE, (c // nbx) * ty, 0, nz) for c in range(ncols)]
    first, used = _first_pieces(segs, ctas)
    T = ncols * nz
    assert used == min(ctas, T)
    for c in range(used):
        p0, p1 = c * T // used, (c + 1) * T // used
        col, z0 = p0 // nz, p0 % nz
        z1 = min(nz, z0 + (p1 - p0))
        assert first[c].tolist() == [(col % nbx) * KTILE, (col // nbx) * ty, z0, z1], c


def test_first_pieces_start_where_the_equal_shares_say():
    rng = np.random.default_rng(7)
    segs = [(int(rng.integers(0, 8)) * 64, int(rng.integers(0, 9)) * 7, int(a), int(a + b))
            for a, b in zip(rng.integers(0, 30, 50), rng.integers(1, 25, 50))]
    T = sum(s[3] - s[2] for s in segs)
    first, used = _first_pieces(segs, 37)
    # the first pieces start where the equal shares say
    starts = np.cumsum([0] + [s[3] - s[2] for s in segs])
    for c in range(used):
        p0 = c * T // used
        k = int(np.searchsorted(starts, p0, side="right") - 1)
        assert first[c][0] == segs[k][0] and first[c][1] == segs[k][1]
        assert first[c][2] == segs[k][2] + (p0 - starts[k])
