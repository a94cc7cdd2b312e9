"""CPU check of the index ranges of the second tensor-core kernel
(paper_2208_08903_gb300/csrc/gf_flow_tc.cu; no GPU), for every shape the
kernel takes: the geometry of its shared-memory plan (positions per channel
group npos, tiles of 96 outputs, the overlapping core matrices of 8 rows
placed 6 positions apart), the A-operand reads of every tile, tap and K-step
(width 8: two taps per K-step, the second at the LBO distance), the x
neighbours the epilogue takes from rows +-1, and the h2 stores.

* every read of a tile stays inside the npos positions of its channel group;
* the rows that store (rows 1..6 of every 8, on interior positions) cover
  every site of the lattice exactly once per layer;
* an output row's x neighbours are rows of the same 8 (the width-8 shuffles).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2208_08903_gb300 import _abi


def plan(nd, L):
    """The kernel's geometry (tc_plan): P, p_first, tiles, npos."""
    P = L + 2
    p_first = 1 + P + (P * P if nd == 3 else 0)
    p_last = p_first * L
    nt = (p_last - p_first + 1 + 95) // 96
    npos = (2 * p_first + nt * 96 + 7) & ~7
    return P, p_first, nt, npos


def taps(nd, P, c):
    """(first position offset, K-direction offset of the second half or None)
    of each K-step's A operand; offsets relative to the tile's first row."""
    PP = P * P
    shift = lambda dz, dy: (dy - 1) * P + (dz - 1) * PP
    out = []
    if c == 8:
        nks = 5 if nd == 3 else 2
        for k in range(nks):
            ta = (2 * k if k < 4 else 7) if nd == 3 else k
            dz, dy = (ta // 3, ta % 3) if nd == 3 else (1, ta)
            lbo = (PP - 2 * P) if (nd == 3 and k == 1) else P
            out.append((shift(dz, dy), lbo))
    else:
        for dz in (range(3) if nd == 3 else (1,)):
            for dy in range(3):
                out.append((shift(dz, dy), None))    # K spans channel groups (other arrays)
    return out


def supported():
    lib = _abi.load()
    shapes = []
    for nd, Ls in ((2, range(4, 66, 2)), (3, range(4, 18, 2))):
        for L in Ls:
            for c in (8, 16, 24, 32):
                if (nd, L, c) == (3, 16, 32):
                    continue                          # the dedicated 3D L=16 kernel
                hid = (C.c_int32 * _abi.GF_MAX_HIDDEN)(*([c, c] + [0] * (_abi.GF_MAX_HIDDEN - 2)))
                sh = _abi.FlowShapeExC(nd, L, 4, 2, hid, 3, 1, 0.01)
                if lib.gf_flow_tensor_core_supported(C.byref(sh)):
                    shapes.append((nd, L, c))
    return shapes


SHAPES = supported()


def test_there_are_shapes():
    assert len(SHAPES) >= 40


@pytest.mark.parametrize("nd,L,c", SHAPES)
def test_tile_reads_stay_in_the_buffer_and_stores_cover_the_lattice(nd, L, c):
    P, p_first, nt, npos = plan(nd, L)
    rows = np.arange(128)
    roff = 6 * (rows >> 3) + (rows & 7)           # row -> position offset in the tile
    store_rows = ((rows & 7) >= 1) & ((rows & 7) <= 6)
    covered = np.zeros(P ** nd, np.int32)
    for t in range(nt):
        first = p_first - 1 + 96 * t
        for off, lbo in taps(nd, P, c):
            lo = first + off + roff.min()
            hi = first + off + roff.max() + (lbo or 0)
            assert lo >= 0 and hi < npos, (t, off, lbo, lo, hi, npos)
        p = first + roff[store_rows]
        px, py = p % P, (p // P) % P
        pz = p // (P * P) if nd == 3 else np.ones_like(p)
        inner = (px >= 1) & (px <= L) & (py >= 1) & (py <= L) & (pz >= 1) & (pz <= L)
        np.add.at(covered, p[inner], 1)
    interior = np.zeros(P ** nd, bool)
    grid = np.indices((P,) * nd).reshape(nd, -1)
    interior[np.all((grid >= 1) & (grid <= L), axis=0)] = True
    assert (covered[interior] == 1).all() and (covered[~interior] == 0).all()


def test_output_rows_find_their_x_neighbours_in_their_own_eight():
    rows = np.arange(128)
    out = ((rows & 7) >= 1) & ((rows & 7) <= 6)
    roff = 6 * (rows >> 3) + (rows & 7)
    for r in rows[out]:
        # the rows one position to the left and right are r - 1 and r + 1, in the same group of 8
        assert (r - 1) >> 3 == r >> 3 == (r + 1) >> 3
        assert roff[r - 1] == roff[r] - 1 and roff[r + 1] == roff[r] + 1
