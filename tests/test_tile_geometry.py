"""Host-side check of the tile geometry that the chained flow launches' per-tile flags rely on.

A tile of a T-step launch loads the window [X0, X0 + LW) x [Y0, Y0 + CH + 2) of U^t, with
X0 = x0 - (T + 1) rounded down to the TMA alignment A (16 bytes of elements) and Y0 = y0 - T,
and writes the output tile [x0, x0 + 130 - 2T) x [y0, y0 + CH + 2 - 2T) (CH = 4 x warps).  A tile
of the next launch waits only for the 3 x 3 tiles around its own in the previous launch.  That is
enough when (a) its window lies inside those nine output tiles (everything it reads was written
by them) and (b) no tile further away has a window that reaches its output tile (every read of the
region it overwrites was made by one of them).  Both are checked here for every steps-per-launch
count, both tile shapes and both element sizes, on image sizes with ragged last tiles.
"""
import itertools

import pytest

CW = 128  # region columns


def geometry(T, warps, elem_bytes):
    A = 16 // elem_bytes
    LW = (CW + 2 + A + A - 1) // A * A
    CH = 4 * warps
    return A, LW, CH, CW + 2 - 2 * T, CH + 2 - 2 * T


def window(T, warps, elem_bytes, tx, ty):
    A, LW, CH, owt, oht = geometry(T, warps, elem_bytes)
    x0, y0 = tx * owt, ty * oht
    X0 = (x0 - (T + 1)) // A * A  # floor, also below 0
    Y0 = y0 - T
    return (X0, X0 + LW), (Y0, Y0 + CH + 2)


def tiles_touched(lo, hi, size, n):
    """Indices of the output tiles of width `size` (n of them) that [lo, hi) overlaps."""
    return {t for t in range(n) if max(lo, t * size) < min(hi, (t + 1) * size)}


@pytest.mark.parametrize("T,warps,elem_bytes", list(itertools.product(range(2, 9), (16, 8), (4, 2))))
def test_windows_stay_within_the_neighbouring_tiles(T, warps, elem_bytes):
    _, _, _, owt, oht = geometry(T, warps, elem_bytes)
    assert owt > 0 and oht > 0
    for h, w in [(2048, 2048), (2047, 1999), (700, 3000)]:
        ntx, nty = -(-w // owt), -(-h // oht)
        for tx, ty in itertools.product(range(ntx), range(nty)):
            (xa, xb), (ya, yb) = window(T, warps, elem_bytes, tx, ty)
            # (a) the window reads only the outputs of the 3 x 3 tiles around its own
            assert tiles_touched(max(xa, 0), min(xb, w), owt, ntx) <= {tx - 1, tx, tx + 1}
            assert tiles_touched(max(ya, 0), min(yb, h), oht, nty) <= {ty - 1, ty, ty + 1}
        # (b) the converse: a window two or more tiles away misses the output tile
        for tx in range(ntx):
            for tx2 in (tx - 2, tx + 2):
                if 0 <= tx2 < ntx:
                    (xa, xb), _ = window(T, warps, elem_bytes, tx2, 0)
                    assert min(xb, w) <= tx * owt or max(xa, 0) >= min((tx + 1) * owt, w)
        for ty in range(nty):
            for ty2 in (ty - 2, ty + 2):
                if 0 <= ty2 < nty:
                    _, (ya, yb) = window(T, warps, elem_bytes, 0, ty2)
                    assert min(yb, h) <= ty * oht or max(ya, 0) >= min((ty + 1) * oht, h)


def test_output_tiles_are_the_exact_part_of_the_window():
    """After T steps the still-exact part of a window starts T + 1 cells in from its unrounded
    left edge x0 - (T + 1) and one row of halo plus T - 1 rows in from its top: exactly the
    output tile's first column and row."""
    for T, warps in itertools.product(range(2, 9), (16, 8)):
        _, _, CH, owt, oht = geometry(T, warps, 4)
        x0, y0 = 5 * owt, 3 * oht
        exact_x = (x0 - (T + 1) + 1 + T, x0 - (T + 1) + CW + 2 + 1 - T)
        exact_y = (y0 - T + T, y0 - T + CH + 2 - T)
        assert exact_x == (x0, x0 + owt)
        assert exact_y == (y0, y0 + oht)
