"""Host-side model of the row-marching two-step kernel's schedule (no GPU).

The kernel computes 128 columns per warp for 120 stored ones, starts
sub-step A two rows and sub-step B one row below its tile, and takes every
neighbour value from a lane shuffle (which wraps at the warp's edges).  This
test follows which values are correct through the two sub-steps of the Yee
update (Eq. (5), then Eq. (3), twice) on one warp's strip and checks that
every stored value is; and that the tile plan stores every cell of a grid
exactly once, with every load inside the pitched arrays."""
import numpy as np
import pytest

KO, KC = 120, 480          # stored columns per warp, per CTA


def strip_correctness(c0, j0, j1, ny, nx):
    """Boolean maps (rows x computed columns) of the values that equal the
    true two-step result, following the kernel's dependencies."""
    cols = np.arange(c0 - 4, c0 + 124)
    W = len(cols)
    jA0, jAe, jB0 = max(j0 - 2, 0), min(j1, ny), max(j0 - 1, 0)
    rows = np.arange(jA0, jAe + 1)
    R = len(rows)
    # inputs (E^n, Hz^{n-1/2}, materials) are loaded for every computed
    # column and row; outside the grid a value is a boundary value (PEC or
    # dead cell) and therefore also "correct".
    # shuffle neighbours: column index k-1 / k+1 inside the warp, wrong at
    # the wrap (k = 0 has no left neighbour, k = W-1 no right one)
    hA = np.zeros((R, W), bool)   # Hz^{n+1/2}
    xA = np.zeros((R, W), bool)   # Ex^{n+1}
    yA = np.zeros((R, W), bool)   # Ey^{n+1}
    for r, j in enumerate(rows):
        for k in range(W):
            # Hz(j, c) needs Ex^n(j), Ex^n(j+1), Ey^n(c), Ey^n(c+1): Ey^n(c+1) by shuffle
            hA[r, k] = k + 1 < W
        for k in range(W):
            # Ex(j, c) needs Hz(j-1, c) (carried; unknown on the first row
            # unless the row is the bottom wall) and Hz(j, c)
            below = (r > 0 and hA[r - 1, k]) or j == 0
            xA[r, k] = hA[r, k] and below
            # Ey(j, c) needs Hz(j, c-1) (shuffle) and Hz(j, c)
            yA[r, k] = hA[r, k] and k - 1 >= 0 and hA[r, k - 1]
    hB = np.zeros((R, W), bool)
    xB = np.zeros((R, W), bool)
    yB = np.zeros((R, W), bool)
    for r, j in enumerate(rows):
        if j < jB0 or r + 1 >= R:
            continue                      # B runs on rows jB0 .. j1-1 (iteration j+1)
        for k in range(W):
            # Hz^{n+3/2}(j, c): Ex^{n+1}(j), Ex^{n+1}(j+1), Ey^{n+1}(c), Ey^{n+1}(c+1) (shuffle), Hz^{n+1/2}(j)
            hB[r, k] = (xA[r, k] and (xA[r + 1, k] or rows[r + 1] == ny) and yA[r, k]
                        and k + 1 < W and yA[r, k + 1] and hA[r, k])
        for k in range(W):
            below = (r > 0 and rows[r - 1] >= jB0 and hB[r - 1, k]) or j == 0
            xB[r, k] = hB[r, k] and below and xA[r, k]
            yB[r, k] = hB[r, k] and k - 1 >= 0 and hB[r, k - 1] and yA[r, k]
    return rows, cols, hB, xB, yB


@pytest.mark.parametrize("c0,j0,j1,ny,nx", [
    (0, 0, 17, 300, 1000), (120, 17, 34, 300, 1000), (480, 282, 300, 300, 1000),
    (960, 1, 40, 40, 1000), (3960, 82, 164, 4096, 4096)])
def test_every_stored_value_is_correct(c0, j0, j1, ny, nx):
    rows, cols, hB, xB, yB = strip_correctness(c0, j0, j1, ny, nx)
    stored_c = (cols >= c0) & (cols < c0 + KO)
    for r, j in enumerate(rows):
        if j0 <= j < j1:
            assert hB[r, stored_c].all() and xB[r, stored_c].all() and yB[r, stored_c].all(), (j, c0)
    # the values at the warp's edges are wrong (the wrapped shuffles): two
    # sub-steps reach three columns to the left and two to the right of the
    # computed range, inside its four spare columns on the left and the
    # fresh column on the right of the stored ones
    r = rows.tolist().index(j0)
    assert not hB[r, 0] and not yB[r, 1] and not hB[r, -2]
    assert cols[np.flatnonzero(yB[r])[0]] == c0 - 2 and cols[np.flatnonzero(hB[r])[-1]] == c0 + KO + 1


def plan(nx, ny, th):
    return [(x0, y0, min(y0 + th, ny)) for y0 in range(0, ny, th) for x0 in range(0, nx, KC)]


@pytest.mark.parametrize("nx,ny,th", [(60, 60, 8), (100, 80, 13), (481, 50, 7), (1023, 517, 40),
                                      (4096, 512, 82), (129, 2, 4), (3, 3, 8)])
def test_plan_stores_each_cell_once_and_loads_stay_inside(nx, ny, th):
    P = ((nx + 1 + 127) // 128) * 128          # pitch: a multiple of 128 columns >= nx + 1
    size = (ny + 1) * P                       # floats per field (float2 per material)
    stored = np.zeros((ny, P), np.int32)
    for (x0, j0, j1) in plan(nx, ny, th):
        for w in range(4):
            c0 = x0 + KO * w
            if c0 >= nx:
                continue
            jA0, jAe, jB0 = max(j0 - 2, 0), min(j1, ny), max(j0 - 1, 0)
            for lane in range(32):
                cl = c0 - 4 + 4 * lane
                if 0 <= cl < P:                 # loads (lanes outside the row read nothing)
                    assert cl + 3 < P
                    for j in range(jA0, jAe + 1):
                        if j < ny:
                            assert (j + 1) * P + cl + 3 < size and j * P + cl >= 0
                if 1 <= lane <= 30 and cl < nx:
                    for r in range(max(jB0, j0), j1):
                        stored[r, cl:cl + 4] += 1
                        assert r * P + cl + 3 < size
    assert (stored[:, :nx] == 1).all()
    assert (stored <= 1).all()
