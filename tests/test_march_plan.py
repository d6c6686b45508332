"""Host-side model of the row-marching two-step kernels' schedules (no GPU).

The forward kernel computes 128 columns per warp for 120 stored ones, starts
sub-step A two rows and sub-step B one row below its tile, and takes every
neighbour value from a lane shuffle (which wraps at the warp's edges).  This
test follows which values are correct through the two sub-steps of the Yee
update (Eq. (5), then Eq. (3), twice) on one warp's strip and checks that
every stored value is; and that the tile plan (CTAs of W = 3 or 4 warps)
stores every cell of a grid exactly once, with every load inside the pitched
arrays.  The same for the reverse sweep's two-step kernel (the transposed
update run twice: A at row j, B at row j - 1, both starting two rows below
the tile with their first row's carried edge terms at zero)."""
import numpy as np
import pytest

KO = 120                   # stored columns per warp (a CTA of W warps: W x 120)


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


def plan(nx, ny, th, W):
    return [(x0, y0, min(y0 + th, ny)) for y0 in range(0, ny, th) for x0 in range(0, nx, KO * W)]


@pytest.mark.parametrize("W", [3, 4])
@pytest.mark.parametrize("nx,ny,th", [(60, 60, 8), (100, 80, 13), (481, 50, 7), (1023, 517, 40),
                                      (4096, 512, 82), (129, 2, 4), (3, 3, 8), (1024, 64, 41)])
def test_plan_stores_each_cell_once_and_loads_stay_inside(nx, ny, th, W):
    P = ((nx + 1 + 127) // 128) * 128          # pitch: a multiple of 128 columns >= nx + 1
    size = (ny + 1) * P                       # floats per field (float2 per material)
    stored = np.zeros((ny, P), np.int32)
    for (x0, j0, j1) in plan(nx, ny, th, W):
        for w in range(W):
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


def reverse_strip_correctness(c0, j0, j1, ny):
    """Which values of the reverse kernel's warp strip equal the true result
    of two reverse steps: A (step t) at rows jA0 .. min(j1, ny - 1), B (step
    t - 1) at rows jA0 .. j1 - 1, both from jA0 = max(j0 - 2, 0) with their
    first row's carried Ex-edge terms and g_H'(row - 1) at zero (A's Ex-edge
    terms of its first row come from memory).  g_H'(j, c) takes the Ex edges
    of rows j, j + 1 and the Ey edges of columns c, c + 1 (the latter by
    shuffle; an Ey edge's coefficient needs the material of column c - 1, by
    shuffle); g_Ex'(j) takes g_H'(j - 1), g_H'(j); g_Ey'(c) takes g_H'(c - 1),
    g_H'(c).  Returns the maps of B's g_H', g_Ex', g_Ey' and of the cells'
    accumulated material terms."""
    W = 128
    jA0 = max(j0 - 2, 0)
    jAe = min(j1, ny - 1)
    ks = np.arange(W)
    rows = list(range(jA0, j1 + 1))
    gnA, vxA, vyA, accA = {}, {}, {}, {}
    muyok = ks >= 1                           # the Ey edge's left material (shuffle)
    for j in rows:
        if j > jAe:                           # row ny: the boundary's Ex edges, zero
            vxA[j] = np.ones(W, bool)
            continue
        gn = muyok & np.append(muyok[1:], False)          # muy(c), muy(c + 1)
        gnA[j] = gn
        below = gnA.get(j - 1)
        vxA[j] = gn & (below if below is not None else np.full(W, j == 0))
        vyA[j] = gn & np.append(False, gn[:-1])
        # A's material terms of row j: edx(j) (from memory, but zero on A's
        # first row unless that row is the wall) and the Ey edges c, c + 1
        accA[j] = gn & (j > jA0 or j == 0)
    gnB, vxB, vyB, acc = {}, {}, {}, {}
    for r in range(jA0, j1):
        first = r == jA0
        muxB = np.full(W, r == 0) if first else vxA[r]      # Ex edges of row r: B's carried term
        mux1 = vxA[r + 1] if r + 1 <= ny - 1 else np.ones(W, bool)
        muyB = muyok & vyA[r]
        gn = gnA[r] & muxB & mux1 & muyB & np.append(muyB[1:], False)
        gnB[r] = gn
        prev = gnB.get(r - 1)
        cgx = np.full(W, r == 0) if first else vxA[r]
        vxB[r] = gn & cgx & (prev if prev is not None else np.full(W, r == 0))
        vyB[r] = gn & np.append(False, gn[:-1]) & vyA[r]
        acc[r] = accA[r] & gn
    return gnB, vxB, vyB, acc


@pytest.mark.parametrize("c0,j0,j1,ny", [(0, 0, 17, 300), (120, 17, 34, 300), (480, 282, 300, 300),
                                         (960, 1, 40, 40), (3960, 82, 164, 4096), (240, 2, 43, 1024)])
def test_every_stored_reverse_value_is_correct(c0, j0, j1, ny):
    gnB, vxB, vyB, acc = reverse_strip_correctness(c0, j0, j1, ny)
    stored = (np.arange(128) >= 4) & (np.arange(128) < 4 + KO)
    for r in range(j0, j1):
        for m in (gnB, vxB, vyB, acc):
            assert m[r][stored].all(), (r, c0)
    # the wrapped shuffles spoil the outer columns only
    r = j0 + 1 if j0 + 1 < j1 else j0
    assert not gnB[r][0] and not gnB[r][-1]


@pytest.mark.parametrize("W", [3, 4])
@pytest.mark.parametrize("nx,ny,th", [(100, 80, 13), (1024, 1024, 41), (481, 50, 7), (129, 2, 4)])
def test_reverse_plan_stores_each_cell_once_and_loads_stay_inside(nx, ny, th, W):
    P = ((nx + 1 + 127) // 128) * 128
    size = (ny + 1) * P
    stored = np.zeros((ny, P), np.int32)
    for (x0, j0, j1) in plan(nx, ny, th, W):
        for w in range(W):
            c0 = x0 + KO * w
            if c0 >= nx:
                continue
            jA0, jAe = max(j0 - 2, 0), min(j1, ny - 1)
            for lane in range(32):
                cl = c0 - 4 + 4 * lane
                if 0 <= cl < P:
                    assert cl + 3 < P
                    for j in range(jA0, jAe + 1):   # row j's loads: rows j and j + 1
                        assert (j + 1) * P + cl + 3 < size and j * P + cl >= 0
                    if jA0 >= 1:                    # the first row's edge terms: mat(jA0 - 1)
                        assert (jA0 - 1) * P + cl >= 0
                if 1 <= lane <= 30 and cl < nx:
                    for r in range(j0, j1):
                        stored[r, cl:cl + 4] += 1
    assert (stored[:, :nx] == 1).all()
    assert (stored <= 1).all()
