"""The adjoint scatter's carry of shared nodes, restated on the CPU: a lane
keeps per cell the sums U0 = sum v (1 - fy), U1 = sum v (1 - fy) f,
V0 = sum v fy, V1 = sum v fy f (corners U0/2 -+ U1 on the lower row,
V0/2 -+ V1 on the upper one); when a ray leaves a cell by a step in x or y,
the two nodes the next cell shares are added to the next cell's sums and only
the other two are written out; after a diagonal step all four.  Along any
path of cells each node must receive exactly the total of the direct method
(every cell's four corners written out), up to rounding."""
import numpy as np


def corners(u, w):
    U0, U1 = u
    V0, V1 = w
    return {(0, 0): 0.5 * U0 - U1, (0, 1): 0.5 * U0 + U1, (1, 0): 0.5 * V0 - V1, (1, 1): 0.5 * V0 + V1}


def carry(x, u, w, y, un, wn, out):
    """Write cell x's non-shared nodes into out, add the shared ones to the
    sums (un, wn) of the next cell y (a restatement of flush_carry)."""
    q = corners(u, w)
    dr, dc = y[0] - x[0], y[1] - x[1]
    r, c = x

    def put(i, j, v):
        out[(r + i, c + j)] = out.get((r + i, c + j), 0.0) + v

    if (dr, dc) == (0, 1):      # +x: the right column carries into the next cell's left column
        put(0, 0, q[(0, 0)]); put(1, 0, q[(1, 0)])
        un = (un[0] + q[(0, 1)], un[1] - 0.5 * q[(0, 1)])
        wn = (wn[0] + q[(1, 1)], wn[1] - 0.5 * q[(1, 1)])
    elif (dr, dc) == (0, -1):   # -x
        put(0, 1, q[(0, 1)]); put(1, 1, q[(1, 1)])
        un = (un[0] + q[(0, 0)], un[1] + 0.5 * q[(0, 0)])
        wn = (wn[0] + q[(1, 0)], wn[1] + 0.5 * q[(1, 0)])
    elif (dr, dc) == (1, 0):    # +y: the upper row becomes the next cell's lower row
        put(0, 0, q[(0, 0)]); put(0, 1, q[(0, 1)])
        un = (un[0] + w[0], un[1] + w[1])
    elif (dr, dc) == (-1, 0):   # -y
        put(1, 0, q[(1, 0)]); put(1, 1, q[(1, 1)])
        wn = (wn[0] + u[0], wn[1] + u[1])
    else:                       # diagonal or a jump: all four
        for k, v in q.items():
            put(*k, v)
    return un, wn


def test_carry_equals_direct_flush_along_random_paths():
    rng = np.random.default_rng(7)
    steps = [(0, 1), (0, -1), (1, 0), (-1, 0), (1, 1), (-1, 1), (1, -1), (-1, -1)]
    for trial in range(300):
        n = int(rng.integers(1, 30))
        cell = (int(rng.integers(5, 10)), int(rng.integers(5, 10)))
        path = [cell]
        for _ in range(n - 1):
            d = steps[int(rng.integers(0, 4 if trial % 3 else 8))]
            cell = (cell[0] + d[0], cell[1] + d[1])
            if cell != path[-1]:
                path.append(cell)
        # each visited cell receives the sums of a few random samples
        sums = []
        for _ in path:
            k = int(rng.integers(1, 6))
            v, fy, f = rng.normal(size=k), rng.uniform(0, 1, k), rng.uniform(-0.5, 0.5, k)
            sums.append(((v * (1 - fy)).sum(), (v * (1 - fy) * f).sum()) + ((v * fy).sum(), (v * fy * f).sum()))
        direct = {}
        for (r, c), s in zip(path, sums):
            for (i, j), val in corners(s[:2], s[2:]).items():
                direct[(r + i, c + j)] = direct.get((r + i, c + j), 0.0) + val
        carried = {}
        u, w = sums[0][:2], sums[0][2:]
        for idx in range(1, len(path)):
            un, wn = sums[idx][:2], sums[idx][2:]
            u, w = carry(path[idx - 1], u, w, path[idx], un, wn, carried)
        for (i, j), val in corners(u, w).items():      # the last cell: all four
            r, c = path[-1]
            carried[(r + i, c + j)] = carried.get((r + i, c + j), 0.0) + val
        keys = set(direct) | set(carried)
        for k in keys:
            assert abs(direct.get(k, 0.0) - carried.get(k, 0.0)) <= 1e-9 * (1 + abs(direct.get(k, 0.0))), (trial, k)
