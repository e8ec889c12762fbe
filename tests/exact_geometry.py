"""Exact (non-sampled) path lengths of a ray through ordered bilinear surfaces.

An independent check of the oracle's sampled march in the hard-indicator case
(gamma = 0): along a ray, the bilinear height of a surface inside one grid cell
is a quadratic in the ray parameter t, so every place where the ray crosses a
surface is a root of a quadratic.  Splitting [0, t_exit] at the grid lines and
at those roots leaves pieces inside a single unit; their lengths are the exact
unit path lengths.  Written with numpy only; it shares nothing with oracle.c.
"""
import numpy as np


def t_exit_box(o, d, box):
    ts = []
    for a in range(3):
        if d[a] > 0:
            ts.append((box[a] - o[a]) / d[a])
        elif d[a] < 0:
            ts.append(-o[a] / d[a])
    return min(ts)


def _cell_quadratic(h, r0, c0, o, d, box, R, Q):
    """Coefficients (t^0, t^1, t^2) of the surface height along the ray in cell (r0, c0)."""
    sx, sy = (Q - 1) / box[0], (R - 1) / box[1]
    ax, bx = o[0] * sx - c0, d[0] * sx          # local x coordinate = ax + bx t
    ay, by = o[1] * sy - r0, d[1] * sy
    h00, h01 = h[r0, c0], h[r0, c0 + 1]
    h10, h11 = h[r0 + 1, c0], h[r0 + 1, c0 + 1]
    A, B, Cc, D = h00, h01 - h00, h10 - h00, h00 - h01 - h10 + h11
    # A + B X + Cc Y + D X Y with X = ax + bx t, Y = ay + by t
    c0_ = A + B * ax + Cc * ay + D * ax * ay
    c1_ = B * bx + Cc * by + D * (ax * by + ay * bx)
    c2_ = D * bx * by
    return c0_, c1_, c2_


def exact_unit_lengths(H, o, d, box):
    """Exact path length per unit for ordered surfaces H[L][R][Q] (hard indicator)."""
    H = np.asarray(H, np.float64)
    L, R, Q = H.shape
    o, d, box = (np.asarray(v, np.float64) for v in (o, d, box))
    T = t_exit_box(o, d, box)
    cuts = {0.0, T}
    for a, n in ((0, Q), (1, R)):
        if d[a] != 0:
            for i in range(n):
                g = i * box[a] / (n - 1)
                t = (g - o[a]) / d[a]
                if 0 < t < T:
                    cuts.add(t)
    cuts = sorted(cuts)
    pieces = []
    for ta, tb in zip(cuts[:-1], cuts[1:]):
        if tb - ta <= 0:
            continue
        tm = 0.5 * (ta + tb)
        gx = min(max((o[0] + tm * d[0]) / box[0] * (Q - 1), 0.0), Q - 1)
        gy = min(max((o[1] + tm * d[1]) / box[1] * (R - 1), 0.0), R - 1)
        c0 = min(int(np.floor(gx)), Q - 2)
        r0 = min(int(np.floor(gy)), R - 2)
        roots = [ta, tb]
        for l in range(L):
            q0, q1, q2 = _cell_quadratic(H[l], r0, c0, o, d, box, R, Q)
            # surface minus ray height
            q0 -= o[2]
            q1 -= d[2]
            coeffs = [q2, q1, q0]
            while len(coeffs) > 1 and abs(coeffs[0]) < 1e-300:
                coeffs = coeffs[1:]
            if len(coeffs) > 1:
                for rt in np.roots(coeffs):
                    if abs(rt.imag) < 1e-12 and ta < rt.real < tb:
                        roots.append(rt.real)
        roots = sorted(roots)
        for sa, sb in zip(roots[:-1], roots[1:]):
            if sb > sa:
                pieces.append((sa, sb, r0, c0))
    lens = np.zeros(L + 1)
    for sa, sb, r0, c0 in pieces:
        tm = 0.5 * (sa + sb)
        z = o[2] + tm * d[2]
        below = 0
        for l in range(L):
            q0, q1, q2 = _cell_quadratic(H[l], r0, c0, o, d, box, R, Q)
            if q0 + q1 * tm + q2 * tm * tm < z:
                below += 1
        lens[below] += sb - sa
    return lens, T
