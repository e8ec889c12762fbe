"""The FP32 march's cell fraction, restated in IEEE FP32 on the CPU.

Per axis the kernel rounds g = fmaf(k, sh, c) (c = fmaf(kc, sl, o), the
block's low part) to its cell i (adding 1.5 * 2^23, nearest in x, down in y)
and then forms the fraction as fmaf(k, sh, -i) + c: the product k sh is
exact inside the fused multiply-add, so the fraction carries the rounding
of a number below one cell.  Checked: i + f reproduces the exact FP64
coordinate to a few ulps of one cell at any distance from the start cell,
whereas g - i (what the kernel formed before) is off by up to half an ulp of
g, 2^-18 cells after 64 cells of travel; and f stays within rounding of its
cell ([-1/2, 1/2] about the midpoint in x, [0, 1) in y)."""
import numpy as np

f32 = np.float32
M = f32(12582912.0)


def fmaf(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def _case(rng, floor_axis):
    G = 384
    step = rng.uniform(0.1, 0.5) * rng.choice([-1.0, 1.0])
    sh = f32(step)
    sl = f32(step - np.float64(sh))
    o = f32(rng.uniform(0.0, 1.0) if floor_axis else rng.uniform(-0.5, 0.5))
    k = np.arange(G)
    kc = (k & ~7) + np.where(k & 1, 4, 3)
    c = fmaf(f32(kc), sl, o)
    g = fmaf(f32(k), sh, c)
    if floor_axis:
        i = np.floor(g.astype(np.float64))                   # 1.5 * 2^23 + g rounded down
    else:
        i = (g.astype(np.float64) + np.float64(M)).astype(np.float32).astype(np.float64) - np.float64(M)
    f_new = (fmaf(f32(k), sh, f32(-i)).astype(np.float64) + c.astype(np.float64)).astype(np.float32)
    f_old = (g.astype(np.float64) - i).astype(np.float32)   # exact
    exact = np.float64(o) + k * np.float64(sh) + kc * np.float64(sl)   # the kernel's intended coordinate
    return exact, i, f_new.astype(np.float64), f_old.astype(np.float64)


def test_fraction_error_does_not_grow_with_travel():
    rng = np.random.default_rng(11)
    worst_new, worst_old_far = 0.0, 0.0
    for t in range(400):
        floor_axis = bool(t & 1)
        exact, i, fn, fo = _case(rng, floor_axis)
        en = np.abs(i + fn - exact)
        eo = np.abs(i + fo - exact)
        worst_new = max(worst_new, en.max())
        far = np.abs(exact) > 32
        if far.any():
            worst_old_far = max(worst_old_far, eo[far].max())
        lo, hi = (0.0, 1.0) if floor_axis else (-0.5, 0.5)
        slack = 2.0 ** -17
        assert fn.min() >= lo - slack and fn.max() <= hi + slack
    assert worst_new <= 2.0 ** -22, worst_new
    assert worst_old_far >= 2.0 ** -20, worst_old_far   # the start-relative fraction's rounding
