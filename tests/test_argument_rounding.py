"""The FP32 march's sigmoid argument, restated in IEEE FP32 on the CPU.

Per sample the kernel forms, with z - ref_l = zhi + rem (zhi on an exact
grid in metres, zlo = kg64 rem in log2 units) and the two rows' records
{h_mid, dx} (offsets from ref_l, exact on the grid of FP32 heights):
    a = fmaf(fx, dxA, hA - zhi),  b = fmaf(fx, dxB, hB - zhi)
    d = fmaf(fy, b - a, a)                       (s_l - zhi)
    arg = fmaf(-kgh, d, fmaf(-kgl, d, zlo))      (kg64 (z - s_l))
Checked against FP64: the differences h - zhi are exact where they are at
most |h| (the case for the records of an offset surface); the argument's
error near the surface, where the logistic's slope
weights it, does not grow with the surface's offset from ref_l (it did when
the lerps were taken on the offsets themselves), and it carries no bias."""
import numpy as np

f32 = np.float32
KG = 1.4426950408889634          # log2(e) / gamma, gamma = 1 m


def fmaf(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def _case(offset_sd, n=400_000, seed=0):
    rng = np.random.default_rng(seed)
    q = 2.0 ** -19                                   # grid of h_mid for heights of 64-128 m
    off = rng.normal(0, offset_sd, n)
    hA = np.round(off / q) * q
    dxA = np.round(rng.normal(0, 2.0, n) / q) * q
    hB = np.round((off + rng.normal(0, 2.0, n)) / q) * q
    dxB = np.round((dxA + rng.normal(0, 0.5, n)) / q) * q
    fx = f32(rng.uniform(-0.5, 0.5, n)).astype(np.float64)
    fy = f32(rng.uniform(0, 1, n)).astype(np.float64)
    s = (1 - fy) * (hA + fx * dxA) + fy * (hB + fx * dxB)
    zr = s + rng.normal(0, 3.0, n)                   # samples within a few metres of the surface
    gm = 2.0 ** -14                                  # grid of z in metres
    zhi = np.round(zr / gm) * gm
    zlo = f32(KG * (zr - zhi))
    exact = KG * (zr - s)
    kgh = f32(KG)
    kgl = f32(KG - np.float64(kgh))
    dA = (hA - zhi).astype(np.float32)
    dB = (hB - zhi).astype(np.float32)
    near = np.abs(hA - zhi) <= np.abs(hA)
    assert np.array_equal(dA[near].astype(np.float64), (hA - zhi)[near])   # exact differences
    a = fmaf(fx, dxA, dA)
    b = fmaf(fx, dxB, dB)
    d = fmaf(fy, (b.astype(np.float64) - a.astype(np.float64)).astype(np.float32), a)
    arg = fmaf(-kgh, d, fmaf(-kgl, d, zlo))
    # the same on the offsets (the earlier form): sl = lerp(h), arg = kg (zr - sl)
    a0 = fmaf(fx, dxA, f32(hA))
    b0 = fmaf(fx, dxB, f32(hB))
    sl = fmaf(fy, (b0.astype(np.float64) - a0.astype(np.float64)).astype(np.float32), a0)
    zhl = f32(KG * zhi)                              # the earlier z in log2 units
    arg0 = (fmaf(-kgh, sl, fmaf(-kgl, sl, f32(KG * zr - np.float64(zhl)))).astype(np.float64)
            + zhl.astype(np.float64)).astype(np.float32)
    psi = 1.0 / (1.0 + 2.0 ** exact)
    w = psi * (1 - psi) * np.log(2.0)               # d psi / d arg
    return w, arg.astype(np.float64) - exact, arg0.astype(np.float64) - exact


def test_argument_error_does_not_grow_with_the_offset():
    rms = {}
    for sd in (3.0, 12.0, 30.0):
        w, e, e0 = _case(sd)
        rms[sd] = (np.sqrt(np.mean((w * e) ** 2)), np.sqrt(np.mean((w * e0) ** 2)))
        assert abs(np.mean(w * e)) < 0.05 * rms[sd][0]            # no bias
    # exact differences: the same error at any offset
    assert rms[30.0][0] < 1.3 * rms[3.0][0], rms
    # on the offsets the error grew with them, and was several times larger
    assert rms[30.0][1] > 3.0 * rms[3.0][1], rms
    assert rms[30.0][1] > 8.0 * rms[30.0][0], rms
