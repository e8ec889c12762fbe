"""The adjoint's float -> fixed-point rounding (add_fixed in adjoint.cu),
restated with IEEE FP32 / integer operations on the CPU and checked against
round-half-to-even over every magnitude it handles: the small branch adds
1.5 * 2^23 and reads the integer from the float's bits (|v| < 2^22); the
large branch shifts the 24-bit significand by the exponent (|v| >= 2^22),
rounding the one bit it drops at 2^22 <= |v| < 2^23 to even."""
import numpy as np

f32 = np.float32


def fixed(v):
    v = f32(v)
    a = abs(v)
    if a < f32(4194304.0):
        t = f32(v + f32(12582912.0))
        return int(np.array(t, np.float32).view(np.int32)) - 0x4B400000
    bits = int(np.array(a, np.float32).view(np.uint32))
    e = min(bits >> 23, 190)
    m = (bits & 0x7FFFFF) | 0x800000
    mag = m << (e - 150) if e >= 150 else (m >> 1) + (m & (m >> 1) & 1)
    return -mag if v < 0 else mag


def rne(v):
    return int(np.rint(np.float64(f32(v))))        # exact for float32 inputs


def test_small_branch_is_round_half_even():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.uniform(-4.2e6, 4.2e6, 200000),
                           np.arange(-40, 40) + 0.5,       # ties
                           [0.0, -0.0, 0.49999997, -0.49999997, 4194303.5, -4194303.5]])
    for v in vals.astype(np.float32):
        if abs(v) < 4194304.0:
            assert fixed(v) == rne(v), v


def test_large_branch_is_exact_or_round_half_even():
    rng = np.random.default_rng(1)
    for e in range(22, 62):
        lo, hi = 2.0 ** e, 2.0 ** (e + 1)
        vals = rng.uniform(lo, hi, 2000).astype(np.float32)
        vals = np.concatenate([vals, -vals, np.array([lo, -lo], np.float32)])
        for v in vals:
            if abs(v) >= 4194304.0:
                assert fixed(v) == rne(v), (e, v)
    # ties at 2^22 <= |v| < 2^23, where the significand has one fractional bit
    for k in range(4194304, 4194304 + 64):
        v = f32(k + 0.5)
        assert fixed(v) == rne(v) and fixed(-v) == rne(-v), v
