"""The FP32 modes' accurate logistic, restated step by step in IEEE FP32
(numpy float32; each fused multiply-add rounded once): 2^x split exactly
into 2^round(x) times a degree-6 polynomial of the fraction, the integer part
added to the exponent bits.  Checked here on the CPU: the error bound over the
arguments the march can see, the absence of a bias (the reason the mode needs
no calibration), the exponent-bit identity the kernel relies on, and that
with it a sample at |a| >= 29.25 log2 units still rounds to exactly 0 units of
2^-28 (the exact-saturation windows)."""
import numpy as np

M = np.float32(12582912.0)  # 1.5 * 2^23
COEF = [np.float32(c) for c in (1.0, 6.931471824645996e-01, 2.4022646248340607e-01, 5.550328642129898e-02,
                                9.618489071726799e-03, 1.3399930903688073e-03, 1.534581242594868e-04)]


def fma32(a, b, c):
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(np.float32)


def exp2_acc(x):
    x = np.minimum(x.astype(np.float32), np.float32(64.0))
    t = (x + M).astype(np.float32)
    f = fma32((t - M).astype(np.float32), np.float32(-1.0), x)
    p = np.full_like(f, COEF[6])
    for k in range(5, -1, -1):
        p = fma32(p, f, COEF[k])
    bits = p.view(np.int32).astype(np.int64) + ((t.view(np.int32).astype(np.int64) << 23) & 0xFFFFFFFF)
    bits = ((bits + 2**31) % 2**32 - 2**31).astype(np.int32)
    return bits.view(np.float32)


def test_exponent_bits_identity():
    """bits(1.5 * 2^23 + i) << 23 == i << 23 modulo 2^32 for every integer
    0 <= i <= 64 (the pattern of 1.5 * 2^23 shifts out)."""
    for i in range(65):
        t = np.float32(12582912.0 + i)
        assert (int(t.view(np.int32)) << 23) % 2**32 == (i << 23) % 2**32


def test_error_bound_and_no_bias():
    x = np.linspace(0.0, 40.0, 2_000_001).astype(np.float32)
    e = exp2_acc(x).astype(np.float64)
    ref = np.exp2(x.astype(np.float64))
    rel = (e - ref) / ref
    assert np.abs(rel).max() < 1.2e-7            # about 2 ulp
    assert abs(rel.mean()) < 2e-9                # no bias: ~0.03 ulp at most
    # the fraction's polynomial alone (its FP32 coefficients in exact
    # arithmetic) is within 2e-8, a third of an ulp
    f = np.linspace(-0.5, 0.5, 100_001)
    p = sum(float(c) * f ** k for k, c in enumerate(COEF))
    assert np.abs(p / np.exp2(f) - 1).max() < 2e-8


def test_clamp_keeps_large_arguments_finite():
    x = np.array([63.5, 64.0, 100.0, 200.0, 1e6], dtype=np.float32)
    e = exp2_acc(x)
    assert np.all(np.isfinite(e)) and np.all(e >= np.float32(2.0 ** 63))


def test_saturated_sample_rounds_to_zero():
    """psi 2^28 = 1 / ((2^|a| + 1) 2^-28) < 1/2 for |a| >= 29.25, with the
    reciprocal's relative error (one Newton step: ~1 ulp) allowed for."""
    a = np.linspace(29.25, 64.0, 100_001).astype(np.float32)
    E = exp2_acc(a).astype(np.float64)
    c = 2.0 ** -28
    e = np.float32(E * c + c).astype(np.float64)
    q = (1.0 / e) * (1 + 2 ** -22)
    assert np.all(q < 0.5)
    # just inside the window a sample does add a unit
    a_in = np.float32(28.9)
    e_in = float(exp2_acc(np.array([a_in]))[0]) * c + c
    assert 1.0 / e_in > 0.5
