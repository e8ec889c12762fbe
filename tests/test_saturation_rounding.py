"""The rounding argument behind the ray kernel's exact saturation windows,
checked in IEEE FP32 on the CPU (numpy float32, round to nearest).

Per surface-sample the BF16 march forms e = 2^a (a = the sigmoid argument
in log2 units), sigma = 1 / (1 + e) and accumulates sigma + 1, whose
mantissa
carries round(sigma * 2^23).  Samples with |a| >= 24.25 are skipped and
their contribution added exactly; that is exact when, for every such a and
for relative errors of the exponential and the reciprocal up to 2^-21 (the
approximate SFU functions are accurate to ~2^-22), sigma + 1 rounds to 1
(a >= 24.25: contributes 0) and 1 + e rounds to 1 (a <= -24.25: sigma is the
reciprocal of 1, contributes 2^23).  Just inside the window the rounding
is not exact, so the threshold cannot be lowered to 24."""
import numpy as np

f32 = np.float32
ERR = (1.0 - 2.0 ** -21, 1.0, 1.0 + 2.0 ** -21)


def _sigma_plus_one(a, ee, er):
    e = f32(f32(2.0 ** a) * f32(ee))
    d = f32(f32(1.0) + e)
    s = f32(f32(f32(1.0) / d) * f32(er))
    return f32(s + f32(1.0)), d


def test_above_the_window_adds_exactly_zero():
    for a in np.linspace(24.25, 60.0, 2000):
        for ee in ERR:
            for er in ERR:
                s1, _ = _sigma_plus_one(a, ee, er)
                assert s1 == f32(1.0), (a, ee, er, s1)


def test_below_the_window_adds_exactly_one():
    for a in np.linspace(-60.0, -24.25, 2000):
        for ee in ERR:
            _, d = _sigma_plus_one(a, ee, 1.0)
            assert d == f32(1.0), (a, ee, d)


def test_inside_the_window_rounding_is_not_exact():
    """At a = 23.9 sigma ~ 2^-23.9 exceeds half an ulp of 1, so sigma + 1 is
    not 1: such samples must be evaluated."""
    s1, _ = _sigma_plus_one(23.9, 1.0, 1.0)
    assert s1 > f32(1.0)
    _, d = _sigma_plus_one(-23.0, 1.0, 1.0)
    assert d > f32(1.0)


# ---------------------------------------------------------------- the FP32 march's complementary logistic
# The approximate-logistic mode's march forms, per sample, psi = 1 / (1 +
# 2^|a|) scaled by 2^28: q = round(rcp(fma(E, c, fma(E, -kappa c, c)))) with
# E = 2^|a| from ex2.approx, c = 2^-28 and kappa the per-device calibration
# (|kappa| < 1e-5 is enforced at set-up), and adds q above the surface,
# 2^28 - q below it.  Samples with |a| >= 29.25 are skipped and add exactly
# 0 / 2^28: exact when q rounds to 0 there, for relative errors of the
# exponential and the reciprocal up to 2^-21.  (The FP32 and compensated
# modes form E with the accurate exp2 instead; tests/test_accurate_logistic.py
# checks the same rounding for it.)


def _q(a, ee, er, kappa):
    c = f32(2.0 ** -28)
    E = f32(f32(2.0 ** a) * f32(ee))
    inner = f32(np.float64(E) * np.float64(f32(-kappa * 2.0 ** -28)) + np.float64(c))
    e = f32(np.float64(E) * np.float64(c) + np.float64(inner))
    y = f32(f32(np.float64(1.0) / np.float64(e)) * f32(er))
    return int(np.rint(np.float64(y)))


def test_psi_beyond_the_march_window_rounds_to_zero():
    for a in np.linspace(29.25, 60.0, 1500):
        for ee in ERR:
            for er in ERR:
                for kappa in (-1e-5, 0.0, 1e-5):
                    assert _q(a, ee, er, kappa) == 0, (a, ee, er, kappa)


def test_psi_inside_the_march_window_is_not_zero():
    """At |a| = 28.5 psi 2^28 ~ 0.7 rounds to 1: such samples must be evaluated."""
    assert _q(28.5, 1.0, 1.0, 0.0) == 1


def test_psi_fixed_point_is_exact_at_the_tie():
    """a = 0 (sample exactly on the surface): psi = 1/2, q = 2^27, so a sample
    above adds 2^27 and one below adds 2^28 - 2^27: the same 1/2 either way
    (the indicator's eta(0) = 1/2)."""
    assert _q(0.0, 1.0, 1.0, 0.0) == 2 ** 27
