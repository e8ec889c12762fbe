"""The rounding argument behind the ray kernel's exact saturation windows,
checked in IEEE FP32 on the CPU (numpy float32, round to nearest).

Per surface-sample the FP32 path forms e = 2^a (a = the sigmoid argument in
log2 units), sigma = 1 / (1 + e) and accumulates sigma + 1, whose mantissa
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
