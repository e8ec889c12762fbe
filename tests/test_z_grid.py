"""The z split of the FP32 march, restated on the CPU: z - ref_l in metres
as zhi = zh + k szh with zh and szh rounded to the grid 2^(e - 24),
2^e > 2 (Lz + max |ref_l| + 1) (the context's choice), plus a remainder.
Checked: zh + k szh is exact in FP32 for every sample k < G of rays across
the box (so the kernel's fmaf(k, szh, zh) is exact), and h_mid - zhi is
exact wherever the distance is at most the record's offset, otherwise
rounded once at the ulp of the distance: the argument's differences never
round at the scale of the offset."""
import math

import numpy as np

f32 = np.float32


def zgrid_m(box_z, refs):
    bound = 2.0 * (box_z + max(abs(r) for r in refs) + 1.0)
    return math.ldexp(1.0, math.frexp(bound)[1] - 1 + 1 - 24)


def test_grid_split_is_exact_along_every_ray():
    rng = np.random.default_rng(5)
    for box_z, refs, G in ((150.0, (40.0, 70.0, 110.0, 140.0), 256), (60.0, (10.0, 30.0), 384),
                           (1.0, (0.25, 0.5, 0.75), 64)):
        g = zgrid_m(box_z, refs)
        for _ in range(300):
            ref = float(f32(rng.choice(refs)))
            z0 = rng.uniform(0, box_z)
            zend = rng.uniform(0, box_z)
            sz = (zend - z0) / G
            zh = np.rint((z0 - ref) / g) * g
            szh = np.rint(sz / g) * g
            assert f32(zh) == zh and f32(szh) == szh
            k = np.arange(G, dtype=np.float64)
            zhi = zh + k * szh                            # the exact value
            assert np.array_equal(zhi.astype(np.float32).astype(np.float64), zhi)   # representable
            assert np.abs(zhi).max() < 2.0 * (box_z + max(refs) + 1.0)


def test_record_minus_z_is_exact_where_the_offset_dominates():
    """h_mid - zhi for any FP32 record h_mid and any zhi on the grid: exact
    where |h_mid - zhi| <= |h_mid| (h_mid's grid is the finer, and the
    difference fits in its binade); elsewhere a single rounding at the ulp
    of the difference, i.e. at the scale of the distance to the surface."""
    rng = np.random.default_rng(6)
    g = zgrid_m(150.0, (40.0, 70.0, 110.0, 140.0))
    hm = (rng.choice([-1.0, 1.0], 200000) * np.exp(rng.uniform(np.log(1e-3), np.log(60.0), 200000)))
    hm = hm.astype(np.float32).astype(np.float64)                   # FP32 records
    zhi = np.rint((hm + rng.uniform(-40, 40, hm.size)) / g) * g
    diff = hm - zhi
    got = diff.astype(np.float32).astype(np.float64)                 # the FP32 subtraction
    small = np.abs(diff) <= np.abs(hm)
    assert small.sum() > 10000
    assert np.array_equal(got[small], diff[small])
    ulp = np.spacing(np.abs(got).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(got - diff) <= 0.5 * ulp)
