"""The integer facts the FP32 ray kernel's cell addressing relies on, checked
in IEEE FP32 / uint32 arithmetic on the CPU:

* adding 1.5 * 2^23 to a cell coordinate c in [-1/2, n - 3/2) rounds it to
  the nearest integer i in [0, n - 2], readable from the float's bits as
  bits - 0x4B400000, with |c - i| <= 1/2;
* the shared-memory byte address bits(ty) * 8Q + bits(tx) * 8 + k0 with
  k0 = base - 8 * 0x4B400000 * (Q + 1), all modulo 2^32, equals
  base + 8 (Q iy + ix), and the record one row up (+ 8Q) still lies inside
  the surface's R x Q plane of 8-byte records;
* the ray table's upper bound, the largest float 8 ulps below n - 3/2, keeps
  the rounded index below n - 1;
* the y axis, taken from the cell's lower edge, adds 1.5 * 2^23 rounding
  toward -infinity: a coordinate in [0, n - 1) gives floor(c) in [0, n - 2],
  read from the bits the same way, the fraction c - floor(c) in [0, 1) is
  exact, and the address algebra is unchanged."""
import numpy as np

f32 = np.float32
M = f32(12582912.0)          # 1.5 * 2^23
MAGIC = 0x4B400000


def _upper(n):
    v = f32(n - 1.5)
    for _ in range(8):
        v = np.nextafter(v, f32(-np.inf), dtype=np.float32)
    return v


def _round_index(c):
    t = (np.asarray(c, np.float32) + M).astype(np.float32)
    return t, t.view(np.uint32).astype(np.int64) - MAGIC


def test_rounding_to_the_cell_index():
    rng = np.random.default_rng(0)
    for n in (2, 3, 7, 64, 100, 1000):
        c = np.concatenate([rng.uniform(-0.5, n - 1.5, 20000).astype(np.float32),
                            np.array([-0.5, 0.0, 0.5, _upper(n)], np.float32)])
        c = c[c < f32(n - 1.5)]
        _, i = _round_index(c)
        assert i.min() >= 0 and i.max() <= n - 2, n
        assert np.all(np.abs(c.astype(np.float64) - i) <= 0.5)


def test_addresses_from_the_float_bits():
    rng = np.random.default_rng(1)
    for (R, Q) in ((2, 2), (5, 7), (64, 64), (100, 100)):
        for base in (0, 2368, 16 * int(rng.integers(0, 14000))):
            gx = rng.uniform(-0.5, Q - 1.5, 5000).astype(np.float32)
            gy = rng.uniform(-0.5, R - 1.5, 5000).astype(np.float32)
            tx, ix = _round_index(gx)
            ty, iy = _round_index(gy)
            k0 = (base - 8 * MAGIC * (Q + 1)) % 2 ** 32
            bx = tx.view(np.uint32).astype(np.uint64)
            by = ty.view(np.uint32).astype(np.uint64)
            addr = (by * np.uint64(8 * Q) + (bx * np.uint64(8) + np.uint64(k0))) % np.uint64(2 ** 32)
            np.testing.assert_array_equal(addr.astype(np.int64), base + 8 * (Q * iy + ix))
            top = base + 8 * (Q * iy + ix) + 8 * Q            # the record one row up
            assert top.max() + 8 <= base + 8 * R * Q


def test_upper_bound_stays_below_the_last_node():
    for n in (2, 3, 64, 100, 4096):
        _, i = _round_index(np.array([_upper(n)], np.float32))
        assert i[0] == n - 2


def _floor_index(c):
    """t = 1.5 * 2^23 + c rounded toward -infinity (ulp 1 there): exactly
    1.5 * 2^23 + floor(c)."""
    c = np.asarray(c, np.float32)
    t = (np.float64(M) + np.floor(c.astype(np.float64))).astype(np.float32)
    return t, t.view(np.uint32).astype(np.int64) - MAGIC


def test_floor_split_of_the_y_axis():
    rng = np.random.default_rng(2)
    for n in (2, 3, 7, 64, 100, 1000):
        top = np.nextafter(f32(n - 1), f32(-np.inf), dtype=np.float32)
        c = np.concatenate([rng.uniform(0.0, n - 1, 20000).astype(np.float32),
                            np.array([0.0, 0.5, 1.0, top], np.float32)])
        c = c[c < f32(n - 1)]
        t, i = _floor_index(c)
        assert i.min() >= 0 and i.max() <= n - 2, n
        f = (c - (t - M).astype(np.float32)).astype(np.float32)   # the kernel's fraction, in FP32
        np.testing.assert_array_equal(f.astype(np.float64), c.astype(np.float64) - i)  # exact
        assert f.min() >= 0.0 and f.max() < 1.0
    # the address algebra with a floored y and a rounded x
    R, Q, base = 64, 64, 4096
    gx = rng.uniform(-0.5, Q - 1.5, 5000).astype(np.float32)
    gy = rng.uniform(0.0, R - 1, 5000).astype(np.float32)
    tx, ix = _round_index(gx)
    ty, iy = _floor_index(gy)
    k0 = (base - 8 * MAGIC * (Q + 1)) % 2 ** 32
    bx = tx.view(np.uint32).astype(np.uint64)
    by = ty.view(np.uint32).astype(np.uint64)
    addr = (by * np.uint64(8 * Q) + (bx * np.uint64(8) + np.uint64(k0))) % np.uint64(2 ** 32)
    np.testing.assert_array_equal(addr.astype(np.int64), base + 8 * (Q * iy + ix))
