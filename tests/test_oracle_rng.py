"""Pins for the oracle's counter-based RNG (Philox4x32-10, section 3.6's need
for independent, evenly distributed per-star streams)."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest


def _curand_host():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and (os.path.exists(cand) or not cand.startswith("/")):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 2**64 - 1])
@pytest.mark.parametrize("offset_blocks", [0, 5, 12_345_678, (5 << 48) + 12_345])
def test_philox_matches_curand_host_generator(orc, seed, offset_blocks):
    """cuRAND's host Philox4_32_10 generator (run, not read) emits block j of
    its stream as Philox4x32-10 of the counter (j >> 16 as words 0-1,
    j mod 2^16 as word 2, 0) with key = seed; the oracle must reproduce it
    word for word.  This pins the round function, both multipliers, the key
    schedule and counter words 0, 1 and 2."""
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * offset_blocks)) == 0
        n = 4 * 512
        buf = (ctypes.c_uint * n)()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    cur = np.array(buf[:], dtype=np.uint32).reshape(-1, 4)
    blk = np.uint64(offset_blocks) + np.arange(cur.shape[0], dtype=np.uint64)
    hi = blk >> np.uint64(16)
    ctr = np.zeros((cur.shape[0], 4), np.uint32)
    ctr[:, 0] = (hi & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctr[:, 1] = (hi >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = (blk & np.uint64(0xFFFF)).astype(np.uint32)
    np.testing.assert_array_equal(orc.philox(ctr, seed), cur)


def test_u01_exact_endpoints(orc):
    assert orc.u01(0, 0) == 2.0 ** -53
    assert orc.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # only the top 52 bits matter
    assert orc.u01(0xFFF, 0) == 2.0 ** -53
    assert orc.u01(0x1000, 0) == 3.0 * 2.0 ** -53


@pytest.mark.parametrize("tag", [0, 1, 2, 3])
def test_uniform_statistics(orc, tag):
    n = 1 << 18
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 1] = 7
    ctr[:, 2] = tag
    w = orc.philox(ctr, 12345)
    u = ((((w[:, 1].astype(np.uint64) << np.uint64(32)) | w[:, 0]) >> np.uint64(12))
         .astype(np.float64) * 2 + 1) * 2.0 ** -53
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 0.01 / 12
    counts = np.histogram(u, bins=64, range=(0, 1))[0]
    chi2 = ((counts - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 120  # 63 d.o.f.; p ~ 1e-5
    # 32-bit words are balanced bit by bit
    bits = np.unpackbits(w.view(np.uint8)).reshape(-1, 8)
    assert np.all(np.abs(bits.mean(axis=0) - 0.5) < 0.005)


def test_disk_angle_is_unit_and_uniform(orc):
    ang = []
    for i in range(20000):
        c, s, rc = orc.disk_angle(99, i, 3, 0)
        assert rc == 0
        assert abs(c * c + s * s - 1.0) < 1e-15
        ang.append(np.arctan2(s, c))
    ang = np.array(ang)
    counts = np.histogram(ang, bins=32, range=(-np.pi, np.pi))[0]
    chi2 = ((counts - len(ang) / 32) ** 2 / (len(ang) / 32)).sum()
    assert chi2 < 70
    assert abs(np.cos(ang).mean()) < 0.03 and abs(np.sin(ang).mean()) < 0.03


def test_disk_test_integer_band_argument():
    """The unit-disk acceptance (u u + v v <= 1 in FP64, u = U 2^-52 with U
    odd and |U| < 2^52) agrees with the exact integer test U^2 + V^2 <=
    2^104 wherever |U^2 + V^2 - 2^104| > 2^54: the FP64 sum of two rounded
    squares below 1 is within 2^-51 of the exact one.  Near-boundary pairs
    (B the integer square root of 2^104 - A^2, and B + 2) exercise both
    sides of the circle; inside the band the two tests do disagree, which is
    why the FP64 expression decides there."""
    import math
    rng = np.random.default_rng(11)
    T, band = 1 << 104, 1 << 54
    outside = disagree_in_band = 0
    for A in rng.integers(1 << 40, 1 << 52, 20000):
        A = int(A) | 1
        B0 = math.isqrt(T - A * A)
        for B in (B0 - 2, B0 - 1, B0, B0 + 1, B0 + 2):
            if B <= 0 or B >= 1 << 52:
                continue
            S = A * A + B * B
            u, v = A * 2.0 ** -52, B * 2.0 ** -52  # exact
            fp = (u * u) + (v * v) <= 1.0
            exact = S <= T
            if abs(S - T) > band:
                outside += 1
                assert fp == exact, (A, B)
            elif fp != exact:
                disagree_in_band += 1
    assert outside > 10000
    assert disagree_in_band > 0
