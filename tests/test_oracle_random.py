"""Pins of the oracle's counter-based random numbers (Philox4x32-10, Box-Muller).

The generator is not named by the paper (it only runs every simulation with
different process noise, Sec. VII-B/C); the oracle and the CUDA path each
implement Philox4x32-10 from Salmon et al. (SC'11).  Pinned here against the
published known-answer vectors, exact arithmetic of the 53-bit uniform, and
the distribution of the Box-Muller normals.
"""
import ctypes as C
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert oracle.philox(ctr, key) == out


def test_philox_counter_sensitivity():
    # every counter/key word must reach the output (a dropped word would not)
    base = oracle.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert oracle.philox(c, [5, 6]) != base
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert oracle.philox([1, 2, 3, 4], k) != base


def test_uniform52_exact_values():
    L = oracle.lib()
    assert L.or_uniform52(0, 0) == 0.5 * 2.0 ** -52
    top = L.or_uniform52(0xFFFFFFFF, 0xFFFFFFFF)
    assert top == 1.0 - 2.0 ** -53
    assert 0.0 < top < 1.0
    # 26 high bits of hi and of lo; low bits ignored
    assert L.or_uniform52(1 << 6, 0) == (2.0 ** 26 + 0.5) * 2.0 ** -52
    assert L.or_uniform52(0, 1 << 6) == 1.5 * 2.0 ** -52
    assert L.or_uniform52(63, 63) == L.or_uniform52(0, 0)


def _normals(n, seed=7):
    L = oracle.lib()
    out = np.empty((n, 2))
    z = np.zeros(2)
    for i in range(n):
        w = oracle.philox([i, 3, 9, 0], [seed, 0])
        L.or_normal_pair((C.c_uint32 * 4)(*w), z.ctypes.data_as(C.POINTER(C.c_double)))
        out[i] = z
    return out


def test_box_muller_distribution():
    from scipy import stats

    z = _normals(100000)
    for col in range(2):
        x = z[:, col]
        assert abs(x.mean()) < 5.0 / math.sqrt(len(x))
        assert abs(x.var() - 1.0) < 0.02
        assert stats.kstest(x, "norm").pvalue > 1e-3
    # the two members of a pair are uncorrelated
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.02


def test_noise_streams_layout():
    """Process noise of substep k of trajectory j uses counters (k, j, 0, 0) and
    (k, j, 1, 0); the measurement of step i uses (i, j, 2, 0); all with key
    (seed_lo, seed_hi)."""
    L = oracle.lib()
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    j, k = 17, 1234
    xi = np.zeros(3)
    L.or_process_noise(seed, j, k, xi.ctypes.data_as(C.POINTER(C.c_double)))
    z = np.zeros(2)
    dp = C.POINTER(C.c_double)
    w = oracle.philox([k, j, 0, 0], key)
    L.or_normal_pair((C.c_uint32 * 4)(*w), z.ctypes.data_as(dp))
    assert xi[0] == z[0] and xi[1] == z[1]
    w = oracle.philox([k, j, 1, 0], key)
    L.or_normal_pair((C.c_uint32 * 4)(*w), z.ctypes.data_as(dp))
    assert xi[2] == z[0]
    w = oracle.philox([k, j, 2, 0], key)
    L.or_normal_pair((C.c_uint32 * 4)(*w), z.ctypes.data_as(dp))
    assert L.or_meas_noise(seed, j, k) == z[0]


def test_process_noise_independent_across_trajectories():
    L = oracle.lib()
    dp = C.POINTER(C.c_double)
    a = np.zeros((2000, 3))
    for j in range(2000):
        xi = np.zeros(3)
        L.or_process_noise(5, j, 11, xi.ctypes.data_as(dp))
        a[j] = xi
    c = np.corrcoef(a.T)
    assert np.all(np.abs(c - np.eye(3)) < 0.1)
    assert np.all(np.abs(a.mean(axis=0)) < 0.1)
