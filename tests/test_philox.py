"""The host definition of the seeded start block (workloads/philox.py)
against the generator's published known-answer vectors, and the
distribution of the normals it yields (CPU)."""
import json
import os

import numpy as np
import pytest

from workloads import philox as PH

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.json")


def _vectors():
    with open(GOLDEN) as f:
        return json.load(f)["vectors"]


@pytest.mark.parametrize("v", _vectors())
def test_philox_known_answers(v):
    ctr = np.array([[int(x, 16) for x in v["ctr"]]], dtype=np.uint64)
    key = tuple(int(x, 16) for x in v["key"])
    out = PH.philox4x32(ctr, key)[0]
    assert [int(x) for x in out] == [int(x, 16) for x in v["out"]]


def test_philox_one_round_by_hand():
    # one round of counter (1, 2, 3, 4) under key (5, 6), multiplied out by hand
    p0, p1 = 1 * PH.M0, 3 * PH.M1
    want = [((p1 >> 32) ^ 2 ^ 5), p1 & 0xFFFFFFFF, ((p0 >> 32) ^ 4 ^ 6), p0 & 0xFFFFFFFF]
    got = PH.philox4x32(np.array([[1, 2, 3, 4]], dtype=np.uint64), (5, 6), rounds=1)[0]
    assert [int(x) for x in got] == want


def test_normals_moments_and_layout():
    n, m = 4001, 25                           # odd n * m: the last pair is half used
    X = PH.start_block_seeded(n, m, seed=123)
    assert X.shape == (m, n)
    z = X.ravel()
    N = z.size
    assert abs(z.mean()) < 5 / np.sqrt(N)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / N)
    assert abs(np.mean(z ** 4) - 3) < 0.1     # Gaussian kurtosis
    assert np.abs(z).max() < 8.6              # r <= sqrt(2 * 53 ln 2) ~ 8.57
    # element e is z0 (even) / z1 (odd) of pair e // 2
    z0, z1 = PH.normal_pairs(3, 123)
    assert np.array_equal(z[:6], np.array([z0[0], z1[0], z0[1], z1[1], z0[2], z1[2]]))
    # a different seed gives a different block; the same seed the same one
    assert not np.array_equal(X, PH.start_block_seeded(n, m, seed=124))
    assert np.array_equal(X, PH.start_block_seeded(n, m, seed=123))


def test_complex_block():
    Z = PH.start_block_seeded(1000, 12, seed=7, complex_=True)
    z0, z1 = PH.normal_pairs(12000, 7)
    assert np.array_equal(Z.ravel().real, z0 * PH.INV_SQRT2)
    assert np.array_equal(Z.ravel().imag, z1 * PH.INV_SQRT2)
    assert abs(np.mean(np.abs(Z) ** 2) - 1) < 0.05
