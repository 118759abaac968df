"""Pins for the oracle's Gaussian test matrix (Algorithm 1 step 1)."""
import os

import numpy as np
import pytest
import scipy.stats

from oracle.philox import gaussian_matrix, philox4x32_10

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    got = philox4x32_10(np.array([ctr], dtype=np.uint64), np.array([key], dtype=np.uint64))[0]
    assert [int(v) for v in got] == out


def test_gaussian_moments_and_normality():
    z = gaussian_matrix(4096, 50, seed=3).ravel()
    assert abs(z.mean()) < 4.0 / np.sqrt(z.size) * 1.5
    assert abs(z.var() - 1.0) < 0.02
    # Kolmogorov-Smirnov against N(0, 1)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    # columns are uncorrelated
    Om = gaussian_matrix(4096, 8, seed=5)
    C = Om @ Om.T / 4096
    assert np.max(np.abs(C - np.eye(8))) < 0.1


def test_gaussian_layout_is_prefix_stable():
    # element (j, i) depends only on the flat index j*N + i and the seed
    a = gaussian_matrix(10, 3, seed=9).ravel()
    b = gaussian_matrix(6, 5, seed=9).ravel()
    assert np.array_equal(a, b[: a.size])
    assert not np.array_equal(gaussian_matrix(10, 3, seed=10), gaussian_matrix(10, 3, seed=9))
