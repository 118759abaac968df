"""Pins for the oracle's orthonormal filter-bank wavelets (Haar and
Daubechies-4, the wavelet of the paper's CT experiments).

* the generic filter bank with the Haar taps reproduces the separately
  written Haar transform;
* the Daubechies-4 taps satisfy the published conditions: sum sqrt 2, unit
  energy, orthogonality to their even shifts, and a high-pass with two
  vanishing moments;
* W is orthonormal (norm preserved, W^T W = W W^T = I) at several depths and
  on non-square images;
* two vanishing moments: a one-level transform of an image that is linear
  along its columns has zero column details away from the periodic wrap, and
  a constant image keeps only its coarsest low-low block (c 2^levels).
"""
import math

import numpy as np
import pytest

from oracle import operators as ops


def test_generic_filter_bank_with_haar_taps_is_the_haar_transform():
    x = np.random.default_rng(0).standard_normal((2, 16, 24))
    for levels in (1, 2, 3):
        a = ops.wavelet_forward(x, levels, "haar")
        b = ops.haar_forward(x, levels)
        assert np.abs(a - b).max() <= 1e-14
        assert np.abs(ops.wavelet_adjoint(a, levels, "haar") - ops.haar_adjoint(b, levels)).max() <= 1e-14


def test_daubechies4_taps():
    h = ops.WAVELET_TAPS["db4"]
    g = ops.qmf_highpass(h)
    assert h.sum() == pytest.approx(math.sqrt(2.0), abs=1e-15)
    assert np.dot(h, h) == pytest.approx(1.0, abs=1e-15)
    assert np.dot(h[:2], h[2:]) == pytest.approx(0.0, abs=1e-15)      # orthogonal to its shift by 2
    k = np.arange(4)
    assert g.sum() == pytest.approx(0.0, abs=1e-15)
    assert np.dot(k, g) == pytest.approx(0.0, abs=1e-14)              # two vanishing moments
    assert np.dot(k * k, g) != pytest.approx(0.0, abs=1e-3)           # not three
    assert np.dot(h, g) == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("shape,levels", [((32, 32), 1), ((32, 48), 3), ((16, 8), 3), ((64, 64), 4)])
def test_daubechies4_is_orthonormal(shape, levels):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3,) + shape)
    c = ops.wavelet_forward(x, levels, "db4")
    assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    assert np.abs(ops.wavelet_adjoint(c, levels, "db4") - x).max() <= 1e-13
    y = rng.standard_normal(shape)
    assert np.abs(ops.wavelet_forward(ops.wavelet_adjoint(y, levels, "db4"), levels, "db4") - y).max() <= 1e-13
    # adjoint identity <W x, y> = <x, W^T y>
    assert np.sum(c[0] * y) == pytest.approx(np.sum(x[0] * ops.wavelet_adjoint(y, levels, "db4")), rel=1e-12)


def test_daubechies4_vanishing_moments_and_constants():
    n1, n2 = 8, 32
    x = np.tile(0.3 + 0.7 * np.arange(n2), (n1, 1))                 # linear along the columns
    c = ops.wavelet_forward(x, 1, "db4")
    col_detail = c[: n1 // 2, n2 // 2:]
    assert np.abs(col_detail[:, :-1]).max() <= 1e-12                # the last one straddles the wrap
    assert np.abs(col_detail[:, -1]).max() > 1.0
    const = np.full((16, 16), 2.5)
    c = ops.wavelet_forward(const, 3, "db4")
    assert np.allclose(c[:2, :2], 2.5 * 8.0, atol=1e-12)
    c[:2, :2] = 0.0
    assert np.abs(c).max() <= 1e-12
