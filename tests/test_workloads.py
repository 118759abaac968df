"""The seeded synthetic inputs follow their stated recipe: phantoms painted
from the documented distributions, unit-sum Gaussian kernels of the stated
width, salt and pepper as two disjoint exact fractions, the four
single-problem presets with the sizes and parameters of the reconstruction
benchmark, and the 64-instance batched workload."""
import math

import numpy as np
import pytest

import workloads as WL


def test_phantom_is_seeded_piecewise_constant_in_unit_range():
    a = WL.phantom(96, 12, 7, "mixed")
    b = WL.phantom(96, 12, 7, "mixed")
    c = WL.phantom(96, 12, 8, "mixed")
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() <= 1.0
    assert len(np.unique(a)) <= 12 + 1                   # one value per shape plus the background


def test_single_ellipse_has_the_drawn_area_value_and_centre():
    # redraw the shape's parameters in the documented order and check the
    # painted area against pi a b (n/2)^2 (semi-axes in units of half the
    # side), to within the pixels along its boundary
    n, checked = 256, 0
    for seed in range(12):
        rng = np.random.default_rng(seed)
        cx, cy = rng.uniform(-0.8, 0.8, size=2)
        a, b = rng.uniform(0.05, 0.4, size=2)
        rng.uniform(0.0, math.pi)
        val = rng.uniform(0.0, 1.0)
        if max(abs(cx), abs(cy)) + max(a, b) > 0.98:
            continue                                       # may cross the image border
        img = WL.phantom(n, 1, seed, "ellipse")
        painted = img > 0
        area = math.pi * a * b * (n / 2) ** 2
        perimeter = 2 * math.pi * max(a, b) * (n / 2)
        assert abs(painted.sum() - area) <= perimeter, (seed, painted.sum(), area)
        assert np.allclose(img[painted], val)
        i, j = np.nonzero(painted)                         # row = y, column = x
        assert abs((j.mean() - (n - 1) / 2) / (n / 2) - cx) < 0.02
        assert abs((i.mean() - (n - 1) / 2) / (n / 2) - cy) < 0.02
        checked += 1
    assert checked >= 3


def test_gaussian_kernel_unit_sum_symmetric_and_width():
    for k, s in ((9, 1.5), (25, 4.0), (7, 2.0)):
        h = WL.gaussian_kernel(k, s)
        assert h.shape == (k, k)
        assert h.sum() == pytest.approx(1.0, abs=1e-15)
        assert np.allclose(h, h.T) and np.allclose(h, h[::-1, ::-1])
        assert np.linalg.matrix_rank(h, tol=1e-12 * h.max()) == 1       # separable
    # a kernel wide enough not to truncate: variance along one axis = sigma^2
    h = WL.gaussian_kernel(41, 3.0)
    a = np.arange(41) - 20.0
    assert (h.sum(1) * a ** 2).sum() == pytest.approx(9.0, rel=1e-9)
    with pytest.raises(ValueError):
        WL.gaussian_kernel(8, 1.0)


def test_salt_and_pepper_sets_two_disjoint_exact_fractions():
    y = np.random.default_rng(0).uniform(0.2, 0.8, (64, 50))
    z = WL.salt_and_pepper(y, 0.10, 5)
    k = int(round(0.10 * y.size))
    assert (z == 1.0).sum() == k and (z == 0.0).sum() == k
    changed = z != y
    assert changed.sum() == 2 * k
    assert np.array_equal(z[~changed], y[~changed])
    assert np.array_equal(z, WL.salt_and_pepper(y, 0.10, 5))


def test_relative_gaussian_noise_scales_with_the_maximum():
    w = WL.scaled(WL.CT512, 32)
    clean = np.full((400, 300), 3.0)
    clean[0, 0] = 50.0
    noise = WL.degrade(w, clean) - clean
    assert noise.std() == pytest.approx(0.01 * 50.0, rel=0.02)


def test_presets_carry_the_benchmark_configurations():
    c1, c2, c3, c4 = WL.DEBLUR64, WL.DEBLUR512, WL.SUPERRES512, WL.CT512
    assert (c1.n, c1.op, c1.reg, c1.lam, c1.ell, c1.iters, c1.dtype) == (64, "blur", "wavelet", 1e-3, 32, 100, "f64")
    assert (c1.blur_k, c1.blur_sigma, c1.haar_levels) == (9, 1.5, 3)
    assert (c2.n, c2.op, c2.reg, c2.lam, c2.ell, c2.iters, c2.dtype) == (512, "blur", "tv", 5e-4, 200, 300, "f32")
    assert (c2.blur_k, c2.blur_sigma) == (25, 4.0)
    assert (c3.n, c3.op, c3.reg, c3.lam, c3.ell, c3.decim) == (512, "blur_decim", "hs", 1e-3, 150, 4)
    assert (c3.blur_k, c3.blur_sigma, c3.fit, c3.huber_delta) == (7, 2.0, "huber", 0.01)
    assert (c3.noise, c3.noise_level) == ("saltpepper", 0.10)
    assert (c4.n, c4.op, c4.reg, c4.lam, c4.ell, c4.n_angles, c4.n_bins) == (512, "radon", "tv", 2e-4, 400, 720, 736)
    assert len(WL.PRESETS) == 4
    assert len({(w.seed_phantom, w.seed_noise, w.seed_omega) for w in WL.PRESETS.values()}) == 4


def test_batched_workload_recipe():
    inst = WL.batch_instances()
    assert len(inst) == 64 and inst == WL.batch_instances()
    assert [d["index"] for d in inst] == list(range(64))
    assert {d["n"] for d in inst} == {128, 256, 384, 512}
    assert all(d["ell"] in (64, 128, 256) for d in inst)
    assert len({d["seed_omega"] for d in inst}) == 64
    for d in inst:
        if d["index"] % 2 == 0:
            assert d["op"] == "blur" and 1.0 <= d["sigma"] <= 4.0
            assert d["k"] == 2 * math.ceil(3 * d["sigma"]) + 1 and d["k"] % 2 == 1
        else:
            assert d["op"] == "radon" and 180 <= d["n_angles"] <= 720
            assert d["n_bins"] == math.ceil(math.sqrt(2.0) * d["n"]) + 2
    # each kind cycles through every size
    for kind in ("blur", "radon"):
        assert {d["n"] for d in inst if d["op"] == kind} == {128, 256, 384, 512}
    x, y = WL.batch_instance_data(inst[0], lambda v: v)
    assert x.shape == (inst[0]["n"],) * 2 and y.shape == x.shape
    assert np.std(y - x) == pytest.approx(0.005, rel=0.05)
