"""Seeded synthetic inputs for the Nystrom-preconditioned reconstruction workloads.

This module is shared by the tests, the benchmark and the CPU oracle.  It holds
only input data: phantoms, blur kernels, noise and the workload presets.  It
contains none of the method's arithmetic (no operator, sketch, factorisation,
preconditioner, prox or iteration), so neither side of a parity test can lean
on the other through it.

Phantoms stand in for the paper's test images, AAPM CT slices and walnut data
(Sec. IV), none of which are available.  Recipe:
  * shapes painted in order, later shapes overwrite earlier ones;
  * centres uniform in [-0.8, 0.8]^2, semi-axes uniform in [0.05, 0.4], angle
    uniform in [0, pi), all in units of half the image side; intensities
    uniform in [0, 1];
  * "mixed" phantoms pick rectangle or ellipse with probability 1/2;
  * the result is clipped to [0, 1].
Blur kernels are sampled Gaussians normalised to unit sum.  Noise is additive
Gaussian, or salt-and-pepper read the way the paper's footnote in Sec. IV-A
defines it: a fraction of pixels set to 1, then a disjoint fraction set to 0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def phantom(n: int, n_shapes: int, seed: int, kind: str = "ellipse") -> np.ndarray:
    """Random piecewise-constant phantom, float64 array of shape (n, n).

    kind: "ellipse" (all ellipses) or "mixed" (rectangle or ellipse, p = 1/2).
    Pixel (i, j) sits at y = (i - (n-1)/2)/(n/2), x = (j - (n-1)/2)/(n/2).
    """
    rng = np.random.default_rng(seed)
    img = np.zeros((n, n), dtype=np.float64)
    half = n / 2.0
    coords = (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) / half
    yy, xx = np.meshgrid(coords, coords, indexing="ij")
    for _ in range(n_shapes):
        cx, cy = rng.uniform(-0.8, 0.8, size=2)
        a, b = rng.uniform(0.05, 0.4, size=2)
        ang = rng.uniform(0.0, math.pi)
        val = rng.uniform(0.0, 1.0)
        rect = (kind == "mixed") and (rng.uniform() < 0.5)
        ca, sa = math.cos(ang), math.sin(ang)
        u = (xx - cx) * ca + (yy - cy) * sa
        v = -(xx - cx) * sa + (yy - cy) * ca
        if rect:
            mask = (np.abs(u) <= a) & (np.abs(v) <= b)
        else:
            mask = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        img[mask] = val
    return np.clip(img, 0.0, 1.0)


def gaussian_kernel(k: int, sigma: float) -> np.ndarray:
    """k x k sampled Gaussian, centred at ((k-1)/2, (k-1)/2), unit sum (float64)."""
    if k < 1 or k % 2 == 0:
        raise ValueError("kernel size must be odd and positive")
    c = (k - 1) / 2.0
    a = np.arange(k, dtype=np.float64) - c
    g = np.exp(-(a[:, None] ** 2 + a[None, :] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def random_kernel(k: int, seed: int) -> np.ndarray:
    """k x k non-separable positive kernel with unit sum (for general-stencil tests)."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.0, 1.0, size=(k, k))
    return h / h.sum()


def gaussian_noise(shape, sigma: float, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).normal(0.0, sigma, size=shape)


def salt_and_pepper(y: np.ndarray, frac: float, seed: int) -> np.ndarray:
    """Set a fraction `frac` of entries to 1, then a disjoint fraction to 0."""
    rng = np.random.default_rng(seed)
    out = np.array(y, dtype=np.float64, copy=True)
    flat = out.reshape(-1)
    m = flat.size
    k = int(round(frac * m))
    perm = rng.permutation(m)
    flat[perm[:k]] = 1.0
    flat[perm[k:2 * k]] = 0.0
    return out


def gaussian_probe_like(shape, seed: int) -> np.ndarray:
    """Plain seeded Gaussian test data (operator inputs for parity tests)."""
    return np.random.default_rng(seed).standard_normal(shape)


@dataclasses.dataclass(frozen=True)
class Workload:
    """A reconstruction workload: image, operator, regulariser and sketch size."""
    name: str
    n: int                      # image side (n x n)
    op: str                     # "blur", "blur_decim", "radon"
    reg: str                    # "wavelet", "tv", "hs"
    lam: float
    ell: int
    iters: int
    dtype: str                  # "f64" or "f32"
    blur_k: int = 0
    blur_sigma: float = 0.0
    decim: int = 1
    n_angles: int = 0
    n_bins: int = 0
    fit: str = "l2"             # "l2" or "huber"
    huber_delta: float = 0.0
    noise: str = "gauss"        # "gauss", "saltpepper", "gauss_rel"
    noise_level: float = 0.0
    phantom_kind: str = "ellipse"
    n_shapes: int = 30
    haar_levels: int = 3
    seed_phantom: int = 0
    seed_noise: int = 0
    seed_omega: int = 0
    n_inner: int = 20


# The four single-problem presets (the batched workload is batch_instances
# below).  Sizes, operators, regularisers, lambda, sketch size and iteration
# counts are the ones the reconstruction benchmark names.
DEBLUR64 = Workload(
    name="deblur64_haar_f64", n=64, op="blur", reg="wavelet", lam=1e-3, ell=32,
    iters=100, dtype="f64", blur_k=9, blur_sigma=1.5, noise="gauss",
    noise_level=0.01, phantom_kind="mixed", n_shapes=8, haar_levels=3,
    seed_phantom=1, seed_noise=2, seed_omega=3)

DEBLUR512 = Workload(
    name="deblur512_tv_f32", n=512, op="blur", reg="tv", lam=5e-4, ell=200,
    iters=300, dtype="f32", blur_k=25, blur_sigma=4.0, noise="gauss",
    noise_level=0.005, phantom_kind="ellipse", n_shapes=30,
    seed_phantom=11, seed_noise=12, seed_omega=13)

SUPERRES512 = Workload(
    name="superres4x_hs_huber_f32", n=512, op="blur_decim", reg="hs", lam=1e-3,
    ell=150, iters=300, dtype="f32", blur_k=7, blur_sigma=2.0, decim=4,
    fit="huber", huber_delta=0.01, noise="saltpepper", noise_level=0.10,
    phantom_kind="ellipse", n_shapes=30, seed_phantom=21, seed_noise=22,
    seed_omega=23)

CT512 = Workload(
    name="ct512_parallel_tv_f32", n=512, op="radon", reg="tv", lam=2e-4,
    ell=400, iters=300, dtype="f32", n_angles=720, n_bins=736,
    noise="gauss_rel", noise_level=0.01, phantom_kind="ellipse", n_shapes=30,
    seed_phantom=31, seed_noise=32, seed_omega=33)

PRESETS = {w.name: w for w in (DEBLUR64, DEBLUR512, SUPERRES512, CT512)}


def scaled(w: Workload, n: int, ell: int | None = None, iters: int | None = None,
           n_angles: int | None = None, n_bins: int | None = None) -> Workload:
    """A smaller copy of a preset (same recipe) for tests the oracle finishes fast."""
    kw = dict(n=n)
    if ell is not None:
        kw["ell"] = ell
    if iters is not None:
        kw["iters"] = iters
    if n_angles is not None:
        kw["n_angles"] = n_angles
    if n_bins is not None:
        kw["n_bins"] = n_bins
    return dataclasses.replace(w, **kw)


def blur_kernel_for(w: Workload) -> np.ndarray:
    return gaussian_kernel(w.blur_k, w.blur_sigma)


def ground_truth(w: Workload) -> np.ndarray:
    return phantom(w.n, w.n_shapes, w.seed_phantom, w.phantom_kind)


def degrade(w: Workload, clean_meas: np.ndarray) -> np.ndarray:
    """Noise the clean measurements A x_true (computed by the caller's operator)."""
    if w.noise == "gauss":
        return clean_meas + gaussian_noise(clean_meas.shape, w.noise_level, w.seed_noise)
    if w.noise == "gauss_rel":
        s = w.noise_level * float(np.max(np.abs(clean_meas)))
        return clean_meas + gaussian_noise(clean_meas.shape, s, w.seed_noise)
    if w.noise == "saltpepper":
        return salt_and_pepper(clean_meas, w.noise_level, w.seed_noise)
    raise ValueError(w.noise)


def batch_instances(count: int = 64, seed: int = 51, sizes=(128, 256, 384, 512), ells=(64, 128, 256),
                    angle_range=(180, 720)):
    """The batched, differentiated workload: `count` instances, alternately blur (Gaussian sigma ~ U[1, 4], kernel side
    2 ceil(3 sigma) + 1, noise 0.005, TV lambda 5e-4) and parallel-beam CT
    (angles ~ U{180..720} over 180 degrees, ceil(sqrt(2) n) + 2 bins, noise 1%
    of the sinogram maximum, TV lambda 2e-4), each kind cycling through the
    image sizes, sketch size drawn from `ells`.
    Returns plain dicts (seeded, no method arithmetic)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = sizes[(i // 2) % len(sizes)]
        inst = dict(index=i, n=n, ell=int(ells[rng.integers(len(ells))]), seed_phantom=1000 + i,
                    seed_noise=2000 + i, seed_omega=3000 + i)
        if i % 2 == 0:
            sigma = float(rng.uniform(1.0, 4.0))
            inst.update(op="blur", sigma=sigma, k=2 * int(np.ceil(3 * sigma)) + 1, lam=5e-4, noise=0.005)
        else:
            inst.update(op="radon", n_angles=int(rng.integers(angle_range[0], angle_range[1] + 1)),
                        n_bins=int(np.ceil(np.sqrt(2.0) * n)) + 2, lam=2e-4, noise=0.01)
        out.append(inst)
    return out


def batch_instance_data(inst: dict, apply_fn) -> tuple:
    """(x_true, y) of one batched instance: the phantom recipe at its size and
    the noisy measurements, with apply_fn(x_true) -> A x_true supplied by the
    caller's operator."""
    x_true = phantom(inst["n"], 30, inst["seed_phantom"], "ellipse")
    clean = np.asarray(apply_fn(x_true), dtype=np.float64)
    scale = inst["noise"] * (float(np.max(np.abs(clean))) if inst["op"] == "radon" else 1.0)
    return x_true, clean + gaussian_noise(clean.shape, scale, inst["seed_noise"])

