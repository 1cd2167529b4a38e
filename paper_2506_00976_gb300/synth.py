"""Seeded synthetic grid measures that stand in for the DOTmark images.

This module generates inputs only: it holds none of the bound computation, and
both the CUDA library's tests and the oracle's tests draw their inputs from it.
Every measure is float64, non-negative, row-major N x N, normalised to mass 1.

Value classes (the paper evaluates 10 images per class, all 45 pairs, Sec. 5):
  white  -- i.i.d. uniform (0, 1] per pixel;
  gauss  -- K ~ U{1..10} isotropic Gaussian blobs, centres uniform on the
            grid, sigma ~ U[2, 6] * N/32 px, amplitudes U[0.5, 1], plus a
            1e-3 floor per pixel;
  cauchy -- the same with the profile 1 / (1 + r^2 / gamma^2),
            gamma ~ U[2, 6] * N/32 px, plus the 1e-3 floor;
  field  -- exp(z) for z a Gaussian-filtered (sigma = 4 px, reflect) standard
            normal field rescaled to unit variance.
The small blob case (``blobs3``) is three Gaussian blobs of amplitude 1 with
sigma ~ U[2, 6] px plus the 1e-3 floor.

Volumes (N x N x N, flat row-major, for the 3-D experiments of the paper, whose
cryo-EM density maps are not available here):
  density -- a compact "molecule": K ~ U{8..24} Gaussian blobs with centres
             drawn around the volume centre (normal, sd N/6, clipped to the
             grid), sigma ~ U[1, 2.5] * N/16 voxels, amplitudes U[0.5, 1],
             plus a 1e-3 floor per voxel;
  field3  -- exp(z) for z a Gaussian-filtered (sigma = 2 voxels, reflect)
             standard normal volume rescaled to unit variance.

Seeds: numpy PCG64 over SeedSequence([250600976, workload, class, image]).
"""
from __future__ import annotations

import itertools

import numpy as np

CLASSES = ("white", "gauss", "cauchy", "field")
_CLASS_ID = {"white": 0, "gauss": 1, "cauchy": 2, "field": 3, "blobs3": 4,
             "density": 5, "field3": 6}
VOLUME_CLASSES = ("density", "field3")
_ROOT_SEED = 250600976


def _rng(workload: int, cls: str, image: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(
        np.random.SeedSequence([_ROOT_SEED, int(workload), _CLASS_ID[cls], int(image)])))


def _blobs(rng, N, count, profile, amp_lo, amp_hi, scale_lo, scale_hi):
    r, c = np.meshgrid(np.arange(N, dtype=np.float64), np.arange(N, dtype=np.float64),
                       indexing="ij")
    img = np.full((N, N), 1e-3)
    for _ in range(count):
        cr, cc = rng.uniform(0.0, N, size=2)
        s = rng.uniform(scale_lo, scale_hi)
        amp = 1.0 if amp_lo == amp_hi else rng.uniform(amp_lo, amp_hi)
        d2 = (r - cr) ** 2 + (c - cc) ** 2
        if profile == "gauss":
            img += amp * np.exp(-0.5 * d2 / (s * s))
        else:
            img += amp / (1.0 + d2 / (s * s))
    return img


def make_measure(N: int, cls: str, workload: int = 0, image: int = 0) -> np.ndarray:
    """One seeded N x N measure of class ``cls`` as a flat float64 array of mass 1."""
    rng = _rng(workload, cls, image)
    scale = N / 32.0
    if cls == "white":
        img = 1.0 - rng.random((N, N))                 # uniform on (0, 1]
    elif cls == "gauss":
        img = _blobs(rng, N, int(rng.integers(1, 11)), "gauss", 0.5, 1.0,
                     2.0 * scale, 6.0 * scale)
    elif cls == "cauchy":
        img = _blobs(rng, N, int(rng.integers(1, 11)), "cauchy", 0.5, 1.0,
                     2.0 * scale, 6.0 * scale)
    elif cls == "blobs3":
        img = _blobs(rng, N, 3, "gauss", 1.0, 1.0, 2.0, 6.0)
    elif cls == "field":
        from scipy.ndimage import gaussian_filter
        z = gaussian_filter(rng.standard_normal((N, N)), sigma=4.0, mode="reflect")
        z = (z - z.mean()) / z.std()
        img = np.exp(z)
    else:
        raise ValueError(f"unknown class {cls!r}")
    img = img.ravel()
    return img / img.sum()


def make_volume(N: int, cls: str, workload: int = 0, image: int = 0) -> np.ndarray:
    """One seeded N x N x N measure of class ``cls`` as a flat float64 array of mass 1."""
    rng = _rng(workload, cls, image)
    if cls == "density":
        x = np.arange(N, dtype=np.float64)
        a, b, c = np.meshgrid(x, x, x, indexing="ij")
        vol = np.full((N, N, N), 1e-3)
        for _ in range(int(rng.integers(8, 25))):
            ctr = np.clip(rng.normal((N - 1) / 2.0, N / 6.0, size=3), 0.0, N - 1.0)
            s = rng.uniform(1.0, 2.5) * N / 16.0
            amp = rng.uniform(0.5, 1.0)
            d2 = (a - ctr[0]) ** 2 + (b - ctr[1]) ** 2 + (c - ctr[2]) ** 2
            vol += amp * np.exp(-0.5 * d2 / (s * s))
    elif cls == "field3":
        from scipy.ndimage import gaussian_filter
        z = gaussian_filter(rng.standard_normal((N, N, N)), sigma=2.0, mode="reflect")
        z = (z - z.mean()) / z.std()
        vol = np.exp(z)
    else:
        raise ValueError(f"unknown volume class {cls!r}")
    vol = vol.ravel()
    return vol / vol.sum()


def volume_pairs(N: int, cls: str, workload: int, count: int = 10):
    """All 45 pairs (mu, nu) of ``count`` volumes of one class, in a fixed order."""
    vols = [make_volume(N, cls, workload, i) for i in range(count)]
    return [(vols[i], vols[j]) for i, j in all_pairs(count)]


def class_images(N: int, cls: str, workload: int, count: int = 10):
    return [make_measure(N, cls, workload, i) for i in range(count)]


def all_pairs(count: int = 10):
    """The 45 unordered pairs (i, j), i < j, of ``count`` images."""
    return list(itertools.combinations(range(count), 2))


def class_pairs(N: int, cls: str, workload: int, count: int = 10):
    """All 45 pairs (mu, nu) of one class, in a fixed order."""
    imgs = class_images(N, cls, workload, count)
    return [(imgs[i], imgs[j]) for i, j in all_pairs(count)]


def uneven_workload(n_pairs: int = 200, workload: int = 3):
    """Pairs with N ~ U{32,64,128,256}, kappa ~ U{4,8}, p ~ U{1,2}, class ~ U(4 classes)."""
    rng = _rng(workload, "white", 10**6)
    out = []
    for t in range(n_pairs):
        N = int(rng.choice([32, 64, 128, 256]))
        kappa = int(rng.choice([4, 8]))
        p = float(rng.choice([1, 2]))
        cls = CLASSES[int(rng.integers(0, 4))]
        mu = make_measure(N, cls, workload, 2 * t)
        nu = make_measure(N, cls, workload, 2 * t + 1)
        out.append({"N": N, "kappa": kappa, "p": p, "cls": cls, "mu": mu, "nu": nu})
    return out


def gaussian_offset_kernel(kappa: int, sigma: float) -> np.ndarray:
    """An upscaling kernel input: K[u, v] over the in-block offsets u, v
    (row-major in the kappa x kappa block) proportional to
    exp(-|u - v|^2 / (2 sigma^2)), scaled to sum 1 -- an input of the
    general-kernel primal pass, like the measures above."""
    g = np.arange(kappa)
    r, c = np.repeat(g, kappa), np.tile(g, kappa)
    d2 = (r[:, None] - r[None, :]) ** 2 + (c[:, None] - c[None, :]) ** 2
    K = np.exp(-d2 / (2.0 * sigma * sigma))
    return K / K.sum()
