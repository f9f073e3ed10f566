"""Seeded synthetic MRI inputs: random-ellipse phantoms, coil maps, k-space.

This module only manufactures inputs.  It holds none of the MX-FFT arithmetic
and is shared by the CUDA path's tests and benchmark and by the CPU oracle's
tests, so both sides see identical bytes.

The public MRI datasets the paper evaluates on (fastMRI brain, SKM-TEA knee;
Sec. 2.3) are not available here; these phantoms stand in for them with the
same structure: fully sampled, centred, multi-coil complex k-space of smooth
anatomy-like images with smooth phase and complex Gaussian noise.

Recipe (all FP64, cast to complex64 at the end):
  * image on [-1, 1]^2 sampled at pixel centres: a body ellipse (semi-axes
    U(0.6, 0.9), intensity 1) plus 7 ellipses (centres U(-0.6, 0.6), semi-axes
    U(0.05, 0.5), rotation U(0, pi), additive intensity U(-0.4, 0.6));
  * smooth phase pi * (c1 x + c2 y + c3 x y + c4 x^2 + c5 y^2), c ~ U(-0.5, 0.5);
  * coil c of C: Gaussian sensitivity exp(-|r - r_c|^2 / (2 w^2)) e^{i psi_c},
    r_c on the circle of radius 1.2 at angle 2 pi c / C + U(-0.1, 0.1),
    w ~ U(0.6, 1.0), psi_c ~ U(0, 2 pi);
  * k-space = fftshift(fft2(coil image)) (centred k-space, no normalisation);
  * complex Gaussian noise n = sigma (g1 + i g2) / sqrt(2) at an SNR of
    10 log10(mean |K|^2 / sigma^2) dB (30 dB by default).
Seeds: numpy SeedSequence([BASE_SEED, config_id, slice, coil]).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20251204


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([BASE_SEED, *[int(k) for k in key]]))


def _grid(n0: int, n1: int):
    y = (np.arange(n0) + 0.5) / n0 * 2.0 - 1.0
    x = (np.arange(n1) + 0.5) / n1 * 2.0 - 1.0
    return np.meshgrid(x, y)  # X varies along n1 (columns), Y along n0 (rows)


def phantom_image(n0: int, n1: int, config_id: int = 0, slice_id: int = 0,
                  n_ellipses: int = 8) -> np.ndarray:
    """Complex128 image [n0, n1]: ellipse magnitude times a smooth phase."""
    rng = _rng(config_id, slice_id, 1_000_000)
    X, Y = _grid(n0, n1)
    img = np.zeros((n0, n1))
    for e in range(n_ellipses):
        if e == 0:
            cx = cy = 0.0
            ax, ay = rng.uniform(0.6, 0.9, size=2)
            th, val = 0.0, 1.0
        else:
            cx, cy = rng.uniform(-0.6, 0.6, size=2)
            ax, ay = rng.uniform(0.05, 0.5, size=2)
            th = rng.uniform(0.0, np.pi)
            val = rng.uniform(-0.4, 0.6)
        c, s = np.cos(th), np.sin(th)
        xr = (X - cx) * c + (Y - cy) * s
        yr = -(X - cx) * s + (Y - cy) * c
        img += val * ((xr / ax) ** 2 + (yr / ay) ** 2 <= 1.0)
    cph = rng.uniform(-0.5, 0.5, size=5)
    phase = np.pi * (cph[0] * X + cph[1] * Y + cph[2] * X * Y + cph[3] * X**2 + cph[4] * Y**2)
    return img * np.exp(1j * phase)


def coil_maps(n0: int, n1: int, ncoils: int, config_id: int = 0) -> np.ndarray:
    """Complex128 Gaussian coil sensitivities [ncoils, n0, n1]."""
    X, Y = _grid(n0, n1)
    maps = np.empty((ncoils, n0, n1), np.complex128)
    for c in range(ncoils):
        rng = _rng(config_id, 2_000_000, c)
        ang = 2.0 * np.pi * c / max(ncoils, 1) + rng.uniform(-0.1, 0.1)
        rx, ry = 1.2 * np.cos(ang), 1.2 * np.sin(ang)
        w = rng.uniform(0.6, 1.0)
        psi = rng.uniform(0.0, 2.0 * np.pi)
        maps[c] = np.exp(-((X - rx) ** 2 + (Y - ry) ** 2) / (2.0 * w * w)) * np.exp(1j * psi)
    return maps


def add_noise(z: np.ndarray, snr_db: float, rng: np.random.Generator) -> np.ndarray:
    """Complex Gaussian noise at 10 log10(mean|z|^2 / sigma^2) = snr_db."""
    p = float(np.mean(np.abs(z) ** 2))
    sigma = np.sqrt(p / 10.0 ** (snr_db / 10.0))
    g = rng.standard_normal(z.shape) + 1j * rng.standard_normal(z.shape)
    return z + sigma * g / np.sqrt(2.0)


def mri_batch(n0: int, n1: int, nslices: int = 1, ncoils: int = 1,
              config_id: int = 0, domain: str = "kspace", snr_db: float = 30.0,
              single_coil_maps: bool = False) -> np.ndarray:
    """complex64 [nslices * ncoils, n0, n1], slice-major then coil.

    domain="kspace": centred k-space (the forward-transform input).
    domain="image":  the noisy coil image (the round-trip input).
    With ncoils == 1 and single_coil_maps False the coil map is 1.
    """
    out = np.empty((nslices * ncoils, n0, n1), np.complex64)
    maps = coil_maps(n0, n1, ncoils, config_id) if (ncoils > 1 or single_coil_maps) else None
    for s in range(nslices):
        img = phantom_image(n0, n1, config_id, s)
        for c in range(ncoils):
            coil_img = img * maps[c] if maps is not None else img
            rng = _rng(config_id, s, c)
            if domain == "kspace":
                z = np.fft.fftshift(np.fft.fft2(coil_img))
            elif domain == "image":
                z = coil_img
            else:
                raise ValueError(domain)
            out[s * ncoils + c] = add_noise(z, snr_db, rng).astype(np.complex64)
    return out


def random_complex(shape, seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """complex64 standard complex Gaussian values (generic test input)."""
    rng = _rng(9_000_000, seed)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return (scale * z / np.sqrt(2.0)).astype(np.complex64)
