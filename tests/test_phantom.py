"""The seeded synthetic inputs follow their stated recipe: deterministic per
(config, slice, coil), centred k-space of the coil image, complex Gaussian
noise at the requested SNR, bounded Gaussian coil sensitivities, unit-variance
generic test values."""
import numpy as np
import pytest

from paper_2512_04317_gb300 import phantom


def test_deterministic_and_distinct_per_slice():
    a = phantom.mri_batch(64, 32, 3, 2, config_id=7)
    b = phantom.mri_batch(64, 32, 3, 2, config_id=7)
    assert a.dtype == np.complex64 and a.shape == (6, 64, 32)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert not np.array_equal(a[0], a[2])            # slice 0 vs slice 1, coil 0
    assert not np.array_equal(a[0], a[1])            # coil 0 vs coil 1
    c = phantom.mri_batch(64, 32, 3, 2, config_id=8)
    assert not np.array_equal(a, c)


@pytest.mark.parametrize("snr_db", [30.0, 10.0])
def test_noise_at_the_requested_snr(snr_db):
    n0, n1 = 128, 96
    noisy = phantom.mri_batch(n0, n1, 1, 1, config_id=3, snr_db=snr_db)[0].astype(np.complex128)
    clean = np.fft.fftshift(np.fft.fft2(phantom.phantom_image(n0, n1, 3, 0)))
    noise = noisy - clean
    snr = 10 * np.log10(np.mean(np.abs(clean) ** 2) / np.mean(np.abs(noise) ** 2))
    assert abs(snr - snr_db) < 0.3, snr
    # complex Gaussian: real and imaginary parts of equal power
    pr, pi = np.mean(noise.real ** 2), np.mean(noise.imag ** 2)
    assert 0.9 < pr / pi < 1.1


def test_kspace_is_centred():
    n0, n1 = 128, 128
    k = phantom.mri_batch(n0, n1, 2, 1, config_id=1)
    for s in range(2):
        r, c = np.unravel_index(np.argmax(np.abs(k[s])), k[s].shape)
        assert abs(r - n0 // 2) <= 2 and abs(c - n1 // 2) <= 2


def test_image_domain_input_is_the_noisy_coil_image():
    n0, n1 = 64, 64
    img = phantom.mri_batch(n0, n1, 1, 1, config_id=2, domain="image")[0].astype(np.complex128)
    clean = phantom.phantom_image(n0, n1, 2, 0)
    snr = 10 * np.log10(np.mean(np.abs(clean) ** 2) / np.mean(np.abs(img - clean) ** 2))
    assert abs(snr - 30.0) < 0.5
    # the body ellipse: the centre is brighter than the corners
    assert np.abs(clean[n0 // 2 - 4:n0 // 2 + 4, n1 // 2 - 4:n1 // 2 + 4]).mean() > \
        5 * np.abs(clean[:4, :4]).mean()


def test_coil_maps():
    m = phantom.coil_maps(96, 96, 8, config_id=4)
    assert m.shape == (8, 96, 96)
    assert np.all(np.abs(m) <= 1.0 + 1e-12)
    # coil c peaks on the side of the field of view facing its centre on the
    # circle of radius 1.2 at angle about 2 pi c / 8
    X, Y = np.meshgrid((np.arange(96) + 0.5) / 96 * 2 - 1, (np.arange(96) + 0.5) / 96 * 2 - 1)
    for c in range(8):
        r, q = np.unravel_index(np.argmax(np.abs(m[c])), (96, 96))
        ang = np.arctan2(Y[r, q], X[r, q])
        d = np.angle(np.exp(1j * (ang - 2 * np.pi * c / 8)))
        assert abs(d) < 0.5, (c, d)
    # the multi-coil batch is the coil image, coil by coil
    k = phantom.mri_batch(96, 96, 1, 8, config_id=4, domain="image", snr_db=200.0)
    img = phantom.phantom_image(96, 96, 4, 0)
    for c in range(8):
        np.testing.assert_allclose(k[c], (img * m[c]).astype(np.complex64), rtol=0, atol=1e-6)


def test_random_complex_unit_variance():
    z = phantom.random_complex((256, 256), seed=1).astype(np.complex128)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.02
    assert abs(np.mean(z)) < 0.02
