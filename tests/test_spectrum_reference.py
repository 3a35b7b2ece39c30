"""Pins of the radial power spectrum used as the reference for the device
spectra (tests/droplets.radial_spectrum): a single Fourier mode puts all its
power in the bin of its wavenumber, with the DFT's closed-form amplitude;
Parseval's theorem ties the binned sums to the field's variance; the mean
does not enter; and the bins count every integer wavevector once."""
import numpy as np

from tests import droplets


def _counts(nx, ny):
    k = np.hypot(*np.meshgrid(np.fft.fftfreq(nx) * nx, np.fft.fftfreq(ny) * ny))
    return np.bincount(np.rint(k).astype(int).ravel())


def test_single_mode_closed_form():
    nx, ny, a = 48, 32, 0.3
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    f = 2.0 + a * np.sin(2 * np.pi * (5 * x / nx - 2 * y / ny))
    s = droplets.radial_spectrum(f, 16)
    b = int(np.rint(np.hypot(5, 2)))
    c = _counts(nx, ny)
    # sin: |F(+-k)| = a nx ny / 2 at the two wavevectors, nothing elsewhere
    assert np.isclose(s[b], 2 * (a * nx * ny / 2) ** 2 / c[b], rtol=1e-12)
    assert np.all(np.delete(s, b) < 1e-20 * s[b])


def test_parseval_and_mean_removed():
    rng = np.random.default_rng(0)
    nx, ny = 32, 16
    f = 5.0 + rng.standard_normal((ny, nx))
    c = _counts(nx, ny)
    nb = len(c)  # every wavevector falls in some bin
    s = droplets.radial_spectrum(f, nb)
    total = (s * c[:nb]).sum()
    assert np.isclose(total, nx * ny * ((f - f.mean()) ** 2).sum(), rtol=1e-12)
    # a constant offset changes nothing
    assert np.allclose(droplets.radial_spectrum(f + 3.0, nb), s, rtol=1e-12, atol=1e-12 * s.max())
    assert c.sum() == nx * ny
