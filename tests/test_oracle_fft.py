"""Pins of the oracle's transforms (CPU only).

The I and J operators (JDFTx paper, Sec. 2.1) are discrete Fourier transforms
on the FFT box.  The oracle's recursive Cooley-Tukey routine is pinned to the
direct O(n^2) sum, to numpy's pocketfft (a library routine), to closed forms
for plane waves and deltas, to Parseval's identity, and its 3-D version to
the direct O(N^2) sum over tiny boxes.
"""
import numpy as np
import pytest

from oracle import cfft

rng = np.random.default_rng(7)


def crandn(*shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n", list(range(1, 41)) + [48, 54, 60, 64, 72, 80, 97, 128, 256])
def test_fft1d_equals_direct_sum(n):
    x = crandn(n)
    for sign in (+1, -1):
        ref = cfft.dft1d(x, sign)
        got = cfft.fft1d(x, sign)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [7, 16, 48, 60, 128])
def test_fft1d_matches_library(n):
    x = crandn(n)
    # numpy's forward transform uses exp(-2 pi i tm/n); its inverse is that with +, over n.
    assert np.allclose(cfft.fft1d(x, -1), np.fft.fft(x), rtol=0, atol=1e-12 * n)
    assert np.allclose(cfft.fft1d(x, +1), n * np.fft.ifft(x), rtol=0, atol=1e-12 * n)


def test_dft1d_delta_is_plane_wave():
    n, t0 = 12, 5
    x = np.zeros(n, complex)
    x[t0] = 1.0
    m = np.arange(n)
    assert np.allclose(cfft.dft1d(x, +1), np.exp(2j * np.pi * t0 * m / n), atol=1e-14)
    assert np.allclose(cfft.dft1d(x, -1), np.exp(-2j * np.pi * t0 * m / n), atol=1e-14)


@pytest.mark.parametrize("S", [(4, 6, 5), (8, 8, 8), (12, 10, 9), (3, 1, 7)])
def test_fft3d_equals_direct_3d_sum(S):
    a = crandn(*S)
    for sign in (+1, -1):
        ref = cfft.dft3d_direct(a, sign)
        got = cfft.fft3d(a, sign)
        assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_fft3d_delta_is_3d_plane_wave():
    S = (6, 4, 10)
    t = (2, 3, 7)
    a = np.zeros(S, complex)
    a[t] = 1.0
    j = np.stack(np.meshgrid(*[np.arange(s) for s in S], indexing="ij"), axis=-1)
    phase = sum(t[d] * j[..., d] / S[d] for d in range(3))
    assert np.allclose(cfft.fft3d(a, +1), np.exp(2j * np.pi * phase), atol=1e-14)


def test_fft3d_parseval_and_inverse():
    S = (16, 12, 15)
    N = np.prod(S)
    a = crandn(*S)
    A = cfft.fft3d(a, -1)
    assert np.isclose(np.sum(np.abs(A) ** 2), N * np.sum(np.abs(a) ** 2), rtol=1e-12)
    back = cfft.fft3d(A, +1) / N
    assert np.max(np.abs(back - a)) < 1e-13


def test_fft3d_batch_independent_boxes():
    a = crandn(3, 6, 5, 4)
    both = cfft.fft3d(a, +1)
    for c in range(3):
        assert np.allclose(both[c], cfft.fft3d(a[c], +1), atol=0, rtol=0)
