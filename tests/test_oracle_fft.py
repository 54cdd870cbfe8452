"""Pins of the oracle's transforms against definitions and library routines.

The oracle's FFT is its own textbook code; these tests tie it to the DFT
definition (brute force), to numpy's pocketfft, to Parseval, the impulse and
shift theorems, and its DCT-I to scipy's REDFT00 and to the even-extension DFT
that Sec. 2.4 of the paper relies on.
"""
import numpy as np
import pytest
import scipy.fft


def _is_235_smooth(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


SMOOTH = [n for n in range(1, 65) if _is_235_smooth(n)]


def _rand(n, seed=0):
    r = np.random.default_rng(seed)
    return r.standard_normal(n) + 1j * r.standard_normal(n)


@pytest.mark.parametrize("n", SMOOTH + [7, 11, 13, 14, 49])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_equals_direct_dft(orc, n, sign):
    x = _rand(n, n)
    a = orc.fft1d(x, sign)
    b = orc.dft1d(x, sign)
    assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))


def test_direct_dft_matches_definition_sign(orc):
    # exp(-2 pi i j k / n) for the forward sign: impulse at j=1 gives the roots.
    n = 12
    x = np.zeros(n, complex)
    x[1] = 1.0
    k = np.arange(n)
    assert np.allclose(orc.dft1d(x, -1), np.exp(-2j * np.pi * k / n), atol=1e-15)
    assert np.allclose(orc.dft1d(x, +1), np.exp(+2j * np.pi * k / n), atol=1e-15)


@pytest.mark.parametrize("n", [96, 128, 160, 192, 256, 320, 384, 512, 1000, 1024, 2048])
def test_fft_matches_pocketfft(orc, n):
    x = _rand(n, 7)
    assert np.max(np.abs(orc.fft1d(x, -1) - np.fft.fft(x))) <= 1e-13 * np.sqrt(n) * np.max(np.abs(x)) * 4
    assert np.max(np.abs(orc.fft1d(x, +1) - n * np.fft.ifft(x))) <= 1e-13 * np.sqrt(n) * np.max(np.abs(x)) * 4


@pytest.mark.parametrize("n", [60, 64, 90])
def test_parseval_impulse_shift(orc, n):
    x = _rand(n, 3)
    X = orc.fft1d(x)
    assert abs(np.sum(np.abs(X) ** 2) - n * np.sum(np.abs(x) ** 2)) <= 1e-12 * n * np.sum(np.abs(x) ** 2)
    # impulse at j0 -> exp(-2 pi i j0 k / n)
    j0 = n // 3
    d = np.zeros(n, complex)
    d[j0] = 1
    k = np.arange(n)
    assert np.allclose(orc.fft1d(d), np.exp(-2j * np.pi * j0 * k / n), atol=1e-14)
    # circular shift by s multiplies by exp(-2 pi i s k / n)
    s = 5
    Xs = orc.fft1d(np.roll(x, s))
    assert np.allclose(Xs, X * np.exp(-2j * np.pi * s * k / n), atol=1e-12 * np.max(np.abs(X)))
    # inverse of forward is n * identity
    assert np.allclose(orc.fft1d(X, +1), n * x, atol=1e-12 * n)


@pytest.mark.parametrize("shape", [(6, 10, 12), (5, 4, 3), (8, 8, 8), (1, 3, 20)])
def test_fft3d_axis_order(orc, shape):
    r = np.random.default_rng(1)
    a = r.standard_normal(shape) + 1j * r.standard_normal(shape)
    assert np.allclose(orc.fft3d(a, -1), np.fft.fftn(a), atol=1e-12)
    assert np.allclose(orc.fft3d(a, +1), np.fft.ifftn(a) * a.size, atol=1e-12)


@pytest.mark.parametrize("M", [1, 2, 3, 4, 8, 15, 16, 33])
def test_dct1_matches_scipy_and_even_extension(orc, M):
    x = np.random.default_rng(M).standard_normal(M + 1)
    X = orc.dct1(x)
    assert np.allclose(X, scipy.fft.dct(x, type=1), atol=1e-12)
    # DFT of the even extension of length 2M is real and equals the DCT-I
    ext = np.concatenate([x, x[-2:0:-1]])
    E = np.fft.fft(ext)
    assert np.allclose(E[: M + 1].real, X, atol=1e-12)
    assert np.max(np.abs(E.imag)) < 1e-11


@pytest.mark.parametrize("M,K", [(4, 4), (8, 4), (12, 6), (16, 8)])
def test_dct1_3d_matches_scipy(orc, M, K):
    x = np.random.default_rng(M + K).standard_normal((M + 1,) * 3)
    got = orc.dct1_3d(x, K)
    ref = scipy.fft.dctn(x, type=1)[: K + 1, : K + 1, : K + 1]
    assert np.allclose(got, ref, atol=1e-10 * np.max(np.abs(ref)))
