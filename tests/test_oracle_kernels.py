"""Pins of the oracle's Green's-function kernels (Sec. 2.2-2.4).

- Eq. green_vico against a 30-digit evaluation (the small-argument series and
  the k = 0 limit included).
- The (4N)^3 inverse transform against the brute-force cosine sum and against
  the sum rule h^3 sum_m T[m] = G_L(0) = L_t^2 / 2 (fixes the (4Nh)^-3 scale
  and the frequency spacing).
- The original (4N)^3 route and the DCT-I (2N+1)^3 route of Sec. 2.4 agree to
  rounding: two independent computations (textbook FFT vs direct cosine sums).
- The spectrum the solve multiplies by equals the DCT-I of T on (N+1)^3 times
  h^3/(2N)^3 (scipy's REDFT00), although the oracle builds it with the full
  complex (2N)^3 FFT of the mirrored kernel.
"""
import numpy as np
import pytest
import scipy.fft


@pytest.mark.parametrize("Lt", [1.0, 1.905, 3.81])
def test_green_vico_hat_high_precision(orc, Lt):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    assert orc.green_vico_hat(0.0, Lt) == pytest.approx(Lt * Lt / 2, rel=1e-15)
    for u in [1e-9, 1e-6, 5e-4, 9.99e-4, 1.001e-3, 0.01, 0.3, 1.0, 3.0, 7.5, 40.0, 123.4]:
        k = 2.0 * u / Lt
        # reference at the exact double argument u = (L_t/2) k the oracle forms,
        # so that only the evaluation itself (sin, division, squares) is tested
        ud = mp.mpf(0.5 * Lt * k)
        ref = 2 * mp.mpf(0.5 * Lt) ** 2 * (mp.sin(ud) / ud) ** 2
        got = orc.green_vico_hat(k, Lt)
        assert abs(got - float(ref)) <= 2e-15 * max(abs(float(ref)), 1e-300) + 1e-300, (u, got, ref)
    # zeros at L_t |k| / 2 = pi
    assert abs(orc.green_vico_hat(2 * np.pi / Lt, Lt)) < 1e-28 * Lt * Lt + 1e-30


@pytest.mark.parametrize("N", [2, 4, 6])
def test_vg_sum_rule_and_realness(orc, N):
    L = 1.0
    full, T = orc.vg_full(N, L)
    h = L / N
    Lt = orc.window(L)
    assert abs(h ** 3 * full.real.sum() - Lt * Lt / 2) <= 1e-12 * Lt * Lt
    assert np.max(np.abs(full.imag)) <= 1e-13 * np.max(np.abs(full.real))
    # T is the [0,N]^3 corner of the real part
    assert np.array_equal(T, full.real[: N + 1, : N + 1, : N + 1])
    # evenness of the (4N)^3 result per axis: value at m equals value at -m
    n4 = 4 * N
    idx = (-np.arange(n4)) % n4
    assert np.allclose(full.real, full.real[idx][:, idx][:, :, idx], atol=1e-13 * np.max(np.abs(full.real)))


@pytest.mark.parametrize("N,L", [(2, 1.0), (3, 1.0), (4, 2.0)])
def test_vg_kernel_by_brute_force(orc, N, L):
    """T[m] = (4Nh)^-3 sum_{j in [-2N,2N)^3} G_L(2 pi |j| / (4Nh)) cos(2 pi j.m / 4N)."""
    h = L / N
    n4 = 4 * N
    Lt = orc.window(L)
    j = np.arange(-2 * N, 2 * N)
    jz, jy, jx = np.meshgrid(j, j, j, indexing="ij")
    kabs = 2 * np.pi / (n4 * h) * np.sqrt(jx ** 2 + jy ** 2 + jz ** 2)
    g = np.vectorize(lambda k: orc.green_vico_hat(k, Lt))(kabs)
    ref = np.empty((N + 1,) * 3)
    for mz in range(N + 1):
        for my in range(N + 1):
            for mx in range(N + 1):
                ph = 2 * np.pi * (jx * mx + jy * my + jz * mz) / n4
                ref[mz, my, mx] = np.sum(g * np.cos(ph)) / (n4 * h) ** 3
    T = orc.kernel_T("vg", N, L)
    assert np.max(np.abs(T - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [3, 4, 8, 12, 16])
def test_vg_equals_vg_dct(orc, N):
    a = orc.kernel_T("vg", N)
    b = orc.kernel_T("vg_dct", N)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("algo", ["he", "vg", "vg_dct"])
@pytest.mark.parametrize("N", [2, 5, 8])
def test_spectrum_is_scaled_dct1_of_kernel(orc, algo, N):
    L = 1.0
    h = L / N
    T = orc.kernel_T(algo, N, L)
    S = orc.spectrum(T, h)
    ref = scipy.fft.dctn(T, type=1) * h ** 3 / (2 * N) ** 3
    assert np.max(np.abs(S - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_vg_window_must_exceed_diagonal(orc):
    """Sec. 2.3: the window exceeds the largest point separation sqrt(3)(N-1)h."""
    for N in (8, 64, 512):
        L = 1.0
        assert orc.window(L) > np.sqrt(3.0) * (N - 1) * (L / N)
        # and the 4N periodisation leaves room: 4Nh - L > L_t
        assert 4 * L - L > orc.window(L)
