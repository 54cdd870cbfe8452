"""Pins of the oracle's field E = -grad phi (Appendix B, Eq. efield).

What fixes each part without the GPU path:
- DST-I and the mixed DST/DCT 3D transform against scipy's RODFT00/REDFT00;
- the Vico-Greengard field kernel by two independent routes: the (4N)^3 DFT
  of -i k_a G_L and the DST/DCT sums on the (2N+1)^3 octant;
- the doubled-grid FFT field against the term-by-term convolution sum (exact:
  the cyclic convolution with an odd kernel equals the aperiodic one);
- Coulomb's law for an impulse (Hockney-Eastwood field kernel), Gauss's law
  for the flux through a cube, the analytic field of a Gaussian;
- E = -grad phi against a fourth-order difference of the oracle's potential;
- the field spectrum against the DST/DCT route, its odd symmetry and zeros.
"""
import numpy as np
import pytest
import scipy.fft as sf

import fsp_inputs as I
from oracle import analytic as A


def test_dst1_matches_rodft00(orc):
    r = np.random.default_rng(11)
    for M in (2, 3, 8, 13):
        x = r.standard_normal(M + 1)
        X = orc.dst1(x)
        assert X[0] == 0.0 and abs(X[M]) < 1e-12 * np.abs(X).max() + 1e-300
        if M > 1:
            np.testing.assert_allclose(X[1:M], sf.dst(x[1:M], type=1), rtol=0, atol=1e-12 * np.abs(X).max())


@pytest.mark.parametrize("odd", [-1, 0, 1, 2])
def test_trig1_3d_matches_scipy(orc, odd):
    r = np.random.default_rng(12 + odd)
    M, K = 6, 4
    x = r.standard_normal((M + 1,) * 3)
    want = x.copy()
    for ax, arr_axis in ((0, 2), (1, 1), (2, 0)):  # x is the last array axis
        if ax == odd:
            inner = np.take(want, np.arange(1, M), axis=arr_axis)
            s = sf.dst(inner, type=1, axis=arr_axis)
            shape = list(want.shape)
            shape[arr_axis] = M + 1
            full = np.zeros(shape)
            idx = [slice(None)] * 3
            idx[arr_axis] = slice(1, M)
            full[tuple(idx)] = s
            want = full
        else:
            want = sf.dct(want, type=1, axis=arr_axis)
    got = orc.trig1_3d(x, odd, K)
    np.testing.assert_allclose(got, want[:K + 1, :K + 1, :K + 1], rtol=0, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("N", [4, 6, 8])
def test_vg_field_kernel_two_routes(orc, N):
    for a in range(3):
        Fv = orc.field_kernel("vg", a, N)
        Fd = orc.field_kernel("vg_dct", a, N)
        np.testing.assert_allclose(Fv, Fd, rtol=0, atol=1e-13 * np.abs(Fv).max())


def test_field_kernel_symmetry(orc):
    """F_a vanishes on m_a = 0, is positive for m_a > 0 near the charge, and
    the three components are the same kernel with axes exchanged (cubic
    symmetry of both Green's functions)."""
    N = 6
    for algo in ("he", "vg_dct"):
        F = [orc.field_kernel(algo, a, N) for a in range(3)]
        assert np.all(F[0][:, :, 0] == 0) or np.abs(F[0][:, :, 0]).max() < 1e-14 * np.abs(F[0]).max()
        assert F[0][0, 0, 1] > 0 and F[1][0, 1, 0] > 0 and F[2][1, 0, 0] > 0
        np.testing.assert_allclose(F[1], np.swapaxes(F[0], 1, 2), rtol=1e-12, atol=1e-14 * np.abs(F[0]).max())
        np.testing.assert_allclose(F[2], np.swapaxes(F[0], 0, 2), rtol=1e-12, atol=1e-14 * np.abs(F[0]).max())


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
@pytest.mark.parametrize("N", [5, 8])
def test_field_fft_equals_direct_sum(orc, algo, N):
    rho = I.random_field(N, 21)
    for a in range(3):
        F = orc.field_kernel(algo, a, N)
        e1 = orc.solve_field_fft(F, a, rho, 1.0 / N)
        e2 = orc.solve_field_direct(F, a, rho, 1.0 / N)
        np.testing.assert_allclose(e1, e2, rtol=0, atol=1e-13 * np.abs(e2).max())


def test_he_impulse_is_coulomb_field(orc):
    """rho = delta_j / h^3 gives E(i) = (x_i - x_j) / (4 pi |x_i - x_j|^3)."""
    N, L = 8, 1.0
    h = L / N
    j = (2, 5, 3)  # (x, y, z)
    rho = I.impulse(N, L, j)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    d = [(x - j[0]) * h, (y - j[1]) * h, (z - j[2]) * h]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    for a in range(3):
        E = orc.solve_field_fft(orc.field_kernel("he", a, N), a, rho, h)
        want = (r > 0) * d[a] / (4 * np.pi * np.where(r > 0, r, 1.0) ** 3)
        np.testing.assert_allclose(E, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
def test_gauss_law_flux_through_a_cube(orc, algo):
    """The flux of E through a cube around a point charge is the charge (1):
    midpoint sums of E.n over the six faces of the cube of half-side R = 6.5h
    centred on the charge, with E sampled at the cell centres of the faces."""
    N, L = 16, 1.0
    h = L / N
    c = 8
    rho = I.impulse(N, L, (c, c, c))
    E = [orc.solve_field_fft(orc.field_kernel(algo, a, N), a, rho, h) for a in range(3)]
    # faces half-way between grid planes c-7/c-6 and c+6/c+7: E averaged over
    # the two planes at each face point, face cells c-6..c+6 in the other axes
    lo, hi = c - 6, c + 7
    s = slice(c - 6, c + 7)
    flux = 0.0
    flux += (0.5 * (E[0][s, s, hi - 1] + E[0][s, s, hi])).sum() - (0.5 * (E[0][s, s, lo - 1] + E[0][s, s, lo])).sum()
    flux += (0.5 * (E[1][s, hi - 1, s] + E[1][s, hi, s])).sum() - (0.5 * (E[1][s, lo - 1, s] + E[1][s, lo, s])).sum()
    flux += (0.5 * (E[2][hi - 1, s, s] + E[2][hi, s, s])).sum() - (0.5 * (E[2][lo - 1, s, s] + E[2][lo, s, s])).sum()
    flux *= h * h
    assert abs(flux - 1.0) < 0.05, flux


def test_vg_field_gaussian_is_spectrally_accurate(orc):
    N = 32
    E = orc.solve_field("vg_dct", I.gaussian(N))
    ex = A.gaussian_field(N)
    err = max(np.abs(E[a] - ex[a]).max() for a in range(3)) / max(np.abs(ex[a]).max() for a in range(3))
    assert err < 1e-5, err


def test_he_field_gaussian_converges(orc):
    errs = []
    for N in (16, 32):
        E = orc.solve_field("he", I.gaussian(N))
        ex = A.gaussian_field(N)
        errs.append(max(np.abs(E[a] - ex[a]).max() for a in range(3)) / max(np.abs(ex[a]).max() for a in range(3)))
    assert errs[1] < 0.1 and errs[0] / errs[1] > 2.5, errs


def test_field_is_minus_gradient_of_potential(orc):
    """E_a against the fourth-order central difference of the oracle's own
    potential, for a smooth Gaussian (sigma = 0.1, N = 32, interior points)."""
    N, L, sig = 32, 1.0, 0.1
    h = L / N
    rho = I.gaussian(N, L, sig)
    phi = orc.solve("vg_dct", rho)
    E = orc.solve_field("vg_dct", rho)
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        p = np.moveaxis(phi, ax, 0)
        d = (-p[4:] + 8 * p[3:-1] - 8 * p[1:-3] + p[:-4]) / (12 * h)
        e = np.moveaxis(E[a], ax, 0)[2:-2]
        assert np.abs(e + d).max() < 2e-3 * np.abs(e).max(), (a, np.abs(e + d).max() / np.abs(e).max())


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
def test_field_spectrum_two_routes(orc, algo):
    """S_a from the full (2N)^3 FFT of the odd doubled kernel equals
    h^3 / (2N)^3 times the DST-I (axis a) / DCT-I (others) of the octant."""
    N = 6
    h = 1.0 / N
    for a in range(3):
        F = orc.field_kernel(algo, a, N)
        S = orc.field_spectrum(F, a, h)
        Fz = F.copy()
        idx = [slice(None)] * 3
        idx[2 - a] = N
        Fz[tuple(idx)] = 0.0  # the odd extension vanishes at m_a = N
        want = orc.trig1_3d(Fz, a) * h ** 3 / (2 * N) ** 3
        np.testing.assert_allclose(S, want, rtol=0, atol=1e-12 * np.abs(want).max())
        zero = [slice(None)] * 3
        zero[2 - a] = 0
        assert np.abs(S[tuple(zero)]).max() < 1e-13 * np.abs(S).max()
