"""Pins of the oracle on non-cubic boxes (n_x x n_y x n_z cells, spacings
h_x, h_y, h_z; the shapes of the paper's weak-scaling runs, Sec. 3.2).

- A cube through the non-cubic functions equals the cubic oracle.
- The doubled-grid FFT equals the term-by-term sum on boxes with three
  different sizes and spacings (exact up to rounding).
- The Vico-Greengard kernel by its (4n_a) DFT route equals its DCT-I route.
- Exchanging two axes (sizes and spacings) transposes the kernel.
- Hockney-Eastwood impulse response in closed form with anisotropic spacing.
- The analytic Gaussian potential (Sec. 3.1): Vico-Greengard spectrally
  accurate on non-cubic boxes.
- The far field of an off-centre Gaussian in the 1 x 1 x 2 box of the
  paper's 512^2 x 1024 runs: pins the window alpha |diagonal|, which both a
  shorter window and one long enough to alias through the 4n_a periodisation
  fail.
"""
import numpy as np
import pytest

import fsp_inputs as I
from oracle import analytic as A

SHAPES = [((6, 4, 5), (0.2, 0.3, 0.25)), ((5, 7, 3), (0.25, 0.18, 0.4)), ((8, 3, 6), (0.1, 0.3, 0.15))]


@pytest.mark.parametrize("algo", ["he", "vg", "vg_dct"])
def test_cube_equals_cubic_oracle(orc, algo):
    for N in (4, 7):
        T = orc.kernel_T(algo, N)
        T3 = orc.kernel_T3(algo, (N, N, N), (1.0 / N,) * 3)
        np.testing.assert_allclose(T3, T, rtol=1e-13, atol=1e-15 * np.abs(T).max())
        rho = I.random_field(N, 3)
        np.testing.assert_allclose(orc.solve_fft3(T3, rho, (1.0 / N,) * 3), orc.solve_fft(T, rho, 1.0 / N),
                                   rtol=0, atol=1e-13)


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
@pytest.mark.parametrize("n,h", SHAPES)
def test_fft_equals_direct_sum(orc, algo, n, h):
    T = orc.kernel_T3(algo, n, h)
    rho = I.random_field3(n, 5)
    a = orc.solve_fft3(T, rho, h)
    b = orc.solve_direct3(T, rho, h)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(b).max())


@pytest.mark.parametrize("n,h", SHAPES)
def test_vg_two_routes(orc, n, h):
    Tv = orc.kernel_T3("vg", n, h)
    Td = orc.kernel_T3("vg_dct", n, h)
    np.testing.assert_allclose(Tv, Td, rtol=0, atol=1e-13 * np.abs(Tv).max())


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
def test_axis_exchange_transposes(orc, algo):
    n, h = (6, 4, 5), (0.2, 0.3, 0.25)
    T = orc.kernel_T3(algo, n, h)
    Txy = orc.kernel_T3(algo, (n[1], n[0], n[2]), (h[1], h[0], h[2]))
    Txz = orc.kernel_T3(algo, (n[2], n[1], n[0]), (h[2], h[1], h[0]))
    np.testing.assert_allclose(Txy, np.swapaxes(T, 1, 2), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Txz, np.swapaxes(T, 0, 2), rtol=1e-12, atol=1e-15)


def test_he_impulse(orc):
    n, h = (7, 5, 6), (0.1, 0.17, 0.13)
    j = (2, 4, 1)
    rho = np.zeros((n[2], n[1], n[0]))
    rho[j[2], j[1], j[0]] = 1.0 / (h[0] * h[1] * h[2])
    phi = orc.solve3("he", rho, h)
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    r = np.sqrt(((x - j[0]) * h[0]) ** 2 + ((y - j[1]) * h[1]) ** 2 + ((z - j[2]) * h[2]) ** 2)
    want = np.where(r > 0, 1.0 / (4 * np.pi * np.where(r > 0, r, 1.0)), 1.0 / (4 * np.pi))
    np.testing.assert_allclose(phi, want, rtol=1e-12)


@pytest.mark.parametrize("n,L,tol", [((40, 32, 48), (1.0, 0.8, 1.2), 1e-10), ((32, 40, 48), (1.0, 1.0, 1.0), 1e-7)])
def test_vg_gaussian_spectral_on_noncubic_box(orc, n, L, tol):
    h = tuple(L[a] / n[a] for a in range(3))
    phi = orc.solve3("vg_dct", I.gaussian3(n, L), h)
    assert A.e_max(phi, A.gaussian_potential3(n, L)) < tol


def _far_field(orc, alpha):
    n, L, c, s = (24, 24, 48), (1.0, 1.0, 2.0), (-0.3, -0.3, -0.8), 0.05
    h = tuple(L[a] / n[a] for a in range(3))
    phi = orc.solve_fft3(orc.kernel_T3("vg_dct", n, h, alpha), I.gaussian3(n, L, s, c), h)
    ex = A.gaussian_potential3(n, L, s, c)
    z = I.cell_centres(n[2], L[2])[:, None, None] - c[2]
    y = I.cell_centres(n[1], L[1])[None, :, None] - c[1]
    x = I.cell_centres(n[0], L[0])[None, None, :] - c[0]
    far = np.sqrt(x * x + y * y + z * z) > 1.2
    return float(np.max(np.abs(phi[far] - ex[far]) / ex[far]))


def test_far_field_pins_the_window(orc):
    assert _far_field(orc, orc.ALPHA) < 1e-3
    # a window of alpha sqrt(3) L_x (too short) and of alpha sqrt(3) L_z
    # (beyond 3 min L_a: aliased by the 4n periodisation) both fail
    assert _far_field(orc, orc.ALPHA * np.sqrt(3) * 1.0 / np.sqrt(6)) > 0.1
    assert _far_field(orc, orc.ALPHA * np.sqrt(3) * 2.0 / np.sqrt(6)) > 0.1


# ---- the field E = -grad phi on non-cubic boxes (Appendix B, Eq. efield)

@pytest.mark.parametrize("algo", ["he", "vg", "vg_dct"])
def test_field_cube_equals_cubic_oracle(orc, algo):
    for a in range(3):
        F = orc.field_kernel(algo, a, 6)
        F3 = orc.field_kernel3(algo, a, (6, 6, 6), (1.0 / 6,) * 3)
        np.testing.assert_allclose(F3, F, rtol=0, atol=1e-13 * np.abs(F).max())


@pytest.mark.parametrize("n,h", SHAPES)
def test_field_fft_equals_direct_and_two_routes(orc, n, h):
    rho = I.random_field3(n, 8)
    for a in range(3):
        Fv, Fd = orc.field_kernel3("vg", a, n, h), orc.field_kernel3("vg_dct", a, n, h)
        np.testing.assert_allclose(Fv, Fd, rtol=0, atol=1e-13 * np.abs(Fv).max())
        for algo in ("he", "vg_dct"):
            F = orc.field_kernel3(algo, a, n, h)
            e1, e2 = orc.solve_field_fft3(F, a, rho, h), orc.solve_field_direct3(F, a, rho, h)
            np.testing.assert_allclose(e1, e2, rtol=0, atol=1e-13 * np.abs(e2).max())


def test_field_he_impulse_is_coulomb(orc):
    n, h, j = (7, 5, 6), (0.1, 0.17, 0.13), (2, 4, 1)
    rho = np.zeros((n[2], n[1], n[0]))
    rho[j[2], j[1], j[0]] = 1.0 / (h[0] * h[1] * h[2])
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    d = [(x - j[0]) * h[0], (y - j[1]) * h[1], (z - j[2]) * h[2]]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    for a in range(3):
        E = orc.solve_field_fft3(orc.field_kernel3("he", a, n, h), a, rho, h)
        want = (r > 0) * d[a] / (4 * np.pi * np.where(r > 0, r, 1.0) ** 3)
        np.testing.assert_allclose(E, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_field_vg_gaussian_on_noncubic_box(orc):
    n, L = (40, 32, 48), (1.0, 0.8, 1.2)
    h = tuple(L[a] / n[a] for a in range(3))
    E = orc.solve_field3("vg_dct", I.gaussian3(n, L), h)
    ex = A.gaussian_field3(n, L)
    err = max(np.abs(E[a] - ex[a]).max() for a in range(3)) / max(np.abs(ex[a]).max() for a in range(3))
    assert err < 1e-8, err


def test_field_is_minus_gradient_on_noncubic_box(orc):
    """E_a against the fourth-order central difference (spacing h_a) of the
    oracle's own potential, smooth Gaussian (sigma = 0.12: the difference's
    own truncation error stays near 1e-3 at h_y = 0.0375), interior points."""
    n, L = (32, 24, 40), (1.0, 0.9, 1.25)
    h = tuple(L[a] / n[a] for a in range(3))
    rho = I.gaussian3(n, L, 0.12)
    phi = orc.solve3("vg_dct", rho, h)
    E = orc.solve_field3("vg_dct", rho, h)
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        p = np.moveaxis(phi, ax, 0)
        d = (-p[4:] + 8 * p[3:-1] - 8 * p[1:-3] + p[:-4]) / (12 * h[a])
        e = np.moveaxis(E[a], ax, 0)[2:-2]
        assert np.abs(e + d).max() < 2e-3 * np.abs(e).max(), (a, np.abs(e + d).max() / np.abs(e).max())


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
@pytest.mark.parametrize("n,h", SHAPES)
def test_spectrum3_is_dct1_of_kernel(orc, algo, n, h):
    """The spectrum from the full doubled-grid FFT equals the type-I DCT of the
    octant (scipy REDFT00 per axis) times h_x h_y h_z / (8 n_x n_y n_z): the
    2n_a DFT of a sequence even about 0 and n_a."""
    import scipy.fft as sf
    T = orc.kernel_T3(algo, n, h)
    want = sf.dctn(T, type=1) * h[0] * h[1] * h[2] / (8.0 * n[0] * n[1] * n[2])
    np.testing.assert_allclose(orc.spectrum3(T, h), want, rtol=0, atol=1e-12 * np.abs(want).max())
