"""Pins of the closed forms the oracle is checked against (Sec. 3.1): the
Gaussian field is minus the gradient of the Gaussian potential (central
differences of the closed form), the non-cubic helpers reduce to the cubic
ones on a cube, and the Gaussian field's flux through a large cube is the
unit charge (Gauss's law).  No GPU."""
import numpy as np

from oracle import analytic as A


def test_gaussian_field_is_minus_gradient_of_potential():
    N, L, sig, c = 48, 1.0, 0.12, (0.05, -0.03, 0.02)
    h = L / N
    E = A.gaussian_field(N, L, sig, c)
    # phi at x +- h/2 e_a is phi at x with the centre moved by -+ h/2 e_a:
    # a central difference at the cell centres
    for a in range(3):
        shift = [0.0, 0.0, 0.0]
        shift[a] = 0.5 * h
        cp = tuple(c[i] - shift[i] for i in range(3))  # phi at x + h/2 e_a
        cm = tuple(c[i] + shift[i] for i in range(3))  # phi at x - h/2 e_a
        d = (A.gaussian_potential(N, L, sig, cp) - A.gaussian_potential(N, L, sig, cm)) / h
        assert np.abs(E[a] + d).max() < 2e-3 * np.abs(E[a]).max(), a


def test_noncubic_helpers_on_a_cube():
    N, L = 20, 1.3
    np.testing.assert_allclose(A.gaussian_potential3((N, N, N), (L, L, L), 0.1, (0.1, 0.0, -0.2)),
                               A.gaussian_potential(N, L, 0.1, (0.1, 0.0, -0.2)), rtol=1e-14)
    for a, b in zip(A.gaussian_field3((N, N, N), (L, L, L), 0.1, (0.1, 0.0, -0.2)),
                    A.gaussian_field(N, L, 0.1, (0.1, 0.0, -0.2))):
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-300)


def test_gauss_law_for_the_closed_form():
    """Flux of the closed-form field through the faces of a cube of half-side
    0.45 around the centre: midpoint rule on a fine face grid, = 1 (the
    Gaussian's mass outside the cube is below 1e-12 for sigma = 0.06)."""
    sig, R, m = 0.06, 0.45, 400
    u = (np.arange(m) + 0.5) / m * 2 * R - R
    U, V = np.meshgrid(u, u, indexing="ij")
    r = np.sqrt(R * R + U * U + V * V)
    s = r / sig
    from scipy.special import erf
    q = erf(s / np.sqrt(2)) - np.sqrt(2 / np.pi) * s * np.exp(-0.5 * s * s)
    en = q / (4 * np.pi * r ** 3) * R  # E . n on one face
    flux = 6 * en.sum() * (2 * R / m) ** 2
    assert abs(flux - 1.0) < 1e-5, flux
