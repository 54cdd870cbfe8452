"""Closed-form potentials and error metrics used to pin the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Sign convention of this
project: phi = G * rho with G = +1/(4 pi |x|), i.e. Lap(phi) = -rho (Sec. 1,
Eq. poisson_eq with eps0 = 1).  The paper's Gaussian test (Sec. 3.1, Eq.
gaussian) prints a negative source with a positive potential; here the source
is the positive unit-charge Gaussian and the potential is the same positive
erf(r / (sqrt(2) sigma)) / (4 pi r).
"""
import numpy as np
from scipy.special import erf


def cell_centres(N, L):
    """Cell-centred coordinates x_i = -L/2 + (i + 1/2) h, h = L/N."""
    h = L / N
    return -0.5 * L + (np.arange(N) + 0.5) * h


def _radius(N, L, centre):
    c = cell_centres(N, L)
    z = c[:, None, None] - centre[2]
    y = c[None, :, None] - centre[1]
    x = c[None, None, :] - centre[0]
    return np.sqrt(x * x + y * y + z * z)


def gaussian_potential(N, L=1.0, sigma=0.05, centre=(0.0, 0.0, 0.0), weight=1.0):
    """Potential of weight * (unit-charge Gaussian of width sigma) (Sec. 3.1).

    phi(r) = weight * erf(r / (sqrt(2) sigma)) / (4 pi r), with the r -> 0 limit
    weight * sqrt(2/pi) / (4 pi sigma).  Shape (N, N, N), index [z, y, x].
    """
    r = _radius(N, L, centre)
    out = np.empty_like(r)
    small = r < 1e-12
    rr = r[~small]
    out[~small] = erf(rr / (np.sqrt(2.0) * sigma)) / (4.0 * np.pi * rr)
    out[small] = np.sqrt(2.0 / np.pi) / (4.0 * np.pi * sigma)
    return weight * out


def sphere_potential(N, L=2.4, radius=1.0, density=1.0, centre=(0.0, 0.0, 0.0)):
    """Potential of a uniform ball (Sec. 3.1, Eq. sphere), this sign convention.

    Inside: density (3 R^2 - r^2) / 6; outside: density R^3 / (3 r).
    """
    r = _radius(N, L, centre)
    R = radius
    inside = density * (3.0 * R * R - r * r) / 6.0
    outside = density * R ** 3 / (3.0 * np.maximum(r, 1e-300))
    return np.where(r <= R, inside, outside)


def e_max(phi, ref):
    """max_i |phi_i - ref_i| / max_i |ref_i| (the tolerance metric)."""
    phi = np.asarray(phi, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(phi - ref)) / np.max(np.abs(ref)))


def rel_l2(phi, ref):
    """||phi - ref||_2 / ||ref||_2 over the mesh points (Sec. 3.1)."""
    phi = np.asarray(phi, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((phi - ref).ravel()) / np.linalg.norm(ref.ravel()))


def gaussian_field(N, L=1.0, sigma=0.05, centre=(0.0, 0.0, 0.0), weight=1.0):
    """Field E = -grad phi of weight * (unit-charge Gaussian of width sigma):
    radial, E_r(r) = weight * Q(r) / (4 pi r^2) with the enclosed charge
    Q(r) = erf(r / (sqrt(2) sigma)) - sqrt(2/pi) (r/sigma) exp(-r^2 / (2 sigma^2))
    (Gauss's law), zero at the centre.  Returns (E_x, E_y, E_z), each of shape
    (N, N, N) indexed [z, y, x]."""
    c = cell_centres(N, L)
    z = np.broadcast_to(c[:, None, None] - centre[2], (N, N, N))
    y = np.broadcast_to(c[None, :, None] - centre[1], (N, N, N))
    x = np.broadcast_to(c[None, None, :] - centre[0], (N, N, N))
    r = np.sqrt(x * x + y * y + z * z)
    s = r / sigma
    q = erf(s / np.sqrt(2.0)) - np.sqrt(2.0 / np.pi) * s * np.exp(-0.5 * s * s)
    er_over_r = np.where(r > 1e-12, q / (4.0 * np.pi * np.maximum(r, 1e-300) ** 3), 0.0)
    return tuple(weight * er_over_r * d for d in (x, y, z))


def gaussian_potential3(n, L, sigma=0.05, centre=(0.0, 0.0, 0.0), weight=1.0):
    """gaussian_potential on a non-cubic box of n = (n_x, n_y, n_z) cells and
    sides L = (L_x, L_y, L_z); shape (n_z, n_y, n_x)."""
    z = cell_centres(n[2], L[2])[:, None, None] - centre[2]
    y = cell_centres(n[1], L[1])[None, :, None] - centre[1]
    x = cell_centres(n[0], L[0])[None, None, :] - centre[0]
    r = np.sqrt(x * x + y * y + z * z)
    out = np.empty_like(r)
    small = r < 1e-12
    rr = r[~small]
    out[~small] = erf(rr / (np.sqrt(2.0) * sigma)) / (4.0 * np.pi * rr)
    out[small] = np.sqrt(2.0 / np.pi) / (4.0 * np.pi * sigma)
    return weight * out


def gaussian_field3(n, L, sigma=0.05, centre=(0.0, 0.0, 0.0), weight=1.0):
    """gaussian_field on a non-cubic box; (E_x, E_y, E_z), shape (n_z, n_y, n_x)."""
    shp = (n[2], n[1], n[0])
    z = np.broadcast_to(cell_centres(n[2], L[2])[:, None, None] - centre[2], shp)
    y = np.broadcast_to(cell_centres(n[1], L[1])[None, :, None] - centre[1], shp)
    x = np.broadcast_to(cell_centres(n[0], L[0])[None, None, :] - centre[0], shp)
    r = np.sqrt(x * x + y * y + z * z)
    s = r / sigma
    q = erf(s / np.sqrt(2.0)) - np.sqrt(2.0 / np.pi) * s * np.exp(-0.5 * s * s)
    er_over_r = np.where(r > 1e-12, q / (4.0 * np.pi * np.maximum(r, 1e-300) ** 3), 0.0)
    return tuple(weight * er_over_r * d for d in (x, y, z))
