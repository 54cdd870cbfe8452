"""Seeded synthetic sources shared by the tests, the benchmark and the oracle.

This module only draws and samples inputs; it holds none of the solver's
arithmetic.  Arrays are float64, shape (N, N, N), index [z, y, x] (x fastest),
on the cell-centred grid x_i = -L/2 + (i + 1/2) h of the cube [-L/2, L/2]^3.

Recipes (the paper's test sources, Sec. 3.1; no external dataset is used):
- gaussian: unit-charge Gaussian, sigma = 0.05, centred in the unit cube.
- gaussian_mixture: 8 Gaussians, centres U[-0.3, 0.3]^3, sigma U[0.03, 0.08],
  weights U[0.5, 1.5], each normalised to unit charge then weighted; numpy
  PCG64 generator seeded with `seed` (default 2405).
- sphere: indicator of the ball of radius 1 in a cube of side 2.4.
- random_field: i.i.d. U[-1, 1] values (parity tests of arbitrary data).
"""
import numpy as np


def cell_centres(N, L):
    h = L / N
    return -0.5 * L + (np.arange(N) + 0.5) * h


def _r2(N, L, centre):
    c = cell_centres(N, L)
    z = c[:, None, None] - centre[2]
    y = c[None, :, None] - centre[1]
    x = c[None, None, :] - centre[0]
    return x * x + y * y + z * z


def gaussian(N, L=1.0, sigma=0.05, centre=(0.0, 0.0, 0.0), weight=1.0):
    """weight * (2 pi sigma^2)^(-3/2) exp(-r^2 / (2 sigma^2)) at the cell centres."""
    norm = (2.0 * np.pi * sigma * sigma) ** -1.5
    return weight * norm * np.exp(-_r2(N, L, centre) / (2.0 * sigma * sigma))


def mixture_params(seed=2405, n=8):
    """(centres (n,3), sigmas (n,), weights (n,)) of the seeded mixture."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-0.3, 0.3, size=(n, 3))
    sigmas = rng.uniform(0.03, 0.08, size=n)
    weights = rng.uniform(0.5, 1.5, size=n)
    return centres, sigmas, weights


def gaussian_mixture(N, L=1.0, seed=2405, n=8):
    """Sum of n seeded unit-charge Gaussians times their weights."""
    centres, sigmas, weights = mixture_params(seed, n)
    rho = np.zeros((N, N, N), dtype=np.float64)
    for c, s, w in zip(centres, sigmas, weights):
        rho += gaussian(N, L, s, tuple(c), w)
    return rho


def sphere(N, L=2.4, radius=1.0, density=1.0):
    """density inside the ball |x| <= radius, 0 outside."""
    return np.where(_r2(N, L, (0.0, 0.0, 0.0)) <= radius * radius, density, 0.0)


def random_field(N, seed=0):
    """i.i.d. uniform values in [-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(N, N, N))


def impulse(N, L=1.0, at=(0, 0, 0)):
    """rho = delta_j / h^3 at grid index `at` = (x, y, z)."""
    h = L / N
    rho = np.zeros((N, N, N), dtype=np.float64)
    rho[at[2], at[1], at[0]] = 1.0 / h ** 3
    return rho


# ---- non-cubic boxes: n = (n_x, n_y, n_z) cells, box sides L = (L_x, L_y, L_z),
# arrays of shape (n_z, n_y, n_x) on the cell centres of [-L/2, L/2] per axis

def _r2_3(n, L, centre):
    z = cell_centres(n[2], L[2])[:, None, None] - centre[2]
    y = cell_centres(n[1], L[1])[None, :, None] - centre[1]
    x = cell_centres(n[0], L[0])[None, None, :] - centre[0]
    return x * x + y * y + z * z


def gaussian3(n, L, sigma=0.05, centre=(0.0, 0.0, 0.0), weight=1.0):
    """The unit-charge Gaussian of `gaussian` on a non-cubic box."""
    norm = (2.0 * np.pi * sigma * sigma) ** -1.5
    return weight * norm * np.exp(-_r2_3(n, L, centre) / (2.0 * sigma * sigma))


def gaussian_mixture3(n, L, seed=2405, k=8):
    """The seeded mixture of `gaussian_mixture` on a non-cubic box."""
    centres, sigmas, weights = mixture_params(seed, k)
    rho = np.zeros((n[2], n[1], n[0]), dtype=np.float64)
    for c, s, w in zip(centres, sigmas, weights):
        rho += gaussian3(n, L, s, tuple(c), w)
    return rho


def random_field3(n, seed=0):
    """i.i.d. uniform values in [-1, 1], shape (n_z, n_y, n_x)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n[2], n[1], n[0]))
