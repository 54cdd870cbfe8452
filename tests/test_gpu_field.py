"""Parity of the field E = -grad phi (Appendix B, Eq. efield) against the
oracle, through fsp_solve_field.

Small sizes: every component of the whole field against the oracle's full
doubled-grid FFT with its own field kernel (the Vico-Greengard kernel from its
(4N)^3 route for "vg", its DST/DCT route for "vg_dct"; the GPU builds both
from the octant), on the specialised kernels (N = 32, 64) and the generic
engine (N = 12, 24, 40: 2N = 24, 48, 80, several tiles and a ragged tail).
N = 256 (the benchmark's size and launch configuration): sampled outputs
against the oracle's direct sum.  The potential returned beside the field is
bitwise the one fsp_solve returns.
"""
import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, e_max, to_dev

pytestmark = pytest.mark.gpu

_F_CACHE = {}


def oracle_F(orc, algo, N, L=1.0):
    key = (algo, N, float(L))
    if key not in _F_CACHE:
        _F_CACHE[key] = [orc.field_kernel(algo, a, N, L) for a in range(3)]
    return _F_CACHE[key]


def check_field(fsp, orc, algo, dtype, N, rho, L=1.0):
    h = L / N
    rho_r = rho.astype(np.float32).astype(np.float64) if dtype == "f32" else rho
    p = fsp.Plan(N, L, algo, dtype)
    out = p.solve_field(to_dev(rho_r, dtype), with_phi=True)
    F = oracle_F(orc, algo, N, L)
    errs = []
    for a in range(3):
        ref = orc.solve_field_fft(F[a], a, rho_r, h)
        errs.append(e_max(out[a].cpu().numpy(), ref))
    phi_ref = p.solve(to_dev(rho_r, dtype))
    same = bool((out[3] == phi_ref).all())
    p.close()
    return errs, same


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64df"])
@pytest.mark.parametrize("algo", ["he", "vg", "vg_dct"])
@pytest.mark.parametrize("N", [32, 64])
def test_field_fast_path(fsp, orc, algo, dtype, N):
    rho = I.gaussian_mixture(N, seed=2405 + N)
    errs, same = check_field(fsp, orc, algo, dtype, N, rho)
    check_emax(max(errs), N, dtype, "field-fast-%s" % algo)
    assert same


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("algo", ["he", "vg_dct"])
@pytest.mark.parametrize("N", [12, 24, 40])
def test_field_generic_engine(fsp, orc, algo, dtype, N):
    rho = I.random_field(N, 7 + N)
    errs, same = check_field(fsp, orc, algo, dtype, N, rho)
    check_emax(max(errs), N, dtype, "field-generic-%s" % algo)
    assert same


def test_field_generic_engine_forced(fsp, orc, monkeypatch):
    """A power-of-two N on the generic engine (FSP_GENERIC_ONLY=1) gives the
    same field as the oracle."""
    monkeypatch.setenv("FSP_GENERIC_ONLY", "1")
    rho = I.gaussian_mixture(32, seed=9)
    errs, same = check_field(fsp, orc, "vg_dct", "f32", 32, rho)
    check_emax(max(errs), 32, "f32", "field-generic-forced")


def test_field_of_impulse_is_coulomb(fsp):
    """Hockney-Eastwood: a unit charge at grid point j gives the Coulomb field
    (x_i - x_j) / (4 pi |x_i - x_j|^3) at every other point, zero at j."""
    N, L = 32, 1.0
    h = L / N
    j = (5, 20, 11)
    p = fsp.Plan(N, L, "he", "f64")
    E = [e.cpu().numpy() for e in p.solve_field(to_dev(I.impulse(N, L, j)))]
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    d = [(x - j[0]) * h, (y - j[1]) * h, (z - j[2]) * h]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    for a in range(3):
        want = (r > 0) * d[a] / (4 * np.pi * np.where(r > 0, r, 1.0) ** 3)
        assert e_max(E[a], want) < 1e-12
    p.close()


def test_field_in_place_and_without_phi(fsp, orc):
    """E_z may overwrite rho; without phi the three components are unchanged."""
    import torch
    N = 32
    rho = I.gaussian_mixture(N, seed=31)
    p = fsp.Plan(N, 1.0, "vg_dct", "f64")
    ex, ey, ez = p.solve_field(to_dev(rho))
    r = to_dev(rho)
    ex2, ey2 = torch.empty_like(r), torch.empty_like(r)
    p.solve_field_into(r, ex2, ey2, r)
    assert bool((ex2 == ex).all()) and bool((ey2 == ey).all()) and bool((r == ez).all())
    p.close()


def test_field_rejects_overlapping_outputs(fsp):
    import torch
    p = fsp.Plan(32, 1.0, "he", "f32")
    a = torch.zeros(32 ** 3, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(fsp.FspError):
        p.solve_field_into(a, b, b, a)
    p.close()


@pytest.mark.parametrize("dtype", ["f32", "f64", "f64df"])
def test_field_n256_sampled_direct_sum(fsp, orc, dtype):
    """N = 256, Vico-Greengard (the benchmark's configuration): the three
    components at sampled points (corners, centre, random) against the
    oracle's direct O(N^3) sum per point."""
    N, L = 256, 1.0
    h = L / N
    rho = I.gaussian_mixture(N).astype(np.float32).astype(np.float64)
    p = fsp.Plan(N, L, "vg", dtype)
    out = p.solve_field(to_dev(rho, dtype))
    rng = np.random.default_rng(256)
    pts = np.concatenate([rng.integers(0, N ** 3, 12), [0, N ** 3 - 1, (N // 2) * (N * N + N + 1), N - 1,
                                                        N * N * (N - 1)]])
    F = oracle_F(orc, "vg_dct", N, L)
    for a in range(3):
        ref = orc.solve_field_direct(F[a], a, rho, h, pts)
        got = out[a].cpu().numpy().ravel()[pts]
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        check_emax(err, N, dtype, "field-n256-sampled-%d" % a)
    p.close()


# ---- non-cubic boxes

ANISO_FIELD = [((12, 20, 9), (1.0, 1.25, 0.9), ["f64", "f32"]), ((24, 24, 48), (1.0, 1.0, 2.0), ["f64", "f32"]),
               ((32, 64, 128), (1.0, 1.0, 2.0), ["f64", "f32", "f64df"]),
               ((64, 32, 32), (1.2, 1.0, 0.8), ["f64", "f32", "f64df"])]


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
@pytest.mark.parametrize("n,L,dtypes", ANISO_FIELD)
def test_field_noncubic(fsp, orc, n, L, dtypes, algo):
    """Every component on non-cubic boxes (generic engine for the first two,
    the specialised kernels with runtime strides for the power-of-two ones)
    against the oracle's doubled-grid FFT; phi beside it bitwise that of
    fsp_solve."""
    h = tuple(L[a] / n[a] for a in range(3))
    rho = I.gaussian_mixture3(n, L, seed=17 + n[0]).astype(np.float32).astype(np.float64)
    F = [orc.field_kernel3(algo, a, n, h) for a in range(3)]
    refs = [orc.solve_field_fft3(F[a], a, rho, h) for a in range(3)]
    for dtype in dtypes:
        p = fsp.Plan(n, L, algo, dtype)
        out = p.solve_field(to_dev(rho, dtype), with_phi=True)
        errs = [e_max(out[a].cpu().numpy(), refs[a]) for a in range(3)]
        check_emax(max(errs), max(n), dtype, "field-%s-%s" % ("x".join(map(str, n)), algo))
        assert bool((out[3] == p.solve(to_dev(rho, dtype))).all())
        p.close()


def test_field_noncubic_impulse_is_coulomb(fsp):
    n, L = (32, 64, 128), (1.0, 1.0, 2.0)
    h = tuple(L[a] / n[a] for a in range(3))
    j = (5, 40, 70)
    rho = np.zeros((n[2], n[1], n[0]))
    rho[j[2], j[1], j[0]] = 1.0 / (h[0] * h[1] * h[2])
    p = fsp.Plan(n, L, "he", "f64")
    E = [e.cpu().numpy() for e in p.solve_field(to_dev(rho))]
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    d = [(x - j[0]) * h[0], (y - j[1]) * h[1], (z - j[2]) * h[2]]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    for a in range(3):
        want = (r > 0) * d[a] / (4 * np.pi * np.where(r > 0, r, 1.0) ** 3)
        assert e_max(E[a], want) < 1e-12
    p.close()
