"""Parity on non-cubic boxes (fsp_plan_create_aniso) against the oracle.

Whole fields against the oracle's full doubled-grid FFT on boxes with three
different sizes and spacings (ragged tiles in every axis, an axis of 2 cells,
the 1 x 1 x 2 shape of the paper's weak-scaling runs), every method in both
precisions, on the generic engine; power-of-two boxes on the specialised
kernels with runtime geometry in all three dtypes (and against the generic
engine); the cubic case returns the cubic plan; the spectrum against the
oracle's; a 256 x 256 x 512 solve at sampled points against the oracle's
direct sum."""
import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, e_max, to_dev

pytestmark = pytest.mark.gpu

BOXES = [((12, 20, 9), (1.0, 1.25, 0.9)), ((16, 24, 40), (1.0, 1.0, 1.5)), ((2, 16, 8), (0.7, 1.0, 1.0)),
         ((24, 24, 48), (1.0, 1.0, 2.0)), ((30, 18, 25), (1.2, 0.9, 1.0))]


def _h(n, L):
    return tuple(L[a] / n[a] for a in range(3))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("algo", ["he", "vg", "vg_dct"])
@pytest.mark.parametrize("n,L", BOXES)
def test_aniso_whole_field(fsp, orc, n, L, algo, dtype):
    h = _h(n, L)
    rho = I.gaussian_mixture3(n, L, seed=3 + n[0])
    if dtype == "f32":
        rho = rho.astype(np.float32).astype(np.float64)
    p = fsp.Plan(n, L, algo, dtype)
    assert not p.fast_path
    phi = p.solve(to_dev(rho, dtype)).cpu().numpy()
    ref = orc.solve_fft3(orc.kernel_T3(algo, n, h), rho, h)
    err = e_max(phi, ref)
    check_emax(err, max(n), dtype, "aniso-%s-%s" % ("x".join(map(str, n)), algo))
    p.close()


FAST_BOXES = [((32, 64, 128), (1.0, 1.0, 2.0)), ((64, 32, 32), (1.2, 1.0, 0.8)), ((128, 32, 64), (1.0, 0.6, 0.8))]


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64df"])
@pytest.mark.parametrize("algo", ["he", "vg_dct"])
@pytest.mark.parametrize("n,L", FAST_BOXES)
def test_aniso_fast_path(fsp, orc, n, L, algo, dtype):
    h = _h(n, L)
    rho = I.gaussian_mixture3(n, L, seed=11 + n[2]).astype(np.float32).astype(np.float64)
    p = fsp.Plan(n, L, algo, dtype)
    assert p.fast_path
    phi = p.solve(to_dev(rho, dtype)).cpu().numpy()
    ref = orc.solve_fft3(orc.kernel_T3(algo, n, h), rho, h)
    err = e_max(phi, ref)
    check_emax(err, max(n), dtype, "aniso-fast-%s-%s" % ("x".join(map(str, n)), algo))
    p.close()


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
def test_aniso_fast_z_lines_of_2048(fsp, orc, algo):
    """An axis of 1024 cells: FP32 column passes of length 2048 (the shape the
    512^2 x 1024 grid needs), whole field against the oracle; FP64 has no
    such shape and takes the generic engine."""
    n, L = (32, 32, 1024), (0.7, 0.7, 1.4)
    h = _h(n, L)
    rho = I.gaussian_mixture3(n, L, seed=1024).astype(np.float32).astype(np.float64)
    p = fsp.Plan(n, L, algo, "f32")
    assert p.fast_path
    phi = p.solve(to_dev(rho, "f32")).cpu().numpy()
    p.close()
    ref = orc.solve_fft3(orc.kernel_T3(algo, n, h), rho, h)
    check_emax(e_max(phi, ref), 1024, "f32", "aniso-z2048-%s" % algo)
    assert not fsp.Plan(n, L, algo, "f64").fast_path


def test_aniso_fast_equals_generic(fsp, monkeypatch):
    n, L = (64, 32, 128), (1.0, 1.0, 1.5)
    rho = to_dev(I.gaussian_mixture3(n, L, seed=5), "f64")
    a = fsp.Plan(n, L, "vg", "f64")
    monkeypatch.setenv("FSP_GENERIC_ONLY", "1")
    b = fsp.Plan(n, L, "vg", "f64")
    assert a.fast_path and not b.fast_path
    assert e_max(a.solve(rho).cpu().numpy(), b.solve(rho).cpu().numpy()) < 1e-14
    a.close()
    b.close()


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
def test_aniso_spectrum(fsp, orc, algo):
    n, L = (12, 20, 9), (1.0, 1.25, 0.9)
    h = _h(n, L)
    p = fsp.Plan(n, L, algo, "f64")
    S = p.spectrum()
    ref = orc.spectrum3(orc.kernel_T3(algo, n, h), h)
    assert S.shape == ref.shape
    assert e_max(S, ref) < 1e-13
    p.close()


def test_aniso_random_data_and_host_path(fsp, orc):
    n, L = (10, 6, 15), (1.0, 0.7, 1.3)
    h = _h(n, L)
    rho = I.random_field3(n, 9)
    p = fsp.Plan(n, L, "vg_dct", "f64")
    ref = orc.solve_direct3(orc.kernel_T3("vg_dct", n, h), rho, h)
    assert e_max(p.solve(to_dev(rho)).cpu().numpy(), ref) < 1e-12
    out = np.empty_like(rho)
    p.solve_host(np.ascontiguousarray(rho), out)
    assert e_max(out, ref) < 1e-12
    p.close()


def test_cube_through_aniso_is_the_cubic_plan(fsp):
    import torch
    rho = to_dev(I.gaussian_mixture(32), "f32")
    a = fsp.Plan((32, 32, 32), (1.0, 1.0, 1.0), "vg", "f32")
    b = fsp.Plan(32, 1.0, "vg", "f32")
    assert a.fast_path and b.fast_path
    assert bool(torch.equal(a.solve(rho), b.solve(rho)))
    a.close()
    b.close()


def test_aniso_plan_rejects_batch(fsp):
    import torch
    p = fsp.Plan((8, 12, 16), (1.0, 1.0, 1.0), "he", "f32")
    rho = torch.zeros(p.npoints, dtype=torch.float32, device="cuda")
    with pytest.raises(fsp.FspError):
        fsp.solve_batched([p], [rho], [torch.empty_like(rho)])
    p.close()


@pytest.mark.parametrize("dtype", ["f32", "f64", "f64df"])
def test_aniso_256x256x512_sampled(fsp, orc, dtype):
    """The 1 x 1 x 2 shape of the weak-scaling runs at 256^2 x 512 (the
    specialised kernels), HE, at sampled points against the oracle's direct
    O(N^3) sum per point."""
    n, L = (256, 256, 512), (1.0, 1.0, 2.0)
    h = _h(n, L)
    rho = I.gaussian_mixture3(n, L).astype(np.float32).astype(np.float64)
    p = fsp.Plan(n, L, "he", dtype)
    assert p.fast_path
    phi = p.solve(to_dev(rho, dtype)).cpu().numpy().ravel()
    rng = np.random.default_rng(2565)
    tot = n[0] * n[1] * n[2]
    pts = np.concatenate([rng.integers(0, tot, 12), [0, tot - 1, tot // 2 + n[0] * n[1] // 2 + n[0] // 2]])
    ref = orc.solve_direct3(orc.kernel_T3("he", n, h), rho, h, pts)
    err = float(np.max(np.abs(phi[pts] - ref)) / np.max(np.abs(ref)))
    check_emax(err, 512, dtype, "aniso-256x256x512-he-sampled")
    p.close()


def test_aniso_512x512x1024_weak_scaling_shape(fsp, orc):
    """The 512^2 x 1024 grid of the paper's weak-scaling runs (Sec. 3.2) on
    one GPU (the specialised kernels; z lines of 2048), HE, FP32-mixed, at
    sampled points against the oracle's direct sum."""
    n, L = (512, 512, 1024), (1.0, 1.0, 2.0)
    h = tuple(L[a] / n[a] for a in range(3))
    rho = I.gaussian_mixture3(n, L).astype(np.float32)
    p = fsp.Plan(n, L, "he", "f32")
    assert p.fast_path
    phi = p.solve(to_dev(rho, "f32")).cpu().numpy().ravel()
    p.close()
    rng = np.random.default_rng(5121024)
    tot = n[0] * n[1] * n[2]
    pts = np.concatenate([rng.integers(0, tot, 4), [tot // 2 + n[0] * n[1] // 2 + n[0] // 2]])
    ref = orc.solve_direct3(orc.kernel_T3("he", n, h), rho.astype(np.float64), h, pts)
    err = float(np.max(np.abs(phi[pts] - ref)) / np.max(np.abs(ref)))
    check_emax(err, 1024, "f32", "aniso-512x512x1024-he-sampled")
