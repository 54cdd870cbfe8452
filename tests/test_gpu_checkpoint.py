"""Restoring plans from a stored spectrum (fsp_plan_create_from_spectrum;
Plan.save / Plan.load): the multiplier of Sec. 2.2 step 3 / Sec. 2.3-2.4 is
the whole of a plan's state that the precompute makes, so a checkpoint of it
brings a plan back without the (4N)^3 (VG) or (2N+1)^3 (VG-DCT) transform.

A restored plan must solve exactly like the plan it was taken from; a plan
restored from the oracle's spectrum must match the oracle's solve; bad inputs
are refused without device work."""
import ctypes

import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, e_max, to_dev

pytestmark = pytest.mark.gpu


def _solve(p, rho, dtype):
    out = p.solve(to_dev(rho, dtype)).double().cpu().numpy()
    p.sync()
    return out


@pytest.mark.parametrize("dtype", ["f32", "f64", "f64df"])
@pytest.mark.parametrize("algo", ["he", "vg", "vg_dct"])
@pytest.mark.parametrize("N", [24, 32, 64])
def test_restored_plan_solves_bitwise_like_fresh(fsp, N, algo, dtype):
    if dtype == "f64df" and N == 24:
        pytest.skip("double-float runs on the specialised power-of-two kernels only")
    L = 1.3
    rho = I.gaussian_mixture(N, seed=5)
    fresh = fsp.Plan(N, L, algo, dtype)
    want = _solve(fresh, rho, dtype)
    src = fresh if dtype != "f64df" else fsp.Plan(N, L, algo, "f64")  # an FP64 spectrum restores any dtype
    S = src.spectrum()
    back = fsp.Plan.from_spectrum(N, L, algo, dtype, S)
    got = _solve(back, rho, dtype)
    assert back.launches == fresh.launches and back.fast_path == fresh.fast_path
    assert np.array_equal(got, want)
    assert np.array_equal(back.spectrum(), fresh.spectrum())
    for p in {id(x): x for x in (fresh, src, back)}.values():
        p.close()


@pytest.mark.parametrize("dtype", ["f32", "f64df"])
def test_fp64_spectrum_restores_lower_dtypes_exactly(fsp, dtype):
    N, L = 64, 1.0
    S64 = fsp.Plan(N, L, "vg_dct", "f64").spectrum()
    fresh = fsp.Plan(N, L, "vg_dct", dtype)
    back = fsp.Plan.from_spectrum(N, L, "vg_dct", dtype, S64)
    rho = I.gaussian_mixture(N, seed=8)
    assert np.array_equal(_solve(back, rho, dtype), _solve(fresh, rho, dtype))
    fresh.close()
    back.close()


@pytest.mark.parametrize("algo", ["he", "vg"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_plan_on_oracle_spectrum_matches_oracle_solve(fsp, orc, algo, dtype):
    """Spectrum and expected field both from the oracle: pins the stored
    layout (octant, x fastest) and scale h^3 / (2N)^3 independently of the
    plan-time precompute."""
    N, L = 32, 1.0
    T = orc.kernel_T(algo, N, L)
    S = np.ascontiguousarray(orc.spectrum(T, L / N))
    rho = I.gaussian_mixture(N, seed=2)
    if dtype == "f32":
        rho = rho.astype(np.float32).astype(np.float64)
    ref = orc.solve_fft(T, rho, L / N)
    p = fsp.Plan.from_spectrum(N, L, algo, dtype, S)
    err = e_max(_solve(p, rho, dtype), ref)
    check_emax(err, N, dtype, "restored-%s" % algo)
    p.close()


def test_save_load_roundtrip(fsp, tmp_path):
    N, L = 64, 2.0
    p = fsp.Plan(N, L, "vg", "f32")
    path = tmp_path / "vg64.npz"
    p.save(path)
    q = fsp.Plan.load(path)
    assert (q.N, q.L, q.algo, q.dtype) == (N, L, "vg", "f32")
    rho = I.gaussian_mixture(N, seed=3)
    assert np.array_equal(_solve(q, rho, "f32"), _solve(p, rho, "f32"))
    print("N=%d VG precompute %.1f ms, restore %.1f ms" % (N, p.precompute_ms, q.precompute_ms))
    p64 = fsp.Plan(N, L, "vg", "f64")
    p64.save(tmp_path / "vg64_f64.npz")
    r = fsp.Plan.load(tmp_path / "vg64_f64.npz", dtype="f32")  # FP64 checkpoint, FP32 plan
    assert r.dtype == "f32"
    assert np.array_equal(_solve(r, rho, "f32"), _solve(p, rho, "f32"))
    for x in (p, q, p64, r):
        x.close()


def test_restore_refuses_bad_inputs(fsp, tmp_path):
    lib = fsp.lib()
    N = 32
    S = fsp.Plan(N, 1.0, "he", "f64").spectrum()
    out = ctypes.c_void_p()
    assert lib.fsp_plan_create_from_spectrum(ctypes.byref(out), N, 1.0, 0, 0, None, None) == fsp.FSP_EINVAL
    assert lib.fsp_plan_create_from_spectrum(None, N, 1.0, 0, 0, ctypes.c_void_p(S.ctypes.data), None) \
        == fsp.FSP_EINVAL
    bad = S.copy()
    bad[3, 2, 1] = np.nan
    with pytest.raises(fsp.FspError) as ei:
        fsp.Plan.from_spectrum(N, 1.0, "he", "f64", bad)
    assert ei.value.status == fsp.FSP_EINVAL
    with pytest.raises(fsp.FspError) as ei:  # shape of another N
        fsp.Plan.from_spectrum(N, 1.0, "he", "f64", S[:-1])
    assert ei.value.status == fsp.FSP_EINVAL
    S7 = np.ones((8, 8, 8))
    with pytest.raises(fsp.FspError) as ei:  # 2N = 14 is not 2/3/5-smooth
        fsp.Plan.from_spectrum(7, 1.0, "he", "f64", S7)
    assert ei.value.status == fsp.FSP_EUNSUPPORTED
    with pytest.raises(fsp.FspError) as ei:  # outside the double-float range
        fsp.Plan.from_spectrum(N, 1.0, "he", "f64df", S * 1e30)
    assert ei.value.status == fsp.FSP_EUNSUPPORTED
    np.savez(tmp_path / "other.npz", format=np.array("something-else"), S=S)
    with pytest.raises(fsp.FspError):
        fsp.Plan.load(tmp_path / "other.npz")
    p = fsp.Plan.from_spectrum(N, 1.0, "he", "f64", S)  # the device is still fine
    p.close()
