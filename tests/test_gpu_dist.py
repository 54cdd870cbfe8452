"""The slab-decomposed solve (fsp_dist_*) with R = 1..4 ranks emulated in this
process on one GPU (device-to-device exchange, paper_2405_02603_gb300.
exchange_local): the gathered field against the oracle's doubled-grid FFT
solve and against the single-GPU fsp_solve on the generic engine, for even
and uneven slab splits (N not divisible by R; N+1 columns)."""
import os

import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, e_max, oracle_T, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("algo", ["he", "vg_dct"])
@pytest.mark.parametrize("N,R", [(8, 2), (15, 2), (16, 4), (24, 3), (32, 4), (48, 4), (10, 1)])
def test_dist_matches_oracle(fsp, orc, N, R, algo, dtype):
    L = 1.0
    rho = I.gaussian_mixture(N, seed=40 + N)
    if dtype == "f32":
        rho = rho.astype(np.float32).astype(np.float64)
    phi = fsp.solve_distributed_local(N, to_dev(rho, dtype), L, algo, dtype, R).double().cpu().numpy()
    ref = orc.solve_fft(oracle_T(orc, algo, N, L), rho, L / N)
    check_emax(e_max(phi, ref), N, dtype, "dist-R%d-%s" % (R, algo))


@pytest.mark.parametrize("N,R", [(32, 2), (64, 4)])
def test_dist_equals_single_gpu_solve(fsp, N, R, monkeypatch):
    """Same generic-engine transforms on both paths: the fields agree to FP64
    rounding of the different line groupings."""
    monkeypatch.setenv("FSP_GENERIC_ONLY", "1")
    rho = to_dev(I.random_field(N, seed=3), "f64")
    p = fsp.Plan(N, 1.0, "vg_dct", "f64")
    one = p.solve(rho).cpu().numpy()
    p.close()
    many = fsp.solve_distributed_local(N, rho, 1.0, "vg_dct", "f64", R).cpu().numpy()
    assert e_max(many, one) <= 1e-13


def test_dist_rejects_bad_arguments(fsp):
    import ctypes
    lib = fsp.lib()
    d = ctypes.c_void_p()
    assert lib.fsp_dist_create(ctypes.byref(d), 8, 1.0, 0, 2, 2, 0, None) == fsp.FSP_EUNSUPPORTED  # double-float
    assert lib.fsp_dist_create(ctypes.byref(d), 8, 1.0, 0, 0, 9, 0, None) == fsp.FSP_EINVAL      # R > N
    assert lib.fsp_dist_create(ctypes.byref(d), 8, 1.0, 0, 0, 2, 2, None) == fsp.FSP_EINVAL      # rank >= R
    p = fsp.DistPlan(8, 1.0, "he", "f64", 2, 0)
    blocks = p.blocks(0, True)
    arr = (ctypes.c_void_p * 2)(blocks[0].data_ptr(), None)
    rho = to_dev(np.zeros((4, 8, 8)), "f64")
    assert lib.fsp_dist_forward(p._d, ctypes.c_void_p(rho.data_ptr()), arr, None) == fsp.FSP_EINVAL
    stale = ctypes.c_void_p(p._d.value)
    p.close()
    assert lib.fsp_dist_destroy(stale) == fsp.FSP_EINVAL  # destroyed: refused without reading it
    assert lib.fsp_dist_middle(stale, arr, arr, None) == fsp.FSP_EINVAL
