"""The TMA-staged persistent P3 (z-FFT * S * z-IFFT of Sec. 2.2 step 4, FP32
lines of 2N = 128, 256, 512) against the default register-direct P3 and
against the oracle, and its bounded wait: a stall injected on the host (each
tile's copy expected to deliver 16 bytes more than it does) must end with
FSP_ETIMEOUT from fsp_plan_sync and leave plan and context usable.

FSP_P3_TMA=1 at plan creation selects the TMA-staged P3; by default (and with
FSP_P3_TMA=0) plans run the register-direct P3 (k_fast_col), which measured
faster on the GB300."""
import os

import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, e_max, to_dev

pytestmark = pytest.mark.gpu


def _plan(fsp, N, algo, tma):
    old = os.environ.get("FSP_P3_TMA")
    os.environ["FSP_P3_TMA"] = "1" if tma else "0"
    try:
        return fsp.Plan(N, 1.0, algo, "f32")
    finally:
        if old is None:
            del os.environ["FSP_P3_TMA"]
        else:
            os.environ["FSP_P3_TMA"] = old


@pytest.mark.parametrize("N", [64, 128, 256])
def test_tma_p3_equals_register_p3(fsp, N):
    """Same transform in both kernels: the fields agree to the last bits
    (1e-7 relative, a few FP32 ulps of the maximum).  At N = 256 the
    register-direct P3 adds in packed two-float form, which rounds the
    spectrum products before the sums that the scalar code of the TMA kernel
    fuses into FMAs: a few ulps more apart there (4e-7)."""
    pt = _plan(fsp, N, "vg_dct", True)
    pr = _plan(fsp, N, "vg_dct", False)
    for seed in (3, 4):
        rho = to_dev(I.gaussian_mixture(N, seed=seed).astype(np.float32), "f32")
        a = pt.solve(rho).double().cpu().numpy()
        b = pr.solve(rho).double().cpu().numpy()
        err = e_max(a, b)
        print("N=%d TMA P3 vs register P3: E_max %.3e, bitwise equal %s" % (N, err, bool(np.array_equal(a, b))))
        assert err <= (4e-7 if N == 256 else 1e-7)
    pt.sync()
    pt.close()
    pr.close()


@pytest.mark.parametrize("algo", ["he", "vg"])
def test_tma_p3_n64_matches_oracle(fsp, orc, algo):
    N, L = 64, 1.0
    rho = I.gaussian_mixture(N, seed=11).astype(np.float32).astype(np.float64)
    ref = orc.solve_fft(orc.kernel_T(algo, N, L), rho, L / N)
    p = _plan(fsp, N, algo, True)
    phi = p.solve(to_dev(rho, "f32")).double().cpu().numpy()
    p.sync()
    err = e_max(phi, ref)
    check_emax(err, N, "f32", "p3tma-%s" % algo)
    p.close()


def test_tma_p3_timeout_leaves_plan_usable(fsp):
    import ctypes
    N = 64
    p = _plan(fsp, N, "vg_dct", True)
    lib = fsp.lib()
    rho = to_dev(I.gaussian_mixture(N).astype(np.float32), "f32")
    good = p.solve(rho).double().cpu().numpy()
    p.sync()
    assert lib.fsp_plan_set_wait_timeout(p.handle, ctypes.c_double(5.0)) == fsp.FSP_OK
    assert lib.fsp_plan_inject_stall(p.handle) == fsp.FSP_OK
    p.solve(rho)
    with pytest.raises(fsp.FspError) as ei:
        p.sync()
    assert ei.value.status == fsp.FSP_ETIMEOUT
    # the flag is cleared and the next solve is whole again
    again = p.solve(rho).double().cpu().numpy()
    p.sync()
    assert np.array_equal(again, good)
    assert lib.fsp_plan_set_wait_timeout(p.handle, ctypes.c_double(0.0)) == fsp.FSP_EINVAL
    p.close()
    pr = _plan(fsp, N, "vg_dct", False)
    assert lib.fsp_plan_inject_stall(pr.handle) == fsp.FSP_EUNSUPPORTED
    pr.close()
