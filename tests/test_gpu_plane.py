"""The fused plane passes against the oracle and against the five-launch
schedule.  Three launches per FP32-mixed solve: PA = pad + x-R2C + y-FFT of
each z-plane in one thread-block cluster, P3, PC = y-IFFT + x-C2R.  They
exist at N = 64, 128, 256 and serve N = 64 by default; FSP_PLANE=1 / 0 at
plan creation forces them on / off.  The packing of the two real columns
k_x = 0 and k_x = N into one complex column changes the rounding order, so
the two schedules agree to FP32 rounding, not bit for bit."""
import os

import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, e_max, to_dev

pytestmark = pytest.mark.gpu


def _plan(fsp, N, algo, plane, dtype="f32"):
    old = os.environ.get("FSP_PLANE")
    os.environ["FSP_PLANE"] = "1" if plane else "0"
    try:
        return fsp.Plan(N, 1.0, algo, dtype)
    finally:
        if old is None:
            del os.environ["FSP_PLANE"]
        else:
            os.environ["FSP_PLANE"] = old


def test_plane_default_sizes(fsp):
    """By default only N = 64 runs the plane passes (measured faster there)."""
    old = os.environ.pop("FSP_PLANE", None)
    try:
        for N, want in ((32, 5), (64, 3), (128, 5), (256, 5)):
            p = fsp.Plan(N, 1.0, "vg_dct", "f32")
            assert p.launches == want, (N, p.launches)
            p.close()
    finally:
        if old is not None:
            os.environ["FSP_PLANE"] = old


@pytest.mark.parametrize("N", [64, 128, 256])
def test_plane_schedule_in_use(fsp, N):
    p3 = _plan(fsp, N, "vg_dct", True)
    p5 = _plan(fsp, N, "vg_dct", False)
    assert p3.launches == 3 and p5.launches == 5
    for dtype in ("f64", "f64df"):
        q = fsp.Plan(N, 1.0, "vg_dct", dtype)
        assert q.launches == 5
        q.close()
    p3.close()
    p5.close()


@pytest.mark.parametrize("algo", ["he", "vg", "vg_dct"])
@pytest.mark.parametrize("N", [64, 128])
def test_plane_matches_oracle(fsp, orc, N, algo):
    L = 1.0
    rho = I.gaussian_mixture(N, seed=21).astype(np.float32).astype(np.float64)
    ref = orc.solve_fft(orc.kernel_T(algo, N, L), rho, L / N)
    p = _plan(fsp, N, algo, True)
    phi = p.solve(to_dev(rho, "f32")).double().cpu().numpy()
    err = e_max(phi, ref)
    check_emax(err, N, "f32", "plane-%s" % algo)
    p.close()


@pytest.mark.parametrize("N", [64, 128, 256])
def test_plane_equals_five_launches(fsp, N):
    pa = _plan(fsp, N, "vg", True)
    pb = _plan(fsp, N, "vg", False)
    for rho_np in (I.gaussian_mixture(N, seed=5).astype(np.float32), I.random_field(N, seed=6).astype(np.float32)):
        rho = to_dev(rho_np, "f32")
        a = pa.solve(rho).double().cpu().numpy()
        b = pb.solve(rho).double().cpu().numpy()
        err = e_max(a, b)
        print("N=%d plane vs five launches E_max %.3e" % (N, err))
        assert err <= 5e-7
    pa.close()
    pb.close()


def test_plane_in_place_and_repeatable(fsp):
    N = 128
    p = _plan(fsp, N, "vg_dct", True)
    rho = to_dev(I.gaussian_mixture(N).astype(np.float32), "f32")
    ref = p.solve(rho).cpu().numpy()
    again = p.solve(rho).cpu().numpy()
    assert np.array_equal(ref, again)  # deterministic
    buf = rho.clone()
    p.solve_into(buf, buf)  # phi == rho
    assert np.array_equal(buf.cpu().numpy(), ref)
    p.close()
