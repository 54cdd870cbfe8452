"""The FP64-accuracy solve in double-float arithmetic (FSP_F64_DF): double
arrays in and out, transforms on float pairs.  Same tolerance as the FP64 path
(E_max <= 1e-12 against the oracle)."""
import numpy as np
import pytest

import fsp_inputs as I
from conftest import e_max, oracle_T, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo", ["he", "vg", "vg_dct"])
@pytest.mark.parametrize("N", [32, 64, 128])
def test_df_matches_oracle(fsp, orc, algo, N):
    rho = I.gaussian_mixture(N) if N != 64 else I.random_field(N, seed=9)
    p = fsp.Plan(N, 1.0, algo, "f64df")
    assert p.fast_path
    phi = p.solve(to_dev(rho)).cpu().numpy()
    ref = orc.solve_fft(oracle_T(orc, algo, N), rho, 1.0 / N)
    err = e_max(phi, ref)
    print("df N=%d %s E_max %.3e" % (N, algo, err))
    assert err <= 1e-12, err
    p.close()


def test_df_agrees_with_native_fp64(fsp):
    N = 256
    rho = to_dev(I.gaussian_mixture(N, seed=5))
    a = fsp.Plan(N, 1.0, "vg_dct", "f64df").solve(rho).cpu().numpy()
    b = fsp.Plan(N, 1.0, "vg_dct", "f64").solve(rho).cpu().numpy()
    assert e_max(a, b) <= 1e-12


def test_df_spectrum_is_fp64_spectrum(fsp):
    N = 64
    s64 = fsp.Plan(N, 1.0, "he", "f64").spectrum()
    sdf = fsp.Plan(N, 1.0, "he", "f64df").spectrum()
    # hi + lo reproduces the double to within the double-float precision
    assert np.max(np.abs(sdf - s64)) <= 2.0 ** -46 * np.max(np.abs(s64))


def test_df_unsupported_sizes_and_batches(fsp):
    import torch
    with pytest.raises(fsp.FspError):
        fsp.Plan(48, 1.0, "he", "f64df")  # no specialised kernels for 48
    p = fsp.Plan(32, 1.0, "he", "f64df")
    r = to_dev(I.gaussian(32))
    with pytest.raises(fsp.FspError):
        fsp.Batch([p], [r], [torch.empty_like(r)])


def test_df_in_place_host_and_deterministic(fsp):
    import torch
    N = 64
    p = fsp.Plan(N, 1.0, "vg_dct", "f64df")
    rho = to_dev(I.gaussian_mixture(N))
    a = p.solve(rho)
    assert torch.equal(a, p.solve(rho))
    x = rho.clone()
    p.solve_into(x, x)
    assert torch.equal(x, a)
    hin = rho.cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    p.solve_host(hin, hout)
    assert torch.equal(hout, a.cpu())
