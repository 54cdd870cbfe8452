"""The specialised kernels (power-of-two N = 32..512, and N = 48, 96, 192,
whose line lengths 3 * 2^k put a radix-3 or radix-6 stage in the middle of
the schedule) against the generic
mixed-radix engine on the same plans' inputs, and against the oracle at
N = 128; the environment switch FSP_GENERIC_ONLY=1 selects the generic engine
at plan creation."""
import os

import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, e_max, oracle_T, to_dev

pytestmark = pytest.mark.gpu


def _plan(fsp, N, algo, dtype, generic):
    old = os.environ.get("FSP_GENERIC_ONLY")
    os.environ["FSP_GENERIC_ONLY"] = "1" if generic else "0"
    try:
        return fsp.Plan(N, 1.0, algo, dtype)
    finally:
        if old is None:
            del os.environ["FSP_GENERIC_ONLY"]
        else:
            os.environ["FSP_GENERIC_ONLY"] = old


FAST = {"f64": [32, 48, 64, 96, 128, 192, 256, 512], "f32": [32, 48, 64, 96, 128, 160, 192, 256, 512]}


@pytest.mark.parametrize("dtype,N", [(d, n) for d in ("f64", "f32") for n in FAST[d]])
def test_fast_equals_generic(fsp, N, dtype):
    pf = _plan(fsp, N, "vg_dct", dtype, generic=False)
    pg = _plan(fsp, N, "vg_dct", dtype, generic=True)
    assert pf.fast_path and not pg.fast_path
    rho = to_dev(I.gaussian_mixture(N, seed=7).astype(np.float32), dtype)
    a = pf.solve(rho).double().cpu().numpy()
    b = pg.solve(rho).double().cpu().numpy()
    check_emax(e_max(a, b), N, dtype, "fast-vs-generic")
    pf.close()
    pg.close()


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fast_n128_against_oracle(fsp, orc, algo, dtype):
    N = 128
    rho = I.random_field(N, seed=11).astype(np.float32).astype(np.float64)
    p = _plan(fsp, N, algo, dtype, generic=False)
    assert p.fast_path
    phi = p.solve(to_dev(rho, dtype)).double().cpu().numpy()
    ref = orc.solve_fft(oracle_T(orc, algo, N), rho, 1.0 / N)
    check_emax(e_max(phi, ref), N, dtype, "fast-n128-%s" % algo)
    p.close()


def test_fast_ragged_and_in_place(fsp):
    import torch
    N = 64
    p = _plan(fsp, N, "he", "f64", generic=False)
    rho = to_dev(I.random_field(N, seed=3))
    a = p.solve(rho)
    x = rho.clone()
    p.solve_into(x, x)
    assert torch.equal(a, x)
    assert torch.equal(a, p.solve(rho))
