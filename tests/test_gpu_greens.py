"""Plan-time Green's functions on the device (FP64) against the oracle:
the real-space kernel T of each method (Sec. 2.2 step 3, Sec. 2.3, Sec. 2.4)
and the spectrum the solve multiplies by."""
import numpy as np
import pytest

from conftest import e_max

pytestmark = pytest.mark.gpu

ALGOS = ["he", "vg", "vg_dct"]
SIZES = [2, 3, 4, 5, 6, 8, 9, 12, 15, 16, 24, 25, 32]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("N", SIZES)
def test_kernel_T_matches_oracle(fsp, orc, algo, N):
    L = 1.0 if N % 2 else 2.0
    got = fsp.kernel_T(N, L, algo).cpu().numpy()
    ref = orc.kernel_T(algo, N, L)
    assert e_max(got, ref) <= 1e-13, e_max(got, ref)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("N", [2, 5, 8, 16, 30])
def test_spectrum_matches_oracle(fsp, orc, algo, N):
    L = 1.0
    p = fsp.Plan(N, L, algo, "f64")
    S = p.spectrum()
    ref = orc.spectrum(orc.kernel_T(algo, N, L), L / N)
    assert e_max(S, ref) <= 1e-12, e_max(S, ref)
    # the mixed plan rounds the same FP64 spectrum once to float32
    q = fsp.Plan(N, L, algo, "f32")
    assert np.array_equal(q.spectrum(), S.astype(np.float32).astype(np.float64))
    p.close()
    q.close()


def test_vg_and_vg_dct_agree_on_device(fsp):
    for N in (8, 24, 64):
        a = fsp.kernel_T(N, 1.0, "vg").cpu().numpy()
        b = fsp.kernel_T(N, 1.0, "vg_dct").cpu().numpy()
        assert e_max(a, b) <= 1e-13

