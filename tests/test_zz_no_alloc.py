"""fsp_solve_noalloc, the solve that allocates no device memory (for callers
that cannot call cudaMalloc), against the plan-based fsp_solve.

Collected last on purpose: if it fails, a run stopped at the first failure has
already run every other test.  It needs nothing from earlier tests and passes
alone in a fresh process too."""
import ctypes

import numpy as np
import pytest

import fsp_inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo", ["he", "vg_dct"])
@pytest.mark.parametrize("N", [8, 15, 32])
def test_noalloc_matches_plan_solve_twice(fsp, algo, N):
    import torch
    plan = fsp.Plan(N, 1.0, algo, "f64")
    S = torch.from_numpy(plan.spectrum()).cuda()
    L = fsp.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((1, 2)):  # two calls in a row, different sources
        rho = torch.from_numpy(I.random_field(N, seed=seed) if call else I.gaussian_mixture(N)).cuda()
        ref = plan.solve(rho)
        phi = torch.full_like(rho, float("nan"))
        st = L.fsp_solve_noalloc(N, ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
                                 ctypes.c_void_p(phi.data_ptr()), stream)
        assert st == fsp.FSP_OK
        torch.cuda.synchronize()
        err = float((phi - ref).abs().max() / ref.abs().max())
        assert err <= 1e-12, (N, algo, call, err)
    plan.close()


@pytest.mark.parametrize("algo", ["he", "vg"])
@pytest.mark.parametrize("N", [6, 16, 32])
def test_noalloc_on_oracle_spectrum_matches_oracle_solve(fsp, orc, algo, N):
    """The spectrum and the expected result both come from the CPU oracle:
    nothing the GPU computed enters the comparison but the solve itself."""
    import torch
    L, h = 1.0, 1.0 / N
    T = orc.kernel_T(algo, N, L)
    S = torch.from_numpy(np.ascontiguousarray(orc.spectrum(T, h))).cuda()
    lib = fsp.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, rho_np in enumerate((I.gaussian_mixture(N), I.random_field(N, seed=7))):
        ref = orc.solve_fft(T, rho_np, h)
        rho = torch.from_numpy(rho_np).cuda()
        phi = torch.full_like(rho, float("nan"))
        st = lib.fsp_solve_noalloc(N, ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
                                   ctypes.c_void_p(phi.data_ptr()), stream)
        assert st == fsp.FSP_OK
        torch.cuda.synchronize()
        got = phi.cpu().numpy()
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert err <= 1e-12, (N, algo, call, err)


def test_noalloc_rejects_sizes_beyond_its_scratch(fsp):
    import torch
    L = fsp.lib()
    buf = torch.zeros(40 ** 3, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert L.fsp_solve_noalloc(33, p, p, p, None) == fsp.FSP_EUNSUPPORTED
    assert L.fsp_solve_noalloc(64, p, p, p, None) == fsp.FSP_EUNSUPPORTED
    assert L.fsp_solve_noalloc(7, p, p, p, None) == fsp.FSP_EUNSUPPORTED
    assert L.fsp_solve_noalloc(1, p, p, p, None) == fsp.FSP_EINVAL
    assert L.fsp_solve_noalloc(8, None, p, p, None) == fsp.FSP_EINVAL
    mis = ctypes.c_void_p(buf.data_ptr() + 8)
    assert L.fsp_solve_noalloc(8, p, mis, p, None) == fsp.FSP_EINVAL
