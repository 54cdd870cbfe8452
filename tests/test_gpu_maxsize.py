"""The largest grids the ABI accepts and degenerate inputs.

N = 1024 (maximum; generic engine, 2048-point columns) and N = 768 (mixed
radix, 2N = 3 * 2^9) against the oracle's compensated direct sum at sampled
points; a zero source gives an exactly zero potential; empty batches and
host-solve lists are rejected or no-ops."""
import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,dtype", [(1024, "f32"), (1024, "f64"), (768, "f64")])
def test_largest_grids_against_direct_sums(fsp, orc, N, dtype):
    import torch
    L = 1.0
    h = L / N
    rho = np.random.default_rng(N).uniform(0.0, 1.0, size=(N, N, N))  # non-negative: no cancellation
    if dtype == "f32":
        rho = rho.astype(np.float32).astype(np.float64)
    p = fsp.Plan(N, L, "he", dtype)
    phi = p.solve(to_dev(rho, dtype)).double().cpu().numpy().ravel()
    p.close()
    torch.cuda.empty_cache()
    rng = np.random.default_rng(7)
    pts = np.concatenate([rng.integers(0, N ** 3, 10), [0, N ** 3 - 1]])
    ref = orc.solve_direct(orc.kernel_T("he", N, L), rho, h, pts)
    err = float(np.max(np.abs(phi[pts] - ref)) / np.max(np.abs(ref)))
    check_emax(err, N, dtype, "maxsize-sampled")


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64df"])
def test_zero_source_gives_zero(fsp, dtype):
    import torch
    p = fsp.Plan(64, 1.0, "vg_dct", dtype)
    z = torch.zeros(64 ** 3, dtype=fsp.torch_dtype(dtype), device="cuda")
    assert bool((p.solve(z) == 0).all())


def test_empty_requests(fsp):
    import ctypes
    p = fsp.Plan(16, 1.0, "he", "f32")
    p.solve_host_many([], [])
    L = fsp.lib()
    assert L.fsp_batch_create(ctypes.byref(ctypes.c_void_p()), None, None, None, 0, None) == fsp.FSP_EINVAL
    assert L.fsp_solve_batched(None, None, None, 0, None) == fsp.FSP_EINVAL
