"""Bounds evidence without a sanitizer.

* Caller buffers: rho and phi are views into larger device arrays whose
  margins hold NaN; after the solve every margin byte is unchanged.
* Plan buffers: plans created with FSP_CHECK_BOUNDS=1 carry 1 MB guard bands
  of one byte pattern around every device buffer (spectrum, workspaces,
  tables, staging, the field's spectra and workspace, plan-time
  temporaries); after solves the guard bytes are all unchanged, and so are
  those of the temporaries freed at plan creation.
Ragged and odd N on the generic engine, power-of-two N on the specialised
kernels (the plane passes at N = 64), non-cubic boxes, the field, every dtype.
Also: the double-float range check refuses spectra outside [2^-80, 2^80]."""
import os

import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, e_max, oracle_T, to_dev

pytestmark = pytest.mark.gpu

MARGIN = 4096  # elements before and after each caller buffer


def _guarded(shape, dtype):
    """A view of `shape` in the middle of a NaN-filled device array."""
    import torch
    n = int(np.prod(shape))
    big = torch.full((n + 2 * MARGIN,), float("nan"), dtype=dtype, device="cuda")
    return big, big[MARGIN:MARGIN + n].view(shape)


def _margins_intact(big, n):
    import torch
    b = big.view(torch.int64) if big.dtype == torch.float64 else big.view(torch.int32)
    nan = torch.full((1,), float("nan"), dtype=big.dtype, device="cuda")
    pat = nan.view(torch.int64) if big.dtype == torch.float64 else nan.view(torch.int32)
    return bool((b[:MARGIN] == pat).all()) and bool((b[MARGIN + n:] == pat).all())


def _plan(fsp, n, L, algo, dtype):
    old = os.environ.get("FSP_CHECK_BOUNDS")
    os.environ["FSP_CHECK_BOUNDS"] = "1"
    try:
        return fsp.Plan(n, L, algo, dtype)
    finally:
        if old is None:
            del os.environ["FSP_CHECK_BOUNDS"]
        else:
            os.environ["FSP_CHECK_BOUNDS"] = old


CASES = [(15, "he", "f64"), (24, "vg_dct", "f32"), (40, "vg", "f64"), (32, "vg_dct", "f32"),
         (64, "vg_dct", "f32"), (64, "he", "f64df"), (128, "vg_dct", "f64"), (256, "vg", "f32")]


@pytest.mark.parametrize("N,algo,dtype", CASES)
def test_guard_bands_unchanged_after_solves(fsp, N, algo, dtype):
    import torch
    freed0 = int(fsp.lib().fsp_bounds_freed_bad())
    p = _plan(fsp, N, 1.0, algo, dtype)
    tdt = fsp.torch_dtype(dtype)
    rbig, rho = _guarded((N, N, N), tdt)
    fbig, phi = _guarded((N, N, N), tdt)
    rho.copy_(torch.from_numpy(I.gaussian_mixture(N, seed=N)).to(tdt))
    for _ in range(2):
        p.solve_into(rho, phi)
    if N <= 64:
        p.field_init()
        ex, ey, ez = (_guarded((N, N, N), tdt) for _ in range(3))
        p.solve_field_into(rho, ex[1], ey[1], ez[1])
        assert all(_margins_intact(b, N ** 3) for b, _ in (ex, ey, ez))
    torch.cuda.synchronize()
    assert _margins_intact(rbig, N ** 3) and _margins_intact(fbig, N ** 3)
    assert not torch.isnan(phi).any()
    assert p.check_bounds() == 0
    p.close()
    assert int(fsp.lib().fsp_bounds_freed_bad()) == freed0


@pytest.mark.parametrize("n,L,dtype", [((12, 20, 9), (1.0, 1.25, 0.9), "f64"), ((32, 64, 128), (1.0, 1.0, 2.0), "f32"),
                                       ((64, 32, 32), (1.2, 1.0, 0.8), "f64df")])
def test_guard_bands_noncubic(fsp, n, L, dtype):
    import torch
    freed0 = int(fsp.lib().fsp_bounds_freed_bad())
    p = _plan(fsp, n, L, "vg_dct", dtype)
    tdt = fsp.torch_dtype(dtype)
    shape = (n[2], n[1], n[0])
    rbig, rho = _guarded(shape, tdt)
    fbig, phi = _guarded(shape, tdt)
    rho.copy_(torch.from_numpy(I.gaussian_mixture3(n, L)).to(tdt))
    p.solve_into(rho, phi)
    p.field_init()
    outs = [_guarded(shape, tdt) for _ in range(3)]
    p.solve_field_into(rho, *[o[1] for o in outs])
    torch.cuda.synchronize()
    tot = int(np.prod(shape))
    assert _margins_intact(rbig, tot) and _margins_intact(fbig, tot)
    assert all(_margins_intact(b, tot) for b, _ in outs)
    assert p.check_bounds() == 0
    p.close()
    assert int(fsp.lib().fsp_bounds_freed_bad()) == freed0


def test_check_bounds_needs_the_variable(fsp):
    p = fsp.Plan(16, 1.0, "he", "f64")
    with pytest.raises(fsp.FspError) as ei:
        p.check_bounds()
    assert ei.value.status == fsp.FSP_EUNSUPPORTED
    p.close()


def test_double_float_range_check(fsp, orc):
    N = 32
    for L in (1e-12, 1e18):
        with pytest.raises(fsp.FspError) as ei:
            fsp.Plan(N, L, "he", "f64df")
        assert ei.value.status == fsp.FSP_EUNSUPPORTED, L
    for L in (1e-6, 1e10):  # inside the range: still FP64-class against the oracle
        rho = I.gaussian_mixture(N)  # the unit-box source's values, on a box of side L
        p = fsp.Plan(N, L, "he", "f64df")
        phi = p.solve(to_dev(rho)).cpu().numpy()
        p.close()
        ref = orc.solve_fft(oracle_T(orc, "he", N, L), rho, L / N)
        check_emax(e_max(phi, ref), N, "f64df", "df-range-L%g" % L)
