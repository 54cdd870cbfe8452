"""Tile autotuner of the generic engine: it returns feasible shapes, the table
round-trips as text, and the tile shape changes no result bit."""
import os

import numpy as np
import pytest

import fsp_inputs as I
from conftest import to_dev

pytestmark = pytest.mark.gpu


def _generic_plan(fsp, N, dtype):
    old = os.environ.get("FSP_GENERIC_ONLY")
    os.environ["FSP_GENERIC_ONLY"] = "1"
    try:
        return fsp.Plan(N, 1.0, "vg_dct", dtype)
    finally:
        if old is None:
            del os.environ["FSP_GENERIC_ONLY"]
        else:
            os.environ["FSP_GENERIC_ONLY"] = old


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_autotune_and_bitwise_independence(fsp, dtype):
    import torch
    N = 48
    saved = fsp.tuning_get()
    lr, lc = fsp.autotune(N, dtype)
    assert 0 <= lr <= 5 and 0 <= lc <= 5
    assert "%d %d %d %d" % (N, fsp.DTYPES[dtype], lr, lc) in fsp.tuning_get()
    rho = to_dev(I.gaussian_mixture(N).astype(np.float32), dtype)
    ref = _generic_plan(fsp, N, dtype).solve(rho)
    for shape in [(0, 0), (2, 3), (5, 1)]:
        fsp.tuning_set("%d %d %d %d\n" % (N, fsp.DTYPES[dtype], shape[0], shape[1]))
        got = _generic_plan(fsp, N, dtype).solve(rho)
        assert torch.equal(got, ref), shape
    fsp.tuning_set(saved or "%d %d %d %d\n" % (N, fsp.DTYPES[dtype], lr, lc))


def test_tuning_text_validation(fsp):
    with pytest.raises(fsp.FspError):
        fsp.tuning_set("48 1 9 1\n")  # lgL out of range
    with pytest.raises(fsp.FspError):
        fsp.tuning_set("garbage")


def test_batch_autotune_keeps_bits(fsp):
    import torch
    Ns = [48, 32, 64, 48]
    plans = [_generic_plan(fsp, N, "f32") for N in Ns]
    rhos = [to_dev(I.gaussian_mixture(N, seed=i).astype(np.float32), "f32") for i, N in enumerate(Ns)]
    phis = [torch.empty_like(r) for r in rhos]
    saved = fsp.tuning_get()
    b = fsp.Batch(plans, rhos, phis)
    b.launch()
    assert b.wait() == fsp.FSP_OK
    before = [f.clone() for f in phis]
    b.autotune()
    b.launch()
    assert b.wait() == fsp.FSP_OK
    for x, y in zip(before, phis):
        assert torch.equal(x, y)
    b.close()
    fsp.tuning_set(saved)
