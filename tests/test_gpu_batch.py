"""Batched solves: one persistent launch over many solves of mixed sizes
(mixed radix 2/3/5), replayed as a CUDA graph.  Each batched result is
bitwise equal to the same plan's single solve through the generic engine
(FSP_GENERIC_ONLY=1), and within tolerance of the oracle; a dependency made
impossible on the host ends the launch with FSP_ETIMEOUT and the context stays
usable."""
import os

import numpy as np
import pytest

import fsp_inputs as I
from conftest import e_max, oracle_T, to_dev

pytestmark = pytest.mark.gpu
SIZES = [32, 48, 64, 96, 128, 160]


def _plans(fsp, Ns, dtype, algo="vg_dct"):
    old = os.environ.get("FSP_GENERIC_ONLY")
    os.environ["FSP_GENERIC_ONLY"] = "1"
    try:
        return [fsp.Plan(N, 1.0, algo, dtype) for N in Ns]
    finally:
        if old is None:
            del os.environ["FSP_GENERIC_ONLY"]
        else:
            os.environ["FSP_GENERIC_ONLY"] = old


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_bitwise_equals_single_solves(fsp, dtype):
    import torch
    rng = np.random.default_rng(2406)
    Ns = [int(x) for x in rng.choice(SIZES, size=12)] + SIZES
    plans = _plans(fsp, Ns, dtype)
    rhos = [to_dev(I.gaussian_mixture(N, seed=2406 + i).astype(np.float32), dtype) for i, N in enumerate(Ns)]
    phis = [torch.full_like(r, float("nan")) for r in rhos]
    b = fsp.Batch(plans, rhos, phis)
    for rep in range(2):  # graph replay gives the same bits
        b.launch()
        assert b.wait() == fsp.FSP_OK
        for p, r, f in zip(plans, rhos, phis):
            assert torch.equal(f, p.solve(r)), (p.N, rep)
    # refill the sources in place and replay
    for r in rhos:
        r.mul_(-0.5)
    b.launch()
    assert b.wait() == fsp.FSP_OK
    for p, r, f in zip(plans, rhos, phis):
        assert torch.equal(f, p.solve(r))
    b.close()


def test_batch_against_oracle(fsp, orc):
    import torch
    Ns = [48, 32, 96]
    plans = _plans(fsp, Ns, "f64", "he")
    srcs = [I.random_field(N, seed=N) for N in Ns]
    rhos = [to_dev(s) for s in srcs]
    phis = [torch.empty_like(r) for r in rhos]
    fsp.solve_batched(plans, rhos, phis)
    for N, s, f in zip(Ns, srcs, phis):
        ref = orc.solve_fft(oracle_T(orc, "he", N), s, 1.0 / N)
        assert e_max(f.cpu().numpy(), ref) <= 1e-12


def test_batch_timeout_is_reported_and_context_survives(fsp):
    import torch
    Ns = [32, 48]
    plans = _plans(fsp, Ns, "f32")
    rhos = [to_dev(I.gaussian_mixture(N), "f32") for N in Ns]
    phis = [torch.zeros_like(r) for r in rhos]
    b = fsp.Batch(plans, rhos, phis)
    b.set_timeout(50.0)
    b.inject_stall()
    b.launch()
    assert b.wait() == fsp.FSP_ETIMEOUT
    b.close()
    # the context is still usable: a normal batch and a plain solve work
    b2 = fsp.Batch(plans, rhos, phis)
    b2.launch()
    assert b2.wait() == fsp.FSP_OK
    for p, r, f in zip(plans, rhos, phis):
        assert torch.equal(f, p.solve(r))
    b2.close()


def test_batch_validation(fsp):
    import torch
    p = _plans(fsp, [32], "f64")[0]
    q = _plans(fsp, [32], "f32")[0]
    r = to_dev(I.gaussian(32))
    r32 = to_dev(I.gaussian(32), "f32")
    with pytest.raises(fsp.FspError):
        fsp.Batch([p, p], [r, r], [torch.empty_like(r), torch.empty_like(r)])  # one workspace twice
    with pytest.raises(fsp.FspError):
        fsp.Batch([p, q], [r, r32], [torch.empty_like(r), torch.empty_like(r32)])  # mixed dtypes


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_graph_of_solves_form_bitwise_equals_single_solves(fsp, dtype):
    """Form 1 replays the solves' own launches (specialised kernels for
    power-of-two N, so plans here are the default ones), several per stream:
    every result is bitwise that plan's fsp_solve."""
    import torch
    rng = np.random.default_rng(2406)
    Ns = [int(x) for x in rng.choice(SIZES, size=20)]
    plans = [fsp.Plan(N, 1.0, "vg_dct", dtype) for N in Ns]
    rhos = [to_dev(I.gaussian_mixture(N, seed=3000 + i).astype(np.float32), dtype) for i, N in enumerate(Ns)]
    phis = [torch.full_like(r, float("nan")) for r in rhos]
    b = fsp.Batch(plans, rhos, phis)
    b.set_form(1)
    for rep in range(2):
        b.launch()
        assert b.wait() == fsp.FSP_OK
        for p, r, f in zip(plans, rhos, phis):
            assert torch.equal(p.solve(r), f)
    b.set_form(0)  # back to the persistent kernel: still a valid batch
    b.launch()
    assert b.wait() == fsp.FSP_OK
    b.close()
    for p in plans:
        p.close()
