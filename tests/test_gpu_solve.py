"""Full solves through the C ABI against the oracle (Sec. 2.2 steps 1-5 with
each method's kernel), at sizes that span several tiles with ragged tails
(N+1 is never a multiple of the tile width; odd N exercises the unpacked
real-row paths), plus invariants, in-place use, determinism and error paths.

Tolerances: FP64 E_max <= 1e-12 (max abs error over max |phi|).  FP32-mixed
is compared with the oracle run on the same float32-rounded source and gated
per size at twice the largest E_max measured on the GB300 at that size
(conftest.f32_gate)."""
import numpy as np
import pytest

import fsp_inputs as I
from conftest import check_emax, e_max, oracle_T, to_dev

pytestmark = pytest.mark.gpu

ALGOS = ["he", "vg", "vg_dct"]
SIZES = [2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 40, 45, 48, 50, 60, 64, 80, 96]


def _src(N, kind):
    if kind == "mix":
        return I.gaussian_mixture(N)
    return I.random_field(N, seed=N)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", SIZES)
def test_solve_matches_oracle(fsp, orc, algo, dtype, N):
    L = 1.0
    kind = "mix" if N % 2 == 0 else "rand"
    rho = _src(N, kind)
    if dtype == "f32":
        rho = rho.astype(np.float32).astype(np.float64)
    p = fsp.Plan(N, L, algo, dtype)
    phi = p.solve(to_dev(rho, dtype)).cpu().numpy()
    ref = orc.solve_fft(oracle_T(orc, algo, N, L), rho, L / N)
    check_emax(e_max(phi, ref), N, dtype, "solve-%s-%s" % (algo, kind))
    p.close()


def test_gaussian_against_analytic_config_c1(fsp):
    """VG FP64, N=32, unit cube, sigma=0.05: about 1e-9 relative L2 (Sec. 3.5 table)."""
    from oracle import analytic as A
    N = 32
    p = fsp.Plan(N, 1.0, "vg", "f64")
    phi = p.solve(to_dev(I.gaussian(N))).cpu().numpy()
    e = A.rel_l2(phi, A.gaussian_potential(N))
    assert 1e-10 <= e <= 1e-8, e


@pytest.fixture(scope="module")
def vg24(fsp):
    N = 24
    return N, fsp.Plan(N, 1.0, "vg_dct", "f64")


def _run(fsp, p, r):
    return p.solve(to_dev(r)).cpu().numpy()


def test_invariants_on_device(fsp, vg24):
    N, p = vg24
    a, b = I.random_field(N, 1), I.random_field(N, 2)
    fa, fb = _run(fsp, p, a), _run(fsp, p, b)
    lin = _run(fsp, p, 2.5 * a - 0.75 * b)
    assert e_max(lin, 2.5 * fa - 0.75 * fb) <= 1e-12
    for ax in range(3):
        assert e_max(_run(fsp, p, np.flip(a, ax).copy()), np.flip(fa, ax)) <= 1e-12
    for perm in [(1, 0, 2), (2, 1, 0), (1, 2, 0)]:
        assert e_max(_run(fsp, p, a.transpose(perm).copy()), fa.transpose(perm)) <= 1e-12
    lhs, rhs = np.sum(a * fb), np.sum(fa * b)
    assert abs(lhs - rhs) <= 1e-11 * np.sum(np.abs(a * fb))
    s = (2, 1, 3)
    r = a.copy()
    r[N - s[0]:], r[:, N - s[1]:], r[:, :, N - s[2]:] = 0, 0, 0
    sh = np.zeros_like(r)
    sh[s[0]:, s[1]:, s[2]:] = r[: N - s[0], : N - s[1], : N - s[2]]
    fr, fs = _run(fsp, p, r), _run(fsp, p, sh)
    assert e_max(fs[s[0]:, s[1]:, s[2]:], fr[: N - s[0], : N - s[1], : N - s[2]]) <= 1e-12


def test_he_positivity_on_device(fsp):
    N = 20
    p = fsp.Plan(N, 1.0, "he", "f64")
    phi = _run(fsp, p, np.abs(I.random_field(N, 8)))
    assert np.all(phi > 0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_in_place_and_deterministic(fsp, dtype):
    import torch
    N = 30
    p = fsp.Plan(N, 1.0, "vg_dct", dtype)
    rho = to_dev(I.gaussian_mixture(N), dtype)
    a = p.solve(rho)
    b = p.solve(rho)
    assert torch.equal(a, b)  # bitwise reproducible
    x = rho.clone()
    p.solve_into(x, x)
    assert torch.equal(x, a)


def test_solve_host_matches_device(fsp):
    import torch
    N = 32
    p = fsp.Plan(N, 1.0, "he", "f32")
    rho = I.gaussian(N).astype(np.float32)
    dev = p.solve(torch.from_numpy(rho).cuda()).cpu().numpy()
    hin = torch.from_numpy(rho).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    p.solve_host(hin, hout)
    assert np.array_equal(hout.numpy(), dev)


def test_error_paths(fsp):
    import ctypes
    import torch
    N = 8
    p = fsp.Plan(N, 1.0, "he", "f64")
    L = fsp.lib()
    buf = torch.zeros(N ** 3 + 2, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    mis = ctypes.c_void_p(buf.data_ptr() + 8)
    ok = ctypes.c_void_p(buf.data_ptr())
    assert L.fsp_solve(p.handle, mis, ok, s) == fsp.FSP_EINVAL
    assert L.fsp_solve(p.handle, ok, None, s) == fsp.FSP_EINVAL
    assert L.fsp_solve(p.handle, ok, ok, s) == fsp.FSP_OK
    h = ctypes.c_void_p(p.handle.value)
    p.close()
    assert L.fsp_solve(h, ok, ok, s) == fsp.FSP_EINVAL  # destroyed plan is detected
    assert L.fsp_plan_destroy(h) == fsp.FSP_EINVAL
    assert fsp.lib().fsp_plan_sync(h, s) == fsp.FSP_EINVAL
    with pytest.raises(fsp.FspError):
        fsp.Plan(14, 1.0, "vg", "f64", h=0.5)


def test_plan_accounting(fsp):
    N = 64
    p = fsp.Plan(N, 1.0, "vg_dct", "f64")
    P = (N + 1 + 15) // 16 * 16
    expect = (N + 1) ** 2 * P * 8 + 3 * N * N * P * 16 + 3 * N * 16
    assert p.bytes == expect
    assert p.precompute_ms > 0


@pytest.mark.parametrize("dtype", ["f32", "f64df"])
def test_solve_host_many_matches_device(fsp, dtype):
    import torch
    N = 64
    p = fsp.Plan(N, 1.0, "vg_dct", dtype)
    srcs = [I.gaussian_mixture(N, seed=s) for s in range(7)]  # every staging slot used twice or more
    tdt = fsp.torch_dtype(dtype)
    hin = [torch.from_numpy(x).to(tdt).pin_memory() for x in srcs]
    hout = [torch.empty_like(h).pin_memory() for h in hin]
    p.solve_host_many(hin, hout)
    for h, o in zip(hin, hout):
        assert torch.equal(o, p.solve(h.cuda()).cpu())
    # a second call starts on the slots and events the first one left
    back = [torch.empty_like(h).pin_memory() for h in hin]
    p.solve_host_many(hin[::-1], back)
    for o, b in zip(hout[::-1], back):
        assert torch.equal(o, b)
    p.solve_host_many([], [])  # nothing to do


@pytest.mark.parametrize("algo,dtype,tol", [("vg", "f64", 1e-5), ("vg_dct", "f64df", 1e-5), ("vg_dct", "f32", 1e-4)])
def test_far_field_uses_the_full_window(fsp, algo, dtype, tol):
    """Off-centre Gaussian (sigma 0.04 at (-0.3,-0.3,-0.3)) against its analytic
    potential more than 1.2 away: the device's truncation window must exceed
    the box diagonal (Sec. 2.3)."""
    from oracle import analytic as A
    N, c, s = 32, (-0.3, -0.3, -0.3), 0.04
    p = fsp.Plan(N, 1.0, algo, dtype)
    phi = p.solve(to_dev(I.gaussian(N, 1.0, s, c), dtype)).double().cpu().numpy()
    ex = A.gaussian_potential(N, 1.0, s, c)
    x = I.cell_centres(N, 1.0)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    far = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) > 1.2
    assert np.max(np.abs(phi[far] - ex[far]) / ex[far]) < tol
