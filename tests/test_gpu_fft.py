"""Line FFT kernels (the building block of every pass) against the oracle's
textbook FFT, for every radix combination the solver uses, both directions,
both precisions, with a line count that leaves a ragged last tile."""
import numpy as np
import pytest

from conftest import e_max

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 20, 24, 25, 27, 30, 32, 45, 48, 60, 64, 75, 80, 96, 100, 120,
         125, 128, 160, 192, 200, 240, 250, 256, 320, 384, 400, 480, 500, 512, 640, 768, 960, 1000, 1024,
         1280, 1536, 2000, 2048, 3072, 4096]
TOL = {"f64": 1e-13, "f32": 3e-6}


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fft_lines_match_oracle(fsp, orc, n, dtype):
    import torch
    count = 37 if n <= 1024 else 9
    r = np.random.default_rng(n)
    x = r.standard_normal((count, n)) + 1j * r.standard_normal((count, n))
    if dtype == "f32":
        x = x.astype(np.complex64).astype(np.complex128)  # the oracle sees the rounded input
    xt = torch.from_numpy(x.astype(np.complex128 if dtype == "f64" else np.complex64)).cuda()
    for sign in (-1, 1):
        got = fsp.fft_c2c(xt, sign).cpu().numpy()
        ref = np.stack([orc.fft1d(row, sign) for row in x])
        assert e_max(got, ref) <= TOL[dtype], (n, dtype, sign, e_max(got, ref))


def test_fft_in_place_and_empty(fsp):
    import ctypes
    import torch
    x = torch.randn(5, 64, dtype=torch.complex128, device="cuda")
    ref = fsp.fft_c2c(x, -1)
    L = fsp.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    fsp.check(L.fsp_fft_c2c(64, 5, 0, -1, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), s))
    torch.cuda.synchronize()
    assert torch.equal(x, ref)
    assert L.fsp_fft_c2c(64, 0, 0, -1, None, None, s) == 0
