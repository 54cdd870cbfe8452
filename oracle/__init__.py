"""FP64 CPU oracle for the free-space spectral Poisson solver (arXiv 2405.02603).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product.  It is independent of the
CUDA path: no shared code, kernels, headers, tables or constant generators.

The arithmetic lives in ``fsp_oracle.c`` (plain C, double precision); this
module marshals numpy arrays to it and adds the analytic potentials and the
error metrics.  Every function names the passage of the paper it follows:

- ``fft1d``/``fft3d``: textbook recursive mixed-radix FFT (the FFT of Sec. 1,
  convolution theorem); ``dft1d``: the DFT by definition.
- ``dct1``/``dct1_3d``: type-I DCT by definition (Sec. 2.4).
- ``kernel_T``: real-space kernel of Hockney-Eastwood (Sec. 2.2, step 3),
  Vico-Greengard on (4N)^3 (Sec. 2.3, Eq. green_vico) or its DCT-I variant on
  (2N+1)^3 (Sec. 2.4).
- ``solve_fft``: Sec. 2.2 steps 1-5 on the full doubled grid.
- ``solve_direct``: the O(N_g^2) discrete convolution sum (Sec. 1).
- ``spectrum``: the multiplier h^3 DFT{G_2}/(2N)^3 on the non-redundant octant.
- ``analytic``: the Gaussian (Sec. 3.1, Eq. gaussian) and uniform-sphere
  (Sec. 3.1, Eq. sphere) potentials, in this project's sign convention, and
  the Gaussian's field.
- ``dst1``/``trig1_3d``: type-I DST by definition, and the separable 3D
  DST-I/DCT-I mix an odd kernel's octant needs.
- ``kernel_T3``, ``solve_fft3``, ``spectrum3``, ``solve_direct3``, ``solve3``:
  the methods on a non-cubic box of n_x x n_y x n_z cells with spacings
  h_x, h_y, h_z (the shapes of the paper's weak-scaling runs, Sec. 3.2), and
  ``field_kernel3``, ``solve_field_fft3``, ``solve_field_direct3``,
  ``solve_field3`` for the field on them.
- ``field_kernel``, ``solve_field_fft``, ``solve_field_direct``,
  ``field_spectrum``, ``solve_field``: the field E = -grad phi (Appendix B,
  Eq. efield) as the convolution of rho with F = -grad G of each method.
"""
import ctypes

import numpy as np

from . import build as _build

HE, VG, VG_DCT = 0, 1, 2
ALGOS = {"he": HE, "vg": VG, "vg_dct": VG_DCT}
ALPHA = 1.1  # Vico-Greengard window factor, Sec. 2.3

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_longlong)
        i, d = ctypes.c_int, ctypes.c_double
        lib.orc_num_threads.restype = i
        lib.orc_set_num_threads.argtypes = [i]
        lib.orc_dft1d.argtypes = [i, dp, dp, i]
        lib.orc_fft1d.argtypes = [i, dp, dp, i]
        lib.orc_fft3d.argtypes = [i, i, i, dp, i]
        lib.orc_dct1_1d.argtypes = [i, dp, dp]
        lib.orc_dct1_3d.argtypes = [i, i, dp, dp]
        lib.orc_green_vico_hat.argtypes = [d, d]
        lib.orc_green_vico_hat.restype = d
        lib.orc_vg_full.argtypes = [i, d, d, dp, dp]
        lib.orc_kernel_T.argtypes = [i, i, d, d, dp]
        lib.orc_solve_fft.argtypes = [i, d, dp, dp, dp]
        lib.orc_spectrum.argtypes = [i, d, dp, dp]
        lib.orc_solve_direct.argtypes = [i, d, dp, dp, lp, ctypes.c_longlong, dp]
        lib.orc_dst1_1d.argtypes = [i, dp, dp]
        lib.orc_trig1_3d.argtypes = [i, i, i, dp, dp]
        lib.orc_field_kernel.argtypes = [i, i, i, d, d, dp]
        lib.orc_solve_field_fft.argtypes = [i, d, i, dp, dp, dp]
        lib.orc_field_spectrum.argtypes = [i, d, i, dp, dp]
        lib.orc_solve_field_direct.argtypes = [i, d, i, dp, dp, lp, ctypes.c_longlong, dp]
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_kernel_T3.argtypes = [i, ip, dp, d, dp]
        lib.orc_solve_fft3.argtypes = [ip, dp, dp, dp, dp]
        lib.orc_spectrum3.argtypes = [ip, dp, dp, dp]
        lib.orc_solve_direct3.argtypes = [ip, dp, dp, dp, lp, ctypes.c_longlong, dp]
        lib.orc_field_kernel3.argtypes = [i, i, ip, dp, d, dp]
        lib.orc_solve_field_fft3.argtypes = [ip, dp, i, dp, dp, dp]
        lib.orc_solve_field_direct3.argtypes = [ip, dp, i, dp, dp, lp, ctypes.c_longlong, dp]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads():
    return _load().orc_num_threads()


def set_num_threads(n):
    _load().orc_set_num_threads(int(n))


def _c128(x):
    return np.ascontiguousarray(x, dtype=np.complex128)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def dft1d(x, sign=-1):
    """X[k] = sum_j x[j] exp(sign 2 pi i jk/n), by definition (O(n^2))."""
    x = _c128(x)
    out = np.empty_like(x)
    _load().orc_dft1d(x.size, _p(x), _p(out), int(sign))
    return out


def fft1d(x, sign=-1):
    """Unnormalised textbook mixed-radix FFT of a 1D array."""
    x = _c128(x)
    out = np.empty_like(x)
    _load().orc_fft1d(x.size, _p(x), _p(out), int(sign))
    return out


def fft3d(a, sign=-1):
    """Unnormalised 3D FFT of a (nz, ny, nx) array (returns a new array)."""
    a = _c128(a).copy()
    nz, ny, nx = a.shape
    _load().orc_fft3d(nx, ny, nz, _p(a), int(sign))
    return a


def dct1(x):
    """Unnormalised DCT-I of M+1 samples (REDFT00 convention), by definition."""
    x = _f64(x)
    out = np.empty_like(x)
    _load().orc_dct1_1d(x.size - 1, _p(x), _p(out))
    return out


def dct1_3d(x, K=None):
    """3D DCT-I of a (M+1)^3 array, evaluated at outputs [0,K]^3."""
    x = _f64(x)
    M = x.shape[0] - 1
    assert x.shape == (M + 1,) * 3
    K = M if K is None else int(K)
    out = np.empty((K + 1,) * 3, dtype=np.float64)
    _load().orc_dct1_3d(M, K, _p(x), _p(out))
    return out


def green_vico_hat(kabs, Lt):
    """Eq. green_vico, G_L(k) = 2 (sin(L_t |k|/2)/|k|)^2 (scalar)."""
    return _load().orc_green_vico_hat(float(kabs), float(Lt))


def window(L, alpha=ALPHA):
    """Truncation window L_t = alpha sqrt(3) L for the cube of side L (Sec. 2.3)."""
    return alpha * np.sqrt(3.0) * L


def kernel_T(algo, N, L=1.0, alpha=ALPHA):
    """Real-space kernel T[m], m in [0,N]^3, shape (N+1,)*3 indexed [z,y,x]."""
    algo = ALGOS.get(algo, algo)
    T = np.empty((N + 1,) * 3, dtype=np.float64)
    _load().orc_kernel_T(int(algo), int(N), float(L), float(alpha), _p(T))
    return T


def vg_full(N, L=1.0, alpha=ALPHA):
    """Vico-Greengard (4N)^3 inverse transform (complex) and its restriction T."""
    h = L / N
    full = np.empty((4 * N,) * 3, dtype=np.complex128)
    T = np.empty((N + 1,) * 3, dtype=np.float64)
    _load().orc_vg_full(int(N), float(h), float(window(L, alpha)), _p(full), _p(T))
    return full, T


def spectrum(T, h):
    """S[q] = h^3 DFT_{2N}{G_2}[q] / (2N)^3 for q in [0,N]^3 (real part)."""
    T = _f64(T)
    N = T.shape[0] - 1
    S = np.empty_like(T)
    _load().orc_spectrum(N, float(h), _p(T), _p(S))
    return S


def solve_fft(T, rho, h):
    """Hockney-Eastwood steps 1-5 on the full doubled grid with kernel T."""
    T, rho = _f64(T), _f64(rho)
    N = rho.shape[0]
    assert rho.shape == (N, N, N) and T.shape == (N + 1,) * 3
    phi = np.empty_like(rho)
    _load().orc_solve_fft(N, float(h), _p(T), _p(rho), _p(phi))
    return phi


def solve_direct(T, rho, h, points=None):
    """phi_i = h^3 sum_j T[|i-j|] rho_j, at flat indices `points` (or all)."""
    T, rho = _f64(T), _f64(rho)
    N = rho.shape[0]
    assert rho.shape == (N, N, N) and T.shape == (N + 1,) * 3
    lib = _load()
    if points is None:
        out = np.empty_like(rho)
        lib.orc_solve_direct(N, float(h), _p(T), _p(rho), None, 0, _p(out))
        return out
    pts = np.ascontiguousarray(points, dtype=np.int64).ravel()
    assert pts.size == 0 or (pts.min() >= 0 and pts.max() < N ** 3)
    out = np.empty(pts.size, dtype=np.float64)
    lib.orc_solve_direct(N, float(h), _p(T), _p(rho),
                         pts.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), pts.size, _p(out))
    return out


def solve(algo, rho, L=1.0, alpha=ALPHA):
    """Kernel construction plus FFT solve for one source (convenience)."""
    N = rho.shape[0]
    T = kernel_T(algo, N, L, alpha)
    return solve_fft(T, rho, L / N)


def dst1(x):
    """Unnormalised DST-I on the interior of x[0..M] (RODFT00), by definition;
    returns X[0..M] with X[0] = X[M] = 0."""
    x = _f64(x)
    out = np.empty_like(x)
    _load().orc_dst1_1d(x.size - 1, _p(x), _p(out))
    return out


def trig1_3d(x, odd, K=None):
    """DST-I along axis `odd` (0 = x, 1 = y, 2 = z; array index order [z,y,x])
    and DCT-I along the others of a (M+1)^3 array, outputs [0,K]^3."""
    x = _f64(x)
    M = x.shape[0] - 1
    assert x.shape == (M + 1,) * 3
    K = M if K is None else int(K)
    out = np.empty((K + 1,) * 3, dtype=np.float64)
    _load().orc_trig1_3d(M, K, int(odd), _p(x), _p(out))
    return out


def field_kernel(algo, a, N, L=1.0, alpha=ALPHA):
    """Field kernel F_a[m] = -dG/dx_a at m h, m in [0,N]^3, component a
    (0 = x, 1 = y, 2 = z), shape (N+1,)*3 indexed [z,y,x]."""
    algo = ALGOS.get(algo, algo)
    F = np.empty((N + 1,) * 3, dtype=np.float64)
    _load().orc_field_kernel(int(algo), int(a), int(N), float(L), float(alpha), _p(F))
    return F


def solve_field_fft(F, a, rho, h):
    """E_a = h^3 sum_j F_a[i-j] rho_j on the full doubled grid (odd kernel)."""
    F, rho = _f64(F), _f64(rho)
    N = rho.shape[0]
    assert rho.shape == (N, N, N) and F.shape == (N + 1,) * 3
    E = np.empty_like(rho)
    _load().orc_solve_field_fft(N, float(h), int(a), _p(F), _p(rho), _p(E))
    return E


def field_spectrum(F, a, h):
    """S_a[q] = -h^3 Im DFT_{2N}{F_2}[q] / (2N)^3 for q in [0,N]^3."""
    F = _f64(F)
    N = F.shape[0] - 1
    S = np.empty_like(F)
    _load().orc_field_spectrum(N, float(h), int(a), _p(F), _p(S))
    return S


def solve_field_direct(F, a, rho, h, points=None):
    """E_a[i] = h^3 sum_j sgn(i_a - j_a) F_a[|i-j|] rho_j, at flat indices
    `points` (or all)."""
    F, rho = _f64(F), _f64(rho)
    N = rho.shape[0]
    assert rho.shape == (N, N, N) and F.shape == (N + 1,) * 3
    lib = _load()
    if points is None:
        out = np.empty_like(rho)
        lib.orc_solve_field_direct(N, float(h), int(a), _p(F), _p(rho), None, 0, _p(out))
        return out
    pts = np.ascontiguousarray(points, dtype=np.int64).ravel()
    assert pts.size == 0 or (pts.min() >= 0 and pts.max() < N ** 3)
    out = np.empty(pts.size, dtype=np.float64)
    lib.orc_solve_field_direct(N, float(h), int(a), _p(F), _p(rho),
                               pts.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), pts.size, _p(out))
    return out


def solve_field(algo, rho, L=1.0, alpha=ALPHA):
    """(E_x, E_y, E_z) for one source: field kernels plus FFT solves."""
    N = rho.shape[0]
    return tuple(solve_field_fft(field_kernel(algo, a, N, L, alpha), a, rho, L / N) for a in range(3))


def _dims(n, h):
    n = (ctypes.c_int * 3)(*[int(v) for v in n])
    h = np.ascontiguousarray(h, dtype=np.float64)
    assert h.shape == (3,)
    return n, h


def kernel_T3(algo, n, h, alpha=ALPHA):
    """Kernel T[m] on a box of n = (n_x, n_y, n_z) cells with spacings
    h = (h_x, h_y, h_z); shape (n_z+1, n_y+1, n_x+1) indexed [z,y,x]."""
    algo = ALGOS.get(algo, algo)
    nn, hh = _dims(n, h)
    T = np.empty((n[2] + 1, n[1] + 1, n[0] + 1), dtype=np.float64)
    _load().orc_kernel_T3(int(algo), nn, _p(hh), float(alpha), _p(T))
    return T


def solve_fft3(T, rho, h):
    """Sec. 2.2 steps 1-5 on the full doubled grid of a non-cubic box."""
    T, rho = _f64(T), _f64(rho)
    n = (rho.shape[2], rho.shape[1], rho.shape[0])
    assert T.shape == (n[2] + 1, n[1] + 1, n[0] + 1)
    nn, hh = _dims(n, h)
    phi = np.empty_like(rho)
    _load().orc_solve_fft3(nn, _p(hh), _p(T), _p(rho), _p(phi))
    return phi


def spectrum3(T, h):
    """S[q] = h_x h_y h_z DFT{G_2}[q] / (8 n_x n_y n_z) on the octant."""
    T = _f64(T)
    n = (T.shape[2] - 1, T.shape[1] - 1, T.shape[0] - 1)
    nn, hh = _dims(n, h)
    S = np.empty_like(T)
    _load().orc_spectrum3(nn, _p(hh), _p(T), _p(S))
    return S


def solve_direct3(T, rho, h, points=None):
    """phi_i = h_x h_y h_z sum_j T[|i-j|] rho_j at flat indices (or all)."""
    T, rho = _f64(T), _f64(rho)
    n = (rho.shape[2], rho.shape[1], rho.shape[0])
    assert T.shape == (n[2] + 1, n[1] + 1, n[0] + 1)
    nn, hh = _dims(n, h)
    lib = _load()
    if points is None:
        out = np.empty_like(rho)
        lib.orc_solve_direct3(nn, _p(hh), _p(T), _p(rho), None, 0, _p(out))
        return out
    pts = np.ascontiguousarray(points, dtype=np.int64).ravel()
    assert pts.size == 0 or (pts.min() >= 0 and pts.max() < rho.size)
    out = np.empty(pts.size, dtype=np.float64)
    lib.orc_solve_direct3(nn, _p(hh), _p(T), _p(rho), pts.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                          pts.size, _p(out))
    return out


def solve3(algo, rho, h, alpha=ALPHA):
    """Kernel plus FFT solve on a non-cubic box (rho indexed [z,y,x])."""
    n = (rho.shape[2], rho.shape[1], rho.shape[0])
    return solve_fft3(kernel_T3(algo, n, h, alpha), rho, h)


def field_kernel3(algo, a, n, h, alpha=ALPHA):
    """Field kernel F_a on a non-cubic box, shape (n_z+1, n_y+1, n_x+1)."""
    algo = ALGOS.get(algo, algo)
    nn, hh = _dims(n, h)
    F = np.empty((n[2] + 1, n[1] + 1, n[0] + 1), dtype=np.float64)
    _load().orc_field_kernel3(int(algo), int(a), nn, _p(hh), float(alpha), _p(F))
    return F


def solve_field_fft3(F, a, rho, h):
    """E_a through the full doubled grid of a non-cubic box."""
    F, rho = _f64(F), _f64(rho)
    n = (rho.shape[2], rho.shape[1], rho.shape[0])
    assert F.shape == (n[2] + 1, n[1] + 1, n[0] + 1)
    nn, hh = _dims(n, h)
    E = np.empty_like(rho)
    _load().orc_solve_field_fft3(nn, _p(hh), int(a), _p(F), _p(rho), _p(E))
    return E


def solve_field_direct3(F, a, rho, h, points=None):
    """E_a by its defining sum on a non-cubic box, at flat indices (or all)."""
    F, rho = _f64(F), _f64(rho)
    n = (rho.shape[2], rho.shape[1], rho.shape[0])
    assert F.shape == (n[2] + 1, n[1] + 1, n[0] + 1)
    nn, hh = _dims(n, h)
    lib = _load()
    if points is None:
        out = np.empty_like(rho)
        lib.orc_solve_field_direct3(nn, _p(hh), int(a), _p(F), _p(rho), None, 0, _p(out))
        return out
    pts = np.ascontiguousarray(points, dtype=np.int64).ravel()
    assert pts.size == 0 or (pts.min() >= 0 and pts.max() < rho.size)
    out = np.empty(pts.size, dtype=np.float64)
    lib.orc_solve_field_direct3(nn, _p(hh), int(a), _p(F), _p(rho),
                                pts.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), pts.size, _p(out))
    return out


def solve_field3(algo, rho, h, alpha=ALPHA):
    """(E_x, E_y, E_z) on a non-cubic box (rho indexed [z,y,x])."""
    n = (rho.shape[2], rho.shape[1], rho.shape[0])
    return tuple(solve_field_fft3(field_kernel3(algo, a, n, h, alpha), a, rho, h) for a in range(3))


from . import analytic  # noqa: E402  (pure-numpy helpers, no C)

__all__ = ["HE", "VG", "VG_DCT", "ALPHA", "dft1d", "fft1d", "fft3d", "dct1", "dct1_3d",
           "green_vico_hat", "window", "kernel_T", "vg_full", "spectrum", "solve_fft",
           "solve_direct", "solve", "analytic", "num_threads", "set_num_threads", "dst1", "trig1_3d",
           "field_kernel", "solve_field_fft", "field_spectrum", "solve_field_direct", "solve_field",
           "kernel_T3", "solve_fft3", "spectrum3", "solve_direct3", "solve3", "field_kernel3",
           "solve_field_fft3", "solve_field_direct3", "solve_field3"]

