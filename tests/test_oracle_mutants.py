"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a flipped
transform sign, a wrong twiddle index, a dropped factor or scale, an
off-by-one in the frequency grid or the mirror fold, a wrong window or series
coefficient, a wrong stride, a padding bound), builds it with gcc on the CPU
and runs the pins against it: at least one must fail.  The mistakes are made
in a temporary copy; the oracle itself is never modified.  The field
functions have their own planted mistakes (a lost odd extension, a wrong
power or sign or axis of the field kernel, a wrong DST factor) and pins, and
so do the non-cubic ones (one axis's size or spacing used for another, the
cubic window, a wrong fold, scale or transform order).
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.fft

import fsp_inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "fsp_oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("fft_direction", "return sign < 0 ? w : conj(w);", "return sign > 0 ? w : conj(w);"),
    ("twiddle_index", "root_of(R, n, (long long)r * k, sign)", "root_of(R, n, (long long)r * (k + 1), sign)"),
    ("dct_interior_factor", "acc += 2.0 * src[j] * c[((long long)j * k) % (2 * M)];\n            dst[k] = acc;",
     "acc += 1.0 * src[j] * c[((long long)j * k) % (2 * M)];\n            dst[k] = acc;"),
    ("dct_endpoint_sign", "double acc = src[0] + ((k & 1) ? -src[M] : src[M]);\n            for (int j = 1; j < M; ++j) acc += 2.0 * src[j] * c[((long long)j * k) % (2 * M)];\n            dst[k] = acc;",
     "double acc = src[0] + src[M];\n            for (int j = 1; j < M; ++j) acc += 2.0 * src[j] * c[((long long)j * k) % (2 * M)];\n            dst[k] = acc;"),
    ("vg_scale_power", "double scale = 1.0 / (((double)n4 * h) * ((double)n4 * h) * ((double)n4 * h));",
     "double scale = 1.0 / (((double)n4 * h) * ((double)n4 * h));"),
    ("vg_negative_freq_offset", "int jx = sx < 2 * N ? sx : sx - n4;", "int jx = sx < 2 * N ? sx : sx - n4 + 1;"),
    ("he_origin_value", ": 1.0 / (4.0 * ORC_PI);", ": 0.0;"),
    ("mirror_fold", "static inline int fold2(int m, int N) { return m <= N ? m : 2 * N - m; }",
     "static inline int fold2(int m, int N) { return m < N ? m : 2 * N - m - 1; }"),
    ("solve_scale", "double scale = h * h * h / (double)tot;\n    for (int z = 0; z < N; ++z)",
     "double scale = h * h / (double)tot;\n    for (int z = 0; z < N; ++z)"),
    ("vg_window", "double Lt = alpha * sqrt(3.0) * L;", "double Lt = alpha * L;"),
    ("sinc_series", "s = 1.0 - u * u / 6.0 + u * u * u * u / 120.0;", "s = 1.0 - u * u / 3.0 + u * u * u * u / 120.0;"),
    ("fft3d_stride", "ptrdiff_t strides[3] = {1, nx, (ptrdiff_t)nx * ny};", "ptrdiff_t strides[3] = {1, ny, (ptrdiff_t)nx * ny};"),
    ("direct_sum_h3", "out[p] = h * h * h * (sum + comp);", "out[p] = h * h * (sum + comp);"),
    ("padding_bound", "for (int z = 0; z < N; ++z)\n        for (int y = 0; y < N; ++y)\n            for (int x = 0; x < N; ++x) r2[",
     "for (int z = 0; z < N; ++z)\n        for (int y = 0; y < N; ++y)\n            for (int x = 1; x < N; ++x) r2["),
    ("spectrum_scale", "S[((size_t)z * k1 + y) * k1 + x] = creal(g2[((size_t)z * n2 + y) * n2 + x]) * scale;",
     "S[((size_t)z * k1 + y) * k1 + x] = creal(g2[((size_t)z * n2 + y) * n2 + x]) * scale * 8.0;"),
    ("spectrum_index", "S[((size_t)z * k1 + y) * k1 + x] = creal(g2[((size_t)z * n2 + y) * n2 + x]) * scale;",
     "S[((size_t)z * k1 + y) * k1 + x] = creal(g2[((size_t)y * n2 + z) * n2 + x]) * scale;"),
]

# planted mistakes in the field functions (caught by _field_pins)
FIELD_MUTANTS = [
    ("odd_extension_even", "return m == 0 || m == N ? 0.0 : (m < N ? 1.0 : -1.0);",
     "return m == 0 || m == N ? 0.0 : (m < N ? 1.0 : 1.0);"),
    ("he_field_power", "(double)m[a] / (4.0 * ORC_PI * h * h * r2 * sqrt(r2))", "(double)m[a] / (4.0 * ORC_PI * h * h * r2)"),
    ("vg_field_sign", "g[idx] = -I * ka * orc_green_vico_hat(kabs, Lt);", "g[idx] = I * ka * orc_green_vico_hat(kabs, Lt);"),
    ("vg_dct_field_axis", "dk * j[a] * orc_green_vico_hat(", "dk * j[0] * orc_green_vico_hat("),
    ("dst_factor", "acc += 2.0 * x[j] * sin(", "acc += 1.0 * x[j] * sin("),
    ("trig_kind_swap", "tab[e] = kind == 0 ? cos(ORC_PI * (double)e / M) : sin(ORC_PI * (double)e / M);",
     "tab[e] = kind == 1 ? cos(ORC_PI * (double)e / M) : sin(ORC_PI * (double)e / M);"),
    ("field_direct_sign", "double sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);", "double sg = d > 0 ? -1.0 : (d < 0 ? 1.0 : 0.0);"),
    ("field_spectrum_sign", "S[((size_t)z * k1 + y) * k1 + x] = -cimag(", "S[((size_t)z * k1 + y) * k1 + x] = cimag("),
    ("field_solve_scale", "double scale = h * h * h / (double)tot;\n    for (int z = 0; z < N; ++z)\n        for (int y = 0; y < N; ++y)\n            for (int x = 0; x < N; ++x)\n                E[",
     "double scale = h * h / (double)tot;\n    for (int z = 0; z < N; ++z)\n        for (int y = 0; y < N; ++y)\n            for (int x = 0; x < N; ++x)\n                E["),
]


def _build(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation target not found: " + name
    path = os.path.join(tmp, name + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))
    lib = os.path.join(tmp, "lib_" + name + ".so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", lib, path, "-lm"], check=True)
    return lib


def _pins(orc):
    """Name -> passed, for a cheap set of the oracle's pins."""
    from oracle import analytic as A
    res = {}
    r = np.random.default_rng(0)
    x = r.standard_normal(30) + 1j * r.standard_normal(30)
    res["fft_vs_pocketfft"] = np.allclose(orc.fft1d(x, -1), np.fft.fft(x), atol=1e-12) and \
        np.allclose(orc.fft1d(x, 1), np.fft.ifft(x) * 30, atol=1e-12)
    a = r.standard_normal((6, 10, 12)) + 0j
    res["fft3d_vs_fftn"] = np.allclose(orc.fft3d(a, -1), np.fft.fftn(a), atol=1e-11)
    g = r.standard_normal((9, 9, 9))
    res["dct1_vs_scipy"] = np.allclose(orc.dct1_3d(g, 4), scipy.fft.dctn(g, type=1)[:5, :5, :5], atol=1e-10)
    Lt = 1.905
    u = 5e-4
    k = 2 * u / Lt
    ref = 2 * (np.sin(u) / u) ** 2 * (Lt / 2) ** 2
    res["vico_hat"] = abs(orc.green_vico_hat(k, Lt) - ref) < 1e-14 * ref
    full, T = orc.vg_full(4)
    res["vg_sum_rule"] = abs((0.25 ** 3) * full.real.sum() - orc.window(1.0) ** 2 / 2) < 1e-10
    res["vg_equals_vg_dct"] = np.allclose(orc.kernel_T("vg", 4), orc.kernel_T("vg_dct", 4), rtol=1e-12, atol=1e-14)
    for algo in ("he", "vg_dct"):
        T = orc.kernel_T(algo, 6)
        rho = I.random_field(6, 1)
        res["fft_eq_direct_" + algo] = np.allclose(orc.solve_fft(T, rho, 1 / 6), orc.solve_direct(T, rho, 1 / 6),
                                                   rtol=1e-12, atol=1e-14)
    N = 8
    phi = orc.solve("he", I.impulse(N, 1.0, (0, 0, 0)))
    z, y, x3 = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    d = np.sqrt(x3 ** 2 + y ** 2 + z ** 2)
    imp = np.where(d > 0, 1 / (4 * np.pi * (1 / N) * np.maximum(d, 1e-300)), 1 / (4 * np.pi))
    res["he_impulse"] = np.allclose(phi, imp, rtol=1e-12)
    e_vg = A.rel_l2(orc.solve("vg", I.gaussian(16)), A.gaussian_potential(16))
    res["gauss_vg16"] = 1e-4 <= e_vg <= 1e-2
    res["vg_far_field"] = _far_field_err(orc, "vg_dct", 16) < 1e-2
    Ts = np.random.default_rng(7).standard_normal((6, 6, 6))  # no symmetry between its axes
    res["spectrum_vs_dctn"] = np.allclose(orc.spectrum(Ts, 0.2), scipy.fft.dctn(Ts, type=1) * 0.2 ** 3 / 10 ** 3,
                                          rtol=0, atol=1e-12 * np.abs(Ts).max())
    return res


def _far_field_err(orc, algo, N, c=(-0.3, -0.3, -0.3), s=0.04):
    """Max relative error of the potential of an off-centre Gaussian at the
    points more than 1.2 from it (beyond a truncation window shorter than the
    box diagonal)."""
    from oracle import analytic as A
    phi = orc.solve(algo, I.gaussian(N, 1.0, s, c))
    ex = A.gaussian_potential(N, 1.0, s, c)
    x = I.cell_centres(N, 1.0)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    far = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) > 1.2
    return float(np.max(np.abs(phi[far] - ex[far]) / ex[far]))


def _field_pins(orc):
    """Name -> passed, for a cheap set of the field pins."""
    import scipy.fft as sf
    from oracle import analytic as A
    res = {}
    r = np.random.default_rng(3)
    x = r.standard_normal(9)
    res["dst1_vs_scipy"] = np.allclose(orc.dst1(x)[1:8], sf.dst(x[1:8], type=1), atol=1e-12)
    g = r.standard_normal((7, 7, 7))
    want = sf.dct(sf.dct(g, type=1, axis=0), type=1, axis=1)
    inner = sf.dst(want[:, :, 1:6], type=1, axis=2)
    full = np.zeros_like(want)
    full[:, :, 1:6] = inner
    res["trig_vs_scipy"] = np.allclose(orc.trig1_3d(g, 0), full, atol=1e-10)
    res["vg_two_routes"] = all(np.allclose(orc.field_kernel("vg", a, 4), orc.field_kernel("vg_dct", a, 4),
                                           rtol=0, atol=1e-13 * np.abs(orc.field_kernel("vg", a, 4)).max())
                               for a in range(3))
    rho = I.random_field(5, 4)
    ok = True
    for algo in ("he", "vg_dct"):
        for a in range(3):
            F = orc.field_kernel(algo, a, 5)
            e1, e2 = orc.solve_field_fft(F, a, rho, 0.2), orc.solve_field_direct(F, a, rho, 0.2)
            ok = ok and np.allclose(e1, e2, rtol=0, atol=1e-12 * np.abs(e2).max())
    res["fft_eq_direct"] = ok
    N, h, j = 6, 1.0 / 6, (1, 4, 2)
    z, y, x3 = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    d = [(x3 - j[0]) * h, (y - j[1]) * h, (z - j[2]) * h]
    rr = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    imp = I.impulse(N, 1.0, j)
    res["coulomb"] = all(np.allclose(orc.solve_field_fft(orc.field_kernel("he", a, N), a, imp, h),
                                     (rr > 0) * d[a] / (4 * np.pi * np.where(rr > 0, rr, 1.0) ** 3), rtol=1e-10, atol=1e-10)
                         for a in range(3))
    E = orc.solve_field("vg_dct", I.gaussian(16, 1.0, 0.1))
    ex = A.gaussian_field(16, 1.0, 0.1)
    res["gaussian_vg16"] = max(np.abs(E[a] - ex[a]).max() for a in range(3)) < 1e-3 * np.abs(ex[0]).max()
    ok = True
    for a in range(3):
        F = orc.field_kernel("vg_dct", a, 4)
        Fz = F.copy()
        idx = [slice(None)] * 3
        idx[2 - a] = 4
        Fz[tuple(idx)] = 0.0
        ok = ok and np.allclose(orc.field_spectrum(F, a, 0.25), orc.trig1_3d(Fz, a) * 0.25 ** 3 / 8 ** 3,
                                rtol=0, atol=1e-12 * np.abs(Fz).max())
    res["spectrum_two_routes"] = ok
    return res


# planted mistakes in the non-cubic functions (caught by _aniso_pins)
ANISO_MUTANTS = [
    ("he3_spacing_axis", "double dx = x * h[0], dy = y * h[1], dz = z * h[2];",
     "double dx = x * h[0], dy = y * h[0], dz = z * h[2];"),
    ("vg3_dk_axis", "for (int a = 0; a < 3; ++a) dk[a] = 2.0 * ORC_PI / ((double)m[a] * h[a]);",
     "for (int a = 0; a < 3; ++a) dk[a] = 2.0 * ORC_PI / ((double)m[a] * h[0]);"),
    ("vgdct3_dk_size", "for (int a = 0; a < 3; ++a) dk[a] = 2.0 * ORC_PI / (4.0 * n[a] * h[a]);",
     "for (int a = 0; a < 3; ++a) dk[a] = 2.0 * ORC_PI / (4.0 * n[0] * h[a]);"),
    ("window_cubic", "double Lt = alpha * sqrt(Lb[0] * Lb[0] + Lb[1] * Lb[1] + Lb[2] * Lb[2]);",
     "double Lt = alpha * sqrt(3.0) * Lb[0];"),
    ("doubled3_fold_axis", "T[((size_t)fold2(z, n[2]) * k[1] + fold2(y, n[1])) * k[0] + fold2(x, n[0])];",
     "T[((size_t)fold2(z, n[2]) * k[1] + fold2(y, n[0])) * k[0] + fold2(x, n[0])];"),
    ("solve3_scale", "double scale = h[0] * h[1] * h[2] / (double)tot;\n    for (int z = 0; z < n[2]; ++z)",
     "double scale = h[0] * h[0] * h[0] / (double)tot;\n    for (int z = 0; z < n[2]; ++z)"),
    ("he_field3_spacing", "double r[3] = {x * h[0], y * h[1], z * h[2]};", "double r[3] = {x * h[0], y * h[0], z * h[2]};"),
    ("field_doubled3_odd_axis", "odd_sign(m[a], n[a]) * F[((size_t)fold2(z, n[2])", "odd_sign(m[a], n[0]) * F[((size_t)fold2(z, n[2])"),
    ("vg_field3_ka_axis", "double ka = j[a] == -2 * n[a] ? 0.0 : dk[a] * j[a];", "double ka = j[a] == -2 * n[a] ? 0.0 : dk[0] * j[a];"),
    ("spectrum3_scale", "S[((size_t)z * k[1] + y) * k[0] + x] = creal(g2[((size_t)z * d[1] + y) * d[0] + x]) * scale;",
     "S[((size_t)z * k[1] + y) * k[0] + x] = creal(g2[((size_t)z * d[1] + y) * d[0] + x]) * scale * 2.0;"),
    ("vgdct3_scale_axis", "double scale = 1.0 / ((4.0 * n[0] * h[0]) * (4.0 * n[1] * h[1]) * (4.0 * n[2] * h[2]));",
     "double scale = 1.0 / ((4.0 * n[0] * h[0]) * (4.0 * n[0] * h[1]) * (4.0 * n[2] * h[2]));"),
]


def _aniso_pins(orc):
    """Name -> passed, for a cheap set of the non-cubic pins."""
    from oracle import analytic as A
    res = {}
    n, h = (6, 4, 5), (0.2, 0.3, 0.25)
    T = orc.kernel_T("vg_dct", 5)
    res["cube_equals_cubic"] = np.allclose(orc.kernel_T3("vg_dct", (5, 5, 5), (0.2,) * 3), T, rtol=1e-12, atol=1e-15)
    ok = True
    for algo in ("he", "vg_dct"):
        T3 = orc.kernel_T3(algo, n, h)
        rho = I.random_field3(n, 2)
        b = orc.solve_direct3(T3, rho, h)
        ok = ok and np.allclose(orc.solve_fft3(T3, rho, h), b, rtol=0, atol=1e-12 * np.abs(b).max())
    res["fft_eq_direct"] = ok
    res["vg_two_routes"] = np.allclose(orc.kernel_T3("vg", n, h), orc.kernel_T3("vg_dct", n, h), rtol=0,
                                       atol=1e-12 * np.abs(orc.kernel_T3("vg", n, h)).max())
    ok = True
    for algo in ("he", "vg_dct"):
        T3 = orc.kernel_T3(algo, n, h)
        ok = ok and np.allclose(orc.kernel_T3(algo, (n[1], n[0], n[2]), (h[1], h[0], h[2])), np.swapaxes(T3, 1, 2),
                                rtol=1e-10, atol=1e-14)
    res["axis_exchange"] = ok
    nn, hh, j = (7, 5, 6), (0.1, 0.17, 0.13), (2, 4, 1)
    rho = np.zeros((nn[2], nn[1], nn[0]))
    rho[j[2], j[1], j[0]] = 1.0 / (hh[0] * hh[1] * hh[2])
    z, y, x = np.meshgrid(np.arange(nn[2]), np.arange(nn[1]), np.arange(nn[0]), indexing="ij")
    r = np.sqrt(((x - j[0]) * hh[0]) ** 2 + ((y - j[1]) * hh[1]) ** 2 + ((z - j[2]) * hh[2]) ** 2)
    want = np.where(r > 0, 1.0 / (4 * np.pi * np.where(r > 0, r, 1.0)), 1.0 / (4 * np.pi))
    res["he_impulse"] = np.allclose(orc.solve3("he", rho, hh), want, rtol=1e-10)
    ng, Lg = (24, 16, 32), (1.0, 0.8, 1.2)
    hg = tuple(Lg[a] / ng[a] for a in range(3))
    e = A.e_max(orc.solve3("vg_dct", I.gaussian3(ng, Lg, 0.08), hg), A.gaussian_potential3(ng, Lg, 0.08))
    res["gaussian_vg"] = e < 1e-6
    nf, Lf, c = (16, 16, 32), (1.0, 1.0, 2.0), (-0.25, -0.25, -0.75)
    hf = tuple(Lf[a] / nf[a] for a in range(3))
    phi = orc.solve3("vg_dct", I.gaussian3(nf, Lf, 0.05, c), hf)
    ex = A.gaussian_potential3(nf, Lf, 0.05, c)
    zz = I.cell_centres(nf[2], Lf[2])[:, None, None] - c[2]
    yy = I.cell_centres(nf[1], Lf[1])[None, :, None] - c[1]
    xx = I.cell_centres(nf[0], Lf[0])[None, None, :] - c[0]
    far = np.sqrt(xx * xx + yy * yy + zz * zz) > 1.2
    res["far_field"] = float(np.max(np.abs(phi[far] - ex[far]) / ex[far])) < 1e-2
    import scipy.fft as sfft
    T3 = orc.kernel_T3("vg_dct", n, h)
    res["spectrum3_vs_dctn"] = np.allclose(orc.spectrum3(T3, h),
                                           sfft.dctn(T3, type=1) * h[0] * h[1] * h[2] / (8.0 * n[0] * n[1] * n[2]),
                                           rtol=0, atol=1e-12 * np.abs(T3).max() * h[0] * h[1] * h[2])
    # the field on a non-cubic box
    nf3, hf3 = (6, 4, 5), (0.2, 0.3, 0.25)
    rr = I.random_field3(nf3, 6)
    ok_routes, ok_direct = True, True
    for a in range(3):
        Fv, Fd = orc.field_kernel3("vg", a, nf3, hf3), orc.field_kernel3("vg_dct", a, nf3, hf3)
        ok_routes = ok_routes and np.allclose(Fv, Fd, rtol=0, atol=1e-12 * np.abs(Fv).max())
        for algo in ("he", "vg_dct"):
            F = orc.field_kernel3(algo, a, nf3, hf3)
            e2 = orc.solve_field_direct3(F, a, rr, hf3)
            ok_direct = ok_direct and np.allclose(orc.solve_field_fft3(F, a, rr, hf3), e2, rtol=0,
                                                  atol=1e-12 * np.abs(e2).max())
    res["field_vg_two_routes"] = ok_routes
    res["field_fft_eq_direct"] = ok_direct
    ni, hi, j = (7, 5, 6), (0.1, 0.17, 0.13), (2, 4, 1)
    rho = np.zeros((ni[2], ni[1], ni[0]))
    rho[j[2], j[1], j[0]] = 1.0 / (hi[0] * hi[1] * hi[2])
    z, y, x = np.meshgrid(np.arange(ni[2]), np.arange(ni[1]), np.arange(ni[0]), indexing="ij")
    d = [(x - j[0]) * hi[0], (y - j[1]) * hi[1], (z - j[2]) * hi[2]]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    res["field_coulomb"] = all(
        np.allclose(orc.solve_field_fft3(orc.field_kernel3("he", a, ni, hi), a, rho, hi),
                    (r > 0) * d[a] / (4 * np.pi * np.where(r > 0, r, 1.0) ** 3), rtol=1e-10, atol=1e-10)
        for a in range(3))
    return res


@pytest.fixture(scope="module")
def baseline(orc):
    return _pins(orc)


def test_pins_pass_on_the_oracle(baseline):
    assert all(baseline.values()), baseline


def test_field_pins_pass_on_the_oracle(orc):
    res = _field_pins(orc)
    assert all(res.values()), res


def _run_mutant(orc, name, old, new, pins):
    with tempfile.TemporaryDirectory() as tmp:
        path = _build(name, old, new, tmp)
        saved = orc._lib
        try:
            orc._lib = None
            mutant = ctypes.CDLL(path)
            orig_build = orc._build.build
            orc._build.build = lambda force=False: path  # load the mutant instead
            orc._load()
            res = pins(orc)
        finally:
            orc._build.build = orig_build
            orc._lib = saved
        del mutant
    return res


def test_aniso_pins_pass_on_the_oracle(orc):
    res = _aniso_pins(orc)
    assert all(res.values()), res


@pytest.mark.parametrize("name,old,new", ANISO_MUTANTS, ids=[m[0] for m in ANISO_MUTANTS])
def test_planted_aniso_mistake_fails_a_pin(orc, name, old, new):
    res = _run_mutant(orc, name, old, new, _aniso_pins)
    failed = [k for k, ok in res.items() if not ok]
    assert failed, "no non-cubic pin caught the planted mistake " + name


@pytest.mark.parametrize("name,old,new", FIELD_MUTANTS, ids=[m[0] for m in FIELD_MUTANTS])
def test_planted_field_mistake_fails_a_pin(orc, name, old, new):
    res = _run_mutant(orc, name, old, new, _field_pins)
    failed = [k for k, ok in res.items() if not ok]
    assert failed, "no field pin caught the planted mistake " + name


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(orc, name, old, new):
    res = _run_mutant(orc, name, old, new, _pins)
    failed = [k for k, ok in res.items() if not ok]
    assert failed, "no pin caught the planted mistake " + name
