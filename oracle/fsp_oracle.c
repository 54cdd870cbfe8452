/*
 * fsp_oracle.c -- plain, slow, FP64 CPU oracle for the free-space spectral
 * Poisson solver of Mayani et al., "A Massively Parallel Performance Portable
 * Free-space Spectral Poisson Solver" (arXiv 2405.02603).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) may link, import or call this file; only the tests, the
 * smoke check and the benchmark's CPU-baseline leg use it.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes (all in double precision, no blocking or fusion beyond the
 * definitions cited below):
 *   - orc_dft1d        : the DFT by its definition, O(n^2).
 *   - orc_fft1d/3d     : a textbook recursive mixed-radix decimation-in-time
 *                        Cooley-Tukey FFT (any n; prime factors > 5 fall back
 *                        to an O(p^2) combine), unnormalised.
 *   - orc_dct1_1d      : the type-I DCT by its definition (Sec. 2.4, "Modified
 *                        Vico-Greengard": the real, even spectrum turns the 4N
 *                        DFT into a DCT; the paper's availability note names
 *                        the DCT of type 1).
 *   - orc_kernel_T     : the real-space discrete kernel T[m], m in [0,N]^3, of
 *                        each method: Hockney-Eastwood (Sec. 2.2, step 3, with
 *                        the regularised origin value), Vico-Greengard on the
 *                        (4N)^3 grid (Sec. 2.3, Eq. green_vico), and the
 *                        memory-reduced (2N+1)^3 DCT-I variant (Sec. 2.4).
 *   - orc_solve_fft    : Hockney-Eastwood steps 1-5 (Sec. 2.2) on the full
 *                        (2N)^3 complex grid, no pruning: pad, FFT rho_2 and
 *                        G_2, multiply, inverse FFT, scale by h^3, restrict.
 *   - orc_solve_direct : the discrete convolution phi_i = h^3 sum_j T[i-j] rho_j
 *                        evaluated term by term (Sec. 1, the O(N_g^2) sum).
 *   - orc_kernel_T3, orc_spectrum3, orc_solve_fft3, orc_solve_direct3 : the
 *                        same method on a box of N_x x N_y x N_z cells with
 *                        spacings h_x, h_y, h_z (the non-cubic grids the
 *                        paper's weak-scaling runs use, Sec. 3.2); the window
 *                        is alpha times the box diagonal.
 *   - orc_field_kernel3, orc_solve_field_fft3, orc_solve_field_direct3 : the
 *                        field on those boxes.
 *   - orc_dst1_1d, orc_trig1_3d, orc_field_kernel, orc_solve_field_fft,
 *     orc_field_spectrum, orc_solve_field_direct : the field E = -grad phi of
 *                        Appendix B (Eq. efield), as the convolution of rho
 *                        with the field kernel F = -grad G of each method (the
 *                        field-kernel reading is stated at orc_field_kernel).
 *
 * Conventions (the readings of the paper this oracle takes):
 *   - Sign: G = +1/(4 pi |x|) with eps0 = 1 (Sec. 1, Eq. convolution_eq), so
 *     phi = G * rho and Lap(phi) = -rho.  The Hockney-Eastwood origin value is
 *     therefore +1/(4 pi) (Sec. 2.2 prints -1/(4 pi) in the paper's opposite
 *     sign convention), used literally, not scaled by h.
 *   - Vico-Greengard window: L_t = alpha * sqrt(3) * L_box with alpha = 1.1
 *     (Sec. 2.3); frequency grid k_j = 2 pi j / (4 N h), j in [-2N, 2N)^3,
 *     stored at index j mod 4N; inverse transform scaled by (4 N h)^-3.
 *   - Arrays are C order with x fastest: index (z*ny + y)*nx + x.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double ORC_PI = 3.14159265358979323846264338327950288;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* exp(sign * 2 pi i * e / n) for an integer exponent e, reduced mod n first. */
static cplx unit_root(long long e, long long n, int sign) {
    long long r = e % n;
    if (r < 0) r += n;
    double a = 2.0 * ORC_PI * (double)r / (double)n;
    return cos(a) + (double)sign * sin(a) * I;
}

/* ---------------------------------------------------------------- DFT -- */
/* X[k] = sum_j x[j] exp(sign 2 pi i j k / n), the definition, O(n^2). */
void orc_dft1d(int n, const cplx *x, cplx *X, int sign) {
    for (int k = 0; k < n; ++k) {
        cplx acc = 0;
        for (int j = 0; j < n; ++j) acc += x[j] * unit_root((long long)j * k, n, sign);
        X[k] = acc;
    }
}

/* ------------------------------------------------- textbook mixed FFT -- */
static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* Roots table for one transform length n: W[e] = exp(-2 pi i e / n). */
typedef struct {
    int n;
    cplx *W;
} roots_t;

static roots_t roots_make(int n) {
    roots_t r;
    r.n = n;
    r.W = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int e = 0; e < n; ++e) r.W[e] = unit_root(e, n, -1);
    return r;
}
static void roots_free(roots_t *r) { free(r->W); r->W = NULL; }

/* exp(sign 2 pi i e / m) for m dividing the table length. */
static inline cplx root_of(const roots_t *R, int m, long long e, int sign) {
    long long r = e % m;
    if (r < 0) r += m;
    cplx w = R->W[(size_t)(r * (R->n / m))];
    return sign < 0 ? w : conj(w);
}

/*
 * Decimation in time: for n = p*m with p the smallest prime factor,
 *   Y_r = FFT_m(x[r], x[r+p], x[r+2p], ...)         r in [0,p)
 *   X[k + m q] = sum_r exp(s 2 pi i r (k + m q) / n) Y_r[k]
 * Input read with a stride, output written contiguously; tmp holds p values.
 */
static void fft_rec(int n, const cplx *in, ptrdiff_t stride, cplx *out, int sign,
                    const roots_t *R, cplx *tmp) {
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_factor(n), m = n / p;
    for (int r = 0; r < p; ++r) fft_rec(m, in + r * stride, stride * p, out + (size_t)r * m, sign, R, tmp);
    for (int k = 0; k < m; ++k) {
        for (int r = 0; r < p; ++r) tmp[r] = out[(size_t)r * m + k] * root_of(R, n, (long long)r * k, sign);
        for (int q = 0; q < p; ++q) {
            cplx acc = 0;
            for (int r = 0; r < p; ++r) acc += tmp[r] * root_of(R, p, (long long)r * q, sign);
            out[(size_t)q * m + k] = acc;
        }
    }
}

/* Largest prime factor bound used for the per-call tmp buffer. */
static int largest_prime(int n) {
    int best = 1;
    while (n > 1) {
        int p = smallest_factor(n);
        if (p > best) best = p;
        n /= p;
    }
    return best;
}

/* Unnormalised 1D FFT, X[k] = sum_j x[j] exp(sign 2 pi i j k / n). */
void orc_fft1d(int n, const cplx *x, cplx *X, int sign) {
    roots_t R = roots_make(n);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)largest_prime(n));
    fft_rec(n, x, 1, X, sign, &R, tmp);
    free(tmp);
    roots_free(&R);
}

/* In-place unnormalised 3D FFT of a (nz, ny, nx) array along every axis. */
void orc_fft3d(int nx, int ny, int nz, cplx *a, int sign) {
    int dims[3] = {nx, ny, nz};
    ptrdiff_t strides[3] = {1, nx, (ptrdiff_t)nx * ny};
    for (int ax = 0; ax < 3; ++ax) {
        int n = dims[ax];
        ptrdiff_t s = strides[ax];
        /* the lines orthogonal to axis ax: two outer index ranges */
        int o1n = dims[(ax + 1) % 3], o2n = dims[(ax + 2) % 3];
        ptrdiff_t o1s = strides[(ax + 1) % 3], o2s = strides[(ax + 2) % 3];
        roots_t R = roots_make(n);
        long long lines = (long long)o1n * o2n;
#pragma omp parallel
        {
            cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)n);
            cplx *res = (cplx *)malloc(sizeof(cplx) * (size_t)n);
            cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)largest_prime(n));
#pragma omp for schedule(static)
            for (long long L = 0; L < lines; ++L) {
                int i1 = (int)(L % o1n), i2 = (int)(L / o1n);
                cplx *base = a + i1 * o1s + i2 * o2s;
                for (int j = 0; j < n; ++j) line[j] = base[j * s];
                fft_rec(n, line, 1, res, sign, &R, tmp);
                for (int j = 0; j < n; ++j) base[j * s] = res[j];
            }
            free(line);
            free(res);
            free(tmp);
        }
        roots_free(&R);
    }
}

/* ------------------------------------------------------------- DCT-I -- */
/*
 * Unnormalised type-I DCT of M+1 samples (FFTW REDFT00 convention):
 *   X[k] = x[0] + (-1)^k x[M] + 2 sum_{j=1}^{M-1} x[j] cos(pi j k / M),  k in [0,M].
 */
void orc_dct1_1d(int M, const double *x, double *X) {
    for (int k = 0; k <= M; ++k) {
        double acc = x[0] + ((k & 1) ? -x[M] : x[M]);
        for (int j = 1; j < M; ++j) acc += 2.0 * x[j] * cos(ORC_PI * (double)(((long long)j * k) % (2 * M)) / M);
        X[k] = acc;
    }
}

/*
 * 3D DCT-I of a (M+1)^3 array as the tensor product of 1D DCT-Is along x, y
 * and z, evaluated only at outputs k in [0,K]^3 (K <= M).  Returns a (K+1)^3
 * array.  Per axis the same direct sum as orc_dct1_1d, with the cosines
 * cos(pi e / M), e in [0, 2M), looked up in a table.
 */
void orc_dct1_3d(int M, int K, const double *x, double *X) {
    int n = M + 1, k1 = K + 1;
    double *c = (double *)malloc(sizeof(double) * (size_t)(2 * M));
    for (int e = 0; e < 2 * M; ++e) c[e] = cos(ORC_PI * (double)e / M);
    /* axis x: (n z, n y, n x) -> (n z, n y, k1 kx) */
    double *t1 = (double *)malloc(sizeof(double) * (size_t)n * n * k1);
#pragma omp parallel for schedule(static)
    for (long long L = 0; L < (long long)n * n; ++L) {
        const double *src = x + L * n;
        double *dst = t1 + L * k1;
        for (int k = 0; k < k1; ++k) {
            double acc = src[0] + ((k & 1) ? -src[M] : src[M]);
            for (int j = 1; j < M; ++j) acc += 2.0 * src[j] * c[((long long)j * k) % (2 * M)];
            dst[k] = acc;
        }
    }
    /* axis y: (n z, n y, k1) -> (n z, k1 ky, k1) */
    double *t2 = (double *)malloc(sizeof(double) * (size_t)n * k1 * k1);
#pragma omp parallel for schedule(static)
    for (long long L = 0; L < (long long)n * k1; ++L) {
        int z = (int)(L / k1), kx = (int)(L % k1);
        const double *src = t1 + (size_t)z * n * k1 + kx;
        double *dst = t2 + (size_t)z * k1 * k1 + kx;
        for (int k = 0; k < k1; ++k) {
            double acc = src[0] + ((k & 1) ? -src[(size_t)M * k1] : src[(size_t)M * k1]);
            for (int j = 1; j < M; ++j) acc += 2.0 * src[(size_t)j * k1] * c[((long long)j * k) % (2 * M)];
            dst[(size_t)k * k1] = acc;
        }
    }
    /* axis z: (n z, k1, k1) -> (k1 kz, k1, k1) */
#pragma omp parallel for schedule(static)
    for (long long L = 0; L < (long long)k1 * k1; ++L) {
        const double *src = t2 + L;
        double *dst = X + L;
        size_t s = (size_t)k1 * k1;
        for (int k = 0; k < k1; ++k) {
            double acc = src[0] + ((k & 1) ? -src[(size_t)M * s] : src[(size_t)M * s]);
            for (int j = 1; j < M; ++j) acc += 2.0 * src[(size_t)j * s] * c[((long long)j * k) % (2 * M)];
            dst[(size_t)k * s] = acc;
        }
    }
    free(t2);
    free(t1);
    free(c);
}

/* ------------------------------------------------------------- DST-I -- */
/*
 * Unnormalised type-I DST of the M-1 interior samples of x[0..M] (FFTW
 * RODFT00 convention, the two zero end points kept in place):
 *   X[k] = 2 sum_{j=1}^{M-1} x[j] sin(pi j k / M),  k in [0,M]  (X[0] = X[M] = 0).
 * x[0] and x[M] are not read.  It is the DFT of length 2M of the odd
 * extension of x, divided by -i.
 */
void orc_dst1_1d(int M, const double *x, double *X) {
    for (int k = 0; k <= M; ++k) {
        double acc = 0.0;
        for (int j = 1; j < M; ++j) acc += 2.0 * x[j] * sin(ORC_PI * (double)(((long long)j * k) % (2 * M)) / M);
        X[k] = acc;
    }
}

/*
 * One axis of a separable transform of a 3D array (x fastest): every line
 * along `axis` (0 = x, 1 = y, 2 = z) of M+1 samples is replaced by its DCT-I
 * (kind 0) or DST-I (kind 1), evaluated at outputs [0,K].  in has extents
 * (nx, ny, nz); out has the same extents except K+1 along `axis`.
 */
static void axis_trig(int M, int K, int kind, int axis, int nx, int ny, int nz, const double *in, double *out) {
    int ext[3] = {nx, ny, nz}, oext[3] = {nx, ny, nz};
    oext[axis] = K + 1;
    size_t istr[3] = {1, (size_t)nx, (size_t)nx * ny};
    size_t ostr[3] = {1, (size_t)oext[0], (size_t)oext[0] * oext[1]};
    int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;  /* the two other axes */
    double *tab = (double *)malloc(sizeof(double) * (size_t)(2 * M));
    for (int e = 0; e < 2 * M; ++e) tab[e] = kind == 0 ? cos(ORC_PI * (double)e / M) : sin(ORC_PI * (double)e / M);
    long long lines = (long long)ext[a1] * ext[a2];
#pragma omp parallel for schedule(static)
    for (long long L = 0; L < lines; ++L) {
        int u = (int)(L % ext[a1]), v = (int)(L / ext[a1]);
        const double *src = in + (size_t)u * istr[a1] + (size_t)v * istr[a2];
        double *dst = out + (size_t)u * ostr[a1] + (size_t)v * ostr[a2];
        size_t si = istr[axis], so = ostr[axis];
        for (int k = 0; k <= K; ++k) {
            double acc = kind == 0 ? src[0] + ((k & 1) ? -src[(size_t)M * si] : src[(size_t)M * si]) : 0.0;
            for (int j = 1; j < M; ++j) acc += 2.0 * src[(size_t)j * si] * tab[((long long)j * k) % (2 * M)];
            dst[(size_t)k * so] = acc;
        }
    }
    free(tab);
}

/*
 * 3D transform of a (M+1)^3 array: DST-I along axis `odd` (0 = x, 1 = y,
 * 2 = z) and DCT-I along the two others (odd < 0: DCT-I along all three),
 * evaluated at outputs [0,K]^3 (K <= M).  Returns a (K+1)^3 array.
 */
void orc_trig1_3d(int M, int K, int odd, const double *x, double *X) {
    int n = M + 1, k1 = K + 1;
    double *t1 = (double *)malloc(sizeof(double) * (size_t)n * n * k1);
    double *t2 = (double *)malloc(sizeof(double) * (size_t)n * k1 * k1);
    axis_trig(M, K, odd == 0, 0, n, n, n, x, t1);
    axis_trig(M, K, odd == 1, 1, k1, n, n, t1, t2);
    axis_trig(M, K, odd == 2, 2, k1, k1, n, t2, X);
    free(t2);
    free(t1);
}

/* ------------------------------------------------- Green's functions -- */
enum { ORC_HE = 0, ORC_VG = 1, ORC_VG_DCT = 2 };

/*
 * Vico-Greengard truncated spectral kernel, Eq. green_vico:
 *   G_L(k) = 2 (sin(L_t |k| / 2) / |k|)^2,   G_L(0) = L_t^2 / 2 (its limit).
 * Written as 2 (L_t/2)^2 sinc^2(L_t |k| / 2); for small arguments the sinc
 * uses its Taylor series 1 - u^2/6 + u^4/120 (error below u^6/5040).
 */
double orc_green_vico_hat(double kabs, double Lt) {
    double u = 0.5 * Lt * kabs;
    double s;
    if (fabs(u) < 1e-3)
        s = 1.0 - u * u / 6.0 + u * u * u * u / 120.0;
    else
        s = sin(u) / u;
    return 2.0 * (0.5 * Lt) * (0.5 * Lt) * s * s;
}

/* Free-space Green's function G(x) = 1/(4 pi |x|) (Sec. 1). */
static double green_free(double r) { return 1.0 / (4.0 * ORC_PI * r); }

/*
 * Vico-Greengard, original method (Sec. 2.3): sample G_L on the (4N)^3
 * frequency grid j in [-2N, 2N)^3 (stored at j mod 4N), inverse DFT, scale,
 * return the full (4N)^3 complex result in `full` (may be NULL) and the
 * restriction T[m], m in [0,N]^3, in T.
 */
void orc_vg_full(int N, double h, double Lt, cplx *full_out, double *T) {
    int n4 = 4 * N;
    size_t tot = (size_t)n4 * n4 * n4;
    cplx *g = (cplx *)malloc(sizeof(cplx) * tot);
    double dk = 2.0 * ORC_PI / ((double)n4 * h);
#pragma omp parallel for schedule(static)
    for (long long idx = 0; idx < (long long)tot; ++idx) {
        int sx = (int)(idx % n4), sy = (int)((idx / n4) % n4), sz = (int)(idx / ((long long)n4 * n4));
        /* storage index s holds frequency j = s for s < 2N, s - 4N otherwise */
        int jx = sx < 2 * N ? sx : sx - n4;
        int jy = sy < 2 * N ? sy : sy - n4;
        int jz = sz < 2 * N ? sz : sz - n4;
        double kabs = dk * sqrt((double)jx * jx + (double)jy * jy + (double)jz * jz);
        g[idx] = orc_green_vico_hat(kabs, Lt);
    }
    orc_fft3d(n4, n4, n4, g, +1);
    double scale = 1.0 / (((double)n4 * h) * ((double)n4 * h) * ((double)n4 * h));
    for (size_t i = 0; i < tot; ++i) g[i] *= scale;
    int k1 = N + 1;
    for (int z = 0; z < k1; ++z)
        for (int y = 0; y < k1; ++y)
            for (int x = 0; x < k1; ++x)
                T[((size_t)z * k1 + y) * k1 + x] = creal(g[((size_t)z * n4 + y) * n4 + x]);
    if (full_out) memcpy(full_out, g, sizeof(cplx) * tot);
    free(g);
}

/*
 * Real-space kernel T[m] for m in [0,N]^3 (x fastest), for the method `algo`.
 * L is the box side (h = L/N), alpha the Vico-Greengard window factor.
 */
void orc_kernel_T(int algo, int N, double L, double alpha, double *T) {
    double h = L / N;
    int k1 = N + 1;
    double Lt = alpha * sqrt(3.0) * L;
    if (algo == ORC_HE) {
        /* Sec. 2.2 step 3: G sampled at m h, with the origin regularised. */
        for (int z = 0; z < k1; ++z)
            for (int y = 0; y < k1; ++y)
                for (int x = 0; x < k1; ++x) {
                    double r = h * sqrt((double)x * x + (double)y * y + (double)z * z);
                    T[((size_t)z * k1 + y) * k1 + x] = (x | y | z) ? green_free(r) : 1.0 / (4.0 * ORC_PI);
                }
    } else if (algo == ORC_VG) {
        orc_vg_full(N, h, Lt, NULL, T);
    } else {
        /* Sec. 2.4: G_L sampled on j in [0,2N]^3, 3D DCT-I, keep [0,N]^3. */
        int M = 2 * N, n = M + 1;
        double *g = (double *)malloc(sizeof(double) * (size_t)n * n * n);
        double dk = 2.0 * ORC_PI / (4.0 * N * h);
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x)
                    g[((size_t)z * n + y) * n + x] =
                        orc_green_vico_hat(dk * sqrt((double)x * x + (double)y * y + (double)z * z), Lt);
        orc_dct1_3d(M, N, g, T);
        double scale = 1.0 / ((4.0 * N * h) * (4.0 * N * h) * (4.0 * N * h));
        for (size_t i = 0; i < (size_t)k1 * k1 * k1; ++i) T[i] *= scale;
        free(g);
    }
}

/* ------------------------------------------------------------ solves -- */
/* Mirror index on the doubled grid: m in [0,2N) -> |m| with m >= N read as m-2N. */
static inline int fold2(int m, int N) { return m <= N ? m : 2 * N - m; }

/*
 * Hockney-Eastwood steps 1-5 (Sec. 2.2), used with the kernel T of any method:
 *   rho_2 = rho zero-padded to (2N)^3, G_2[m] = T[fold(m)] on (2N)^3,
 *   phi_2 = h^3 IDFT{ DFT{rho_2} DFT{G_2} }  (IDFT includes 1/(2N)^3),
 *   phi   = phi_2 restricted to [0,N)^3.
 * rho, phi: N^3 doubles.  T: (N+1)^3 doubles.  Full (2N)^3 complex grids.
 */
void orc_solve_fft(int N, double h, const double *T, const double *rho, double *phi) {
    int n2 = 2 * N, k1 = N + 1;
    size_t tot = (size_t)n2 * n2 * n2;
    cplx *r2 = (cplx *)calloc(tot, sizeof(cplx));
    cplx *g2 = (cplx *)malloc(sizeof(cplx) * tot);
    for (int z = 0; z < N; ++z)
        for (int y = 0; y < N; ++y)
            for (int x = 0; x < N; ++x) r2[((size_t)z * n2 + y) * n2 + x] = rho[((size_t)z * N + y) * N + x];
    for (int z = 0; z < n2; ++z)
        for (int y = 0; y < n2; ++y)
            for (int x = 0; x < n2; ++x)
                g2[((size_t)z * n2 + y) * n2 + x] =
                    T[((size_t)fold2(z, N) * k1 + fold2(y, N)) * k1 + fold2(x, N)];
    orc_fft3d(n2, n2, n2, r2, -1);
    orc_fft3d(n2, n2, n2, g2, -1);
    for (size_t i = 0; i < tot; ++i) r2[i] *= g2[i];
    orc_fft3d(n2, n2, n2, r2, +1);
    double scale = h * h * h / (double)tot;
    for (int z = 0; z < N; ++z)
        for (int y = 0; y < N; ++y)
            for (int x = 0; x < N; ++x)
                phi[((size_t)z * N + y) * N + x] = creal(r2[((size_t)z * n2 + y) * n2 + x]) * scale;
    free(g2);
    free(r2);
}

/*
 * The spectrum the solve multiplies by, on the (N+1)^3 non-redundant octant:
 *   S[q] = h^3 / (2N)^3 * DFT_{2N}{G_2}[q],  q in [0,N]^3  (real part).
 * Computed through the full (2N)^3 complex FFT of the mirrored kernel G_2.
 */
void orc_spectrum(int N, double h, const double *T, double *S) {
    int n2 = 2 * N, k1 = N + 1;
    size_t tot = (size_t)n2 * n2 * n2;
    cplx *g2 = (cplx *)malloc(sizeof(cplx) * tot);
    for (int z = 0; z < n2; ++z)
        for (int y = 0; y < n2; ++y)
            for (int x = 0; x < n2; ++x)
                g2[((size_t)z * n2 + y) * n2 + x] =
                    T[((size_t)fold2(z, N) * k1 + fold2(y, N)) * k1 + fold2(x, N)];
    orc_fft3d(n2, n2, n2, g2, -1);
    double scale = h * h * h / (double)tot;
    for (int z = 0; z < k1; ++z)
        for (int y = 0; y < k1; ++y)
            for (int x = 0; x < k1; ++x)
                S[((size_t)z * k1 + y) * k1 + x] = creal(g2[((size_t)z * n2 + y) * n2 + x]) * scale;
    free(g2);
}

/*
 * The discrete convolution by its definition (Sec. 1, the O(N_g^2) sum):
 *   phi_i = h^3 sum_{j in [0,N)^3} T[|i_x-j_x|, |i_y-j_y|, |i_z-j_z|] rho_j
 * evaluated at the `npts` flat output indices `pts` (all N^3 if pts == NULL).
 * The N^3 products are accumulated with Neumaier's compensated summation, so
 * the sum is exact to a few roundings whatever N (plain accumulation of N^3
 * terms drifts by about N^3 eps).
 */
void orc_solve_direct(int N, double h, const double *T, const double *rho, const long long *pts, long long npts,
                      double *out) {
    int k1 = N + 1;
    long long total = pts ? npts : (long long)N * N * N;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long p = 0; p < total; ++p) {
        long long i = pts ? pts[p] : p;
        int ix = (int)(i % N), iy = (int)((i / N) % N), iz = (int)(i / ((long long)N * N));
        double sum = 0.0, comp = 0.0;
        for (int jz = 0; jz < N; ++jz)
            for (int jy = 0; jy < N; ++jy) {
                const double *Trow = T + ((size_t)abs(iz - jz) * k1 + abs(iy - jy)) * k1;
                const double *rrow = rho + ((size_t)jz * N + jy) * N;
                for (int jx = 0; jx < N; ++jx) {
                    double t = Trow[abs(ix - jx)] * rrow[jx];
                    double s = sum + t;
                    if (fabs(sum) >= fabs(t))
                        comp += (sum - s) + t;
                    else
                        comp += (t - s) + sum;
                    sum = s;
                }
            }
        out[p] = h * h * h * (sum + comp);
    }
}

/* ---------------------------------------------------------- the field -- */
/*
 * Field kernel F_a[m] = -dG/dx_a at x = m h, m in [0,N]^3 (a = 0, 1, 2 for
 * x, y, z), so that E_a = h^3 sum_j F_a[i-j] rho_j is the field E = -grad phi
 * of Appendix B (Eq. efield) for the potential phi = G * rho of Sec. 1.  F_a is
 * odd in m_a and even in the two other indices, so the octant fixes it.  The
 * paper does not say how the gradient is discretised; the reading taken here
 * differentiates each method's Green's function before sampling:
 *   HE (Sec. 2.2): the gradient of 1/(4 pi |x|) sampled at m h,
 *       F_a[m] = m_a / (4 pi h^2 |m|^3), and F_a[0] = 0 (odd symmetry).
 *   VG (Sec. 2.3): the inverse transform of -i k_a G_L(k) on the (4N)^3 grid
 *       (the gradient of the truncated kernel), with the Nyquist plane
 *       j_a = -2N set to zero (k_a has no odd value there), scaled by
 *       (4Nh)^-3, real part.
 *   VG-DCT (Sec. 2.4): the same sum through the (2N+1)^3 octant: k_a G_L(k)
 *       sampled at j in [0,2N]^3 is odd in j_a, so the 4N sum becomes a DST-I
 *       along a and DCT-I along the others, scaled by (4Nh)^-3.
 */
void orc_field_kernel(int algo, int a, int N, double L, double alpha, double *F) {
    double h = L / N;
    int k1 = N + 1;
    double Lt = alpha * sqrt(3.0) * L;
    if (algo == ORC_HE) {
        for (int z = 0; z < k1; ++z)
            for (int y = 0; y < k1; ++y)
                for (int x = 0; x < k1; ++x) {
                    int m[3] = {x, y, z};
                    double r2 = (double)x * x + (double)y * y + (double)z * z;
                    F[((size_t)z * k1 + y) * k1 + x] =
                        (x | y | z) ? (double)m[a] / (4.0 * ORC_PI * h * h * r2 * sqrt(r2)) : 0.0;
                }
    } else if (algo == ORC_VG) {
        int n4 = 4 * N;
        size_t tot = (size_t)n4 * n4 * n4;
        cplx *g = (cplx *)malloc(sizeof(cplx) * tot);
        double dk = 2.0 * ORC_PI / ((double)n4 * h);
#pragma omp parallel for schedule(static)
        for (long long idx = 0; idx < (long long)tot; ++idx) {
            int s3[3] = {(int)(idx % n4), (int)((idx / n4) % n4), (int)(idx / ((long long)n4 * n4))};
            int j[3];
            for (int c = 0; c < 3; ++c) j[c] = s3[c] < 2 * N ? s3[c] : s3[c] - n4;
            double kabs = dk * sqrt((double)j[0] * j[0] + (double)j[1] * j[1] + (double)j[2] * j[2]);
            double ka = j[a] == -2 * N ? 0.0 : dk * j[a];
            g[idx] = -I * ka * orc_green_vico_hat(kabs, Lt);
        }
        orc_fft3d(n4, n4, n4, g, +1);
        double scale = 1.0 / (((double)n4 * h) * ((double)n4 * h) * ((double)n4 * h));
        for (int z = 0; z < k1; ++z)
            for (int y = 0; y < k1; ++y)
                for (int x = 0; x < k1; ++x)
                    F[((size_t)z * k1 + y) * k1 + x] = creal(g[((size_t)z * n4 + y) * n4 + x]) * scale;
        free(g);
    } else {
        int M = 2 * N, n = M + 1;
        double *g = (double *)malloc(sizeof(double) * (size_t)n * n * n);
        double dk = 2.0 * ORC_PI / (4.0 * N * h);
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    int j[3] = {x, y, z};
                    g[((size_t)z * n + y) * n + x] =
                        dk * j[a] * orc_green_vico_hat(dk * sqrt((double)x * x + (double)y * y + (double)z * z), Lt);
                }
        orc_trig1_3d(M, N, a, g, F);
        double scale = 1.0 / ((4.0 * N * h) * (4.0 * N * h) * (4.0 * N * h));
        for (size_t i = 0; i < (size_t)k1 * k1 * k1; ++i) F[i] *= scale;
        free(g);
    }
}

/* Sign of the odd extension on the doubled grid: +1 on (0,N), -1 on (N,2N),
 * 0 at 0 and at N (an odd sequence of period 2N vanishes there; no physical
 * output reads index N, since |i - j| <= N-1). */
static inline double odd_sign(int m, int N) { return m == 0 || m == N ? 0.0 : (m < N ? 1.0 : -1.0); }

/* F_2 on the (2N)^3 doubled grid from the octant of a kernel odd in axis a. */
static void field_doubled(int N, int a, const double *F, cplx *g2) {
    int n2 = 2 * N, k1 = N + 1;
    for (int z = 0; z < n2; ++z)
        for (int y = 0; y < n2; ++y)
            for (int x = 0; x < n2; ++x) {
                int m[3] = {x, y, z};
                g2[((size_t)z * n2 + y) * n2 + x] =
                    odd_sign(m[a], N) * F[((size_t)fold2(z, N) * k1 + fold2(y, N)) * k1 + fold2(x, N)];
            }
}

/*
 * E_a = h^3 sum_j F_a[i-j] rho_j through Sec. 2.2 steps 1-5 on the full
 * (2N)^3 complex grid with the odd field kernel in place of G: pad rho, FFT
 * rho_2 and F_2, multiply, inverse FFT (1/(2N)^3), scale by h^3, restrict.
 */
void orc_solve_field_fft(int N, double h, int a, const double *F, const double *rho, double *E) {
    int n2 = 2 * N;
    size_t tot = (size_t)n2 * n2 * n2;
    cplx *r2 = (cplx *)calloc(tot, sizeof(cplx));
    cplx *g2 = (cplx *)malloc(sizeof(cplx) * tot);
    for (int z = 0; z < N; ++z)
        for (int y = 0; y < N; ++y)
            for (int x = 0; x < N; ++x) r2[((size_t)z * n2 + y) * n2 + x] = rho[((size_t)z * N + y) * N + x];
    field_doubled(N, a, F, g2);
    orc_fft3d(n2, n2, n2, r2, -1);
    orc_fft3d(n2, n2, n2, g2, -1);
    for (size_t i = 0; i < tot; ++i) r2[i] *= g2[i];
    orc_fft3d(n2, n2, n2, r2, +1);
    double scale = h * h * h / (double)tot;
    for (int z = 0; z < N; ++z)
        for (int y = 0; y < N; ++y)
            for (int x = 0; x < N; ++x)
                E[((size_t)z * N + y) * N + x] = creal(r2[((size_t)z * n2 + y) * n2 + x]) * scale;
    free(g2);
    free(r2);
}

/*
 * The field multiplier on the non-redundant octant.  DFT_{2N}{F_2} is purely
 * imaginary (F_2 real, odd in a, even in the others); the value returned is
 *   S_a[q] = -h^3 / (2N)^3 * Im DFT_{2N}{F_2}[q],  q in [0,N]^3,
 * so that the solve multiplies by -i S_a[q] for q_a <= N (and by +i S_a at
 * the mirrored index for q_a > N).  Computed through the full complex FFT.
 */
void orc_field_spectrum(int N, double h, int a, const double *F, double *S) {
    int n2 = 2 * N, k1 = N + 1;
    size_t tot = (size_t)n2 * n2 * n2;
    cplx *g2 = (cplx *)malloc(sizeof(cplx) * tot);
    field_doubled(N, a, F, g2);
    orc_fft3d(n2, n2, n2, g2, -1);
    double scale = h * h * h / (double)tot;
    for (int z = 0; z < k1; ++z)
        for (int y = 0; y < k1; ++y)
            for (int x = 0; x < k1; ++x)
                S[((size_t)z * k1 + y) * k1 + x] = -cimag(g2[((size_t)z * n2 + y) * n2 + x]) * scale;
    free(g2);
}

/*
 * The field's discrete convolution by its definition:
 *   E_a[i] = h^3 sum_{j in [0,N)^3} sgn(i_a - j_a) F_a[|i - j|] rho_j
 * at the `npts` flat output indices `pts` (all N^3 if pts == NULL), with
 * Neumaier's compensated summation as in orc_solve_direct.
 */
void orc_solve_field_direct(int N, double h, int a, const double *F, const double *rho, const long long *pts,
                            long long npts, double *out) {
    int k1 = N + 1;
    long long total = pts ? npts : (long long)N * N * N;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long p = 0; p < total; ++p) {
        long long i = pts ? pts[p] : p;
        int ix = (int)(i % N), iy = (int)((i / N) % N), iz = (int)(i / ((long long)N * N));
        int ii[3] = {ix, iy, iz};
        double sum = 0.0, comp = 0.0;
        for (int jz = 0; jz < N; ++jz)
            for (int jy = 0; jy < N; ++jy) {
                const double *Frow = F + ((size_t)abs(iz - jz) * k1 + abs(iy - jy)) * k1;
                const double *rrow = rho + ((size_t)jz * N + jy) * N;
                for (int jx = 0; jx < N; ++jx) {
                    int jj[3] = {jx, jy, jz};
                    int d = ii[a] - jj[a];
                    double sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
                    double t = sg * Frow[abs(ix - jx)] * rrow[jx];
                    double s = sum + t;
                    if (fabs(sum) >= fabs(t))
                        comp += (sum - s) + t;
                    else
                        comp += (t - s) + sum;
                    sum = s;
                }
            }
        out[p] = h * h * h * (sum + comp);
    }
}

/* ------------------------------------------------- non-cubic boxes -- */
/*
 * The methods on a box of n[0] x n[1] x n[2] cells (x, y, z) with spacings
 * h[0], h[1], h[2]: the same definitions per axis, with N and h of that axis.
 * Arrays are (n_z, n_y, n_x) with x fastest; kernels and spectra are
 * (n_z+1, n_y+1, n_x+1).
 *   HE:     T[m] = 1/(4 pi |(m_x h_x, m_y h_y, m_z h_z)|), T[0] = 1/(4 pi).
 *   VG:     G_L sampled on the (4n_x, 4n_y, 4n_z) frequency grid,
 *           k_a = 2 pi j_a / (4 n_a h_a), j_a in [-2n_a, 2n_a), inverse DFT,
 *           scaled by 1 / prod_a (4 n_a h_a), restricted to [0,n_a] per axis.
 *           The window is L_t = alpha |(L_x, L_y, L_z)| (alpha sqrt(3) L for a
 *           cube), L_a = n_a h_a.
 *   VG-DCT: the same through the (2n_a+1) octant and a DCT-I per axis.
 */
void orc_kernel_T3(int algo, const int *n, const double *h, double alpha, double *T) {
    int k[3] = {n[0] + 1, n[1] + 1, n[2] + 1};
    double Lb[3] = {n[0] * h[0], n[1] * h[1], n[2] * h[2]};
    double Lt = alpha * sqrt(Lb[0] * Lb[0] + Lb[1] * Lb[1] + Lb[2] * Lb[2]);
    if (algo == ORC_HE) {
        for (int z = 0; z < k[2]; ++z)
            for (int y = 0; y < k[1]; ++y)
                for (int x = 0; x < k[0]; ++x) {
                    double dx = x * h[0], dy = y * h[1], dz = z * h[2];
                    T[((size_t)z * k[1] + y) * k[0] + x] =
                        (x | y | z) ? green_free(sqrt(dx * dx + dy * dy + dz * dz)) : 1.0 / (4.0 * ORC_PI);
                }
    } else if (algo == ORC_VG) {
        int m[3] = {4 * n[0], 4 * n[1], 4 * n[2]};
        size_t tot = (size_t)m[0] * m[1] * m[2];
        cplx *g = (cplx *)malloc(sizeof(cplx) * tot);
        double dk[3];
        for (int a = 0; a < 3; ++a) dk[a] = 2.0 * ORC_PI / ((double)m[a] * h[a]);
#pragma omp parallel for schedule(static)
        for (long long idx = 0; idx < (long long)tot; ++idx) {
            int s3[3] = {(int)(idx % m[0]), (int)((idx / m[0]) % m[1]), (int)(idx / ((long long)m[0] * m[1]))};
            double k2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                int j = s3[a] < 2 * n[a] ? s3[a] : s3[a] - m[a];
                k2 += (dk[a] * j) * (dk[a] * j);
            }
            g[idx] = orc_green_vico_hat(sqrt(k2), Lt);
        }
        orc_fft3d(m[0], m[1], m[2], g, +1);
        double scale = 1.0 / (((double)m[0] * h[0]) * ((double)m[1] * h[1]) * ((double)m[2] * h[2]));
        for (int z = 0; z < k[2]; ++z)
            for (int y = 0; y < k[1]; ++y)
                for (int x = 0; x < k[0]; ++x)
                    T[((size_t)z * k[1] + y) * k[0] + x] = creal(g[((size_t)z * m[1] + y) * m[0] + x]) * scale;
        free(g);
    } else {
        int M[3] = {2 * n[0], 2 * n[1], 2 * n[2]}, q[3] = {M[0] + 1, M[1] + 1, M[2] + 1};
        double dk[3];
        for (int a = 0; a < 3; ++a) dk[a] = 2.0 * ORC_PI / (4.0 * n[a] * h[a]);
        double *g = (double *)malloc(sizeof(double) * (size_t)q[0] * q[1] * q[2]);
        for (int z = 0; z < q[2]; ++z)
            for (int y = 0; y < q[1]; ++y)
                for (int x = 0; x < q[0]; ++x) {
                    double kx = dk[0] * x, ky = dk[1] * y, kz = dk[2] * z;
                    g[((size_t)z * q[1] + y) * q[0] + x] = orc_green_vico_hat(sqrt(kx * kx + ky * ky + kz * kz), Lt);
                }
        /* DCT-I along x, y, z in turn, each keeping outputs [0, n_a] */
        double *t1 = (double *)malloc(sizeof(double) * (size_t)k[0] * q[1] * q[2]);
        double *t2 = (double *)malloc(sizeof(double) * (size_t)k[0] * k[1] * q[2]);
        axis_trig(M[0], n[0], 0, 0, q[0], q[1], q[2], g, t1);
        axis_trig(M[1], n[1], 0, 1, k[0], q[1], q[2], t1, t2);
        axis_trig(M[2], n[2], 0, 2, k[0], k[1], q[2], t2, T);
        double scale = 1.0 / ((4.0 * n[0] * h[0]) * (4.0 * n[1] * h[1]) * (4.0 * n[2] * h[2]));
        for (size_t i = 0; i < (size_t)k[0] * k[1] * k[2]; ++i) T[i] *= scale;
        free(t2);
        free(t1);
        free(g);
    }
}

/* G_2 on the (2n_x, 2n_y, 2n_z) doubled grid from the octant T. */
static void doubled3(const int *n, const double *T, cplx *g2) {
    int d[3] = {2 * n[0], 2 * n[1], 2 * n[2]}, k[3] = {n[0] + 1, n[1] + 1, n[2] + 1};
    for (int z = 0; z < d[2]; ++z)
        for (int y = 0; y < d[1]; ++y)
            for (int x = 0; x < d[0]; ++x)
                g2[((size_t)z * d[1] + y) * d[0] + x] =
                    T[((size_t)fold2(z, n[2]) * k[1] + fold2(y, n[1])) * k[0] + fold2(x, n[0])];
}

/* Sec. 2.2 steps 1-5 on the full (2n_x, 2n_y, 2n_z) complex grid. */
void orc_solve_fft3(const int *n, const double *h, const double *T, const double *rho, double *phi) {
    int d[3] = {2 * n[0], 2 * n[1], 2 * n[2]};
    size_t tot = (size_t)d[0] * d[1] * d[2];
    cplx *r2 = (cplx *)calloc(tot, sizeof(cplx));
    cplx *g2 = (cplx *)malloc(sizeof(cplx) * tot);
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x)
                r2[((size_t)z * d[1] + y) * d[0] + x] = rho[((size_t)z * n[1] + y) * n[0] + x];
    doubled3(n, T, g2);
    orc_fft3d(d[0], d[1], d[2], r2, -1);
    orc_fft3d(d[0], d[1], d[2], g2, -1);
    for (size_t i = 0; i < tot; ++i) r2[i] *= g2[i];
    orc_fft3d(d[0], d[1], d[2], r2, +1);
    double scale = h[0] * h[1] * h[2] / (double)tot;
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x)
                phi[((size_t)z * n[1] + y) * n[0] + x] = creal(r2[((size_t)z * d[1] + y) * d[0] + x]) * scale;
    free(g2);
    free(r2);
}

/* S[q] = h_x h_y h_z / (8 n_x n_y n_z) * DFT{G_2}[q], q in the octant (real part). */
void orc_spectrum3(const int *n, const double *h, const double *T, double *S) {
    int d[3] = {2 * n[0], 2 * n[1], 2 * n[2]}, k[3] = {n[0] + 1, n[1] + 1, n[2] + 1};
    size_t tot = (size_t)d[0] * d[1] * d[2];
    cplx *g2 = (cplx *)malloc(sizeof(cplx) * tot);
    doubled3(n, T, g2);
    orc_fft3d(d[0], d[1], d[2], g2, -1);
    double scale = h[0] * h[1] * h[2] / (double)tot;
    for (int z = 0; z < k[2]; ++z)
        for (int y = 0; y < k[1]; ++y)
            for (int x = 0; x < k[0]; ++x)
                S[((size_t)z * k[1] + y) * k[0] + x] = creal(g2[((size_t)z * d[1] + y) * d[0] + x]) * scale;
    free(g2);
}

/* phi_i = h_x h_y h_z sum_j T[|i - j|] rho_j by its definition (Neumaier). */
void orc_solve_direct3(const int *n, const double *h, const double *T, const double *rho, const long long *pts,
                       long long npts, double *out) {
    int k[3] = {n[0] + 1, n[1] + 1, n[2] + 1};
    long long total = pts ? npts : (long long)n[0] * n[1] * n[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (long long p = 0; p < total; ++p) {
        long long i = pts ? pts[p] : p;
        int ix = (int)(i % n[0]), iy = (int)((i / n[0]) % n[1]), iz = (int)(i / ((long long)n[0] * n[1]));
        double sum = 0.0, comp = 0.0;
        for (int jz = 0; jz < n[2]; ++jz)
            for (int jy = 0; jy < n[1]; ++jy) {
                const double *Trow = T + ((size_t)abs(iz - jz) * k[1] + abs(iy - jy)) * k[0];
                const double *rrow = rho + ((size_t)jz * n[1] + jy) * n[0];
                for (int jx = 0; jx < n[0]; ++jx) {
                    double t = Trow[abs(ix - jx)] * rrow[jx];
                    double s = sum + t;
                    if (fabs(sum) >= fabs(t))
                        comp += (sum - s) + t;
                    else
                        comp += (t - s) + sum;
                    sum = s;
                }
            }
        out[p] = h[0] * h[1] * h[2] * (sum + comp);
    }
}

/* ------------------------------------------- the field, non-cubic boxes -- */
/*
 * Field kernel F_a[m] = -dG/dx_a at (m_x h_x, m_y h_y, m_z h_z), m in the
 * (n_x+1, n_y+1, n_z+1) octant, for a box of n cells with spacings h (the
 * readings of orc_field_kernel, per axis):
 *   HE:     m_a h_a / (4 pi |r|^3), F_a[0] = 0.
 *   VG:     the inverse DFT of -i k_a G_L on the (4n_x, 4n_y, 4n_z) grid, the
 *           Nyquist plane j_a = -2n_a at zero, over prod_a (4 n_a h_a), real.
 *   VG-DCT: the octant samples k_a G_L, DST-I along a and DCT-I along the
 *           others, over prod_a (4 n_a h_a).
 * The window is alpha |(L_x, L_y, L_z)| as in orc_kernel_T3.
 */
void orc_field_kernel3(int algo, int a, const int *n, const double *h, double alpha, double *F) {
    int k[3] = {n[0] + 1, n[1] + 1, n[2] + 1};
    double Lb[3] = {n[0] * h[0], n[1] * h[1], n[2] * h[2]};
    double Lt = alpha * sqrt(Lb[0] * Lb[0] + Lb[1] * Lb[1] + Lb[2] * Lb[2]);
    if (algo == ORC_HE) {
        for (int z = 0; z < k[2]; ++z)
            for (int y = 0; y < k[1]; ++y)
                for (int x = 0; x < k[0]; ++x) {
                    double r[3] = {x * h[0], y * h[1], z * h[2]};
                    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    F[((size_t)z * k[1] + y) * k[0] + x] = (x | y | z) ? r[a] / (4.0 * ORC_PI * r2 * sqrt(r2)) : 0.0;
                }
    } else if (algo == ORC_VG) {
        int m[3] = {4 * n[0], 4 * n[1], 4 * n[2]};
        size_t tot = (size_t)m[0] * m[1] * m[2];
        cplx *g = (cplx *)malloc(sizeof(cplx) * tot);
        double dk[3];
        for (int c = 0; c < 3; ++c) dk[c] = 2.0 * ORC_PI / ((double)m[c] * h[c]);
#pragma omp parallel for schedule(static)
        for (long long idx = 0; idx < (long long)tot; ++idx) {
            int s3[3] = {(int)(idx % m[0]), (int)((idx / m[0]) % m[1]), (int)(idx / ((long long)m[0] * m[1]))};
            int j[3];
            double k2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                j[c] = s3[c] < 2 * n[c] ? s3[c] : s3[c] - m[c];
                k2 += (dk[c] * j[c]) * (dk[c] * j[c]);
            }
            double ka = j[a] == -2 * n[a] ? 0.0 : dk[a] * j[a];
            g[idx] = -I * ka * orc_green_vico_hat(sqrt(k2), Lt);
        }
        orc_fft3d(m[0], m[1], m[2], g, +1);
        double scale = 1.0 / (((double)m[0] * h[0]) * ((double)m[1] * h[1]) * ((double)m[2] * h[2]));
        for (int z = 0; z < k[2]; ++z)
            for (int y = 0; y < k[1]; ++y)
                for (int x = 0; x < k[0]; ++x)
                    F[((size_t)z * k[1] + y) * k[0] + x] = creal(g[((size_t)z * m[1] + y) * m[0] + x]) * scale;
        free(g);
    } else {
        int M[3] = {2 * n[0], 2 * n[1], 2 * n[2]}, q[3] = {M[0] + 1, M[1] + 1, M[2] + 1};
        double dk[3];
        for (int c = 0; c < 3; ++c) dk[c] = 2.0 * ORC_PI / (4.0 * n[c] * h[c]);
        double *g = (double *)malloc(sizeof(double) * (size_t)q[0] * q[1] * q[2]);
        for (int z = 0; z < q[2]; ++z)
            for (int y = 0; y < q[1]; ++y)
                for (int x = 0; x < q[0]; ++x) {
                    double kk[3] = {dk[0] * x, dk[1] * y, dk[2] * z};
                    g[((size_t)z * q[1] + y) * q[0] + x] =
                        kk[a] * orc_green_vico_hat(sqrt(kk[0] * kk[0] + kk[1] * kk[1] + kk[2] * kk[2]), Lt);
                }
        double *t1 = (double *)malloc(sizeof(double) * (size_t)k[0] * q[1] * q[2]);
        double *t2 = (double *)malloc(sizeof(double) * (size_t)k[0] * k[1] * q[2]);
        axis_trig(M[0], n[0], a == 0, 0, q[0], q[1], q[2], g, t1);
        axis_trig(M[1], n[1], a == 1, 1, k[0], q[1], q[2], t1, t2);
        axis_trig(M[2], n[2], a == 2, 2, k[0], k[1], q[2], t2, F);
        double scale = 1.0 / ((4.0 * n[0] * h[0]) * (4.0 * n[1] * h[1]) * (4.0 * n[2] * h[2]));
        for (size_t i = 0; i < (size_t)k[0] * k[1] * k[2]; ++i) F[i] *= scale;
        free(t2);
        free(t1);
        free(g);
    }
}

/* F_2 on the (2n_x, 2n_y, 2n_z) doubled grid, odd in axis a (odd_sign). */
static void field_doubled3(const int *n, int a, const double *F, cplx *g2) {
    int d[3] = {2 * n[0], 2 * n[1], 2 * n[2]}, k[3] = {n[0] + 1, n[1] + 1, n[2] + 1};
    for (int z = 0; z < d[2]; ++z)
        for (int y = 0; y < d[1]; ++y)
            for (int x = 0; x < d[0]; ++x) {
                int m[3] = {x, y, z};
                g2[((size_t)z * d[1] + y) * d[0] + x] =
                    odd_sign(m[a], n[a]) * F[((size_t)fold2(z, n[2]) * k[1] + fold2(y, n[1])) * k[0] + fold2(x, n[0])];
            }
}

/* E_a = h_x h_y h_z sum_j F_a[i - j] rho_j through the full doubled grid. */
void orc_solve_field_fft3(const int *n, const double *h, int a, const double *F, const double *rho, double *E) {
    int d[3] = {2 * n[0], 2 * n[1], 2 * n[2]};
    size_t tot = (size_t)d[0] * d[1] * d[2];
    cplx *r2 = (cplx *)calloc(tot, sizeof(cplx));
    cplx *g2 = (cplx *)malloc(sizeof(cplx) * tot);
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x)
                r2[((size_t)z * d[1] + y) * d[0] + x] = rho[((size_t)z * n[1] + y) * n[0] + x];
    field_doubled3(n, a, F, g2);
    orc_fft3d(d[0], d[1], d[2], r2, -1);
    orc_fft3d(d[0], d[1], d[2], g2, -1);
    for (size_t i = 0; i < tot; ++i) r2[i] *= g2[i];
    orc_fft3d(d[0], d[1], d[2], r2, +1);
    double scale = h[0] * h[1] * h[2] / (double)tot;
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x)
                E[((size_t)z * n[1] + y) * n[0] + x] = creal(r2[((size_t)z * d[1] + y) * d[0] + x]) * scale;
    free(g2);
    free(r2);
}

/* E_a[i] = h_x h_y h_z sum_j sgn(i_a - j_a) F_a[|i - j|] rho_j (Neumaier). */
void orc_solve_field_direct3(const int *n, const double *h, int a, const double *F, const double *rho,
                             const long long *pts, long long npts, double *out) {
    int k[3] = {n[0] + 1, n[1] + 1, n[2] + 1};
    long long total = pts ? npts : (long long)n[0] * n[1] * n[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (long long p = 0; p < total; ++p) {
        long long i = pts ? pts[p] : p;
        int ii[3] = {(int)(i % n[0]), (int)((i / n[0]) % n[1]), (int)(i / ((long long)n[0] * n[1]))};
        double sum = 0.0, comp = 0.0;
        for (int jz = 0; jz < n[2]; ++jz)
            for (int jy = 0; jy < n[1]; ++jy) {
                const double *Frow = F + ((size_t)abs(ii[2] - jz) * k[1] + abs(ii[1] - jy)) * k[0];
                const double *rrow = rho + ((size_t)jz * n[1] + jy) * n[0];
                for (int jx = 0; jx < n[0]; ++jx) {
                    int jj[3] = {jx, jy, jz};
                    int dd = ii[a] - jj[a];
                    double sg = dd > 0 ? 1.0 : (dd < 0 ? -1.0 : 0.0);
                    double t = sg * Frow[abs(ii[0] - jx)] * rrow[jx];
                    double s = sum + t;
                    if (fabs(sum) >= fabs(t))
                        comp += (sum - s) + t;
                    else
                        comp += (t - s) + sum;
                    sum = s;
                }
            }
        out[p] = h[0] * h[1] * h[2] * (sum + comp);
    }
}
