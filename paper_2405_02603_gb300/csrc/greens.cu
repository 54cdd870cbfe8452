// greens.cu -- plan-time sampling kernels of the Green's functions (always
// FP64): the Hockney-Eastwood kernel (Sec. 2.2 step 3), the Vico-Greengard
// truncated spectral kernel sampled on the (4N)^3 frequency grid (Sec. 2.3,
// Eq. green_vico) and on its (2N+1)^3 non-negative octant (Sec. 2.4), the
// same two for the field kernel F = -grad G (Appendix B, Eq. efield), plus
// scaling and the rounding of the spectrum to the solve's type.
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "greens.h"

namespace fsp {

// 1/(4 pi)
__device__ __forceinline__ double inv4pi() { return 0.079577471545947667884441881686257; }

// Eq. green_vico: G_L(k) = 2 (sin(L_t |k| / 2) / |k|)^2, evaluated as
// 2 (L_t/2)^2 sinc^2(u), u = L_t |k| / 2; for |u| < 1e-3 the sinc uses its
// Taylor series 1 - u^2/6 + u^4/120 (truncation below u^6/5040), so the k -> 0
// limit L_t^2 / 2 is reached without cancellation.
__device__ __forceinline__ double green_vico_hat(double kabs, double Lt) {
    const double u = 0.5 * Lt * kabs;
    double s;
    if (fabs(u) < 1e-3) {
        const double u2 = u * u;
        s = 1.0 - u2 / 6.0 + u2 * u2 / 120.0;
    } else {
        s = sin(u) / u;
    }
    const double hl = 0.5 * Lt;
    return 2.0 * hl * hl * s * s;
}

// T[m] = 1/(4 pi h |m|), T[0] = 1/(4 pi); m in [0,N]^3, x fastest.
__global__ void k_he_T(double *T, int N, double h) {
    const int k1 = N + 1;
    const long long tot = (long long)k1 * k1 * k1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % k1), y = (int)((i / k1) % k1), z = (int)(i / ((long long)k1 * k1));
        const double r = sqrt((double)x * x + (double)y * y + (double)z * z);
        T[i] = (x | y | z) ? inv4pi() / (h * r) : inv4pi();
    }
}

// g[j] = G_L(dk |j|) for j in [0,M]^3 (M = 2N), dk = 2 pi / (4 N h).
__global__ void k_vg_sample_octant(double *g, int M, double dk, double Lt) {
    const int n = M + 1;
    const long long tot = (long long)n * n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((long long)n * n));
        g[i] = green_vico_hat(dk * sqrt((double)x * x + (double)y * y + (double)z * z), Lt);
    }
}

// g[s] = G_L(dk |j|) on the (4N)^3 grid, storage index s holding frequency
// j = s for s < 2N and j = s - 4N otherwise (the Nyquist plane j = -2N
// included).  Complex, imaginary part zero.
__global__ void k_vg_sample_full(double2 *g, int n4, double dk, double Lt) {
    const long long tot = (long long)n4 * n4 * n4;
    const int half = n4 / 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % n4), y = (int)((i / n4) % n4), z = (int)(i / ((long long)n4 * n4));
        x = x < half ? x : x - n4;
        y = y < half ? y : y - n4;
        z = z < half ? z : z - n4;
        g[i] = double2{green_vico_hat(dk * sqrt((double)x * x + (double)y * y + (double)z * z), Lt), 0.0};
    }
}

// Field kernel of Hockney-Eastwood: F_a[m] = m_a / (4 pi h^2 |m|^3), F_a[0] = 0,
// m in [0,N]^3, x fastest (a = 0, 1, 2 for x, y, z).
__global__ void k_he_F(double *F, int N, double h, int a) {
    const int k1 = N + 1;
    const long long tot = (long long)k1 * k1 * k1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % k1), y = (int)((i / k1) % k1), z = (int)(i / ((long long)k1 * k1));
        const int ma = a == 0 ? x : (a == 1 ? y : z);
        const double r2 = (double)x * x + (double)y * y + (double)z * z;
        F[i] = (x | y | z) ? inv4pi() * (double)ma / (h * h * r2 * sqrt(r2)) : 0.0;
    }
}

// g[j] = dk j_a G_L(dk |j|) for j in [0,M]^3 (M = 2N): the octant of k_a G_L,
// odd in j_a, whose DST-I (axis a) / DCT-I (others) gives the field kernel.
__global__ void k_vg_sample_octant_grad(double *g, int M, double dk, double Lt, int a) {
    const int n = M + 1;
    const long long tot = (long long)n * n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((long long)n * n));
        const int ja = a == 0 ? x : (a == 1 ? y : z);
        g[i] = dk * (double)ja * green_vico_hat(dk * sqrt((double)x * x + (double)y * y + (double)z * z), Lt);
    }
}

// Non-cubic boxes (n_x x n_y x n_z cells, spacings h_x, h_y, h_z).
// T[m] = 1/(4 pi |(m_x h_x, m_y h_y, m_z h_z)|), T[0] = 1/(4 pi); m in the
// (n_x+1, n_y+1, n_z+1) octant, x fastest.
__global__ void k_he_T3(double *T, int kx, int ky, int kz, double hx, double hy, double hz) {
    const long long tot = (long long)kx * ky * kz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % kx), y = (int)((i / kx) % ky), z = (int)(i / ((long long)kx * ky));
        const double dx = x * hx, dy = y * hy, dz = z * hz;
        T[i] = (x | y | z) ? inv4pi() / sqrt(dx * dx + dy * dy + dz * dz) : inv4pi();
    }
}

// g[j] = G_L(|(dk_x j_x, dk_y j_y, dk_z j_z)|) for j in the (q_x, q_y, q_z)
// octant, q_a = 2 n_a + 1.
__global__ void k_vg_sample_octant3(double *g, int qx, int qy, int qz, double dkx, double dky, double dkz, double Lt) {
    const long long tot = (long long)qx * qy * qz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % qx), y = (int)((i / qx) % qy), z = (int)(i / ((long long)qx * qy));
        const double kx = dkx * x, ky = dky * y, kz = dkz * z;
        g[i] = green_vico_hat(sqrt(kx * kx + ky * ky + kz * kz), Lt);
    }
}

// g[s] = G_L(|k|) on the (4n_x, 4n_y, 4n_z) grid, storage index s holding
// frequency j_a = s_a for s_a < 2 n_a and s_a - 4 n_a otherwise.
__global__ void k_vg_sample_full3(double2 *g, int mx, int my, int mz, double dkx, double dky, double dkz, double Lt) {
    const long long tot = (long long)mx * my * mz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % mx), y = (int)((i / mx) % my), z = (int)(i / ((long long)mx * my));
        x = x < mx / 2 ? x : x - mx;
        y = y < my / 2 ? y : y - my;
        z = z < mz / 2 ? z : z - mz;
        const double kx = dkx * x, ky = dky * y, kz = dkz * z;
        g[i] = double2{green_vico_hat(sqrt(kx * kx + ky * ky + kz * kz), Lt), 0.0};
    }
}

// Field kernels on a non-cubic box: F_a[m] = m_a h_a / (4 pi |r|^3), r =
// (m_x h_x, m_y h_y, m_z h_z), F_a[0] = 0; and the octant of k_a G_L(|k|),
// k = (dk_x j_x, dk_y j_y, dk_z j_z).
__global__ void k_he_F3(double *F, int kx, int ky, int kz, double hx, double hy, double hz, int a) {
    const long long tot = (long long)kx * ky * kz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % kx), y = (int)((i / kx) % ky), z = (int)(i / ((long long)kx * ky));
        const double rx = x * hx, ry = y * hy, rz = z * hz;
        const double ra = a == 0 ? rx : (a == 1 ? ry : rz);
        const double r2 = rx * rx + ry * ry + rz * rz;
        F[i] = (x | y | z) ? inv4pi() * ra / (r2 * sqrt(r2)) : 0.0;
    }
}

__global__ void k_vg_sample_octant_grad3(double *g, int qx, int qy, int qz, double dkx, double dky, double dkz, double Lt,
                                         int a) {
    const long long tot = (long long)qx * qy * qz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % qx), y = (int)((i / qx) % qy), z = (int)(i / ((long long)qx * qy));
        const double kx = dkx * x, ky = dky * y, kz = dkz * z;
        const double ka = a == 0 ? kx : (a == 1 ? ky : kz);
        g[i] = ka * green_vico_hat(sqrt(kx * kx + ky * ky + kz * kz), Lt);
    }
}

__global__ void k_scale(double *a, long long n, double s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] *= s;
}

// S[qz][qy][qx] (row pitch P) = scale * Sd[qz][qy][qx] rounded to T; rows of
// kx values, `rows` = (n_z+1)(n_y+1) of them.
template <typename T> __global__ void k_store_S(const double *Sd, T *S, int kx, long long rows, int P, double scale) {
    const long long tot = (long long)kx * rows;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % kx);
        const long long row = i / kx;  // qz*(n_y+1) + qy
        S[row * P + x] = (T)(scale * Sd[i]);
    }
}

// S (pitch P, type T) -> dense rows of kx doubles
template <typename T> __global__ void k_load_S(const T *S, double *Sd, int kx, long long rows, int P) {
    const long long tot = (long long)kx * rows;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % kx);
        Sd[i] = (double)S[(i / kx) * P + x];
    }
}

static unsigned grid_for(long long tot) {
    long long b = (tot + 255) / 256;
    if (b > 152LL * 64) b = 152LL * 64;
    if (b < 1) b = 1;
    return (unsigned)b;
}

cudaError_t launch_he_T(double *T, int N, double h, cudaStream_t s) {
    const long long tot = (long long)(N + 1) * (N + 1) * (N + 1);
    k_he_T<<<grid_for(tot), 256, 0, s>>>(T, N, h);
    return cudaGetLastError();
}

cudaError_t launch_vg_sample_octant(double *g, int N, double h, double Lt, cudaStream_t s) {
    const int M = 2 * N;
    const long long tot = (long long)(M + 1) * (M + 1) * (M + 1);
    const double dk = 6.283185307179586476925286766559 / (4.0 * N * h);
    k_vg_sample_octant<<<grid_for(tot), 256, 0, s>>>(g, M, dk, Lt);
    return cudaGetLastError();
}

cudaError_t launch_vg_sample_full(void *g, int N, double h, double Lt, cudaStream_t s) {
    const int n4 = 4 * N;
    const long long tot = (long long)n4 * n4 * n4;
    const double dk = 6.283185307179586476925286766559 / (4.0 * N * h);
    k_vg_sample_full<<<grid_for(tot), 256, 0, s>>>(reinterpret_cast<double2 *>(g), n4, dk, Lt);
    return cudaGetLastError();
}

cudaError_t launch_he_F(double *F, int N, double h, int a, cudaStream_t s) {
    const long long tot = (long long)(N + 1) * (N + 1) * (N + 1);
    k_he_F<<<grid_for(tot), 256, 0, s>>>(F, N, h, a);
    return cudaGetLastError();
}

cudaError_t launch_vg_sample_octant_grad(double *g, int N, double h, double Lt, int a, cudaStream_t s) {
    const int M = 2 * N;
    const long long tot = (long long)(M + 1) * (M + 1) * (M + 1);
    const double dk = 6.283185307179586476925286766559 / (4.0 * N * h);
    k_vg_sample_octant_grad<<<grid_for(tot), 256, 0, s>>>(g, M, dk, Lt, a);
    return cudaGetLastError();
}

cudaError_t launch_scale(double *a, long long n, double sc, cudaStream_t s) {
    k_scale<<<grid_for(n), 256, 0, s>>>(a, n, sc);
    return cudaGetLastError();
}

cudaError_t launch_he_F3(double *F, const int *n, const double *h, int a, cudaStream_t s) {
    const long long tot = (long long)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
    k_he_F3<<<grid_for(tot), 256, 0, s>>>(F, n[0] + 1, n[1] + 1, n[2] + 1, h[0], h[1], h[2], a);
    return cudaGetLastError();
}

cudaError_t launch_vg_sample_octant_grad3(double *g, const int *n, const double *h, double Lt, int a, cudaStream_t s) {
    const int q[3] = {2 * n[0] + 1, 2 * n[1] + 1, 2 * n[2] + 1};
    double dk[3];
    for (int c = 0; c < 3; ++c) dk[c] = 6.283185307179586476925286766559 / (4.0 * n[c] * h[c]);
    k_vg_sample_octant_grad3<<<grid_for((long long)q[0] * q[1] * q[2]), 256, 0, s>>>(g, q[0], q[1], q[2], dk[0], dk[1],
                                                                                     dk[2], Lt, a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_store_S3(const double *Sd, void *S, int kx, long long rows, int P, double scale, cudaStream_t s) {
    k_store_S<T><<<grid_for((long long)kx * rows), 256, 0, s>>>(Sd, reinterpret_cast<T *>(S), kx, rows, P, scale);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_load_S3(const void *S, double *Sd, int kx, long long rows, int P, cudaStream_t s) {
    k_load_S<T><<<grid_for((long long)kx * rows), 256, 0, s>>>(reinterpret_cast<const T *>(S), Sd, kx, rows, P);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_store_S(const double *Sd, void *S, int N, int P, double scale, cudaStream_t s) {
    return launch_store_S3<T>(Sd, S, N + 1, (long long)(N + 1) * (N + 1), P, scale, s);
}

template <typename T> cudaError_t launch_load_S(const void *S, double *Sd, int N, int P, cudaStream_t s) {
    return launch_load_S3<T>(S, Sd, N + 1, (long long)(N + 1) * (N + 1), P, s);
}

cudaError_t launch_he_T3(double *T, const int *n, const double *h, cudaStream_t s) {
    const long long tot = (long long)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
    k_he_T3<<<grid_for(tot), 256, 0, s>>>(T, n[0] + 1, n[1] + 1, n[2] + 1, h[0], h[1], h[2]);
    return cudaGetLastError();
}

cudaError_t launch_vg_sample_octant3(double *g, const int *n, const double *h, double Lt, cudaStream_t s) {
    const int q[3] = {2 * n[0] + 1, 2 * n[1] + 1, 2 * n[2] + 1};
    double dk[3];
    for (int a = 0; a < 3; ++a) dk[a] = 6.283185307179586476925286766559 / (4.0 * n[a] * h[a]);
    k_vg_sample_octant3<<<grid_for((long long)q[0] * q[1] * q[2]), 256, 0, s>>>(g, q[0], q[1], q[2], dk[0], dk[1], dk[2], Lt);
    return cudaGetLastError();
}

cudaError_t launch_vg_sample_full3(void *g, const int *n, const double *h, double Lt, cudaStream_t s) {
    const int m[3] = {4 * n[0], 4 * n[1], 4 * n[2]};
    double dk[3];
    for (int a = 0; a < 3; ++a) dk[a] = 6.283185307179586476925286766559 / (4.0 * n[a] * h[a]);
    k_vg_sample_full3<<<grid_for((long long)m[0] * m[1] * m[2]), 256, 0, s>>>(reinterpret_cast<double2 *>(g), m[0], m[1],
                                                                                m[2], dk[0], dk[1], dk[2], Lt);
    return cudaGetLastError();
}

template cudaError_t launch_store_S<float>(const double *, void *, int, int, double, cudaStream_t);
template cudaError_t launch_store_S<df>(const double *, void *, int, int, double, cudaStream_t);
template cudaError_t launch_load_S<df>(const void *, double *, int, int, cudaStream_t);
template cudaError_t launch_store_S<double>(const double *, void *, int, int, double, cudaStream_t);
template cudaError_t launch_load_S<float>(const void *, double *, int, int, cudaStream_t);
template cudaError_t launch_load_S<double>(const void *, double *, int, int, cudaStream_t);
template cudaError_t launch_store_S3<float>(const double *, void *, int, long long, int, double, cudaStream_t);
template cudaError_t launch_store_S3<double>(const double *, void *, int, long long, int, double, cudaStream_t);
template cudaError_t launch_load_S3<float>(const void *, double *, int, long long, int, cudaStream_t);
template cudaError_t launch_load_S3<double>(const void *, double *, int, long long, int, cudaStream_t);
template cudaError_t launch_store_S3<df>(const double *, void *, int, long long, int, double, cudaStream_t);
template cudaError_t launch_load_S3<df>(const void *, double *, int, long long, int, cudaStream_t);

}  // namespace fsp
