// greens.h -- host launchers of the plan-time Green's-function kernels.
#pragma once
#include <cuda_runtime.h>

namespace fsp {
cudaError_t launch_he_T(double *T, int N, double h, cudaStream_t s);
cudaError_t launch_vg_sample_octant(double *g, int N, double h, double Lt, cudaStream_t s);
cudaError_t launch_vg_sample_full(void *g, int N, double h, double Lt, cudaStream_t s);
cudaError_t launch_he_F(double *F, int N, double h, int a, cudaStream_t s);
cudaError_t launch_vg_sample_octant_grad(double *g, int N, double h, double Lt, int a, cudaStream_t s);
cudaError_t launch_scale(double *a, long long n, double sc, cudaStream_t s);
template <typename T> cudaError_t launch_store_S(const double *Sd, void *S, int N, int P, double scale, cudaStream_t s);
template <typename T> cudaError_t launch_load_S(const void *S, double *Sd, int N, int P, cudaStream_t s);
// non-cubic boxes: n = (n_x, n_y, n_z), h = (h_x, h_y, h_z); spectra as rows
// of kx = n_x + 1 values, rows = (n_z + 1)(n_y + 1)
cudaError_t launch_he_T3(double *T, const int *n, const double *h, cudaStream_t s);
cudaError_t launch_vg_sample_octant3(double *g, const int *n, const double *h, double Lt, cudaStream_t s);
cudaError_t launch_vg_sample_full3(void *g, const int *n, const double *h, double Lt, cudaStream_t s);
cudaError_t launch_he_F3(double *F, const int *n, const double *h, int a, cudaStream_t s);
cudaError_t launch_vg_sample_octant_grad3(double *g, const int *n, const double *h, double Lt, int a, cudaStream_t s);
template <typename T>
cudaError_t launch_store_S3(const double *Sd, void *S, int kx, long long rows, int P, double scale, cudaStream_t s);
template <typename T> cudaError_t launch_load_S3(const void *S, double *Sd, int kx, long long rows, int P, cudaStream_t s);
}  // namespace fsp
