// api.cu -- the C ABI of include/fsp.h: plan registry, argument validation,
// the plan-time Green's spectrum pipeline and the five-pass solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <tuple>
#include <type_traits>
#include <unordered_set>
#include <vector>

#include "../../include/fsp.h"
#include "batch.h"
#include "fast_field.h"
#include "df.cuh"
#include "fast.h"
#include "greens.h"
#include "kernels.cuh"
#include "tiles.h"
#include "internal.h"

using namespace fsp;

namespace {

constexpr uint64_t kMagic = 0x46535050'4c414e31ULL;  // "FSPPLAN1"
constexpr int kMaxN = 1024;
// device staging slots of the host-buffer pipeline (fsp_solve_host_many):
// with three, a step's copies have the time of two solves to finish
constexpr int kPipeSlots = 3;
constexpr double kAlpha = 1.1;  // Vico-Greengard window factor (Sec. 2.3)

std::mutex g_mu;
std::unordered_set<const fsp_plan *> g_plans;

// Tile shapes (log2 lines per CTA) of the generic engine chosen by the
// autotuner or loaded from a table, per (N, dtype): {rows, columns}.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, std::pair<int, int>> g_tuning;

bool tuned_lgL(int N, int dtype, int &row, int &col) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuning.find({N, dtype});
    if (it == g_tuning.end()) return false;
    row = it->second.first, col = it->second.second;
    return true;
}

fsp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FSP_OK : FSP_ECUDA; }

#define FSP_TRY_CUDA(expr)                              \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return FSP_ECUDA;        \
    } while (0)

// Device memory owned by one scope: freed on every exit path.
// Bounds checking without a sanitizer (opt-in, FSP_CHECK_BOUNDS=1 in the
// environment at plan creation): every device buffer the plan allocates --
// spectrum, workspaces, tables, plan-time temporaries -- gets kGuard bytes of
// the pattern kGuardByte on each side.  A kernel that stores outside its
// buffer by less than that changes the pattern; fsp_plan_check_bounds counts
// changed bytes around the plan's live buffers, and freeing a guarded buffer
// (a temporary, or a destroyed plan's) adds its changed bytes to a process-
// wide count.  Nothing traps: the counts are read on the host.
constexpr size_t kGuard = 1 << 20;
constexpr unsigned char kGuardByte = 0xA5;
thread_local size_t t_guard = 0;  // guard of allocations made by this thread now
std::mutex g_guard_mu;
struct Guarded {
    void *base;
    size_t bytes;
};
std::map<const void *, Guarded> g_guarded;
std::atomic<unsigned long long> g_guard_freed_bad{0};

// max |x| over n doubles (the bit patterns of non-negative doubles order as
// unsigned integers)
__global__ void k_abs_max(const double *x, long long n, unsigned long long *out) {
    unsigned long long m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(fabs(x[i])));
    atomicMax(out, m);
}

fsp_status abs_max(const double *x, long long n, cudaStream_t s, double *out) {
    unsigned long long *d = nullptr, h = 0;
    if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) {
        cudaGetLastError();
        return FSP_ENOMEM;
    }
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(*d), s);
    if (e == cudaSuccess) {
        k_abs_max<<<256, 256, 0, s>>>(x, n, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    std::memcpy(out, &h, sizeof(*out));
    return e == cudaSuccess ? FSP_OK : FSP_ECUDA;
}

// Double-float keeps FP32's exponent range: a spectrum whose largest value is
// outside [2^-80, 2^80] would lose the low words of its smaller entries to
// underflow (or overflow outright), so such plans are refused.
constexpr double kDfMinS = 0x1p-80, kDfMaxS = 0x1p80;

bool bounds_check_requested() {
    const char *e = std::getenv("FSP_CHECK_BOUNDS");
    return e && e[0] == '1';
}

__global__ void k_count_not(const unsigned char *a, size_t n, unsigned char v, unsigned long long *out) {
    unsigned long long c = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        c += a[i] != v;
    if (c) atomicAdd(out, c);
}

// changed guard bytes around the guarded buffer at p (synchronous)
unsigned long long guard_bad(const void *p, const Guarded &g) {
    unsigned long long *d = nullptr, h = 0;
    if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return ~0ull;
    cudaMemset(d, 0, sizeof(*d));
    const unsigned char *base = static_cast<const unsigned char *>(g.base);
    k_count_not<<<64, 256>>>(base, kGuard, kGuardByte, d);
    k_count_not<<<64, 256>>>(base + kGuard + g.bytes, kGuard, kGuardByte, d);
    cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    (void)p;
    return h;
}

void dev_free(void *p) {
    if (!p) return;
    Guarded g{nullptr, 0};
    {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        auto it = g_guarded.find(p);
        if (it != g_guarded.end()) {
            g = it->second;
            g_guarded.erase(it);
        }
    }
    if (!g.base) {
        cudaFree(p);
        return;
    }
    cudaDeviceSynchronize();
    g_guard_freed_bad += guard_bad(p, g);
    cudaFree(g.base);
}

cudaError_t dev_malloc(void **p, size_t bytes) {
    if (!t_guard) return cudaMalloc(p, bytes);
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, bytes + 2 * kGuard);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemset(base, kGuardByte, bytes + 2 * kGuard)) != cudaSuccess) {
        cudaFree(base);
        return e;
    }
    *p = static_cast<char *>(base) + kGuard;
    std::lock_guard<std::mutex> lk(g_guard_mu);
    g_guarded[*p] = Guarded{base, bytes};
    return cudaSuccess;
}

// Allocations made while this object lives get guard bands when `on`.
struct GuardScope {
    size_t prev;
    explicit GuardScope(bool on) : prev(t_guard) { t_guard = on ? kGuard : 0; }
    ~GuardScope() { t_guard = prev; }
};

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) dev_free(p);
    }
    cudaError_t alloc(size_t bytes) { return dev_malloc(&p, bytes); }
    void *release() {
        void *q = p;
        p = nullptr;
        return q;
    }
};

fsp_status alloc_or_nomem(DevBuf &b, size_t bytes) {
    cudaError_t e = b.alloc(bytes);
    if (e == cudaSuccess) return FSP_OK;
    cudaGetLastError();  // clear the sticky-free allocation error
    return e == cudaErrorMemoryAllocation ? FSP_ENOMEM : FSP_ECUDA;
}

// FP64 forward-roots table of length n in a scope-owned buffer.
fsp_status roots_f64(DevBuf &b, int n, cudaStream_t s) {
    fsp_status st = alloc_or_nomem(b, sizeof(double2) * (size_t)n);
    if (st != FSP_OK) return st;
    return cuda_status(launch_roots<double>(b.p, n, s));
}

// -------------------------------------------------------- plan-time kernels
// Real-space kernel T[m], m in [0,N]^3, into t_dev (FP64).  Asynchronous on s;
// temporaries are owned by `keep` and must outlive the enqueued work.
struct Temps {
    DevBuf g, a1, a2, tw, tw_y, tw_z;
};

// Roots tables of lengths len[0..2] (FP64): one per distinct length, so that
// a cube uses a single table; tab[a] points at axis a's.
fsp_status roots_3(Temps &tmp, const int *len, const void **tab, cudaStream_t s) {
    fsp_status st;
    if ((st = roots_f64(tmp.tw, len[0], s)) != FSP_OK) return st;
    tab[0] = tmp.tw.p;
    if (len[1] == len[0]) {
        tab[1] = tmp.tw.p;
    } else {
        if ((st = roots_f64(tmp.tw_y, len[1], s)) != FSP_OK) return st;
        tab[1] = tmp.tw_y.p;
    }
    if (len[2] == len[0]) {
        tab[2] = tmp.tw.p;
    } else if (len[2] == len[1]) {
        tab[2] = tab[1];
    } else {
        if ((st = roots_f64(tmp.tw_z, len[2], s)) != FSP_OK) return st;
        tab[2] = tmp.tw_z.p;
    }
    return FSP_OK;
}

// DCT-I (kind false) or DST-I (kind true) of real lines, FP64.
cudaError_t launch_trig(bool dst, const LinesArgs &a, cudaStream_t s) {
    return dst ? launch_lines<double, IN_REAL_ODD, OUT_REAL, M_FWD>(a, s)
               : launch_lines<double, IN_REAL_EVEN, OUT_REAL, M_FWD>(a, s);
}

// Separable transform of the octant g of (2n_x+1, 2n_y+1, 2n_z+1) samples
// (M_a = 2n_a per axis, extended to 4n_a): DST-I along axis `odd` (0 = x,
// 1 = y, 2 = z; -1: none) and DCT-I along the others, outputs [0,n_a] per
// axis into out ((n_z+1)(n_y+1)(n_x+1)), FP64.  This is the (4n)^3 DFT of a
// sequence even (or, along `odd`, odd) in every axis (Sec. 2.4).
// Temporaries in tmp.a1, tmp.a2 and the roots tables.
fsp_status enqueue_octant_transform3(const int *nn, int odd, const double *g, double *out, cudaStream_t s, Temps &tmp) {
    const int k[3] = {nn[0] + 1, nn[1] + 1, nn[2] + 1};
    const int q[3] = {2 * nn[0] + 1, 2 * nn[1] + 1, 2 * nn[2] + 1};
    const int len[3] = {4 * nn[0], 4 * nn[1], 4 * nn[2]};
    fsp_status st;
    TileCfg c[3];
    for (int a = 0; a < 3; ++a)
        if (!make_cfg(len[a], len[a], sizeof(double2), 3, c[a])) return FSP_EUNSUPPORTED;
    if ((st = alloc_or_nomem(tmp.a1, sizeof(double) * (size_t)q[2] * q[1] * k[0])) != FSP_OK) return st;
    if ((st = alloc_or_nomem(tmp.a2, sizeof(double) * (size_t)q[2] * k[1] * k[0])) != FSP_OK) return st;
    const void *tab[3];
    if ((st = roots_3(tmp, len, tab, s)) != FSP_OK) return st;
    LinesArgs a{};
    // x: rows of q_x reals -> rows of k_x
    a.tw = tab[0], a.st = c[0].st, a.tpl = c[0].tpl, a.lgL = c[0].lgL;
    a.in = g;
    a.out = tmp.a1.p;
    a.in_pos = 1, a.in_line = q[0], a.in_batch = 0;
    a.out_pos = 1, a.out_line = k[0], a.out_batch = 0;
    a.n_out = k[0], a.nlines = q[1] * q[2], a.nbatch = 1;
    FSP_TRY_CUDA(launch_trig(odd == 0, a, s));
    // y: columns (x in [0,n_x]) of a1[z][y][x]
    a.tw = tab[1], a.st = c[1].st, a.tpl = c[1].tpl, a.lgL = c[1].lgL;
    a.in = tmp.a1.p;
    a.out = tmp.a2.p;
    a.in_pos = k[0], a.in_line = 1, a.in_batch = (long long)q[1] * k[0];
    a.out_pos = k[0], a.out_line = 1, a.out_batch = (long long)k[1] * k[0];
    a.n_out = k[1], a.nlines = k[0], a.nbatch = q[2];
    FSP_TRY_CUDA(launch_trig(odd == 1, a, s));
    // z: columns of a2[z][y][x], batch y
    a.tw = tab[2], a.st = c[2].st, a.tpl = c[2].tpl, a.lgL = c[2].lgL;
    a.in = tmp.a2.p;
    a.out = out;
    a.in_pos = (long long)k[1] * k[0], a.in_line = 1, a.in_batch = k[0];
    a.out_pos = (long long)k[1] * k[0], a.out_line = 1, a.out_batch = k[0];
    a.n_out = k[2], a.nlines = k[0], a.nbatch = k[1];
    FSP_TRY_CUDA(launch_trig(odd == 2, a, s));
    return FSP_OK;
}

fsp_status enqueue_octant_transform(int N, int odd, const double *g, double *out, cudaStream_t s, Temps &tmp) {
    const int nn[3] = {N, N, N};
    return enqueue_octant_transform3(nn, odd, g, out, s, tmp);
}

// Vico-Greengard on the (4n_x, 4n_y, 4n_z) grid (Sec. 2.3): the sampled G_L in
// tmp.g (complex), unnormalised inverse DFT per axis keeping outputs [0,n_a]
// (three pruned passes), real part into t_dev, unscaled.
fsp_status enqueue_vg_inverse3(const int *nn, double *t_dev, cudaStream_t s, Temps &tmp) {
    const int k[3] = {nn[0] + 1, nn[1] + 1, nn[2] + 1};
    const int m[3] = {4 * nn[0], 4 * nn[1], 4 * nn[2]};
    fsp_status st;
    TileCfg c[3];
    for (int a = 0; a < 3; ++a)
        if (!make_cfg(m[a], m[a], sizeof(double2), 3, c[a])) return FSP_EUNSUPPORTED;
    if ((st = alloc_or_nomem(tmp.a1, sizeof(double2) * (size_t)m[2] * m[1] * k[0])) != FSP_OK) return st;
    if ((st = alloc_or_nomem(tmp.a2, sizeof(double2) * (size_t)m[2] * k[1] * k[0])) != FSP_OK) return st;
    const void *tab[3];
    if ((st = roots_3(tmp, m, tab, s)) != FSP_OK) return st;
    LinesArgs a{};
    a.tw = tab[0], a.st = c[0].st, a.tpl = c[0].tpl, a.lgL = c[0].lgL;
    a.in = tmp.g.p, a.out = tmp.a1.p;
    a.in_pos = 1, a.in_line = m[0], a.in_batch = 0;
    a.out_pos = 1, a.out_line = k[0], a.out_batch = 0;
    a.n_in = m[0], a.n_out = k[0], a.nlines = m[1] * m[2], a.nbatch = 1;
    FSP_TRY_CUDA((launch_lines<double, IN_CPLX, OUT_CPLX, M_INV>(a, s)));
    a.tw = tab[1], a.st = c[1].st, a.tpl = c[1].tpl, a.lgL = c[1].lgL;
    a.in = tmp.a1.p, a.out = tmp.a2.p;
    a.in_pos = k[0], a.in_line = 1, a.in_batch = (long long)m[1] * k[0];
    a.out_pos = k[0], a.out_line = 1, a.out_batch = (long long)k[1] * k[0];
    a.n_in = m[1], a.n_out = k[1], a.nlines = k[0], a.nbatch = m[2];
    FSP_TRY_CUDA((launch_lines<double, IN_CPLX, OUT_CPLX, M_INV>(a, s)));
    a.tw = tab[2], a.st = c[2].st, a.tpl = c[2].tpl, a.lgL = c[2].lgL;
    a.in = tmp.a2.p, a.out = t_dev;
    a.in_pos = (long long)k[1] * k[0], a.in_line = 1, a.in_batch = k[0];
    a.out_pos = (long long)k[1] * k[0], a.out_line = 1, a.out_batch = k[0];
    a.n_in = m[2], a.n_out = k[2], a.nlines = k[0], a.nbatch = k[1];
    FSP_TRY_CUDA((launch_lines<double, IN_CPLX, OUT_REAL, M_INV>(a, s)));
    return FSP_OK;
}

fsp_status enqueue_kernel_T(int N, double L, fsp_algo algo, double *t_dev, cudaStream_t s, Temps &tmp) {
    const double h = L / N;
    const int k1 = N + 1;
    const double Lt = kAlpha * std::sqrt(3.0) * L;
    fsp_status st;
    if (algo == FSP_HE) return cuda_status(launch_he_T(t_dev, N, h, s));

    const double scale = 1.0 / ((4.0 * N * h) * (4.0 * N * h) * (4.0 * N * h));
    if (algo == FSP_VG_DCT) {
        // Sec. 2.4: G_L on [0,2N]^3, DCT-I per axis (M = 2N, even extension to
        // 4N), keeping outputs [0,N] of each axis, then (4Nh)^-3.
        const int nm = 2 * N + 1;
        if ((st = alloc_or_nomem(tmp.g, sizeof(double) * (size_t)nm * nm * nm)) != FSP_OK) return st;
        FSP_TRY_CUDA(launch_vg_sample_octant((double *)tmp.g.p, N, h, Lt, s));
        if ((st = enqueue_octant_transform(N, -1, (double *)tmp.g.p, t_dev, s, tmp)) != FSP_OK) return st;
        return cuda_status(launch_scale(t_dev, (long long)k1 * k1 * k1, scale, s));
    }
    // FSP_VG, Sec. 2.3: G_L on the (4N)^3 grid, unnormalised inverse DFT per
    // axis, restricted to [0,N] per axis, real part, times (4Nh)^-3.
    const int n4 = 4 * N;
    if ((st = alloc_or_nomem(tmp.g, sizeof(double2) * (size_t)n4 * n4 * n4)) != FSP_OK) return st;
    FSP_TRY_CUDA(launch_vg_sample_full(tmp.g.p, N, h, Lt, s));
    const int nn[3] = {N, N, N};
    if ((st = enqueue_vg_inverse3(nn, t_dev, s, tmp)) != FSP_OK) return st;
    return cuda_status(launch_scale(t_dev, (long long)k1 * k1 * k1, scale, s));
}

// Real-space kernel T on a non-cubic box (n_x x n_y x n_z cells, spacings
// h_x, h_y, h_z), (n_z+1)(n_y+1)(n_x+1) FP64 values into t_dev: the methods
// of Sec. 2.2-2.4 per axis, the Vico-Greengard window alpha |(L_x, L_y, L_z)|.
fsp_status enqueue_kernel_T3(const int *nn, const double *hh, fsp_algo algo, double *t_dev, cudaStream_t s, Temps &tmp) {
    const long long tot = (long long)(nn[0] + 1) * (nn[1] + 1) * (nn[2] + 1);
    if (algo == FSP_HE) return cuda_status(launch_he_T3(t_dev, nn, hh, s));
    const double Lb[3] = {nn[0] * hh[0], nn[1] * hh[1], nn[2] * hh[2]};
    const double Lt = kAlpha * std::sqrt(Lb[0] * Lb[0] + Lb[1] * Lb[1] + Lb[2] * Lb[2]);
    const double scale = 1.0 / ((4.0 * nn[0] * hh[0]) * (4.0 * nn[1] * hh[1]) * (4.0 * nn[2] * hh[2]));
    fsp_status st;
    if (algo == FSP_VG_DCT) {
        const size_t q = (size_t)(2 * nn[0] + 1) * (2 * nn[1] + 1) * (2 * nn[2] + 1);
        if ((st = alloc_or_nomem(tmp.g, sizeof(double) * q)) != FSP_OK) return st;
        FSP_TRY_CUDA(launch_vg_sample_octant3((double *)tmp.g.p, nn, hh, Lt, s));
        if ((st = enqueue_octant_transform3(nn, -1, (double *)tmp.g.p, t_dev, s, tmp)) != FSP_OK) return st;
    } else {
        const size_t m = (size_t)(4 * nn[0]) * (4 * nn[1]) * (4 * nn[2]);
        if ((st = alloc_or_nomem(tmp.g, sizeof(double2) * m)) != FSP_OK) return st;
        FSP_TRY_CUDA(launch_vg_sample_full3(tmp.g.p, nn, hh, Lt, s));
        if ((st = enqueue_vg_inverse3(nn, t_dev, s, tmp)) != FSP_OK) return st;
    }
    return cuda_status(launch_scale(t_dev, tot, scale, s));
}

// Spectrum of the mirrored kernel: DCT-I of length n_a+1 per axis on T in
// place (the 2n_a DFT of a real sequence even about 0 and n_a), FP64.  For a
// field kernel odd in axis `odd` (0 = x, 1 = y, 2 = z) that axis takes the
// DST-I instead: the 2N DFT of the odd extension is -i times the result.
fsp_status enqueue_trig_spectrum3(const int *nn, int odd, double *t_dev, cudaStream_t s, Temps &tmp) {
    const int k[3] = {nn[0] + 1, nn[1] + 1, nn[2] + 1};
    const int len[3] = {2 * nn[0], 2 * nn[1], 2 * nn[2]};
    TileCfg c[3];
    for (int a = 0; a < 3; ++a)
        if (!make_cfg(len[a], len[a], sizeof(double2), 3, c[a])) return FSP_EUNSUPPORTED;
    const void *tab[3];
    fsp_status st = roots_3(tmp, len, tab, s);
    if (st != FSP_OK) return st;
    LinesArgs a{};
    a.in = a.out = t_dev;
    // x: rows
    a.tw = tab[0], a.st = c[0].st, a.tpl = c[0].tpl, a.lgL = c[0].lgL;
    a.n_out = k[0];
    a.in_pos = a.out_pos = 1, a.in_line = a.out_line = k[0], a.in_batch = a.out_batch = 0;
    a.nlines = k[1] * k[2], a.nbatch = 1;
    FSP_TRY_CUDA(launch_trig(odd == 0, a, s));
    // y: columns, batch z
    a.tw = tab[1], a.st = c[1].st, a.tpl = c[1].tpl, a.lgL = c[1].lgL;
    a.n_out = k[1];
    a.in_pos = a.out_pos = k[0], a.in_line = a.out_line = 1, a.in_batch = a.out_batch = (long long)k[1] * k[0];
    a.nlines = k[0], a.nbatch = k[2];
    FSP_TRY_CUDA(launch_trig(odd == 1, a, s));
    // z: columns, batch y
    a.tw = tab[2], a.st = c[2].st, a.tpl = c[2].tpl, a.lgL = c[2].lgL;
    a.n_out = k[2];
    a.in_pos = a.out_pos = (long long)k[1] * k[0], a.in_batch = a.out_batch = k[0];
    a.nlines = k[0], a.nbatch = k[1];
    FSP_TRY_CUDA(launch_trig(odd == 2, a, s));
    return FSP_OK;
}

fsp_status enqueue_trig_spectrum(int N, int odd, double *t_dev, cudaStream_t s, Temps &tmp) {
    const int nn[3] = {N, N, N};
    return enqueue_trig_spectrum3(nn, odd, t_dev, s, tmp);
}

fsp_status enqueue_dct_spectrum(int N, double *t_dev, cudaStream_t s, Temps &tmp) {
    return enqueue_trig_spectrum(N, -1, t_dev, s, tmp);
}

// Field kernel F_a[m] = -dG/dx_a (m h), m in [0,N]^3, into f_dev (FP64), for
// E = -grad phi (Appendix B, Eq. efield).  Hockney-Eastwood: the sampled
// gradient of 1/(4 pi |x|), zero at the origin.  Vico-Greengard (both forms):
// the inverse transform of -i k_a G_L (Sec. 2.3) through the (2N+1)^3 octant,
// where k_a G_L is odd in j_a: DST-I along a, DCT-I along the others, times
// (4Nh)^-3 (the octant form of the (4N)^3 sum with its Nyquist plane j_a = -2N
// at zero).
fsp_status enqueue_field_kernel(int N, double L, fsp_algo algo, int axis, double *f_dev, cudaStream_t s, Temps &tmp) {
    const double h = L / N;
    const int k1 = N + 1, nm = 2 * N + 1;
    if (algo == FSP_HE) return cuda_status(launch_he_F(f_dev, N, h, axis, s));
    const double Lt = kAlpha * std::sqrt(3.0) * L;
    fsp_status st;
    if ((st = alloc_or_nomem(tmp.g, sizeof(double) * (size_t)nm * nm * nm)) != FSP_OK) return st;
    FSP_TRY_CUDA(launch_vg_sample_octant_grad((double *)tmp.g.p, N, h, Lt, axis, s));
    if ((st = enqueue_octant_transform(N, axis, (double *)tmp.g.p, f_dev, s, tmp)) != FSP_OK) return st;
    const double scale = 1.0 / ((4.0 * N * h) * (4.0 * N * h) * (4.0 * N * h));
    return cuda_status(launch_scale(f_dev, (long long)k1 * k1 * k1, scale, s));
}

// The same on a non-cubic box (per-axis sizes and spacings, window
// 1.1 |(L_x, L_y, L_z)|), (n_z+1)(n_y+1)(n_x+1) values.
fsp_status enqueue_field_kernel3(const int *nn, const double *hh, fsp_algo algo, int axis, double *f_dev, cudaStream_t s,
                                 Temps &tmp) {
    if (algo == FSP_HE) return cuda_status(launch_he_F3(f_dev, nn, hh, axis, s));
    const double Lb[3] = {nn[0] * hh[0], nn[1] * hh[1], nn[2] * hh[2]};
    const double Lt = kAlpha * std::sqrt(Lb[0] * Lb[0] + Lb[1] * Lb[1] + Lb[2] * Lb[2]);
    fsp_status st;
    const size_t q = (size_t)(2 * nn[0] + 1) * (2 * nn[1] + 1) * (2 * nn[2] + 1);
    if ((st = alloc_or_nomem(tmp.g, sizeof(double) * q)) != FSP_OK) return st;
    FSP_TRY_CUDA(launch_vg_sample_octant_grad3((double *)tmp.g.p, nn, hh, Lt, axis, s));
    if ((st = enqueue_octant_transform3(nn, axis, (double *)tmp.g.p, f_dev, s, tmp)) != FSP_OK) return st;
    const double scale = 1.0 / ((4.0 * nn[0] * hh[0]) * (4.0 * nn[1] * hh[1]) * (4.0 * nn[2] * hh[2]));
    return cuda_status(launch_scale(f_dev, (long long)(nn[0] + 1) * (nn[1] + 1) * (nn[2] + 1), scale, s));
}

fsp_status validate_size(int N, double L, fsp_algo algo) {
    if (N < 2 || N > kMaxN) return N < 2 ? FSP_EINVAL : FSP_EUNSUPPORTED;
    if (!(L > 0.0) || !std::isfinite(L)) return FSP_EINVAL;
    if (algo != FSP_HE && algo != FSP_VG && algo != FSP_VG_DCT) return FSP_EINVAL;
    if (!is_235_smooth(2LL * N)) return FSP_EUNSUPPORTED;
    if (algo == FSP_VG && !is_235_smooth(4LL * N)) return FSP_EUNSUPPORTED;
    return FSP_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// ------------------------------------------------------------------ plan --
struct fsp_plan {
    uint64_t magic = 0;
    int N = 0, P = 0, device = 0;
    double L = 0, h = 0;
    fsp_algo algo = FSP_HE;
    fsp_dtype dtype = FSP_F64;
    size_t rsize = 8;  // bytes per real
    void *S = nullptr, *W1 = nullptr, *W2 = nullptr, *tw_n = nullptr, *tw_2n = nullptr;
    void *stage_rho = nullptr, *stage_phi = nullptr;
    // pipelined host solves: kPipeSlots staging slots, copy streams, events
    void *pipe_rho[kPipeSlots] = {}, *pipe_phi[kPipeSlots] = {};
    cudaStream_t pipe_h2d = nullptr, pipe_d2h = nullptr;
    cudaEvent_t ev_in[kPipeSlots] = {}, ev_comp[kPipeSlots] = {}, ev_out[kPipeSlots] = {};
    TileCfg row, col;
    bool fast = false;  // specialised power-of-two kernels (fast.cuh) serve this N
    bool p3_tma = false;  // P3 by the TMA-staged persistent kernel (p3_tma.cuh)
    bool plane = false;   // three launches: fused plane passes PA, PC around P3 (plane.cuh)
    unsigned *err = nullptr;  // device word: bit 0 = a bounded device-side wait timed out
    unsigned long long wait_timeout_ns = 1000000000ull;  // per device-side wait
    mutable std::atomic<unsigned> inject_tx{0};  // fault injection, consumed by the next solve
    // field solves (fsp_plan_field_init): the spectra of F_x, F_y, F_z and the
    // third workspace the out-of-place P3 of each component writes
    void *SF[3] = {}, *W3 = nullptr;
    // a non-cubic box (fsp_plan_create_aniso): n3 cells and h3 spacings per
    // axis, the generic engine with its own tiles and roots for the y (2 n_y)
    // and z (2 n_z) lines; rows use tw_n / tw_2n of n_x
    bool aniso = false;
    int n3[3] = {};
    double h3[3] = {};
    TileCfg colz;
    void *tw_y = nullptr, *tw_z = nullptr;
    cudaEvent_t ev[6] = {};
    bool timing = false;
    bool guarded = false;  // FSP_CHECK_BOUNDS=1 at creation: buffers with guard bands
    size_t bytes = 0;
    double precompute_ms = 0;
};

namespace {

bool plan_live(const fsp_plan *p) {
    std::lock_guard<std::mutex> lk(g_mu);
    return p && g_plans.count(p) && p->magic == kMagic;
}

// grid points of a plan's source / result
size_t plan_points(const fsp_plan *p) {
    return p->aniso ? (size_t)p->n3[0] * p->n3[1] * p->n3[2] : (size_t)p->N * p->N * p->N;
}

void plan_free(fsp_plan *p) {
    for (void *q : {p->S, p->W1, p->W2, p->tw_n, p->tw_2n, p->stage_rho, p->stage_phi, p->SF[0], p->SF[1], p->SF[2],
                    p->W3, p->tw_y, p->tw_z, (void *)p->err})
        if (q) dev_free(q);
    for (int i = 0; i < kPipeSlots; ++i)
        for (void *q : {p->pipe_rho[i], p->pipe_phi[i]})
            if (q) dev_free(q);
    for (cudaStream_t q : {p->pipe_h2d, p->pipe_d2h})
        if (q) cudaStreamDestroy(q);
    for (int i = 0; i < kPipeSlots; ++i)
        for (cudaEvent_t q : {p->ev_in[i], p->ev_comp[i], p->ev_out[i]})
            if (q) cudaEventDestroy(q);
    p->magic = 0;
    delete p;
}

// Three launches: PA (P1 + P2 per z-plane, W1 through L2 only), P3, PC (P4 +
// P5 per z-plane).  The timing hook's six events then bracket PA as the first
// pass and PC as the fourth (the second and fifth are empty).
cudaError_t enqueue_solve_plane(const fsp_plan *p, const void *rho, void *phi, void *W1, void *W2, cudaStream_t s) {
    const int N = p->N;
    const long long P = p->P;
    cudaError_t e;
    auto mark = [&](int i) { return p->timing ? cudaEventRecord(p->ev[i], s) : cudaSuccess; };
    fast::PlaneArgs pa{rho, phi, W1, W2, p->tw_n, p->tw_2n};
    if ((e = mark(0)) != cudaSuccess) return e;
    if ((e = fast::plane_fwd<float>(N, pa, s)) != cudaSuccess) return e;  // PA
    if ((e = mark(1)) != cudaSuccess || (e = mark(2)) != cudaSuccess) return e;
    fast::ColArgs a{};
    a.tw = p->tw_2n, a.nlines = N + 1;
    a.in = a.out = W2;  // P3: z-FFT * S * z-IFFT, in place, batch ky
    a.in_pos = a.out_pos = 2LL * N * P, a.in_batch = a.out_batch = P;
    a.S = p->S, a.s_pos = (long long)(N + 1) * P, a.s_batch = P, a.half = N;
    if (p->p3_tma) {
        fast::P3Wait w{p->err, p->wait_timeout_ns, p->inject_tx.exchange(0)};
        e = fast::p3_tma<float>(N, W2, p->S, p->tw_2n, w, s);
    } else {
        e = fast::p3<float>(N, a, 2 * N, s);
    }
    if (e != cudaSuccess) return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    if ((e = fast::plane_inv<float>(N, pa, s)) != cudaSuccess) return e;  // PC
    if ((e = mark(4)) != cudaSuccess) return e;
    return mark(5);
}

template <typename T>
cudaError_t enqueue_solve_fast(const fsp_plan *p, const void *rho, void *phi, void *W1, void *W2, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value)
        if (p->plane) return enqueue_solve_plane(p, rho, phi, W1, W2, s);
    const int N = p->N;
    const long long P = p->P;
    cudaError_t e;
    auto mark = [&](int i) { return p->timing ? cudaEventRecord(p->ev[i], s) : cudaSuccess; };
    fast::RowArgs r{};
    r.x = rho, r.c = W1, r.x_row = N, r.c_row = P, r.nrows = N * N, r.tw = p->tw_n, r.tw2 = p->tw_2n;
    fast::ColArgs a{};
    a.tw = p->tw_2n, a.nlines = N + 1;
    if ((e = mark(0)) != cudaSuccess) return e;
    if ((e = fast::p1<T>(N, r, s)) != cudaSuccess) return e;  // P1: pad + x-R2C
    if ((e = mark(1)) != cudaSuccess) return e;
    a.in = W1, a.out = W2;  // P2: y-FFT, W1[z][y][kx] -> W2[z][ky][kx]
    a.in_pos = P, a.in_batch = (long long)N * P, a.out_pos = P, a.out_batch = 2LL * N * P;
    if ((e = fast::p2<T>(N, a, N, s)) != cudaSuccess) return e;
    if ((e = mark(2)) != cudaSuccess) return e;
    a.in = a.out = W2;  // P3: z-FFT * S * z-IFFT, in place, batch ky
    a.in_pos = a.out_pos = 2LL * N * P, a.in_batch = a.out_batch = P;
    a.S = p->S, a.s_pos = (long long)(N + 1) * P, a.s_batch = P, a.half = N;
    if constexpr (std::is_same<T, float>::value) {
        if (p->p3_tma) {
            fast::P3Wait w{p->err, p->wait_timeout_ns, p->inject_tx.exchange(0)};
            e = fast::p3_tma<float>(N, W2, p->S, p->tw_2n, w, s);
        }
        else
            e = fast::p3<T>(N, a, 2 * N, s);
    } else {
        e = fast::p3<T>(N, a, 2 * N, s);
    }
    if (e != cudaSuccess) return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    a.in = W2, a.out = W1;  // P4: y-IFFT, W2 -> W1 (y < N)
    a.in_pos = P, a.in_batch = 2LL * N * P, a.out_pos = P, a.out_batch = (long long)N * P;
    if ((e = fast::p4<T>(N, a, N, s)) != cudaSuccess) return e;
    if ((e = mark(4)) != cudaSuccess) return e;
    r.x = phi;  // P5: x-C2R, W1 rows -> phi
    if ((e = fast::p5<T>(N, r, s)) != cudaSuccess) return e;
    return mark(5);
}

template <typename T>
cudaError_t enqueue_solve_generic(const fsp_plan *p, const void *rho, void *phi, void *W1, void *W2, cudaStream_t s) {
    const int N = p->N;
    const long long P = p->P;
    cudaError_t e;
    auto mark = [&](int i) { return p->timing ? cudaEventRecord(p->ev[i], s) : cudaSuccess; };
    // P1: pad + x-R2C (rows of rho -> W1[z][y][kx])
    if ((e = mark(0)) != cudaSuccess) return e;
    RowsArgs r{};
    r.x = rho, r.c = W1, r.x_row = N, r.c_row = P, r.N = N, r.nrows = N * N;
    r.lgL = p->row.lgL, r.tpl = p->row.tpl, r.st = p->row.st, r.tw = p->tw_n, r.tw2 = p->tw_2n;
    if ((e = launch_r2c_rows<T>(r, s)) != cudaSuccess) return e;
    if ((e = mark(1)) != cudaSuccess) return e;
    // P2: y-FFT (columns kx of W1[z][y][.], y < N zero-padded to 2N) -> W2[z][ky][kx]
    LinesArgs a{};
    a.st = p->col.st, a.tpl = p->col.tpl, a.lgL = p->col.lgL, a.tw = p->tw_2n;
    a.in = W1, a.out = W2;
    a.in_pos = P, a.in_line = 1, a.in_batch = (long long)N * P;
    a.out_pos = P, a.out_line = 1, a.out_batch = 2LL * N * P;
    a.n_in = N, a.n_out = 2 * N, a.nlines = N + 1, a.nbatch = N;
    if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD>(a, s)) != cudaSuccess) return e;
    if ((e = mark(2)) != cudaSuccess) return e;
    // P3: z-FFT, multiply by S, z-IFFT, keep z < N (in place in W2, batch ky)
    a.in = a.out = W2;
    a.in_pos = a.out_pos = 2LL * N * P, a.in_batch = a.out_batch = P;
    a.n_in = N, a.n_out = N, a.nbatch = 2 * N;
    a.S = p->S, a.s_pos = (long long)(N + 1) * P, a.s_batch = P, a.half = N;
    if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD_MUL_INV>(a, s)) != cudaSuccess) return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    // P4: y-IFFT, keep y < N: W2[z][ky][kx] -> W1[z][y][kx]
    a.in = W2, a.out = W1;
    a.in_pos = P, a.in_batch = 2LL * N * P;
    a.out_pos = P, a.out_batch = (long long)N * P;
    a.n_in = 2 * N, a.n_out = N, a.nbatch = N;
    if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_INV>(a, s)) != cudaSuccess) return e;
    if ((e = mark(4)) != cudaSuccess) return e;
    // P5: x-C2R, keep x < N: W1 rows -> phi
    r.x = phi;
    if ((e = launch_c2r_rows<T>(r, s)) != cudaSuccess) return e;
    return mark(5);
}

// The field E = -grad phi (and phi, when out[3] is set): P1 and P2 once, then
// per output P3 (W2 -> W3 with that output's spectrum), P4 (W3 -> W1), P5
// (W1 -> output).  out[0..2] = E_x, E_y, E_z, out[3] = phi or null.  The odd
// axis of component a is the line (k_x), the batch (k_y) or the position (z)
// of the P3 pass.
constexpr int kP3Odd[3] = {3, 2, 1};

template <typename T>
cudaError_t enqueue_field_fast(const fsp_plan *p, const void *rho, void *const out[4], cudaStream_t s) {
    const int N = p->N;
    const long long P = p->P;
    cudaError_t e;
    fast::RowArgs r{};
    r.x = rho, r.c = p->W1, r.x_row = N, r.c_row = P, r.nrows = N * N, r.tw = p->tw_n, r.tw2 = p->tw_2n;
    fast::ColArgs a{};
    a.tw = p->tw_2n, a.nlines = N + 1;
    a.in = p->W1, a.out = p->W2;
    a.in_pos = P, a.in_batch = (long long)N * P, a.out_pos = P, a.out_batch = 2LL * N * P;
    if constexpr (std::is_same<T, float>::value) {
        if (p->plane) {  // the solve's own passes: PA once, then P3 and PC per output
            fast::PlaneArgs pa{rho, nullptr, p->W1, p->W2, p->tw_n, p->tw_2n};
            if ((e = fast::plane_fwd<float>(N, pa, s)) != cudaSuccess) return e;
            for (int c = 3; c >= 0; --c) {
                if (!out[c]) continue;
                fast::ColArgs b = a;
                b.in = p->W2, b.out = p->W3;
                b.in_pos = b.out_pos = 2LL * N * P, b.in_batch = b.out_batch = P;
                b.S = c == 3 ? p->S : p->SF[c], b.s_pos = (long long)(N + 1) * P, b.s_batch = P, b.half = N;
                b.odd = c == 3 ? 0 : kP3Odd[c];
                if ((e = c == 3 ? fast::p3<T>(N, b, 2 * N, s) : fast::p3_odd<T>(N, b, 2 * N, s)) != cudaSuccess)
                    return e;
                fast::PlaneArgs pc{nullptr, out[c], p->W1, p->W3, p->tw_n, p->tw_2n};
                if ((e = fast::plane_inv<float>(N, pc, s)) != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
    }
    if ((e = fast::p1<T>(N, r, s)) != cudaSuccess) return e;
    if ((e = fast::p2<T>(N, a, N, s)) != cudaSuccess) return e;
    for (int c = 3; c >= 0; --c) {
        if (!out[c]) continue;
        fast::ColArgs b = a;
        b.in = p->W2, b.out = p->W3;
        b.in_pos = b.out_pos = 2LL * N * P, b.in_batch = b.out_batch = P;
        b.S = c == 3 ? p->S : p->SF[c], b.s_pos = (long long)(N + 1) * P, b.s_batch = P, b.half = N;
        b.odd = c == 3 ? 0 : kP3Odd[c];
        if ((e = c == 3 ? fast::p3<T>(N, b, 2 * N, s) : fast::p3_odd<T>(N, b, 2 * N, s)) != cudaSuccess) return e;
        b.in = p->W3, b.out = p->W1, b.odd = 0;
        b.in_pos = P, b.in_batch = 2LL * N * P, b.out_pos = P, b.out_batch = (long long)N * P;
        if ((e = fast::p4<T>(N, b, N, s)) != cudaSuccess) return e;
        r.x = out[c];
        if ((e = fast::p5<T>(N, r, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t enqueue_field_generic(const fsp_plan *p, const void *rho, void *const out[4], cudaStream_t s) {
    const int N = p->N;
    const long long P = p->P;
    cudaError_t e;
    RowsArgs r{};
    r.x = rho, r.c = p->W1, r.x_row = N, r.c_row = P, r.N = N, r.nrows = N * N;
    r.lgL = p->row.lgL, r.tpl = p->row.tpl, r.st = p->row.st, r.tw = p->tw_n, r.tw2 = p->tw_2n;
    if ((e = launch_r2c_rows<T>(r, s)) != cudaSuccess) return e;
    LinesArgs a{};
    a.st = p->col.st, a.tpl = p->col.tpl, a.lgL = p->col.lgL, a.tw = p->tw_2n;
    a.in = p->W1, a.out = p->W2;
    a.in_pos = P, a.in_line = 1, a.in_batch = (long long)N * P;
    a.out_pos = P, a.out_line = 1, a.out_batch = 2LL * N * P;
    a.n_in = N, a.n_out = 2 * N, a.nlines = N + 1, a.nbatch = N;
    if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD>(a, s)) != cudaSuccess) return e;
    for (int c = 3; c >= 0; --c) {
        if (!out[c]) continue;
        LinesArgs b = a;
        b.in = p->W2, b.out = p->W3;
        b.in_pos = b.out_pos = 2LL * N * P, b.in_batch = b.out_batch = P;
        b.n_in = N, b.n_out = N, b.nbatch = 2 * N;
        b.S = c == 3 ? p->S : p->SF[c], b.s_pos = (long long)(N + 1) * P, b.s_batch = P, b.half = N;
        b.odd = c == 3 ? 0 : kP3Odd[c];
        if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD_MUL_INV>(b, s)) != cudaSuccess) return e;
        b.in = p->W3, b.out = p->W1, b.odd = 0;
        b.in_pos = P, b.in_batch = 2LL * N * P;
        b.out_pos = P, b.out_batch = (long long)N * P;
        b.n_in = 2 * N, b.n_out = N, b.nbatch = N;
        if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_INV>(b, s)) != cudaSuccess) return e;
        r.x = out[c];
        if ((e = launch_c2r_rows<T>(r, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The field on a non-cubic box: P1, P2 once, then per output P3 (W2 -> W3,
// S folded at n_z in z and n_y in k_y), P4, P5; generic engine or the
// specialised kernels with runtime strides.
template <typename T>
cudaError_t enqueue_field_aniso(const fsp_plan *p, const void *rho, void *const out[4], cudaStream_t s) {
    const int nx = p->n3[0], ny = p->n3[1], nz = p->n3[2];
    const long long P = p->P;
    cudaError_t e;
    if (p->fast) {
        fast::RowArgs r{};
        r.x = rho, r.c = p->W1, r.x_row = nx, r.c_row = P, r.nrows = ny * nz, r.tw = p->tw_n, r.tw2 = p->tw_2n;
        if ((e = fast::p1<T>(nx, r, s)) != cudaSuccess) return e;
        fast::ColArgs a{};
        a.nlines = nx + 1;
        a.tw = p->tw_y, a.in = p->W1, a.out = p->W2;
        a.in_pos = P, a.in_batch = (long long)ny * P, a.out_pos = P, a.out_batch = 2LL * ny * P;
        if ((e = fast::col_rg<T>(fast::COL_FWD, 2 * ny, a, nz, s)) != cudaSuccess) return e;
        for (int c = 3; c >= 0; --c) {
            if (!out[c]) continue;
            fast::ColArgs b = a;
            b.tw = p->tw_z, b.in = p->W2, b.out = p->W3;
            b.in_pos = b.out_pos = 2LL * ny * P, b.in_batch = b.out_batch = P;
            b.S = c == 3 ? p->S : p->SF[c], b.s_pos = (long long)(ny + 1) * P, b.s_batch = P, b.half = nz, b.half_b = ny;
            b.odd = c == 3 ? 0 : kP3Odd[c];
            if ((e = c == 3 ? fast::col_rg<T>(fast::COL_FMI, 2 * nz, b, 2 * ny, s)
                            : fast::p3_odd_rg<T>(2 * nz, b, 2 * ny, s)) != cudaSuccess)
                return e;
            b.tw = p->tw_y, b.in = p->W3, b.out = p->W1, b.odd = 0;
            b.in_pos = P, b.in_batch = 2LL * ny * P, b.out_pos = P, b.out_batch = (long long)ny * P;
            if ((e = fast::col_rg<T>(fast::COL_INV, 2 * ny, b, nz, s)) != cudaSuccess) return e;
            r.x = out[c];
            if ((e = fast::p5<T>(nx, r, s)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if constexpr (std::is_same<T, df>::value) {
        return cudaErrorInvalidValue;  // double-float plans always have the specialised kernels
    } else {
        RowsArgs r{};
        r.x = rho, r.c = p->W1, r.x_row = nx, r.c_row = P, r.N = nx, r.nrows = ny * nz;
        r.lgL = p->row.lgL, r.tpl = p->row.tpl, r.st = p->row.st, r.tw = p->tw_n, r.tw2 = p->tw_2n;
        if ((e = launch_r2c_rows<T>(r, s)) != cudaSuccess) return e;
        LinesArgs a{};
        a.st = p->col.st, a.tpl = p->col.tpl, a.lgL = p->col.lgL, a.tw = p->tw_y;
        a.in = p->W1, a.out = p->W2;
        a.in_pos = P, a.in_line = 1, a.in_batch = (long long)ny * P;
        a.out_pos = P, a.out_line = 1, a.out_batch = 2LL * ny * P;
        a.n_in = ny, a.n_out = 2 * ny, a.nlines = nx + 1, a.nbatch = nz;
        if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD>(a, s)) != cudaSuccess) return e;
        for (int c = 3; c >= 0; --c) {
            if (!out[c]) continue;
            LinesArgs b = a;
            b.st = p->colz.st, b.tpl = p->colz.tpl, b.lgL = p->colz.lgL, b.tw = p->tw_z;
            b.in = p->W2, b.out = p->W3;
            b.in_pos = b.out_pos = 2LL * ny * P, b.in_batch = b.out_batch = P;
            b.n_in = nz, b.n_out = nz, b.nbatch = 2 * ny;
            b.S = c == 3 ? p->S : p->SF[c], b.s_pos = (long long)(ny + 1) * P, b.s_batch = P, b.half = nz, b.half_b = ny;
            b.odd = c == 3 ? 0 : kP3Odd[c];
            if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD_MUL_INV>(b, s)) != cudaSuccess) return e;
            b.st = p->col.st, b.tpl = p->col.tpl, b.lgL = p->col.lgL, b.tw = p->tw_y;
            b.in = p->W3, b.out = p->W1, b.odd = 0, b.half_b = 0;
            b.in_pos = P, b.in_batch = 2LL * ny * P;
            b.out_pos = P, b.out_batch = (long long)ny * P;
            b.n_in = 2 * ny, b.n_out = ny, b.nbatch = nz;
            if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_INV>(b, s)) != cudaSuccess) return e;
            r.x = out[c];
            if ((e = launch_c2r_rows<T>(r, s)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
}

cudaError_t enqueue_field(const fsp_plan *p, const void *rho, void *const out[4], cudaStream_t s) {
    if (p->aniso)
        return p->dtype == FSP_F64      ? enqueue_field_aniso<double>(p, rho, out, s)
               : p->dtype == FSP_F64_DF ? enqueue_field_aniso<df>(p, rho, out, s)
                                        : enqueue_field_aniso<float>(p, rho, out, s);
    if (p->dtype == FSP_F64_DF) return enqueue_field_fast<df>(p, rho, out, s);
    if (p->fast)
        return p->dtype == FSP_F64 ? enqueue_field_fast<double>(p, rho, out, s)
                                   : enqueue_field_fast<float>(p, rho, out, s);
    return p->dtype == FSP_F64 ? enqueue_field_generic<double>(p, rho, out, s)
                               : enqueue_field_generic<float>(p, rho, out, s);
}

// Sec. 2.2 steps 1-5 on a non-cubic box, generic engine: P1 rows of n_x, P2
// y lines of 2 n_y (batch z), P3 z lines of 2 n_z (batch k_y; S folded at n_z
// in z and n_y in k_y), P4, P5.  W1 = n_z n_y P, W2 = n_z 2 n_y P complex.
template <typename T>
cudaError_t enqueue_solve_aniso(const fsp_plan *p, const void *rho, void *phi, void *W1, void *W2, cudaStream_t s) {
    const int nx = p->n3[0], ny = p->n3[1], nz = p->n3[2];
    const long long P = p->P;
    cudaError_t e;
    auto mark = [&](int i) { return p->timing ? cudaEventRecord(p->ev[i], s) : cudaSuccess; };
    if ((e = mark(0)) != cudaSuccess) return e;
    RowsArgs r{};
    r.x = rho, r.c = W1, r.x_row = nx, r.c_row = P, r.N = nx, r.nrows = ny * nz;
    r.lgL = p->row.lgL, r.tpl = p->row.tpl, r.st = p->row.st, r.tw = p->tw_n, r.tw2 = p->tw_2n;
    if ((e = launch_r2c_rows<T>(r, s)) != cudaSuccess) return e;
    if ((e = mark(1)) != cudaSuccess) return e;
    LinesArgs a{};
    a.st = p->col.st, a.tpl = p->col.tpl, a.lgL = p->col.lgL, a.tw = p->tw_y;
    a.in = W1, a.out = W2;
    a.in_pos = P, a.in_line = 1, a.in_batch = (long long)ny * P;
    a.out_pos = P, a.out_line = 1, a.out_batch = 2LL * ny * P;
    a.n_in = ny, a.n_out = 2 * ny, a.nlines = nx + 1, a.nbatch = nz;
    if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD>(a, s)) != cudaSuccess) return e;
    if ((e = mark(2)) != cudaSuccess) return e;
    a.st = p->colz.st, a.tpl = p->colz.tpl, a.lgL = p->colz.lgL, a.tw = p->tw_z;
    a.in = a.out = W2;
    a.in_pos = a.out_pos = 2LL * ny * P, a.in_batch = a.out_batch = P;
    a.n_in = nz, a.n_out = nz, a.nbatch = 2 * ny;
    a.S = p->S, a.s_pos = (long long)(ny + 1) * P, a.s_batch = P, a.half = nz, a.half_b = ny;
    if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD_MUL_INV>(a, s)) != cudaSuccess) return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    a.st = p->col.st, a.tpl = p->col.tpl, a.lgL = p->col.lgL, a.tw = p->tw_y;
    a.in = W2, a.out = W1;
    a.in_pos = P, a.in_batch = 2LL * ny * P;
    a.out_pos = P, a.out_batch = (long long)ny * P;
    a.n_in = 2 * ny, a.n_out = ny, a.nbatch = nz;
    if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_INV>(a, s)) != cudaSuccess) return e;
    if ((e = mark(4)) != cudaSuccess) return e;
    r.x = phi;
    if ((e = launch_c2r_rows<T>(r, s)) != cudaSuccess) return e;
    return mark(5);
}

// The same on the specialised kernels (every n_a a power of two in [32, 512]):
// the rows depend on n_x only; the column passes take runtime geometry.
template <typename T>
cudaError_t enqueue_solve_aniso_fast(const fsp_plan *p, const void *rho, void *phi, void *W1, void *W2, cudaStream_t s) {
    const int nx = p->n3[0], ny = p->n3[1], nz = p->n3[2];
    const long long P = p->P;
    cudaError_t e;
    auto mark = [&](int i) { return p->timing ? cudaEventRecord(p->ev[i], s) : cudaSuccess; };
    fast::RowArgs r{};
    r.x = rho, r.c = W1, r.x_row = nx, r.c_row = P, r.nrows = ny * nz, r.tw = p->tw_n, r.tw2 = p->tw_2n;
    if ((e = mark(0)) != cudaSuccess) return e;
    if ((e = fast::p1<T>(nx, r, s)) != cudaSuccess) return e;
    if ((e = mark(1)) != cudaSuccess) return e;
    fast::ColArgs a{};
    a.nlines = nx + 1;
    a.tw = p->tw_y, a.in = W1, a.out = W2;
    a.in_pos = P, a.in_batch = (long long)ny * P, a.out_pos = P, a.out_batch = 2LL * ny * P;
    if ((e = fast::col_rg<T>(fast::COL_FWD, 2 * ny, a, nz, s)) != cudaSuccess) return e;
    if ((e = mark(2)) != cudaSuccess) return e;
    a.tw = p->tw_z, a.in = a.out = W2;
    a.in_pos = a.out_pos = 2LL * ny * P, a.in_batch = a.out_batch = P;
    a.S = p->S, a.s_pos = (long long)(ny + 1) * P, a.s_batch = P, a.half = nz, a.half_b = ny;
    if ((e = fast::col_rg<T>(fast::COL_FMI, 2 * nz, a, 2 * ny, s)) != cudaSuccess) return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    a.tw = p->tw_y, a.in = W2, a.out = W1;
    a.in_pos = P, a.in_batch = 2LL * ny * P, a.out_pos = P, a.out_batch = (long long)ny * P;
    if ((e = fast::col_rg<T>(fast::COL_INV, 2 * ny, a, nz, s)) != cudaSuccess) return e;
    if ((e = mark(4)) != cudaSuccess) return e;
    r.x = phi;
    if ((e = fast::p5<T>(nx, r, s)) != cudaSuccess) return e;
    return mark(5);
}

// One solve of plan p with the given workspace (W1: N*N*P, W2: 2*N*N*P complex).
cudaError_t enqueue_solve_ws(const fsp_plan *p, const void *rho, void *phi, void *W1, void *W2, cudaStream_t s) {
    if (p->aniso) {
        if (p->fast)
            return p->dtype == FSP_F64      ? enqueue_solve_aniso_fast<double>(p, rho, phi, W1, W2, s)
                   : p->dtype == FSP_F64_DF ? enqueue_solve_aniso_fast<df>(p, rho, phi, W1, W2, s)
                                            : enqueue_solve_aniso_fast<float>(p, rho, phi, W1, W2, s);
        return p->dtype == FSP_F64 ? enqueue_solve_aniso<double>(p, rho, phi, W1, W2, s)
                                   : enqueue_solve_aniso<float>(p, rho, phi, W1, W2, s);
    }
    if (p->dtype == FSP_F64_DF) return enqueue_solve_fast<df>(p, rho, phi, W1, W2, s);
    if (p->fast)
        return p->dtype == FSP_F64 ? enqueue_solve_fast<double>(p, rho, phi, W1, W2, s)
                                   : enqueue_solve_fast<float>(p, rho, phi, W1, W2, s);
    return p->dtype == FSP_F64 ? enqueue_solve_generic<double>(p, rho, phi, W1, W2, s)
                               : enqueue_solve_generic<float>(p, rho, phi, W1, W2, s);
}

}  // namespace

extern "C" {

const char *fsp_status_str(fsp_status s) {
    switch (s) {
    case FSP_OK: return "FSP_OK";
    case FSP_EINVAL: return "FSP_EINVAL: invalid argument";
    case FSP_EUNSUPPORTED: return "FSP_EUNSUPPORTED: unsupported size";
    case FSP_ENOMEM: return "FSP_ENOMEM: out of device memory or over budget";
    case FSP_ECUDA: return "FSP_ECUDA: CUDA error";
    case FSP_EBUSY: return "FSP_EBUSY: busy";
    case FSP_ETIMEOUT: return "FSP_ETIMEOUT: device-side wait timed out";
    }
    return "FSP_?: unknown status";
}

}  // extern "C"

namespace {
// s_host: null to compute the spectrum (Sec. 2.2-2.4), else (N+1)^3 doubles
// of a stored one (the octant fsp_plan_spectrum writes, already scaled)
fsp_status plan_create_impl(fsp_plan **out, int N, double L, double h, fsp_algo algo, fsp_dtype dtype,
                            fsp_stream stream, bool with_workspace, const double *s_host = nullptr) {
    if (!out) return FSP_EINVAL;
    *out = nullptr;
    fsp_status st = validate_size(N, L, algo);
    if (st != FSP_OK) return st;
    if (dtype != FSP_F64 && dtype != FSP_F32_MIXED && dtype != FSP_F64_DF) return FSP_EINVAL;
    if (!(std::fabs(h - L / N) <= 1e-12 * std::fabs(L / N))) return FSP_EINVAL;
    if (dtype == FSP_F64_DF && !fast::has<df>(N)) return FSP_EUNSUPPORTED;  // specialised kernels only
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();

    fsp_plan *p = new fsp_plan();
    p->guarded = bounds_check_requested();
    GuardScope guard_scope(p->guarded);
    p->N = N, p->L = L, p->h = L / N, p->algo = algo, p->dtype = dtype;
    p->rsize = dtype == FSP_F32_MIXED ? 4 : 8;  // caller's reals; a double-float is 8 bytes too
    p->P = ((N + 1) + 15) / 16 * 16;
    const size_t csize = 2 * p->rsize;
    // tiles: rows (length-N FFT, N+1 positions), columns (length 2N)
    int row_lgL = dtype == FSP_F32_MIXED ? 4 : 3, col_lgL = dtype == FSP_F32_MIXED ? 4 : 3;
    tuned_lgL(N, (int)dtype, row_lgL, col_lgL);
    if (!make_cfg(N, N + 1, csize, row_lgL, p->row) || !make_cfg(2 * N, 2 * N, csize, col_lgL, p->col)) {
        delete p;
        return FSP_EUNSUPPORTED;
    }
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return FSP_ECUDA;
    }
    // specialised kernels for power-of-two N unless FSP_GENERIC_ONLY=1 (A/B and tests)
    {
        const char *g = std::getenv("FSP_GENERIC_ONLY");
        const bool generic_only = g && g[0] == '1';
        p->fast = dtype == FSP_F64_DF ||
                  (!generic_only && (dtype == FSP_F64 ? fast::has<double>(N) : fast::has<float>(N)));
        // the TMA-staged P3 only with FSP_P3_TMA=1: measured slower than the
        // register-direct P3 on the GB300 (kept for the A/B and its tests)
        const char *t = std::getenv("FSP_P3_TMA");
        p->p3_tma = p->fast && dtype == FSP_F32_MIXED && fast::has_p3_tma<float>(N) && t && t[0] == '1';
        // the fused plane passes where they measured faster; FSP_PLANE=1 / 0
        // forces them on (every size that has them) / off, for the A/B
        const char *pl = std::getenv("FSP_PLANE");
        const bool plane_ok = p->fast && dtype == FSP_F32_MIXED && fast::has_plane<float>(N);
        p->plane = plane_ok && (pl && pl[0] == '1' ? true : pl && pl[0] == '0' ? false : fast::plane_default<float>(N));
    }
    auto fail = [&](fsp_status e) {
        cudaStreamSynchronize(s);
        plan_free(p);
        return e;
    };
    const size_t k1 = N + 1;
    const size_t sbytes = k1 * k1 * p->P * p->rsize;
    const size_t w1 = (size_t)N * N * p->P * csize, w2 = 2 * w1;
    DevBuf bS, bW1, bW2, bt1, bt2, berr;
    if ((st = alloc_or_nomem(berr, 16)) != FSP_OK) return fail(st);
    p->err = static_cast<unsigned *>(berr.release());
    if (cudaMemsetAsync(p->err, 0, 16, s) != cudaSuccess) return fail(FSP_ECUDA);
    if ((st = alloc_or_nomem(bS, sbytes)) != FSP_OK) return fail(st);
    if (with_workspace && (st = alloc_or_nomem(bW1, w1)) != FSP_OK) return fail(st);
    if (with_workspace && (st = alloc_or_nomem(bW2, w2)) != FSP_OK) return fail(st);
    if ((st = alloc_or_nomem(bt1, csize * N)) != FSP_OK) return fail(st);
    // the cubic FP32 P3's stage twiddle tables follow the 2N roots
    const int tt_len = p->fast && dtype == FSP_F32_MIXED ? fast::p3_table_len<float>(N) : 0;
    if ((st = alloc_or_nomem(bt2, csize * (2 * N + tt_len))) != FSP_OK) return fail(st);
    p->S = bS.release(), p->W1 = bW1.release(), p->W2 = bW2.release();
    p->tw_n = bt1.release(), p->tw_2n = bt2.release();
    p->bytes = sbytes + (with_workspace ? w1 + w2 : 0) + csize * (3 * N + tt_len);
    cudaError_t e;
    if (dtype == FSP_F64) {
        e = launch_roots<double>(p->tw_n, N, s);
        if (e == cudaSuccess) e = launch_roots<double>(p->tw_2n, 2 * N, s);
    } else if (dtype == FSP_F64_DF) {
        e = launch_roots<df>(p->tw_n, N, s);
        if (e == cudaSuccess) e = launch_roots<df>(p->tw_2n, 2 * N, s);
    } else {
        e = launch_roots<float>(p->tw_n, N, s);
        if (e == cudaSuccess) e = launch_roots<float>(p->tw_2n, 2 * N, s);
        if (e == cudaSuccess && tt_len) e = fast::p3_table_fill<float>(N, p->tw_2n, s);
    }
    if (e != cudaSuccess) return fail(FSP_ECUDA);

    {  // plan-time spectrum, FP64 throughout
        Temps tmp, tw;
        DevBuf Td;
        if ((st = alloc_or_nomem(Td, sizeof(double) * k1 * k1 * k1)) != FSP_OK) return fail(st);
        const double hh = p->h;
        double scale = hh * hh * hh / ((2.0 * N) * (2.0 * N) * (2.0 * N));
        if (s_host) {  // a stored spectrum: upload it as it is
            if (cudaMemcpyAsync(Td.p, s_host, sizeof(double) * k1 * k1 * k1, cudaMemcpyHostToDevice, s) !=
                cudaSuccess)
                return fail(FSP_ECUDA);
            scale = 1.0;
        } else {
            if ((st = enqueue_kernel_T(N, L, algo, (double *)Td.p, s, tmp)) != FSP_OK) return fail(st);
            if ((st = enqueue_dct_spectrum(N, (double *)Td.p, s, tw)) != FSP_OK) return fail(st);
        }
        if (dtype == FSP_F64_DF) {
            double mx = 0;
            if ((st = abs_max((const double *)Td.p, (long long)(k1 * k1 * k1), s, &mx)) != FSP_OK) return fail(st);
            mx *= std::fabs(scale);
            if (!(mx >= kDfMinS && mx <= kDfMaxS)) return fail(FSP_EUNSUPPORTED);
        }
        e = dtype == FSP_F64      ? launch_store_S<double>((double *)Td.p, p->S, N, p->P, scale, s)
            : dtype == FSP_F64_DF ? launch_store_S<df>((double *)Td.p, p->S, N, p->P, scale, s)
                                  : launch_store_S<float>((double *)Td.p, p->S, N, p->P, scale, s);
        if (e != cudaSuccess) return fail(FSP_ECUDA);
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(FSP_ECUDA);
    }
    p->precompute_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    p->magic = kMagic;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_plans.insert(p);
    }
    *out = p;
    return FSP_OK;
}
}  // namespace

namespace fsp {
namespace internal {

fsp_status spectrum_plan_create(fsp_plan **out, int N, double L, fsp_algo algo, fsp_dtype dtype, cudaStream_t s) {
    return plan_create_impl(out, N, L, L / N, algo, dtype, reinterpret_cast<fsp_stream>(s), false);
}

bool plan_view(const fsp_plan *p, PlanView *v) {
    if (!plan_live(p) || !v || p->aniso) return false;
    v->N = p->N, v->P = p->P, v->device = p->device, v->dtype = p->dtype, v->rsize = p->rsize;
    v->S = p->S, v->tw_n = p->tw_n, v->tw_2n = p->tw_2n, v->row = p->row, v->col = p->col;
    return true;
}

}  // namespace internal
}  // namespace fsp

extern "C" {

fsp_status fsp_plan_create(fsp_plan **out, int N, double L, double h, fsp_algo algo, fsp_dtype dtype,
                           fsp_stream stream) {
    return plan_create_impl(out, N, L, h, algo, dtype, stream, true);
}

fsp_status fsp_plan_create_from_spectrum(fsp_plan **out, int N, double L, fsp_algo algo, fsp_dtype dtype,
                                         const double *s_host, fsp_stream stream) {
    if (!out) return FSP_EINVAL;
    *out = nullptr;
    if (!s_host) return FSP_EINVAL;
    if (N >= 2 && N <= kMaxN) {  // every value finite (a truncated or corrupt file shows here first)
        const size_t tot = (size_t)(N + 1) * (N + 1) * (N + 1);
        for (size_t i = 0; i < tot; ++i)
            if (!std::isfinite(s_host[i])) return FSP_EINVAL;
    }
    return plan_create_impl(out, N, L, L / N, algo, dtype, stream, true, s_host);
}

fsp_status fsp_plan_create_aniso(fsp_plan **out, int nx, int ny, int nz, double hx, double hy, double hz,
                                 fsp_algo algo, fsp_dtype dtype, fsp_stream stream) {
    if (!out) return FSP_EINVAL;
    *out = nullptr;
    const int nn[3] = {nx, ny, nz};
    const double hh[3] = {hx, hy, hz};
    if (algo != FSP_HE && algo != FSP_VG && algo != FSP_VG_DCT) return FSP_EINVAL;
    if (dtype != FSP_F64 && dtype != FSP_F32_MIXED && dtype != FSP_F64_DF) return FSP_EINVAL;
    for (int a = 0; a < 3; ++a) {
        if (nn[a] < 2 || !(hh[a] > 0.0) || !std::isfinite(hh[a])) return FSP_EINVAL;
        if (nn[a] > kMaxN || !is_235_smooth(2LL * nn[a])) return FSP_EUNSUPPORTED;
        if (algo == FSP_VG && !is_235_smooth(4LL * nn[a])) return FSP_EUNSUPPORTED;
    }
    if (nx == ny && ny == nz && hx == hy && hy == hz)  // a cube: the cubic plan and its kernels
        return plan_create_impl(out, nx, nx * hx, hx, algo, dtype, stream, true);
    // the specialised kernels when every n_a has them (and FSP_GENERIC_ONLY is not 1)
    bool fast_ok;
    {
        const char *g = std::getenv("FSP_GENERIC_ONLY");
        const bool generic_only = g && g[0] == '1';
        // rows of n_x; column passes of 2 n_y and 2 n_z
        fast_ok = dtype == FSP_F64 ? fast::has<double>(nx) && fast::has_col_rg<double>(2 * ny) &&
                                         fast::has_col_rg<double>(2 * nz)
                  : dtype == FSP_F64_DF ? fast::has<df>(nx) && fast::has_col_rg<df>(2 * ny) &&
                                              fast::has_col_rg<df>(2 * nz)
                                        : fast::has<float>(nx) && fast::has_col_rg<float>(2 * ny) &&
                                              fast::has_col_rg<float>(2 * nz);
        fast_ok = fast_ok && ny >= 32 && nz >= 32;
        if (dtype != FSP_F64_DF) fast_ok = fast_ok && !generic_only;
    }
    if (dtype == FSP_F64_DF && !fast_ok) return FSP_EUNSUPPORTED;  // double-float: specialised kernels only
    if (algo != FSP_HE) {
        // the (4 n_a h_a) periodisation of the truncated kernel must not reach
        // the box: 3 min_a L_a >= L_t = alpha |(L_x, L_y, L_z)|
        const double Lb[3] = {nx * hx, ny * hy, nz * hz};
        const double Lt = kAlpha * std::sqrt(Lb[0] * Lb[0] + Lb[1] * Lb[1] + Lb[2] * Lb[2]);
        if (3.0 * std::min(Lb[0], std::min(Lb[1], Lb[2])) < Lt) return FSP_EUNSUPPORTED;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();
    fsp_plan *p = new fsp_plan();
    p->guarded = bounds_check_requested();
    GuardScope guard_scope(p->guarded);
    p->aniso = true;
    p->fast = fast_ok;
    for (int a = 0; a < 3; ++a) p->n3[a] = nn[a], p->h3[a] = hh[a];
    p->N = nx, p->L = nx * hx, p->h = hx, p->algo = algo, p->dtype = dtype;
    p->rsize = dtype == FSP_F32_MIXED ? 4 : 8;
    p->P = ((nx + 1) + 15) / 16 * 16;
    const size_t csize = 2 * p->rsize;
    const int lg = dtype == FSP_F32_MIXED ? 4 : 3;
    if (!make_cfg(nx, nx + 1, csize, lg, p->row) || !make_cfg(2 * ny, 2 * ny, csize, lg, p->col) ||
        !make_cfg(2 * nz, 2 * nz, csize, lg, p->colz)) {
        delete p;
        return FSP_EUNSUPPORTED;
    }
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return FSP_ECUDA;
    }
    auto fail = [&](fsp_status e) {
        cudaStreamSynchronize(s);
        plan_free(p);
        return e;
    };
    const size_t sbytes = (size_t)(nz + 1) * (ny + 1) * p->P * p->rsize;
    const size_t w1 = (size_t)nz * ny * p->P * csize, w2 = 2 * w1;
    fsp_status st;
    DevBuf bS, bW1, bW2, b1, b2, by, bz;
    if ((st = alloc_or_nomem(bS, sbytes)) != FSP_OK) return fail(st);
    if ((st = alloc_or_nomem(bW1, w1)) != FSP_OK) return fail(st);
    if ((st = alloc_or_nomem(bW2, w2)) != FSP_OK) return fail(st);
    if ((st = alloc_or_nomem(b1, csize * nx)) != FSP_OK) return fail(st);
    if ((st = alloc_or_nomem(b2, csize * 2 * nx)) != FSP_OK) return fail(st);
    if ((st = alloc_or_nomem(by, csize * 2 * ny)) != FSP_OK) return fail(st);
    if ((st = alloc_or_nomem(bz, csize * 2 * nz)) != FSP_OK) return fail(st);
    p->S = bS.release(), p->W1 = bW1.release(), p->W2 = bW2.release();
    p->tw_n = b1.release(), p->tw_2n = b2.release(), p->tw_y = by.release(), p->tw_z = bz.release();
    p->bytes = sbytes + w1 + w2 + csize * (3 * nx + 2 * ny + 2 * nz);
    cudaError_t e;
    if (dtype == FSP_F64) {
        e = launch_roots<double>(p->tw_n, nx, s);
        if (e == cudaSuccess) e = launch_roots<double>(p->tw_2n, 2 * nx, s);
        if (e == cudaSuccess) e = launch_roots<double>(p->tw_y, 2 * ny, s);
        if (e == cudaSuccess) e = launch_roots<double>(p->tw_z, 2 * nz, s);
    } else if (dtype == FSP_F64_DF) {
        e = launch_roots<df>(p->tw_n, nx, s);
        if (e == cudaSuccess) e = launch_roots<df>(p->tw_2n, 2 * nx, s);
        if (e == cudaSuccess) e = launch_roots<df>(p->tw_y, 2 * ny, s);
        if (e == cudaSuccess) e = launch_roots<df>(p->tw_z, 2 * nz, s);
    } else {
        e = launch_roots<float>(p->tw_n, nx, s);
        if (e == cudaSuccess) e = launch_roots<float>(p->tw_2n, 2 * nx, s);
        if (e == cudaSuccess) e = launch_roots<float>(p->tw_y, 2 * ny, s);
        if (e == cudaSuccess) e = launch_roots<float>(p->tw_z, 2 * nz, s);
    }
    if (e != cudaSuccess) return fail(FSP_ECUDA);
    {  // plan-time spectrum, FP64 throughout
        Temps tmp, tw;
        DevBuf Td;
        const long long rows = (long long)(ny + 1) * (nz + 1);
        if ((st = alloc_or_nomem(Td, sizeof(double) * (size_t)(nx + 1) * rows)) != FSP_OK) return fail(st);
        if ((st = enqueue_kernel_T3(nn, hh, algo, (double *)Td.p, s, tmp)) != FSP_OK) return fail(st);
        if ((st = enqueue_trig_spectrum3(nn, -1, (double *)Td.p, s, tw)) != FSP_OK) return fail(st);
        const double scale = hx * hy * hz / ((2.0 * nx) * (2.0 * ny) * (2.0 * nz));
        if (dtype == FSP_F64_DF) {
            double mx = 0;
            if ((st = abs_max((const double *)Td.p, (long long)(nx + 1) * rows, s, &mx)) != FSP_OK) return fail(st);
            mx *= std::fabs(scale);
            if (!(mx >= kDfMinS && mx <= kDfMaxS)) return fail(FSP_EUNSUPPORTED);
        }
        e = dtype == FSP_F64      ? launch_store_S3<double>((double *)Td.p, p->S, nx + 1, rows, p->P, scale, s)
            : dtype == FSP_F64_DF ? launch_store_S3<df>((double *)Td.p, p->S, nx + 1, rows, p->P, scale, s)
                                  : launch_store_S3<float>((double *)Td.p, p->S, nx + 1, rows, p->P, scale, s);
        if (e != cudaSuccess) return fail(FSP_ECUDA);
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(FSP_ECUDA);
    }
    p->precompute_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    p->magic = kMagic;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_plans.insert(p);
    }
    *out = p;
    return FSP_OK;
}

fsp_status fsp_solve(fsp_plan *plan, const void *rho, void *phi, fsp_stream stream) {
    if (!plan_live(plan)) return FSP_EINVAL;
    if (!rho || !phi || !aligned16(rho) || !aligned16(phi)) return FSP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    if (dev != plan->device) return FSP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!plan->W1) return FSP_EINVAL;  // a spectrum-only plan (server cache) has no workspace
    const cudaError_t e = enqueue_solve_ws(plan, rho, phi, plan->W1, plan->W2, s);
    return cuda_status(e);
}

fsp_status fsp_plan_field_init(fsp_plan *plan, fsp_stream stream) {
    if (!plan_live(plan)) return FSP_EINVAL;
    if (!plan->W1) return FSP_EINVAL;
    if (plan->W3) return FSP_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    if (dev != plan->device) return FSP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();
    GuardScope guard_scope(plan->guarded);
    const int N = plan->N;
    // the box: cubic, or the plan's non-cubic sizes and spacings
    const int nn[3] = {plan->aniso ? plan->n3[0] : N, plan->aniso ? plan->n3[1] : N, plan->aniso ? plan->n3[2] : N};
    const double hb[3] = {plan->aniso ? plan->h3[0] : plan->h, plan->aniso ? plan->h3[1] : plan->h,
                          plan->aniso ? plan->h3[2] : plan->h};
    const int kx = nn[0] + 1;
    const long long rows = (long long)(nn[1] + 1) * (nn[2] + 1);
    const size_t sbytes = (size_t)rows * plan->P * plan->rsize;
    const size_t w2 = 2 * (size_t)nn[2] * nn[1] * plan->P * 2 * plan->rsize;
    DevBuf bs[3], bw;
    fsp_status st;
    for (auto &b : bs)
        if ((st = alloc_or_nomem(b, sbytes)) != FSP_OK) return st;
    if ((st = alloc_or_nomem(bw, w2)) != FSP_OK) return st;
    const double scale = hb[0] * hb[1] * hb[2] / ((2.0 * nn[0]) * (2.0 * nn[1]) * (2.0 * nn[2]));
    for (int axis = 0; axis < 3; ++axis) {
        // plan-time field spectrum S_a = h^3 / (2N)^3 * DST/DCT of F_a, FP64,
        // rounded to the plan's type; each component's temporaries live
        // until its work has finished
        Temps tmp, tw;
        DevBuf Fd;
        if ((st = alloc_or_nomem(Fd, sizeof(double) * (size_t)kx * rows)) != FSP_OK) return st;
        st = plan->aniso ? enqueue_field_kernel3(nn, hb, plan->algo, axis, (double *)Fd.p, s, tmp)
                         : enqueue_field_kernel(N, plan->L, plan->algo, axis, (double *)Fd.p, s, tmp);
        if (st != FSP_OK) {
            cudaStreamSynchronize(s);
            return st;
        }
        if ((st = enqueue_trig_spectrum3(nn, axis, (double *)Fd.p, s, tw)) != FSP_OK) {
            cudaStreamSynchronize(s);
            return st;
        }
        cudaError_t e =
            plan->dtype == FSP_F64      ? launch_store_S3<double>((double *)Fd.p, bs[axis].p, kx, rows, plan->P, scale, s)
            : plan->dtype == FSP_F64_DF ? launch_store_S3<df>((double *)Fd.p, bs[axis].p, kx, rows, plan->P, scale, s)
                                        : launch_store_S3<float>((double *)Fd.p, bs[axis].p, kx, rows, plan->P, scale, s);
        if (cudaStreamSynchronize(s) != cudaSuccess || e != cudaSuccess) return FSP_ECUDA;
    }
    for (int axis = 0; axis < 3; ++axis) plan->SF[axis] = bs[axis].release();
    plan->W3 = bw.release();
    plan->bytes += 3 * sbytes + w2;
    plan->precompute_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return FSP_OK;
}

fsp_status fsp_solve_field(fsp_plan *plan, const void *rho, void *phi, void *ex, void *ey, void *ez,
                           fsp_stream stream) {
    if (!plan_live(plan)) return FSP_EINVAL;
    if (!rho || !ex || !ey || !ez || !aligned16(rho) || !aligned16(ex) || !aligned16(ey) || !aligned16(ez))
        return FSP_EINVAL;
    if (phi && !aligned16(phi)) return FSP_EINVAL;
    if (ex == ey || ey == ez || ex == ez || (phi && (phi == ex || phi == ey || phi == ez))) return FSP_EINVAL;
    if (!plan->W1) return FSP_EINVAL;
    fsp_status st = fsp_plan_field_init(plan, stream);
    if (st != FSP_OK) return st;
    void *const out[4] = {ex, ey, ez, phi};
    return cuda_status(enqueue_field(plan, rho, out, reinterpret_cast<cudaStream_t>(stream)));
}

fsp_status fsp_solve_host(fsp_plan *plan, const void *rho_host, void *phi_host, fsp_stream stream) {
    if (!plan_live(plan)) return FSP_EINVAL;
    if (!rho_host || !phi_host) return FSP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    if (dev != plan->device) return FSP_EINVAL;
    const size_t bytes = plan_points(plan) * plan->rsize;
    if (!plan->stage_rho) {
        DevBuf a, b;
        fsp_status st;
        if ((st = alloc_or_nomem(a, bytes)) != FSP_OK) return st;
        if ((st = alloc_or_nomem(b, bytes)) != FSP_OK) return st;
        plan->stage_rho = a.release();
        plan->stage_phi = b.release();
        plan->bytes += 2 * bytes;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    FSP_TRY_CUDA(cudaMemcpyAsync(plan->stage_rho, rho_host, bytes, cudaMemcpyHostToDevice, s));
    fsp_status st = fsp_solve(plan, plan->stage_rho, plan->stage_phi, stream);
    if (st != FSP_OK) return st;
    FSP_TRY_CUDA(cudaMemcpyAsync(phi_host, plan->stage_phi, bytes, cudaMemcpyDeviceToHost, s));
    return cuda_status(cudaStreamSynchronize(s));
}

fsp_status fsp_solve_host_many(fsp_plan *plan, const void *const *rho_host, void *const *phi_host, int count,
                               fsp_stream stream) {
    if (!plan_live(plan) || count < 0 || (count > 0 && (!rho_host || !phi_host))) return FSP_EINVAL;
    if (!plan->W1) return FSP_EINVAL;
    for (int i = 0; i < count; ++i)
        if (!rho_host[i] || !phi_host[i]) return FSP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    if (dev != plan->device) return FSP_EINVAL;
    if (count == 0) return FSP_OK;
    const size_t bytes = plan_points(plan) * plan->rsize;
    if (!plan->pipe_h2d) {  // first use: staging slots, copy streams, events
        GuardScope guard_scope(plan->guarded);
        DevBuf a[kPipeSlots], b[kPipeSlots];
        fsp_status st;
        for (int i = 0; i < kPipeSlots; ++i)
            if ((st = alloc_or_nomem(a[i], bytes)) != FSP_OK || (st = alloc_or_nomem(b[i], bytes)) != FSP_OK)
                return st;
        cudaStream_t h2d = nullptr, d2h = nullptr;
        cudaEvent_t ev[3 * kPipeSlots] = {};
        bool ok = cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 3 * kPipeSlots && ok; ++i)
            ok = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            for (cudaStream_t q : {h2d, d2h})
                if (q) cudaStreamDestroy(q);
            for (cudaEvent_t q : ev)
                if (q) cudaEventDestroy(q);
            return FSP_ECUDA;
        }
        for (int i = 0; i < kPipeSlots; ++i) {
            plan->pipe_rho[i] = a[i].release(), plan->pipe_phi[i] = b[i].release();
            plan->ev_in[i] = ev[i], plan->ev_comp[i] = ev[kPipeSlots + i], plan->ev_out[i] = ev[2 * kPipeSlots + i];
        }
        plan->pipe_h2d = h2d, plan->pipe_d2h = d2h;
        plan->bytes += 2 * kPipeSlots * bytes;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // all three streams start after prior work on `stream`
    cudaError_t e = cudaEventRecord(plan->ev_out[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->pipe_h2d, plan->ev_out[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->pipe_d2h, plan->ev_out[0], 0);
    for (int k = 0; k < kPipeSlots && e == cudaSuccess; ++k) {
        e = cudaEventRecord(plan->ev_comp[k], s);
        if (e == cudaSuccess && k > 0) e = cudaEventRecord(plan->ev_out[k], s);
    }
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        const int k = i % kPipeSlots;
        // copy in: slot k's source buffer is free once the solve of i-3 ran
        e = cudaStreamWaitEvent(plan->pipe_h2d, plan->ev_comp[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(plan->pipe_rho[k], rho_host[i], bytes, cudaMemcpyHostToDevice, plan->pipe_h2d);
        if (e == cudaSuccess) e = cudaEventRecord(plan->ev_in[k], plan->pipe_h2d);
        // solve: after its copy-in and after the copy-out of i-3 freed slot k
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->ev_in[k], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->ev_out[k], 0);
        if (e == cudaSuccess) e = enqueue_solve_ws(plan, plan->pipe_rho[k], plan->pipe_phi[k], plan->W1, plan->W2, s);
        if (e == cudaSuccess) e = cudaEventRecord(plan->ev_comp[k], s);
        // copy out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->pipe_d2h, plan->ev_comp[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(phi_host[i], plan->pipe_phi[k], bytes, cudaMemcpyDeviceToHost, plan->pipe_d2h);
        if (e == cudaSuccess) e = cudaEventRecord(plan->ev_out[k], plan->pipe_d2h);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(plan->pipe_d2h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(e);
}

fsp_status fsp_plan_sync(fsp_plan *plan, fsp_stream stream) {
    if (!plan_live(plan)) return FSP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return FSP_ECUDA;
    if (!plan->err) return FSP_OK;
    // a bounded device-side wait that expired since the last check
    unsigned flags = 0;
    if (cudaMemcpyAsync(&flags, plan->err, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FSP_ECUDA;
    if (flags == 0) return FSP_OK;
    if (cudaMemsetAsync(plan->err, 0, sizeof(flags), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return FSP_ECUDA;
    return FSP_ETIMEOUT;
}

fsp_status fsp_plan_destroy(fsp_plan *plan) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!plan || !g_plans.count(plan)) return FSP_EINVAL;
        g_plans.erase(plan);
    }
    cudaError_t e = cudaDeviceSynchronize();
    plan_free(plan);
    return cuda_status(e);
}

fsp_status fsp_plan_set_timing(fsp_plan *plan, void *const *events, int nevents) {
    if (!plan_live(plan)) return FSP_EINVAL;
    if (nevents == 0) {
        plan->timing = false;
        return FSP_OK;
    }
    if (nevents != 6 || !events) return FSP_EINVAL;
    for (int i = 0; i < 6; ++i)
        if (!events[i]) return FSP_EINVAL;
    for (int i = 0; i < 6; ++i) plan->ev[i] = reinterpret_cast<cudaEvent_t>(events[i]);
    plan->timing = true;
    return FSP_OK;
}

fsp_status fsp_plan_set_wait_timeout(fsp_plan *plan, double ms) {
    if (!plan_live(plan) || !(ms > 0.0) || !(ms < 1e9)) return FSP_EINVAL;
    plan->wait_timeout_ns = (unsigned long long)(ms * 1e6);
    return FSP_OK;
}

fsp_status fsp_plan_inject_stall(fsp_plan *plan) {
    if (!plan_live(plan)) return FSP_EINVAL;
    if (!plan->p3_tma) return FSP_EUNSUPPORTED;
    plan->inject_tx.store(16);
    return FSP_OK;
}

int fsp_plan_uses_fast_path(const fsp_plan *plan) { return plan_live(plan) ? (plan->fast ? 1 : 0) : -1; }

fsp_status fsp_plan_check_bounds(const fsp_plan *plan, unsigned long long *bad_bytes) {
    if (!plan_live(plan) || !bad_bytes) return FSP_EINVAL;
    *bad_bytes = 0;
    if (!plan->guarded) return FSP_EUNSUPPORTED;
    if (cudaDeviceSynchronize() != cudaSuccess) return FSP_ECUDA;
    const fsp_plan *p = plan;
    const void *bufs[] = {p->S,          p->W1,          p->W2,          p->tw_n,        p->tw_2n,
                          p->stage_rho,  p->stage_phi,   p->pipe_rho[0], p->pipe_rho[1], p->pipe_rho[2],
                          p->pipe_phi[0], p->pipe_phi[1], p->pipe_phi[2], p->SF[0],      p->SF[1],
                          p->SF[2],      p->W3,          p->tw_y,        p->tw_z,        (const void *)p->err};
    static_assert(kPipeSlots == 3, "the list above names every staging slot");
    for (const void *q : bufs) {
        if (!q) continue;
        Guarded g{nullptr, 0};
        {
            std::lock_guard<std::mutex> lk(g_guard_mu);
            auto it = g_guarded.find(q);
            if (it != g_guarded.end()) g = it->second;
        }
        if (!g.base) continue;
        const unsigned long long b = guard_bad(q, g);
        if (b == ~0ull) return FSP_ENOMEM;
        *bad_bytes += b;
    }
    return FSP_OK;
}

unsigned long long fsp_bounds_freed_bad(void) { return g_guard_freed_bad.load(); }

int fsp_plan_launches(const fsp_plan *plan) { return plan_live(plan) ? (plan->plane ? 3 : 5) : -1; }

size_t fsp_plan_bytes(const fsp_plan *plan) { return plan_live(plan) ? plan->bytes : 0; }

double fsp_plan_precompute_ms(const fsp_plan *plan) { return plan_live(plan) ? plan->precompute_ms : -1.0; }

fsp_status fsp_plan_spectrum(const fsp_plan *plan, double *s_host) {
    if (!plan_live(plan) || !s_host) return FSP_EINVAL;
    if (plan->aniso) {
        const int kx = plan->n3[0] + 1;
        const long long rows = (long long)(plan->n3[1] + 1) * (plan->n3[2] + 1);
        const size_t tot = (size_t)kx * rows;
        DevBuf d;
        fsp_status st = alloc_or_nomem(d, sizeof(double) * tot);
        if (st != FSP_OK) return st;
        cudaError_t e = plan->dtype == FSP_F64      ? launch_load_S3<double>(plan->S, (double *)d.p, kx, rows, plan->P, 0)
                        : plan->dtype == FSP_F64_DF ? launch_load_S3<df>(plan->S, (double *)d.p, kx, rows, plan->P, 0)
                                                    : launch_load_S3<float>(plan->S, (double *)d.p, kx, rows, plan->P, 0);
        if (e != cudaSuccess) return FSP_ECUDA;
        return cuda_status(cudaMemcpy(s_host, d.p, sizeof(double) * tot, cudaMemcpyDeviceToHost));
    }
    const size_t k1 = plan->N + 1, tot = k1 * k1 * k1;
    DevBuf d;
    fsp_status st = alloc_or_nomem(d, sizeof(double) * tot);
    if (st != FSP_OK) return st;
    cudaError_t e = plan->dtype == FSP_F64      ? launch_load_S<double>(plan->S, (double *)d.p, plan->N, plan->P, 0)
                    : plan->dtype == FSP_F64_DF ? launch_load_S<df>(plan->S, (double *)d.p, plan->N, plan->P, 0)
                                                : launch_load_S<float>(plan->S, (double *)d.p, plan->N, plan->P, 0);
    if (e != cudaSuccess) return FSP_ECUDA;
    return cuda_status(cudaMemcpy(s_host, d.p, sizeof(double) * tot, cudaMemcpyDeviceToHost));
}

fsp_status fsp_kernel_T(int N, double L, fsp_algo algo, double *t_dev, fsp_stream stream) {
    fsp_status st = validate_size(N, L, algo);
    if (st != FSP_OK) return st;
    if (!t_dev || !aligned16(t_dev)) return FSP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Temps tmp;
    st = enqueue_kernel_T(N, L, algo, t_dev, s, tmp);
    cudaError_t e = cudaStreamSynchronize(s);
    if (st != FSP_OK) return st;
    return cuda_status(e);
}

fsp_status fsp_fft_c2c(int n, int count, fsp_dtype dtype, int sign, const void *in, void *out, fsp_stream stream) {
    if (n < 1 || n > 4096 || count < 0 || (sign != -1 && sign != 1)) return FSP_EINVAL;
    if (dtype != FSP_F64 && dtype != FSP_F32_MIXED) return FSP_EINVAL;
    if (!is_235_smooth(n)) return FSP_EUNSUPPORTED;
    if (count == 0) return FSP_OK;
    if (!in || !out || !aligned16(in) || !aligned16(out)) return FSP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    const size_t csize = dtype == FSP_F64 ? 16 : 8;
    TileCfg c;
    if (!make_cfg(n, n, csize, dtype == FSP_F64 ? 3 : 4, c)) return FSP_EUNSUPPORTED;
    // roots tables are cached per (device, dtype, n) for the life of the process
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, void *> cache;
    void *tw = nullptr;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto key = std::make_tuple(dev, (int)dtype, n);
        auto it = cache.find(key);
        if (it != cache.end()) {
            tw = it->second;
        } else {
            DevBuf b;
            fsp_status st = alloc_or_nomem(b, csize * n);
            if (st != FSP_OK) return st;
            cudaError_t e = dtype == FSP_F64 ? launch_roots<double>(b.p, n, s) : launch_roots<float>(b.p, n, s);
            if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return FSP_ECUDA;
            tw = b.release();
            cache[key] = tw;
        }
    }
    LinesArgs a{};
    a.in = in, a.out = out, a.tw = tw, a.st = c.st, a.tpl = c.tpl, a.lgL = c.lgL;
    a.in_pos = a.out_pos = 1, a.in_line = a.out_line = n, a.in_batch = a.out_batch = 0;
    a.n_in = a.n_out = n, a.nlines = count, a.nbatch = 1;
    cudaError_t e;
    if (dtype == FSP_F64)
        e = sign < 0 ? launch_lines<double, IN_CPLX, OUT_CPLX, M_FWD>(a, s)
                     : launch_lines<double, IN_CPLX, OUT_CPLX, M_INV>(a, s);
    else
        e = sign < 0 ? launch_lines<float, IN_CPLX, OUT_CPLX, M_FWD>(a, s)
                     : launch_lines<float, IN_CPLX, OUT_CPLX, M_INV>(a, s);
    return cuda_status(e);
}

}  // extern "C"

// ------------------------------------------------------------- batches --
struct fsp_batch {
    uint64_t magic = 0;
    int device = 0, count = 0;
    fsp_dtype dtype = FSP_F64;
    std::vector<fsp_plan *> plans;
    std::vector<const void *> rho;
    std::vector<void *> phi;
    std::map<int, std::pair<int, int>> shape;  // per N: (lgL_row, lgL_col) of its tiles
    std::vector<BatchSolve> solves;
    std::vector<BatchSeg> segs;
    int total = 0;
    BatchSolve *d_solves = nullptr;
    BatchSeg *d_segs = nullptr;
    BatchCtl *d_ctl = nullptr;
    size_t ctl_bytes = 0;
    BatchLaunch launch{};
    double timeout_ms = 1000.0;
    int form = 0;  // 0: one persistent kernel; 1: the solves' own launches on several streams
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr uint64_t kBatchMagic = 0x46535042'41544348ULL;  // "FSPBATCH"
std::unordered_set<const fsp_batch *> g_batches;

bool batch_live(const fsp_batch *b) {
    std::lock_guard<std::mutex> lk(g_mu);
    return b && g_batches.count(b) && b->magic == kBatchMagic;
}

void batch_free(fsp_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void *q : {(void *)b->d_solves, (void *)b->d_segs, (void *)b->d_ctl})
        if (q) dev_free(q);
    b->magic = 0;
    delete b;
}

// Fill the device-side descriptor of one solve from its plan (generic engine
// tile shapes; workspace reads through L2).
BatchSolve batch_solve_of(const fsp_plan *p, const void *rho, void *phi, const TileCfg &row, const TileCfg &col) {
    const int N = p->N;
    const long long P = p->P;
    BatchSolve b{};
    RowsArgs r{};
    r.c = p->W1, r.x_row = N, r.c_row = P, r.N = N, r.nrows = N * N;
    r.lgL = row.lgL, r.tpl = row.tpl, r.st = row.st, r.tw = p->tw_n, r.tw2 = p->tw_2n;
    b.r1 = r, b.r5 = r;
    b.r1.x = rho;
    b.r5.x = phi;
    LinesArgs a{};
    a.st = col.st, a.tpl = col.tpl, a.lgL = col.lgL, a.tw = p->tw_2n;
    a.nlines = N + 1;
    LinesArgs c2 = a;
    c2.in = p->W1, c2.out = p->W2;
    c2.in_pos = P, c2.in_line = 1, c2.in_batch = (long long)N * P;
    c2.out_pos = P, c2.out_line = 1, c2.out_batch = 2LL * N * P;
    c2.n_in = N, c2.n_out = 2 * N, c2.nbatch = N;
    LinesArgs c3 = a;
    c3.in = c3.out = p->W2;
    c3.in_pos = c3.out_pos = 2LL * N * P, c3.in_line = c3.out_line = 1, c3.in_batch = c3.out_batch = P;
    c3.n_in = N, c3.n_out = N, c3.nbatch = 2 * N;
    c3.S = p->S, c3.s_pos = (long long)(N + 1) * P, c3.s_batch = P, c3.half = N;
    LinesArgs c4 = a;
    c4.in = p->W2, c4.out = p->W1;
    c4.in_pos = P, c4.in_line = 1, c4.in_batch = 2LL * N * P;
    c4.out_pos = P, c4.out_line = 1, c4.out_batch = (long long)N * P;
    c4.n_in = 2 * N, c4.n_out = N, c4.nbatch = N;
    b.c2 = c2, b.c3 = c3, b.c4 = c4;
    b.ntx = (N + 1 + (1 << col.lgL) - 1) >> col.lgL;
    const int ntr = (N * N + (1 << row.lgL) - 1) >> row.lgL;
    b.ntiles[0] = ntr, b.ntiles[1] = b.ntx * N, b.ntiles[2] = b.ntx * 2 * N, b.ntiles[3] = b.ntx * N, b.ntiles[4] = ntr;
    return b;
}

fsp_status batch_build_graph(fsp_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec), b->exec = nullptr;
    if (b->graph) cudaGraphDestroy(b->graph), b->graph = nullptr;
    b->launch.timeout_ns = (unsigned long long)(b->timeout_ms * 1e6);
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return FSP_ECUDA;
    // form 1: kStreams capture streams forked from cs; a plan's solves stay on
    // one stream (they share its workspace), plans are dealt round-robin
    constexpr int kStreams = 8;
    cudaStream_t fs[kStreams] = {};
    cudaEvent_t fev[kStreams + 1] = {};
    cudaError_t e = cudaSuccess;
    if (b->form == 1) {
        for (int i = 0; i < kStreams && e == cudaSuccess; ++i)
            e = cudaStreamCreateWithFlags(&fs[i], cudaStreamNonBlocking);
        for (int i = 0; i <= kStreams && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&fev[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemsetAsync(b->d_ctl, 0, b->ctl_bytes, cs);
        cudaError_t e2 = e1;
        if (e1 == cudaSuccess && b->form == 0) {
            e2 = b->dtype == FSP_F64 ? launch_batch_kernel<double>(b->launch, cs)
                                     : launch_batch_kernel<float>(b->launch, cs);
        } else if (e1 == cudaSuccess) {
            e2 = cudaEventRecord(fev[kStreams], cs);
            for (int i = 0; i < kStreams && e2 == cudaSuccess; ++i) e2 = cudaStreamWaitEvent(fs[i], fev[kStreams], 0);
            std::map<const fsp_plan *, int> lane;
            for (int i = 0; i < b->count && e2 == cudaSuccess; ++i) {
                auto it = lane.find(b->plans[i]);
                if (it == lane.end()) it = lane.emplace(b->plans[i], (int)lane.size() % kStreams).first;
                const fsp_plan *p = b->plans[i];
                e2 = enqueue_solve_ws(p, b->rho[i], b->phi[i], p->W1, p->W2, fs[it->second]);
            }
            for (int i = 0; i < kStreams && e2 == cudaSuccess; ++i) {
                e2 = cudaEventRecord(fev[i], fs[i]);
                if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(cs, fev[i], 0);
            }
        }
        e = cudaStreamEndCapture(cs, &b->graph);
        if (e == cudaSuccess) e = e2;
    }
    for (int i = 0; i < kStreams; ++i) {
        if (fs[i]) cudaStreamDestroy(fs[i]);
        if (fev[i]) cudaEventDestroy(fev[i]);
    }
    if (fev[kStreams]) cudaEventDestroy(fev[kStreams]);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    return cuda_status(e);
}

}  // namespace

namespace {

// Tile shapes a batch uses for one of its plans: the per-N override if set,
// else the plan's own generic-engine shapes.
void batch_tiles(const fsp_batch *b, const fsp_plan *p, TileCfg &row, TileCfg &col) {
    row = p->row, col = p->col;
    auto it = b->shape.find(p->N);
    if (it == b->shape.end()) return;
    const size_t csize = 2 * p->rsize;
    TileCfg r = row, c = col;
    if (choose_tile(p->N + 1, r.tpl, csize, it->second.first, r.lgL)) row = r;
    if (choose_tile(2 * p->N, c.tpl, csize, it->second.second, c.lgL)) col = c;
}

// (Re)build descriptors, work list, device arrays and graph of a batch.
fsp_status batch_build(fsp_batch *b, cudaStream_t s) {
    const int count = b->count;
    const size_t csize = 2 * b->plans[0]->rsize;
    b->solves.clear();
    b->segs.clear();
    int threads = 32;
    size_t smem = 0;
    for (int i = 0; i < count; ++i) {
        const fsp_plan *p = b->plans[i];
        TileCfg row, col;
        batch_tiles(b, p, row, col);
        b->solves.push_back(batch_solve_of(p, b->rho[i], b->phi[i], row, col));
        threads = std::max(threads, std::max((1 << row.lgL) * row.tpl, (1 << col.lgL) * col.tpl));
        smem = std::max(smem, std::max((size_t)(p->N + 1) * ((1 << row.lgL) + 1) * csize,
                                       (size_t)(2 * p->N) * ((1 << col.lgL) + 1) * csize));
    }
    threads = (threads + 31) / 32 * 32;
    // pass-major work list; within a pass, larger solves first
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->plans[x]->N > b->plans[y]->N; });
    int first = 0;
    for (int pass = 0; pass < 5; ++pass)
        for (int i : order) {
            BatchSeg g{};
            g.solve = i, g.pass = pass, g.first = first, g.ntiles = b->solves[i].ntiles[pass];
            g.need_prev = pass ? b->solves[i].ntiles[pass - 1] : 0;
            first += g.ntiles;
            b->segs.push_back(g);
        }
    b->total = first;
    for (void *q : {(void *)b->d_solves, (void *)b->d_segs, (void *)b->d_ctl})
        if (q) dev_free(q);
    b->d_solves = nullptr, b->d_segs = nullptr, b->d_ctl = nullptr;
    b->ctl_bytes = sizeof(BatchCtl) + sizeof(int) * (5 * (size_t)count);
    DevBuf ds, dg, dc;
    fsp_status st;
    if ((st = alloc_or_nomem(ds, sizeof(BatchSolve) * count)) != FSP_OK) return st;
    if ((st = alloc_or_nomem(dg, sizeof(BatchSeg) * b->segs.size())) != FSP_OK) return st;
    if ((st = alloc_or_nomem(dc, b->ctl_bytes)) != FSP_OK) return st;
    b->d_solves = (BatchSolve *)ds.release(), b->d_segs = (BatchSeg *)dg.release(), b->d_ctl = (BatchCtl *)dc.release();
    if (cudaMemcpyAsync(b->d_solves, b->solves.data(), sizeof(BatchSolve) * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(b->d_segs, b->segs.data(), sizeof(BatchSeg) * b->segs.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FSP_ECUDA;
    const int per_sm = b->dtype == FSP_F64 ? batch_blocks_per_sm<double>(threads, smem) : batch_blocks_per_sm<float>(threads, smem);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (per_sm < 1 || sms < 1) return FSP_EUNSUPPORTED;
    b->launch.solves = b->d_solves, b->launch.segs = b->d_segs, b->launch.nseg = (int)b->segs.size();
    b->launch.total = b->total, b->launch.ctl = b->d_ctl;
    b->launch.grid = (unsigned)std::min<long long>((long long)sms * per_sm, b->total);
    b->launch.threads = threads, b->launch.smem = smem;
    return batch_build_graph(b);
}

}  // namespace

extern "C" fsp_status fsp_batch_create(fsp_batch **out, fsp_plan *const *plans, const void *const *rho,
                                       void *const *phi, int count, fsp_stream stream) {
    if (!out) return FSP_EINVAL;
    *out = nullptr;
    if (count < 1 || !plans || !rho || !phi) return FSP_EINVAL;
    std::unordered_set<const fsp_plan *> seen;
    for (int i = 0; i < count; ++i) {
        if (!plan_live(plans[i]) || !seen.insert(plans[i]).second) return FSP_EINVAL;  // distinct live plans
        if (plans[i]->dtype != plans[0]->dtype || plans[i]->device != plans[0]->device) return FSP_EINVAL;
        if (plans[i]->dtype == FSP_F64_DF) return FSP_EUNSUPPORTED;  // batches use the generic engine
        if (plans[i]->aniso) return FSP_EUNSUPPORTED;                // and cubic boxes
        if (!rho[i] || !phi[i] || !aligned16(rho[i]) || !aligned16(phi[i])) return FSP_EINVAL;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    if (dev != plans[0]->device) return FSP_EINVAL;
    fsp_batch *b = new fsp_batch();
    b->device = dev, b->count = count, b->dtype = plans[0]->dtype;
    b->plans.assign(plans, plans + count);
    b->rho.assign(rho, rho + count);
    b->phi.assign(phi, phi + count);
    const fsp_status st = batch_build(b, reinterpret_cast<cudaStream_t>(stream));
    if (st != FSP_OK) {
        batch_free(b);
        return st;
    }
    b->magic = kBatchMagic;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_batches.insert(b);
    }
    *out = b;
    return FSP_OK;
}

extern "C" fsp_status fsp_batch_launch(fsp_batch *b, fsp_stream stream) {
    if (!batch_live(b)) return FSP_EINVAL;
    return cuda_status(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" fsp_status fsp_batch_wait(fsp_batch *b, fsp_stream stream) {
    if (!batch_live(b)) return FSP_EINVAL;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return FSP_ECUDA;
    int status = 0;
    if (cudaMemcpy(&status, &b->d_ctl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FSP_ECUDA;
    return status == 0 ? FSP_OK : (fsp_status)status;
}

extern "C" fsp_status fsp_batch_set_timeout(fsp_batch *b, double ms) {
    if (!batch_live(b) || !(ms > 0.0) || ms > 3.6e6) return FSP_EINVAL;
    b->timeout_ms = ms;
    return batch_build_graph(b);
}

extern "C" fsp_status fsp_batch_set_form(fsp_batch *b, int form) {
    if (!batch_live(b) || (form != 0 && form != 1)) return FSP_EINVAL;
    if (form == 1)
        for (const fsp_plan *p : b->plans)
            if (!p->W1) return FSP_EINVAL;
    b->form = form;
    return batch_build_graph(b);
}

extern "C" fsp_status fsp_batch_inject_stall(fsp_batch *b) {
    if (!batch_live(b)) return FSP_EINVAL;
    // the last segment of pass 1 waits for one more pass-0 tile than exists
    for (int i = (int)b->segs.size() - 1; i >= 0; --i)
        if (b->segs[i].pass == 1) {
            b->segs[i].need_prev += 1;
            break;
        }
    if (cudaMemcpy(b->d_segs, b->segs.data(), sizeof(BatchSeg) * b->segs.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return FSP_ECUDA;
    return FSP_OK;
}

namespace {
// Best of `reps` launches of the batch's graph, in ms; negative on error.
double time_batch(fsp_batch *b, cudaStream_t s, int reps) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    cudaError_t e = cudaGraphLaunch(b->exec, s);  // warm-up
    for (int i = 0; i < reps && e == cudaSuccess; ++i) {
        cudaEventRecord(e0, s);
        e = cudaGraphLaunch(b->exec, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) e = cudaErrorUnknown;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int status = 0;
    cudaMemcpy(&status, &b->d_ctl->status, sizeof(int), cudaMemcpyDeviceToHost);
    return (e == cudaSuccess && status == 0) ? best : -1.0;
}
}  // namespace

extern "C" fsp_status fsp_batch_autotune(fsp_batch *b, fsp_stream stream) {
    if (!batch_live(b)) return FSP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<int> Ns;
    for (auto *p : b->plans)
        if (std::find(Ns.begin(), Ns.end(), p->N) == Ns.end()) Ns.push_back(p->N);
    std::sort(Ns.begin(), Ns.end(), std::greater<int>());
    for (int N : Ns)
        for (auto *p : b->plans)
            if (p->N == N && !b->shape.count(N)) b->shape[N] = {p->row.lgL, p->col.lgL};
    fsp_status st = batch_build(b, s);
    if (st != FSP_OK) return st;
    double best = time_batch(b, s, 3);
    if (best < 0) return FSP_ECUDA;
    // coordinate descent, largest N first: columns, then rows
    for (int N : Ns)
        for (int which = 1; which >= 0; --which)
            for (int lg = 0; lg <= 5; ++lg) {
                auto keep = b->shape[N];
                auto trial = keep;
                (which ? trial.second : trial.first) = lg;
                if (trial == keep) continue;
                b->shape[N] = trial;
                if ((st = batch_build(b, s)) != FSP_OK) return st;
                const double t = time_batch(b, s, 3);
                if (t > 0 && t < best)
                    best = t;
                else
                    b->shape[N] = keep;
            }
    if ((st = batch_build(b, s)) != FSP_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : b->shape) g_tuning[{kv.first, (int)b->dtype}] = kv.second;
    return FSP_OK;
}

extern "C" fsp_status fsp_batch_destroy(fsp_batch *b) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!b || !g_batches.count(b)) return FSP_EINVAL;
        g_batches.erase(b);
    }
    cudaError_t e = cudaDeviceSynchronize();
    batch_free(b);
    return cuda_status(e);
}

extern "C" fsp_status fsp_solve_batched(fsp_plan *const *plans, const void *const *rho, void *const *phi, int count,
                                        fsp_stream stream) {
    fsp_batch *b = nullptr;
    fsp_status st = fsp_batch_create(&b, plans, rho, phi, count, stream);
    if (st != FSP_OK) return st;
    st = fsp_batch_launch(b, stream);
    fsp_status w = fsp_batch_wait(b, stream);
    fsp_batch_destroy(b);
    return st != FSP_OK ? st : w;
}

// -------------------------------------------------------------- server --
// Continuous batching: a worker thread owned by the server retires finished
// solves and admits queued requests into free slots (one CUDA stream each)
// whenever the device-memory budget allows, so that requests arriving while
// others run start as soon as a slot and memory free up, and their kernels
// overlap on the device.  Spectra are cached per (N, L, algo, dtype) (a plan
// without workspace) and evicted least-recently-used when the budget needs
// room; workspaces are pooled per (N, dtype).
struct fsp_server {
    uint64_t magic = 0;
    int device = 0;
    size_t budget = 0, used = 0;
    int max_slots = 0, max_queue = 0;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::thread worker;
    struct Req {
        int N;
        double L;
        fsp_algo algo;
        fsp_dtype dtype;
        const void *rho;
        void *phi;
        std::chrono::steady_clock::time_point t_submit, t_done;
        int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
        fsp_status status = FSP_OK;
    };
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<uint64_t> queue;
    uint64_t next_ticket = 1;
    struct Spec {
        fsp_plan *plan = nullptr;
        size_t bytes = 0;     // held in the budget: the plan's, or the build's reservation
        uint64_t last_use = 0;
        int refs = 0;
        bool ready = true;    // false while the builder thread computes it
        fsp_status status = FSP_OK;  // the build's result
    };
    // spectra missing from the cache are built by a thread of their own, on
    // its own stream, without the worker's lock: admission and retirement of
    // other requests go on meanwhile
    struct Build {
        std::tuple<int, uint64_t, int, int> key;
        int N;
        double L;
        fsp_algo algo;
        fsp_dtype dtype;
    };
    std::deque<Build> builds;
    std::thread builder;
    cudaStream_t build_stream = nullptr;
    int builds_in_flight = 0;
    size_t peak = 0;
    std::map<std::tuple<int, uint64_t, int, int>, Spec> specs;
    struct WS {
        void *W1 = nullptr, *W2 = nullptr;
        size_t bytes = 0;
        int N = 0;
        fsp_dtype dtype = FSP_F64;
    };
    std::vector<WS> idle_ws;
    struct Slot {
        cudaStream_t stream = nullptr;
        cudaEvent_t ev = nullptr;
        bool busy = false;
        uint64_t ticket = 0;
        WS ws;
        std::tuple<int, uint64_t, int, int> key;
    };
    std::vector<Slot> slots;
    uint64_t clock = 0;
    fsp_server_stats st{};
};

namespace {

constexpr uint64_t kServerMagic = 0x46535053'45525645ULL;  // "FSPSERVE"
std::unordered_set<const fsp_server *> g_servers;

bool server_live(const fsp_server *v) {
    std::lock_guard<std::mutex> lk(g_mu);
    return v && g_servers.count(v) && v->magic == kServerMagic;
}

uint64_t bits_of(double x) {
    uint64_t u;
    std::memcpy(&u, &x, sizeof(u));
    return u;
}

// Device bytes a spectrum-only plan holds once built (spectrum, roots tables,
// error word), and the peak of the temporaries its creation allocates (the
// real-space kernel and the method's sample grid with its transform buffers).
size_t spec_bytes(int N, fsp_dtype dtype) {
    const size_t P = ((N + 1) + 15) / 16 * 16, rs = dtype == FSP_F32_MIXED ? 4 : 8;
    return (size_t)(N + 1) * (N + 1) * P * rs + 3 * (size_t)N * 2 * rs + 16;
}
size_t plan_temp_bytes(int N, fsp_algo algo) {
    const size_t k = N + 1;
    size_t b = k * k * k * sizeof(double) + (size_t)64 * 1024 + 48 * (size_t)N;  // kernel T, roots
    if (algo == FSP_VG_DCT) {
        const size_t q = 2 * (size_t)N + 1;  // the (2N+1)^3 octant and its two pruned transforms
        b += (q * q * q + q * q * k + q * k * k) * sizeof(double);
    } else if (algo == FSP_VG) {
        const size_t m = 4 * (size_t)N;  // the (4N)^3 complex grid and its two pruned transforms
        b += (m * m * m + m * m * k + m * k * k) * sizeof(double2);
    }
    return b;
}

size_t ws_bytes(int N, fsp_dtype dtype) {
    const size_t P = ((N + 1) + 15) / 16 * 16;
    return (size_t)N * N * P * (dtype == FSP_F32_MIXED ? 8 : 16) * 3;
}

// Free idle workspaces, then unreferenced spectra (least recently used first),
// until `need` more bytes fit in the budget.  Caller holds v->mu.
bool server_make_room(fsp_server *v, size_t need) {
    while (v->used + need > v->budget && !v->idle_ws.empty()) {
        fsp_server::WS w = v->idle_ws.back();
        v->idle_ws.pop_back();
        cudaFree(w.W1);
        cudaFree(w.W2);
        v->used -= w.bytes;
    }
    while (v->used + need > v->budget) {
        auto victim = v->specs.end();
        for (auto it = v->specs.begin(); it != v->specs.end(); ++it)
            if (it->second.refs == 0 && it->second.ready &&
                (victim == v->specs.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == v->specs.end()) return false;
        if (victim->second.plan) fsp_plan_destroy(victim->second.plan);
        v->used -= victim->second.bytes;
        v->specs.erase(victim);
        v->st.evictions++;
    }
    return true;
}

void server_loop(fsp_server *v) {
    cudaSetDevice(v->device);
    std::unique_lock<std::mutex> lk(v->mu);
    while (!v->stop) {
        bool progress = false, running = false;
        // retire finished solves
        for (auto &sl : v->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) {
                running = true;
                continue;
            }
            auto &r = v->reqs[sl.ticket];
            r.t_done = std::chrono::steady_clock::now();
            r.state = q == cudaSuccess ? 2 : 3;
            r.status = q == cudaSuccess ? FSP_OK : FSP_ECUDA;
            if (q != cudaSuccess) cudaGetLastError();
            v->st.completed++;
            v->idle_ws.push_back(sl.ws);
            v->specs[sl.key].refs--;
            sl.busy = false;
            progress = true;
        }
        // admit queued requests into free slots, in arrival order
        auto none_busy = [&]() {
            for (auto &x : v->slots)
                if (x.busy) return false;
            return true;
        };
        // FIFO over the requests whose spectrum is ready; a request whose
        // spectrum is still being built keeps its place without holding back
        // the ones behind it
        for (size_t qi = 0; qi < v->queue.size();) {
            int si = -1;
            for (int i = 0; i < (int)v->slots.size(); ++i)
                if (!v->slots[i].busy) {
                    si = i;
                    break;
                }
            if (si < 0) break;
            const uint64_t t = v->queue[qi];
            auto &r = v->reqs[t];
            auto key = std::make_tuple(r.N, bits_of(r.L), (int)r.algo, (int)r.dtype);
            auto fail_at = [&](fsp_status why) {
                r.state = 3, r.status = why, r.t_done = std::chrono::steady_clock::now();
                v->queue.erase(v->queue.begin() + qi);
                v->st.completed++;
                progress = true;
            };
            auto it = v->specs.find(key);
            if (it == v->specs.end()) {
                // reserve the spectrum and its build's temporaries, then hand
                // the build to the builder thread
                const size_t need = spec_bytes(r.N, r.dtype) + plan_temp_bytes(r.N, r.algo);
                if (!server_make_room(v, need)) {
                    if (none_busy() && v->builds_in_flight == 0) {
                        fail_at(FSP_ENOMEM);  // cannot fit even with nothing running
                        continue;
                    }
                    break;  // wait for running solves and builds to release memory
                }
                fsp_server::Spec sp;
                sp.ready = false, sp.bytes = need, sp.last_use = ++v->clock;
                v->used += need;
                v->peak = std::max(v->peak, v->used);
                v->specs.emplace(key, sp);
                v->builds.push_back({key, r.N, r.L, r.algo, r.dtype});
                v->builds_in_flight++;
                v->st.spec_misses++;
                v->cv.notify_all();
                progress = true;
                ++qi;
                continue;
            }
            if (!it->second.ready) {  // being built: look further down the queue
                ++qi;
                continue;
            }
            if (it->second.status != FSP_OK) {  // the build failed: so does every request for it
                const fsp_status why = it->second.status;
                if (it->second.refs == 0) v->specs.erase(it);
                fail_at(why);
                continue;
            }
            v->st.spec_hits++;
            it->second.refs++;  // pinned while a workspace is sought
            fsp_server::WS ws;
            bool have = false;
            for (size_t i = 0; i < v->idle_ws.size(); ++i)
                if (v->idle_ws[i].N == r.N && v->idle_ws[i].dtype == r.dtype) {
                    ws = v->idle_ws[i];
                    v->idle_ws.erase(v->idle_ws.begin() + i);
                    have = true;
                    break;
                }
            if (!have) {
                const size_t wb = ws_bytes(r.N, r.dtype);
                if (!server_make_room(v, wb)) {
                    it->second.refs--;
                    if (none_busy() && v->builds_in_flight == 0) {
                        fail_at(FSP_ENOMEM);
                        continue;
                    }
                    break;
                }
                const size_t w1 = wb / 3;
                if (cudaMalloc(&ws.W1, w1) != cudaSuccess || cudaMalloc(&ws.W2, 2 * w1) != cudaSuccess) {
                    cudaGetLastError();
                    if (ws.W1) cudaFree(ws.W1);
                    ws.W1 = nullptr;
                    it->second.refs--;
                    if (none_busy() && v->builds_in_flight == 0) {
                        fail_at(FSP_ENOMEM);
                        continue;
                    }
                    break;
                }
                ws.bytes = wb, ws.N = r.N, ws.dtype = r.dtype;
                v->used += wb;
                v->peak = std::max(v->peak, v->used);
            }
            auto &sl = v->slots[si];
            it->second.last_use = ++v->clock;
            const cudaError_t e = enqueue_solve_ws(it->second.plan, r.rho, r.phi, ws.W1, ws.W2, sl.stream);
            const cudaError_t e2 = e == cudaSuccess ? cudaEventRecord(sl.ev, sl.stream) : e;
            v->queue.erase(v->queue.begin() + qi);
            if (e2 != cudaSuccess) {
                cudaGetLastError();
                r.state = 3, r.status = FSP_ECUDA, r.t_done = std::chrono::steady_clock::now();
                v->idle_ws.push_back(ws);
                it->second.refs--;
                v->st.completed++;
            } else {
                sl.busy = true, sl.ticket = t, sl.ws = ws, sl.key = key;
                r.state = 1;
                v->st.admitted++;
                running = true;
            }
            progress = true;
        }
        if (progress) continue;
        if (running) {
            // a solve is on the device: poll its event closely (latency)
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else {
            v->cv.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
}

// The builder thread: builds queued spectra on its own stream, outside the
// worker's lock, then swaps the build's reservation in the budget for the
// plan's actual size.
void server_build_loop(fsp_server *v) {
    cudaSetDevice(v->device);
    std::unique_lock<std::mutex> lk(v->mu);
    while (!v->stop) {
        if (v->builds.empty()) {
            v->cv.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        const fsp_server::Build b = v->builds.front();
        v->builds.pop_front();
        lk.unlock();
        fsp_plan *p = nullptr;
        const fsp_status cs = plan_create_impl(&p, b.N, b.L, b.L / b.N, b.algo, b.dtype,
                                               reinterpret_cast<fsp_stream>(v->build_stream), false);
        lk.lock();
        auto &sp = v->specs[b.key];
        v->used -= sp.bytes;
        sp.status = cs, sp.ready = true, sp.plan = cs == FSP_OK ? p : nullptr;
        sp.bytes = cs == FSP_OK ? p->bytes : 0;
        v->used += sp.bytes;
        v->builds_in_flight--;
        v->cv.notify_all();
    }
}

}  // namespace

extern "C" fsp_status fsp_server_create(fsp_server **out, size_t hbm_budget_bytes, int max_slots) {
    if (!out) return FSP_EINVAL;
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 64) return FSP_EINVAL;
    fsp_server *v = new fsp_server();
    if (cudaGetDevice(&v->device) != cudaSuccess) {
        delete v;
        return FSP_ECUDA;
    }
    v->budget = hbm_budget_bytes, v->max_slots = max_slots, v->max_queue = 1 << 16;
    v->slots.resize(max_slots);
    for (auto &sl : v->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            for (auto &x : v->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.ev) cudaEventDestroy(x.ev);
            }
            delete v;
            return FSP_ECUDA;
        }
    }
    if (cudaStreamCreateWithFlags(&v->build_stream, cudaStreamNonBlocking) != cudaSuccess) {
        for (auto &x : v->slots) cudaStreamDestroy(x.stream), cudaEventDestroy(x.ev);
        delete v;
        return FSP_ECUDA;
    }
    v->magic = kServerMagic;
    v->worker = std::thread(server_loop, v);
    v->builder = std::thread(server_build_loop, v);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_servers.insert(v);
    }
    *out = v;
    return FSP_OK;
}

extern "C" fsp_status fsp_server_submit(fsp_server *v, int N, double L, fsp_algo algo, fsp_dtype dtype,
                                        const void *rho, void *phi, uint64_t *ticket) {
    if (!server_live(v) || !ticket) return FSP_EINVAL;
    fsp_status st = validate_size(N, L, algo);
    if (st != FSP_OK) return st;
    if (dtype != FSP_F64 && dtype != FSP_F32_MIXED && dtype != FSP_F64_DF) return FSP_EINVAL;
    if (dtype == FSP_F64_DF && !fast::has<df>(N)) return FSP_EUNSUPPORTED;
    if (!rho || !phi || !aligned16(rho) || !aligned16(phi)) return FSP_EINVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    if ((int)v->queue.size() >= v->max_queue) return FSP_EBUSY;
    fsp_server::Req r;
    r.N = N, r.L = L, r.algo = algo, r.dtype = dtype, r.rho = rho, r.phi = phi;
    r.t_submit = std::chrono::steady_clock::now();
    const uint64_t t = v->next_ticket++;
    v->reqs.emplace(t, r);
    v->queue.push_back(t);
    v->st.submitted++;
    *ticket = t;
    v->cv.notify_one();
    return FSP_OK;
}

extern "C" fsp_status fsp_server_poll(fsp_server *v, uint64_t ticket, int *state, double *latency_ms) {
    if (!server_live(v) || !state) return FSP_EINVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    auto it = v->reqs.find(ticket);
    if (it == v->reqs.end()) return FSP_EINVAL;
    *state = it->second.state;
    if (it->second.state >= 2) {
        if (latency_ms)
            *latency_ms = std::chrono::duration<double, std::milli>(it->second.t_done - it->second.t_submit).count();
        const fsp_status rs = it->second.status;
        v->reqs.erase(it);  // a finished request is reported once
        return rs;
    }
    if (latency_ms) *latency_ms = -1.0;
    return FSP_OK;
}

extern "C" fsp_status fsp_server_get_stats(fsp_server *v, fsp_server_stats *out) {
    if (!server_live(v) || !out) return FSP_EINVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    *out = v->st;
    out->queued = v->queue.size();
    out->running = 0;
    for (auto &sl : v->slots) out->running += sl.busy ? 1 : 0;
    out->bytes_in_use = v->used;
    out->budget = v->budget;
    out->cached_spectra = v->specs.size();
    out->builds_in_flight = (uint64_t)v->builds_in_flight;
    out->peak_bytes_in_use = v->peak;
    return FSP_OK;
}

extern "C" fsp_status fsp_server_destroy(fsp_server *v) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!v || !g_servers.count(v)) return FSP_EINVAL;
        g_servers.erase(v);
    }
    {
        std::lock_guard<std::mutex> lk(v->mu);
        v->stop = true;
    }
    v->cv.notify_all();
    if (v->worker.joinable()) v->worker.join();
    if (v->builder.joinable()) v->builder.join();  // finishes the build in progress, if any
    cudaSetDevice(v->device);
    const cudaError_t e = cudaDeviceSynchronize();
    for (auto &sl : v->slots) {
        if (sl.busy) cudaFree(sl.ws.W1), cudaFree(sl.ws.W2);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.ev);
    }
    for (auto &w : v->idle_ws) cudaFree(w.W1), cudaFree(w.W2);
    for (auto &kv : v->specs)
        if (kv.second.plan) fsp_plan_destroy(kv.second.plan);
    cudaStreamDestroy(v->build_stream);
    v->magic = 0;
    delete v;
    return cuda_status(e);
}

// ------------------------------------------------------------ autotune --
namespace {

// Time `reps` generic-engine solves of plan p with tile shapes (lr, lc); the
// best of three rounds, in ms per solve, or a negative value when the shape
// does not fit (threads or shared memory).
double time_generic(fsp_plan *p, int lr, int lc, const void *rho, void *phi, cudaStream_t s, int reps) {
    const size_t csize = 2 * p->rsize;
    TileCfg row = p->row, col = p->col;
    if (!choose_tile(p->N + 1, row.tpl, csize, lr, row.lgL) || row.lgL != lr) return -1.0;
    if (!choose_tile(2 * p->N, col.tpl, csize, lc, col.lgL) || col.lgL != lc) return -1.0;
    const TileCfg save_r = p->row, save_c = p->col;
    p->row = row, p->col = col;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double best = 1e30;
    cudaError_t e = cudaSuccess;
    for (int round = 0; round < 4 && e == cudaSuccess; ++round) {
        cudaEventRecord(a, s);
        for (int i = 0; i < reps && e == cudaSuccess; ++i)
            e = p->dtype == FSP_F64 ? enqueue_solve_generic<double>(p, rho, phi, p->W1, p->W2, s)
                                    : enqueue_solve_generic<float>(p, rho, phi, p->W1, p->W2, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (round > 0) best = std::min(best, (double)ms / reps);  // round 0 warms up
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    p->row = save_r, p->col = save_c;
    return e == cudaSuccess ? best : -2.0;
}

}  // namespace

extern "C" fsp_status fsp_autotune(int N, fsp_dtype dtype, fsp_stream stream, int *lgL_row, int *lgL_col) {
    fsp_status st = validate_size(N, 1.0, FSP_HE);
    if (st != FSP_OK) return st;
    if (dtype != FSP_F64 && dtype != FSP_F32_MIXED) return FSP_EINVAL;  // generic engine only
    fsp_plan *p = nullptr;
    if ((st = plan_create_impl(&p, N, 1.0, 1.0 / N, FSP_HE, dtype, stream, true)) != FSP_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)N * N * N * p->rsize;
    DevBuf rho, phi;
    if ((st = alloc_or_nomem(rho, bytes)) != FSP_OK || (st = alloc_or_nomem(phi, bytes)) != FSP_OK) {
        fsp_plan_destroy(p);
        return st;
    }
    cudaMemsetAsync(rho.p, 0, bytes, s);
    // enough solves per round for a few milliseconds of work
    const int reps = std::max(2, std::min(200, (int)(4e6 / ((double)N * N * N))));
    int best_r = p->row.lgL, best_c = p->col.lgL;
    double best = time_generic(p, best_r, best_c, rho.p, phi.p, s, reps);
    for (int lr = 0; lr <= 5; ++lr) {  // rows, columns at their current best
        const double t = time_generic(p, lr, best_c, rho.p, phi.p, s, reps);
        if (t > 0 && t < best) best = t, best_r = lr;
    }
    for (int lc = 0; lc <= 5; ++lc) {
        const double t = time_generic(p, best_r, lc, rho.p, phi.p, s, reps);
        if (t > 0 && t < best) best = t, best_c = lc;
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    fsp_plan_destroy(p);
    if (e != cudaSuccess || best <= 0 || best >= 1e30) return FSP_ECUDA;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuning[{N, (int)dtype}] = {best_r, best_c};
    }
    if (lgL_row) *lgL_row = best_r;
    if (lgL_col) *lgL_col = best_c;
    return FSP_OK;
}

// Table text: one entry per line, "N dtype lgL_row lgL_col".
extern "C" fsp_status fsp_tuning_get(char *buf, size_t cap, size_t *len) {
    std::string out;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto &kv : g_tuning)
            out += std::to_string(kv.first.first) + " " + std::to_string(kv.first.second) + " " +
                   std::to_string(kv.second.first) + " " + std::to_string(kv.second.second) + "\n";
    }
    if (len) *len = out.size() + 1;
    if (!buf) return FSP_OK;
    if (cap < out.size() + 1) return FSP_EINVAL;
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return FSP_OK;
}

extern "C" fsp_status fsp_tuning_set(const char *text) {
    if (!text) return FSP_EINVAL;
    std::map<std::pair<int, int>, std::pair<int, int>> t;
    const char *c = text;
    while (*c) {
        int N, dt, lr, lc, used = 0;
        if (std::sscanf(c, " %d %d %d %d%n", &N, &dt, &lr, &lc, &used) != 4) {
            while (*c == ' ' || *c == '\n' || *c == '\t' || *c == '\r') ++c;
            if (*c) return FSP_EINVAL;
            break;
        }
        if (N < 2 || N > kMaxN || (dt != FSP_F64 && dt != FSP_F32_MIXED) || lr < 0 || lr > 5 || lc < 0 || lc > 5)
            return FSP_EINVAL;
        t[{N, dt}] = {lr, lc};
        c += used;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : t) g_tuning[kv.first] = kv.second;
    return FSP_OK;
}
