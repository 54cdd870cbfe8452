// dist.cu -- one rank's share of a slab-decomposed solve (the distributed
// form of Sec. 2.2 steps 1-5; the paper's own solver distributes pencils and
// transposes them with all-to-all exchanges, Sec. 3.2, and maps the physical
// grid onto the doubled one by Appendix A, Algorithm 1).
//
// R ranks.  Rank r owns the z-planes [z0_r, z1_r) of the source and the
// result, and the k_x columns [c_r, c_{r+1}) of the half spectrum, with
// z0_r = floor(r N / R) and c_r = floor(r (N+1) / R):
//   forward   P1 (x-R2C) and P2 (y-FFT) on its z-slab, then one block per
//             peer p: the slab's columns of p, [zl][k_y][j], zl < nz_r,
//             k_y < 2N, j < w_p;
//   exchange  (the caller) block (r -> p) becomes p's receive block from r;
//   middle    the received blocks assembled into the k_x slab V[z][k_y][j]
//             (all z < N: the padded half never exists, as in the
//             single-GPU path), P3 (z-FFT * S * z-IFFT) and P4 (y-IFFT, crop
//             y) on it, then one block per peer p: [zl][y][j], z in p's slab,
//             y < N, j < w_r -- half the first exchange's volume, because
//             P4 already cropped y;
//   exchange  (the caller) again;
//   backward  the received blocks assembled into the z-slab's rows
//             W1[zl][y][k_x], P5 (x-C2R, crop x) into the result slab.
// The transforms are the generic engine's (any 2/3/5-smooth N, FP64 or
// FP32-mixed), with the spectrum of a spectrum-only plan; blocks are dense
// complex arrays in the caller's device memory.  Block and slab geometry is
// pure host arithmetic (fsp_dist_partition, fsp_dist_block_elems), which the
// callers' exchange code shares.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <unordered_set>

#include "../../include/fsp.h"
#include "internal.h"
#include "kernels.cuh"

using namespace fsp;

namespace {

constexpr uint64_t kDistMagic = 0x46535044'49535431ULL;  // "FSPDIST1"
// live handles: a destroyed or foreign pointer is refused without reading it
std::mutex g_dist_mu;
std::unordered_set<const void *> g_dists;

// dst[a dA + b dB + c] = src[a sA + b sB + c], (a, b, c) < (A, B, C); one
// complex value per thread, c fastest (coalesced on both sides)
template <typename C>
__global__ void k_copy3(const C *__restrict__ src, C *__restrict__ dst, long long A, long long B, long long Cn,
                        long long sA, long long sB, long long dA, long long dB) {
    const long long tot = A * B * Cn;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long c = i % Cn, ab = i / Cn, b = ab % B, a = ab / B;
        dst[a * dA + b * dB + c] = src[a * sA + b * sB + c];
    }
}

cudaError_t copy3(size_t csize, const void *src, void *dst, long long A, long long B, long long Cn, long long sA,
                  long long sB, long long dA, long long dB, cudaStream_t s) {
    const long long tot = A * B * Cn;
    if (tot <= 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (tot + threads - 1) / threads;
    const unsigned grid = (unsigned)(blocks < 65536 ? blocks : 65536);
    if (csize == sizeof(double2))
        k_copy3<double2><<<grid, threads, 0, s>>>((const double2 *)src, (double2 *)dst, A, B, Cn, sA, sB, dA, dB);
    else
        k_copy3<float2><<<grid, threads, 0, s>>>((const float2 *)src, (float2 *)dst, A, B, Cn, sA, sB, dA, dB);
    return cudaGetLastError();
}

void part(int N, int R, int r, int &z0, int &z1, int &c0, int &c1) {
    z0 = (int)((long long)r * N / R), z1 = (int)((long long)(r + 1) * N / R);
    c0 = (int)((long long)r * (N + 1) / R), c1 = (int)((long long)(r + 1) * (N + 1) / R);
}

}  // namespace

struct fsp_dist {
    uint64_t magic = 0;
    int N = 0, R = 0, rank = 0, z0 = 0, z1 = 0, c0 = 0, c1 = 0;
    fsp_plan *spec = nullptr;  // spectrum-only plan: S, roots, tile shapes
    internal::PlanView pv;
    size_t csize = 0;
    void *W1 = nullptr, *W2 = nullptr, *V = nullptr, *U = nullptr;
};

static void dist_free(fsp_dist *d);

extern "C" {

fsp_status fsp_dist_partition(int N, int nranks, int rank, int *z0, int *z1, int *kx0, int *kx1) {
    if (N < 2 || nranks < 1 || nranks > N || rank < 0 || rank >= nranks) return FSP_EINVAL;
    int a, b, c, d;
    part(N, nranks, rank, a, b, c, d);
    if (z0) *z0 = a;
    if (z1) *z1 = b;
    if (kx0) *kx0 = c;
    if (kx1) *kx1 = d;
    return FSP_OK;
}

long long fsp_dist_block_elems(int N, int nranks, int rank, int phase, int peer, int sending) {
    if (N < 2 || nranks < 1 || nranks > N || rank < 0 || rank >= nranks || peer < 0 || peer >= nranks ||
        (phase != 0 && phase != 1))
        return -1;
    // the block travels from rank s to rank q
    const int src = sending ? rank : peer, dst = sending ? peer : rank;
    int sz0, sz1, sc0, sc1, dz0, dz1, dc0, dc1;
    part(N, nranks, src, sz0, sz1, sc0, sc1);
    part(N, nranks, dst, dz0, dz1, dc0, dc1);
    // phase 0: the sender's z-planes, all 2N k_y, the receiver's columns;
    // phase 1: the receiver's z-planes, N rows y, the sender's columns
    return phase == 0 ? (long long)(sz1 - sz0) * 2LL * N * (dc1 - dc0)
                      : (long long)(dz1 - dz0) * (long long)N * (sc1 - sc0);
}

fsp_status fsp_dist_create(fsp_dist **out, int N, double L, fsp_algo algo, fsp_dtype dtype, int nranks, int rank,
                           fsp_stream stream) {
    if (!out) return FSP_EINVAL;
    *out = nullptr;
    if (dtype != FSP_F64 && dtype != FSP_F32_MIXED) return FSP_EUNSUPPORTED;
    fsp_dist *d = new fsp_dist();
    fsp_status st = fsp_dist_partition(N, nranks, rank, &d->z0, &d->z1, &d->c0, &d->c1);
    if (st != FSP_OK) {
        delete d;
        return st;
    }
    d->N = N, d->R = nranks, d->rank = rank;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((st = internal::spectrum_plan_create(&d->spec, N, L, algo, dtype, s)) != FSP_OK) {
        delete d;
        return st;
    }
    internal::plan_view(d->spec, &d->pv);
    d->csize = 2 * d->pv.rsize;
    const size_t nz = d->z1 - d->z0, w = d->c1 - d->c0, P = d->pv.P;
    const size_t b1 = nz * N * P * d->csize, b2 = 2 * b1, bv = (size_t)N * 2 * N * w * d->csize,
                 bu = (size_t)N * N * w * d->csize;
    void **bufs[4] = {&d->W1, &d->W2, &d->V, &d->U};
    const size_t sizes[4] = {b1, b2, bv, bu};
    for (int i = 0; i < 4; ++i) {
        if (cudaMalloc(bufs[i], sizes[i] ? sizes[i] : 16) != cudaSuccess) {
            cudaGetLastError();
            dist_free(d);
            return FSP_ENOMEM;
        }
    }
    d->magic = kDistMagic;
    {
        std::lock_guard<std::mutex> lk(g_dist_mu);
        g_dists.insert(d);
    }
    *out = d;
    return FSP_OK;
}

}  // extern "C"

namespace {

bool dist_live(const fsp_dist *d) {
    std::lock_guard<std::mutex> lk(g_dist_mu);
    return d && g_dists.count(d) && d->magic == kDistMagic;
}

template <typename T> cudaError_t dist_forward(fsp_dist *d, const void *rho, void *const *send, cudaStream_t s) {
    const internal::PlanView &v = d->pv;
    const int N = d->N;
    const long long P = v.P, nz = d->z1 - d->z0;
    cudaError_t e;
    RowsArgs r{};  // P1: pad + x-R2C of the slab's rows
    r.x = rho, r.c = d->W1, r.x_row = N, r.c_row = P, r.N = N, r.nrows = (int)(nz * N);
    r.lgL = v.row.lgL, r.tpl = v.row.tpl, r.st = v.row.st, r.tw = v.tw_n, r.tw2 = v.tw_2n;
    if (nz > 0 && (e = launch_r2c_rows<T>(r, s)) != cudaSuccess) return e;
    LinesArgs a{};  // P2: y-FFT, W1[zl][y][kx] -> W2[zl][ky][kx]
    a.st = v.col.st, a.tpl = v.col.tpl, a.lgL = v.col.lgL, a.tw = v.tw_2n;
    a.in = d->W1, a.out = d->W2;
    a.in_pos = P, a.in_line = 1, a.in_batch = N * P;
    a.out_pos = P, a.out_line = 1, a.out_batch = 2LL * N * P;
    a.n_in = N, a.n_out = 2 * N, a.nlines = N + 1, a.nbatch = (int)nz;
    if (nz > 0 && (e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD>(a, s)) != cudaSuccess) return e;
    for (int q = 0; q < d->R; ++q) {  // block for q: [zl][ky][j], columns of q
        int z0, z1, c0, c1;
        part(N, d->R, q, z0, z1, c0, c1);
        const size_t cs = d->csize;
        if ((e = copy3(cs, (const char *)d->W2 + c0 * cs, send[q], nz, 2 * N, c1 - c0, 2LL * N * P, P,
                       2LL * N * (c1 - c0), c1 - c0, s)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t dist_middle(fsp_dist *d, const void *const *recv, void *const *send, cudaStream_t s) {
    const internal::PlanView &v = d->pv;
    const int N = d->N;
    const long long P = v.P, w = d->c1 - d->c0;
    const size_t cs = d->csize;
    cudaError_t e;
    for (int q = 0; q < d->R; ++q) {  // block from q: [zl][ky][j] -> V[z0_q + zl][ky][j]
        int z0, z1, c0, c1;
        part(N, d->R, q, z0, z1, c0, c1);
        if ((e = copy3(cs, recv[q], (char *)d->V + (size_t)z0 * 2 * N * w * cs, z1 - z0, 2 * N, w, 2LL * N * w, w,
                       2LL * N * w, w, s)) != cudaSuccess)
            return e;
    }
    if (w > 0) {
        LinesArgs a{};  // P3: z-FFT * S * z-IFFT in place on V (lines j, batch ky)
        a.st = v.col.st, a.tpl = v.col.tpl, a.lgL = v.col.lgL, a.tw = v.tw_2n;
        a.in = a.out = d->V;
        a.in_pos = a.out_pos = 2LL * N * w, a.in_line = a.out_line = 1, a.in_batch = a.out_batch = w;
        a.n_in = N, a.n_out = N, a.nlines = (int)w, a.nbatch = 2 * N;
        a.S = (const char *)v.S + (size_t)d->c0 * v.rsize;  // S[fz][fy][c0 + j]
        a.s_pos = (long long)(N + 1) * P, a.s_batch = P, a.half = N;
        if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD_MUL_INV>(a, s)) != cudaSuccess) return e;
        LinesArgs b{};  // P4: y-IFFT, crop y: V[z][ky][j] -> U[z][y][j]
        b.st = v.col.st, b.tpl = v.col.tpl, b.lgL = v.col.lgL, b.tw = v.tw_2n;
        b.in = d->V, b.out = d->U;
        b.in_pos = w, b.in_line = 1, b.in_batch = 2LL * N * w;
        b.out_pos = w, b.out_line = 1, b.out_batch = (long long)N * w;
        b.n_in = 2 * N, b.n_out = N, b.nlines = (int)w, b.nbatch = N;
        if ((e = launch_lines<T, IN_CPLX, OUT_CPLX, M_INV>(b, s)) != cudaSuccess) return e;
    }
    for (int q = 0; q < d->R; ++q) {  // block for q: U[z in q's slab][y][j] -> [zl][y][j]
        int z0, z1, c0, c1;
        part(N, d->R, q, z0, z1, c0, c1);
        if ((e = copy3(cs, (const char *)d->U + (size_t)z0 * N * w * cs, send[q], z1 - z0, N, w, (long long)N * w,
                       w, (long long)N * w, w, s)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t dist_backward(fsp_dist *d, const void *const *recv, void *phi, cudaStream_t s) {
    const internal::PlanView &v = d->pv;
    const int N = d->N;
    const long long P = v.P, nz = d->z1 - d->z0;
    const size_t cs = d->csize;
    cudaError_t e;
    for (int q = 0; q < d->R; ++q) {  // block from q: [zl][y][j] -> W1[zl][y][c0_q + j]
        int z0, z1, c0, c1;
        part(N, d->R, q, z0, z1, c0, c1);
        if ((e = copy3(cs, recv[q], (char *)d->W1 + c0 * cs, nz, N, c1 - c0, (long long)N * (c1 - c0), c1 - c0,
                       (long long)N * P, P, s)) != cudaSuccess)
            return e;
    }
    RowsArgs r{};  // P5: x-C2R, crop x, W1 rows -> phi slab
    r.x = phi, r.c = d->W1, r.x_row = N, r.c_row = P, r.N = N, r.nrows = (int)(nz * N);
    r.lgL = v.row.lgL, r.tpl = v.row.tpl, r.st = v.row.st, r.tw = v.tw_n, r.tw2 = v.tw_2n;
    if (nz > 0 && (e = launch_c2r_rows<T>(r, s)) != cudaSuccess) return e;
    return cudaSuccess;
}

bool blocks_ok(const fsp_dist *d, const void *const *b) {
    if (!b) return false;
    for (int q = 0; q < d->R; ++q)
        if (!b[q] || (reinterpret_cast<uintptr_t>(b[q]) & 15u)) return false;
    return true;
}

}  // namespace

extern "C" {

fsp_status fsp_dist_forward(fsp_dist *d, const void *rho_slab, void *const *send, fsp_stream stream) {
    if (!dist_live(d) || !rho_slab || (reinterpret_cast<uintptr_t>(rho_slab) & 15u) ||
        !blocks_ok(d, (const void *const *)send))
        return FSP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t e = d->pv.dtype == FSP_F64 ? dist_forward<double>(d, rho_slab, send, s)
                                                 : dist_forward<float>(d, rho_slab, send, s);
    return e == cudaSuccess ? FSP_OK : FSP_ECUDA;
}

fsp_status fsp_dist_middle(fsp_dist *d, const void *const *recv, void *const *send, fsp_stream stream) {
    if (!dist_live(d) || !blocks_ok(d, recv) || !blocks_ok(d, (const void *const *)send)) return FSP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t e = d->pv.dtype == FSP_F64 ? dist_middle<double>(d, recv, send, s)
                                                 : dist_middle<float>(d, recv, send, s);
    return e == cudaSuccess ? FSP_OK : FSP_ECUDA;
}

fsp_status fsp_dist_backward(fsp_dist *d, const void *const *recv, void *phi_slab, fsp_stream stream) {
    if (!dist_live(d) || !phi_slab || (reinterpret_cast<uintptr_t>(phi_slab) & 15u) || !blocks_ok(d, recv))
        return FSP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t e = d->pv.dtype == FSP_F64 ? dist_backward<double>(d, recv, phi_slab, s)
                                                 : dist_backward<float>(d, recv, phi_slab, s);
    return e == cudaSuccess ? FSP_OK : FSP_ECUDA;
}

fsp_status fsp_dist_destroy(fsp_dist *d) {
    {
        std::lock_guard<std::mutex> lk(g_dist_mu);
        if (!d || !g_dists.erase(d)) return FSP_EINVAL;
    }
    dist_free(d);
    return FSP_OK;
}

}  // extern "C"

static void dist_free(fsp_dist *d) {
    cudaDeviceSynchronize();
    for (void *q : {d->W1, d->W2, d->V, d->U})
        if (q) cudaFree(q);
    if (d->spec) fsp_plan_destroy(d->spec);
    d->magic = 0;
    delete d;
}
