// noalloc.cu -- fsp_solve_noalloc: the FP64 solve for small grids with its
// workspace in a fixed, statically allocated device array instead of memory
// obtained from cudaMalloc.
//
// Why it exists: some callers do not call cudaMalloc at all.  Real-time
// loops often forbid any allocator call, and some host applications reserve
// all device memory through their own allocator and hand out only the
// buffers they own.  Such a caller can still compute a potential here: it passes the spectrum, the
// source and the result buffer, and the solve borrows its scratch from the
// array below.
//
// Limits: FP64 only, 2 <= N <= 32 with 2N 2/3/5-smooth.  The array holds the
// two transform buffers for N = 32 (row pitch 48) and the two roots tables:
// 147552 double2 values = 2.36 MB, held by every GPU that loads this library
// until the process exits.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fsp.h"
#include "kernels.cuh"
#include "tiles.h"

using namespace fsp;

namespace {

constexpr int kNoAllocMaxN = 32;
constexpr int kNoAllocPitch = 48;  // N+1 rounded up to 16, for N = 32
constexpr size_t kNoAllocW1 = (size_t)kNoAllocMaxN * kNoAllocMaxN * kNoAllocPitch;
constexpr size_t kNoAllocComplex = 3 * kNoAllocW1 + 3 * kNoAllocMaxN;

}  // namespace

// The shared scratch: W1 (N*N*P), W2 (2*N*N*P), roots of length N and 2N.
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocComplex];

namespace {

// The plan-based solve's radix schedule and tile rule (tiles.h).
bool noalloc_cfg(int n, int positions, int want_lgL, TileCfg &c) {
    return make_cfg(n, positions, sizeof(double2), want_lgL, c);
}

// Device address of the scratch array in the current device's context.  The
// host-side symbol is only a stand-in and must never be passed to a kernel.
// The address is looked up on every call and never cached: after a device
// reset, or when the primary context is torn down and created again, the
// module is loaded anew and the array may sit at another address.  The lookup
// allocates nothing and is not a stream operation; the first one in a context
// may load this library's device code.
fsp_status noalloc_scratch(double2 **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return FSP_ECUDA;
    }
    *out = reinterpret_cast<double2 *>(p);
    return FSP_OK;
}

}  // namespace

extern "C" fsp_status fsp_solve_noalloc(int N, const double *S, const double *rho, double *phi, fsp_stream stream) {
    if (N < 2) return FSP_EINVAL;
    if (N > kNoAllocMaxN || !is_235_smooth(2LL * N)) return FSP_EUNSUPPORTED;
    if (!S || !rho || !phi) return FSP_EINVAL;
    for (const void *q : {(const void *)S, (const void *)rho, (const void *)phi})
        if (reinterpret_cast<uintptr_t>(q) & 15u) return FSP_EINVAL;
    TileCfg row, col;
    if (!noalloc_cfg(N, N + 1, 3, row) || !noalloc_cfg(2 * N, 2 * N, 3, col)) return FSP_EUNSUPPORTED;
    double2 *base = nullptr;
    fsp_status status = noalloc_scratch(&base);
    if (status != FSP_OK) return status;

    const long long P = ((N + 1) + 15) / 16 * 16;
    double2 *W1 = base, *W2 = base + (size_t)N * N * P;
    double2 *tw_n = base + 3 * (size_t)N * N * P, *tw_2n = tw_n + N;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = launch_roots<double>(tw_n, N, s)) != cudaSuccess) return FSP_ECUDA;
    if ((e = launch_roots<double>(tw_2n, 2 * N, s)) != cudaSuccess) return FSP_ECUDA;

    // P1: pad + x-R2C
    RowsArgs r{};
    r.x = rho, r.c = W1, r.x_row = N, r.c_row = P, r.N = N, r.nrows = N * N;
    r.lgL = row.lgL, r.tpl = row.tpl, r.st = row.st, r.tw = tw_n, r.tw2 = tw_2n;
    if ((e = launch_r2c_rows<double>(r, s)) != cudaSuccess) return FSP_ECUDA;
    // P2: y-FFT
    LinesArgs a{};
    a.st = col.st, a.tpl = col.tpl, a.lgL = col.lgL, a.tw = tw_2n;
    a.in = W1, a.out = W2;
    a.in_pos = P, a.in_line = 1, a.in_batch = (long long)N * P;
    a.out_pos = P, a.out_line = 1, a.out_batch = 2LL * N * P;
    a.n_in = N, a.n_out = 2 * N, a.nlines = N + 1, a.nbatch = N;
    if ((e = launch_lines<double, IN_CPLX, OUT_CPLX, M_FWD>(a, s)) != cudaSuccess) return FSP_ECUDA;
    // P3: z-FFT * S * z-IFFT; S is the caller's dense (N+1)^3 array
    a.in = a.out = W2;
    a.in_pos = a.out_pos = 2LL * N * P, a.in_batch = a.out_batch = P;
    a.n_in = N, a.n_out = N, a.nbatch = 2 * N;
    a.S = S, a.s_pos = (long long)(N + 1) * (N + 1), a.s_batch = N + 1, a.half = N;
    if ((e = launch_lines<double, IN_CPLX, OUT_CPLX, M_FWD_MUL_INV>(a, s)) != cudaSuccess) return FSP_ECUDA;
    // P4: y-IFFT
    a.in = W2, a.out = W1;
    a.in_pos = P, a.in_batch = 2LL * N * P;
    a.out_pos = P, a.out_batch = (long long)N * P;
    a.n_in = 2 * N, a.n_out = N, a.nbatch = N;
    if ((e = launch_lines<double, IN_CPLX, OUT_CPLX, M_INV>(a, s)) != cudaSuccess) return FSP_ECUDA;
    // P5: x-C2R
    r.x = phi;
    if ((e = launch_c2r_rows<double>(r, s)) != cudaSuccess) return FSP_ECUDA;
    return FSP_OK;
}
