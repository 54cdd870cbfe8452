// fast.h -- host interface of the specialised power-of-two pass kernels
// (fast.cuh): argument blocks and one launcher per solve pass.
#pragma once
#include <cuda_runtime.h>

namespace fsp {
namespace fast {

// Column pass: line c of batch b, position p at base + b*batch + c + p*pos.
struct ColArgs {
    const void *in;
    void *out;
    long long in_pos, in_batch, out_pos, out_batch;
    int nlines;
    const void *tw;  // forward roots exp(-2 pi i e / n), n = 2N
    const void *S;   // P3: real spectrum S[fold(p)*s_pos + fold(b)*s_batch + c]
    long long s_pos, s_batch;
    int half;        // N
    // p3_odd: 1, 2, 3 for a field component's spectrum odd in z (the
    // position), k_y (the batch) or k_x (the line): the multiplier is
    // -i S[fold], negated where z or k_y > N.  Ignored by p3.
    int odd;
    // col_rg (a non-cubic box): the fold of the batch index k_y in P3 (n_y);
    // nbatch and xrows are set by the launcher
    int half_b;
    int nbatch, xrows;
};

// Row pass: rows of N reals (x, stride x_row) <-> rows of N+1 complex (c,
// stride c_row).
struct RowArgs {
    const void *x;
    void *c;
    long long x_row, c_row;
    int nrows;
    const void *tw;   // roots of length N
    const void *tw2;  // roots of length 2N
};

enum ColMode { COL_FWD = 0, COL_INV = 1, COL_FMI = 2, COL_FMO = 3 };

// true when the specialised kernels cover this N (N = 32, 64, 128, 256, 512)
template <typename T> bool has(int N);
// P1 pad + x-R2C, P2 y-FFT, P3 z-FFT*S*z-IFFT, P4 y-IFFT, P5 x-C2R
template <typename T> cudaError_t p1(int N, const RowArgs &a, cudaStream_t s);
template <typename T> cudaError_t p2(int N, const ColArgs &a, int nbatch, cudaStream_t s);
template <typename T> cudaError_t p3(int N, const ColArgs &a, int nbatch, cudaStream_t s);
// The cubic P3 of some sizes reads its twiddles from per-stage tables stored
// right after the 2N roots in the same buffer (ColArgs::tw): p3_table_len
// complex entries (0: none), written by p3_table_fill from the roots, which
// must already be in place.  Every buffer handed to p3 as tw must hold them.
template <typename T> int p3_table_len(int N);
template <typename T> cudaError_t p3_table_fill(int N, void *tw2n, cudaStream_t s);
template <typename T> cudaError_t p4(int N, const ColArgs &a, int nbatch, cudaStream_t s);
template <typename T> cudaError_t p5(int N, const RowArgs &a, cudaStream_t s);
// A column pass (mode COL_FWD, COL_INV or COL_FMI) of length n on a non-cubic
// box: strides from `a`, lines k_x <= a.nlines - 1, P3's k_y fold at a.half_b
template <typename T> cudaError_t col_rg(int mode, int n, const ColArgs &a, int nbatch, cudaStream_t s);
// true when col_rg has a shape for lines of length n (64 .. 1024; FP32 also 2048)
template <typename T> bool has_col_rg(int n);
// P3 of a field component: z-FFT * (-i S_a, odd in the axis a.odd) * z-IFFT
template <typename T> cudaError_t p3_odd(int N, const ColArgs &a, int nbatch, cudaStream_t s);
// P3 as a persistent kernel with TMA-staged input tiles (p3_tma.cuh), in
// place on W2 of the cubic layout.  Each wait for a tile is bounded by
// timeout_ns; on expiry bit 0 of *err is set.  extra_tx > 0 (fault injection)
// makes every wait expire.
struct P3Wait {
    unsigned *err;
    unsigned long long timeout_ns;
    unsigned extra_tx;
};
template <typename T> bool has_p3_tma(int N);

// The fused plane passes (plane.cuh): PA = P1 + P2 and PC = P4 + P5 of each
// z-plane in one thread-block cluster, W1 exchanged through L2 only.
struct PlaneArgs {
    const void *rho;    // PA: source, N^3 reals
    void *phi;          // PC: result, N^3 reals (may be the source)
    void *w1;           // W1[z][y][k_x], pitch P: the plane exchange (k_x = 0 packs X[0], X[N])
    void *w2;           // W2[z][k_y][k_x], pitch P
    const void *tw_n;   // roots of length N
    const void *tw_2n;  // roots of length 2N
};
template <typename T> bool has_plane(int N);
// the sizes whose plans use the plane passes by default (measured faster than
// five launches on the GB300)
template <typename T> bool plane_default(int N);
template <typename T> cudaError_t plane_fwd(int N, const PlaneArgs &a, cudaStream_t s);
template <typename T> cudaError_t plane_inv(int N, const PlaneArgs &a, cudaStream_t s);
template <typename T> cudaError_t p3_tma(int N, void *w2, const void *S, const void *tw, const P3Wait &w, cudaStream_t s);

}  // namespace fast
}  // namespace fsp
