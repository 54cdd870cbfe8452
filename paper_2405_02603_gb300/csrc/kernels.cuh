// kernels.cuh -- the line-transform kernels of the solver and their host
// launchers (declarations; definitions in kernels_impl.cuh, instantiated for
// float in kernels_f32.cu and for double in kernels_f64.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"

namespace fsp {

enum InKind { IN_CPLX = 0, IN_REAL_EVEN = 1, IN_REAL_ODD = 2 };
enum OutKind { OUT_CPLX = 0, OUT_REAL = 1 };
enum Mode { M_FWD = 0, M_INV = 1, M_FWD_MUL_INV = 2 };

// One batched line transform over strided views.  Line `c` of batch `b`,
// position `p` lives at base + b*batch + c*line + p*pos (in elements of the
// input / output type).  Column mode (line stride 1) is used for the y and z
// axes, row mode (position stride 1) for the x axis.
struct LinesArgs {
    const void *in;
    void *out;
    long long in_pos, in_line, in_batch;
    long long out_pos, out_line, out_batch;
    int n_in;    // IN_CPLX: positions loaded, the rest of the n are zero (padding);
                 // IN_REAL_EVEN: M+1 real samples, even-extended to n = 2M (DCT-I);
                 // IN_REAL_ODD: the M-1 interior samples, i times their odd
                 // extension to n = 2M, whose DFT is real: the DST-I
    int n_out;   // positions stored (0..n_out-1): the crop
    int nlines;  // valid lines per batch
    int nbatch;
    int lgL;     // lines per CTA = 2^lgL
    int tpl;     // threads per line
    Stages st;   // transform length st.n
    const void *tw;  // forward roots exp(-2 pi i e / n), e in [0,n)
    // M_FWD_MUL_INV: multiply position p of line c in batch b by the real
    // S[fold(p)*s_pos + fold_b(b)*s_batch + c], fold(k) = min(k, 2*half - k),
    // fold_b the same with half_b (0: half_b = half; a non-cubic box folds k_y
    // at n_y and z at n_z)
    const void *S;
    long long s_pos, s_batch;
    int half, half_b;
    // 0: S is even in every index (the potential).  1, 2, 3: S holds a
    // spectrum odd in the position, batch or line index (a field component):
    // the multiplier is -i S[fold], negated where that index exceeds half.
    int odd;
};

// Real rows <-> half spectra of their zero-padded length-2N extension, through
// a complex FFT of length N (st.n == N).  r2c: rows of N reals (row stride
// x_row) -> rows of N+1 complex (row stride c_row); c2r the reverse, keeping
// the first N of the 2N real outputs.
struct RowsArgs {
    const void *x;   // reals
    void *c;         // complex
    long long x_row, c_row;
    int N;
    int nrows;
    int lgL;
    int tpl;
    Stages st;       // length N
    const void *tw;  // length-N roots
    const void *tw2; // length-2N roots
};

inline int smem_pitch(int lgL) { return (1 << lgL) + 1; }

template <typename T> size_t lines_smem_bytes(const LinesArgs &a);
template <typename T> size_t rows_smem_bytes(const RowsArgs &a);

template <typename T, int IN, int OUT, int MODE> cudaError_t launch_lines(const LinesArgs &a, cudaStream_t s);
template <typename T> cudaError_t launch_r2c_rows(const RowsArgs &a, cudaStream_t s);
template <typename T> cudaError_t launch_c2r_rows(const RowsArgs &a, cudaStream_t s);

// exp(-2 pi i e / n), e in [0,n), computed in double precision (sincospi) and
// rounded to T.
template <typename T> cudaError_t launch_roots(void *tw, int n, cudaStream_t s);

}  // namespace fsp
