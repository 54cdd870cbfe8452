// kernels_impl.cuh -- definitions of the line-transform kernels (included once
// per real type by kernels_f32.cu / kernels_f64.cu).
#pragma once
#include "kernels.cuh"

namespace fsp {

constexpr int kMaxThreads = 512;

// Loads of data another CTA of the same launch may have written (the
// persistent batched kernel) bypass L1, which is not coherent across SMs.
template <bool COH, typename V> __device__ __forceinline__ V ldw(const V *p) {
    if constexpr (COH)
        return __ldcg(p);
    else
        return *p;
}

// ---------------------------------------------------------- lines_tile --
// One tile of a batched line transform: lines [bx*L, bx*L + L) of batch `by`.
// Every thread of the CTA must call it (barriers); threads beyond L*tpl idle.
template <typename T, int IN, int OUT, int MODE, bool COH>
__device__ __forceinline__ void lines_tile(const LinesArgs &a, int bx, long long by, unsigned char *smem_raw) {
    using C = cx_t<T>;
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int L = 1 << a.lgL, lmask = L - 1;
    const int ld = L + 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int line0 = bx << a.lgL;
    const long long b = by;
    const int n = a.st.n;

    // ---- load (with zero padding / even extension); U loads of a thread are
    // issued before their shared-memory stores, so that several are in flight
    constexpr int U = 4;
    if (IN == IN_CPLX) {
        const C *in = reinterpret_cast<const C *>(a.in) + b * a.in_batch;
        const int cnt = L * a.n_in;
        if (a.in_line == 1) {
            for (int base = tid; base < cnt; base += U * nth) {
                C q[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int idx = base + u * nth, l = idx & lmask, p = idx >> a.lgL;
                    q[u] = C{T(0), T(0)};
                    if (idx < cnt && line0 + l < a.nlines)
                        q[u] = ldw<COH>(in + ((long long)(line0 + l) + (long long)p * a.in_pos));
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int idx = base + u * nth;
                    if (idx < cnt) buf[(idx >> a.lgL) * ld + (idx & lmask)] = q[u];
                }
            }
        } else {
            for (int base = tid; base < cnt; base += U * nth) {
                C q[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int idx = base + u * nth, p = idx % a.n_in, l = idx / a.n_in;
                    q[u] = C{T(0), T(0)};
                    if (idx < cnt && line0 + l < a.nlines)
                        q[u] = ldw<COH>(in + ((long long)(line0 + l) * a.in_line + (long long)p * a.in_pos));
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int idx = base + u * nth;
                    if (idx < cnt) buf[(idx % a.n_in) * ld + idx / a.n_in] = q[u];
                }
            }
        }
        const int zc = L * (n - a.n_in);
        for (int idx = tid; idx < zc; idx += nth) buf[(a.n_in + (idx >> a.lgL)) * ld + (idx & lmask)] = C{T(0), T(0)};
    } else {
        // DCT-I through the DFT of the even extension: y[j] = x[j] for j <= M,
        // y[2M - j] = x[j] for 0 < j < M.  DST-I through the DFT of
        // y[j] = i x[j], y[2M - j] = -i x[j] for 0 < j < M, y[0] = y[M] = 0,
        // which is 2 sum_j x[j] sin(pi j k / M), real.
        const T *in = reinterpret_cast<const T *>(a.in) + b * a.in_batch;
        const int M = n >> 1, np = M + 1, cnt = L * np;
        const bool col = (a.in_line == 1);
        for (int idx = tid; idx < cnt; idx += nth) {
            int l, p;
            if (col) {
                l = idx & lmask;
                p = idx >> a.lgL;
            } else {
                p = idx % np;
                l = idx / np;
            }
            T x = T(0);
            if (line0 + l < a.nlines) x = ldw<COH>(in + ((long long)(line0 + l) * a.in_line + (long long)p * a.in_pos));
            const bool inner = p > 0 && p < M;
            if (IN == IN_REAL_EVEN) {
                buf[p * ld + l] = C{x, T(0)};
                if (inner) buf[(n - p) * ld + l] = C{x, T(0)};
            } else {
                buf[p * ld + l] = C{T(0), inner ? x : T(0)};
                if (inner) buf[(n - p) * ld + l] = C{T(0), -x};
            }
        }
    }
    __syncthreads();

    const int l = tid & lmask, sub = tid >> a.lgL;
    const bool act = (line0 + l) < a.nlines && sub < a.tpl;
    const C *tw = reinterpret_cast<const C *>(a.tw);
    if (MODE == M_INV)
        Engine<T, +1>::run(buf, ld, a.st, tw, l, sub, a.tpl, act);
    else
        Engine<T, -1>::run(buf, ld, a.st, tw, l, sub, a.tpl, act);

    if (MODE == M_FWD_MUL_INV) {
        const T *S = reinterpret_cast<const T *>(a.S);
        const int h2 = 2 * a.half;
        const int hb = a.half_b ? a.half_b : a.half;
        const int fy = (int)b <= hb ? (int)b : 2 * hb - (int)b;
        const int cnt = L * n;
        const int odd = a.odd;
        const T sb = odd == 2 && (int)b > hb ? T(-1) : T(1);
        for (int idx = tid; idx < cnt; idx += nth) {
            const int ll = idx & lmask, p = idx >> a.lgL;
            if (line0 + ll < a.nlines) {
                const int fz = p <= a.half ? p : h2 - p;
                T s = S[(long long)fz * a.s_pos + (long long)fy * a.s_batch + line0 + ll];
                C v = buf[p * ld + ll];
                if (odd == 0) {
                    v.x *= s;
                    v.y *= s;
                } else {
                    // -i s v; the line index (k_x <= half) never flips the sign
                    if (odd == 1 && p > a.half) s = -s;
                    s *= sb;
                    v = C{s * v.y, -(s * v.x)};
                }
                buf[p * ld + ll] = v;
            }
        }
        __syncthreads();
        Engine<T, +1>::run(buf, ld, a.st, tw, l, sub, a.tpl, act);
    }

    // ---- store (crop to n_out positions)
    const int cnt = L * a.n_out;
    const bool col = (a.out_line == 1);
    if (OUT == OUT_CPLX) {
        C *out = reinterpret_cast<C *>(a.out) + b * a.out_batch;
        for (int idx = tid; idx < cnt; idx += nth) {
            int ll, p;
            if (col) {
                ll = idx & lmask;
                p = idx >> a.lgL;
            } else {
                p = idx % a.n_out;
                ll = idx / a.n_out;
            }
            if (line0 + ll < a.nlines) out[(long long)(line0 + ll) * a.out_line + (long long)p * a.out_pos] = buf[p * ld + ll];
        }
    } else {
        T *out = reinterpret_cast<T *>(a.out) + b * a.out_batch;
        for (int idx = tid; idx < cnt; idx += nth) {
            int ll, p;
            if (col) {
                ll = idx & lmask;
                p = idx >> a.lgL;
            } else {
                p = idx % a.n_out;
                ll = idx / a.n_out;
            }
            if (line0 + ll < a.nlines)
                out[(long long)(line0 + ll) * a.out_line + (long long)p * a.out_pos] = buf[p * ld + ll].x;
        }
    }
}

template <typename T, int IN, int OUT, int MODE>
__global__ void __launch_bounds__(kMaxThreads) k_lines(const LinesArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    lines_tile<T, IN, OUT, MODE, false>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// ------------------------------------------------------------ r2c_tile --
// Sec. 2.2 steps 2 and 4 along x: each row of N reals, zero-padded to 2N, is
// transformed to its N+1 non-redundant coefficients.  With z[m] = x[2m] +
// i x[2m+1] (zero for 2m >= N) and Z = FFT_N(z):
//   E = (Z[k] + conj Z[N-k]) / 2,  O = -i (Z[k] - conj Z[N-k]) / 2,
//   X[k] = E + w^k O,  X[N-k] = conj(E - w^k O),  w = exp(-2 pi i / 2N).
template <typename T, bool COH>
__device__ __forceinline__ void r2c_tile(const RowsArgs &a, int bx, unsigned char *smem_raw) {
    using C = cx_t<T>;
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int L = 1 << a.lgL, lmask = L - 1, ld = L + 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const long long row0 = (long long)bx << a.lgL;
    const int N = a.N, Mh = (N + 1) >> 1;
    const T *x = reinterpret_cast<const T *>(a.x);

    const int cnt = L * Mh;
    constexpr int U = 4;  // loads in flight per thread
    for (int base = tid; base < cnt; base += U * nth) {
        C q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * nth, m = idx % Mh, l = idx / Mh;
            q[u] = C{T(0), T(0)};
            if (idx < cnt && row0 + l < a.nrows) {
                const T *xr = x + (row0 + l) * a.x_row;
                if ((N & 1) == 0) {
                    q[u] = ldw<COH>(reinterpret_cast<const C *>(xr) + m);
                } else {
                    q[u].x = ldw<COH>(xr + 2 * m);
                    q[u].y = (2 * m + 1 < N) ? ldw<COH>(xr + 2 * m + 1) : T(0);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * nth;
            if (idx < cnt) buf[(idx % Mh) * ld + idx / Mh] = q[u];
        }
    }
    const int zc = L * (N - Mh);
    for (int idx = tid; idx < zc; idx += nth) buf[(Mh + (idx >> a.lgL)) * ld + (idx & lmask)] = C{T(0), T(0)};
    __syncthreads();

    const int l = tid & lmask, sub = tid >> a.lgL;
    const bool act = (row0 + l) < a.nrows && sub < a.tpl;
    Engine<T, -1>::run(buf, ld, a.st, reinterpret_cast<const C *>(a.tw), l, sub, a.tpl, act);

    const C *tw2 = reinterpret_cast<const C *>(a.tw2);
    if (act) {
        for (int k = sub; 2 * k <= N; k += a.tpl) {
            const int kc = (k == 0) ? 0 : N - k;
            const C zk = buf[k * ld + l], zc = buf[kc * ld + l];
            const C e = C{T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y)};
            const C o = C{T(0.5) * (zk.y + zc.y), T(-0.5) * (zk.x - zc.x)};
            const C wo = cmul(tw2[k], o);
            if (k == 0) {
                buf[0 * ld + l] = cadd(e, o);
                buf[N * ld + l] = csub(e, o);
            } else {
                buf[k * ld + l] = cadd(e, wo);
                if (2 * k != N) buf[kc * ld + l] = cconj(csub(e, wo));
            }
        }
    }
    __syncthreads();

    C *c = reinterpret_cast<C *>(a.c);
    const int np = N + 1, cnt2 = L * np;
    for (int idx = tid; idx < cnt2; idx += nth) {
        const int k = idx % np, ll = idx / np;
        if (row0 + ll < a.nrows) c[(row0 + ll) * a.c_row + k] = buf[k * ld + ll];
    }
}

template <typename T> __global__ void __launch_bounds__(kMaxThreads) k_r2c_rows(const RowsArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    r2c_tile<T, false>(a, blockIdx.x, smem_raw);
}

// ------------------------------------------------------------ c2r_tile --
// Sec. 2.2 steps 4 and 5 along x: from the N+1 coefficients X[k] of a real
// length-2N signal y, y[j] = sum_k X[k] exp(+2 pi i jk / 2N), keep j < N.
// With A = X[k] + conj X[N-k], B = X[k] - conj X[N-k], w = exp(-2 pi i/2N):
//   Z[k] = A + i conj(w^k) B,  Z[N-k] = conj A + i w^k conj B,
//   z = IFFT_N(Z) (unnormalised),  y[2m] = Re z[m],  y[2m+1] = Im z[m].
template <typename T, bool COH>
__device__ __forceinline__ void c2r_tile(const RowsArgs &a, int bx, unsigned char *smem_raw) {
    using C = cx_t<T>;
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int L = 1 << a.lgL, ld = L + 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const long long row0 = (long long)bx << a.lgL;
    const int N = a.N, np = N + 1;
    const C *c = reinterpret_cast<const C *>(a.c);

    const int cnt = L * np;
    constexpr int U = 4;  // loads in flight per thread
    for (int base = tid; base < cnt; base += U * nth) {
        C q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * nth, k = idx % np, l = idx / np;
            q[u] = C{T(0), T(0)};
            if (idx < cnt && row0 + l < a.nrows) q[u] = ldw<COH>(c + ((row0 + l) * a.c_row + k));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * nth;
            if (idx < cnt) buf[(idx % np) * ld + idx / np] = q[u];
        }
    }
    __syncthreads();

    const int l = tid & (L - 1), sub = tid >> a.lgL;
    const bool act = (row0 + l) < a.nrows && sub < a.tpl;
    const C *tw2 = reinterpret_cast<const C *>(a.tw2);
    if (act) {
        for (int k = sub; 2 * k <= N; k += a.tpl) {
            const int kc = N - k;
            const C xk = buf[k * ld + l], xc = buf[kc * ld + l];
            const C A = C{xk.x + xc.x, xk.y - xc.y};
            const C B = C{xk.x - xc.x, xk.y + xc.y};
            const C w = tw2[k];
            buf[k * ld + l] = cadd(A, cmuli(cmul(cconj(w), B)));
            if (k != 0 && 2 * k != N) buf[kc * ld + l] = cadd(cconj(A), cmuli(cmul(w, cconj(B))));
        }
    }
    __syncthreads();
    Engine<T, +1>::run(buf, ld, a.st, reinterpret_cast<const C *>(a.tw), l, sub, a.tpl, act);

    T *x = reinterpret_cast<T *>(const_cast<void *>(a.x));
    const int Mh = (N + 1) >> 1, cnt2 = L * Mh;
    for (int idx = tid; idx < cnt2; idx += nth) {
        const int m = idx % Mh, ll = idx / Mh;
        if (row0 + ll < a.nrows) {
            T *xr = x + (row0 + ll) * a.x_row;
            const C v = buf[m * ld + ll];
            if ((N & 1) == 0) {
                reinterpret_cast<C *>(xr)[m] = v;
            } else {
                xr[2 * m] = v.x;
                if (2 * m + 1 < N) xr[2 * m + 1] = v.y;
            }
        }
    }
}

template <typename T> __global__ void __launch_bounds__(kMaxThreads) k_c2r_rows(const RowsArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2r_tile<T, false>(a, blockIdx.x, smem_raw);
}

// -------------------------------------------------------------- k_roots --
template <typename T> __global__ void k_roots(cx_t<T> *tw, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) {
        // angle -2 pi e/n reduced to (-pi, pi]: sincospi of -2e/n
        const int er = (2 * e > n) ? e - n : e;
        double s, c;
        sincospi(-2.0 * (double)er / (double)n, &s, &c);
        tw[e] = cx_t<T>{T(c), T(s)};
    }
}

// ---------------------------------------------------------------- hosts --
template <typename T> size_t lines_smem_bytes(const LinesArgs &a) {
    int np = a.st.n;
    return (size_t)np * smem_pitch(a.lgL) * sizeof(cx_t<T>);
}
template <typename T> size_t rows_smem_bytes(const RowsArgs &a) {
    return (size_t)(a.N + 1) * smem_pitch(a.lgL) * sizeof(cx_t<T>);
}

template <typename K> static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int IN, int OUT, int MODE> cudaError_t launch_lines(const LinesArgs &a, cudaStream_t s) {
    const size_t sm = lines_smem_bytes<T>(a);
    auto kern = k_lines<T, IN, OUT, MODE>;
    cudaError_t e = set_smem(kern, sm);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.nlines + (1 << a.lgL) - 1) >> a.lgL), (unsigned)a.nbatch);
    kern<<<grid, (1 << a.lgL) * a.tpl, sm, s>>>(a);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_r2c_rows(const RowsArgs &a, cudaStream_t s) {
    const size_t sm = rows_smem_bytes<T>(a);
    cudaError_t e = set_smem(k_r2c_rows<T>, sm);
    if (e != cudaSuccess) return e;
    k_r2c_rows<T><<<(unsigned)((a.nrows + (1 << a.lgL) - 1) >> a.lgL), (1 << a.lgL) * a.tpl, sm, s>>>(a);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_c2r_rows(const RowsArgs &a, cudaStream_t s) {
    const size_t sm = rows_smem_bytes<T>(a);
    cudaError_t e = set_smem(k_c2r_rows<T>, sm);
    if (e != cudaSuccess) return e;
    k_c2r_rows<T><<<(unsigned)((a.nrows + (1 << a.lgL) - 1) >> a.lgL), (1 << a.lgL) * a.tpl, sm, s>>>(a);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_roots(void *tw, int n, cudaStream_t s) {
    k_roots<T><<<(n + 255) / 256, 256, 0, s>>>(reinterpret_cast<cx_t<T> *>(tw), n);
    return cudaGetLastError();
}

#define FSP_INSTANTIATE(T)                                                                          \
    template cudaError_t launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD>(const LinesArgs &, cudaStream_t); \
    template cudaError_t launch_lines<T, IN_CPLX, OUT_CPLX, M_INV>(const LinesArgs &, cudaStream_t); \
    template cudaError_t launch_lines<T, IN_CPLX, OUT_CPLX, M_FWD_MUL_INV>(const LinesArgs &, cudaStream_t); \
    template cudaError_t launch_r2c_rows<T>(const RowsArgs &, cudaStream_t);                         \
    template cudaError_t launch_c2r_rows<T>(const RowsArgs &, cudaStream_t);                         \
    template cudaError_t launch_roots<T>(void *, int, cudaStream_t);                                 \
    template size_t lines_smem_bytes<T>(const LinesArgs &);                                          \
    template size_t rows_smem_bytes<T>(const RowsArgs &);

}  // namespace fsp
