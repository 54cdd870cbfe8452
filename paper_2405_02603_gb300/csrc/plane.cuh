// plane.cuh -- the two transforms of one z-plane fused into one kernel, for
// power-of-two N: the forward pass PA = P1 (pad + x-R2C of the plane's rows)
// then P2 (y-FFT of its columns), and the inverse pass PC = P4 (y-IFFT of
// the columns, crop y) then P5 (x-C2R of the rows, crop x); Sec. 2.2 steps 2
// and 5 along x and y.  With P3 between them a solve is three launches.
//
// One thread-block cluster of C CTAs works on one plane.  The rows and the
// columns of the plane are split between its CTAs; between the two phases the
// plane goes through W1 once, but only through L2: each CTA writes its part,
// the cluster barrier (release / acquire at cluster scope) orders those writes
// before the other CTAs' reads, the readers load with ld.global.cg (L2 only)
// and then discard every 128-byte line they consumed (discard.global.L2: the
// line is dropped without being written back).  So W1 never reaches HBM, and
// the HBM traffic of a solve falls from 12 N^2(N+1) to 8 N^2(N+1) complex
// values (plus the source, the result and the spectrum).
//
// The two real columns k_x = 0 and k_x = N of a real row's half spectrum are
// carried as one complex column (X[0] + i X[N]), so a plane has exactly N
// columns; the y-FFT of that column is split back into the two Hermitian
// transforms, A[k] = (Y[k] + conj Y[-k]) / 2 and B[k] = (Y[k] - conj Y[-k]) /
// 2i, and the inverse packs A + i B before its y-IFFT.  The row and column
// transforms are the register-resident ones of fast.cuh.
#pragma once
#include <cooperative_groups.h>

#include "fast.cuh"

namespace fsp {
namespace fast {

// Per (type, N): CTAs per cluster (one plane), the row shape (values per
// thread, rows per tile, radices of the length-N packed FFT) and the column
// shape (length 2N), with equal thread counts.
// MINB: CTAs per SM the register budget is sized for (__launch_bounds__).
template <typename T, int N> struct PlaneCfg {
    static constexpr bool Ok = false;
    static constexpr int C = 1, MINB = 1, RV = 8, RL = 8, RR1 = 8, RR2 = 1, RR3 = 1, CV = 8, CLn = 8, CR1 = 8,
                         CR2 = 1, CR3 = 1;
};
#define FSP_PLANE_CFG(TT, NN, CC, MB, RV_, RL_, A1, A2, A3, CV_, CL_, B1, B2, B3)                                 \
    template <> struct PlaneCfg<TT, NN> {                                                                         \
        static constexpr bool Ok = true;                                                                          \
        static constexpr int C = CC, MINB = MB, RV = RV_, RL = RL_, RR1 = A1, RR2 = A2, RR3 = A3, CV = CV_,     \
                             CLn = CL_, CR1 = B1, CR2 = B2, CR3 = B3;                                             \
    };
FSP_PLANE_CFG(float, 64, 4, 4, 8, 16, 8, 8, 1, 16, 16, 8, 16, 1)
FSP_PLANE_CFG(float, 128, 4, 2, 16, 32, 8, 16, 1, 16, 16, 16, 16, 1)
FSP_PLANE_CFG(float, 256, 8, 2, 16, 16, 16, 16, 1, 32, 16, 16, 32, 1)
#undef FSP_PLANE_CFG

template <typename T, int N> struct PlaneGeo {
    using K = PlaneCfg<T, N>;
    static constexpr int n = 2 * N, P = row_pitch(N);
    static constexpr int NTH = K::RL * (N / K::RV);
    static constexpr int PER = N / K::C;  // rows and packed columns of one CTA
    static_assert(!K::Ok || NTH == K::CLn * (n / K::CV), "row and column shapes need equal thread counts");
    static_assert(!K::Ok || (PER % K::RL == 0 && PER % K::CLn == 0), "tiles must cover a CTA's share");
    static_assert(!K::Ok || K::CLn * sizeof(cx_t<T>) == 128, "a column tile's row segment is one 128-byte line");
    static_assert(!K::Ok || K::RR1 * K::RR2 * K::RR3 == N, "row radices multiply to N");
    static_assert(!K::Ok || K::CR1 * K::CR2 * K::CR3 == n, "column radices multiply to 2N");
    static_assert(!K::Ok || (K::RV % K::RR1 == 0 && K::RV % K::RR2 == 0 && K::RV % K::RR3 == 0 &&
                             K::CV % K::CR1 == 0 && K::CV % K::CR2 == 0 && K::CV % K::CR3 == 0),
                  "every radix divides the values per thread");
    static constexpr size_t SMEM_ROW = (size_t)(N + 1) * (K::RL + 1) * sizeof(cx_t<T>);
    static constexpr size_t SMEM_COL = (size_t)n * (K::CLn + 1) * sizeof(cx_t<T>);
    static constexpr size_t SMEM = SMEM_ROW > SMEM_COL ? SMEM_ROW : SMEM_COL;
};

__device__ __forceinline__ void discard_l2(const void *p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// ---------------------------------------------------------------- rows --
// L rows of N reals (x: first row, stride N) -> packed half spectra (W1 rows,
// stride P): X[1..N-1] at k_x = 1..N-1, (X[0], X[N]) as the real and
// imaginary parts at k_x = 0.  Through the length-N FFT of the packed pairs
// z[m] = x[2m] + i x[2m+1] (zero for m >= N/2, the padding).
template <typename T, int N, int V, int L, int R1, int R2, int R3>
__device__ __forceinline__ void plane_r2c_tile(const typename io_of<T>::t *x, cx_t<T> *w1, cx_t<T> *buf,
                                               const cx_t<T> *tw, const cx_t<T> *tw2) {
    using C = cx_t<T>;
    constexpr int TPL = N / V, LD = L + 1, NTH = L * TPL, H = N / 2, P = row_pitch(N);
    constexpr int RL = LastR<R1, R2, R3>::value;
    const int tid = threadIdx.x, l = tid % L, t = tid / L;
    {
        constexpr int PER = (L * H + NTH - 1) / NTH;
        C q[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = tid + i * NTH, m = idx % H, rr = idx / H;
            q[i] = idx < L * H ? load_pair<T>(x + rr * N, m) : C{T(0), T(0)};
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = tid + i * NTH;
            if (idx < L * H) buf[(idx % H) * LD + idx / H] = q[i];
        }
    }
    __syncthreads();
    using S = Stg<T, -1, N, V, L>;
    C v[V];
#pragma unroll
    for (int k = 0; k < V / R1; ++k)
#pragma unroll
        for (int r = 0; r < R1 / 2; ++r) v[k * R1 + r] = buf[(t + k * TPL + r * (N / R1)) * LD + l];
    S::template compute<R1, 1, true, false>(v, t, tw);
    run_rest<T, -1, N, V, L, R1, R2, R3, false>(v, buf, t, l, tw, true);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V / RL; ++k)
#pragma unroll
        for (int r = 0; r < RL; ++r) buf[(t + k * TPL + r * (N / RL)) * LD + l] = v[k * RL + r];
    __syncthreads();
    // X[k] = E + w^k O, X[N-k] = conj(E - w^k O), E/O from Z[k], Z[N-k]
    for (int k = t; 2 * k <= N; k += TPL) {
        const int kc = k == 0 ? 0 : N - k;
        const C zk = buf[k * LD + l], zc = buf[kc * LD + l];
        const C e = C{T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y)};
        const C o = C{T(0.5) * (zk.y + zc.y), T(-0.5) * (zk.x - zc.x)};
        const C wo = cmul(ldg_c(tw2 + k), o);
        if (k == 0) {  // X[0] and X[N] are real: packed as one value
            buf[l] = C{e.x + o.x, e.x - o.x};
        } else {
            buf[k * LD + l] = cadd(e, wo);
            if (2 * k != N) buf[kc * LD + l] = cconj(csub(e, wo));
        }
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (int rr = warp; rr < L; rr += NTH / 32) {
        C *crow = w1 + (long long)rr * P;
#pragma unroll
        for (int k = lane; k < N; k += 32) crow[k] = buf[k * LD + rr];
    }
}

// L rows of packed half spectra (W1) -> the first N of the 2N real outputs.
// The W1 lines are read through L2 only and discarded after use.
template <typename T, int N, int V, int L, int R1, int R2, int R3>
__device__ __forceinline__ void plane_c2r_tile(cx_t<T> *w1, typename io_of<T>::t *x, cx_t<T> *buf,
                                               const cx_t<T> *tw, const cx_t<T> *tw2) {
    using C = cx_t<T>;
    constexpr int TPL = N / V, LD = L + 1, NTH = L * TPL, H = N / 2, P = row_pitch(N);
    constexpr int RL = LastR<R1, R2, R3>::value;
    constexpr int LINE = 128 / (int)sizeof(C);  // complex values per 128-byte line
    const int tid = threadIdx.x, l = tid % L, t = tid / L;
    const int warp = tid >> 5, lane = tid & 31;
    {
        constexpr int NW = NTH / 32, RPW = (L + NW - 1) / NW, KPL = N / 32;
        C q[RPW * KPL];
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int rr = warp + i * NW;
            const C *crow = w1 + (long long)(rr < L ? rr : 0) * P;
#pragma unroll
            for (int j = 0; j < KPL; ++j) q[i * KPL + j] = rr < L ? ldcg_c(crow + lane + 32 * j) : C{T(0), T(0)};
        }
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int rr = warp + i * NW;
            if (rr >= L) continue;
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const int k = lane + 32 * j;
                const C qv = q[i * KPL + j];
                if (k == 0) {  // (X[0], X[N]) packed: both real
                    buf[rr] = C{qv.x, T(0)};
                    buf[N * LD + rr] = C{qv.y, T(0)};
                } else {
                    buf[k * LD + rr] = qv;
                }
            }
        }
    }
    __syncthreads();
    // every load of these rows has completed: drop their lines from L2
    for (int i = tid; i < L * (N / LINE); i += NTH) discard_l2(w1 + (long long)(i / (N / LINE)) * P + (i % (N / LINE)) * LINE);
    // Z[k] = A + i conj(w^k) B, Z[N-k] = conj A + i w^k conj B
    for (int k = t; 2 * k <= N; k += TPL) {
        const int kc = N - k;
        const C xk = buf[k * LD + l], xc = buf[kc * LD + l];
        const C A = C{xk.x + xc.x, xk.y - xc.y};
        const C B = C{xk.x - xc.x, xk.y + xc.y};
        const C w = ldg_c(tw2 + k);
        buf[k * LD + l] = cadd(A, cmuli(cmul(cconj(w), B)));
        if (k != 0 && 2 * k != N) buf[kc * LD + l] = cadd(cconj(A), cmuli(cmul(w, cconj(B))));
    }
    __syncthreads();
    using S = Stg<T, +1, N, V, L>;
    C v[V];
    S::template load_in<R1>(v, buf, t, l);
    S::template compute<R1, 1, false, false>(v, t, tw);
    run_rest<T, +1, N, V, L, R1, R2, R3, true>(v, buf, t, l, tw, true);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V / RL; ++k)
#pragma unroll
        for (int r = 0; r < RL / 2; ++r) buf[(t + k * TPL + r * (N / RL)) * LD + l] = v[k * RL + r];
    __syncthreads();
#pragma unroll 4
    for (int idx = tid; idx < L * H; idx += NTH) {
        const int m = idx % H, rr = idx / H;
        store_pair<T>(x + (long long)rr * N, m, buf[m * LD + rr]);
    }
}

// ------------------------------------------------------------- columns --
// Forward: L columns k_x0 .. k_x0+L-1 of the plane, N positions y of W1
// (pitch P), zero-padded, length-2N FFT -> all 2N outputs k_y into W2 (pitch
// P).  `packed`: the tile's first column is the packed (X[0], X[N]) column,
// split into the columns k_x = 0 and k_x = N of W2.
template <typename T, int n, int V, int L, int R1, int R2, int R3>
__device__ __forceinline__ void plane_col_fwd_tile(const cx_t<T> *in, cx_t<T> *out, bool packed, cx_t<T> *buf,
                                                   const cx_t<T> *tw, bool first_sync) {
    using C = cx_t<T>;
    constexpr int TPL = n / V, N = n / 2, P = row_pitch(N), NTH = L * TPL;
    constexpr int RL = LastR<R1, R2, R3>::value;
    const int l = threadIdx.x % L, t = threadIdx.x / L;
    const C *in_t = in + l + (long long)t * P;
    C v[V];
    StaticFor<0, V / R1>::run([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        StaticFor<0, R1 / 2>::run([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            constexpr long long c = k * TPL + r * (n / R1);
            v[k * R1 + r] = ldcg_c(in_t + c * P);
        });
    });
    Stg<T, -1, n, V, L>::template compute<R1, 1, true, false>(v, t, tw);
    run_rest<T, -1, n, V, L, R1, R2, R3, false>(v, buf, t, l, tw, first_sync);
    // every thread's loads have completed (their values passed through the
    // exchange and its barriers): drop the tile's W1 lines from L2
    if (l == 0) {
        StaticFor<0, V / R1>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            StaticFor<0, R1 / 2>::run([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                constexpr long long c = k * TPL + r * (n / R1);
                discard_l2(in + (long long)t * P + c * P);
            });
        });
    }
    if (!packed || l != 0) {
        StaticFor<0, V / RL>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            StaticFor<0, RL>::run([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                constexpr long long c = k * TPL + r * (n / RL);
                out[l + ((long long)t + c) * P] = v[k * RL + r];
            });
        });
    }
    if (packed) {  // uniform over the CTA
        __syncthreads();  // every thread is done with the exchange buffer
        if (l == 0) {
            StaticFor<0, V / RL>::run([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                StaticFor<0, RL>::run([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    constexpr int c = k * TPL + r * (n / RL);
                    buf[t + c] = v[k * RL + r];
                });
            });
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += NTH) {
            const C yk = buf[k], ym = buf[(n - k) & (n - 1)];
            out[(long long)k * P] = C{T(0.5) * (yk.x + ym.x), T(0.5) * (yk.y - ym.y)};      // A[k]
            out[(long long)k * P + N] = C{T(0.5) * (yk.y + ym.y), T(-0.5) * (yk.x - ym.x)};  // B[k]
        }
    }
}

// Inverse: L columns of W2 (2N positions k_y) -> y-IFFT -> the first N
// positions into W1.  `packed`: the tile's first column is formed as
// A + i B from W2's columns k_x = 0 (A) and k_x = N (B).
template <typename T, int n, int V, int L, int R1, int R2, int R3>
__device__ __forceinline__ void plane_col_inv_tile(const cx_t<T> *in, cx_t<T> *out, bool packed, cx_t<T> *buf,
                                                   const cx_t<T> *tw, bool first_sync) {
    using C = cx_t<T>;
    constexpr int TPL = n / V, N = n / 2, P = row_pitch(N);
    constexpr int RL = LastR<R1, R2, R3>::value;
    const int l = threadIdx.x % L, t = threadIdx.x / L;
    const C *in_t = in + l + (long long)t * P;
    const bool pk = packed && l == 0;
    C v[V];
    StaticFor<0, V / R1>::run([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        StaticFor<0, R1>::run([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            constexpr long long c = k * TPL + r * (n / R1);
            v[k * R1 + r] = ldcg_c(in_t + c * P);
        });
    });
    if (pk) {
        StaticFor<0, V / R1>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            StaticFor<0, R1>::run([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                constexpr long long c = k * TPL + r * (n / R1);
                const C b = ldcg_c(in_t + N + c * P);
                const C a = v[k * R1 + r];
                v[k * R1 + r] = C{a.x - b.y, a.y + b.x};
            });
        });
    }
    Stg<T, +1, n, V, L>::template compute<R1, 1, false, false>(v, t, tw);
    run_rest<T, +1, n, V, L, R1, R2, R3, true>(v, buf, t, l, tw, first_sync);
    StaticFor<0, V / RL>::run([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        StaticFor<0, RL / 2>::run([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            constexpr long long c = k * TPL + r * (n / RL);
            out[l + ((long long)t + c) * P] = v[k * RL + r];
        });
    });
}

// ------------------------------------------------------------- kernels --
template <typename T, int N>
__global__ void __launch_bounds__(PlaneGeo<T, N>::NTH, PlaneCfg<T, N>::MINB) k_plane_fwd(const PlaneArgs a) {
    using K = PlaneCfg<T, N>;
    using G = PlaneGeo<T, N>;
    using C = cx_t<T>;
    using R = typename io_of<T>::t;
    constexpr int n = G::n, P = G::P;
    extern __shared__ __align__(16) unsigned char plane_smem[];
    C *buf = reinterpret_cast<C *>(plane_smem);
    cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
    const int c = (int)cluster.block_rank();
    const long long z = blockIdx.x / K::C;
    const R *rho = reinterpret_cast<const R *>(a.rho);
    C *W1 = reinterpret_cast<C *>(a.w1), *W2 = reinterpret_cast<C *>(a.w2);
    const C *tw_n = reinterpret_cast<const C *>(a.tw_n), *tw_2n = reinterpret_cast<const C *>(a.tw_2n);
#pragma unroll 1
    for (int g = 0; g < G::PER / K::RL; ++g) {
        const long long y0 = (long long)c * G::PER + g * K::RL;
        if (g) __syncthreads();
        plane_r2c_tile<T, N, K::RV, K::RL, K::RR1, K::RR2, K::RR3>(rho + (z * N + y0) * N, W1 + (z * N + y0) * P, buf,
                                                                   tw_n, tw_2n);
    }
    // the plane's rows are in W1 (L2): every CTA of the cluster may read them
    cluster.sync();
#pragma unroll 1
    for (int g = 0; g < G::PER / K::CLn; ++g) {
        const int kx0 = c * G::PER + g * K::CLn;
        plane_col_fwd_tile<T, n, K::CV, K::CLn, K::CR1, K::CR2, K::CR3>(W1 + z * N * P + kx0, W2 + z * n * P + kx0,
                                                                        kx0 == 0, buf, tw_2n, true);
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(PlaneGeo<T, N>::NTH, PlaneCfg<T, N>::MINB) k_plane_inv(const PlaneArgs a) {
    using K = PlaneCfg<T, N>;
    using G = PlaneGeo<T, N>;
    using C = cx_t<T>;
    using R = typename io_of<T>::t;
    constexpr int n = G::n, P = G::P;
    extern __shared__ __align__(16) unsigned char plane_smem[];
    C *buf = reinterpret_cast<C *>(plane_smem);
    cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
    const int c = (int)cluster.block_rank();
    const long long z = blockIdx.x / K::C;
    R *phi = reinterpret_cast<R *>(a.phi);
    C *W1 = reinterpret_cast<C *>(a.w1), *W2 = reinterpret_cast<C *>(a.w2);
    const C *tw_n = reinterpret_cast<const C *>(a.tw_n), *tw_2n = reinterpret_cast<const C *>(a.tw_2n);
#pragma unroll 1
    for (int g = 0; g < G::PER / K::CLn; ++g) {
        const int kx0 = c * G::PER + g * K::CLn;
        plane_col_inv_tile<T, n, K::CV, K::CLn, K::CR1, K::CR2, K::CR3>(W2 + z * n * P + kx0, W1 + z * N * P + kx0,
                                                                        kx0 == 0, buf, tw_2n, g > 0);
    }
    // the plane's columns are in W1 (L2): every CTA of the cluster may read them
    cluster.sync();
#pragma unroll 1
    for (int g = 0; g < G::PER / K::RL; ++g) {
        const long long y0 = (long long)c * G::PER + g * K::RL;
        if (g) __syncthreads();
        plane_c2r_tile<T, N, K::RV, K::RL, K::RR1, K::RR2, K::RR3>(W1 + (z * N + y0) * P, phi + (z * N + y0) * N, buf,
                                                                   tw_n, tw_2n);
    }
}

}  // namespace fast
}  // namespace fsp
