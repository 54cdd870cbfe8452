// fast.cuh -- compile-time specialised, register-resident line transforms for
// power-of-two lengths (the solve passes P1..P5 for N = 32..512).
//
// Compared with the generic shared-memory engine (fft_engine.cuh):
//  * the radix schedule, strides and tile shape are template constants, so all
//    index arithmetic folds into immediate offsets;
//  * every thread keeps V values in registers; only the exchanges between
//    stages go through shared memory;
//  * the first stage of a zero-padded transform reads straight from global
//    memory and skips the zero half (its butterflies have half-zero inputs),
//    and the last stage of a cropped transform computes and stores only the
//    kept half (Sec. 2.2 steps 2 and 5, pruned);
//  * in P3 the multiply by S happens in registers and the inverse transform
//    runs the forward radix schedule in reverse, so its first stage works on
//    the very registers the forward's last stage produced (no exchange);
//  * P3 also has an odd-spectrum mode (COL_FMO, the field E = -grad phi:
//    multiplier -i S_a) and every column pass a runtime-geometry form (RG,
//    non-cubic boxes: strides, line count and k_y fold from the arguments);
//  * per (type, pass) compile-time choices: the tile shape (Cfg, ColCfg) and
//    the memory options (ColOpt: L2-only streamed loads, L1 prefetch of the
//    spectrum, roots table in shared memory), each kept where it measured
//    faster on the GB300.
//
// Stage s (radix R, Ns = product of the earlier radices) on butterflies
// b = t + k*TPL (k < V/R) of thread t: inputs at positions b + r n/R,
// twiddles w_n^(r (b mod Ns) n/(Ns R)), outputs at (b - b mod Ns) R +
// b mod Ns + r Ns -- the self-sorting Stockham form of the generic engine.
#pragma once
#include <type_traits>
#include <utility>

#include "df.cuh"
#include "fast.h"
#include "kernels.cuh"

namespace fsp {
namespace fast {

// ------------------------------------------------------------ constants --
// cos(2 pi m / 32), m in [0, 8]
__host__ __device__ constexpr double c32_base(int m) {
    return m == 0   ? 1.0
           : m == 1 ? 0.98078528040323044912618
           : m == 2 ? 0.92387953251128675612818
           : m == 3 ? 0.83146961230254523707879
           : m == 4 ? 0.70710678118654752440084
           : m == 5 ? 0.55557023301960222474283
           : m == 6 ? 0.38268343236508977172846
           : m == 7 ? 0.19509032201612826784828
                    : 0.0;
}
__host__ __device__ constexpr double cos32(int m) {
    m &= 31;
    return m <= 8 ? c32_base(m) : m <= 16 ? -c32_base(16 - m) : m <= 24 ? -c32_base(m - 16) : c32_base(32 - m);
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }

// Type of the caller's real arrays (rho, phi): the compute type itself, except
// for double-float, whose solves read and write double.
template <typename T> struct io_of {
    using t = T;
};
template <> struct io_of<df> {
    using t = double;
};
template <typename T> __device__ __forceinline__ cx_t<T> load_pair(const typename io_of<T>::t *row, int m) {
    if constexpr (std::is_same<T, df>::value) {
        const double2 q = reinterpret_cast<const double2 *>(row)[m];
        return cdf{df_from_double(q.x), df_from_double(q.y)};
    } else {
        return reinterpret_cast<const cx_t<T> *>(row)[m];
    }
}
template <typename T> __device__ __forceinline__ void store_pair(typename io_of<T>::t *row, int m, cx_t<T> v) {
    if constexpr (std::is_same<T, df>::value)
        reinterpret_cast<double2 *>(row)[m] = double2{df_to_double(v.x), df_to_double(v.y)};
    else
        reinterpret_cast<cx_t<T> *>(row)[m] = v;
}

// loads that bypass L1 (ld.global.cg): streamed data and spectrum values
// are read once per CTA, so they should not evict the twiddle table from L1
__device__ __forceinline__ float2 ldcg_c(const float2 *p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg_c(const double2 *p) { return __ldcg(p); }
__device__ __forceinline__ cdf ldcg_c(const cdf *p) {
    const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
    return cdf{df(q.x, q.y, 0), df(q.z, q.w, 0)};
}
__device__ __forceinline__ float ldcg_r(const float *p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg_r(const double *p) { return __ldcg(p); }
__device__ __forceinline__ df ldcg_r(const df *p) {
    const float2 q = __ldcg(reinterpret_cast<const float2 *>(p));
    return df(q.x, q.y, 0);
}

template <int I, int E> struct StaticFor {
    template <class F> static __device__ __forceinline__ void run(F &&f) {
        if constexpr (I < E) {
            f(std::integral_constant<int, I>{});
            StaticFor<I + 1, E>::run(f);
        }
    }
};

// ------------------------------------------------------- register DFTs --
// v'[q] = sum_r v[r] exp(D 2 pi i r q / R).  HZ: inputs r >= R/2 are zero
// (not read).  HO: only outputs q < R/2 are produced.  PK (FP32 only): the
// complex sums as packed two-float instructions (cadd_pk, csub_pk) and the
// +-i rotations of the radix-4 butterflies per component, so that no pair
// has to be rebuilt for the packed form; kernels choose it where it
// measured faster.
template <typename T, int D, bool PK = false> struct RD {
    using C = cx_t<T>;
    static_assert(!PK || std::is_same<T, float>::value, "packed sums are FP32");
    static __device__ __forceinline__ C rot(C a) { return D < 0 ? cmulmi(a) : cmuli(a); }  // exp(D i pi/2)
    static __device__ __forceinline__ C add(C a, C b) {
        if constexpr (PK)
            return cadd_pk(a, b);
        else
            return cadd(a, b);
    }
    static __device__ __forceinline__ C sub(C a, C b) {
        if constexpr (PK)
            return csub_pk(a, b);
        else
            return csub(a, b);
    }

    // multiply by exp(D 2 pi i M / 32)
    template <int M> static __device__ __forceinline__ C w32(C a) {
        constexpr int m = ((M % 32) + 32) % 32;
        if constexpr (m == 0) {
            return a;
        } else if constexpr (m == 8) {
            return rot(a);
        } else if constexpr (m == 16) {
            return C{-a.x, -a.y};
        } else if constexpr (m == 24) {
            return D < 0 ? cmuli(a) : cmulmi(a);
        } else {
            constexpr T c = T(cos32(m)), s = T(D * sin32(m));
            return cmul(a, C{c, s});
        }
    }

    // t + rot(d) and t - rot(d) per component (PK; the sign folds into the adds)
    static __device__ __forceinline__ C addrot(C t, C d) {
        return D < 0 ? C{t.x + d.y, t.y - d.x} : C{t.x - d.y, t.y + d.x};
    }
    static __device__ __forceinline__ C subrot(C t, C d) {
        return D < 0 ? C{t.x - d.y, t.y + d.x} : C{t.x + d.y, t.y - d.x};
    }

    template <bool HZ, bool HO> static __device__ __forceinline__ void d2(C *v) {
        if constexpr (HZ) {
            v[1] = v[0];
        } else {
            const C a = v[0], b = v[1];
            v[0] = add(a, b);
            if constexpr (!HO) v[1] = sub(a, b);
        }
    }
    template <bool HZ, bool HO> static __device__ __forceinline__ void d4(C *v) {
        if constexpr (PK) {
            C t0, t1, t2, d;  // outputs 1 and 3 are t1 +- rot(d)
            if constexpr (HZ) {
                t0 = v[0], t1 = v[0], t2 = v[1], d = v[1];
            } else {
                t0 = add(v[0], v[2]), t1 = sub(v[0], v[2]);
                t2 = add(v[1], v[3]), d = sub(v[1], v[3]);
            }
            v[0] = add(t0, t2);
            v[1] = addrot(t1, d);
            if constexpr (!HO) {
                v[2] = sub(t0, t2);
                v[3] = subrot(t1, d);
            }
        } else {
            C t0, t1, t2, t3;
            if constexpr (HZ) {
                t0 = v[0], t1 = v[0], t2 = v[1], t3 = rot(v[1]);
            } else {
                t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
                t2 = cadd(v[1], v[3]), t3 = rot(csub(v[1], v[3]));
            }
            v[0] = cadd(t0, t2);
            v[1] = cadd(t1, t3);
            if constexpr (!HO) {
                v[2] = csub(t0, t2);
                v[3] = csub(t1, t3);
            }
        }
    }
    template <bool HZ, bool HO> static __device__ __forceinline__ void d8(C *v) {
        C e[4], o[4];
        e[0] = v[0], e[1] = v[2], o[0] = v[1], o[1] = v[3];
        if constexpr (!HZ) e[2] = v[4], e[3] = v[6], o[2] = v[5], o[3] = v[7];
        d4<HZ, false>(e);
        d4<HZ, false>(o);
        o[1] = w32<4>(o[1]);
        o[3] = w32<12>(o[3]);
        if constexpr (PK) {  // o[2] takes w32<8> = rot in addrot / subrot
            v[0] = add(e[0], o[0]), v[1] = add(e[1], o[1]);
            v[2] = addrot(e[2], o[2]), v[3] = add(e[3], o[3]);
            if constexpr (!HO) {
                v[4] = sub(e[0], o[0]), v[5] = sub(e[1], o[1]);
                v[6] = subrot(e[2], o[2]), v[7] = sub(e[3], o[3]);
            }
        } else {
            o[2] = w32<8>(o[2]);
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = cadd(e[q], o[q]);
            if constexpr (!HO) {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q + 4] = csub(e[q], o[q]);
            }
        }
    }
    // R = 4 B (B = 4 or 8): x[B n1 + n2] -> DFT_4 over n1 per n2, twiddle
    // w_R^(n2 k1), DFT_B over n2 per k1 -> X[k1 + 4 k2].
    template <int R, bool HZ, bool HO> static __device__ __forceinline__ void dct4(C *v) {
        constexpr int B = R / 4;
        C y[R];
        StaticFor<0, B>::run([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            C g[4];
            g[0] = v[n2], g[1] = v[B + n2];
            if constexpr (!HZ) g[2] = v[2 * B + n2], g[3] = v[3 * B + n2];
            d4<HZ, false>(g);
            y[n2 * 4 + 0] = g[0];
            y[n2 * 4 + 1] = w32<n2 * 1 * (32 / R)>(g[1]);
            y[n2 * 4 + 2] = w32<n2 * 2 * (32 / R)>(g[2]);
            y[n2 * 4 + 3] = w32<n2 * 3 * (32 / R)>(g[3]);
        });
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C h[B];
#pragma unroll
            for (int n2 = 0; n2 < B; ++n2) h[n2] = y[n2 * 4 + k1];
            if constexpr (B == 4)
                d4<false, HO>(h);
            else
                d8<false, HO>(h);
#pragma unroll
            for (int k2 = 0; k2 < (HO ? B / 2 : B); ++k2) v[k1 + 4 * k2] = h[k2];
        }
    }
    // Radix 3: X1, X2 = a - (b + c)/2 +- i D (sqrt 3 / 2)(b - c).  Never a
    // padded first or a cropped last stage (those stay even).
    template <bool HZ, bool HO> static __device__ __forceinline__ void d3(C *v) {
        static_assert(!HZ && !HO, "radix 3 runs only as a middle stage");
        constexpr T s3 = T(D * 0.86602540378443864676372317075294);
        const C a = v[0], t = add(v[1], v[2]), d = sub(v[1], v[2]);
        const C u = C{a.x - T(0.5) * t.x, a.y - T(0.5) * t.y};
        const C w = C{-s3 * d.y, s3 * d.x};
        v[0] = add(a, t);
        v[1] = add(u, w);
        v[2] = sub(u, w);
    }
    // Radix 5: with t1 = v1 + v4, t2 = v2 + v3, t3 = v1 - v4, t4 = v2 - v3,
    // X1,4 = v0 + c1 t1 + c2 t2 +- i D (s1 t3 + s2 t4), X2,3 = v0 + c2 t1 +
    // c1 t2 +- i D (s2 t3 - s1 t4); c_k = cos(2 pi k / 5), s_k = sin(2 pi k / 5).
    template <bool HZ, bool HO> static __device__ __forceinline__ void d5(C *v) {
        static_assert(!HZ && !HO, "radix 5 runs only as a middle stage");
        constexpr T c1 = T(0.30901699437494742410229341718282), c2 = T(-0.80901699437494742410229341718282);
        constexpr T s1 = T(D * 0.95105651629515357211643933337938), s2 = T(D * 0.58778525229247312916870595463907);
        const C v0 = v[0], t1 = add(v[1], v[4]), t2 = add(v[2], v[3]), t3 = sub(v[1], v[4]),
                t4 = sub(v[2], v[3]);
        const C m1 = C{v0.x + c1 * t1.x + c2 * t2.x, v0.y + c1 * t1.y + c2 * t2.y};
        const C m2 = C{v0.x + c2 * t1.x + c1 * t2.x, v0.y + c2 * t1.y + c1 * t2.y};
        const C n1 = C{s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y};
        const C n2 = C{s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y};
        v[0] = C{v0.x + t1.x + t2.x, v0.y + t1.y + t2.y};
        v[1] = C{m1.x - n1.y, m1.y + n1.x};
        v[4] = C{m1.x + n1.y, m1.y - n1.x};
        v[2] = C{m2.x - n2.y, m2.y + n2.x};
        v[3] = C{m2.x + n2.y, m2.y - n2.x};
    }
    // Radix 6 = 2 x 3: E = DFT3 of the even inputs, O of the odd ones,
    // X[q] = E[q] + w6^q O[q], X[q+3] = E[q] - w6^q O[q], w6 = exp(D 2 pi i / 6).
    template <bool HZ, bool HO> static __device__ __forceinline__ void d6(C *v) {
        static_assert(!HZ && !HO, "radix 6 runs only as a middle stage");
        constexpr T s3 = T(D * 0.86602540378443864676372317075294);
        C e[3] = {v[0], v[2], v[4]}, o[3] = {v[1], v[3], v[5]};
        d3<false, false>(e);
        d3<false, false>(o);
        const C o1 = C{T(0.5) * o[1].x - s3 * o[1].y, s3 * o[1].x + T(0.5) * o[1].y};    // w6 o1
        const C o2 = C{-T(0.5) * o[2].x - s3 * o[2].y, s3 * o[2].x - T(0.5) * o[2].y};   // w6^2 o2
        v[0] = add(e[0], o[0]), v[3] = sub(e[0], o[0]);
        v[1] = add(e[1], o1), v[4] = sub(e[1], o1);
        v[2] = add(e[2], o2), v[5] = sub(e[2], o2);
    }
    template <int R, bool HZ, bool HO> static __device__ __forceinline__ void dft(C *v) {
        if constexpr (R == 2)
            d2<HZ, HO>(v);
        else if constexpr (R == 3)
            d3<HZ, HO>(v);
        else if constexpr (R == 4)
            d4<HZ, HO>(v);
        else if constexpr (R == 5)
            d5<HZ, HO>(v);
        else if constexpr (R == 6)
            d6<HZ, HO>(v);
        else if constexpr (R == 8)
            d8<HZ, HO>(v);
        else
            dct4<R, HZ, HO>(v);
    }
};

// ---------------------------------------------------------------- stages --
// n: transform length; V: values per thread; L: lines per CTA (pitch L+1).
// TWS: the roots table is in shared memory (generic loads) rather than read
// through the read-only global path.
template <typename T, int D, int n, int V, int L, bool TWS = false, bool PK = false> struct Stg {
    using C = cx_t<T>;
    static constexpr int TPL = n / V;
    static constexpr int LD = L + 1;

    // exp(D 2 pi i e / n) from the forward roots table
    static __device__ __forceinline__ C twid(const C *__restrict__ tw, int e) {
        C w;
        if constexpr (TWS)
            w = tw[e];
        else
            w = ldg_c(tw + e);
        if (D > 0) w.y = -w.y;
        return w;
    }

    template <int R, int Ns, bool HZ, bool HO>
    static __device__ __forceinline__ void compute(C *v, int t, const C *__restrict__ tw) {
        static_assert(V % R == 0, "radix must divide the values per thread");
        StaticFor<0, V / R>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            if constexpr (Ns > 1) {
                const unsigned b = (unsigned)(t + k * TPL);
                const unsigned j = b % (unsigned)Ns;
                constexpr int tws = n / (Ns * R);
#pragma unroll
                for (int r = 1; r < R; ++r) v[k * R + r] = cmul(v[k * R + r], twid(tw, (int)(r * j) * tws));
            }
            RD<T, D, PK>::template dft<R, HZ, HO>(v + k * R);
        });
    }

    // compute with this stage's table tt[j R + r] = w_n^(r j n/(Ns R)) (the
    // same roots as twid reads; r = 0 unused); FP32 only (pairs as float4)
    template <int R, int Ns, bool HZ, bool HO>
    static __device__ __forceinline__ void compute_tt(C *v, int t, const C *__restrict__ tt) {
        static_assert(std::is_same<T, float>::value && R % 2 == 0 && Ns > 1, "FP32 twiddled stages only");
        StaticFor<0, V / R>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const unsigned j = (unsigned)(t + k * TPL) % (unsigned)Ns;
            const float4 *row = reinterpret_cast<const float4 *>(tt + j * R);
#pragma unroll
            for (int q = 0; q < R / 2; ++q) {
                const float4 w2 = __ldg(row + q);
                C w0 = C{w2.x, w2.y}, w1 = C{w2.z, w2.w};
                if (D > 0) w0.y = -w0.y, w1.y = -w1.y;
                if (q > 0) v[k * R + 2 * q] = cmul(v[k * R + 2 * q], w0);
                v[k * R + 2 * q + 1] = cmul(v[k * R + 2 * q + 1], w1);
            }
            RD<T, D, PK>::template dft<R, HZ, HO>(v + k * R);
        });
    }

    template <int R> static __device__ __forceinline__ void load_in(C *v, const C *buf, int t, int l) {
#pragma unroll
        for (int k = 0; k < V / R; ++k)
#pragma unroll
            for (int r = 0; r < R; ++r) v[k * R + r] = buf[(t + k * TPL + r * (n / R)) * LD + l];
    }

    template <int R, int Ns> static __device__ __forceinline__ void store_out(C *buf, const C *v, int t, int l) {
#pragma unroll
        for (int k = 0; k < V / R; ++k) {
            const unsigned b = (unsigned)(t + k * TPL);
            const unsigned j = b % (unsigned)Ns;
            const int base = (int)((b - j) * R + j);
#pragma unroll
            for (int r = 0; r < R; ++r) buf[(base + r * Ns) * LD + l] = v[k * R + r];
        }
    }
};

// Run stages 1.. of schedule (R1, R2, R3) after stage 0 has been computed in
// registers: exchange through shared memory, compute; leaves the last
// stage's outputs in registers.  `first_sync` is needed when shared memory
// was read just before (the caller's previous stage loaded from it).
template <typename T, int D, int n, int V, int L, int R1, int R2, int R3, bool HO_LAST, bool TWS = false,
          bool PK = false>
__device__ __forceinline__ void run_rest(cx_t<T> *v, cx_t<T> *buf, int t, int l, const cx_t<T> *tw, bool first_sync) {
    using S = Stg<T, D, n, V, L, TWS, PK>;
    if (first_sync) __syncthreads();
    S::template store_out<R1, 1>(buf, v, t, l);
    __syncthreads();
    S::template load_in<R2>(v, buf, t, l);
    if constexpr (R3 == 1) {
        S::template compute<R2, R1, false, HO_LAST>(v, t, tw);
    } else {
        S::template compute<R2, R1, false, false>(v, t, tw);
        __syncthreads();
        S::template store_out<R2, R1>(buf, v, t, l);
        __syncthreads();
        S::template load_in<R3>(v, buf, t, l);
        S::template compute<R3, R1 * R2, false, HO_LAST>(v, t, tw);
    }
}

// Positions of the last stage's outputs: register k*R + r holds position
// t + k*TPL + r*(n/R) (the last stage's butterflies have b < Ns).
template <int R1, int R2, int R3> struct LastR {
    static constexpr int value = R3 > 1 ? R3 : R2;
};

// ---------------------------------------------------- column pass kernel --
// Lines are columns (consecutive lines contiguous in memory): P2 (COL_FWD,
// half-zero input, all n outputs), P4 (COL_INV, all inputs, first n/2
// outputs), P3 (COL_FMI: forward with half-zero input, times S, inverse, first
// n/2 outputs).  The last tile may be partial (N+1 lines, not a multiple of
// L).  The workspace geometry is fixed by n = 2N (row pitch P = N+1 rounded up
// to 16; W1 [z][y][kx], W2 [z][ky][kx], S [qz][qy][qx]), so every stride is a
// compile-time constant and every address offset an immediate.
__host__ __device__ constexpr int row_pitch(int N) { return ((N + 1) + 15) / 16 * 16; }

template <int n, int MODE> struct ColGeo {
    static constexpr int N = n / 2, P = row_pitch(N);
    static constexpr bool ZL = MODE == COL_FMI || MODE == COL_FMO;  // P3: z lines, batch k_y
    static constexpr long long NP = (long long)N * P;
    static constexpr long long IN_POS = ZL ? 2 * NP : P;
    static constexpr long long IN_BATCH = MODE == COL_FWD ? NP : ZL ? P : 2 * NP;
    static constexpr long long OUT_POS = ZL ? 2 * NP : P;
    static constexpr long long OUT_BATCH = MODE == COL_FWD ? 2 * NP : ZL ? P : NP;
    static constexpr long long S_POS = (long long)(N + 1) * P, S_BATCH = P;
};

// Per (type, pass) choices, each measured on the GB300 at N = 256:
//   PF:  prefetch the thread's spectrum values into L1 before the forward
//        transform (P3: their latency overlaps the transform; FP32 P3 -5 %).
//   TWS: roots table in shared memory: double-float P3 -11 % and P2 -2 %,
//        the FP32 field P3 (COL_FMO) and the FP32 P3 on lines of 1024 (-4 %)
//        faster too; the FP32 P3 of the potential on lines of 512, native
//        FP64 and every P4 are slower or unchanged with it.
template <typename T, int MODE, int n> struct ColOpt {
    static constexpr bool ZL = MODE == COL_FMI || MODE == COL_FMO;
    static constexpr bool DF = std::is_same<T, df>::value;
    static constexpr bool F32 = std::is_same<T, float>::value;
    static constexpr bool PF = ZL && !DF;
    // CTAs per SM the register allocation must allow (2: k_fast_col_occ2):
    // two 256-thread tiles of the FP32 P3 on lines of 512 (N = 256)
    static constexpr int MINB = ZL && F32 && n == 512 ? 2 : 1;
    // PK: packed two-float complex sums in the register DFTs, on the FP32
    // lines of 512 of P3 (0.206 -> 0.191 ms) and P2 (0.090 -> 0.084 ms);
    // P4 unchanged by them, the lines of 1024 6-8 % slower, so off there
    static constexpr bool PK = F32 && n == 512 && (ZL || MODE == COL_FWD);
    // INL: k_fast_col_inl for the FP32 P2 on lines of 512 (0.084 ms against
    // 0.088 with the body in the kernel)
    static constexpr bool INL = F32 && n == 512 && MODE == COL_FWD;
    // TT: the twiddled stages of the cubic P3 read per-stage tables [j][r]
    // (after the n roots; see p3_table_fill): a pair of twiddles per 16-byte
    // load at an immediate offset, no index arithmetic per twiddle
    // (measured: N = 256 P3 0.191 -> 0.183 ms; N = 128 2 % slower, so off there)
    static constexpr bool TT = MODE == COL_FMI && F32 && n == 512;
    static constexpr bool TWS = (DF && MODE != COL_INV) || (MODE == COL_FMO && !std::is_same<T, double>::value) ||
                                (MODE == COL_FMI && F32 && n == 1024);
};

// RG (a non-cubic box): the strides, the number of lines (k_x <= n_x) and the
// fold of the batch index (k_y <= n_y) come from the arguments instead of
// ColGeo; the cube keeps its compile-time geometry.
// The column pass kernels, one body source (fast_col_body.inc).  k_fast_col:
// the body in the kernel, the plain launch bound.  k_fast_col_occ2: a bound
// of two CTAs per SM (ColOpt::MINB), the body inlined from fast_col_body.
// k_fast_col_inl: the plain bound, the body inlined (ColOpt::INL).  The
// compiler's code differs between the forms; each pass takes the one it
// measured fastest with.
template <typename T, int n, int V, int L, int R1, int R2, int R3, int MODE, bool RG>
__device__ __forceinline__ void fast_col_body(const ColArgs &a) {
#include "fast_col_body.inc"
}
template <typename T, int n, int V, int L, int R1, int R2, int R3, int MODE, bool RG = false>
__global__ void __launch_bounds__(L *(n / V)) k_fast_col(const ColArgs a) {
#include "fast_col_body.inc"
}
template <typename T, int n, int V, int L, int R1, int R2, int R3, int MODE, bool RG = false>
__global__ void __launch_bounds__(L *(n / V), 2) k_fast_col_occ2(const ColArgs a) {
    fast_col_body<T, n, V, L, R1, R2, R3, MODE, RG>(a);
}
template <typename T, int n, int V, int L, int R1, int R2, int R3, int MODE, bool RG = false>
__global__ void __launch_bounds__(L *(n / V)) k_fast_col_inl(const ColArgs a) {
    fast_col_body<T, n, V, L, R1, R2, R3, MODE, RG>(a);
}
template <typename T, int n, int V, int L, int R1, int R2, int R3, int MODE, bool RG>
constexpr auto col_kernel() {
    if constexpr (ColOpt<T, MODE, n>::MINB == 2)
        return k_fast_col_occ2<T, n, V, L, R1, R2, R3, MODE, RG>;
    else if constexpr (ColOpt<T, MODE, n>::INL)
        return k_fast_col_inl<T, n, V, L, R1, R2, R3, MODE, RG>;
    else
        return k_fast_col<T, n, V, L, R1, R2, R3, MODE, RG>;
}


// ------------------------------------------------------- row kernels --
// P1: rows of N reals -> N+1 coefficients of the zero-padded length-2N row,
// through the length-N FFT of z[m] = x[2m] + i x[2m+1] (zero for m >= N/2).
template <typename T, int N, int V, int L, int R1, int R2, int R3>
__global__ void __launch_bounds__(L *(N / V)) k_fast_r2c(const RowArgs a) {
    using C = cx_t<T>;
    constexpr int TPL = N / V, LD = L + 1, NTH = L * TPL, H = N / 2;
    static_assert(NTH % 32 == 0, "row kernels use whole warps per row");
    constexpr int RL = LastR<R1, R2, R3>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int tid = threadIdx.x, l = tid % L, t = tid / L;
    const long long row0 = (long long)blockIdx.x * L;
    using R = typename io_of<T>::t;
    const R *x = reinterpret_cast<const R *>(a.x);
    // coalesced row loads of the packed pairs (x[2m], x[2m+1]), m < N/2, all
    // of a thread's loads issued before the first shared-memory store
    {
        constexpr int PER = (L * H + NTH - 1) / NTH;
        C q[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = tid + i * NTH, m = idx % H, rr = idx / H;
            q[i] = idx < L * H && row0 + rr < a.nrows ? load_pair<T>(x + (row0 + rr) * N, m) : C{T(0), T(0)};
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = tid + i * NTH;
            if (idx < L * H) buf[(idx % H) * LD + idx / H] = q[i];
        }
    }
    __syncthreads();
    const C *tw = reinterpret_cast<const C *>(a.tw);
    using S = Stg<T, -1, N, V, L>;
    C v[V];
#pragma unroll
    for (int k = 0; k < V / R1; ++k)
#pragma unroll
        for (int r = 0; r < R1 / 2; ++r) v[k * R1 + r] = buf[(t + k * TPL + r * (N / R1)) * LD + l];
    S::template compute<R1, 1, true, false>(v, t, tw);
    run_rest<T, -1, N, V, L, R1, R2, R3, false>(v, buf, t, l, tw, true);
    // natural-order spectrum Z back to shared memory
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V / RL; ++k)
#pragma unroll
        for (int r = 0; r < RL; ++r) buf[(t + k * TPL + r * (N / RL)) * LD + l] = v[k * RL + r];
    __syncthreads();
    // X[k] = E + w^k O, X[N-k] = conj(E - w^k O), E/O from Z[k], Z[N-k]
    const C *tw2 = reinterpret_cast<const C *>(a.tw2);
    for (int k = t; 2 * k <= N; k += TPL) {
        const int kc = k == 0 ? 0 : N - k;
        const C zk = buf[k * LD + l], zc = buf[kc * LD + l];
        const C e = C{T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y)};
        const C o = C{T(0.5) * (zk.y + zc.y), T(-0.5) * (zk.x - zc.x)};
        const C wo = cmul(ldg_c(tw2 + k), o);
        if (k == 0) {
            buf[l] = cadd(e, o);
            buf[N * LD + l] = csub(e, o);
        } else {
            buf[k * LD + l] = cadd(e, wo);
            if (2 * k != N) buf[kc * LD + l] = cconj(csub(e, wo));
        }
    }
    __syncthreads();
    // one warp per row: coalesced stores of the N+1 coefficients
    C *c = reinterpret_cast<C *>(a.c);
    const int warp = tid >> 5, lane = tid & 31;
    for (int rr = warp; rr < L; rr += NTH / 32) {
        if (row0 + rr < a.nrows) {
            C *crow = c + (row0 + rr) * row_pitch(N);
            for (int k = lane; k <= N; k += 32) crow[k] = buf[k * LD + rr];
        }
    }
}

// P5: N+1 coefficients -> first N of the 2N real outputs.
template <typename T, int N, int V, int L, int R1, int R2, int R3>
__global__ void __launch_bounds__(L *(N / V)) k_fast_c2r(const RowArgs a) {
    using C = cx_t<T>;
    constexpr int TPL = N / V, LD = L + 1, NTH = L * TPL, H = N / 2;
    constexpr int RL = LastR<R1, R2, R3>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int tid = threadIdx.x, l = tid % L, t = tid / L;
    const long long row0 = (long long)blockIdx.x * L;
    // one warp per row: coalesced loads of the N+1 coefficients, all of a
    // thread's loads issued before the first shared-memory store
    const C *c = reinterpret_cast<const C *>(a.c);
    const int warp = tid >> 5, lane = tid & 31;
    {
        constexpr int NW = NTH / 32, RPW = (L + NW - 1) / NW, KPL = (N + 32) / 32;
        C q[RPW * KPL];
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int rr = warp + i * NW;
            const bool okr = rr < L && row0 + rr < a.nrows;
            const C *crow = c + (okr ? row0 + rr : 0) * row_pitch(N);
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const int k = lane + 32 * j;
                q[i * KPL + j] = okr && k <= N ? crow[k] : C{T(0), T(0)};
            }
        }
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int rr = warp + i * NW;
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const int k = lane + 32 * j;
                if (rr < L && k <= N) buf[k * LD + rr] = q[i * KPL + j];
            }
        }
    }
    __syncthreads();
    // Z[k] = A + i conj(w^k) B, Z[N-k] = conj A + i w^k conj B
    const C *tw2 = reinterpret_cast<const C *>(a.tw2);
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
    const C *tw = reinterpret_cast<const C *>(a.tw);
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
    using R = typename io_of<T>::t;
    R *x = reinterpret_cast<R *>(const_cast<void *>(a.x));
#pragma unroll 4
    for (int idx = tid; idx < L * H; idx += NTH) {
        const int m = idx % H, rr = idx / H;
        if (row0 + rr < a.nrows) store_pair<T>(x + (row0 + rr) * N, m, buf[m * LD + rr]);
    }
}

// ------------------------------------ row kernels, one lane per position --
// FP32 rows with a two-stage schedule whose last radix is V (N = 32 .. 512):
// the TPL threads of a row are consecutive lanes, so position p = t + TPL c of
// the row is register c of lane t.  The first stage's inputs and the last
// stage's outputs then move between registers and global memory directly
// (TPL lanes cover TPL consecutive complex values), and the one exchange
// between the stages uses a row-major shared buffer with one pad slot per
// TPL positions, free of bank conflicts for both of its access patterns.
// Both pair Z[p] (P1) or X[p] (P5) with the value at N - p by a warp
// shuffle: lane TPL - t, register V-1-c (lane 0: its own register (V-c) mod V,
// and X[N] for p = 0 in P5).
template <typename T, int N, int V, int R1, int R2, int R3> struct LaneRow {
    static constexpr int TPL = N / V;
    static constexpr bool ok = std::is_same<T, float>::value && R3 == 1 && R2 == V && V % R1 == 0 &&
                               TPL >= 4 && 32 % TPL == 0;
    // row stride: room for positions 0..N (N + N/TPL + 1 slots), rounded up to
    // TPL mod 16, so that the rows of one half-warp start on distinct banks
    static constexpr int LDT = (N + V + 1) + ((TPL - (N + V + 1)) % 16 + 16) % 16;
    static __device__ __forceinline__ int idx(int pos, int l) { return l * LDT + pos + pos / TPL; }
};
// CTAs per SM for the launch bound, from a register target per thread: 64
// at N = 128, 256 (measured: P5 at N = 256 0.044 ms with 64 registers
// against 0.047 with the compiler's 72), 48 at N = 64 and 64 at N = 32 (what
// the compiler takes there by itself), 128 at N = 512 (two 256-thread CTAs)
template <int N, int V, int L> constexpr int lane_row_minb() {
    return 65536 / (L * (N / V) * (N == 64 ? 48 : N <= 256 ? 64 : 128));
}
template <typename T, int N, int V, int L> constexpr size_t lane_row_smem() {
    return (size_t)L * LaneRow<T, N, V, 1, V, 1>::LDT * sizeof(cx_t<T>);
}

// the exchange between the two stages: stage-0 outputs of butterfly
// b = t + k TPL at b R1 + r, stage-1 inputs at t + r TPL
template <typename T, int D, int N, int V, int L, int R1>
__device__ __forceinline__ void lane_row_stages(cx_t<T> *v, cx_t<T> *buf, int t, int l, const cx_t<T> *tw,
                                                bool hz, bool ho) {
    using X = LaneRow<T, N, V, R1, V, 1>;
    using S = Stg<T, D, N, V, L, false, true>;  // packed sums (FP32 only, as LaneRow::ok)
    constexpr int TPL = N / V;
    if (hz)
        S::template compute<R1, 1, true, false>(v, t, tw);
    else
        S::template compute<R1, 1, false, false>(v, t, tw);
#pragma unroll
    for (int k = 0; k < V / R1; ++k)
#pragma unroll
        for (int r = 0; r < R1; ++r) buf[X::idx((t + k * TPL) * R1 + r, l)] = v[k * R1 + r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < V; ++r) v[r] = buf[X::idx(t + r * TPL, l)];
    if (ho)
        S::template compute<V, R1, false, true>(v, t, tw);
    else
        S::template compute<V, R1, false, false>(v, t, tw);
}

// P1, lane per position: same arithmetic as k_fast_r2c
template <typename T, int N, int V, int L, int R1>
__global__ void __launch_bounds__(L *(N / V), (lane_row_minb<N, V, L>())) k_lane_r2c(const RowArgs a) {
    using C = cx_t<T>;
    constexpr int TPL = N / V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int tid = threadIdx.x, t = tid % TPL, l = tid / TPL;
    const long long row = (long long)blockIdx.x * L + l;
    const bool live = row < a.nrows;
    using R = typename io_of<T>::t;
    const R *xr = reinterpret_cast<const R *>(a.x) + (live ? row : 0) * N;
    const C *tw = reinterpret_cast<const C *>(a.tw);
    C v[V];
    // stage 0 (zero upper half): z[m] = (x[2m], x[2m+1]) at m = t + k TPL + r N/R1 < N/2
#pragma unroll
    for (int k = 0; k < V / R1; ++k)
#pragma unroll
        for (int r = 0; r < R1 / 2; ++r)
            v[k * R1 + r] = live ? load_pair<T>(xr, t + k * TPL + r * (N / R1)) : C{T(0), T(0)};
    lane_row_stages<T, -1, N, V, L, R1>(v, buf, t, l, tw, true, false);
    // v[c] = Z[t + c TPL].  X[q] = E + w^q O, X[N-q] = conj(E - w^q O) for
    // q <= N/2, E, O from (Z[q], Z[N-q]); each lane computes its own positions
    const C *tw2 = reinterpret_cast<const C *>(a.tw2);
    C *crow = reinterpret_cast<C *>(a.c) + (live ? row : 0) * row_pitch(N);
    const int lane = tid & 31, src = (lane & ~(TPL - 1)) | ((TPL - t) & (TPL - 1));
#pragma unroll
    for (int c = 0; c < V; ++c) {
        C zp;  // Z[N - p], p = t + c TPL
        zp.x = __shfl_sync(0xffffffffu, v[V - 1 - c].x, src);
        zp.y = __shfl_sync(0xffffffffu, v[V - 1 - c].y, src);
        if (t == 0) zp = v[(V - c) % V];
        const int p = t + c * TPL;
        const bool lo = c < V / 2 || p == N / 2;  // p <= N/2
        const C zk = lo ? v[c] : zp, zc = lo ? zp : v[c];
        const C e = C{T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y)};
        const C o = C{T(0.5) * (zk.y + zc.y), T(-0.5) * (zk.x - zc.x)};
        if (p == 0) {
            if (live) {
                crow[0] = cadd(e, o);
                crow[N] = csub(e, o);
            }
        } else {
            const C wo = cmul(ldg_c(tw2 + (lo ? p : N - p)), o);
            if (live) crow[p] = lo ? cadd(e, wo) : cconj(csub(e, wo));
        }
    }
}

// P5, lane per position: same arithmetic as k_fast_c2r
template <typename T, int N, int V, int L, int R1>
__global__ void __launch_bounds__(L *(N / V), (lane_row_minb<N, V, L>())) k_lane_c2r(const RowArgs a) {
    using C = cx_t<T>;
    constexpr int TPL = N / V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int tid = threadIdx.x, t = tid % TPL, l = tid / TPL;
    const long long row = (long long)blockIdx.x * L + l;
    const bool live = row < a.nrows;
    const C *crow = reinterpret_cast<const C *>(a.c) + (live ? row : 0) * row_pitch(N);
    C x[V];
#pragma unroll
    for (int c = 0; c < V; ++c) x[c] = live ? crow[t + c * TPL] : C{T(0), T(0)};
    const C xn = live && t == 0 ? crow[N] : C{T(0), T(0)};
    // Z[q] = A + i conj(w^q) B, Z[N-q] = conj A + i w^q conj B for q <= N/2,
    // A, B from (X[q], X[N-q]).  Positions t + c TPL and t + (V-1-c) TPL are
    // done together: their partners are registers V-1-c and c of lane TPL - t
    // (lane 0: X[N] or its own register V - c, and its register c + 1), so each
    // coefficient is last read in the iteration that consumes it.  Z[t + c TPL]
    // goes to stage 0's register (c mod (V/R1)) R1 + c / (V/R1) (its position
    // t + k TPL + r N/R1).
    const C *tw2 = reinterpret_cast<const C *>(a.tw2);
    const int lane = tid & 31, src = (lane & ~(TPL - 1)) | ((TPL - t) & (TPL - 1));
    C v[V];
    auto zof = [&](int c, C xc_own, C xp) {
        const int p = t + c * TPL;
        const bool lo = c < V / 2 || p == N / 2;
        const C xk = lo ? xc_own : xp, xc = lo ? xp : xc_own;
        const C A = C{xk.x + xc.x, xk.y - xc.y};
        const C B = C{xk.x - xc.x, xk.y + xc.y};
        const C w = ldg_c(tw2 + (lo ? p : N - p));
        v[(c % (V / R1)) * R1 + c / (V / R1)] =
            lo ? cadd(A, cmuli(cmul(cconj(w), B))) : cadd(cconj(A), cmuli(cmul(w, cconj(B))));
    };
#pragma unroll
    for (int c = 0; c < V / 2; ++c) {
        const int cc = V - 1 - c;
        C p0, p1;  // partners of positions t + c TPL and t + cc TPL
        p0.x = __shfl_sync(0xffffffffu, x[cc].x, src);
        p0.y = __shfl_sync(0xffffffffu, x[cc].y, src);
        p1.x = __shfl_sync(0xffffffffu, x[c].x, src);
        p1.y = __shfl_sync(0xffffffffu, x[c].y, src);
        if (t == 0) {
            p0 = c == 0 ? xn : x[V - c];
            p1 = x[c + 1];
        }
        zof(c, x[c], p0);
        zof(cc, x[cc], p1);
    }
    lane_row_stages<T, +1, N, V, L, R1>(v, buf, t, l, reinterpret_cast<const C *>(a.tw), false, true);
    // the first N/2 positions t + c TPL (c < V/2) hold z[m] = (x[2m], x[2m+1])
    using R = typename io_of<T>::t;
    R *xr = reinterpret_cast<R *>(const_cast<void *>(a.x)) + (live ? row : 0) * N;
    if (live) {
#pragma unroll
        for (int c = 0; c < V / 2; ++c) store_pair<T>(xr, t + c * TPL, v[c]);
    }
}

// ----------------------------------------------------- configurations --
// Tile shape and radix schedule per (type, length); Ok = false: no fast path.
template <typename T, int n> struct Cfg {
    static constexpr bool Ok = false;
    static constexpr int V = 8, L = 8, R1 = 8, R2 = 8, R3 = 1;
};
#define FSP_CFG(TT, NN, VV, LL, A, B, CC)                                   \
    template <> struct Cfg<TT, NN> {                                       \
        static constexpr bool Ok = true;                                   \
        static constexpr int V = VV, L = LL, R1 = A, R2 = B, R3 = CC;      \
    };
FSP_CFG(float, 32, 8, 16, 4, 8, 1)
// 3 * 2^k: the odd radix as the middle stage (the first and last stay even
// for the padded loads and the cropped stores)
FSP_CFG(float, 48, 12, 16, 4, 3, 4)
FSP_CFG(float, 96, 24, 16, 4, 3, 8)
FSP_CFG(float, 192, 24, 16, 8, 3, 8)
FSP_CFG(float, 384, 24, 16, 8, 6, 8)
// 5 * 2^k (N = 160): radix 5 in the middle
FSP_CFG(float, 160, 40, 16, 4, 5, 8)
FSP_CFG(float, 320, 40, 16, 8, 5, 8)
FSP_CFG(float, 64, 8, 16, 8, 8, 1)
FSP_CFG(float, 128, 16, 16, 8, 16, 1)
FSP_CFG(float, 256, 16, 16, 16, 16, 1)
FSP_CFG(float, 512, 32, 16, 16, 32, 1)
FSP_CFG(float, 1024, 16, 16, 16, 16, 4)
FSP_CFG(float, 2048, 16, 8, 16, 16, 8)  // column passes of non-cubic boxes only (an axis of 1024)
FSP_CFG(double, 32, 8, 16, 4, 8, 1)
FSP_CFG(double, 48, 12, 8, 4, 3, 4)
FSP_CFG(double, 96, 24, 8, 4, 3, 8)
FSP_CFG(double, 192, 24, 8, 8, 3, 8)
FSP_CFG(double, 384, 24, 8, 8, 6, 8)
FSP_CFG(double, 64, 8, 16, 8, 8, 1)
FSP_CFG(double, 128, 16, 8, 8, 16, 1)
FSP_CFG(double, 256, 16, 8, 16, 16, 1)
FSP_CFG(double, 512, 8, 8, 8, 8, 8)
FSP_CFG(double, 1024, 16, 8, 16, 8, 8)
FSP_CFG(df, 32, 8, 16, 4, 8, 1)
FSP_CFG(df, 64, 8, 16, 8, 8, 1)
FSP_CFG(df, 128, 16, 8, 8, 16, 1)
FSP_CFG(df, 256, 8, 8, 8, 8, 4)
FSP_CFG(df, 512, 8, 8, 8, 8, 8)
FSP_CFG(df, 1024, 16, 8, 16, 8, 8)
#undef FSP_CFG

// A column pass may override its length's shape (each measured on the GB300):
// at n = 1024 the FP32 inverse-only pass (P4) is faster with V = 32, L = 8,
// 32*32 (0.66 vs 0.80 ms at N = 512), the passes with a forward transform with
// V = 16, L = 16, 16*16*4; at n = 512 P4 is faster with V = 16, L = 16,
// 16*16*2 (0.078 vs 0.092 ms at N = 256), P2 and P3 with V = 32, L = 16, 16*32.
template <typename T, int n, int MODE> struct ColCfg : Cfg<T, n> {};
template <> struct ColCfg<float, 1024, COL_INV> {
    static constexpr bool Ok = true;
    static constexpr int V = 32, L = 8, R1 = 32, R2 = 32, R3 = 1;
};
template <> struct ColCfg<float, 512, COL_INV> {
    static constexpr bool Ok = true;
    static constexpr int V = 16, L = 16, R1 = 16, R2 = 16, R3 = 2;
};
template <> struct ColCfg<float, 512, COL_FWD> {
    static constexpr bool Ok = true;
    static constexpr int V = 16, L = 16, R1 = 16, R2 = 16, R3 = 2;
};

template <typename T, int n> constexpr size_t smem_for(int positions) {
    return (size_t)positions * (Cfg<T, n>::L + 1) * sizeof(cx_t<T>);
}

}  // namespace fast
}  // namespace fsp

// --------------------------------------------------------------- launchers
namespace fsp {
namespace fast {

// The per-stage tables of the cubic P3 (ColOpt::TT), gathered from the n
// roots tw[e] = w_n^e so that they hold exactly the values the other
// kernels read: forward stage (radix R2 over Ns = R1) [j][r] = tw[r j n/(R1
// R2)] for j < R1, r < R2, then the inverse's (radix R1 over Ns = R2) [j][r]
// for j < R2, r < R1.
template <typename T, int n, int R1, int R2> __global__ void k_p3_table(cx_t<T> *tw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * n) return;
    constexpr int tws = n / (R1 * R2);
    const int fwd = i < n, ii = fwd ? i : i - n, R = fwd ? R2 : R1;
    const int j = ii / R, r = ii % R;
    tw[n + i] = tw[r * j * tws];
}
template <typename T, int n> constexpr int p3_table_len_n() {
    using K = ColCfg<T, n, COL_FMI>;
    if constexpr (!K::Ok)
        return 0;
    else
        return ColOpt<T, COL_FMI, n>::TT && K::R3 == 1 ? 2 * n : 0;
}
template <typename T, int n> cudaError_t p3_table_fill_n(void *tw2n, cudaStream_t s) {
    if constexpr (p3_table_len_n<T, n>() == 0) {
        return cudaSuccess;
    } else {
        using K = ColCfg<T, n, COL_FMI>;
        static_assert(n % (K::R1 * K::R2) == 0, "stage tables cover the two-stage schedule");
        k_p3_table<T, n, K::R1, K::R2><<<(2 * n + 255) / 256, 256, 0, s>>>(reinterpret_cast<cx_t<T> *>(tw2n));
        return cudaGetLastError();
    }
}

template <typename T, int n, int MODE> cudaError_t launch_col_n(const ColArgs &a, int nbatch, cudaStream_t s) {
    using K = ColCfg<T, n, MODE>;
    if constexpr (!K::Ok) {
        return cudaErrorInvalidValue;
    } else {
        auto kern = col_kernel<T, n, K::V, K::L, K::R1, K::R2, K::R3, MODE, false>();
        const size_t sm = sizeof(cx_t<T>) * n * (K::L + 1) + (ColOpt<T, MODE, n>::TWS ? sizeof(cx_t<T>) * n : 0);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        // N/L full tiles per batch row, plus nbatch/N block rows of Nyquist tiles
        constexpr int N = n / 2;
        static_assert(N % K::L == 0, "tiles must cover k_x < N exactly");
        if (nbatch % N != 0) return cudaErrorInvalidValue;
        dim3 grid((unsigned)(N / K::L), (unsigned)(nbatch + nbatch / N));
        kern<<<grid, K::L * (n / K::V), sm, s>>>(a);
        return cudaGetLastError();
    }
}

// Non-cubic box: lines k_x <= n_x = nlines - 1 (a multiple of L), nbatch a
// multiple of L; ceil(nbatch / n_x) leading block rows hold the Nyquist tiles.
template <typename T, int n, int MODE> cudaError_t launch_col_rg_n(const ColArgs &a, int nbatch, cudaStream_t s) {
    using K = ColCfg<T, n, MODE>;
    if constexpr (!K::Ok) {
        return cudaErrorInvalidValue;
    } else {
        auto kern = col_kernel<T, n, K::V, K::L, K::R1, K::R2, K::R3, MODE, true>();
        const int nx = a.nlines - 1;
        if (nx <= 0 || nx % K::L != 0 || nbatch % K::L != 0) return cudaErrorInvalidValue;
        ColArgs b = a;
        b.nbatch = nbatch;
        b.xrows = (nbatch / K::L + nx / K::L - 1) / (nx / K::L);
        const size_t sm = sizeof(cx_t<T>) * n * (K::L + 1) + (ColOpt<T, MODE, n>::TWS ? sizeof(cx_t<T>) * n : 0);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)(nx / K::L), (unsigned)(nbatch + b.xrows));
        kern<<<grid, K::L * (n / K::V), sm, s>>>(b);
        return cudaGetLastError();
    }
}

template <typename T, int MODE> cudaError_t launch_col_rg(int n, const ColArgs &a, int nbatch, cudaStream_t s) {
    switch (n) {
    case 64: return launch_col_rg_n<T, 64, MODE>(a, nbatch, s);
    case 128: return launch_col_rg_n<T, 128, MODE>(a, nbatch, s);
    case 256: return launch_col_rg_n<T, 256, MODE>(a, nbatch, s);
    case 512: return launch_col_rg_n<T, 512, MODE>(a, nbatch, s);
    case 1024: return launch_col_rg_n<T, 1024, MODE>(a, nbatch, s);
    case 2048: return launch_col_rg_n<T, 2048, MODE>(a, nbatch, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int N, bool R2C> cudaError_t launch_row_n(const RowArgs &a, cudaStream_t s) {
    using K = Cfg<T, N>;
    if constexpr (!K::Ok) {
        return cudaErrorInvalidValue;
    } else {
        constexpr bool lane = LaneRow<T, N, K::V, K::R1, K::R2, K::R3>::ok;
        void (*kern)(const RowArgs);
        size_t sm;
        if constexpr (lane) {
            kern = R2C ? k_lane_r2c<T, N, K::V, K::L, K::R1> : k_lane_c2r<T, N, K::V, K::L, K::R1>;
            sm = lane_row_smem<T, N, K::V, K::L>();
        } else {
            kern = R2C ? k_fast_r2c<T, N, K::V, K::L, K::R1, K::R2, K::R3>
                       : k_fast_c2r<T, N, K::V, K::L, K::R1, K::R2, K::R3>;
            sm = smem_for<T, N>(N + 1);
        }
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)((a.nrows + K::L - 1) / K::L), K::L * (N / K::V), sm, s>>>(a);
        return cudaGetLastError();
    }
}

template <typename T, int MODE> cudaError_t launch_col(int n, const ColArgs &a, int nbatch, cudaStream_t s) {
    switch (n) {
    case 96: return launch_col_n<T, 96, MODE>(a, nbatch, s);
    case 192: return launch_col_n<T, 192, MODE>(a, nbatch, s);
    case 384: return launch_col_n<T, 384, MODE>(a, nbatch, s);
    case 320: return launch_col_n<T, 320, MODE>(a, nbatch, s);
    case 64: return launch_col_n<T, 64, MODE>(a, nbatch, s);
    case 128: return launch_col_n<T, 128, MODE>(a, nbatch, s);
    case 256: return launch_col_n<T, 256, MODE>(a, nbatch, s);
    case 512: return launch_col_n<T, 512, MODE>(a, nbatch, s);
    case 1024: return launch_col_n<T, 1024, MODE>(a, nbatch, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T, bool R2C> cudaError_t launch_row(int N, const RowArgs &a, cudaStream_t s) {
    switch (N) {
    case 48: return launch_row_n<T, 48, R2C>(a, s);
    case 96: return launch_row_n<T, 96, R2C>(a, s);
    case 192: return launch_row_n<T, 192, R2C>(a, s);
    case 160: return launch_row_n<T, 160, R2C>(a, s);
    case 32: return launch_row_n<T, 32, R2C>(a, s);
    case 64: return launch_row_n<T, 64, R2C>(a, s);
    case 128: return launch_row_n<T, 128, R2C>(a, s);
    case 256: return launch_row_n<T, 256, R2C>(a, s);
    case 512: return launch_row_n<T, 512, R2C>(a, s);
    }
    return cudaErrorInvalidValue;
}

#define FSP_FAST_INSTANTIATE(T)                                                                                \
    template <> bool has<T>(int N) {                                                                           \
        return N == 32 || N == 64 || N == 128 || N == 256 || N == 512 ||                                      \
               (N == 48 && Cfg<T, 48>::Ok && Cfg<T, 96>::Ok) || (N == 96 && Cfg<T, 96>::Ok && Cfg<T, 192>::Ok) || \
               (N == 192 && Cfg<T, 192>::Ok && Cfg<T, 384>::Ok) || (N == 160 && Cfg<T, 160>::Ok && Cfg<T, 320>::Ok); \
    }                                                                                                          \
    template <> cudaError_t p1<T>(int N, const RowArgs &a, cudaStream_t s) { return launch_row<T, true>(N, a, s); } \
    template <> cudaError_t p5<T>(int N, const RowArgs &a, cudaStream_t s) { return launch_row<T, false>(N, a, s); } \
    template <> cudaError_t p2<T>(int N, const ColArgs &a, int nb, cudaStream_t s) {                            \
        return launch_col<T, COL_FWD>(2 * N, a, nb, s);                                                        \
    }                                                                                                          \
    template <> cudaError_t p3<T>(int N, const ColArgs &a, int nb, cudaStream_t s) {                            \
        return launch_col<T, COL_FMI>(2 * N, a, nb, s);                                                        \
    }                                                                                                          \
    template <> int p3_table_len<T>(int N) {                                                                   \
        switch (N) {                                                                                           \
        case 32: return p3_table_len_n<T, 64>();                                                               \
        case 64: return p3_table_len_n<T, 128>();                                                              \
        case 128: return p3_table_len_n<T, 256>();                                                             \
        case 256: return p3_table_len_n<T, 512>();                                                             \
        }                                                                                                      \
        return 0;                                                                                              \
    }                                                                                                          \
    template <> cudaError_t p3_table_fill<T>(int N, void *tw2n, cudaStream_t s) {                               \
        switch (N) {                                                                                           \
        case 32: return p3_table_fill_n<T, 64>(tw2n, s);                                                       \
        case 64: return p3_table_fill_n<T, 128>(tw2n, s);                                                      \
        case 128: return p3_table_fill_n<T, 256>(tw2n, s);                                                     \
        case 256: return p3_table_fill_n<T, 512>(tw2n, s);                                                     \
        }                                                                                                      \
        return cudaSuccess;                                                                                    \
    }                                                                                                          \
    template <> cudaError_t p4<T>(int N, const ColArgs &a, int nb, cudaStream_t s) {                            \
        return launch_col<T, COL_INV>(2 * N, a, nb, s);                                                        \
    }

// the column passes of non-cubic boxes (runtime geometry), in translation
// units of their own
#define FSP_FAST_RG_INSTANTIATE(T)                                                                             \
    template <> bool has_col_rg<T>(int n) {                                                                    \
        switch (n) {                                                                                           \
        case 64: return Cfg<T, 64>::Ok;                                                                        \
        case 128: return Cfg<T, 128>::Ok;                                                                      \
        case 256: return Cfg<T, 256>::Ok;                                                                      \
        case 512: return Cfg<T, 512>::Ok;                                                                      \
        case 1024: return Cfg<T, 1024>::Ok;                                                                    \
        case 2048: return Cfg<T, 2048>::Ok;                                                                    \
        }                                                                                                      \
        return false;                                                                                          \
    }                                                                                                          \
    template <> cudaError_t col_rg<T>(int mode, int n, const ColArgs &a, int nb, cudaStream_t s) {              \
        switch (mode) {                                                                                        \
        case COL_FWD: return launch_col_rg<T, COL_FWD>(n, a, nb, s);                                           \
        case COL_INV: return launch_col_rg<T, COL_INV>(n, a, nb, s);                                           \
        case COL_FMI: return launch_col_rg<T, COL_FMI>(n, a, nb, s);                                           \
        }                                                                                                      \
        return cudaErrorInvalidValue;                                                                          \
    }

// the field's P3 (odd spectrum), in translation units of its own
#define FSP_FAST_FIELD_INSTANTIATE(T)                                                                          \
    template <> cudaError_t p3_odd<T>(int N, const ColArgs &a, int nb, cudaStream_t s) {                        \
        return launch_col<T, COL_FMO>(2 * N, a, nb, s);                                                        \
    }

}  // namespace fast
}  // namespace fsp
