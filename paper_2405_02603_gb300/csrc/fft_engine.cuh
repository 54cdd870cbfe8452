// fft_engine.cuh -- shared-memory mixed-radix (2/3/4/5/8) Stockham FFT engine
// for batches of lines, the building block of every transform of the solver
// (the FFTs of Sec. 2.2 step 4 and the plan-time transforms of Sec. 2.3/2.4).
//
// Layout: a CTA holds L = 2^lgL lines of one length-n transform in shared
// memory, element (line l, position p) at buf[p*ld + l] with an odd pitch
// ld = L + 1, so that both "all lines at one position" (column) and "one line
// at consecutive positions" (row) accesses are free of bank conflicts.
// Thread t works on line l = t & (L-1) as sub-thread sub = t >> lgL of tpl.
//
// Stage s with radix R and Ns = product of the earlier radices performs, for
// each butterfly b in [0, n/R):
//   v[r] = buf[b + r n/R] * w_n^(r (b mod Ns) n/(Ns R)),  r in [0,R)
//   v    = DFT_R(v)
//   buf[(b - b mod Ns) R + b mod Ns + r Ns] = v[r]
// (decimation in time, self-sorting: natural order in and out).  All loads of
// a stage complete (barrier) before any store, so one buffer suffices.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace fsp {

template <typename T> struct cx;
template <> struct cx<float> { using t = float2; };
template <> struct cx<double> { using t = double2; };
template <typename T> using cx_t = typename cx<T>::t;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
// FP32 complex sums as one packed two-float instruction (add/sub .f32x2,
// sm_100 and later): each component is rounded exactly as by the scalar add,
// in half the issue slots.  Used where a kernel measured faster with them
// (the register DFTs' PK option).
__device__ __forceinline__ float2 cadd_pk(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __fadd2_rn(a, b);
#else
    return cadd(a, b);
#endif
}
__device__ __forceinline__ float2 csub_pk(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pr, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
#else
    return csub(a, b);
#endif
}

template <typename C> __device__ __forceinline__ C ldg_c(const C *p) { return __ldg(p); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// multiply by i and by -i
template <typename C> __device__ __forceinline__ C cmuli(C a) { return C{-a.y, a.x}; }
template <typename C> __device__ __forceinline__ C cmulmi(C a) { return C{a.y, -a.x}; }

constexpr int kMaxV = 16;  // complex values a thread holds within one stage

// Compile-time loop: f(integral_constant<int, I>) for I in [B, E).
template <int B, int E> struct Unroll {
    template <class F> static __device__ __forceinline__ void run(F &&f) {
        if constexpr (B < E) {
            f(std::integral_constant<int, B>{});
            Unroll<B + 1, E>::run(f);
        }
    }
};

// Radix schedule of a length-n transform, always in the order: n5 radix-5
// stages, n3 radix-3 stages, n8 radix-8 stages, then one radix-`last` stage
// (last = 4, 2 or 0 for none).  A fixed order keeps each radix in its own
// loop, so the register arrays of different radices never share a live range.
struct Stages {
    int n;
    int n5, n3, n8, last;
};

// Size-R DFT in registers, v'[q] = sum_r v[r] exp(D 2 pi i r q / R), D = -1
// (forward) or +1 (inverse).
template <typename T, int D> struct Dft {
    using C = cx_t<T>;
    // the sign-dependent multiply by -i (forward) / +i (inverse): exp(D i pi/2)
    static __device__ __forceinline__ C rot(C a) { return D < 0 ? cmulmi(a) : cmuli(a); }

    static __device__ __forceinline__ void r2(C *v) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
    static __device__ __forceinline__ void r3(C *v) {
        // exp(D 2 pi i/3) = -1/2 + D i sqrt(3)/2
        const T h = T(0.5), s = T(0.86602540378443864676372317075294);
        C t = cadd(v[1], v[2]);
        C d = csub(v[1], v[2]);
        C m = C{v[0].x - h * t.x, v[0].y - h * t.y};
        // D i s d
        C sd = C{-T(D) * s * d.y, T(D) * s * d.x};
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, sd);
        v[2] = csub(m, sd);
    }
    static __device__ __forceinline__ void r4(C *v) {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = rot(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
    static __device__ __forceinline__ void r5(C *v) {
        // c1 = cos(2pi/5), c2 = cos(4pi/5), s1 = sin(2pi/5), s2 = sin(4pi/5)
        const T c1 = T(0.30901699437494742410229341718282), c2 = T(-0.80901699437494742410229341718282);
        const T s1 = T(0.95105651629515357211643933337938), s2 = T(0.58778525229247312916870595463907);
        C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        C x0 = v[0];
        C m1 = C{x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y};
        C m2 = C{x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y};
        // n1 = s1 b1 + s2 b2, n2 = s2 b1 - s1 b2; X1 = m1 + D i n1, X2 = m2 + D i n2
        C n1 = C{s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y};
        C n2 = C{s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y};
        C in1 = C{-T(D) * n1.y, T(D) * n1.x};
        C in2 = C{-T(D) * n2.y, T(D) * n2.x};
        v[0] = C{x0.x + a1.x + a2.x, x0.y + a1.y + a2.y};
        v[1] = cadd(m1, in1);
        v[4] = csub(m1, in1);
        v[2] = cadd(m2, in2);
        v[3] = csub(m2, in2);
    }
    static __device__ __forceinline__ void r8(C *v) {
        // two radix-4 on even / odd inputs, then combine with exp(D i pi q/4)
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        r4(e);
        r4(o);
        const T r = T(0.70710678118654752440084436210485);
        // o1 *= exp(D i pi/4) = r (1 + D i); o2 *= D i; o3 *= exp(3 D i pi/4) = r (-1 + D i)
        C o1 = C{r * (o[1].x - T(D) * o[1].y), r * (o[1].y + T(D) * o[1].x)};
        C o2 = C{-T(D) * o[2].y, T(D) * o[2].x};
        C o3 = C{r * (-o[3].x - T(D) * o[3].y), r * (-o[3].y + T(D) * o[3].x)};
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <typename T, int D> struct Engine {
    using C = cx_t<T>;

    // exp(D 2 pi i e / n) from the forward table tw[e] = exp(-2 pi i e / n)
    static __device__ __forceinline__ C twid(const C *__restrict__ tw, int e) {
        C w = tw[e];
        if (D > 0) w.y = -w.y;
        return w;
    }

    // The loops over butterflies and over the radix are unrolled by
    // construction (Unroll), not by pragma: inside an outer loop (the
    // persistent batched kernel) pragma unrolling is not guaranteed, and a
    // partially unrolled loop would send the register array v to local memory.
    template <int R>
    static __device__ __forceinline__ void stage(C *buf, int ld, int n, int Ns, const C *__restrict__ tw, int l,
                                                 int sub, int tpl, bool act) {
        constexpr int KMAX = kMaxV / R;
        const int nb = n / R;
        // Defined on entry: the loads below are predicated, and inside an outer
        // loop an array that might be read before written stays live around
        // the back-edge, so ptxas keeps every radix's array allocated at once.
        C v[KMAX * R];
        Unroll<0, KMAX * R>::run([&](auto ic) { v[decltype(ic)::value] = C{T(0), T(0)}; });
        Unroll<0, KMAX>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const int b = sub + k * tpl;
            if (act && b < nb) {
                Unroll<0, R>::run([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    v[k * R + r] = buf[(b + r * nb) * ld + l];
                });
            }
        });
        __syncthreads();
        const int tws = n / (Ns * R);
        Unroll<0, KMAX>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const int b = sub + k * tpl;
            if (act && b < nb) {
                const int j = b % Ns;
                if (j != 0) {
                    Unroll<1, R>::run([&](auto rc) {
                        constexpr int r = decltype(rc)::value;
                        v[k * R + r] = cmul(v[k * R + r], twid(tw, r * j * tws));
                    });
                }
                if constexpr (R == 2) Dft<T, D>::r2(v + k * R);
                if constexpr (R == 3) Dft<T, D>::r3(v + k * R);
                if constexpr (R == 4) Dft<T, D>::r4(v + k * R);
                if constexpr (R == 5) Dft<T, D>::r5(v + k * R);
                if constexpr (R == 8) Dft<T, D>::r8(v + k * R);
                const int base = (b - j) * R + j;
                Unroll<0, R>::run([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    buf[(base + r * Ns) * ld + l] = v[k * R + r];
                });
            }
        });
        __syncthreads();
    }

    // Transform all lines held in buf in place.  Every thread of the CTA must
    // call this (it contains barriers); `act` only gates the arithmetic.
    static __device__ __forceinline__ void run(C *buf, int ld, const Stages &st, const C *__restrict__ tw, int l,
                                               int sub, int tpl, bool act) {
        int Ns = 1;
        for (int s = 0; s < st.n5; ++s, Ns *= 5) stage<5>(buf, ld, st.n, Ns, tw, l, sub, tpl, act);
        for (int s = 0; s < st.n3; ++s, Ns *= 3) stage<3>(buf, ld, st.n, Ns, tw, l, sub, tpl, act);
        for (int s = 0; s < st.n8; ++s, Ns *= 8) stage<8>(buf, ld, st.n, Ns, tw, l, sub, tpl, act);
        if (st.last == 4) stage<4>(buf, ld, st.n, Ns, tw, l, sub, tpl, act);
        if (st.last == 2) stage<2>(buf, ld, st.n, Ns, tw, l, sub, tpl, act);
    }
};

}  // namespace fsp
