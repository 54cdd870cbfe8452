// p3_tma.cuh -- P3 (z-FFT * S * z-IFFT, crop z; Sec. 2.2 steps 2-5 along
// the last axis) as a persistent kernel whose input tiles are staged in
// shared memory by the tensor memory accelerator.
//
// The register-resident transform is the one of k_fast_col<COL_FMI>
// (fast.cuh); what differs is how a tile's inputs arrive and the order in
// which a CTA takes tiles:
//  * each CTA owns a contiguous run of tiles.  A tile is L consecutive k_x
//    lines of one k_y row, z in [0, N): one 3D cp.async.bulk.tensor box of
//    L x 1 x N complex values (128-byte rows), completed on an mbarrier.
//    As soon as the current tile's stage-0 values are in registers the next
//    tile's box is requested, so its HBM latency overlaps the whole
//    transform of the current one (the register-direct kernel has nothing in
//    flight while it computes);
//  * within a block of k_x lines the k_y rows are ordered 0, N, 1, 2N-1, 2,
//    2N-2, ...: the two rows that fold to the same spectrum row (k_y and
//    2N - k_y) run back to back on one CTA, so the second finds its spectrum
//    values in L1 and S is read from HBM about once;
//  * the Nyquist column k_x = N (lines 8 KB apart, not a box of rows) runs in
//    the first tiles with register-direct loads, as in k_fast_col.
// Every wait on the mbarrier is bounded by %globaltimer: on expiry the CTA
// records the timeout in the caller's error word, waits (bounded again) for
// its copy in flight and returns; the launch ends with the context usable.
#pragma once
#include <cuda.h>

#include "fast.cuh"

namespace fsp {
namespace fast {

__device__ __forceinline__ unsigned long long tma_gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// true once the phase of the given parity has completed; false after
// timeout_ns nanoseconds without completion
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned long long timeout_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = tma_gtimer();
    while (!mbar_try(bar, parity))
        if (tma_gtimer() - t0 > timeout_ns) return false;
    return true;
}

// One thread: expect `bytes` on the barrier and request the box at (x, y, z).
__device__ __forceinline__ void tma_box3(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar,
                                         uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

struct P3TmaArgs {
    void *w2;          // W2[z][k_y][k_x], pitch P (in place)
    const void *S;     // S[q_z][q_y][q_x], pitch P
    const void *tw;    // forward roots of length 2N
    unsigned *err;     // bit 0 set when a wait timed out
    unsigned long long timeout_ns;
    unsigned extra_tx; // fault injection: bytes expected beyond each box (0)
    int ntiles_nyq;    // Nyquist tiles (first)
    int ntiles;        // all tiles
};

// the register-direct P3's options with the roots-table placement chosen here
template <typename T, int n, bool TWS_> struct ColOptP3 {
    static constexpr bool PF = ColOpt<T, COL_FMI, n>::PF, TWS = TWS_;
};

// Bytes of shared memory: exchange buffer, roots table (TWS), staging box,
// mbarrier.
template <typename T, int n, int L, bool TWS> constexpr size_t p3_tma_stage_off() {
    return (sizeof(cx_t<T>) * n * (L + 1) + (TWS ? sizeof(cx_t<T>) * n : 0) + 127) / 128 * 128;
}
template <typename T, int n, int L, bool TWS> constexpr size_t p3_tma_smem() {
    return p3_tma_stage_off<T, n, L, TWS>() + sizeof(cx_t<T>) * (n / 2) * L + 16;
}

template <typename T, int n, int V, int L, int R1, int R2, int R3, bool TWS_>
__global__ void __launch_bounds__(L *(n / V), 2) k_p3_tma(const __grid_constant__ CUtensorMap tmap, const P3TmaArgs a) {
    using C = cx_t<T>;
    using G = ColGeo<n, COL_FMI>;
    using O = ColOptP3<T, n, TWS_>;
    constexpr int TPL = n / V, N = G::N, NTH = L * TPL;
    constexpr int RL = LastR<R1, R2, R3>::value;
    constexpr uint32_t BOX_BYTES = (uint32_t)(sizeof(C) * N * L);
    constexpr int XE = (int)(sizeof(C) / 4);  // 4-byte tensor elements per complex value
    static_assert(N <= 256, "one box covers the N positions of a tile");
    extern __shared__ __align__(128) unsigned char p3_smem[];
    C *buf = reinterpret_cast<C *>(p3_smem);
    const C *stg = reinterpret_cast<const C *>(p3_smem + p3_tma_stage_off<T, n, L, TWS_>());
    uint64_t *barp = reinterpret_cast<uint64_t *>(p3_smem + p3_tma_stage_off<T, n, L, TWS_>() + sizeof(C) * N * L);
    const uint32_t bar = smem_addr(barp), stg_s = smem_addr(stg);
    const int l = threadIdx.x % L, t = threadIdx.x / L;

    const C *tw = reinterpret_cast<const C *>(a.tw);
    if constexpr (O::TWS) {
        C *tws = buf + (size_t)n * (L + 1);
        for (int e = threadIdx.x; e < n; e += NTH) tws[e] = ldg_c(tw + e);
        tw = tws;
    }
    // CTA b: Nyquist tile b (b < ntiles_nyq <= gridDim.x), then a contiguous
    // run of main tiles; every CTA takes floor or ceil(ntiles / gridDim.x)
    // tiles.  Tile index i < ntiles_nyq: Nyquist tile i; else main tile
    // i - ntiles_nyq.
    const int b = blockIdx.x, nq = a.ntiles_nyq;
    const int m0 = (int)((long long)b * a.ntiles / gridDim.x) - min(b, nq);
    const int m1 = (int)((long long)(b + 1) * a.ntiles / gridDim.x) - min(b + 1, nq);
    const int i0 = b < nq ? b : nq + m0;  // first tile
    const int cnt = (b < nq ? 1 : 0) + (m1 - m0);
    auto tile_at = [&](int q) { return b < nq ? (q == 0 ? b : nq + m0 + q - 1) : nq + m0 + q; };
    // main tile u: block xb of L lines, k_y in the order 0, N, 1, 2N-1, 2, ...
    auto main_tile = [&](int i, int &x0, int &ky) {
        const int u = i - a.ntiles_nyq;
        const int j = u % (2 * N);
        x0 = (u / (2 * N)) * L;
        ky = j == 0 ? 0 : j == 1 ? N : (j & 1) ? 2 * N - ((j - 2) / 2 + 1) : (j - 2) / 2 + 1;
    };
    auto request = [&](int i) {
        int x0, ky;
        main_tile(i, x0, ky);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tma_box3(stg_s, &tmap, x0 * XE, ky, 0, bar, BOX_BYTES + a.extra_tx);
    };
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (cnt > 0 && i0 >= nq) request(i0);
    }
    __syncthreads();
    uint32_t parity = 0;
    C *W2 = reinterpret_cast<C *>(a.w2);
    const T *Sb = reinterpret_cast<const T *>(a.S);

    for (int q = 0; q < cnt; ++q) {
        const int i = tile_at(q);
        const bool is_main = i >= nq;
        int line;
        long long bt;
        C v[V];
        if (is_main) {
            int x0, ky;
            main_tile(i, x0, ky);
            line = x0 + l, bt = ky;
            const bool ok = mbar_wait_bounded(bar, parity, a.timeout_ns);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    atomicOr(a.err, 1u);
                    mbar_wait_bounded(bar, parity, a.timeout_ns);  // the copy in flight
                }
                return;
            }
            parity ^= 1u;
            StaticFor<0, V / R1>::run([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                StaticFor<0, R1 / 2>::run([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    constexpr int c = k * TPL + r * (n / R1);
                    v[k * R1 + r] = stg[(t + c) * L + l];
                });
            });
        } else {
            line = N, bt = (long long)i * L + l;
            const C *in_t = W2 + bt * G::IN_BATCH + line + (long long)t * G::IN_POS;
            StaticFor<0, V / R1>::run([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                StaticFor<0, R1 / 2>::run([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    constexpr long long c = k * TPL + r * (n / R1);
                    v[k * R1 + r] = ldcg_c(in_t + c * G::IN_POS);
                });
            });
        }
        // every thread is done with the staging box (and with the exchange
        // buffer of the previous tile): the next box may land
        __syncthreads();
        if (threadIdx.x == 0 && q + 1 < cnt) request(tile_at(q + 1));  // always a main tile

        const int fy = (int)bt <= N ? (int)bt : 2 * N - (int)bt;
        const T *Sy = Sb + (long long)fy * G::S_BATCH + line;
        if constexpr (O::PF) {
            StaticFor<0, V / RL>::run([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                StaticFor<0, RL>::run([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    constexpr int c = k * TPL + r * (n / RL);
                    const int p = t + c;
                    const int fz = p <= N ? p : n - p;
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(Sy + (long long)fz * G::S_POS));
                });
            });
        }
        Stg<T, -1, n, V, L, O::TWS>::template compute<R1, 1, true, false>(v, t, tw);
        run_rest<T, -1, n, V, L, R1, R2, R3, false, O::TWS>(v, buf, t, l, tw, false);

        // multiply by the real, even spectrum at the folded frequency
        const T *S_up = Sy + (long long)t * G::S_POS, *S_dn = Sy - (long long)t * G::S_POS;
        StaticFor<0, V / RL>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            StaticFor<0, RL>::run([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                constexpr int c = k * TPL + r * (n / RL);
                T s;
                if constexpr (c + TPL - 1 <= N) {
                    s = S_up[(long long)c * G::S_POS];
                } else if constexpr (c > N) {
                    s = S_dn[(long long)(n - c) * G::S_POS];
                } else {
                    const int p = t + c;
                    const int fz = p <= N ? p : n - p;
                    s = Sy[(long long)fz * G::S_POS];
                }
                v[k * RL + r].x *= s;
                v[k * RL + r].y *= s;
            });
        });
        using SI = Stg<T, +1, n, V, L, O::TWS>;
        if constexpr (R3 > 1) {
            SI::template compute<R3, 1, false, false>(v, t, tw);
            run_rest<T, +1, n, V, L, R3, R2, R1, true, O::TWS>(v, buf, t, l, tw, true);
        } else {
            SI::template compute<R2, 1, false, false>(v, t, tw);
            run_rest<T, +1, n, V, L, R2, R1, 1, true, O::TWS>(v, buf, t, l, tw, true);
        }
        C *out_t = W2 + bt * G::OUT_BATCH + line + (long long)t * G::OUT_POS;
        constexpr int RF = R1;
        StaticFor<0, V / RF>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            StaticFor<0, RF / 2>::run([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                constexpr long long c = k * TPL + r * (n / RF);
                out_t[c * G::OUT_POS] = v[k * RF + r];
            });
        });
    }
}

}  // namespace fast
}  // namespace fsp
