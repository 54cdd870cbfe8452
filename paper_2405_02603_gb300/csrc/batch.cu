// batch.cu -- many independent solves of mixed sizes in one persistent launch
// (the batched systems form; the paper solves one grid at a time).
//
// Work list: every solve contributes 5 segments (P1..P5) of tiles; segments
// are ordered pass-major (all P1 segments, then all P2, ...).  Each CTA of the
// persistent kernel repeatedly takes the next item with an atomic cursor.  A
// tile of pass p > 0 first waits until all tiles of pass p-1 of the same solve
// are done (a per-(solve, pass) counter).  Because items are taken in index
// order, every item a CTA waits for has a smaller index and was taken by a
// running CTA, so the waits always end.  Each wait is nevertheless bounded by
// a time limit (%globaltimer): on expiry the CTA records FSP_ETIMEOUT in a
// status word that every CTA checks before taking work, and the launch ends
// normally so that the host can read the status and the context stays usable.
//
// Memory ordering: a finished tile is published with barrier + fence + atomic
// increment by thread 0; the consumer's thread 0 reads the counter with
// acquire semantics before a barrier, and all tiles of this kernel read
// workspace data through L2 (ld.global.cg), since L1 is not coherent.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/fsp.h"
#include "batch.h"
#include "kernels_impl.cuh"

namespace fsp {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__global__ void __launch_bounds__(512) k_batch(const BatchSolve *__restrict__ solves, const BatchSeg *__restrict__ segs,
                                               int nseg, int total, BatchCtl *ctl, unsigned long long timeout_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_seg, s_stop;
    // the current tile's argument block, staged in shared memory so that the
    // tile code reads its fields from there (a reference into global memory
    // makes ptxas spill the engine's registers)
    __shared__ __align__(16) union {
        RowsArgs r;
        LinesArgs l;
    } s_args;
    for (;;) {
        if (threadIdx.x == 0) {
            cuda::atomic_ref<int, cuda::thread_scope_device> status(ctl->status);
            int item = total, seg = -1, stop = 0;
            if (status.load(cuda::memory_order_relaxed) == 0) item = atomicAdd(&ctl->cursor, 1);
            if (item < total) {
                int lo = 0, hi = nseg - 1;  // last segment with first <= item
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (segs[mid].first <= item)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                seg = lo;
                const BatchSeg g = segs[seg];
                if (g.pass > 0) {
                    const int need = g.need_prev;
                    cuda::atomic_ref<int, cuda::thread_scope_device> prev(ctl->done[g.solve * 5 + g.pass - 1]);
                    const unsigned long long t0 = global_ns();
                    unsigned sleep = 32;
                    while (prev.load(cuda::memory_order_acquire) < need) {
                        if (status.load(cuda::memory_order_relaxed) != 0) {
                            stop = 1;
                            break;
                        }
                        if (global_ns() - t0 > timeout_ns) {
                            int expected = 0;
                            status.compare_exchange_strong(expected, (int)FSP_ETIMEOUT);
                            stop = 1;
                            break;
                        }
                        __nanosleep(sleep);
                        if (sleep < 2048) sleep <<= 1;
                    }
                }
            }
            s_item = item, s_seg = seg, s_stop = stop;
        }
        __syncthreads();
        const int item = s_item, seg = s_seg;
        if (item >= total || s_stop) break;
        const BatchSeg g = segs[seg];
        const int tile = item - g.first;
        const BatchSolve &sv = solves[g.solve];
        {
            const void *src = g.pass == 0   ? (const void *)&sv.r1
                              : g.pass == 1 ? (const void *)&sv.c2
                              : g.pass == 2 ? (const void *)&sv.c3
                              : g.pass == 3 ? (const void *)&sv.c4
                                            : (const void *)&sv.r5;
            const int words = (g.pass == 0 || g.pass == 4) ? (int)(sizeof(RowsArgs) / 4) : (int)(sizeof(LinesArgs) / 4);
            for (int w = threadIdx.x; w < words; w += blockDim.x)
                reinterpret_cast<int *>(&s_args)[w] = reinterpret_cast<const int *>(src)[w];
        }
        const int ntx = sv.ntx;
        __syncthreads();
        switch (g.pass) {
        case 0: r2c_tile<T, true>(s_args.r, tile, smem_raw); break;
        case 1: lines_tile<T, IN_CPLX, OUT_CPLX, M_FWD, true>(s_args.l, tile % ntx, tile / ntx, smem_raw); break;
        case 2: lines_tile<T, IN_CPLX, OUT_CPLX, M_FWD_MUL_INV, true>(s_args.l, tile % ntx, tile / ntx, smem_raw); break;
        case 3: lines_tile<T, IN_CPLX, OUT_CPLX, M_INV, true>(s_args.l, tile % ntx, tile / ntx, smem_raw); break;
        default: c2r_tile<T, true>(s_args.r, tile, smem_raw); break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            cuda::atomic_ref<int, cuda::thread_scope_device> d(ctl->done[g.solve * 5 + g.pass]);
            d.fetch_add(1, cuda::memory_order_release);
        }
    }
}

// The caller sets the shared-memory attribute beforehand (batch_blocks_per_sm)
// so that this launch can be captured into a graph.
template <typename T> cudaError_t launch_batch_kernel(const BatchLaunch &L, cudaStream_t s) {
    k_batch<T><<<L.grid, L.threads, L.smem, s>>>(L.solves, L.segs, L.nseg, L.total, L.ctl, L.timeout_ns);
    return cudaGetLastError();
}

template <typename T> int batch_blocks_per_sm(int threads, size_t smem) {
    int nb = 0;
    cudaFuncSetAttribute(k_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<T>, threads, smem) != cudaSuccess) return 0;
    return nb;
}

template cudaError_t launch_batch_kernel<float>(const BatchLaunch &, cudaStream_t);
template cudaError_t launch_batch_kernel<double>(const BatchLaunch &, cudaStream_t);
template int batch_blocks_per_sm<float>(int, size_t);
template int batch_blocks_per_sm<double>(int, size_t);

}  // namespace fsp
