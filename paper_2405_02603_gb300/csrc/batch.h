// batch.h -- device descriptors of the persistent batched kernel (batch.cu).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace fsp {

// One solve of a batch: the argument blocks of its five passes.
struct BatchSolve {
    RowsArgs r1, r5;           // P1 (x = rho), P5 (x = phi)
    LinesArgs c2, c3, c4;      // P2, P3, P4
    int ntx;                   // column tiles per batch index
    int ntiles[5];
};

// A run of consecutive work items: the tiles of one pass of one solve.
struct BatchSeg {
    int solve, pass, first, ntiles;
    int need_prev;  // tiles of the previous pass that must be done first
};

// Per-launch control block, zeroed before every launch.
struct BatchCtl {
    int cursor;
    int status;
    int done[1];  // 5 * nsolves counters (allocated beyond the struct)
};

struct BatchLaunch {
    const BatchSolve *solves;
    const BatchSeg *segs;
    int nseg, total;
    BatchCtl *ctl;
    unsigned long long timeout_ns;
    unsigned grid;
    int threads;
    size_t smem;
};

template <typename T> cudaError_t launch_batch_kernel(const BatchLaunch &L, cudaStream_t s);
template <typename T> int batch_blocks_per_sm(int threads, size_t smem);

}  // namespace fsp
