// internal.h -- what other translation units of the library may read of a
// plan (api.cu owns the plan type): its spectrum, roots tables and generic-
// engine tile shapes.
#pragma once
#include <cuda_runtime.h>

#include "../../include/fsp.h"
#include "tiles.h"

namespace fsp {
namespace internal {

struct PlanView {
    int N = 0, P = 0, device = 0;
    fsp_dtype dtype = FSP_F64;
    size_t rsize = 8;                      // bytes per real of the solve's arrays
    const void *S = nullptr;               // S[q_z][q_y][q_x], pitch P, (N+1)^2 rows
    const void *tw_n = nullptr, *tw_2n = nullptr;  // roots of length N and 2N
    TileCfg row, col;                      // generic engine: rows (length N), columns (length 2N)
};

// A plan that holds the spectrum and the tables but no workspace.
fsp_status spectrum_plan_create(fsp_plan **out, int N, double L, fsp_algo algo, fsp_dtype dtype, cudaStream_t s);
bool plan_view(const fsp_plan *p, PlanView *v);

}  // namespace internal
}  // namespace fsp
