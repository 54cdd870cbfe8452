// fast_field.h -- host interface of the field's P3 on non-cubic boxes: the
// odd-spectrum column pass (COL_FMO) with runtime geometry, instantiated with
// the cubic field P3 in fast_{f32,f64,df}_field.cu.
#pragma once
#include <cuda_runtime.h>

#include "fast.h"

namespace fsp {
namespace fast {

// z-FFT * (-i S_a, odd in the axis a.odd) * z-IFFT of length n, strides from
// `a`, lines k_x <= a.nlines - 1, the k_y fold at a.half_b
template <typename T> cudaError_t p3_odd_rg(int n, const ColArgs &a, int nbatch, cudaStream_t s);

}  // namespace fast
}  // namespace fsp
