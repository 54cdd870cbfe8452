// kernels_f32.cu -- single-precision instantiation of the line kernels
// (the FSP_F32_MIXED solve).
#include "kernels_impl.cuh"

namespace fsp {
FSP_INSTANTIATE(float)
}  // namespace fsp
