// kernels_f64.cu -- double-precision instantiation of the line kernels (the
// FSP_F64 solve and every plan-time transform, which always runs in FP64).
#include "kernels_impl.cuh"

namespace fsp {
FSP_INSTANTIATE(double)
// plan-time forms: DCT-I of real lines (Sec. 2.4), DST-I of real lines (the
// field kernels' odd axis) and the real part of the last inverse pass of the
// (4N)^3 transform (Sec. 2.3)
template cudaError_t launch_lines<double, IN_REAL_EVEN, OUT_REAL, M_FWD>(const LinesArgs &, cudaStream_t);
template cudaError_t launch_lines<double, IN_REAL_ODD, OUT_REAL, M_FWD>(const LinesArgs &, cudaStream_t);
template cudaError_t launch_lines<double, IN_CPLX, OUT_REAL, M_INV>(const LinesArgs &, cudaStream_t);
}  // namespace fsp
