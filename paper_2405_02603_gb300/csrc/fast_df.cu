// fast_df.cu -- double-float instantiation of the specialised passes (the
// FSP_F64_DF solve) and of its roots tables.
#include "fast.cuh"
#include "kernels_impl.cuh"

namespace fsp {
namespace fast {
FSP_FAST_INSTANTIATE(df)
}  // namespace fast
template cudaError_t launch_roots<df>(void *, int, cudaStream_t);
}  // namespace fsp
