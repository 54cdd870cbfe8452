// fast_f32.cu -- single-precision instantiation of the specialised passes.
#include "fast.cuh"

namespace fsp {
namespace fast {
FSP_FAST_INSTANTIATE(float)
}  // namespace fast
}  // namespace fsp
