// fast_f64.cu -- double-precision instantiation of the specialised passes.
#include "fast.cuh"

namespace fsp {
namespace fast {
FSP_FAST_INSTANTIATE(double)
}  // namespace fast
}  // namespace fsp
