// fast_f32_rg.cu -- FP32 instantiation of the specialised column passes with
// runtime geometry (non-cubic boxes), apart from the cubic ones so that the
// translation units compile in parallel.
#include "fast.cuh"

namespace fsp {
namespace fast {
FSP_FAST_RG_INSTANTIATE(float)
}  // namespace fast
}  // namespace fsp
