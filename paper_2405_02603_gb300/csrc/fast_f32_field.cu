// fast_f32_field.cu -- FP32 instantiation of the field's P3 (the odd spectrum
// of E = -grad phi), kept apart from the solve's passes so that the two
// translation units compile in parallel.
#include "fast.cuh"

namespace fsp {
namespace fast {
FSP_FAST_FIELD_INSTANTIATE(float)
}  // namespace fast
}  // namespace fsp
