// fast_f64_field.cu -- FP64 instantiation of the field's P3 (the odd
// spectrum of E = -grad phi) on cubic and non-cubic boxes, kept apart from the
// solve's passes so that the translation units compile in parallel.
#include "fast.cuh"
#include "fast_field.h"

namespace fsp {
namespace fast {
FSP_FAST_FIELD_INSTANTIATE(double)
template <> cudaError_t p3_odd_rg<double>(int n, const ColArgs &a, int nb, cudaStream_t s) {
    return launch_col_rg<double, COL_FMO>(n, a, nb, s);
}
}  // namespace fast
}  // namespace fsp
