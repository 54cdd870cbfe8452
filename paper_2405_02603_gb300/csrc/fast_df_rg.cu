// fast_df_rg.cu -- double-float instantiation of the specialised column passes with
// runtime geometry (non-cubic boxes), apart from the cubic ones so that the
// translation units compile in parallel.
#include "fast.cuh"

namespace fsp {
namespace fast {
FSP_FAST_RG_INSTANTIATE(df)
}  // namespace fast
}  // namespace fsp
