// FP32-mixed update-pass kernels with compile-time y transform lengths.
#include "pfc_line_fixed.cuh"

namespace pfc {
PFC_INSTANTIATE_LINE_FIXED(float)
}  // namespace pfc
