// FP32-mixed psi^3 row-pass kernels with compile-time row lengths.
#include "pfc_row_fixed.cuh"

namespace pfc {
PFC_INSTANTIATE_ROW_FIXED(float)
}  // namespace pfc
