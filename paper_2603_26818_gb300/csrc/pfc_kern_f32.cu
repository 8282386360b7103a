// FP32-mixed instantiation of the pass and reduction kernels.
#include "pfc_kern.cuh"

namespace pfc {
PFC_INSTANTIATE_LAUNCH(float)
}  // namespace pfc
