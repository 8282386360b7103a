// FP32-mixed instantiation of the persistent batch kernel (pfc_persist.cuh), 512-thread blocks.
#include "pfc_persist_launch.cuh"

namespace pfc {
PFC_INSTANTIATE_PERSIST(float, 512)
}  // namespace pfc
