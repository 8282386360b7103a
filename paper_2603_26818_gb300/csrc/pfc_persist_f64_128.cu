// FP64 instantiation of the persistent batch kernel (pfc_persist.cuh), 128-thread blocks.
#include "pfc_persist_launch.cuh"

namespace pfc {
PFC_INSTANTIATE_PERSIST(double, 128)
}  // namespace pfc
