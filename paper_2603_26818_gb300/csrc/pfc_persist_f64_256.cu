// FP64 instantiation of the persistent batch kernel (pfc_persist.cuh), 256-thread blocks.
#include "pfc_persist_launch.cuh"

namespace pfc {
PFC_INSTANTIATE_PERSIST(double, 256)
}  // namespace pfc
