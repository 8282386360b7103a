// Launch functions of the persistent batch kernel (declared in pfc_launch.h); included by the
// per-precision translation units only.
#pragma once

#include "pfc_launch.h"

namespace pfc {

// One cooperative launch of grid blocks of NT threads (all resident at once, or the launch
// fails with cudaErrorCooperativeLaunchTooLarge).
template <typename R, int NT>
cudaError_t launch_batch_persist(const PbArgs<R> &a, int grid, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_persist<R, NT>, a);
}

// Allows smem bytes of dynamic shared memory and returns the blocks of NT threads that fit an SM.
template <typename R, int NT> cudaError_t persist_occupancy(size_t smem, int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_persist<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_persist<R, NT>, NT, smem);
}

#define PFC_INSTANTIATE_PERSIST(R, NT)                                                             \
    template cudaError_t launch_batch_persist<R, NT>(const PbArgs<R> &, int, size_t, cudaStream_t); \
    template cudaError_t persist_occupancy<R, NT>(size_t, int *);

}  // namespace pfc
