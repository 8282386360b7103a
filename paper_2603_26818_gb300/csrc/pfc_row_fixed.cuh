// psi^3 row-pass kernels with the row transform length 2^LM fixed at compile time, LM in
// [ROW_FIXED_MIN, ROW_FIXED_MAX]; included by the per-precision translation units only.
#pragma once

#include "pfc_launch.h"

namespace pfc {

template <typename R, int LM>
static void launch_row_fixed_t(const LaunchCfg &c, const RowArgs<R> &a, int nf) {
    dim3 grid(c.g.QR / c.g.gpc, nf);
    k_row<R, ROW_CUBE, LM><<<grid, c.nt_row, c.smem_row, c.stream>>>(c.g, a);
}

template <typename R> void launch_row_cube_fixed(const LaunchCfg &c, const RowArgs<R> &a, int nf) {
    switch (c.g.lM) {
        case 5: launch_row_fixed_t<R, 5>(c, a, nf); break;
        case 6: launch_row_fixed_t<R, 6>(c, a, nf); break;
        case 7: launch_row_fixed_t<R, 7>(c, a, nf); break;
        case 8: launch_row_fixed_t<R, 8>(c, a, nf); break;
        case 9: launch_row_fixed_t<R, 9>(c, a, nf); break;
        default: launch_row_fixed_t<R, 10>(c, a, nf); break;
    }
}

template <typename R> cudaError_t set_smem_attrs_row_fixed(const LaunchCfg &c) {
    cudaError_t e;
    const int bytes = (int)c.smem_row;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_row<R, ROW_CUBE, 5>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row<R, ROW_CUBE, 6>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row<R, ROW_CUBE, 7>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row<R, ROW_CUBE, 8>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row<R, ROW_CUBE, 9>, at, bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_row<R, ROW_CUBE, 10>, at, bytes);
}

static_assert(ROW_FIXED_MIN == 5 && ROW_FIXED_MAX == 10, "fixed-length row kernels cover 2^5 .. 2^10");

#define PFC_INSTANTIATE_ROW_FIXED(R)                                                              \
    template void launch_row_cube_fixed<R>(const LaunchCfg &, const RowArgs<R> &, int);          \
    template cudaError_t set_smem_attrs_row_fixed<R>(const LaunchCfg &);

}  // namespace pfc
