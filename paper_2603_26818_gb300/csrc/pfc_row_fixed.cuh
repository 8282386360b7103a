// psi^3 row-pass kernels with the row transform length 2^LM fixed at compile time, LM in
// [ROW_FIXED_MIN, ROW_FIXED_MAX]; included by the per-precision translation units only.
#pragma once

#include "pfc_launch.h"

namespace pfc {

template <typename R, int LM, int PY = 0>
static void launch_row_fixed_t(const LaunchCfg &c, const RowArgs<R> &a, int nf) {
    dim3 grid(c.g.QR / c.g.gpc, nf);
    k_row<R, ROW_CUBE, LM, PY><<<grid, c.nt_row, c.smem_row, c.stream>>>(c.g, a);
}

// FP32 2D plans (Pz == 1) with rows of at most 2^8 + 1 bins (the batch classes): Py fixed at
// compile time too, which drops the unused register slots of the y-part (a quarter of them at
// Py = 2)
template <typename R, int LM> static bool launch_row_fixed_py(const LaunchCfg &c, const RowArgs<R> &a, int nf) {
    if (c.g.Pz != 1) return false;
    switch (c.g.Py) {
        case 1: launch_row_fixed_t<R, LM, 1>(c, a, nf); return true;
        case 2: launch_row_fixed_t<R, LM, 2>(c, a, nf); return true;
        case 4: launch_row_fixed_t<R, LM, 4>(c, a, nf); return true;
        case 8: launch_row_fixed_t<R, LM, 8>(c, a, nf); return true;
        default: return false;
    }
}

template <typename R> void launch_row_cube_fixed(const LaunchCfg &c, const RowArgs<R> &a, int nf) {
    if constexpr (sizeof(R) == 4) {
        bool done = false;
        switch (c.g.lM) {
            case 5: done = launch_row_fixed_py<R, 5>(c, a, nf); break;
            case 6: done = launch_row_fixed_py<R, 6>(c, a, nf); break;
            case 7: done = launch_row_fixed_py<R, 7>(c, a, nf); break;
            case 8: done = launch_row_fixed_py<R, 8>(c, a, nf); break;
            default: break;
        }
        if (done) return;
    }
    switch (c.g.lM) {
        case 5: launch_row_fixed_t<R, 5>(c, a, nf); break;
        case 6: launch_row_fixed_t<R, 6>(c, a, nf); break;
        case 7: launch_row_fixed_t<R, 7>(c, a, nf); break;
        case 8: launch_row_fixed_t<R, 8>(c, a, nf); break;
        case 9: launch_row_fixed_t<R, 9>(c, a, nf); break;
        default: launch_row_fixed_t<R, 10>(c, a, nf); break;
    }
}

template <typename R, int LM> static cudaError_t set_smem_py(int bytes) {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_row<R, ROW_CUBE, LM, 1>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row<R, ROW_CUBE, LM, 2>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row<R, ROW_CUBE, LM, 4>, at, bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_row<R, ROW_CUBE, LM, 8>, at, bytes);
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
    if constexpr (sizeof(R) == 4) {
        if ((e = set_smem_py<R, 5>(bytes)) != cudaSuccess) return e;
        if ((e = set_smem_py<R, 6>(bytes)) != cudaSuccess) return e;
        if ((e = set_smem_py<R, 7>(bytes)) != cudaSuccess) return e;
        if ((e = set_smem_py<R, 8>(bytes)) != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(k_row<R, ROW_CUBE, 10>, at, bytes);
}

static_assert(ROW_FIXED_MIN == 5 && ROW_FIXED_MAX == 10, "fixed-length row kernels cover 2^5 .. 2^10");

#define PFC_INSTANTIATE_ROW_FIXED(R)                                                              \
    template void launch_row_cube_fixed<R>(const LaunchCfg &, const RowArgs<R> &, int);          \
    template cudaError_t set_smem_attrs_row_fixed<R>(const LaunchCfg &);

}  // namespace pfc
