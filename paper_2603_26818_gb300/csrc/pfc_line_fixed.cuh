// Update-pass kernels with the transform lengths fixed at compile time (see line_fixed_fits);
// included by the per-precision translation units only.
#pragma once

#include "pfc_launch.h"

namespace pfc {

template <typename R, int MAXT, int LY, int LZ>
static void launch_fixed_t(const LaunchCfg &c, const LineArgs<R> &a, int nf) {
    dim3 grid(c.g.ncg, c.g.P * c.g.R, nf);
    k_line<R, LINE_STEP, MAXT, LY, LZ><<<grid, c.nt_line, c.smem_line, c.stream>>>(c.g, a);
}

template <typename R> void launch_line_step_fixed(const LaunchCfg &c, const LineArgs<R> &a, int nf) {
    if (c.g.Qz > 1) {
        const int ly = c.g.lQy, lz = c.g.lQz;
        if constexpr (sizeof(R) == 4) {
            if (ly == 6 && lz == 6) {
                launch_fixed_t<R, 1024, 6, 6>(c, a, nf);
                return;
            }
        }
        if (ly == 5 && lz == 5) launch_fixed_t<R, 512, 5, 5>(c, a, nf);
        else if (ly == 5 && lz == 4) launch_fixed_t<R, 512, 5, 4>(c, a, nf);
        else launch_fixed_t<R, 512, 6, 4>(c, a, nf);
        return;
    }
    switch (c.g.lQy) {
        case 6: launch_fixed_t<R, 512, 6, 0>(c, a, nf); break;
        case 7: launch_fixed_t<R, 512, 7, 0>(c, a, nf); break;
        case 8: launch_fixed_t<R, 512, 8, 0>(c, a, nf); break;
        case 9: launch_fixed_t<R, 512, 9, 0>(c, a, nf); break;
        default: launch_fixed_t<R, 512, 10, 0>(c, a, nf); break;
    }
}

template <typename R> cudaError_t set_smem_attrs_fixed(const LaunchCfg &c) {
    cudaError_t e;
    const int bytes = (int)c.smem_line;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 6, 0>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 7, 0>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 8, 0>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 9, 0>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 10, 0>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 5, 5>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 5, 4>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 6, 4>, at, bytes)) != cudaSuccess) return e;
    if constexpr (sizeof(R) == 4)
        return cudaFuncSetAttribute(k_line<R, LINE_STEP, 1024, 6, 6>, at, bytes);
    return cudaSuccess;
}

static_assert(LINE_FIXED_MIN == 6 && LINE_FIXED_MAX == 10, "fixed-length kernels cover 2^6 .. 2^10");

#define PFC_INSTANTIATE_LINE_FIXED(R)                                                            \
    template void launch_line_step_fixed<R>(const LaunchCfg &, const LineArgs<R> &, int);       \
    template cudaError_t set_smem_attrs_fixed<R>(const LaunchCfg &);

}  // namespace pfc
