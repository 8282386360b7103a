// Update-pass kernels with the y transform length 2^LY fixed at compile time, LY in
// [LINE_FIXED_MIN, LINE_FIXED_MAX]; included by the per-precision translation units only.
#pragma once

#include "pfc_launch.h"

namespace pfc {

template <typename R, int LY>
static void launch_fixed_t(const LaunchCfg &c, const LineArgs<R> &a, int nf) {
    dim3 grid(c.g.ncg, c.g.P, nf);
    k_line<R, LINE_STEP, 512, LY><<<grid, c.nt_line, c.smem_line, c.stream>>>(c.g, a);
}

template <typename R> void launch_line_step_fixed(const LaunchCfg &c, const LineArgs<R> &a, int nf) {
    switch (c.g.lQy) {
        case 6: launch_fixed_t<R, 6>(c, a, nf); break;
        case 7: launch_fixed_t<R, 7>(c, a, nf); break;
        case 8: launch_fixed_t<R, 8>(c, a, nf); break;
        case 9: launch_fixed_t<R, 9>(c, a, nf); break;
        default: launch_fixed_t<R, 10>(c, a, nf); break;
    }
}

template <typename R> cudaError_t set_smem_attrs_fixed(const LaunchCfg &c) {
    cudaError_t e;
    const int bytes = (int)c.smem_line;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 6>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 7>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 8>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 9>, at, bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_line<R, LINE_STEP, 512, 10>, at, bytes);
}

static_assert(LINE_FIXED_MIN == 6 && LINE_FIXED_MAX == 10, "fixed-length kernels cover 2^6 .. 2^10");

#define PFC_INSTANTIATE_LINE_FIXED(R)                                                            \
    template void launch_line_step_fixed<R>(const LaunchCfg &, const LineArgs<R> &, int);       \
    template cudaError_t set_smem_attrs_fixed<R>(const LaunchCfg &);

}  // namespace pfc
