// FP32-mixed update-pass kernels with compile-time y transform lengths.
#include "pfc_line_fixed.cuh"

namespace pfc {
PFC_INSTANTIATE_LINE_FIXED(float)
}  // namespace pfc

#include <cstdlib>

namespace pfc {

// k_line_v2 where the tile width is even (single field or a batch class); PFC_LINE_V2=0 keeps the
// one-column pass (to compare the two)
bool line_v2_on(const LaunchCfg &c) {
    static const bool off = [] {
        const char *e = std::getenv("PFC_LINE_V2");
        return e && e[0] == '0';
    }();
    return !off && c.g.W >= 2 && c.nt_line / 2 <= 512 && c.nt_line >= 64;
}

template <int LY, int LZ> static void v2_t(const LaunchCfg &c, const LineArgs<float> &a, int nf) {
    const Geom gv = v2_view(c.g);
    const dim3 grid(c.g.ncg, c.g.P * c.g.R, nf);
    k_line_v2<512, LY, LZ><<<grid, c.nt_line / 2, c.smem_line, c.stream>>>(c.g, gv, a);
}

void launch_line_v2(const LaunchCfg &c, const LineArgs<float> &a, int nf) {
    const int ly = c.g.lQy, lz = c.g.Qz > 1 ? c.g.lQz : 0;
    if (ly == 9 && lz == 0) v2_t<9, 0>(c, a, nf);
    else if (ly == 8 && lz == 0) v2_t<8, 0>(c, a, nf);
    else if (ly == 10 && lz == 0) v2_t<10, 0>(c, a, nf);
    else if (ly == 6 && lz == 6) v2_t<6, 6>(c, a, nf);
    else if (ly == 6 && lz == 4) v2_t<6, 4>(c, a, nf);
    else if (ly == 7 && lz == 5) v2_t<7, 5>(c, a, nf);
    else v2_t<0, 0>(c, a, nf);
}

cudaError_t set_smem_attrs_v2(const LaunchCfg &c) {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int bytes = (int)c.smem_line;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_line_v2<512, 9, 0>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line_v2<512, 8, 0>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line_v2<512, 10, 0>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line_v2<512, 6, 6>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line_v2<512, 6, 4>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line_v2<512, 7, 5>, at, bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_line_v2<512, 0, 0>, at, bytes);
}

}  // namespace pfc
