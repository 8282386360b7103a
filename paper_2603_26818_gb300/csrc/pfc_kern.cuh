// Definitions of the launch functions of pfc_launch.h; included by the per-precision
// translation units only.
#pragma once

#include "pfc_launch.h"
#include "pfc_reduce.cuh"
#include "pfc_row_cluster.cuh"

#include <algorithm>

namespace pfc {

template <typename K> static cudaError_t allow_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// 3D clustered psi^3 row pass, row length M = 2^8, 2^9 or 2^10 fixed at compile time
template <typename R> void launch_row_cube_cl3(const LaunchCfg &c, const RowArgs<R> &a, int nf) {
    const dim3 grid(2 * c.g.QR, nf);
    if (c.g.lM == 8) k_row_cube_cl3<R, 8><<<grid, c.nt_row_cs, c.smem_row_cs, c.stream>>>(c.g, a);
    else if (c.g.lM == 9) k_row_cube_cl3<R, 9><<<grid, c.nt_row_cs, c.smem_row_cs, c.stream>>>(c.g, a);
    else k_row_cube_cl3<R, 10><<<grid, c.nt_row_cs, c.smem_row_cs, c.stream>>>(c.g, a);
}

template <typename R> void launch_row(const LaunchCfg &c, int mode, const RowArgs<R> &a, int nf) {
    if constexpr (sizeof(R) == 4) {
        if (mode == ROW_CUBE && c.row_cs == 2) {
            if (c.g.Pz == 1)
                k_row_cube_cl<R, 2, 11><<<dim3(2 * c.g.QR, nf), c.nt_row_cs, c.smem_row_cs, c.stream>>>(c.g, a);
            else
                launch_row_cube_cl3<R>(c, a, nf);
            return;
        }
    }
    if (mode == ROW_CUBE && c.g.lM >= ROW_FIXED_MIN && c.g.lM <= ROW_FIXED_MAX) {
        launch_row_cube_fixed<R>(c, a, nf);
        return;
    }
    dim3 grid(c.g.QR / c.g.gpc, nf);
    if (mode == ROW_CUBE) k_row<R, ROW_CUBE><<<grid, c.nt_row, c.smem_row, c.stream>>>(c.g, a);
    else if (mode == ROW_FWD) k_row<R, ROW_FWD><<<grid, c.nt_row, c.smem_row, c.stream>>>(c.g, a);
    else if (mode == ROW_INV) k_row<R, ROW_INV><<<grid, c.nt_row, c.smem_row, c.stream>>>(c.g, a);
    else k_row<R, ROW_ADJ_MIX><<<grid, c.nt_row, c.smem_row, c.stream>>>(c.g, a);
}

template <typename R, int MAXT>
static void launch_line_t(const LaunchCfg &c, int mode, const LineArgs<R> &a, int nf) {
    dim3 grid(c.g.ncg, c.g.P * c.g.R, nf);
    if (mode == LINE_STEP) k_line<R, LINE_STEP, MAXT><<<grid, c.nt_line, c.smem_line, c.stream>>>(c.g, a);
    else if (mode == LINE_SCHEME) k_line<R, LINE_SCHEME, MAXT><<<grid, c.nt_line, c.smem_line, c.stream>>>(c.g, a);
    else if (mode == LINE_FWD) k_line<R, LINE_FWD, MAXT><<<grid, c.nt_line, c.smem_line, c.stream>>>(c.g, a);
    else k_line<R, LINE_INV, MAXT><<<grid, c.nt_line, c.smem_line, c.stream>>>(c.g, a);
}

template <typename R> void launch_line(const LaunchCfg &c, int mode, const LineArgs<R> &a, int nf) {
    if constexpr (sizeof(R) == 4) {
        if (mode == LINE_STEP && line_v2_on(c)) {
            launch_line_v2(c, a, nf);
            return;
        }
    }
    if (mode == LINE_STEP && line_fixed_fits<R>(c)) {
        launch_line_step_fixed<R>(c, a, nf);
        return;
    }
    if constexpr (sizeof(R) == 4) {
        if (c.nt_line > 512) {
            launch_line_t<R, 1024>(c, mode, a, nf);
            return;
        }
    }
    launch_line_t<R, 512>(c, mode, a, nf);
}

template <typename R> cudaError_t set_smem_attrs(const LaunchCfg &c) {
    cudaError_t e;
    if ((e = allow_smem(k_row<R, ROW_CUBE>, c.smem_row)) != cudaSuccess) return e;
    if ((e = allow_smem(k_row<R, ROW_FWD>, c.smem_row)) != cudaSuccess) return e;
    if ((e = allow_smem(k_row<R, ROW_INV>, c.smem_row)) != cudaSuccess) return e;
    if ((e = allow_smem(k_row<R, ROW_ADJ_MIX>, c.smem_row)) != cudaSuccess) return e;
    if ((e = allow_smem(k_line_adj<R>, c.smem_line)) != cudaSuccess) return e;
    if ((e = allow_smem(k_line_step2<R>, c.smem_line)) != cudaSuccess) return e;
    if ((e = allow_smem(k_line<R, LINE_STEP, 512>, c.smem_line)) != cudaSuccess) return e;
    if ((e = allow_smem(k_line<R, LINE_SCHEME, 512>, c.smem_line)) != cudaSuccess) return e;
    if ((e = allow_smem(k_line<R, LINE_FWD, 512>, c.smem_line)) != cudaSuccess) return e;
    if ((e = allow_smem(k_line<R, LINE_INV, 512>, c.smem_line)) != cudaSuccess) return e;
    if constexpr (sizeof(R) == 4) {
        if ((e = allow_smem(k_line<R, LINE_STEP, 1024>, c.smem_line)) != cudaSuccess) return e;
        if ((e = allow_smem(k_line<R, LINE_SCHEME, 1024>, c.smem_line)) != cudaSuccess) return e;
        if ((e = allow_smem(k_line<R, LINE_FWD, 1024>, c.smem_line)) != cudaSuccess) return e;
        if ((e = allow_smem(k_line<R, LINE_INV, 1024>, c.smem_line)) != cudaSuccess) return e;
    }
    if constexpr (sizeof(R) == 4) {
        if (c.row_cs == 2 && c.g.Pz == 1 &&
            (e = allow_smem(k_row_cube_cl<R, 2, 11>, c.smem_row_cs)) != cudaSuccess) return e;
        if (c.row_cs == 2 && c.g.Pz > 1) {
            if ((e = allow_smem(k_row_cube_cl3<R, 8>, c.smem_row_cs)) != cudaSuccess) return e;
            if ((e = allow_smem(k_row_cube_cl3<R, 9>, c.smem_row_cs)) != cudaSuccess) return e;
            if ((e = allow_smem(k_row_cube_cl3<R, 10>, c.smem_row_cs)) != cudaSuccess) return e;
        }
    }
    if ((e = set_smem_attrs_row_fixed<R>(c)) != cudaSuccess) return e;
    if constexpr (sizeof(R) == 4)
        if ((e = set_smem_attrs_v2(c)) != cudaSuccess) return e;
    return set_smem_attrs_fixed<R>(c);
}

template <typename R> void launch_line_adj(const LaunchCfg &c, const AdjArgs<R> &a) {
    dim3 grid(c.g.ncg, c.g.P * c.g.R);
    k_line_adj<R><<<grid, c.nt_line, c.smem_line, c.stream>>>(c.g, a);
}

template <typename R> void launch_line_step2(const LaunchCfg &c, const Step2Args<R> &a) {
    dim3 grid(c.g.ncg, c.g.P * c.g.R);
    k_line_step2<R><<<grid, c.nt_line, c.smem_line, c.stream>>>(c.g, a);
}

template <typename R> void launch_mid(const LaunchCfg &c, int dir, const MidArgs<R> &a) {
    const dim3 grid(a.edges ? 1 : (c.g.xs + MID_CW - 1) / MID_CW, c.g.Q, c.g.P);
    if (dir < 0) k_mid<R, -1><<<grid, MID_THREADS, 0, c.stream>>>(c.g, a);
    else k_mid<R, +1><<<grid, MID_THREADS, 0, c.stream>>>(c.g, a);
}

template <typename R>
void launch_onchip(cudaStream_t s, const Geom &g, const OnchipArgs<R> &a, int members, size_t smem) {
    k_onchip<R><<<members, ONCHIP_THREADS, smem, s>>>(g, a);
}
template <typename R> cudaError_t set_smem_onchip(size_t smem) {
    return allow_smem(k_onchip<R>, smem);
}
template <typename R>
void launch_row_adj2(cudaStream_t s, const Geom &g, int nt, size_t smem, const RowArgs<R> &a) {
    k_row_adj2<R><<<g.QR / g.gpc, nt, smem, s>>>(g, a);
}
template <typename R> cudaError_t set_smem_adj2(size_t smem) {
    return allow_smem(k_row_adj2<R>, smem);
}

template <typename R>
void launch_hyd_spec(cudaStream_t s, int kind, const HydArgs<R> &a, int64_t n, void *x, const void *y,
                     const void *z, int axis) {
    using V = typename VT<R>::V;
    V *xv = reinterpret_cast<V *>(x);
    const V *yv = reinterpret_cast<const V *>(y), *zv = reinterpret_cast<const V *>(z);
    const int blocks = (int)std::min<int64_t>(4 * 304, (n + 255) / 256);
    if (kind == HYD_DERIV) k_hyd_spec<R, HYD_DERIV><<<blocks, 256, 0, s>>>(a, n, xv, yv, zv, axis);
    else if (kind == HYD_PSI) k_hyd_spec<R, HYD_PSI><<<blocks, 256, 0, s>>>(a, n, xv, yv, zv, axis);
    else if (kind == HYD_MU) k_hyd_spec<R, HYD_MU><<<blocks, 256, 0, s>>>(a, n, xv, yv, zv, axis);
    else k_hyd_spec<R, HYD_VEL><<<blocks, 256, 0, s>>>(a, n, xv, yv, zv, axis);
}
template <typename R> void launch_hyd_real(cudaStream_t s, int kind, int64_t n, const R *p, const R *q, R *out) {
    const int blocks = (int)std::min<int64_t>(4 * 304, (n + 255) / 256);
    if (kind == HYD_CUBE) k_hyd_real<R, HYD_CUBE><<<blocks, 256, 0, s>>>(n, p, q, out);
    else if (kind == HYD_FMA) k_hyd_real<R, HYD_FMA><<<blocks, 256, 0, s>>>(n, p, q, out);
    else k_hyd_real<R, HYD_MUL><<<blocks, 256, 0, s>>>(n, p, q, out);
}

template <typename R>
void launch_mr_row(cudaStream_t s, int mode, const MrGeom &g, const MrArgs<R> &a, const void *in, void *out,
                   void *E, int rows_per_block) {
    const int64_t rows = (int64_t)g.ny * g.nz;
    const unsigned blocks = (unsigned)((rows + rows_per_block - 1) / rows_per_block);
    const int threads = 32 * rows_per_block;
    const size_t smem = mr_row_smem(g.M, rows_per_block, sizeof(typename VT<R>::V));
    if (mode == MR_ROW_CUBE) k_mr_row<R, MR_ROW_CUBE><<<blocks, threads, smem, s>>>(g, a, in, out, E);
    else if (mode == MR_ROW_FWD) k_mr_row<R, MR_ROW_FWD><<<blocks, threads, smem, s>>>(g, a, in, out, E);
    else k_mr_row<R, MR_ROW_INV><<<blocks, threads, smem, s>>>(g, a, in, out, E);
}
template <typename R>
void launch_mr_col(cudaStream_t s, int mode, const MrGeom &g, const MrArgs<R> &a, int axis, int W, int ncols,
                   const void *in, void *out, int G) {
    const dim3 grid((ncols + W - 1) / W, axis == 1 ? g.nz : g.ny);
    const size_t smem = mr_col_smem(g.ax[axis].n, W, sizeof(typename VT<R>::V));
    const int nt = 32 * W * G;
    if (mode == MR_COL_FWD) k_mr_col<R, MR_COL_FWD><<<grid, nt, smem, s>>>(g, a, axis, ncols, in, out, G);
    else if (mode == MR_COL_INV) k_mr_col<R, MR_COL_INV><<<grid, nt, smem, s>>>(g, a, axis, ncols, in, out, G);
    else k_mr_col<R, MR_COL_UPDATE><<<grid, nt, smem, s>>>(g, a, axis, ncols, in, out, G);
}
template <typename R>
void launch_mr_edges(cudaStream_t s, const MrGeom &g, const void *E, void *S, double scale) {
    using V = typename VT<R>::V;
    k_mr_edges<R><<<304, 256, 0, s>>>(g, reinterpret_cast<const V *>(E), reinterpret_cast<V *>(S), (R)scale);
}
template <typename R> cudaError_t set_smem_mr(size_t row, size_t col) {
    cudaError_t e;
    if ((e = allow_smem(k_mr_row<R, MR_ROW_CUBE>, row)) != cudaSuccess) return e;
    if ((e = allow_smem(k_mr_row<R, MR_ROW_FWD>, row)) != cudaSuccess) return e;
    if ((e = allow_smem(k_mr_row<R, MR_ROW_INV>, row)) != cudaSuccess) return e;
    if ((e = allow_smem(k_mr_col<R, MR_COL_FWD>, col)) != cudaSuccess) return e;
    if ((e = allow_smem(k_mr_col<R, MR_COL_INV>, col)) != cudaSuccess) return e;
    return allow_smem(k_mr_col<R, MR_COL_UPDATE>, col);
}

template <typename R>
void launch_batch_mean(cudaStream_t s, const R *base, const int64_t *off, const int64_t *n,
                       int members, double *mean, int *status) {
    k_batch_mean<R><<<members, RED_THREADS, 0, s>>>(base, off, n, mean, status);
}

template <typename R>
void launch_reduce_real(cudaStream_t s, int kind, const R *x, const R *y, int64_t n,
                        double *partials, int *status) {
    if (kind == RED_SUM) k_reduce_real<R, RED_SUM><<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, y, n, partials, status);
    else if (kind == RED_POW4) k_reduce_real<R, RED_POW4><<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, y, n, partials, status);
    else k_reduce_real<R, RED_DOT><<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, y, n, partials, status);
}

template <typename R>
void launch_reduce_spec(cudaStream_t s, const Geom &g, OpDev op, double dx, const void *X,
                        const double *mean, double *partials, int *status) {
    k_reduce_spec<R><<<RED_BLOCKS, RED_THREADS, 0, s>>>(
        g, op, dx, reinterpret_cast<const typename VT<R>::V *>(X), mean, partials, status);
}

#define PFC_INSTANTIATE_LAUNCH(R)                                                          \
    template void launch_row<R>(const LaunchCfg &, int, const RowArgs<R> &, int);          \
    template void launch_line<R>(const LaunchCfg &, int, const LineArgs<R> &, int);        \
    template cudaError_t set_smem_attrs<R>(const LaunchCfg &);                             \
    template void launch_line_adj<R>(const LaunchCfg &, const AdjArgs<R> &);               \
    template void launch_line_step2<R>(const LaunchCfg &, const Step2Args<R> &);           \
    template void launch_mid<R>(const LaunchCfg &, int, const MidArgs<R> &);               \
    template void launch_onchip<R>(cudaStream_t, const Geom &, const OnchipArgs<R> &, int, size_t); \
    template cudaError_t set_smem_onchip<R>(size_t);                                       \
    template void launch_row_adj2<R>(cudaStream_t, const Geom &, int, size_t, const RowArgs<R> &); \
    template cudaError_t set_smem_adj2<R>(size_t);                                         \
    template void launch_hyd_spec<R>(cudaStream_t, int, const HydArgs<R> &, int64_t, void *, const void *, \
                                     const void *, int);                                  \
    template void launch_hyd_real<R>(cudaStream_t, int, int64_t, const R *, const R *, R *); \
    template void launch_mr_row<R>(cudaStream_t, int, const MrGeom &, const MrArgs<R> &, const void *, void *, \
                                   void *, int);                                            \
    template void launch_mr_col<R>(cudaStream_t, int, const MrGeom &, const MrArgs<R> &, int, int, int,  \
                                   const void *, void *, int);                              \
    template void launch_mr_edges<R>(cudaStream_t, const MrGeom &, const void *, void *, double); \
    template cudaError_t set_smem_mr<R>(size_t, size_t);                                   \
    template void launch_batch_mean<R>(cudaStream_t, const R *, const int64_t *,           \
                                       const int64_t *, int, double *, int *);             \
    template void launch_reduce_real<R>(cudaStream_t, int, const R *, const R *, int64_t,  \
                                        double *, int *);                                  \
    template void launch_reduce_spec<R>(cudaStream_t, const Geom &, OpDev, double,         \
                                        const void *, const double *, double *, int *);

}  // namespace pfc
