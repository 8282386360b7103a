// Host-side launch interface of the pass and reduction kernels. The kernels are compiled in
// translation units per precision (pfc_kern_f32.cu, pfc_kern_f64.cu, pfc_line_fixed_f32.cu,
// pfc_line_fixed_f64.cu), which instantiate these functions; the plan logic in pfc_api.cu only
// calls them.
#pragma once

#include <cuda_runtime.h>

#include "pfc_adjoint.cuh"
#include "pfc_coupled.cuh"
#include "pfc_mid.cuh"
#include "pfc_line_v2.cuh"
#include "pfc_onchip.cuh"
#include "pfc_adjoint_row.cuh"
#include "pfc_hydro.cuh"
#include "pfc_mixed.cuh"
#include "pfc_persist.cuh"

namespace pfc {

struct LaunchCfg {
    Geom g;
    int nt_row, nt_line;
    size_t smem_row, smem_line;
    cudaStream_t stream;
    // ROW_CUBE over clusters of row_cs blocks (k_row_cube_cl, FP32 only); 0: single blocks
    int row_cs = 0, nt_row_cs = 0;
    size_t smem_row_cs = 0;
};

constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs
constexpr int RED_THREADS = 256;
enum { RED_SUM = 0, RED_POW4 = 1, RED_DOT = 2 };

template <typename R> void launch_row(const LaunchCfg &c, int mode, const RowArgs<R> &a, int nf);
template <typename R> void launch_line(const LaunchCfg &c, int mode, const LineArgs<R> &a, int nf);
template <typename R> cudaError_t set_smem_attrs(const LaunchCfg &c);
// partials[b] (b < RED_BLOCKS) = block sums of x, x^4 or x y over n values, FP64
template <typename R>
void launch_reduce_real(cudaStream_t s, int kind, const R *x, const R *y, int64_t n,
                        double *partials, int *status);
// partials = block sums of w_k Lk(k) |psi_hat_k|^2 over a standard half spectrum
template <typename R>
void launch_reduce_spec(cudaStream_t s, const Geom &g, OpDev op, double dx, const void *X,
                        const double *mean, double *partials, int *status);
// out[0] = scale * sum of nb partials, in a fixed order (added to out[0] if accumulate)
void launch_finish(cudaStream_t s, const double *partials, int nb, double scale, double *out,
                   bool accumulate = false);
// per-member means of a packed batch (one block per member)
template <typename R>
void launch_batch_mean(cudaStream_t s, const R *base, const int64_t *off, const int64_t *n,
                       int members, double *mean, int *status);
// adjoint line pass (blocks of nt_line <= 512 threads), one partial per block
template <typename R> void launch_line_adj(const LaunchCfg &c, const AdjArgs<R> &a);
// coupled two-field line pass (blocks of nt_line <= 512 threads, smem_line for three tiles)
template <typename R> void launch_line_step2(const LaunchCfg &c, const Step2Args<R> &a);
// on-chip steps of small batch domains (pfc_onchip.cuh): one block per member, smem bytes
template <typename R>
void launch_onchip(cudaStream_t s, const Geom &g, const OnchipArgs<R> &a, int members, size_t smem);
template <typename R> cudaError_t set_smem_onchip(size_t smem);
// fused adjoint row pass (pfc_adjoint_row.cuh) on geometry g (its gpc), nt threads, smem bytes
template <typename R>
void launch_row_adj2(cudaStream_t s, const Geom &g, int nt, size_t smem, const RowArgs<R> &a);
template <typename R> cudaError_t set_smem_adj2(size_t smem);
// pointwise kernels of the hydrodynamic step (pfc_hydro.cuh): spectral (standard half spectra of
// n complex values) and real (n values)
template <typename R>
void launch_hyd_spec(cudaStream_t s, int kind, const HydArgs<R> &a, int64_t n, void *x, const void *y,
                     const void *z, int axis);
template <typename R> void launch_hyd_real(cudaStream_t s, int kind, int64_t n, const R *p, const R *q, R *out);
// passes of the mixed-radix schedule (pfc_mixed.cuh)
template <typename R>
void launch_mr_row(cudaStream_t s, int mode, const MrGeom &g, const MrArgs<R> &a, const void *in, void *out,
                   void *E, int rows_per_block);
template <typename R>
void launch_mr_col(cudaStream_t s, int mode, const MrGeom &g, const MrArgs<R> &a, int axis, int W, int ncols,
                   const void *in, void *out, int G);
template <typename R>
void launch_mr_edges(cudaStream_t s, const MrGeom &g, const void *E, void *S, double scale);
template <typename R> cudaError_t set_smem_mr(size_t row, size_t col);
// the persistent batch kernel (pfc_persist.cuh), NT = 128, 256 or 512 threads a block: one
// cooperative launch of grid blocks; persist_occupancy allows smem bytes and returns the blocks
// that fit an SM
template <typename R, int NT> cudaError_t launch_batch_persist(const PbArgs<R> &a, int grid, size_t smem, cudaStream_t s);
template <typename R, int NT> cudaError_t persist_occupancy(size_t smem, int *blocks_per_sm);
// middle pass of a three-pass plan (g.R > 1): dir -1 forward, +1 inverse (pfc_mid.cuh)
template <typename R> void launch_mid(const LaunchCfg &c, int dir, const MidArgs<R> &a);

// The update pass (LINE_STEP) with its transform lengths fixed at compile time, compiled in
// pfc_line_fixed_f32.cu / pfc_line_fixed_f64.cu: one-axis tiles (Qz = 1) with Qy = 2^6 .. 2^10
// in blocks of at most 512 threads, and the two-axis tiles of the common 3D plans (log2 Qy,
// log2 Qz) = (5, 5), (5, 4), (6, 4) in blocks of at most 512 threads and (6, 6) in blocks of up
// to 1024. launch_line takes it whenever line_fixed_fits.
constexpr int LINE_FIXED_MIN = 6, LINE_FIXED_MAX = 10;
// (6, 6) is built for FP32 only (FP64 line blocks have at most 512 threads and no such plan)
template <typename R> inline bool line_fixed_fits(const LaunchCfg &c) {
    const int ly = c.g.lQy, lz = c.g.lQz, nt = c.nt_line;
    if (c.g.Qz == 1) return nt <= 512 && ly >= LINE_FIXED_MIN && ly <= LINE_FIXED_MAX;
    if (nt <= 512 && ((ly == 5 && lz == 5) || (ly == 5 && lz == 4) || (ly == 6 && lz == 4))) return true;
    return sizeof(R) == 4 && nt <= 1024 && ly == 6 && lz == 6;
}
template <typename R> void launch_line_step_fixed(const LaunchCfg &c, const LineArgs<R> &a, int nf);
// The FP32 update pass with two kx columns per element (k_line_v2), for tiles of even width.
bool line_v2_on(const LaunchCfg &c);
void launch_line_v2(const LaunchCfg &c, const LineArgs<float> &a, int nf);
cudaError_t set_smem_attrs_v2(const LaunchCfg &c);
// The psi^3 row pass with its row length M = 2^lM fixed at compile time, lM in [ROW_FIXED_MIN,
// ROW_FIXED_MAX] (compiled in pfc_row_fixed_f32.cu / pfc_row_fixed_f64.cu).
constexpr int ROW_FIXED_MIN = 5, ROW_FIXED_MAX = 10;
template <typename R> void launch_row_cube_fixed(const LaunchCfg &c, const RowArgs<R> &a, int nf);
template <typename R> cudaError_t set_smem_attrs_row_fixed(const LaunchCfg &c);
template <typename R> cudaError_t set_smem_attrs_fixed(const LaunchCfg &c);

#define PFC_DECLARE_LAUNCH(R)                                                                   \
    extern template void launch_row<R>(const LaunchCfg &, int, const RowArgs<R> &, int);        \
    extern template void launch_line<R>(const LaunchCfg &, int, const LineArgs<R> &, int);      \
    extern template void launch_line_step_fixed<R>(const LaunchCfg &, const LineArgs<R> &, int); \
    extern template void launch_row_cube_fixed<R>(const LaunchCfg &, const RowArgs<R> &, int);   \
    extern template cudaError_t set_smem_attrs_row_fixed<R>(const LaunchCfg &);                 \
    extern template cudaError_t set_smem_attrs_fixed<R>(const LaunchCfg &);                     \
    extern template cudaError_t set_smem_attrs<R>(const LaunchCfg &);                           \
    extern template void launch_line_adj<R>(const LaunchCfg &, const AdjArgs<R> &);             \
    extern template void launch_line_step2<R>(const LaunchCfg &, const Step2Args<R> &);         \
    extern template void launch_mid<R>(const LaunchCfg &, int, const MidArgs<R> &);             \
    extern template void launch_onchip<R>(cudaStream_t, const Geom &, const OnchipArgs<R> &, int, size_t); \
    extern template cudaError_t set_smem_onchip<R>(size_t);                                      \
    extern template void launch_row_adj2<R>(cudaStream_t, const Geom &, int, size_t, const RowArgs<R> &); \
    extern template cudaError_t set_smem_adj2<R>(size_t);                                        \
    extern template void launch_hyd_spec<R>(cudaStream_t, int, const HydArgs<R> &, int64_t, void *, \
                                            const void *, const void *, int);                    \
    extern template void launch_hyd_real<R>(cudaStream_t, int, int64_t, const R *, const R *, R *); \
    extern template void launch_mr_row<R>(cudaStream_t, int, const MrGeom &, const MrArgs<R> &, const void *, \
                                          void *, void *, int);                                  \
    extern template void launch_mr_col<R>(cudaStream_t, int, const MrGeom &, const MrArgs<R> &, int, int, \
                                          int, const void *, void *, int);                       \
    extern template void launch_mr_edges<R>(cudaStream_t, const MrGeom &, const void *, void *, double); \
    extern template cudaError_t set_smem_mr<R>(size_t, size_t);                                  \
    extern template void launch_batch_mean<R>(cudaStream_t, const R *, const int64_t *,         \
                                              const int64_t *, int, double *, int *);           \
    extern template void launch_reduce_real<R>(cudaStream_t, int, const R *, const R *, int64_t, \
                                               double *, int *);                                \
    extern template void launch_reduce_spec<R>(cudaStream_t, const Geom &, OpDev, double,       \
                                               const void *, const double *, double *, int *);
#define PFC_DECLARE_PERSIST(R)                                                                     \
    extern template cudaError_t launch_batch_persist<R, 128>(const PbArgs<R> &, int, size_t, cudaStream_t); \
    extern template cudaError_t launch_batch_persist<R, 256>(const PbArgs<R> &, int, size_t, cudaStream_t); \
    extern template cudaError_t launch_batch_persist<R, 512>(const PbArgs<R> &, int, size_t, cudaStream_t); \
    extern template cudaError_t persist_occupancy<R, 128>(size_t, int *);                          \
    extern template cudaError_t persist_occupancy<R, 256>(size_t, int *);                          \
    extern template cudaError_t persist_occupancy<R, 512>(size_t, int *);
PFC_DECLARE_PERSIST(float)
PFC_DECLARE_PERSIST(double)
#undef PFC_DECLARE_PERSIST
PFC_DECLARE_LAUNCH(float)
PFC_DECLARE_LAUNCH(double)
#undef PFC_DECLARE_LAUNCH

}  // namespace pfc
