// Deterministic FP64 reductions for mass and energy (Eq. (5)).
// A fixed grid of RED_BLOCKS blocks each sums a fixed strided slice in FP64 and writes one
// partial; a single block then adds the partials in index order. The result does not depend
// on scheduling, so two runs are bitwise equal. Any NaN or Inf met sets STATUS_NONFINITE.
#pragma once

#include "pfc_launch.h"

namespace pfc {


__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] += sh[tid + s];
        __syncthreads();
    }
    return sh[0];
}


// partial[b] = sum over this block's slice of f(x[i], y[i]); f = x, x^4 or x y.
template <typename R, int KIND>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_real(const R *__restrict__ x,
                                                             const R *__restrict__ y, int64_t n,
                                                             double *partials, int *status) {
    __shared__ double sh[RED_THREADS];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = (double)x[i];
        if (!isfinite(v)) bad = true;
        if (KIND == RED_SUM) acc += v;
        else if (KIND == RED_POW4) { const double v2 = v * v; acc += v2 * v2; }
        else acc += v * (double)y[i];
    }
    if (bad) atomicOr(status, STATUS_NONFINITE);
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out[0] = scale * sum_{b < nb} partials[b] (+ out[0] when accumulate), summed by one block in
// a fixed order.
static __global__ void __launch_bounds__(RED_THREADS) k_finish(const double *__restrict__ partials, int nb,
                                                               double scale, double *out, int accumulate) {
    __shared__ double sh[RED_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partials[i];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = (accumulate ? out[0] : 0.0) + s * scale;
}

// Spectral part of the energy for one field from its standard half spectrum X of psi - m,
// m = mean rounded to R:  sum_k w_k Lk(k) |psi_hat_k|^2 with w_k = 1 on the kx = 0 and
// kx = nx/2 planes and 2 elsewhere, and psi_hat_0 = N m + X_0.
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_spec(const Geom g, OpDev op, double dx,
                                                             const typename VT<R>::V *__restrict__ X,
                                                             const double *__restrict__ mean,
                                                             double *partials, int *status) {
    __shared__ double sh[RED_THREADS];
    const int64_t n = g.nstd;
    const int M1 = g.M + 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double two_pi = 6.28318530717958647692528676655900576839;
    const double cx = two_pi / (g.nx * dx), cy = two_pi / (g.ny * dx), cz = two_pi / (g.nz * dx);
    double acc = 0.0;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int kx = (int)(i % M1);
        const int64_t row = i / M1;
        const int ky = (int)(row % g.ny), kz = (int)(row / g.ny);
        const int my = ky <= g.ny / 2 ? ky : ky - g.ny;
        const int mz = kz <= g.nz / 2 ? kz : kz - g.nz;
        const double fx = cx * kx, fy = cy * my, fz = cz * mz;
        const double k2 = fx * fx + fy * fy + fz * fz;
        const double a = 1.0 - k2;
        double lk;
        if (op.kind == 0) lk = op.r + a * a;
        else { const double b = op.q2 * op.q2 - k2; lk = op.r + a * a * (op.R1 + b * b); }
        double re = (double)X[i].x, im = (double)X[i].y;
        if (!isfinite(re) || !isfinite(im)) bad = true;
        if (i == 0) { re += (double)g.nreal * (double)(R)mean[0]; im = 0.0; }
        const double wk = (kx == 0 || kx == g.M) ? 1.0 : 2.0;
        acc += wk * lk * (re * re + im * im);
    }
    if (bad) atomicOr(status, STATUS_NONFINITE);
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Mean of every member of a packed batch: block m sums member m (n_m values at offset off[m])
// in FP64 in a fixed order and writes mean[m].
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_batch_mean(const R *__restrict__ base,
                                                            const int64_t *__restrict__ off,
                                                            const int64_t *__restrict__ n,
                                                            double *mean, int *status) {
    __shared__ double sh[RED_THREADS];
    const int m = blockIdx.x;
    const R *x = base + off[m];
    const int64_t nm = n[m];
    double acc = 0.0;
    bool bad = false;
    for (int64_t i = threadIdx.x; i < nm; i += blockDim.x) {
        const double v = (double)x[i];
        if (!isfinite(v)) bad = true;
        acc += v;
    }
    if (bad) atomicOr(status, STATUS_NONFINITE);
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) mean[m] = s / (double)nm;
}

}  // namespace pfc
