// Pointwise kernels of the hydrodynamic PFC step (the paper's multiphysics example, Eq. (hpfc)):
//     d_t psi = lap(mu) - v . grad psi,      rho d_t v = Gamma lap v - < psi grad mu >,
//     mu = Lk psi + psi^3,   < . > = multiplication by exp(-a0^2 k^2 / 2) in Fourier space.
// The step (pfc_hydro_step in pfc_api.cu) runs the library's transforms between these kernels;
// the spectral kernels work on standard half spectra (nz, ny, nx/2 + 1), the real kernels on
// real fields, with grid-stride loops.
#pragma once

#include "pfc_pass.cuh"

namespace pfc {

template <typename R> struct HydArgs {
    int nx, ny, nz;
    R cx, cy, cz;        // 2 pi / (n dx) per axis
    R dt, vf, gamma, a0sq;   // vf = dt / rho (0 for rho = inf)
    OpR<R> op;
};

enum { HYD_DERIV = 0, HYD_PSI = 1, HYD_MU = 2, HYD_VEL = 3 };
enum { HYD_CUBE = 0, HYD_MUL = 1, HYD_FMA = 2, HYD_MUL_SET = 3 };

// wavenumbers of half-spectrum index i; nyq[j] is set at the Nyquist index of axis j
template <typename R>
__device__ __forceinline__ void hyd_k(const HydArgs<R> &a, int64_t i, R &kx, R &ky, R &kz, bool (&nyq)[3]) {
    const int nxh = a.nx / 2 + 1;
    const int ikx = (int)(i % nxh);
    const int64_t rest = i / nxh;
    const int iy = (int)(rest % a.ny), iz = (int)(rest / a.ny);
    kx = a.cx * (R)ikx;
    ky = a.cy * (R)(iy <= a.ny / 2 ? iy : iy - a.ny);
    kz = a.cz * (R)(iz <= a.nz / 2 ? iz : iz - a.nz);
    nyq[0] = 2 * ikx == a.nx;
    nyq[1] = 2 * iy == a.ny;
    nyq[2] = a.nz > 1 && 2 * iz == a.nz;
}

// kind HYD_DERIV: x = i k_axis y (zero at the axis' Nyquist index: the spectral first derivative
//                 of a real field);
// kind HYD_PSI:   x = (x - dt k^2 y - dt z) / (1 + dt k^2 Lk)   (density, y = FFT psi^3, z = FFT advection);
// kind HYD_MU:    x = y + Lk z                                (mu_hat, y = FFT psi^3, z = psi_hat);
// kind HYD_VEL:   x = (x - vf G y) / (1 + vf Gamma k^2)       (velocity, y = FFT(psi d_j mu)).
template <typename R, int KIND>
__global__ void __launch_bounds__(256) k_hyd_spec(const HydArgs<R> a, int64_t n, typename VT<R>::V *x,
                                                  const typename VT<R>::V *y, const typename VT<R>::V *z,
                                                  int axis) {
    using V = typename VT<R>::V;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        R kx, ky, kz;
        bool nyq[3];
        hyd_k(a, i, kx, ky, kz, nyq);
        const R k2 = kx * kx + ky * ky + kz * kz;
        if (KIND == HYD_DERIV) {
            const R kj = nyq[axis] ? (R)0 : (axis == 0 ? kx : axis == 1 ? ky : kz);
            const V u = y[i];
            x[i] = V{-kj * u.y, kj * u.x};
        } else if (KIND == HYD_PSI) {
            const R lk = lin_symbol<R>(a.op, k2);
            const V u = x[i], nn = y[i], ad = z[i];
            const R inv = (R)1 / ((R)1 + a.dt * k2 * lk);
            x[i] = V{(u.x - a.dt * k2 * nn.x - a.dt * ad.x) * inv, (u.y - a.dt * k2 * nn.y - a.dt * ad.y) * inv};
        } else if (KIND == HYD_MU) {
            const R lk = lin_symbol<R>(a.op, k2);
            const V nn = y[i], p = z[i];
            x[i] = V{nn.x + lk * p.x, nn.y + lk * p.y};
        } else {
            const R gk = exp(-(R)0.5 * a.a0sq * k2);
            const R inv = (R)1 / ((R)1 + a.vf * a.gamma * k2);
            const V u = x[i], f = y[i];
            x[i] = V{(u.x - a.vf * gk * f.x) * inv, (u.y - a.vf * gk * f.y) * inv};
        }
    }
}

// kind HYD_CUBE: out = p^3;  HYD_MUL: out = p q;  HYD_FMA: out += p q;  HYD_MUL_SET: as HYD_MUL.
template <typename R, int KIND>
__global__ void __launch_bounds__(256) k_hyd_real(int64_t n, const R *p, const R *q, R *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R u = p[i];
        if (KIND == HYD_CUBE) out[i] = u * u * u;
        else if (KIND == HYD_FMA) out[i] += u * q[i];
        else out[i] = u * q[i];
    }
}

}  // namespace pfc
