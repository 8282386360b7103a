// Line pass of the coupled two-field step (density psi and composition c, both conserved).
//
// With chemical potentials mu_psi = Lk_psi psi + psi^3 + alpha c and mu_c = Lk_c c + c^3 +
// alpha psi and d_t = lap mu for both fields, the semi-implicit step takes the linear terms
// (both operators and the alpha coupling) implicitly and the cubes explicitly, so every mode
// solves
//   [1 + dt k^2 Lk_psi,  dt k^2 alpha    ] [psi_hat']   [psi_hat - dt k^2 N_psi]
//   [dt k^2 alpha,       1 + dt k^2 Lk_c ] [c_hat'  ] = [c_hat   - dt k^2 N_c  ]
// by Cramer's rule. In the X' scaling of the single-field pass the right-hand side entries are
// e = T_hat / Q - dt k^2 (2/N) C_hat, and the inverse transforms take the solution directly.
// The k = 0 mode of both fluctuation fields stays zero (each mean is carried in FP64).
#pragma once

#include "pfc_pass.cuh"

namespace pfc {

template <typename R> struct Step2Args {
    void *x0, *x1;        // X' of psi and of c (in/out)
    const void *c0, *c1;  // C' of psi and of c
    R alpha;
    UpdR<R> up;           // op[0] for psi, op[1] for c
    StageTw<typename VT<R>::V> st;
};

template <typename R>
__global__ void __launch_bounds__(512) k_line_step2(const Geom g, const Step2Args<R> a) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const int cg = blockIdx.x, kp = blockIdx.y;
    const int tsz = g.tsz;
    V *T0 = sm;                 // psi transform
    V *T1 = sm + tsz;           // c transform (natural order)
    V *N0 = sm + 2 * tsz;       // psi^3 transform (natural order)
    V *N1 = sm + 3 * tsz;       // c^3 transform (natural order)
    const LineMap mp = line_map(g, threadIdx.x);
    const PadTileAddr ady = tile_y(g, mp);
    const TileAddr adz = tile_z(g, mp);
    const bool two_axes = g.Qz > 1;
    const int kpy = kp % g.Py, kpz = kp / g.Py;
    V v[8];

    auto forward = [&](const V *src, V *tile, bool to_regs) {
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = src[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)];
        fft_run<-1>(v, tile, ady, g.lQy, mp.jy, true, true, to_regs && !two_axes, a.st);
        if (two_axes) fft_run<-1>(v, tile, adz, g.lQz, mp.jz, true, false, to_regs, a.st);
    };
    forward(reinterpret_cast<const V *>(a.c0), N0, false);
    forward(reinterpret_cast<const V *>(a.c1), N1, false);
    forward(reinterpret_cast<const V *>(a.x1), T1, false);
    forward(reinterpret_cast<const V *>(a.x0), T0, true);

    const int kx = cg * g.W + mp.w;
    const R fx = a.up.cx * (R)kx;
    const R dt = a.up.dt, invQ = a.up.invQ, ihn = a.up.inv_halfN;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int kqy = two_axes ? mp.yq : mp.jy + m * mp.ny8;
        const int kqz = two_axes ? mp.jz + m * mp.nz8 : 0;
        const int ky = kpy + (kqy << g.lPy), kz = kpz + (kqz << g.lPz);
        const int my = ky <= (g.ny >> 1) ? ky : ky - g.ny;
        const int mz = kz <= (g.nz >> 1) ? kz : kz - g.nz;
        const R fy = a.up.cy * (R)my, fz = a.up.cz * (R)mz;
        const R k2 = fx * fx + fy * fy + fz * fz;
        const R dk = dt * k2;
        const R m11 = (R)1 + dk * lin_symbol<R>(a.up.op[0], k2);
        const R m22 = (R)1 + dk * lin_symbol<R>(a.up.op[1], k2);
        const R m12 = dk * a.alpha;
        const R idet = (R)1 / (m11 * m22 - m12 * m12);
        const int pos = tile_slot(mp, two_axes, ady, adz, m);
        const V n0 = N0[pos], n1 = N1[pos], t1 = T1[pos];
        const V e1 = V{v[m].x * invQ - dk * ihn * n0.x, v[m].y * invQ - dk * ihn * n0.y};
        const V e2 = V{t1.x * invQ - dk * ihn * n1.x, t1.y * invQ - dk * ihn * n1.y};
        V s0 = V{(m22 * e1.x - m12 * e2.x) * idet, (m22 * e1.y - m12 * e2.y) * idet};
        V s1 = V{(m11 * e2.x - m12 * e1.x) * idet, (m11 * e2.y - m12 * e1.y) * idet};
        if (kx == 0 && ky == 0 && kz == 0) {
            s0 = V{(R)0, (R)0};
            s1 = V{(R)0, (R)0};
        }
        v[m] = s0;
        T1[pos] = s1;   // own position: no other thread reads it before the barrier below
    }
    V *X0 = reinterpret_cast<V *>(a.x0);
    V *X1 = reinterpret_cast<V *>(a.x1);
    if (two_axes) {
        fft_run<+1>(v, T0, adz, g.lQz, mp.jz, true, true, false, a.st);
        fft_run<+1>(v, T0, ady, g.lQy, mp.jy, true, false, true, a.st);
    } else {
        fft_run<+1>(v, T0, ady, g.lQy, mp.jy, true, true, true, a.st);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) X0[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)] = v[m];
    __syncthreads();
    if (two_axes) {
        fft_run<+1>(v, T1, adz, g.lQz, mp.jz, true, false, false, a.st);
        fft_run<+1>(v, T1, ady, g.lQy, mp.jy, true, false, true, a.st);
    } else {
        fft_run<+1>(v, T1, ady, g.lQy, mp.jy, true, false, true, a.st);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) X1[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)] = v[m];
}

}  // namespace pfc
