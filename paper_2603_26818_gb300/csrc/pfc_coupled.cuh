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

// Three tiles of shared memory: A keeps, per register slot of its owner thread, first N0 then
// e1 and finally the solved c field; N holds N1; B is the transforms' workspace. Only one
// register set is live at a time.
// The body of one block (column group cg, split index kp); k_line_step2 runs it as its own
// block, the persistent batch kernel once per work item.
template <typename R>
__device__ __forceinline__ void line_step2_body(const Geom &g, const Step2Args<R> &a, int cg, int kp) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    V *A = sm;
    V *B = sm + g.tsz;
    V *N = sm + 2 * g.tsz;
    const LineMap mp = line_map(g, threadIdx.x);
    const PadTileAddr ady = tile_y(g, mp);
    const TileAddr adz = tile_z(g, mp);
    const bool two_axes = g.Qz > 1;
    int kpy, kpz;
    line_kp(g, kp, kpy, kpz);
    const int lsy = g.lPy + g.lRy, lsz = g.lPz + g.lRz;
    V v[8];

    const int kx = cg * g.W + mp.w;
    const R fx = a.up.cx * (R)kx;
    const R dt = a.up.dt, invQ = a.up.invQ, ihn = a.up.inv_halfN;
    // k^2 of register slot m (and its ky, kz)
#define PFC_KSQ(m, ky, kz, k2)                                                                \
    do {                                                                                      \
        const int kqy_ = two_axes ? mp.yq : mp.jy + (m) * mp.ny8;                             \
        const int kqz_ = two_axes ? mp.jz + (m) * mp.nz8 : 0;                                 \
        ky = kpy + (kqy_ << lsy);                                                           \
        kz = kpz + (kqz_ << lsz);                                                           \
        const int my_ = ky <= (g.ny >> 1) ? ky : ky - g.ny;                                   \
        const int mz_ = kz <= (g.nz >> 1) ? kz : kz - g.nz;                                   \
        const R fy_ = a.up.cy * (R)my_, fz_ = a.up.cz * (R)mz_;                               \
        k2 = fx * fx + fy_ * fy_ + fz_ * fz_;                                                 \
    } while (0)
    // 1. N0 into A (natural order)
    line_forward(v, g, mp, kp, cg, reinterpret_cast<const V *>(a.c0), A, ady, adz, false, a.st);
    // 2. T0 into registers; e1 = T0/Q - dt k^2 (2/N) N0 replaces N0 at the thread's own slots
    line_forward(v, g, mp, kp, cg, reinterpret_cast<const V *>(a.x0), B, ady, adz, true, a.st);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        int ky, kz;
        R k2;
        PFC_KSQ(m, ky, kz, k2);
        const R dk = dt * k2;
        const int pos = tile_slot(mp, two_axes, ady, adz, m);
        const V n0 = A[pos];
        A[pos] = V{v[m].x * invQ - dk * ihn * n0.x, v[m].y * invQ - dk * ihn * n0.y};
    }
    // 3. N1 into N (natural order); 4. T1 into registers
    line_forward(v, g, mp, kp, cg, reinterpret_cast<const V *>(a.c1), N, ady, adz, false, a.st);
    line_forward(v, g, mp, kp, cg, reinterpret_cast<const V *>(a.x1), B, ady, adz, true, a.st);
    // 5. per-mode 2x2 solve (Cramer), one slot at a time from shared memory: T1 goes to B at the
    // own slots, psi replaces it there and c replaces e1 in A
#pragma unroll
    for (int m = 0; m < 8; ++m) B[tile_slot(mp, two_axes, ady, adz, m)] = v[m];
#pragma unroll 1
    for (int m = 0; m < 8; ++m) {
        int ky, kz;
        R k2;
        PFC_KSQ(m, ky, kz, k2);
        const R dk = dt * k2;
        const R m11 = (R)1 + dk * lin_symbol<R>(a.up.op[0], k2);
        const R m22 = (R)1 + dk * lin_symbol<R>(a.up.op[1], k2);
        const R m12 = dk * a.alpha;
        const R idet = (R)1 / (m11 * m22 - m12 * m12);
        const int pos = tile_slot(mp, two_axes, ady, adz, m);
        const V e1 = A[pos], n1 = N[pos], t1 = B[pos];
        const V e2 = V{t1.x * invQ - dk * ihn * n1.x, t1.y * invQ - dk * ihn * n1.y};
        V s0 = V{(m22 * e1.x - m12 * e2.x) * idet, (m22 * e1.y - m12 * e2.y) * idet};
        V s1 = V{(m11 * e2.x - m12 * e1.x) * idet, (m11 * e2.y - m12 * e1.y) * idet};
        if (kx == 0 && ky == 0 && kz == 0) {
            s0 = V{(R)0, (R)0};
            s1 = V{(R)0, (R)0};
        }
        B[pos] = s0;
        A[pos] = s1;
    }
    __syncthreads();   // every thread's slots of A and B written
    // 6. inverse of psi from B
    V *X0 = reinterpret_cast<V *>(a.x0);
    V *X1 = reinterpret_cast<V *>(a.x1);
    if (two_axes) {
        fft_run<+1>(v, B, adz, g.lQz, mp.jz, true, false, false, a.st);
        fft_run<+1>(v, B, ady, g.lQy, mp.jy, true, false, true, a.st);
    } else {
        fft_run<+1>(v, B, ady, g.lQy, mp.jy, true, false, true, a.st);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) __stcg(&X0[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)], v[m]);
    // 7. inverse of c from A
    if (two_axes) {
        fft_run<+1>(v, A, adz, g.lQz, mp.jz, true, false, false, a.st);
        fft_run<+1>(v, A, ady, g.lQy, mp.jy, true, false, true, a.st);
    } else {
        fft_run<+1>(v, A, ady, g.lQy, mp.jy, true, false, true, a.st);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) __stcg(&X1[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)], v[m]);
}
#undef PFC_KSQ

template <typename R>
__global__ void __launch_bounds__(512, 1) k_line_step2(const Geom g, const Step2Args<R> a) {
    line_step2_body<R>(g, a, blockIdx.x, blockIdx.y);
}

}  // namespace pfc
