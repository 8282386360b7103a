// Line pass of the adjoint step (single field).
//
// One semi-implicit step is psi' = A psi - B psi^3 with A = IFFT a FFT, B = IFFT b FFT,
// a = 1/D, b = dt k^2 / D, D = 1 + dt k^2 Lk(k) (the update of Listing 1 applied to Eq. (6)).
// A and B are real and symmetric, so the transpose of the Jacobian J = A - B diag(3 psi^2) is
// J^T = A - diag(3 psi^2) B, and with dD/dr = dt k^2,  d psi'/dr = IFFT(-b psi_hat').
//
// From the X' forms Lam' (of lam_next), Psi' (of psi_n) and C' (of psi_n^3) of one tile this
// kernel forms, per mode,
//     psi_hat' = a psi_hat - b N_hat,   g = -b psi_hat',
//     partial  += w_k Re(conj(Lam_hat) g)       (Parseval, w_k = 1 on kx = 0, nx/2 else 2)
// and writes U' = X' form of A lam_next over Lam' and V' = X' form of B lam_next over Psi'.
// The row passes then give lam_out = U - 3 psi_n^2 V.
//
// Scaling: an X' form holds F_p(x) / (P M), so F(x) = P M DFT_Q(X'); C' holds F_p(psi^3)
// unscaled. With P M = N / (2 Q) the caller scales the partial sums by 1/(2 Q).
#pragma once

#include "pfc_pass.cuh"

namespace pfc {

template <typename R> struct AdjArgs {
    void *lam;            // in: Lam', out: U'
    void *psi;            // in: Psi', out: V' (when vout is null)
    void *vout;           // V' (null: over psi)
    const void *c;        // C'
    double *partials;     // one per block
    UpdR<R> up;
    R PM;                 // P M
    StageTw<typename VT<R>::V> st;
};

template <typename R>
__global__ void __launch_bounds__(512) k_line_adj(const Geom g, const AdjArgs<R> a) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[512];
    V *sm = reinterpret_cast<V *>(smraw);
    const int cg = blockIdx.x, kp = blockIdx.y;
    V *T = sm;
    V *Cs = sm + g.tsz;
    const LineMap mp = line_map(g, threadIdx.x);
    const PadTileAddr ady = tile_y(g, mp);
    const TileAddr adz = tile_z(g, mp);
    const bool two_axes = g.Qz > 1;
    int kpy, kpz;
    line_kp(g, kp, kpy, kpz);
    const int lsy = g.lPy + g.lRy, lsz = g.lPz + g.lRz;
    V v[8];


    // multipliers a, b of register slot m
    const int kx = cg * g.W + mp.w;
    const R fx = a.up.cx * (R)kx;
    auto mult = [&](int m, R &ca, R &cb) {
        const int kqy = two_axes ? mp.yq : mp.jy + m * mp.ny8;
        const int kqz = two_axes ? mp.jz + m * mp.nz8 : 0;
        const int ky = kpy + (kqy << lsy), kz = kpz + (kqz << lsz);
        const int my = ky <= (g.ny >> 1) ? ky : ky - g.ny;
        const int mz = kz <= (g.nz >> 1) ? kz : kz - g.nz;
        const R fy = a.up.cy * (R)my, fz = a.up.cz * (R)mz;
        const R k2 = fx * fx + fy * fy + fz * fz;
        const R inv = (R)1 / ((R)1 + a.up.dt * k2 * lin_symbol<R>(a.up.op[0], k2));
        ca = inv;
        cb = a.up.dt * k2 * inv;
    };

    // 1. N_hat into Cs, psi_hat into registers; g = -b (a P M psi_hat - b N_hat) into Cs
    line_forward(v, g, mp, kp, cg, reinterpret_cast<const V *>(a.c), Cs, ady, adz, false, a.st);
    line_forward(v, g, mp, kp, cg, reinterpret_cast<const V *>(a.psi), T, ady, adz, true, a.st);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        R ca, cb;
        mult(m, ca, cb);
        const int pos = tile_slot(mp, two_axes, ady, adz, m);
        const V n = Cs[pos];
        const R s = ca * a.PM;
        const V p1 = V{s * v[m].x - cb * n.x, s * v[m].y - cb * n.y};
        Cs[pos] = V{-cb * p1.x, -cb * p1.y};
    }
    // 2. Lam_hat into registers; partial sum; B-input into Cs, A-input stays in registers
    line_forward(v, g, mp, kp, cg, reinterpret_cast<const V *>(a.lam), T, ady, adz, true, a.st);
    const R wk = kx == 0 || kx == g.M ? (R)1 : (kx < g.M ? (R)2 : (R)0);
    const R invQ = a.up.invQ;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        R ca, cb;
        mult(m, ca, cb);
        const int pos = tile_slot(mp, two_axes, ady, adz, m);
        const V gv = Cs[pos];
        // padding columns (kx > nx/2) take no part: their contents are whatever the arrays held
        if (kx <= g.M) acc += (double)(wk * (v[m].x * gv.x + v[m].y * gv.y));
        Cs[pos] = V{cb * invQ * v[m].x, cb * invQ * v[m].y};
        v[m] = V{ca * invQ * v[m].x, ca * invQ * v[m].y};
    }
    // 3. U' = inverse of the registers -> lam; V' = inverse of Cs -> psi
    V *U = reinterpret_cast<V *>(a.lam);
    V *Vo = reinterpret_cast<V *>(a.vout ? a.vout : a.psi);
    if (two_axes) {
        fft_run<+1>(v, T, adz, g.lQz, mp.jz, true, true, false, a.st);
        fft_run<+1>(v, T, ady, g.lQy, mp.jy, true, false, true, a.st);
    } else {
        fft_run<+1>(v, T, ady, g.lQy, mp.jy, true, true, true, a.st);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) U[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)] = v[m];
    __syncthreads();   // the B-inputs written to Cs by every thread
    if (two_axes) {
        fft_run<+1>(v, Cs, adz, g.lQz, mp.jz, true, false, false, a.st);
        fft_run<+1>(v, Cs, ady, g.lQy, mp.jy, true, false, true, a.st);
    } else {
        fft_run<+1>(v, Cs, ady, g.lQy, mp.jy, true, false, true, a.st);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) Vo[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)] = v[m];

    // 4. deterministic block sum of the partials
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 1; s < (int)blockDim.x; s <<= 1) {
        if ((threadIdx.x & (2 * s - 1)) == 0 && threadIdx.x + s < blockDim.x) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.partials[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

}  // namespace pfc
