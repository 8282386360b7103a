// Middle pass of the three-pass schedule (sm_103a): the R-point part of the y/z transforms.
//
// The y (and z) transform of length n = P R Q is split in three (see pfc_pass.cuh):
//   Yhat[k_p + P (k_r + R k_q)] = sum_{y_q} W_Q^{y_q k_q} W_{RQ}^{y_q k_r}
//                                 sum_{y_r} W_R^{y_r k_r} A[y_q + Q y_r][k_p],
// where A is the row pass's output (P-part done, its twiddle applied). For one k_p, one y/z
// offset q = (z_q, y_q) and a chunk of kx columns, this pass maps the R = Ry Rz rows
// r = y_r + Ry z_r of A to the R rows k_r = k_ry + Ry k_rz of B (the line pass's input):
//   forward  B[k_r] = s W_{Ry Qy}^{y_q k_ry} W_{Rz Qz}^{z_q k_rz} sum_{y_r, z_r} A[r] W_Ry^{y_r k_ry} W_Rz^{z_r k_rz}
//   inverse  A[r]   = s sum_{k_r} conj(W_{Ry Qy}^{y_q k_ry} W_{Rz Qz}^{z_q k_rz}) B[k_r] W_Ry^{-y_r k_ry} W_Rz^{-z_r k_rz}
// with s the caller's scale (the inverse is unnormalised). Rows r and k_r of one (k_p, q) are
// the same R rows of the array, kp QR + r Q + q, so the pass can run in place: a block reads all
// of its values before it writes any. Each element is read once and written once (two sweeps).
//
// Block: MID_CW columns x 8 threads. Phase 1: thread (c, t) takes z index t (< Rz), its Ry values
// from global memory (inverse: twiddled on load), the Ry-point DFT, into shared memory. Phase 2:
// thread (c, t) takes y index t (< Ry), its Rz values from shared memory, the Rz-point DFT
// (forward: then the twiddle), the scale, and writes global memory.
#pragma once

#include "pfc_pass.cuh"

namespace pfc {

constexpr int MID_CW = 32;            // kx columns per block (256 B of FP32 complex per row)
constexpr int MID_THREADS = MID_CW * 8;

template <typename R> struct MidArgs {
    const void *in;       // X' layout (all R rows of every (k_p, q))
    void *out;            // may equal in
    R scale;
    const typename VT<R>::V *tw;   // full table, 2^ltab entries, forward sign
    int edges;            // 1: only the kx = 0 and kx = nx/2 columns (one block per (k_p, q))
};

// W_{Ry Qy}^{y_q k} W_{Rz Qz}^{z_q m}, forward sign
template <typename V>
__device__ __forceinline__ V mid_twiddle(const Geom &g, const V *__restrict__ tw, int yq, int zq, int k, int m) {
    V t = __ldg(&tw[(yq * k) << (g.ltab - g.lRy - g.lQy)]);
    if (g.Rz > 1) t = cmul(t, __ldg(&tw[(zq * m) << (g.ltab - g.lRz - g.lQz)]));
    return t;
}

// DIR = -1 forward, +1 inverse. grid = (column chunks (1 when edges), Q, P).
template <typename R, int DIR>
__global__ void __launch_bounds__(MID_THREADS) k_mid(const Geom g, const MidArgs<R> a) {
    using V = typename VT<R>::V;
    __shared__ V S[64 * MID_CW];
    const int c = threadIdx.x % MID_CW, t = threadIdx.x / MID_CW;
    const int q = blockIdx.y, kp = blockIdx.z;
    const int yq = q & (g.Qy - 1), zq = q >> g.lQy;
    int col;
    bool act;
    if (a.edges) {
        col = c == 0 ? 0 : g.M;
        act = c < 2;
    } else {
        col = blockIdx.x * MID_CW + c;
        act = col < g.xs;
    }
    const V *in = reinterpret_cast<const V *>(a.in);
    V *out = reinterpret_cast<V *>(a.out);
    // element (r, col) of this (k_p, q): row kp QR + r Q + q
    auto at = [&](int r) -> size_t { return (size_t)((kp * g.R + r) * g.Q + q) * g.xs + col; };

    // phase 1: the Ry-point DFT along y_r (forward) or k_ry (inverse) for z index t
    if (act && t < g.Rz) {
        V v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j < g.Ry) {
                v[j] = __ldcg(&in[at(j + g.Ry * t)]);
                if (DIR > 0) v[j] = cscale(ctw<+1>(v[j], mid_twiddle(g, a.tw, yq, zq, j, t)), a.scale);
            }
        }
        dft_small<DIR>(v, g.Ry);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < g.Ry) S[(j + g.Ry * t) * MID_CW + c] = v[j];
    }
    __syncthreads();
    // phase 2: the Rz-point DFT along z_r (forward) or k_rz (inverse) for y index t
    if (act && t < g.Ry) {
        V v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if (m < g.Rz) v[m] = S[(t + g.Ry * m) * MID_CW + c];
        dft_small<DIR>(v, g.Rz);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            if (m < g.Rz) {
                V x = v[m];
                if (DIR < 0) x = cscale(cmul(x, mid_twiddle(g, a.tw, yq, zq, t, m)), a.scale);
                __stcg(&out[at(t + g.Ry * m)], x);
            }
        }
    }
}

}  // namespace pfc
