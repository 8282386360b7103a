// Row pass of the fused adjoint step (single field, two-pass plans).
//
// The adjoint of one semi-implicit step is lam_n = A lam_{n+1} - 3 psi_n^2 (B lam_{n+1})
// (pfc_adjoint.cuh gives A, B). The adjoint line pass leaves U' and V', the X' forms of
// A lam_{n+1} and B lam_{n+1}; the state's X' form Psi'_n is kept from the forward run. Per row
// group this pass takes all three back to row space (the inverse P-part, the real-transform
// pre-processing and the inverse x transform of the psi^3 row pass), forms
//     lam_n = u - 3 (psi_n)^2 v,    psi_n = (row inverse of Psi'_n) + mean,
// and transforms lam_n forward to its X' form (scale 1 / (P M)) for the next adjoint line pass:
// three reads and one write of a half spectrum, where the separate row passes of the one-step
// adjoint read the real psi_n and lam, write lam_out and read it back.
//
// Shared memory: two buffers of the group's rows (A, B), the split twiddles and the saved edge
// values of the row pass layout. A: psi_n, then 3 psi_n^2; B: v, then 3 psi_n^2 v; A: u, then
// lam_n (in registers between the inverse and forward transforms).
#pragma once

#include "pfc_pass.cuh"

namespace pfc {

template <typename R>
__global__ void __launch_bounds__(512, 1) k_row_adj2(const Geom g, const RowArgs<R> a) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *A = reinterpret_cast<V *>(smraw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int P = g.P, rows = g.gpc * P, M = g.M, lM = g.lM;
    const int grp0 = blockIdx.x * g.gpc;
    V *B = A + rows * g.rs;
    V *stw = B + rows * g.rs;
    const R mean = a.mean ? (R)a.mean[0] : (R)0;
    for (int t = tid; t < rows; t += nt) {
        const int gi = t / P, kp = t % P;
        stw[t] = split_twiddle(g, a.tw, grp0 + gi, kp / g.Py, kp % g.Py);
    }
    __syncthreads();
    // row space of an X'-layout array into buffer S (phases A and B of the row pass)
    auto to_rows = [&](const void *src, V *S) {
        const V *X = reinterpret_cast<const V *>(src);
        if (g.Pz > 1) {
            row_phase_a<R>(g, S, X, grp0, stw);
            __syncthreads();
            row_phase_b<R, false>(g, S, nullptr, X, grp0, a.tw, stw, nullptr);
        } else {
            row_phase_b<R, true>(g, S, nullptr, X, grp0, a.tw, stw, nullptr);
        }
        __syncthreads();
    };
    const int Tr = M >> 3, RB = nt / Tr;
    const RowBarrier bar = Tr <= 32 ? RowBarrier{0, Tr} : RowBarrier{0, nt};

    // A = 3 psi_n^2
    to_rows(a.aux3, A);
    for (int rb = 0; rb < rows; rb += RB) {
        const int r = rb + tid / Tr, j = tid % Tr;
        const bool act = r < rows;
        const RowAddr ad{(act ? r : 0) * g.rs};
        V v[8];
        fft_run<+1>(v, A, ad, lM, j, act, false, true, a.st, bar);
        bar.sync();   // the row's last-stage loads are done before its slots are overwritten
        if (act) {
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const R p0 = v[m].x + mean, p1 = v[m].y + mean;
                A[ad.at(j + m * Tr)] = V{(R)3 * p0 * p0, (R)3 * p1 * p1};
            }
        }
    }
    __syncthreads();
    // B = 3 psi_n^2 v
    to_rows(a.aux2, B);
    for (int rb = 0; rb < rows; rb += RB) {
        const int r = rb + tid / Tr, j = tid % Tr;
        const bool act = r < rows;
        const RowAddr ad{(act ? r : 0) * g.rs};
        V v[8];
        fft_run<+1>(v, B, ad, lM, j, act, false, true, a.st, bar);
        bar.sync();
        if (act) {
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const V w = A[ad.at(j + m * Tr)];
                B[ad.at(j + m * Tr)] = V{w.x * v[m].x, w.y * v[m].y};
            }
        }
    }
    __syncthreads();
    // A = u, then lam_n = u - B, forward
    to_rows(a.in, A);
    for (int rb = 0; rb < rows; rb += RB) {
        const int r = rb + tid / Tr, j = tid % Tr;
        const bool act = r < rows;
        const RowAddr ad{(act ? r : 0) * g.rs};
        V v[8];
        fft_run<+1>(v, A, ad, lM, j, act, false, true, a.st, bar);
        if (act) {
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const V w = B[ad.at(j + m * Tr)];
                v[m] = V{v[m].x - w.x, v[m].y - w.y};
            }
        }
        fft_run<-1>(v, A, ad, lM, j, act, true, false, a.st, bar);
    }
    __syncthreads();
    V *out = reinterpret_cast<V *>(a.out);
    row_phase_d<R>(g, A, out, grp0, a.tw, stw, a.scale);
    if (g.Pz > 1) {
        __syncthreads();
        row_phase_e<R>(g, A, out, grp0, stw, a.scale);
    }
}

// shared memory of k_row_adj2 for a geometry: two row buffers and the split twiddles
inline size_t row_adj2_smem(const Geom &g, size_t vb) {
    return (size_t)(2 * g.gpc * g.P * g.rs + g.gpc * g.P) * vb;
}

}  // namespace pfc
