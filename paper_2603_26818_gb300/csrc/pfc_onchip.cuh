// Small 2D domains stepped entirely in shared memory: one block per domain keeps the domain's
// half spectrum on chip for all the steps of a call (zero HBM sweeps per step; the real field is
// read once at the entry and written once at the exit).
//
// A domain of ny x nx points (ny <= 128, nx <= 128) holds two half spectra of ny rows of
// nx/2 + 1 bins in shared memory (rows at a stride rs, the XOR swizzle of pfc_fft.cuh inside a
// row): S0, the carried state F(psi - mean) / (ny M) (M = nx/2, the mean carried in FP64 as in
// the plans), and S1, the work array. One semi-implicit step (the update of Listing 1):
//   S1 = S0; inverse y transforms of the columns; the kx = 0 and nx/2 columns, which must be real
//   in row space, projected and written back to S0; per row the real-transform pre-processing
//   and the inverse x transform (the row-pass conventions of pfc_pass.cuh); psi^3 - mean^3 in
//   registers; the forward x transform and post-processing; forward y transforms: S1 = F(psi^3);
//   then per bin S0 <- (S0 - dt k^2 S1 / (ny M)) / (1 + dt k^2 Lk(k)), S0 = 0 at k = 0.
// Transforms of one row or column are done by nx/16 or ny/8 threads of one warp (warp barriers).
#pragma once

#include <type_traits>

#include "pfc_pass.cuh"

namespace pfc {

constexpr int ONCHIP_THREADS = 256;
constexpr int ONCHIP_MAX = 128;   // largest extent of an on-chip domain

template <typename R> struct OnchipArgs {
    void *state;              // packed real state of the batch (in/out)
    const int64_t *moff;      // element offset of each member in the packed state
    const double *mean;       // each member's FP64 mean
    const R *r;               // each member's r (one-mode operator)
    int64_t nsteps;
    UpdR<R> up;               // dt, cx, cy, inv_halfN = 2 / N; op[0] for the kind
    const typename VT<R>::V *tw;   // full table, 2^ltab entries
    StageTw<typename VT<R>::V> st;
};

// shared-memory bytes of an on-chip domain: S0, S1 and two projection columns
__host__ __device__ inline size_t onchip_smem(int ny, int nx, size_t vb) {
    const int rs = ((nx / 2 + 1) + 15) / 16 * 16;
    return (size_t)(2 * ny * rs + 2 * ny) * vb;
}

// The steps of one member by one block (any block size that is a multiple of 32 and at least
// 2 ny / 8); k_onchip runs it as its own block, the persistent batch kernel once per on-chip item.
template <typename R>
__device__ __forceinline__ void onchip_body(const Geom &g, const OnchipArgs<R> &a, int member) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *S0 = reinterpret_cast<V *>(smraw);
    V *S1 = S0 + g.ny * g.rs;
    V *E = S1 + g.ny * g.rs;   // two projection columns of ny values
    const int tid = threadIdx.x, nt = blockDim.x;
    const int M = g.M, lM = g.lM, hM = M >> 1, ny = g.ny, rs = g.rs;
    const R mean = (R)a.mean[member];
    V *field = reinterpret_cast<V *>(a.state) + a.moff[member] / 2;   // rows of M real pairs
    const R sc = (R)1 / ((R)ny * (R)M);

    // a column transform of length ny: Ty threads per column, columns in rounds
    const int Ty = ny >> 3, CPB = nt / Ty;
    const int ncolr = (M + 1 + CPB - 1) / CPB;
    auto cols = [&](V *S, auto sgn) {
        constexpr int SG = decltype(sgn)::value;
        for (int rd = 0; rd < ncolr; ++rd) {
            const int kx = rd * CPB + tid / Ty, j = tid % Ty;
            const bool act = kx <= M;
            const TileAddr ad{row_swz(act ? kx : 0), rs};
            V v[8];
            fft_run<SG>(v, S, ad, g.lny, j, act, false, false, a.st, RowBarrier{0, Ty});
        }
    };
    // the x transforms of every row: Tr threads per row, rows in rounds
    const int Tr = M >> 3, RPB = nt / Tr;
    const int nrowr = (ny + RPB - 1) / RPB;
    // real-transform post-processing (forward) of every row's column pairs, in place
    auto post = [&](V *S) {
        for (int e = tid; e < ny * (hM + 1); e += nt) {
            const int y = e / (hM + 1), kk = e % (hM + 1);
            const bool k0 = kk == 0, self = kk == hM;
            const int ca = kk, cb = k0 ? M : M - kk;
            V *row = S + y * rs;
            const V w = __ldg(&a.tw[ca << (g.ltab - g.lnx)]);
            const V za = row[row_swz(k0 ? 0 : ca)];
            const V zb = (k0 || self) ? za : row[row_swz(cb)];
            V xa, xb;
            r2c_post_pair<V, R>(za, zb, w, k0, xa, xb);
            row[row_swz(ca)] = xa;
            if (!self) row[row_swz(cb)] = xb;
        }
    };
    // real-transform pre-processing (inverse) of every row's column pairs, in place
    auto pre = [&](V *S) {
        for (int e = tid; e < ny * (hM + 1); e += nt) {
            const int y = e / (hM + 1), kk = e % (hM + 1);
            const bool k0 = kk == 0, self = kk == hM;
            const int ca = kk, cb = k0 ? M : M - kk;
            V *row = S + y * rs;
            const V w = __ldg(&a.tw[ca << (g.ltab - g.lnx)]);
            const V xa = row[row_swz(ca)], xb = self ? xa : row[row_swz(cb)];
            V za, zb;
            c2r_pre_pair<V, R>(xa, xb, w, k0, za, zb);
            row[row_swz(ca)] = za;
            if (!k0 && !self) row[row_swz(cb)] = zb;
        }
    };

    // ---- entry: S0 = F(psi - mean) / (ny M) ----
    for (int e = tid; e < ny * M; e += nt) {
        const int y = e >> lM, i = e & (M - 1);
        V v = field[(size_t)y * M + i];
        S0[y * rs + row_swz(i)] = V{v.x - mean, v.y - mean};
    }
    __syncthreads();
    for (int rd = 0; rd < nrowr; ++rd) {
        const int y = rd * RPB + tid / Tr, j = tid % Tr;
        V v[8];
        fft_run<-1>(v, S0, RowAddr{(y < ny ? y : 0) * rs}, lM, j, y < ny, false, false, a.st, RowBarrier{0, Tr});
    }
    __syncthreads();
    post(S0);
    __syncthreads();
    cols(S0, std::integral_constant<int, -1>());
    __syncthreads();
    for (int e = tid; e < ny * (M + 1); e += nt) {
        const int y = e / (M + 1), k = e % (M + 1);
        V &x = S0[y * rs + row_swz(k)];
        x = cscale(x, sc);
    }
    __syncthreads();

    OpR<R> op = a.up.op[0];
    op.r = a.r[member];
    for (int64_t s = 0; s < a.nsteps; ++s) {
        for (int e = tid; e < ny * rs; e += nt) S1[e] = S0[e];
        __syncthreads();
        cols(S1, std::integral_constant<int, +1>());
        __syncthreads();
        // Hermitian projection of the kx = 0 and nx/2 columns: their row-space values must be
        // real; the imaginary parts (rounding) are invisible to psi^3 but would be multiplied by
        // 1/D > 1 at the unstable wavenumbers every step. S0 gets F_y of the real parts.
        for (int e = tid; e < 2 * ny; e += nt) {
            const int c = e / ny, y = e % ny;
            E[c * ny + y] = V{S1[y * rs + row_swz(c ? M : 0)].x, (R)0};
        }
        __syncthreads();
        {
            const int c = tid / Ty, j = tid % Ty;
            V v[8];
            fft_run<-1>(v, E, TileAddr{(c < 2 ? c : 0) * ny, 1}, g.lny, j, c < 2, false, false, a.st, RowBarrier{0, Ty});
        }
        __syncthreads();
        for (int e = tid; e < 2 * ny; e += nt) {
            const int c = e / ny, y = e % ny;
            S0[y * rs + row_swz(c ? M : 0)] = cscale(E[c * ny + y], (R)1 / (R)ny);
        }
        pre(S1);
        __syncthreads();
        for (int rd = 0; rd < nrowr; ++rd) {
            const int y = rd * RPB + tid / Tr, j = tid % Tr;
            const bool act = y < ny;
            const RowAddr ad{(act ? y : 0) * rs};
            V v[8];
            fft_run<+1>(v, S1, ad, lM, j, act, false, true, a.st, RowBarrier{0, Tr});
            cube_shifted(v, mean);
            fft_run<-1>(v, S1, ad, lM, j, act, true, false, a.st, RowBarrier{0, Tr});
        }
        __syncthreads();
        post(S1);
        __syncthreads();
        cols(S1, std::integral_constant<int, -1>());
        __syncthreads();
        for (int e = tid; e < ny * (M + 1); e += nt) {
            const int y = e / (M + 1), kx = e % (M + 1);
            const int my = y <= (ny >> 1) ? y : y - ny;
            const R fx = a.up.cx * (R)kx, fy = a.up.cy * (R)my;
            const R k2 = fx * fx + fy * fy;
            const R inv = (R)1 / ((R)1 + a.up.dt * k2 * lin_symbol<R>(op, k2));
            const R ca = inv, cb = a.up.dt * k2 * inv * a.up.inv_halfN;
            const int pos = y * rs + row_swz(kx);
            const V x = S0[pos], c = S1[pos];
            S0[pos] = (kx == 0 && y == 0) ? V{(R)0, (R)0} : V{ca * x.x - cb * c.x, ca * x.y - cb * c.y};
        }
        __syncthreads();
    }

    // ---- exit: psi = F^-1(S0) + mean ----
    cols(S0, std::integral_constant<int, +1>());
    __syncthreads();
    pre(S0);
    __syncthreads();
    for (int rd = 0; rd < nrowr; ++rd) {
        const int y = rd * RPB + tid / Tr, j = tid % Tr;
        V v[8];
        fft_run<+1>(v, S0, RowAddr{(y < ny ? y : 0) * rs}, lM, j, y < ny, false, false, a.st, RowBarrier{0, Tr});
    }
    __syncthreads();
    for (int e = tid; e < ny * M; e += nt) {
        const int y = e >> lM, i = e & (M - 1);
        const V v = S0[y * rs + row_swz(i)];
        field[(size_t)y * M + i] = V{v.x + mean, v.y + mean};
    }
}

template <typename R>
__global__ void __launch_bounds__(ONCHIP_THREADS) k_onchip(const Geom g, const OnchipArgs<R> a) {
    onchip_body<R>(g, a, blockIdx.x);
}

}  // namespace pfc
