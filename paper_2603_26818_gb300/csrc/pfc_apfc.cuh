// Amplitude-expansion PFC (pfc_apfc_* of pfc.h): n complex amplitude fields eta_j on a
// periodic grid, the density psi = psibar + sum_j [eta_j exp(i k_j . r) + c.c.]. One step is the
// semi-implicit update of Listing 1 per amplitude at the shifted wavevector:
//   S_j <- (S_j - dt Q C_j / N) / (1 + dt Q L(Q)),   Q = |k_j + q|^2,
// S_j = F(eta_j) / N the carried state, C_j = F(N_j) and N_j the component of psi^3 at k_j:
//   N_j = 3 psibar^2 eta_j + sum over the resonances of amplitude j of coef e_a e_b (e_c),
// e_{+m} = eta_m, e_{-m} = conj(eta_m), the resonances (k_a + k_b = k_j with coef 3 psibar times
// the ordered count, k_a + k_b + k_c = k_j with the ordered count) listed by the host.
// Transforms are complex (c2c), mixed radix (2, 3, 4, 5, 7, 8), one warp a line, with the
// Stockham engine of pfc_mixed.cuh; a step in 2D is the y inverse pass (S -> T), the x pass (per
// row: every amplitude's inverse x transform, N_j at every point from all amplitudes' values,
// the forward x transforms; T in place) and the y forward pass with the update (T, S -> S):
// 7 sweeps of the amplitude fields; in 3D the z and y passes on both sides, 11 sweeps.
#pragma once

#include "pfc_mixed.cuh"

namespace pfc {

constexpr int AP_MAXAMP = 16;

struct ApGeom {
    int nx, ny, nz, ndim, namp;
    MrAxis ax[3];       // x, y, z (complex lengths)
    int64_t npts;       // points of one amplitude field
};

template <typename R> struct ApArgs {
    const typename VT<R>::V *tw;   // the axes' stage twiddles
    R scale;                       // output scale of a forward column pass
    R dt, inv_n;                   // the update's dt and 1 / npts
    R cx, cy, cz;                  // 2 pi / (n dx) per axis
    R kx[AP_MAXAMP], ky[AP_MAXAMP], kz[AP_MAXAMP];   // k_j
    OpR<R> op;
    R c1;                          // 3 psibar^2
    const int *term_beg;           // terms of amplitude j: [term_beg[j], term_beg[j + 1])
    const int4 *terms;             // (a, b, c, 0): signed modes, c = 0 for a quadratic term
    const R *coef;                 // the terms' coefficients
};

// signed mode s of the amplitudes at one point: X(j) is the buffer of amplitude j
template <typename V>
__device__ __forceinline__ V ap_mode(const V *base, size_t stride, int s, int i) {
    const V v = base[(size_t)((s > 0 ? s : -s) - 1) * stride + i];
    return s > 0 ? v : V{v.x, -v.y};
}

template <typename V> __device__ __forceinline__ V ap_mul(V p, V q) {
    return V{p.x * q.x - p.y * q.y, p.x * q.y + p.y * q.x};
}

enum { AP_ROW_FWD = 0, AP_ROW_INV = 1 };

// Entry and exit x passes: one warp a line (row r of amplitude f), blockDim.x / 32 lines a
// block; forward (unscaled) or inverse (unnormalised) transform from in to out.
template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_ap_row_io(const __grid_constant__ ApGeom g, const __grid_constant__ ApArgs<R> a,
                                                   const void *in, void *out) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rows = (int64_t)g.ny * g.nz;
    const int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;   // f rows + r
    if (line >= rows * g.namp) return;   // a whole warp; the kernel has no block barrier
    const int n = g.nx;
    V *A = reinterpret_cast<V *>(smraw) + (size_t)warp * 2 * n;
    V *B = A + n;
    mr_warp_load(A, reinterpret_cast<const V *>(in) + line * n, n, lane);
    __syncwarp();
    const V *Z = MODE == AP_ROW_FWD ? mr_fft<-1>(A, B, g.ax[0], a.tw, lane) : mr_fft<+1>(A, B, g.ax[0], a.tw, lane);
    V *dst = reinterpret_cast<V *>(out) + line * n;
    for (int i = lane; i < n; i += 32) __stcg(&dst[i], Z[i]);
}

// The x pass of a step, T in place: rows_per_block rows a block, the namp warps of a row one
// amplitude each. Every warp takes its amplitude's row to real space; after a block barrier each
// warp forms N_f at every point of its row from all the row's amplitudes; after a second barrier
// (the real-space buffers are free) each warp transforms its N_f forward and stores it.
template <typename R>
__global__ void __launch_bounds__(512) k_ap_row_nl(const __grid_constant__ ApGeom g, const __grid_constant__ ApArgs<R> a,
                                                   void *T, int rows_per_block) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rr = warp / g.namp, f = warp - rr * g.namp;
    const int64_t r = (int64_t)blockIdx.x * rows_per_block + rr;
    const bool act = rr < rows_per_block && r < (int64_t)g.ny * g.nz;
    const int n = g.nx;
    // buffers of line (rr, f): A at (rr namp + f) 2n, B = A + n; the real-space values end in A
    // or B by the parity of the stage count (the same for every line)
    V *rowbase = reinterpret_cast<V *>(smraw) + (size_t)rr * g.namp * 2 * n;
    V *A = rowbase + (size_t)f * 2 * n;
    V *B = A + n;
    const bool odd = g.ax[0].nst & 1;
    V *X = odd ? B : A, *Y = odd ? A : B;
    V *line = reinterpret_cast<V *>(T) + (size_t)f * g.npts + (size_t)(act ? r : 0) * n;
    if (act) {
        mr_warp_load(A, line, n, lane);
        __syncwarp();
        mr_fft<+1>(A, B, g.ax[0], a.tw, lane);
    }
    __syncthreads();
    if (act) {
        const V *Xs = rowbase + (odd ? n : 0);   // amplitude j's real-space row at Xs + j 2n
        const size_t js = 2 * (size_t)n;
        const int t0 = a.term_beg[f], t1 = a.term_beg[f + 1];
        // four points a lane at a time (i0, i0 + 32, ...): one read of each term for the four
        constexpr int PU = 4;
        for (int i0 = lane; i0 < n; i0 += 32 * PU) {
            int ii[PU];
            V acc[PU];
#pragma unroll
            for (int u = 0; u < PU; ++u) {
                const int i = i0 + 32 * u;
                ii[u] = i < n ? i : n - 1;   // past the end: a valid point, not stored
                const V e = X[ii[u]];
                acc[u] = V{a.c1 * e.x, a.c1 * e.y};
            }
            for (int t = t0; t < t1; ++t) {
                const int4 tm = __ldg(&a.terms[t]);
                const R c = __ldg(&a.coef[t]);
#pragma unroll
                for (int u = 0; u < PU; ++u) {
                    V p = ap_mul(ap_mode(Xs, js, tm.x, ii[u]), ap_mode(Xs, js, tm.y, ii[u]));
                    if (tm.z != 0) p = ap_mul(p, ap_mode(Xs, js, tm.z, ii[u]));
                    acc[u].x += c * p.x;
                    acc[u].y += c * p.y;
                }
            }
#pragma unroll
            for (int u = 0; u < PU; ++u)
                if (i0 + 32 * u < n) Y[i0 + 32 * u] = acc[u];
        }
    }
    __syncthreads();
    if (act) {
        const V *Z = mr_fft<-1>(Y, X, g.ax[0], a.tw, lane);
        for (int i = lane; i < n; i += 32) __stcg(&line[i], Z[i]);
    }
}

enum { AP_COL_FWD = 0, AP_COL_INV = 1, AP_COL_UPDATE = 2 };

// The wavenumber index of FFT bin i of an axis of n points (the middle bin of an even axis is
// the negative frequency -n/2)
__device__ __forceinline__ int ap_freq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

// A pass along axis (1 = y, 2 = z) on W = blockDim.x / 32 columns of amplitude blockIdx.z, one
// warp a column; grid = (column chunks, the other axis' extent, namp).
//   AP_COL_FWD / AP_COL_INV: out = scale * F(in) / out = F^-1(in) (in may equal out);
//   AP_COL_UPDATE (the last forward axis): C = F(in), then
//     S <- (S - dt Q C / N) / (1 + dt Q L(Q)) with S = out (read and written).
template <typename R, int MODE>
__global__ void __launch_bounds__(512) k_ap_col(const __grid_constant__ ApGeom g, const __grid_constant__ ApArgs<R> a,
                                                int axis, const void *in, void *out) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    const MrAxis &ax = g.ax[axis];
    const int n = ax.n, tid = threadIdx.x, nt = blockDim.x, W = nt >> 5, lW = __ffs(W) - 1;
    const int warp = tid >> 5, lane = tid & 31;
    const int CS = mr_col_stride(n);
    V *A = reinterpret_cast<V *>(smraw);
    V *B = A + (size_t)W * CS;
    const int c0 = blockIdx.x * W, other = blockIdx.y, f = blockIdx.z;
    const int64_t step = axis == 1 ? (int64_t)g.nx : (int64_t)g.ny * g.nx;
    const int64_t base0 = (size_t)f * g.npts + (axis == 1 ? (int64_t)other * g.ny * g.nx : (int64_t)other * g.nx) + c0;
    const int wv = min(W, g.nx - c0);
    const int total = n << lW;
    const V *src = reinterpret_cast<const V *>(in);
    for (int e0 = tid; e0 < total; e0 += nt * MR_U) {
        V t[MR_U];
#pragma unroll
        for (int u = 0; u < MR_U; ++u) {
            const int e = e0 + u * nt, i = e >> lW, w = e & (W - 1);
            t[u] = V{(R)0, (R)0};
            if (e < total && w < wv) t[u] = __ldcg(&src[base0 + i * step + w]);
        }
#pragma unroll
        for (int u = 0; u < MR_U; ++u) {
            const int e = e0 + u * nt, i = e >> lW, w = e & (W - 1);
            if (e < total) A[w * CS + i] = t[u];
        }
    }
    __syncthreads();
    const V *res;
    if (MODE == AP_COL_INV) res = mr_fft<+1>(A + warp * CS, B + warp * CS, ax, a.tw, lane);
    else res = mr_fft<-1>(A + warp * CS, B + warp * CS, ax, a.tw, lane);
    res -= warp * CS;   // the same buffer for every column (the same number of stages)
    __syncthreads();
    V *dst = reinterpret_cast<V *>(out);
    R kjx = 0, kjy = 0, kjz = 0;
    if (MODE == AP_COL_UPDATE) {
        kjx = a.kx[f];
        kjy = a.ky[f];
        kjz = a.kz[f];
    }
    for (int e0 = tid; e0 < total; e0 += nt * MR_U) {
        V sv[MR_U];
        if (MODE == AP_COL_UPDATE) {
#pragma unroll
            for (int u = 0; u < MR_U; ++u) {
                const int e = e0 + u * nt, i = e >> lW, w = e & (W - 1);
                if (e < total && w < wv) sv[u] = __ldcg(&dst[base0 + i * step + w]);
            }
        }
#pragma unroll
        for (int u = 0; u < MR_U; ++u) {
            const int e = e0 + u * nt, i = e >> lW, w = e & (W - 1);
            if (e >= total || w >= wv) continue;
            const V c = res[w * CS + i];
            const int64_t idx = base0 + i * step + w;
            if (MODE != AP_COL_UPDATE) {
                __stcg(&dst[idx], MODE == AP_COL_FWD ? cscale(c, a.scale) : c);
                continue;
            }
            const int ix = c0 + w;
            const int iy = axis == 1 ? i : other, iz = axis == 1 ? other : i;
            const R qx = kjx + a.cx * (R)ap_freq(ix, g.nx);
            const R qy = kjy + a.cy * (R)ap_freq(iy, g.ny);
            const R qz = g.nz > 1 ? kjz + a.cz * (R)ap_freq(iz, g.nz) : kjz;
            const R Q = qx * qx + qy * qy + qz * qz;
            const R inv = (R)1 / ((R)1 + a.dt * Q * lin_symbol<R>(a.op, Q));
            const R cb = a.dt * Q * inv * a.inv_n;
            __stcg(&dst[idx], V{inv * sv[u].x - cb * c.x, inv * sv[u].y - cb * c.y});
        }
    }
}

// shared-memory bytes of the passes
inline size_t ap_row_smem(int nx, int lines, size_t vb) { return (size_t)lines * 2 * nx * vb; }

}  // namespace pfc
