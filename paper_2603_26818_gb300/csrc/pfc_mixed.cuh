// Grids whose extents are not all powers of two (n = 2^a 3^b 5^c 7^d, nx even): the paper's own
// sizes (750^3, 900^3, 1400^3). One pass per axis, each transform a mixed-radix Stockham FFT in
// shared memory:
//   state S = F(psi - mean) / (ny nz M), the standard half spectrum (nz, ny, nx/2 + 1), rows of xs;
//   one semi-implicit step (the update of Listing 1):
//     z inverse S -> T, y inverse T (2D: S -> T), x pass T -> C (per row: real-transform
//     pre-processing, inverse M-point transform, psi^3 - mean^3 in registers, forward transform,
//     post-processing; the real parts of the kx = 0 and nx/2 columns saved in E), y forward C,
//     [the Hermitian projection: E forward in y and z, into S's kx = 0 and nx/2 columns],
//     z forward C with the update S <- (S - dt k^2 C / (ny nz M)) / (1 + dt k^2 Lk)
//     (2D: y forward with the update): 11 sweeps of a half spectrum a step in 3D, 7 in 2D.
// A transform of length n: stages of radix r in {2, 3, 4, 5, 7, 8} (Stockham auto-sort, stage s
// with Ns = the product of the earlier radices: butterfly b in [0, n/r) takes x[b + m n/r],
// m < r, multiplies by W_{r Ns}^{m (b mod Ns)}, and stores the r-point DFT at
// (b - b mod Ns) r + b mod Ns + m Ns). One warp owns a line: the stages alternate between two
// shared-memory buffers (out of place, a __syncwarp between stages), a lane takes butterflies
// b = lane, lane + 32, ... one at a time, so a thread holds at most 8 values. The odd radices
// come first: the stride-r stores of the first stage (Ns = 1) then hit distinct banks, and once
// Ns > 1 a warp's stores are runs of consecutive elements. Reads are always consecutive. Twiddles are FP64-generated on the host (rounded once for FP32); the roots of the
// odd radices are constants of the small-DFT code.
//
// Global memory is read in batches: a thread issues MR_U loads before it stores any of them to
// shared memory (a warp a line leaves few threads an SM, and one load in flight a thread keeps
// HBM far from busy).
#pragma once

#include "pfc_pass.cuh"

namespace pfc {

constexpr int MR_MAXST = 14;

// One transform length: its radices and where its tables start.
struct MrAxis {
    int n, nst;
    int radix[MR_MAXST];
    int ns[MR_MAXST];
    int twoff[MR_MAXST];   // stage s's twiddles W_{r Ns}^{m k} at twoff[s] + m Ns + k
};

struct MrGeom {
    int nx, ny, nz, M, xs;      // xs: complex stride of the half spectrum's rows
    int ndim;
    MrAxis ax[3];               // x (length M), y, z
    int64_t nstd;               // complex values of the half spectrum (nz ny xs)
    int64_t nreal;
};

template <typename R> struct MrArgs {
    const typename VT<R>::V *tw;   // the axes' stage twiddles (ax[a].twoff indexes into it)
    const typename VT<R>::V *twx;  // exp(-2 pi i t / nx), t < nx (real-transform processing)
    const double *mean;
    R scale;
    UpdR<R> up;                    // dt, cx, cy, cz, inv_halfN = 1 / (ny nz M); op[0]
};

// cos and sin of 2 pi m / R for the odd radices, m = 1 .. (R - 1) / 2
__host__ __device__ constexpr double odd_cos(int R, int m) {
    return R == 3 ? -0.5
         : R == 5 ? (m == 1 ? 0.3090169943749474241023 : -0.8090169943749474241023)
                  : (m == 1 ? 0.6234898018587335305250 : m == 2 ? -0.2225209339563144042889 : -0.9009688679024191262361);
}
__host__ __device__ constexpr double odd_sin(int R, int m) {
    return R == 3 ? 0.8660254037844386467637
         : R == 5 ? (m == 1 ? 0.9510565162951535721164 : 0.5877852522924731291687)
                  : (m == 1 ? 0.7818314824680298087084 : m == 2 ? 0.9749279121818236070181 : 0.4338837391175581204758);
}

// x[k] <- sum_j x[j] exp(S 2 pi i j k / R), natural order. Odd R: with a_j = x_j + x_{R-j},
// b_j = x_j - x_{R-j} (j = 1 .. (R-1)/2), X_k = x_0 + sum_j cos(2 pi j k / R) a_j
// + S i sum_j sin(2 pi j k / R) b_j and X_{R-k} the same with -S i.
template <int S, int R, typename V>
__device__ __forceinline__ void mr_dft(V (&x)[R]) {
    if constexpr (R == 2) {
        dft2<S>(x[0], x[1]);
    } else if constexpr (R == 4) {
        dft4<S>(x[0], x[1], x[2], x[3]);
    } else if constexpr (R == 8) {
        dft8<S>(x);
    } else {
        using T = typename ElemOf<V>::R;
        constexpr int H = (R - 1) / 2;
        V a[H], b[H];
        V y0 = x[0];
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            a[j - 1] = cadd(x[j], x[R - j]);
            b[j - 1] = csub(x[j], x[R - j]);
            y0 = cadd(y0, a[j - 1]);
        }
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            V re = x[0], im{(T)0, (T)0};
#pragma unroll
            for (int j = 1; j <= H; ++j) {
                const int m = (j * k) % R;
                const int mp = m <= H ? m : R - m;
                re = cadd(re, cscale(a[j - 1], (T)odd_cos(R, mp)));
                im = cadd(im, cscale(b[j - 1], (T)(m <= H ? odd_sin(R, mp) : -odd_sin(R, mp))));
            }
            const V si = cmul_i<S>(im);
            x[k] = cadd(re, si);
            x[R - k] = csub(re, si);
        }
        x[0] = y0;
    }
}


// one stage of radix R, src -> dst, the butterflies strided over the T threads of the line:
// butterfly b = q Ns + k (th, th + T, ...), with q and k stepped, not divided, from one b to the
// next
template <int S, int R, typename V>
__device__ __forceinline__ void mr_stage(const V *src, V *dst, const MrAxis &ax, int s, const V *tw, int th,
                                         int T) {
    const int nb = ax.n / R, Ns = ax.ns[s];
    const V *t = tw + ax.twoff[s];
    const int dq = T / Ns, dk = T - dq * Ns;
    int q = th / Ns, k = th - q * Ns;
    for (int b = th; b < nb; b += T) {
        V v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = src[b + m * nb];
        if (Ns > 1) {
#pragma unroll
            for (int m = 1; m < R; ++m) v[m] = ctw<S>(v[m], __ldg(&t[m * Ns + k]));
        }
        mr_dft<S, R>(v);
        V *d = dst + q * (R * Ns) + k;
#pragma unroll
        for (int m = 0; m < R; ++m) d[m * Ns] = v[m];
        q += dq;
        k += dk;
        if (k >= Ns) {
            k -= Ns;
            ++q;
        }
    }
}

// The transform of one line by the T threads of a line group (th its thread index): input in
// buffer a (natural order), b the other buffer; returns the buffer that holds the result. Every
// thread of the group calls it. Between stages the group syncs on its warp (T = 32) or on the
// named barrier bar_id over T threads.
template <int S, typename V>
__device__ __forceinline__ V *mr_fft_g(V *a, V *b, const MrAxis &ax, const V *tw, int th, int T, int bar_id) {
    for (int s = 0; s < ax.nst; ++s) {
        switch (ax.radix[s]) {
            case 2: mr_stage<S, 2>(a, b, ax, s, tw, th, T); break;
            case 3: mr_stage<S, 3>(a, b, ax, s, tw, th, T); break;
            case 4: mr_stage<S, 4>(a, b, ax, s, tw, th, T); break;
            case 5: mr_stage<S, 5>(a, b, ax, s, tw, th, T); break;
            case 7: mr_stage<S, 7>(a, b, ax, s, tw, th, T); break;
            default: mr_stage<S, 8>(a, b, ax, s, tw, th, T); break;
        }
        if (T == 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(T) : "memory");
        V *t = a;
        a = b;
        b = t;
    }
    return a;
}

// The transform of one line by one warp (lane its lane index).
template <int S, typename V>
__device__ __forceinline__ V *mr_fft(V *a, V *b, const MrAxis &ax, const V *tw, int lane) {
    return mr_fft_g<S>(a, b, ax, tw, lane, 32, 0);
}

enum { MR_ROW_CUBE = 0, MR_ROW_FWD = 1, MR_ROW_INV = 2 };

constexpr int MR_U = 8;   // global loads a thread issues before it stores them to shared memory

// buf[i] = src[i], i < cnt, by the 32 lanes of a warp in batches of MR_U loads a lane
template <typename V>
__device__ __forceinline__ void mr_warp_load(V *buf, const V *src, int cnt, int lane) {
    for (int i0 = lane; i0 < cnt; i0 += 32 * MR_U) {
        V t[MR_U];
#pragma unroll
        for (int u = 0; u < MR_U; ++u) {
            const int i = i0 + 32 * u;
            if (i < cnt) t[u] = __ldcg(&src[i]);
        }
#pragma unroll
        for (int u = 0; u < MR_U; ++u) {
            const int i = i0 + 32 * u;
            if (i < cnt) buf[i] = t[u];
        }
    }
}

// The x pass: one warp a row (z, y), blockDim.x / 32 rows a block, two buffers of M + 1 values a
// row in shared memory.
//   MR_ROW_CUBE  in: rows of T (y/z in row space) -> out: C rows = F_x(psi^3 - mean^3); E gets the
//                real parts of the kx = 0 and nx/2 bins (for the Hermitian projection)
//   MR_ROW_FWD   in: real rows -> out: scale F_x(psi - mean)
//   MR_ROW_INV   in: rows -> out: real rows, scale (row inverse + mean)
// The real transform of nx points is an M-point complex one (x[2i] + i x[2i + 1]) with the
// pre-/post-processing of pfc_pass.cuh on the pairs (k, M - k).
template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_mr_row(const __grid_constant__ MrGeom g, const __grid_constant__ MrArgs<R> a,
                                                const void *in, void *out, void *E) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;   // row index z ny + y
    if (r >= (int64_t)g.ny * g.nz) return;   // a whole warp; the kernel has no block barrier
    const int M = g.M, L = (M + 1);
    V *A = reinterpret_cast<V *>(smraw) + (size_t)warp * 2 * L;
    V *B = A + L;
    const R mean = a.mean ? (R)a.mean[0] : (R)0;
    const int npairs = M / 2 + 1;      // kk = 0 takes (0, M); kk = M/2 (M even) is self-paired
    if (MODE == MR_ROW_FWD) {
        mr_warp_load(A, reinterpret_cast<const V *>(in) + r * M, M, lane);
        __syncwarp();
        for (int i = lane; i < M; i += 32) {
            const V v = A[i];
            A[i] = V{v.x - mean, v.y - mean};
        }
    } else {
        // the row's M + 1 bins into B, then the real-transform pre-processing B -> A
        mr_warp_load(B, reinterpret_cast<const V *>(in) + r * g.xs, M + 1, lane);
        __syncwarp();
        if (MODE == MR_ROW_CUBE && lane < 2) {
            V *e = reinterpret_cast<V *>(E);
            e[2 * r + lane] = V{B[lane ? M : 0].x, (R)0};
        }
        for (int kk = lane; kk < npairs; kk += 32) {
            const bool k0 = kk == 0, self = 2 * kk == M;
            const int ca = kk, cb = k0 ? M : M - kk;
            const V xa = B[ca], xb = self ? xa : B[cb];
            V za, zb;
            c2r_pre_pair<V, R>(xa, xb, __ldg(&a.twx[ca]), k0, za, zb);
            A[ca] = za;
            if (!k0 && !self) A[cb] = zb;
        }
    }
    __syncwarp();
    V *X = A, *Y = B;
    if (MODE != MR_ROW_FWD) {
        X = mr_fft<+1>(A, B, g.ax[0], a.tw, lane);
        Y = X == A ? B : A;
    }
    if (MODE == MR_ROW_INV) {
        V *dst = reinterpret_cast<V *>(out) + r * M;
        for (int i = lane; i < M; i += 32) {
            const V v = X[i];
            __stcg(&dst[i], V{(v.x + mean) * a.scale, (v.y + mean) * a.scale});
        }
        return;
    }
    if (MODE == MR_ROW_CUBE) {
        // (v + mean)^3 - mean^3 with v = psi - mean
        const R c3 = (R)3 * mean * mean, b3 = (R)3 * mean;
        for (int i = lane; i < M; i += 32) {
            const V v = X[i];
            X[i] = V{v.x * (c3 + v.x * (b3 + v.x)), v.y * (c3 + v.y * (b3 + v.y))};
        }
        __syncwarp();
    }
    const V *Z = mr_fft<-1>(X, Y, g.ax[0], a.tw, lane);
    // real-transform post-processing (forward)
    V *dst = reinterpret_cast<V *>(out) + r * g.xs;
    const R sc = MODE == MR_ROW_FWD ? a.scale : (R)1;
    for (int kk = lane; kk < npairs; kk += 32) {
        const bool k0 = kk == 0, self = 2 * kk == M;
        const int ca = kk, cb = k0 ? M : M - kk;
        const V za = Z[ca], zb = (k0 || self) ? za : Z[cb];
        V xa, xb;
        r2c_post_pair<V, R>(za, zb, __ldg(&a.twx[ca]), k0, xa, xb);
        __stcg(&dst[ca], cscale(xa, sc));
        if (!self) __stcg(&dst[cb], cscale(xb, sc));
    }
}

// column stride of the column pass' buffers (odd, so that a row of W columns hits W banks)
__host__ __device__ __forceinline__ int mr_col_stride(int n) { return n | 1; }

enum { MR_COL_FWD = 0, MR_COL_INV = 1, MR_COL_UPDATE = 2 };

// A pass along axis (1 = y, 2 = z) on W = blockDim.x / (32 G) columns of the half spectrum, G
// warps a column (synced on the column's named barrier 1 + c when G > 1); grid = (column chunks,
// the other axis' extent). The block loads the W columns (rows of W adjacent values, W vb bytes
// apiece) into the first buffer of each column, the column groups transform, the block stores.
// MR_COL_FWD / MR_COL_INV: out = scale * transform(in) (in may equal out);
// MR_COL_UPDATE (the last forward axis): C = forward(in), then
// S <- (S - dt k^2 C inv_halfN) / (1 + dt k^2 Lk), S = 0 at k = 0 (out = S, read and written).
template <typename R, int MODE>
__global__ void __launch_bounds__(512) k_mr_col(const __grid_constant__ MrGeom g, const __grid_constant__ MrArgs<R> a,
                                                int axis, int ncols, const void *in, void *out, int G) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    const MrAxis &ax = g.ax[axis];
    const int n = ax.n, tid = threadIdx.x, nt = blockDim.x, W = (nt >> 5) / G, lW = __ffs(W) - 1;
    const int col = (tid >> 5) / G, th = tid - col * 32 * G;   // column of the thread, index in its group
    const int CS = mr_col_stride(n);
    V *A = reinterpret_cast<V *>(smraw);
    V *B = A + (size_t)W * CS;
    const int c0 = blockIdx.x * W, other = blockIdx.y;
    const int64_t step = axis == 1 ? (int64_t)g.xs : (int64_t)g.ny * g.xs;
    const int64_t base0 = (axis == 1 ? (int64_t)other * g.ny * g.xs : (int64_t)other * g.xs) + c0;
    const int wv = min(W, ncols - c0);   // valid columns of the chunk
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
    if (MODE == MR_COL_INV) res = mr_fft_g<+1>(A + col * CS, B + col * CS, ax, a.tw, th, 32 * G, 1 + col);
    else res = mr_fft_g<-1>(A + col * CS, B + col * CS, ax, a.tw, th, 32 * G, 1 + col);
    res -= col * CS;   // the same buffer for every column (the same number of stages)
    __syncthreads();
    V *dst = reinterpret_cast<V *>(out);
    for (int e0 = tid; e0 < total; e0 += nt * MR_U) {
        V sv[MR_U];
        if (MODE == MR_COL_UPDATE) {
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
            if (MODE != MR_COL_UPDATE) {
                __stcg(&dst[idx], cscale(c, a.scale));
                continue;
            }
            const int kx = c0 + w;
            const int iy = axis == 1 ? i : other, iz = axis == 1 ? other : i;
            const int my = iy <= g.ny / 2 ? iy : iy - g.ny, mz = iz <= g.nz / 2 ? iz : iz - g.nz;
            const R fx = a.up.cx * (R)kx, fy = a.up.cy * (R)my, fz = a.up.cz * (R)mz;
            const R k2 = fx * fx + fy * fy + fz * fz;
            const R inv = (R)1 / ((R)1 + a.up.dt * k2 * lin_symbol<R>(a.up.op[0], k2));
            const R cb = a.up.dt * k2 * inv * a.up.inv_halfN;
            __stcg(&dst[idx], (kx == 0 && iy == 0 && iz == 0) ? V{(R)0, (R)0}
                                                             : V{inv * sv[u].x - cb * c.x, inv * sv[u].y - cb * c.y});
        }
    }
}

// S's kx = 0 and nx/2 columns <- scale * E (E: two complex columns per (z, y), the projection)
template <typename R>
__global__ void k_mr_edges(const MrGeom g, const typename VT<R>::V *E, typename VT<R>::V *S, R scale) {
    const int64_t rows = (int64_t)g.ny * g.nz;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * rows; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e >> 1;
        const int c = (int)(e & 1);
        S[r * g.xs + (c ? g.M : 0)] = cscale(E[e], scale);
    }
}

// shared-memory bytes of the x pass (rows a block) and of a column pass (W columns of length n)
inline size_t mr_row_smem(int M, int rows, size_t vb) { return (size_t)rows * 2 * (M + 1) * vb; }
inline size_t mr_col_smem(int n, int W, size_t vb) { return (size_t)W * 2 * mr_col_stride(n) * vb; }

// Warps a column of a column pass of W columns: up to want (1, 2 or 4) while the block keeps at
// most 512 threads and every column has its own named barrier (W <= 15).
inline int mr_col_group(int W, int want) {
    int G = want == 4 ? 4 : want == 1 ? 1 : 2;
    while (G > 1 && (32 * W * G > 512 || W > 15)) G /= 2;
    return G;
}

}  // namespace pfc
