// Pass kernels of the fused semi-implicit PFC step (sm_103a).
//
// One step of Eq. (6) with the semi-implicit update of Listing 1,
//     psi_hat <- (psi_hat - dt k^2 FFT(psi^3)) / (1 + dt k^2 Lk(k)),
// runs as two passes over HBM (5 sweeps of a half spectrum):
//
//   row pass   reads X' (the carried state), undoes the P-part of the y/z transforms across
//              the rows it holds, transforms each row back to real space along x, forms
//              psi^3 in registers, transforms forward along x, applies the P-part forward and
//              writes C'.
//   line pass  reads the X' and C' tiles of one P-frequency, completes the y/z transforms
//              (the Q-part), applies the update with the multipliers computed from k^2 on the
//              fly, transforms the new state back (Q-part inverse) and writes X'.
//
// The y (and z) transform of length n = P Q is split Cooley-Tukey style:
//   y = y_q + Q y_p,  ky = k_p + P k_q,
//   Yhat[k_p + P k_q] = sum_{y_q} W_Q^{y_q k_q} [ W_n^{y_q k_p} sum_{y_p} x[y_q + Q y_p] W_P^{y_p k_p} ].
// The row pass owns the inner P-point sums of one y_q (its P rows are Q apart in y); the line
// pass owns the outer Q-point sums of one k_p. X' is stored as rows [k_p][y_q] (k_p = k_pz Py + k_py,
// y_q = z_q Qy + y_q) of xs complex values along kx, so a line-pass tile is contiguous.
//
// Scaling: X' = F_p(psi - mean) / (P M) with M = nx/2, so the row-pass inverse chain returns
// psi - mean exactly; the update multipliers fold the remaining 1/N.
#pragma once

#include "pfc_fft.cuh"

namespace pfc {

struct Geom {
    int nx, ny, nz, M;
    int lnx, lny, lnz, lM;
    int xs;                          // complex stride of X'/C' rows (multiple of W)
    int Py, Pz, Qy, Qz, lPy, lPz, lQy, lQz;
    int P, Q, lQ;
    int ltab;                        // twiddle table has 2^ltab entries
    int W, lW, ncg;                  // line pass: columns per tile, column groups
    int tpsh;                        // tile padding shift
    int rs;                          // row pass smem row stride (elements)
    int gpc;                         // row groups per row-pass CTA
    int64_t nreal;                   // real values per field (N)
    int64_t nhalf;                   // complex values per field of X'/C' (P Q xs)
    int64_t nstd;                    // complex values per field of the standard half spectrum
};

struct OpDev {
    int kind;
    double r, R1, q2;
};

enum { ROW_CUBE = 0, ROW_FWD = 1, ROW_INV = 2, ROW_ADJ_MIX = 3 };
enum { LINE_STEP = 0, LINE_FWD = 1, LINE_INV = 2, LINE_STEP2 = 3, LINE_ADJ = 4 };
enum { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2 };

template <typename R> struct RowArgs {
    const void *in;       // ROW_FWD: real; else X' layout
    void *out;            // ROW_INV: real; else X' layout
    const void *in2;      // ROW_ADJ_MIX: second X' input (V = B lam) ; real psi_n in in3
    const void *in3;
    void *proj;           // ROW_CUBE: X' to receive the projected kx = 0 and nx/2 columns
    const double *mean;   // per field, may be null
    R scale;
    const typename VT<R>::V *tw;
};

template <typename R> struct LineArgs {
    void *x;              // X' (in/out)
    const void *c;        // C'
    const void *std_in;   // LINE_INV input (standard half spectrum)
    void *std_out;        // LINE_FWD output (standard half spectrum)
    void *x2;             // second output (adjoint: B lam) or second field
    R scale;              // LINE_INV / LINE_FWD output scale
    double dt;
    double dx;
    OpDev op0, op1;
    double alpha;         // two-field coupling
    const typename VT<R>::V *tw;
    double *partials;     // adjoint: per-CTA dr partial sums
};

// ------------------------------------------------------------------------------------------
// P-part: small DFTs across the rows of one group, plus the split twiddles
// W_ny^{y_q k_py} W_nz^{z_q k_pz}. Rows of group gi live at smem rows gi P + (a Py + b).
// ------------------------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ V split_twiddle(const Geom &g, const V *__restrict__ tw, int grp,
                                           int kpz, int kpy) {
    const int zq = grp >> g.lQy, yq = grp & (g.Qy - 1);
    V t = __ldg(&tw[(yq * kpy) << (g.ltab - g.lny)]);
    if (g.Pz > 1) t = cmul(t, __ldg(&tw[(zq * kpz) << (g.ltab - g.lnz)]));
    return t;
}

// Inverse P-part in place: rows (k_pz, k_py) -> (z_p, y_p).
template <typename R>
__device__ void ppart_inverse(const Geom &g, typename VT<R>::V *sm, int grp0,
                              const typename VT<R>::V *__restrict__ tw) {
    using V = typename VT<R>::V;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int M1 = g.M + 1, P = g.P;
    // z first (with the twiddle), then y
    if (g.Pz > 1) {
        const int cnt = g.gpc * g.Py * M1;
        for (int e = tid; e < cnt; e += nt) {
            const int k = e % M1, rest = e / M1;
            const int kpy = rest % g.Py, gi = rest / g.Py;
            V t[8];
            for (int a = 0; a < g.Pz; ++a) {
                V x = sm[(gi * P + a * g.Py + kpy) * g.rs + row_pad(k)];
                t[a] = ctw<+1>(x, split_twiddle(g, tw, grp0 + gi, a, kpy));
            }
            dft_small<+1>(t, g.Pz);
            for (int a = 0; a < g.Pz; ++a) sm[(gi * P + a * g.Py + kpy) * g.rs + row_pad(k)] = t[a];
        }
        __syncthreads();
    }
    if (g.Py > 1) {
        const int cnt = g.gpc * g.Pz * M1;
        for (int e = tid; e < cnt; e += nt) {
            const int k = e % M1, rest = e / M1;
            const int zp = rest % g.Pz, gi = rest / g.Pz;
            V t[8];
            for (int b = 0; b < g.Py; ++b) {
                V x = sm[(gi * P + zp * g.Py + b) * g.rs + row_pad(k)];
                if (g.Pz == 1) x = ctw<+1>(x, split_twiddle(g, tw, grp0 + gi, 0, b));
                t[b] = x;
            }
            dft_small<+1>(t, g.Py);
            for (int b = 0; b < g.Py; ++b) sm[(gi * P + zp * g.Py + b) * g.rs + row_pad(k)] = t[b];
        }
        __syncthreads();
    }
}

// Forward P-part: rows (z_p, y_p) -> (k_pz, k_py), then scale and write X' rows
// (k_p Q + grp) of the output.
template <typename R>
__device__ void ppart_forward_store(const Geom &g, typename VT<R>::V *sm, int grp0,
                                    const typename VT<R>::V *__restrict__ tw,
                                    typename VT<R>::V *__restrict__ out, R scale) {
    using V = typename VT<R>::V;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int M1 = g.M + 1, P = g.P;
    if (P == 1) {
        const int cnt = g.gpc * M1;
        for (int e = tid; e < cnt; e += nt) {
            const int k = e % M1, gi = e / M1;
            out[(size_t)(grp0 + gi) * g.xs + k] = cscale(sm[gi * g.rs + row_pad(k)], scale);
        }
        return;
    }
    // y first
    {
        const int cnt = g.gpc * g.Pz * M1;
        for (int e = tid; e < cnt; e += nt) {
            const int k = e % M1, rest = e / M1;
            const int zp = rest % g.Pz, gi = rest / g.Pz;
            V t[8];
            for (int b = 0; b < g.Py; ++b) t[b] = sm[(gi * P + zp * g.Py + b) * g.rs + row_pad(k)];
            dft_small<-1>(t, g.Py);
            if (g.Pz == 1) {
                for (int b = 0; b < g.Py; ++b) {
                    V x = cmul(t[b], split_twiddle(g, tw, grp0 + gi, 0, b));
                    out[(size_t)(b * g.Q + grp0 + gi) * g.xs + k] = cscale(x, scale);
                }
            } else {
                for (int b = 0; b < g.Py; ++b) sm[(gi * P + zp * g.Py + b) * g.rs + row_pad(k)] = t[b];
            }
        }
    }
    if (g.Pz > 1) {
        __syncthreads();
        const int cnt = g.gpc * g.Py * M1;
        for (int e = tid; e < cnt; e += nt) {
            const int k = e % M1, rest = e / M1;
            const int kpy = rest % g.Py, gi = rest / g.Py;
            V t[8];
            for (int a = 0; a < g.Pz; ++a) t[a] = sm[(gi * P + a * g.Py + kpy) * g.rs + row_pad(k)];
            dft_small<-1>(t, g.Pz);
            for (int a = 0; a < g.Pz; ++a) {
                V x = cmul(t[a], split_twiddle(g, tw, grp0 + gi, a, kpy));
                out[(size_t)((a * g.Py + kpy) * g.Q + grp0 + gi) * g.xs + k] = cscale(x, scale);
            }
        }
    }
}

// Hermitian projection of the carried state. The kx = 0 and kx = nx/2 columns of X' are
// redundant: in row space (after the inverse P-part) they must be real, and the row inverse
// ignores their imaginary parts. Rounding leaves a small imaginary part there which psi^3
// never sees and which the update multiplies by 1/D(k) > 1 at the linearly unstable
// wavenumbers, so without projection it grows until it overflows. After the inverse P-part
// this writes the real parts of both columns back to X' through the forward P-part
// (X' = DFT_P(row values) / P), two values per row.
template <typename R>
__device__ void project_edge_columns(const Geom &g, const typename VT<R>::V *sm, int grp0,
                                     const typename VT<R>::V *__restrict__ tw,
                                     typename VT<R>::V *__restrict__ xout) {
    using V = typename VT<R>::V;
    const int P = g.P;
    const R invP = (R)1 / (R)P;
    for (int t = threadIdx.x; t < 2 * g.gpc; t += blockDim.x) {
        const int gi = t >> 1, k = (t & 1) ? g.M : 0, grp = grp0 + gi;
        V vals[64];
        for (int pr = 0; pr < P; ++pr) vals[pr] = V{sm[(gi * P + pr) * g.rs + row_pad(k)].x, (R)0};
        V tt[8];
        if (g.Py > 1) {
            for (int zp = 0; zp < g.Pz; ++zp) {
                for (int b = 0; b < g.Py; ++b) tt[b] = vals[zp * g.Py + b];
                dft_small<-1>(tt, g.Py);
                for (int b = 0; b < g.Py; ++b) vals[zp * g.Py + b] = tt[b];
            }
        }
        if (g.Pz > 1) {
            for (int kpy = 0; kpy < g.Py; ++kpy) {
                for (int a = 0; a < g.Pz; ++a) tt[a] = vals[a * g.Py + kpy];
                dft_small<-1>(tt, g.Pz);
                for (int a = 0; a < g.Pz; ++a) vals[a * g.Py + kpy] = tt[a];
            }
        }
        for (int kpz = 0; kpz < g.Pz; ++kpz)
            for (int kpy = 0; kpy < g.Py; ++kpy) {
                V x = vals[kpz * g.Py + kpy];
                if (P > 1) x = cmul(x, split_twiddle(g, tw, grp, kpz, kpy));
                xout[(size_t)((kpz * g.Py + kpy) * g.Q + grp) * g.xs + k] = cscale(x, invP);
            }
    }
}

// ------------------------------------------------------------------------------------------
// Real transform along x via a half-length complex transform (M = nx/2):
//   z[j] = x[2j] + i x[2j+1],  Z = DFT_M z,
//   X[k] = (Z[k] + conj Z[M-k])/2 - (i/2) W^k (Z[k] - conj Z[M-k]),  W = exp(-2 pi i / nx).
// The inverse builds E[k] = (X[k] + conj X[M-k])/2, O[k] = (X[k] - conj X[M-k])/2 conj(W^k),
// Z = E + i O (imaginary parts of X[0], X[M] ignored); IDFT_M Z = M (x_even + i x_odd).
// ------------------------------------------------------------------------------------------
template <typename R>
__device__ void c2r_pre_rows(const Geom &g, typename VT<R>::V *sm, int rows,
                             const typename VT<R>::V *__restrict__ tw) {
    using V = typename VT<R>::V;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int M = g.M, half = M / 2 + 1, sh = g.ltab - g.lnx;
    const int cnt = rows * half;
    for (int e = tid; e < cnt; e += nt) {
        const int k = e % half, r = e / half;
        V *row = sm + r * g.rs;
        if (k == 0) {
            const V x0 = row[row_pad(0)], xm = row[row_pad(M)];
            row[row_pad(0)] = V{(R)0.5 * (x0.x + xm.x), (R)0.5 * (x0.x - xm.x)};
        } else {
            const V xk = row[row_pad(k)], xm = row[row_pad(M - k)];
            const V w = __ldg(&tw[k << sh]);              // W^k
            // index k
            V e1 = cscale(cadd(xk, cconj(xm)), (R)0.5);
            V o1 = ctw<+1>(cscale(csub(xk, cconj(xm)), (R)0.5), w);
            // index M - k: conj(W^{M-k}) = -W^k
            V e2 = cscale(cadd(xm, cconj(xk)), (R)0.5);
            V o2 = cmul(cscale(csub(xm, cconj(xk)), (R)-0.5), w);
            row[row_pad(k)] = V{e1.x - o1.y, e1.y + o1.x};
            row[row_pad(M - k)] = V{e2.x - o2.y, e2.y + o2.x};
        }
    }
}

template <typename R>
__device__ void r2c_post_rows(const Geom &g, typename VT<R>::V *sm, int rows,
                              const typename VT<R>::V *__restrict__ tw) {
    using V = typename VT<R>::V;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int M = g.M, half = M / 2 + 1, sh = g.ltab - g.lnx;
    const int cnt = rows * half;
    for (int e = tid; e < cnt; e += nt) {
        const int k = e % half, r = e / half;
        V *row = sm + r * g.rs;
        if (k == 0) {
            const V z0 = row[row_pad(0)];
            row[row_pad(0)] = V{z0.x + z0.y, (R)0};
            row[row_pad(M)] = V{z0.x - z0.y, (R)0};
        } else {
            const V zk = row[row_pad(k)], zm = row[row_pad(M - k)];
            const V w = __ldg(&tw[k << sh]);              // W^k ; W^{M-k} = -conj(W^k)
            V a1 = cscale(cadd(zk, cconj(zm)), (R)0.5);
            V d1 = cmul(cscale(csub(zk, cconj(zm)), (R)0.5), w);
            V a2 = cscale(cadd(zm, cconj(zk)), (R)0.5);
            V d2 = cmul(cscale(csub(zm, cconj(zk)), (R)-0.5), cconj(w));
            // X = a - i d
            row[row_pad(k)] = V{a1.x + d1.y, a1.y - d1.x};
            row[row_pad(M - k)] = V{a2.x + d2.y, a2.y - d2.x};
        }
    }
}

// ------------------------------------------------------------------------------------------
// Row pass.
//   ROW_CUBE  X' -> C' = F_p(psi^3), psi = (row inverse of X') + mean.
//   ROW_FWD   real psi -> X' = scale F_p(psi - mean)
//   ROW_INV   X' -> real psi = (row inverse of X') + mean
// grid = (row groups / gpc, nfields); block = threads (multiple of M/8).
// ------------------------------------------------------------------------------------------
template <typename R, int MODE>
__global__ void __launch_bounds__(512) k_row(const Geom g, const RowArgs<R> a) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int field = blockIdx.y;
    const int P = g.P, rows = g.gpc * P, M = g.M, lM = g.lM;
    const int grp0 = blockIdx.x * g.gpc;
    const R mean = a.mean ? (R)a.mean[field] : (R)0;

    // ---- load ----
    if (MODE == ROW_FWD) {
        const V *in = reinterpret_cast<const V *>(a.in) + (size_t)field * (g.nreal / 2);
        const int cnt = rows << lM;
        for (int e = tid; e < cnt; e += nt) {
            const int i = e & (M - 1), r = e >> lM;
            const int gi = r / P, pr = r % P;
            const int grp = grp0 + gi;
            const int zq = grp >> g.lQy, yq = grp & (g.Qy - 1);
            const int zp = pr >> g.lPy, yp = pr & (g.Py - 1);
            const int z = zq + g.Qz * zp, y = yq + g.Qy * yp;
            V v = in[((size_t)z * g.ny + y) * M + i];
            v.x -= mean;
            v.y -= mean;
            sm[r * g.rs + row_pad(i)] = v;
        }
    } else {
        const V *in = reinterpret_cast<const V *>(a.in) + (size_t)field * g.nhalf;
        const int cnt = rows << lM;
        for (int e = tid; e < cnt; e += nt) {
            const int i = e & (M - 1), r = e >> lM;
            const int gi = r / P, kp = r % P;
            sm[r * g.rs + row_pad(i)] = in[(size_t)(kp * g.Q + grp0 + gi) * g.xs + i];
        }
        for (int r = tid; r < rows; r += nt) {
            const int gi = r / P, kp = r % P;
            sm[r * g.rs + row_pad(M)] = in[(size_t)(kp * g.Q + grp0 + gi) * g.xs + M];
        }
    }
    __syncthreads();

    if (MODE != ROW_FWD) {
        ppart_inverse<R>(g, sm, grp0, a.tw);
        if (MODE == ROW_CUBE) {
            V *xw = reinterpret_cast<V *>(a.proj) + (size_t)field * g.nhalf;
            project_edge_columns<R>(g, sm, grp0, a.tw, xw);
            __syncthreads();
        }
        c2r_pre_rows<R>(g, sm, rows, a.tw);
        __syncthreads();
    }

    // ---- per-row transforms ----
    const int Tr = M >> 3;
    const int RB = nt / Tr;
    for (int rb = 0; rb < rows; rb += RB) {
        const int r = rb + tid / Tr, j = tid % Tr;
        const bool act = r < rows;
        const RowAddr ad{r * g.rs};
        V v[8];
        if (MODE == ROW_CUBE) {
            fft_run<+1>(v, sm, ad, lM, j, act, false, true, a.tw, g.ltab);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const R p0 = v[m].x + mean, p1 = v[m].y + mean;
                v[m] = V{p0 * p0 * p0, p1 * p1 * p1};
            }
            fft_run<-1>(v, sm, ad, lM, j, act, true, false, a.tw, g.ltab);
        } else if (MODE == ROW_FWD) {
            fft_run<-1>(v, sm, ad, lM, j, act, false, false, a.tw, g.ltab);
        } else {
            fft_run<+1>(v, sm, ad, lM, j, act, false, true, a.tw, g.ltab);
            if (act) {
                const int gi = r / P, pr = r % P;
                const int grp = grp0 + gi;
                const int zq = grp >> g.lQy, yq = grp & (g.Qy - 1);
                const int zp = pr >> g.lPy, yp = pr & (g.Py - 1);
                const int z = zq + g.Qz * zp, y = yq + g.Qy * yp;
                V *out = reinterpret_cast<V *>(a.out) + (size_t)field * (g.nreal / 2) +
                         ((size_t)z * g.ny + y) * M;
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    out[j + m * Tr] = V{(v[m].x + mean) * a.scale, (v[m].y + mean) * a.scale};
            }
        }
    }

    if (MODE != ROW_INV) {
        r2c_post_rows<R>(g, sm, rows, a.tw);
        __syncthreads();
        V *out = reinterpret_cast<V *>(a.out) + (size_t)field * g.nhalf;
        ppart_forward_store<R>(g, sm, grp0, a.tw, out, a.scale);
    }
}

// ------------------------------------------------------------------------------------------
// Line pass: tiles of Q = Qz Qy complex values x W columns, interleaved (w fastest).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int tile_pad(int e, int sh) { return e + (e >> sh); }

// y-transforms (length Qy) of every (z_q, w) column, then z-transforms (length Qz).
// Thread t (of tot = Q W / 8) maps to (w fastest, then the butterfly index j, then the other
// column index); when tot exceeds the block, each thread takes NJ = tot / blockDim slots.
template <int S, int NJ, typename V>
__device__ void tile_fft_nj(const Geom &g, V *tile, const V *__restrict__ tw, bool y_first) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int tot = (g.Q * g.W) >> 3;
    for (int pass = 0; pass < 2; ++pass) {
        const bool doy = (pass == 0) == y_first;
        if (doy ? g.Qy == 1 : g.Qz == 1) continue;
        TileAddr ad[NJ];
        int j[NJ];
        bool act[NJ];
#pragma unroll
        for (int u = 0; u < NJ; ++u) {
            const int t = u * nt + tid;
            act[u] = t < tot;
            const int w = t & (g.W - 1);
            if (doy) {
                const int ly8 = g.lQy - 3;
                j[u] = (t >> g.lW) & ((1 << ly8) - 1);
                const int zq = t >> (g.lW + ly8);
                ad[u] = TileAddr{zq * g.Qy * g.W + w, g.W, g.tpsh};
            } else {
                const int yq = (t >> g.lW) & (g.Qy - 1);
                j[u] = t >> (g.lW + g.lQy);
                ad[u] = TileAddr{yq * g.W + w, g.Qy * g.W, g.tpsh};
            }
        }
        fft_run_multi<S, NJ>(tile, ad, doy ? g.lQy : g.lQz, j, act, tw, g.ltab);
    }
}

template <int S, typename V>
__device__ void tile_fft(const Geom &g, V *tile, const V *__restrict__ tw, bool y_first) {
    const int tot = (g.Q * g.W) >> 3;
    const int nt = blockDim.x;
    if (tot <= nt) tile_fft_nj<S, 1>(g, tile, tw, y_first);
    else if (tot <= 2 * nt) tile_fft_nj<S, 2>(g, tile, tw, y_first);
    else tile_fft_nj<S, 4>(g, tile, tw, y_first);
}

template <typename R>
__device__ __forceinline__ R lin_symbol(const OpDev &op, R k2) {
    const R a = (R)1 - k2;
    if (op.kind == 0) return (R)op.r + a * a;
    const R b = (R)(op.q2 * op.q2) - k2;
    return (R)op.r + a * a * ((R)op.R1 + b * b);
}

// k^2 of tile element e (after the forward Q-part) in column group cg and P-frequency kp.
template <typename R>
__device__ __forceinline__ R tile_k2(const Geom &g, double dx, int e, int cg, int kp, int *kx_o,
                                     int *ky_o, int *kz_o) {
    const int w = e & (g.W - 1), q = e >> g.lW;
    const int kqy = q & (g.Qy - 1), kqz = q >> g.lQy;
    const int kpy = kp % g.Py, kpz = kp / g.Py;
    const int kx = cg * g.W + w;
    const int ky = kpy + (kqy << g.lPy), kz = kpz + (kqz << g.lPz);
    const int my = ky <= g.ny / 2 ? ky : ky - g.ny;
    const int mz = kz <= g.nz / 2 ? kz : kz - g.nz;
    const R two_pi = (R)6.28318530717958647692528676655900576839;
    const R cx = two_pi / (R)(g.nx * dx), cy = two_pi / (R)(g.ny * dx), cz = two_pi / (R)(g.nz * dx);
    const R fx = cx * (R)kx, fy = cy * (R)my, fz = cz * (R)mz;
    *kx_o = kx;
    *ky_o = ky;
    *kz_o = kz;
    return fx * fx + fy * fy + fz * fz;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(512) k_line(const Geom g, const LineArgs<R> a) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int cg = blockIdx.x, kp = blockIdx.y, field = blockIdx.z;
    const int QW = g.Q * g.W;
    const int tsz = tile_pad(QW - 1, g.tpsh) + 1;
    V *T = sm;
    V *C = sm + tsz;
    const int kpy = kp % g.Py, kpz = kp / g.Py;

    auto gidx = [&](int e) -> size_t {       // X' element of tile element e
        const int w = e & (g.W - 1), q = e >> g.lW;
        return (size_t)(kp * g.Q + q) * g.xs + cg * g.W + w;
    };
    auto sidx = [&](int e, int *valid) -> size_t {   // standard half-spectrum element
        const int w = e & (g.W - 1), q = e >> g.lW;
        const int kqy = q & (g.Qy - 1), kqz = q >> g.lQy;
        const int kx = cg * g.W + w;
        const int ky = kpy + (kqy << g.lPy), kz = kpz + (kqz << g.lPz);
        *valid = kx <= g.M;
        return ((size_t)kz * g.ny + ky) * (g.M + 1) + kx;
    };

    if (MODE == LINE_STEP) {
        const V *X = reinterpret_cast<const V *>(a.x) + (size_t)field * g.nhalf;
        const V *Cc = reinterpret_cast<const V *>(a.c) + (size_t)field * g.nhalf;
        for (int e = tid; e < QW; e += nt) {
            const size_t gi = gidx(e);
            T[tile_pad(e, g.tpsh)] = X[gi];
            C[tile_pad(e, g.tpsh)] = Cc[gi];
        }
        __syncthreads();
        tile_fft<-1>(g, T, a.tw, true);
        tile_fft<-1>(g, C, a.tw, true);
        // update: T <- a' T - b' C, a' = 1/(Q D), b' = dt k^2 / ((N/2) D)
        const OpDev &op = field == 0 ? a.op0 : a.op1;
        const R invQ = (R)1 / (R)g.Q;
        const R inv_halfN = (R)(2.0 / ((double)g.nreal));
        const R dt = (R)a.dt;
        for (int e = tid; e < QW; e += nt) {
            int kx, ky, kz;
            const R k2 = tile_k2<R>(g, a.dx, e, cg, kp, &kx, &ky, &kz);
            const R lk = lin_symbol<R>(op, k2);
            const R inv = (R)1 / ((R)1 + dt * k2 * lk);
            const R ca = inv * invQ, cb = dt * k2 * inv * inv_halfN;
            const int s = tile_pad(e, g.tpsh);
            V t = T[s];
            const V c = C[s];
            t = V{ca * t.x - cb * c.x, ca * t.y - cb * c.y};
            if (kx == 0 && ky == 0 && kz == 0) t = V{(R)0, (R)0};
            T[s] = t;
        }
        __syncthreads();
        tile_fft<+1>(g, T, a.tw, false);
        V *Xo = reinterpret_cast<V *>(a.x) + (size_t)field * g.nhalf;
        for (int e = tid; e < QW; e += nt) Xo[gidx(e)] = T[tile_pad(e, g.tpsh)];
    } else if (MODE == LINE_FWD) {
        const V *X = reinterpret_cast<const V *>(a.x) + (size_t)field * g.nhalf;
        for (int e = tid; e < QW; e += nt) T[tile_pad(e, g.tpsh)] = X[gidx(e)];
        __syncthreads();
        tile_fft<-1>(g, T, a.tw, true);
        V *O = reinterpret_cast<V *>(a.std_out) + (size_t)field * g.nstd;
        for (int e = tid; e < QW; e += nt) {
            int valid;
            const size_t si = sidx(e, &valid);
            if (valid) O[si] = cscale(T[tile_pad(e, g.tpsh)], a.scale);
        }
    } else if (MODE == LINE_INV) {
        const V *I = reinterpret_cast<const V *>(a.std_in) + (size_t)field * g.nstd;
        for (int e = tid; e < QW; e += nt) {
            int valid;
            const size_t si = sidx(e, &valid);
            T[tile_pad(e, g.tpsh)] = valid ? I[si] : V{(R)0, (R)0};
        }
        __syncthreads();
        tile_fft<+1>(g, T, a.tw, false);
        V *Xo = reinterpret_cast<V *>(a.x) + (size_t)field * g.nhalf;
        for (int e = tid; e < QW; e += nt) Xo[gidx(e)] = cscale(T[tile_pad(e, g.tpsh)], a.scale);
    }
}

}  // namespace pfc
