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
//
// Three-pass form (grids whose row groups and line tiles cannot both fit shared memory): the
// y (and z) length is split in three, n = P R Q,
//   y = y_q + Q (y_r + R y_p),  ky = k_p + P (k_r + R k_q),
//   Yhat = sum_{y_q} W_Q^{y_q k_q} W_{RQ}^{y_q k_r} sum_{y_r} W_R^{y_r k_r}
//          [ W_n^{(y_q + Q y_r) k_p} sum_{y_p} x W_P^{y_p k_p} ].
// The row pass is the two-pass row pass with R Q groups (group (r, q) holds the rows
// y_q + Q y_r + Q R y_p); a middle pass (pfc_mid.cuh) owns the R-point sums and the twiddle
// W_{RQ}^{y_q k_r}; the line pass owns the Q-point sums of one (k_p, k_r). Rows of X' are
// [k_p][r][q] in both forms (r = y_r + Ry z_r before the middle pass, k_ry + Ry k_rz after it),
// so a line tile is still contiguous. With R = 1 everything reduces to the two-pass form.
#pragma once

#include "pfc_fft.cuh"

namespace pfc {

struct Geom {
    int nx, ny, nz, M;
    int lnx, lny, lnz, lM;
    int xs;                          // complex stride of X'/C' rows (multiple of W)
    int Py, Pz, Qy, Qz, lPy, lPz, lQy, lQz;
    int P, Q, lQ;
    int Ry, Rz, R, lRy, lRz, lR;     // middle-pass split (1 in the two-pass form)
    int QR;                          // row groups = R Q
    int ltab;                        // full twiddle table has 2^ltab entries
    int W, lW, ncg;                  // line pass: columns per tile, column groups
    int tsz;                         // line pass tile size in elements, (Q + Q/8) W (see tile_y)
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
enum { LINE_STEP = 0, LINE_FWD = 1, LINE_INV = 2, LINE_SCHEME = 3 };
enum { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2 };

template <typename R> struct RowArgs {
    const void *in;       // ROW_FWD: real; else X' layout
    void *out;            // ROW_INV: real; else X' layout
    void *proj;           // ROW_CUBE: X' to receive the projected kx = 0 and nx/2 columns
    const void *aux;      // ROW_ADJ_MIX: real psi_n
    const void *aux2;     // k_row_adj2: V' and Psi' (X' layout)
    const void *aux3;
    const int64_t *moff;  // batched members: element offset of member m in the real arrays
    const double *mean;   // per field, may be null
    R scale;
    const typename VT<R>::V *tw;
    StageTw<typename VT<R>::V> st;
};

// Operator and update constants in the path's precision, prepared on the host so that an
// FP32 kernel executes no FP64 instruction (GB300's FP64 rate is a small fraction of FP32).
template <typename R> struct OpR {
    int kind;
    R r, R1, q2sq;        // q2sq = q2^2
};
template <typename R> struct UpdR {
    R dt;
    R cx, cy, cz;         // 2 pi / (n dx) per axis
    R invQ, inv_halfN;    // 1/Q and 2/N
    OpR<R> op[2];         // per field
    // LINE_SCHEME: psi_hat' = (1 + dt k^2 S) inv X - d1 dt k^2 inv C, inv = 1 / (d0 + d1 dt k^2 (Lk + S)),
    // X and C the combinations xw0 X + xw1 Xprev and cw0 C + cw1 Cprev (Xprev, Cprev may be null)
    R d0, d1, S;
    R xw0, xw1, cw0, cw1;
};

template <typename R> struct LineArgs {
    void *x;              // X' (in/out; LINE_SCHEME: in)
    const void *c;        // C'
    const void *xprev;    // LINE_SCHEME: the previous level's X' and C' (null: not used)
    const void *cprev;
    void *xout;           // LINE_STEP, LINE_SCHEME: output X' (null: x, in place; may equal xprev)
    const void *std_in;   // LINE_INV input (standard half spectrum)
    void *std_out;        // LINE_FWD output (standard half spectrum)
    R scale;              // LINE_INV / LINE_FWD output scale
    UpdR<R> up;
    const R *rmem;        // batched members: r of member m (overrides up.op[0].r), may be null
    StageTw<typename VT<R>::V> st;
};

// ------------------------------------------------------------------------------------------
// Helpers
// ------------------------------------------------------------------------------------------
// Row group grp = r Q + q (q = z_q Qy + y_q, r = y_r + Ry z_r) -> the y and z offsets of its
// rows, yo = y_q + Qy y_r and zo = z_q + Qz z_r; its rows are y = yo + Qy Ry y_p,
// z = zo + Qz Rz z_p.
__device__ __forceinline__ void grp_yz(const Geom &g, int grp, int &zo, int &yo) {
    const int q = grp & (g.Q - 1), r = grp >> g.lQ;
    yo = (q & (g.Qy - 1)) + g.Qy * (r & (g.Ry - 1));
    zo = (q >> g.lQy) + g.Qz * (r >> g.lRy);
}

// Row of row group grp for (z_p, y_p) in the caller's real array (z, y).
__device__ __forceinline__ void grp_row(const Geom &g, int grp, int zp, int yp, int &z, int &y) {
    int zo, yo;
    grp_yz(g, grp, zo, yo);
    z = zo + g.Qz * g.Rz * zp;
    y = yo + g.Qy * g.Ry * yp;
}

// Line tile kp = k_p R + k_r -> the low parts of its wavenumber indices, ky = kpy + Py Ry k_qy,
// kz = kpz + Pz Rz k_qz.
__device__ __forceinline__ void line_kp(const Geom &g, int kp, int &kpy, int &kpz) {
    const int p = kp >> g.lR, r = kp & (g.R - 1);
    kpy = (p & (g.Py - 1)) + g.Py * (r & (g.Ry - 1));
    kpz = (p >> g.lPy) + g.Pz * (r >> g.lRy);
}

// Split twiddle W_ny^{yo k_py} W_nz^{zo k_pz} of row group grp (forward sign).
template <typename V>
__device__ __forceinline__ V split_twiddle(const Geom &g, const V *__restrict__ tw, int grp,
                                           int kpz, int kpy) {
    int zo, yo;
    grp_yz(g, grp, zo, yo);
    V t = __ldg(&tw[(yo * kpy) << (g.ltab - g.lny)]);
    if (g.Pz > 1) t = cmul(t, __ldg(&tw[(zo * kpz) << (g.ltab - g.lnz)]));
    return t;
}

// Real-transform pre-processing (inverse direction) of one row pair (a = X[k], b = X[M-k]):
// E = (X[k] + conj X[M-k]) / 2, O = (X[k] - conj X[M-k]) / 2 conj(W^k), Z = E + i O; at k = 0 the
// imaginary parts of X[0] and X[M] are ignored. w = W^k = exp(-2 pi i k / nx).
template <typename V, typename R>
__device__ __forceinline__ void c2r_pre_pair(V a, V b, V w, bool k0, V &za, V &zb) {
    if (k0) {
        za = V{(R)0.5 * (a.x + b.x), (R)0.5 * (a.x - b.x)};
        zb = za;
        return;
    }
    const V e1 = cscale(cadd(a, cconj(b)), (R)0.5);
    const V o1 = ctw<+1>(cscale(csub(a, cconj(b)), (R)0.5), w);
    const V e2 = cscale(cadd(b, cconj(a)), (R)0.5);
    const V o2 = cmul(cscale(csub(b, cconj(a)), (R)-0.5), w);   // conj(W^{M-k}) = -W^k
    za = V{e1.x - o1.y, e1.y + o1.x};
    zb = V{e2.x - o2.y, e2.y + o2.x};
}

// Real-transform post-processing (forward direction): from Z[k], Z[M-k] to X[k], X[M-k],
// X[k] = (Z[k] + conj Z[M-k])/2 - (i/2) W^k (Z[k] - conj Z[M-k]); at k = 0, X[0] and X[M].
template <typename V, typename R>
__device__ __forceinline__ void r2c_post_pair(V za, V zb, V w, bool k0, V &xa, V &xb) {
    if (k0) {
        xa = V{za.x + za.y, (R)0};
        xb = V{za.x - za.y, (R)0};
        return;
    }
    const V a1 = cscale(cadd(za, cconj(zb)), (R)0.5);
    const V d1 = cmul(cscale(csub(za, cconj(zb)), (R)0.5), w);
    const V a2 = cscale(cadd(zb, cconj(za)), (R)0.5);
    const V d2 = cmul(cscale(csub(zb, cconj(za)), (R)-0.5), cconj(w));   // W^{M-k} = -conj(W^k)
    xa = V{a1.x + d1.y, a1.y - d1.x};
    xb = V{a2.x + d2.y, a2.y - d2.x};
}

// Decompose a flat index over (gi, s, kk), kk in [0, M/2), s in [0, S) (S a power of two). The
// item kk = 0 covers the column pair (0, M) and also the self-paired column M/2, so that
// gpc*S*(M/2) items cover all M + 1 columns with no second round.
__device__ __forceinline__ void pair_index(const Geom &g, int e, int lS, int &kk, int &s, int &gi) {
    const int lh = g.lM - 1;
    kk = e & ((1 << lh) - 1);
    const int rest = e >> lh;
    s = rest & ((1 << lS) - 1);
    gi = rest >> lS;
}

// ------------------------------------------------------------------------------------------
// Row pass phases
// ------------------------------------------------------------------------------------------
// Phase A (Pz > 1): z-part inverse from X' in global memory into smem rows, with the full split
// twiddle; rows (k_pz, k_py) become (z_p, k_py).
template <typename R>
__device__ void row_phase_a(const Geom &g, typename VT<R>::V *sm, const typename VT<R>::V *X,
                            int grp0, const typename VT<R>::V *stw) {
    using V = typename VT<R>::V;
    const int P = g.P, M = g.M, lM = g.lM;
    const int main = (g.gpc * g.Py) << lM;
    const int cnt = main + g.gpc * g.Py;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int k, rest;
        if (e < main) { k = e & (M - 1); rest = e >> lM; }
        else { k = M; rest = e - main; }
        const int kpy = rest % g.Py, gi = rest / g.Py, grp = grp0 + gi;
        V t[8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
            if (a < g.Pz)
                t[a] = ctw<+1>(X[(size_t)((a * g.Py + kpy) * g.QR + grp) * g.xs + k],
                               stw[gi * P + a * g.Py + kpy]);
        dft_small<+1>(t, g.Pz);
#pragma unroll
        for (int a = 0; a < 8; ++a)
            if (a < g.Pz) sm[(gi * P + a * g.Py + kpy) * g.rs + row_swz(k)] = t[a];
    }
}

// Phase B: y-part inverse of the column pair (kk, M - kk) of the Py rows of (gi, z_p), then the
// real-transform pre-processing; rows end physical (z_p, y_p). FROM_GLOBAL (Pz == 1) reads X'
// and applies the y twiddle; otherwise reads smem left by phase A. When edge is set, the real
// parts of the kx = 0 and kx = M columns are saved there for the projection.
// PY > 0: the plan's Py fixed at compile time (the unused register slots drop out).
template <typename R, bool FROM_GLOBAL, int PY = 0>
__device__ __forceinline__ void row_pair_b(const Geom &g, typename VT<R>::V *sm, R *edge,
                                           const typename VT<R>::V *X, int gi, int grp, int zp,
                                           int ca, int cb, bool k0,
                                           const typename VT<R>::V *__restrict__ tw,
                                           const typename VT<R>::V *stw, typename VT<R>::V *proj) {
    using V = typename VT<R>::V;
    const int P = PY > 0 ? PY : g.P;   // (PY > 0 only with Pz == 1)
    const int Py = PY > 0 ? PY : g.Py;
    V a[8], b[8];
#pragma unroll
    for (int yy = 0; yy < 8; ++yy) {
        if (yy < Py) {
            if (FROM_GLOBAL) {
                const V *src = X + (size_t)(yy * g.QR + grp) * g.xs;
                const V w = stw[gi * P + yy];
                a[yy] = ctw<+1>(__ldcg(&src[ca]), w);
                b[yy] = ctw<+1>(__ldcg(&src[cb]), w);
            } else {
                const int row = gi * P + zp * Py + yy;
                a[yy] = sm[row * g.rs + row_swz(ca)];
                b[yy] = sm[row * g.rs + row_swz(cb)];
            }
        }
    }
    dft_small<+1>(a, Py);
    dft_small<+1>(b, Py);
    const V w = __ldg(&tw[ca << (g.ltab - g.lnx)]);
#pragma unroll
    for (int yy = 0; yy < 8; ++yy) {
        if (yy < Py) {
            const int row = gi * P + zp * Py + yy;
            if (edge && k0) {
                edge[(gi * 2) * P + zp * Py + yy] = a[yy].x;
                edge[(gi * 2 + 1) * P + zp * Py + yy] = b[yy].x;
            }
            V za, zb;
            c2r_pre_pair<V, R>(a[yy], b[yy], w, k0, za, zb);
            sm[row * g.rs + row_swz(ca)] = za;
            if (!k0 && cb != ca) sm[row * g.rs + row_swz(cb)] = zb;
        }
    }
    if (FROM_GLOBAL && proj && k0) {
        // Hermitian projection (see project_edge_columns_par) done here when the thread holds every
        // row of the kx = 0 and kx = M columns (Pz == 1): X' = DFT_P(real parts) / P. a and b are
        // reused: the pre-processing above no longer needs them.
#pragma unroll
        for (int yy = 0; yy < 8; ++yy) {
            a[yy].y = (R)0;
            b[yy].y = (R)0;
        }
        dft_small<-1>(a, Py);
        dft_small<-1>(b, Py);
        const R invP = (R)1 / (R)P;
#pragma unroll
        for (int yy = 0; yy < 8; ++yy) {
            if (yy < Py) {
                V *dst = proj + (size_t)(yy * g.QR + grp) * g.xs;
                dst[0] = cscale(cmul(a[yy], stw[gi * P + yy]), invP);
                dst[g.M] = cscale(cmul(b[yy], stw[gi * P + yy]), invP);
            }
        }
    }
}

// Phase B: y-part inverse of the column pair (kk, M - kk) of the Py rows of (gi, z_p), then the
// real-transform pre-processing; rows end physical (z_p, y_p). FROM_GLOBAL (Pz == 1) reads X'
// and applies the y twiddle; otherwise reads smem left by phase A. When edge is set, the real
// parts of the kx = 0 and kx = M columns are saved there for the projection.
template <typename R, bool FROM_GLOBAL, int PY = 0>
__device__ void row_phase_b(const Geom &g, typename VT<R>::V *sm, R *edge,
                            const typename VT<R>::V *X, int grp0,
                            const typename VT<R>::V *__restrict__ tw,
                            const typename VT<R>::V *stw, typename VT<R>::V *proj) {
    const int M = g.M, hM = M >> 1;
    const int cnt = (g.gpc * g.Pz) << (g.lM - 1);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int kk, zp, gi;
        pair_index(g, e, g.lPz, kk, zp, gi);
        const int grp = grp0 + gi;
        // kk = 0 handles the pair (0, M) and then the self-paired column M/2 (one body, so the
        // code is not duplicated)
        const int npass = kk == 0 ? 2 : 1;
#pragma unroll 1
        for (int pp = 0; pp < npass; ++pp) {
            const bool k0 = kk == 0 && pp == 0;
            const int ca = pp ? hM : kk, cb = pp ? hM : (kk == 0 ? M : M - kk);
            row_pair_b<R, FROM_GLOBAL, PY>(g, sm, k0 ? edge : nullptr, X, gi, grp, zp, ca, cb, k0, tw, stw, proj);
        }
    }
}

// Hermitian projection of the carried state. The kx = 0 and kx = nx/2 columns of X' are
// redundant: in row space (after the inverse P-part) they must be real, and the row inverse
// ignores their imaginary parts. Rounding leaves a small imaginary part there which psi^3
// never sees and which the update multiplies by 1/D(k) > 1 at the linearly unstable
// wavenumbers, so without projection it grows until it overflows. This writes the saved real
// parts of both columns back to X' through the forward P-part (X' = DFT_P(row values) / P).
// Spread over threads: the y-part of every (group, column, z_p), then the z-part, twiddle and
// store of every (group, column, k_py), through S (2 gpc P complex values of shared memory).
// Called by every thread of the block (it contains a barrier).
template <typename R>
__device__ void project_edge_columns_par(const Geom &g, const R *edge, int grp0,
                                         const typename VT<R>::V *stw, typename VT<R>::V *__restrict__ xout,
                                         typename VT<R>::V *S) {
    using V = typename VT<R>::V;
    const int P = g.P, Py = g.Py, Pz = g.Pz;
    const R invP = (R)1 / (R)P;
    for (int t = threadIdx.x; t < 2 * g.gpc * Pz; t += blockDim.x) {
        const int gc = t / Pz, zp = t % Pz;   // gc = 2 gi + c
        V tt[8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (b < Py) tt[b] = V{edge[gc * P + zp * Py + b], (R)0};
        dft_small<-1>(tt, Py);
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (b < Py) S[gc * P + zp * Py + b] = tt[b];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * g.gpc * Py; t += blockDim.x) {
        const int gc = t / Py, kpy = t % Py, gi = gc >> 1, k = (gc & 1) ? g.M : 0, grp = grp0 + gi;
        V tt[8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
            if (a < Pz) tt[a] = S[gc * P + a * Py + kpy];
        dft_small<-1>(tt, Pz);
#pragma unroll
        for (int kpz = 0; kpz < 8; ++kpz) {
            if (kpz < Pz) {
                V x = tt[kpz];
                if (P > 1) x = cmul(x, stw[gi * P + kpz * Py + kpy]);
                xout[(size_t)((kpz * Py + kpy) * g.QR + grp) * g.xs + k] = cscale(x, invP);
            }
        }
    }
}

template <typename R, int PY = 0>
__device__ __forceinline__ void row_pair_d(const Geom &g, typename VT<R>::V *sm,
                                           typename VT<R>::V *out, int gi, int grp, int zp,
                                           int ca, int cb, bool k0,
                                           const typename VT<R>::V *__restrict__ tw,
                                           const typename VT<R>::V *stw, R scale) {
    using V = typename VT<R>::V;
    const int P = PY > 0 ? PY : g.P;   // (PY > 0 only with Pz == 1)
    const int Py = PY > 0 ? PY : g.Py;
    const V w = __ldg(&tw[ca << (g.ltab - g.lnx)]);
    V a[8], b[8];
#pragma unroll
    for (int yy = 0; yy < 8; ++yy) {
        if (yy < Py) {
            const int row = gi * P + zp * Py + yy;
            const V za = sm[row * g.rs + row_swz(ca)];
            const V zb = (k0 || cb == ca) ? za : sm[row * g.rs + row_swz(cb)];
            r2c_post_pair<V, R>(za, zb, w, k0, a[yy], b[yy]);
        }
    }
    dft_small<-1>(a, Py);
    dft_small<-1>(b, Py);
#pragma unroll
    for (int yy = 0; yy < 8; ++yy) {
        if (yy < Py) {
            if (g.Pz == 1) {
                const V t = stw[gi * P + yy];
                V *dst = out + (size_t)(yy * g.QR + grp) * g.xs;
                __stcg(&dst[ca], cscale(cmul(a[yy], t), scale));
                if (cb != ca) __stcg(&dst[cb], cscale(cmul(b[yy], t), scale));
            } else {
                const int row = gi * P + zp * Py + yy;
                sm[row * g.rs + row_swz(ca)] = a[yy];
                if (cb != ca) sm[row * g.rs + row_swz(cb)] = b[yy];
            }
        }
    }
}

// Phase D: real-transform post-processing of the pair (kk, M - kk) of the Py rows of (gi, z_p),
// then the y-part forward. With Pz == 1 it applies the y twiddle and the scale and writes X'
// rows (k_py Q + grp) of out; otherwise it writes smem rows (z_p, k_py) for phase E.
template <typename R, int PY = 0>
__device__ void row_phase_d(const Geom &g, typename VT<R>::V *sm, typename VT<R>::V *out,
                            int grp0, const typename VT<R>::V *__restrict__ tw,
                            const typename VT<R>::V *stw, R scale) {
    const int M = g.M, hM = M >> 1;
    const int cnt = (g.gpc * g.Pz) << (g.lM - 1);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int kk, zp, gi;
        pair_index(g, e, g.lPz, kk, zp, gi);
        const int grp = grp0 + gi;
        const int npass = kk == 0 ? 2 : 1;
#pragma unroll 1
        for (int pp = 0; pp < npass; ++pp) {
            const bool k0 = kk == 0 && pp == 0;
            const int ca = pp ? hM : kk, cb = pp ? hM : (kk == 0 ? M : M - kk);
            row_pair_d<R, PY>(g, sm, out, gi, grp, zp, ca, cb, k0, tw, stw, scale);
        }
    }
}

// Phase E (Pz > 1): z-part forward of each column, twiddle, scale, write X' rows.
template <typename R>
__device__ void row_phase_e(const Geom &g, const typename VT<R>::V *sm, typename VT<R>::V *out,
                            int grp0, const typename VT<R>::V *stw, R scale) {
    using V = typename VT<R>::V;
    const int P = g.P, M = g.M, lM = g.lM;
    const int main = (g.gpc * g.Py) << lM;
    const int cnt = main + g.gpc * g.Py;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int k, rest;
        if (e < main) { k = e & (M - 1); rest = e >> lM; }
        else { k = M; rest = e - main; }
        const int kpy = rest % g.Py, gi = rest / g.Py, grp = grp0 + gi;
        V t[8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
            if (a < g.Pz) t[a] = sm[(gi * P + a * g.Py + kpy) * g.rs + row_swz(k)];
        dft_small<-1>(t, g.Pz);
#pragma unroll
        for (int a = 0; a < 8; ++a)
            if (a < g.Pz)
                out[(size_t)((a * g.Py + kpy) * g.QR + grp) * g.xs + k] =
                    cscale(cmul(t[a], stw[gi * P + a * g.Py + kpy]), scale);
    }
}

// psi^3 - mean^3 of the 16 real values held in v (both halves of each complex slot), psi = v +
// mean, as v (3 mean^2 + v (3 mean + v)). The constant mean^3 would only change the k = 0 bin of
// C', which the update multiplies by k^2 = 0; leaving it out keeps the rounding of C' relative to
// the fluctuation's part of psi^3 instead of to mean^3 (in FP32, ten times smaller for a 0.01
// fluctuation about a mean of -0.3).
template <typename V, typename R>
__device__ __forceinline__ void cube_shifted(V (&v)[8], R mean) {
    const R a = (R)3 * mean * mean, b = (R)3 * mean;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const R p0 = v[m].x, p1 = v[m].y;
        v[m] = V{p0 * (a + p0 * (b + p0)), p1 * (a + p1 * (b + p1))};
    }
}

// ------------------------------------------------------------------------------------------
// Row pass.
//   ROW_CUBE  X' -> C' = F_p(psi^3), psi = (row inverse of X') + mean; X' edge columns projected
//   ROW_FWD   real psi -> X' = scale F_p(psi - mean)
//   ROW_INV   X' -> real psi = scale ((row inverse of X') + mean)
// grid = (row groups / gpc, nfields); block = threads (a multiple of M/8).
// ------------------------------------------------------------------------------------------
// row transform of a row pass: length 2^LM fixed at compile time when LM > 0 (a kernel with one
// transform length is a fraction of the size of the all-lengths one: small rows are bound by
// instruction fetch otherwise), else the plan's length
template <int S, int LM, typename V, typename Bar>
__device__ __forceinline__ void row_fft(V (&v)[8], V *sm, const RowAddr &ad, int lM, int j, bool act,
                                        bool in_regs, bool out_regs, const StageTw<typename ElemOf<V>::Tw> &tw, const Bar &bar) {
    if constexpr (LM > 0) fft_run_t<S, LM>(v, sm, ad, j, act, in_regs, out_regs, tw, bar);
    else fft_run<S>(v, sm, ad, lM, j, act, in_regs, out_regs, tw, bar);
}

// LM > 0: the kernel only serves plans with M = 2^LM.
// The body of one row-pass block (block index bx, field or batch member `field`); k_row runs it
// as its own block, the persistent batch kernel once per work item.
// PY > 0: only for plans with Pz == 1 and Py == PY.
template <typename R, int MODE, int LM = 0, int PY = 0>
__device__ __forceinline__ void row_body(const Geom &g, const RowArgs<R> &a, int bx, int field) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int P = g.P, rows = g.gpc * P, M = g.M, lM = g.lM;
    const int grp0 = bx * g.gpc;
    const R mean = a.mean ? (R)a.mean[field] : (R)0;
    // smem: rows | split twiddles of this block's groups (gpc P) | saved edge values (2 gpc P)
    V *stw = sm + rows * g.rs;
    R *edge = reinterpret_cast<R *>(stw + rows);
    for (int t = tid; t < rows; t += nt) {
        const int gi = t / P, kp = t % P;
        stw[t] = split_twiddle(g, a.tw, grp0 + gi, kp / g.Py, kp % g.Py);
    }

    if (MODE == ROW_FWD) {
        const V *in = reinterpret_cast<const V *>(a.in) +
                      (a.moff ? (size_t)(a.moff[field] / 2) : (size_t)field * (g.nreal / 2));
        const int cnt = rows << lM;
        for (int e = tid; e < cnt; e += nt) {
            const int i = e & (M - 1), r = e >> lM;
            const int gi = r / P, pr = r % P;
            const int grp = grp0 + gi;
            int z, y;
            grp_row(g, grp, pr >> g.lPy, pr & (g.Py - 1), z, y);
            V v = in[((size_t)z * g.ny + y) * M + i];
            v.x -= mean;
            v.y -= mean;
            sm[r * g.rs + row_swz(i)] = v;
        }
    } else {
        const V *X = reinterpret_cast<const V *>(a.in) + (size_t)field * g.nhalf;
        R *ed = MODE == ROW_CUBE ? edge : nullptr;
        __syncthreads();
        V *pw = MODE == ROW_CUBE ? reinterpret_cast<V *>(a.proj) + (size_t)field * g.nhalf : nullptr;
        if (g.Pz > 1) {
            row_phase_a<R>(g, sm, X, grp0, stw);
            __syncthreads();
            row_phase_b<R, false>(g, sm, ed, X, grp0, a.tw, stw, nullptr);
        } else {
            row_phase_b<R, true, PY>(g, sm, nullptr, X, grp0, a.tw, stw, pw);
        }
    }
    __syncthreads();

    // ---- per-row transforms ----
    const int Tr = M >> 3;
    const int RB = nt / Tr;
    // groups of Tr threads take rows gidx, gidx + RB, ...; a group syncs on its own warp (Tr <=
    // 32), on its own named barrier, or (more groups than barriers, or ragged rounds) on the block
    const bool grouped = Tr >= 32 && RB <= 15 && rows % RB == 0;
    const int gidx = tid / Tr;
    const RowBarrier nbar = Tr <= 32 ? RowBarrier{0, Tr} : grouped ? RowBarrier{1 + gidx, Tr} : RowBarrier{0, nt};
    for (int rb = 0; rb < rows; rb += RB) {
        const int r = rb + gidx, j = tid % Tr;
        const bool act = r < rows;
        const RowAddr ad{r * g.rs};
        V v[8];
        if (MODE == ROW_CUBE) {
            row_fft<+1, LM>(v, sm, ad, lM, j, act, false, true, a.st, nbar);
            cube_shifted(v, mean);
            row_fft<-1, LM>(v, sm, ad, lM, j, act, true, false, a.st, nbar);
        } else if (MODE == ROW_FWD) {
            row_fft<-1, LM>(v, sm, ad, lM, j, act, false, false, a.st, nbar);
        } else {   // ROW_INV, ROW_ADJ_MIX
            row_fft<+1, LM>(v, sm, ad, lM, j, act, false, true, a.st, nbar);
            if (act) {
                const int gi = r / P, pr = r % P;
                const int grp = grp0 + gi;
                int z, y;
                grp_row(g, grp, pr >> g.lPy, pr & (g.Py - 1), z, y);
                V *out = reinterpret_cast<V *>(a.out) +
                         (a.moff ? (size_t)(a.moff[field] / 2) : (size_t)field * (g.nreal / 2)) +
                         ((size_t)z * g.ny + y) * M;
                if (MODE == ROW_INV) {
#pragma unroll
                    for (int m = 0; m < 8; ++m)
                        out[j + m * Tr] = V{(v[m].x + mean) * a.scale, (v[m].y + mean) * a.scale};
                } else {
                    // adjoint: out <- out - 3 psi_n^2 (this row inverse)
                    const V *ps = reinterpret_cast<const V *>(a.aux) + (size_t)field * (g.nreal / 2) +
                                  ((size_t)z * g.ny + y) * M;
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const V u = out[j + m * Tr], p = ps[j + m * Tr];
                        out[j + m * Tr] = V{u.x - (R)3 * p.x * p.x * (v[m].x * a.scale),
                                            u.y - (R)3 * p.y * p.y * (v[m].y * a.scale)};
                    }
                }
            }
        }
    }

    __syncthreads();
    if (MODE == ROW_CUBE || MODE == ROW_FWD) {
        V *out = reinterpret_cast<V *>(a.out) + (size_t)field * g.nhalf;
        row_phase_d<R, PY>(g, sm, out, grp0, a.tw, stw, a.scale);
        if (g.Pz > 1) {
            __syncthreads();
            row_phase_e<R>(g, sm, out, grp0, stw, a.scale);
        }
    }
    // the edge values were saved in phase B in their own smem area; nothing waits on this
    if (MODE == ROW_CUBE && g.Pz > 1) {   // (Pz == 1 projects in phase B)
        V *xw = reinterpret_cast<V *>(a.proj) + (size_t)field * g.nhalf;
        __syncthreads();   // phase E has read the rows; they serve as the projection's scratch
        project_edge_columns_par<R>(g, edge, grp0, stw, xw, sm);
    }
}

template <typename R, int MODE, int LM = 0, int PY = 0>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? 2 : 1) k_row(const Geom g, const RowArgs<R> a) {
    row_body<R, MODE, LM, PY>(g, a, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------------------------------
// Line pass: one tile of Q = Qz Qy complex values x W columns per block, interleaved (w
// fastest, one padding row after every 8 tile rows), block = Q W / 8 threads. y-transforms use
// the thread map (w, j, z_q), z-transforms (w, y_q, j). The first forward stage reads global memory into registers, the last forward
// stage, the update and the first inverse stage stay in registers, and the last inverse stage
// writes global memory from registers.
// ------------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R lin_symbol(const OpR<R> &op, R k2) {
    const R a = (R)1 - k2;
    if (op.kind == 0) return op.r + a * a;
    const R b = op.q2sq - k2;
    return op.r + a * a * (op.R1 + b * b);
}

struct LineMap {
    int w, jy, zq;   // y map
    int yq, jz;      // z map
    int ny8, nz8;
};

__device__ __forceinline__ LineMap line_map(const Geom &g, int t) {
    LineMap m;
    m.w = t & (g.W - 1);
    const int ly8 = g.lQy - 3;
    m.jy = (t >> g.lW) & ((1 << ly8) - 1);
    m.zq = t >> (g.lW + ly8);
    m.yq = (t >> g.lW) & (g.Qy - 1);
    m.jz = g.Qz > 1 ? (t >> (g.lW + g.lQy)) : 0;
    m.ny8 = g.Qy >> 3;
    m.nz8 = g.Qz > 1 ? (g.Qz >> 3) : 0;
    return m;
}

// X' element of tile element (z_q, y_q) in column w of tile (cg, kp).
// Line tile layout: tile row q (W elements) at row_pad(q) W, one padding row after every 8 rows
// (bank spreading, see PadTileAddr). Qy is a multiple of 8, so a y column (fixed z_q) and a z
// column (fixed y_q) are:
__device__ __forceinline__ PadTileAddr tile_y(const Geom &g, const LineMap &mp) {
    return PadTileAddr{row_pad(mp.zq * g.Qy) * g.W + mp.w, g.W};
}
__device__ __forceinline__ TileAddr tile_z(const Geom &g, const LineMap &mp) {
    return TileAddr{row_pad(mp.yq) * g.W + mp.w, row_pad(g.Qy) * g.W};
}
// smem position of register slot m after a forward transform that ends in registers
__device__ __forceinline__ int tile_slot(const LineMap &mp, bool two_axes, const PadTileAddr &ady,
                                         const TileAddr &adz, int m) {
    return two_axes ? adz.at(mp.jz + m * mp.nz8) : ady.at(mp.jy + m * mp.ny8);
}

// Forward y (and z) transform of one X'-layout array for a line tile: the first stage reads
// global memory into v; the last stage leaves the result in v (to_regs) or in the tile in
// natural order.
template <typename V>
__device__ __forceinline__ void line_forward(V (&v)[8], const Geom &g, const LineMap &mp, int kp, int cg,
                                             const V *src, V *tile, const PadTileAddr &ady,
                                             const TileAddr &adz, bool to_regs, const StageTw<typename ElemOf<V>::Tw> &st);

// X' and C' are streamed once per pass: the passes read them with __ldcg and write them with
// __stcg (cached in L2 only), so they do not evict the twiddle tables and register spills that
// the transforms keep in L1.
__device__ __forceinline__ size_t xprime_index(const Geom &g, int kp, int cg, int zq, int yq, int w) {
    return (size_t)(kp * g.Q + zq * g.Qy + yq) * g.xs + cg * g.W + w;
}

template <typename V>
__device__ __forceinline__ void line_forward(V (&v)[8], const Geom &g, const LineMap &mp, int kp, int cg,
                                             const V *src, V *tile, const PadTileAddr &ady,
                                             const TileAddr &adz, bool to_regs, const StageTw<typename ElemOf<V>::Tw> &st) {
    const bool two_axes = g.Qz > 1;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = __ldcg(&src[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)]);
    fft_run<-1>(v, tile, ady, g.lQy, mp.jy, true, true, to_regs && !two_axes, st);
    if (two_axes) fft_run<-1>(v, tile, adz, g.lQz, mp.jz, true, false, to_regs, st);
}

// y transform of a line tile: length 2^LY fixed at compile time when LY > 0 (one-axis tiles;
// straight-line code with no switch over lengths, fewer live registers), else the plan's length
template <int S, int LY, typename V>
__device__ __forceinline__ void line_yfft(V (&v)[8], V *sm, const PadTileAddr &ad, const Geom &g, int j,
                                          bool in_regs, bool out_regs, const StageTw<typename ElemOf<V>::Tw> &tw) {
    if constexpr (LY > 0) fft_run_t<S, LY>(v, sm, ad, j, true, in_regs, out_regs, tw, BlockBarrier());
    else fft_run<S>(v, sm, ad, g.lQy, j, true, in_regs, out_regs, tw);
}

// z transform of a two-axis line tile: length 2^LZ fixed at compile time when LZ > 0
template <int S, int LZ, typename V>
__device__ __forceinline__ void line_zfft(V (&v)[8], V *sm, const TileAddr &ad, const Geom &g, int j,
                                          bool in_regs, bool out_regs, const StageTw<typename ElemOf<V>::Tw> &tw) {
    if constexpr (LZ > 0) fft_run_t<S, LZ>(v, sm, ad, j, true, in_regs, out_regs, tw, BlockBarrier());
    else fft_run<S>(v, sm, ad, g.lQz, j, true, in_regs, out_regs, tw);
}

// LY > 0, LZ = 0: the kernel only serves plans with Qz = 1 and Qy = 2^LY; LY, LZ > 0: plans with
// Qy = 2^LY and Qz = 2^LZ; LY = LZ = 0: any plan (lengths at run time).
// The body of one line-pass block (column group cg, split index kp, field or batch member);
// k_line runs it as its own block, the persistent batch kernel once per work item.
template <typename R, int MODE, int LY = 0, int LZ = 0>
__device__ __forceinline__ void line_body(const Geom &g, const LineArgs<R> &a, int cg, int kp, int field) {
    using V = typename VT<R>::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    V *T = sm;
    V *Cs = sm + g.tsz;
    const LineMap mp = line_map(g, threadIdx.x);
    const PadTileAddr ady = tile_y(g, mp);
    const TileAddr adz = tile_z(g, mp);
    const bool two_axes = LZ > 0 || (LY == 0 && g.Qz > 1);
    int kpy, kpz;
    line_kp(g, kp, kpy, kpz);
    const int lsy = g.lPy + g.lRy, lsz = g.lPz + g.lRz;   // ky = kpy + (k_qy << lsy), kz likewise
    V vt[8], vc[8];

    if (MODE == LINE_STEP || MODE == LINE_SCHEME) {
        // C' first, completely into smem (natural order), so that only one register set is live
        const V *C = reinterpret_cast<const V *>(a.c) + (size_t)field * g.nhalf;
#pragma unroll
        for (int m = 0; m < 8; ++m) vc[m] = __ldcg(&C[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)]);
        if constexpr (MODE == LINE_SCHEME) {
            if (a.cprev) {
                const V *Cp = reinterpret_cast<const V *>(a.cprev) + (size_t)field * g.nhalf;
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const V u = __ldcg(&Cp[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)]);
                    vc[m] = V{a.up.cw0 * vc[m].x + a.up.cw1 * u.x, a.up.cw0 * vc[m].y + a.up.cw1 * u.y};
                }
            }
        }
        line_yfft<-1, LY>(vc, Cs, ady, g, mp.jy, true, false, a.st);
        if (two_axes) line_zfft<-1, LZ>(vc, Cs, adz, g, mp.jz, false, false, a.st);
    }
    if (MODE == LINE_STEP || MODE == LINE_FWD || MODE == LINE_SCHEME) {
        const V *X = reinterpret_cast<const V *>(a.x) + (size_t)field * g.nhalf;
#pragma unroll
        for (int m = 0; m < 8; ++m) vt[m] = __ldcg(&X[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)]);
        if constexpr (MODE == LINE_SCHEME) {
            if (a.xprev) {
                const V *Xp = reinterpret_cast<const V *>(a.xprev) + (size_t)field * g.nhalf;
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const V u = __ldcg(&Xp[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)]);
                    vt[m] = V{a.up.xw0 * vt[m].x + a.up.xw1 * u.x, a.up.xw0 * vt[m].y + a.up.xw1 * u.y};
                }
            }
        }
        line_yfft<-1, LY>(vt, T, ady, g, mp.jy, true, !two_axes, a.st);
        if (two_axes) line_zfft<-1, LZ>(vt, T, adz, g, mp.jz, false, true, a.st);
    }


    if (MODE == LINE_FWD) {
        // registers hold k_qy = jy + m ny8 (one axis) or k_qz = jz + m nz8 (two axes)
        V *O = reinterpret_cast<V *>(a.std_out) + (size_t)field * g.nstd;
        const int kx = cg * g.W + mp.w;
        if (kx <= g.M) {
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int kqy = two_axes ? mp.yq : mp.jy + m * mp.ny8;
                const int kqz = two_axes ? mp.jz + m * mp.nz8 : 0;
                const int ky = kpy + (kqy << lsy), kz = kpz + (kqz << lsz);
                O[((size_t)kz * g.ny + ky) * (g.M + 1) + kx] = cscale(vt[m], a.scale);
            }
        }
        return;
    }

    if (MODE == LINE_STEP || MODE == LINE_SCHEME) {
        OpR<R> op = field == 0 ? a.up.op[0] : a.up.op[1];
        if (a.rmem) op.r = a.rmem[field];
        const R invQ = a.up.invQ, inv_halfN = a.up.inv_halfN, dt = a.up.dt;
        const R cy = a.up.cy, cz = a.up.cz;
        const int kx = cg * g.W + mp.w;
        const R fx = a.up.cx * (R)kx;
        // the C transform's outputs at this thread's register positions, read one at a time
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const V c = Cs[tile_slot(mp, two_axes, ady, adz, m)];
            const int kqy = two_axes ? mp.yq : mp.jy + m * mp.ny8;
            const int kqz = two_axes ? mp.jz + m * mp.nz8 : 0;
            const int ky = kpy + (kqy << lsy), kz = kpz + (kqz << lsz);
            const int my = ky <= (g.ny >> 1) ? ky : ky - g.ny;
            const int mz = kz <= (g.nz >> 1) ? kz : kz - g.nz;
            const R fy = cy * (R)my, fz = cz * (R)mz;
            const R k2 = fx * fx + fy * fy + fz * fz;
            const R lk = lin_symbol<R>(op, k2);
            R ca, cb;
            if constexpr (MODE == LINE_SCHEME) {
                const R dk = dt * k2;
                const R inv = (R)1 / (a.up.d0 + a.up.d1 * dk * (lk + a.up.S));
                ca = ((R)1 + dk * a.up.S) * inv * invQ;
                cb = a.up.d1 * dk * inv * inv_halfN;
            } else {
                const R inv = (R)1 / ((R)1 + dt * k2 * lk);
                ca = inv * invQ;
                cb = dt * k2 * inv * inv_halfN;
            }
            V t = V{ca * vt[m].x - cb * c.x, ca * vt[m].y - cb * c.y};
            if (kx == 0 && ky == 0 && kz == 0) t = V{(R)0, (R)0};
            vt[m] = t;
        }
    }

    if (MODE == LINE_INV) {
        const V *I = reinterpret_cast<const V *>(a.std_in) + (size_t)field * g.nstd;
        const int kx = cg * g.W + mp.w;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int kqy = two_axes ? mp.yq : mp.jy + m * mp.ny8;
            const int kqz = two_axes ? mp.jz + m * mp.nz8 : 0;
            const int ky = kpy + (kqy << lsy), kz = kpz + (kqz << lsz);
            vt[m] = kx <= g.M ? I[((size_t)kz * g.ny + ky) * (g.M + 1) + kx] : V{(R)0, (R)0};
        }
    }

    // inverse: the last forward axis first, from registers
    if (two_axes) {
        line_zfft<+1, LZ>(vt, T, adz, g, mp.jz, true, false, a.st);
        line_yfft<+1, LY>(vt, T, ady, g, mp.jy, false, true, a.st);
    } else {
        line_yfft<+1, LY>(vt, T, ady, g, mp.jy, true, true, a.st);
    }
    V *Xo = reinterpret_cast<V *>(MODE != LINE_INV && a.xout ? a.xout : a.x) + (size_t)field * g.nhalf;
    const R sc = MODE == LINE_INV ? a.scale : (R)1;
#pragma unroll
    for (int m = 0; m < 8; ++m)
        __stcg(&Xo[xprime_index(g, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)], cscale(vt[m], sc));
}

template <typename R, int MODE, int MAXT, int LY = 0, int LZ = 0>
__global__ void __launch_bounds__(MAXT, (sizeof(R) == 4 && MAXT == 512) ? 2 : 1) k_line(const Geom g, const LineArgs<R> a) {
    line_body<R, MODE, LY, LZ>(g, a, blockIdx.x, blockIdx.y, blockIdx.z);
}

}  // namespace pfc
