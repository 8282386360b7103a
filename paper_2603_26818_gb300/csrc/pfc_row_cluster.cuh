// Row pass psi^3 (ROW_CUBE) with one row group split over a cluster of CS thread blocks.
//
// The single-block row kernel keeps all P rows of its group in shared memory. With Py = 8 rows of
// nx = 4096 (18 KB each in FP32) that is 147 KB, so only one block fits an SM and its load,
// transform and store phases cannot overlap with another block's. Here the CS blocks of a cluster
// share the group: block h keeps rows y_p in [h Py/CS, (h+1) Py/CS) in its own shared memory, so
// two blocks (of two different groups) fit an SM. Phase B (load of X', y twiddle, inverse P-part
// across the Py rows, real-transform pre-processing) and phase D (post-processing, forward
// P-part, twiddle, store of C') give each thread all Py rows of one column pair; the rows held by
// the other blocks of the cluster are written and read through distributed shared memory. The
// blocks split the column pairs between them. The per-row transforms and psi^3 are the single-
// block kernel's, on the block's own rows. Used for Pz = 1, Py = 8, one group per cluster.
#pragma once

#include <cooperative_groups.h>

#include "pfc_pass.cuh"

namespace pfc {

constexpr int ROWCL_PY = 8;

// Cluster barrier without memory ordering (barrier.cluster.arrive.relaxed, then wait).
__device__ __forceinline__ void cluster_sync_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// LM = log2 M, the row transform length, fixed at compile time (the planner uses this kernel
// for nx = 4096 only).
template <typename R, int CS, int LM>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(512, 2)
    k_row_cube_cl(const Geom g, const RowArgs<R> a) {
    using V = typename VT<R>::V;
    namespace cg = cooperative_groups;
    constexpr int RPC = ROWCL_PY / CS;   // rows per block
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const cg::cluster_group cl = cg::this_cluster();
    const int h = (int)cl.block_rank();
    const int tid = threadIdx.x, nt = blockDim.x;
    const int field = blockIdx.y;
    const int M = g.M, hM = M >> 1;
    const int grp = blockIdx.x / CS;
    const R mean = a.mean ? (R)a.mean[field] : (R)0;
    // smem: RPC rows | one scratch row per row in flight (ping-pong transforms) | split
    // twiddles of the group's Py rows
    const int Tr = M >> 3;
    const int RB = nt / Tr;
    V *stw = sm + (RPC + RB) * g.rs;
    for (int t = tid; t < ROWCL_PY; t += nt) stw[t] = split_twiddle(g, a.tw, grp, 0, t);
    V *rows[CS];                // row 0 of each block of the cluster (generic addresses)
#pragma unroll
    for (int c = 0; c < CS; ++c) rows[c] = cl.map_shared_rank(sm, c);
    // stw visible in the block; every block of the cluster has started (its shared memory
    // exists) before any block writes into it. Nothing is published across blocks yet, so the
    // cluster barrier needs no release ordering.
    __syncthreads();
    cluster_sync_relaxed();

    // ---- phase B: this block's share of the column pairs (kk, M - kk), kk in [0, M/2) ----
    {
        const V *X = reinterpret_cast<const V *>(a.in) + (size_t)field * g.nhalf;
        V *pw = reinterpret_cast<V *>(a.proj) + (size_t)field * g.nhalf;
        const int per = hM / CS;
        for (int e = tid; e < per; e += nt) {
            const int kk = h * per + e;
            const int npass = kk == 0 ? 2 : 1;   // kk = 0: the pair (0, M), then the column M/2
#pragma unroll 1
            for (int pp = 0; pp < npass; ++pp) {
                const bool k0 = kk == 0 && pp == 0;
                const int ca = pp ? hM : kk, cb = pp ? hM : (kk == 0 ? M : M - kk);
                V va[ROWCL_PY], vb[ROWCL_PY];
#pragma unroll
                for (int yy = 0; yy < ROWCL_PY; ++yy) {
                    const V *src = X + (size_t)(yy * g.QR + grp) * g.xs;
                    const V w = stw[yy];
                    va[yy] = ctw<+1>(__ldcg(&src[ca]), w);
                    vb[yy] = ctw<+1>(__ldcg(&src[cb]), w);
                }
                dft8<+1>(va);
                dft8<+1>(vb);
                const V w = __ldg(&a.tw[ca << (g.ltab - g.lnx)]);
#pragma unroll
                for (int yy = 0; yy < ROWCL_PY; ++yy) {
                    V za, zb;
                    c2r_pre_pair<V, R>(va[yy], vb[yy], w, k0, za, zb);
                    V *dst = rows[yy / RPC] + (yy % RPC) * g.rs;
                    dst[row_swz(ca)] = za;
                    if (!k0 && cb != ca) dst[row_swz(cb)] = zb;
                }
                if (k0 && a.proj) {
                    // Hermitian projection of the kx = 0 and nx/2 columns (see
                    // project_edge_columns_par): X' = DFT_P(real parts of the row values) / P
#pragma unroll
                    for (int yy = 0; yy < ROWCL_PY; ++yy) {
                        va[yy].y = (R)0;
                        vb[yy].y = (R)0;
                    }
                    dft8<-1>(va);
                    dft8<-1>(vb);
                    const R invP = (R)1 / (R)ROWCL_PY;
#pragma unroll
                    for (int yy = 0; yy < ROWCL_PY; ++yy) {
                        V *dst = pw + (size_t)(yy * g.QR + grp) * g.xs;
                        dst[0] = cscale(cmul(va[yy], stw[yy]), invP);
                        dst[M] = cscale(cmul(vb[yy], stw[yy]), invP);
                    }
                }
            }
        }
    }
    cl.sync();

    // ---- per-row transforms and psi^3 on this block's rows ----
    {
        const bool grouped = Tr >= 32 && RB <= 15 && RPC % RB == 0;
        const int gidx = tid / Tr;
        const NamedBarrier nbar{1 + gidx, Tr};
        for (int rb = 0; rb < RPC; rb += RB) {
            const int r = rb + gidx, j = tid % Tr;
            const bool act = r < RPC;
            const RowAddr ad{r * g.rs};
            V v[8];
            // ping-pong through this row group's scratch row
            const RowAddr sc{(RPC + gidx) * g.rs};
            if (grouped) fft_run_pp_t<+1, LM>(v, sm, ad, sc, j, act, false, true, a.st, nbar);
            else fft_run_pp_t<+1, LM>(v, sm, ad, sc, j, act, false, true, a.st, BlockBarrier());
            cube_shifted(v, mean);
            if (grouped) fft_run_pp_t<-1, LM>(v, sm, ad, sc, j, act, true, false, a.st, nbar);
            else fft_run_pp_t<-1, LM>(v, sm, ad, sc, j, act, true, false, a.st, BlockBarrier());
        }
    }
    cl.sync();

    // ---- phase D: this block's share of the column pairs ----
    {
        V *out = reinterpret_cast<V *>(a.out) + (size_t)field * g.nhalf;
        const int per = hM / CS;
        for (int e = tid; e < per; e += nt) {
            const int kk = h * per + e;
            const int npass = kk == 0 ? 2 : 1;
#pragma unroll 1
            for (int pp = 0; pp < npass; ++pp) {
                const bool k0 = kk == 0 && pp == 0;
                const int ca = pp ? hM : kk, cb = pp ? hM : (kk == 0 ? M : M - kk);
                const V w = __ldg(&a.tw[ca << (g.ltab - g.lnx)]);
                V va[ROWCL_PY], vb[ROWCL_PY];
#pragma unroll
                for (int yy = 0; yy < ROWCL_PY; ++yy) {
                    const V *src = rows[yy / RPC] + (yy % RPC) * g.rs;
                    const V za = src[row_swz(ca)];
                    const V zb = (k0 || cb == ca) ? za : src[row_swz(cb)];
                    r2c_post_pair<V, R>(za, zb, w, k0, va[yy], vb[yy]);
                }
                dft8<-1>(va);
                dft8<-1>(vb);
#pragma unroll
                for (int yy = 0; yy < ROWCL_PY; ++yy) {
                    const V t = stw[yy];
                    V *dst = out + (size_t)(yy * g.QR + grp) * g.xs;
                    if constexpr (sizeof(R) == 4) {
                        st_keep_l2(&dst[ca], cscale(cmul(va[yy], t), a.scale));
                        if (cb != ca) st_keep_l2(&dst[cb], cscale(cmul(vb[yy], t), a.scale));
                    } else {
                        __stcg(&dst[ca], cscale(cmul(va[yy], t), a.scale));
                        if (cb != ca) __stcg(&dst[cb], cscale(cmul(vb[yy], t), a.scale));
                    }
                }
            }
        }
    }
    // no block leaves while another may still read its rows. Every read of phase D fed a store
    // issued before this point, so a barrier without release ordering suffices (it does not wait
    // for this block's global stores to complete).
    cluster_sync_relaxed();
}

}  // namespace pfc

namespace pfc {

// The psi^3 row pass of a 3D plan with Pz = 8 on clusters of two blocks: block h keeps the rows
// of z_p in [4h, 4h + 4) (4 Py rows), so that a group of 8 Py rows too large for two blocks per
// SM is split in two. Phase A (z-part inverse from X') and phase E (z-part forward to C') give
// each thread all eight z_p rows of one (k_py, column) item, the block's own and, through
// distributed shared memory, the partner's; the items are split between the blocks. Phases B
// and D (y-part and real-transform processing) and the row transforms touch only the block's
// own rows. The real parts of the kx = 0 and nx/2 columns are gathered in block 0, which does
// the Hermitian projection (project_edge_columns_par) for the group.
// LM = log2 M fixed at compile time (the planner uses this kernel for nx = 512, 1024 and 2048).
template <typename R, int LM>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512, 2)
    k_row_cube_cl3(const Geom g, const RowArgs<R> a) {
    using V = typename VT<R>::V;
    namespace cg = cooperative_groups;
    constexpr int PZ = 8, ZPB = 4;   // z_p rows per block
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const cg::cluster_group cl = cg::this_cluster();
    const int h = (int)cl.block_rank();
    const int tid = threadIdx.x, nt = blockDim.x;
    const int field = blockIdx.y;
    const int M = g.M, lM = g.lM, hM = M >> 1, Py = g.Py, P = g.P;
    const int grp = blockIdx.x >> 1;
    const int rows = ZPB * Py;
    const R mean = a.mean ? (R)a.mean[field] : (R)0;
    // smem: rows (z_p local, k_py or y_p) | split twiddles of the group (P) | edge values (2 P,
    // used in block 0) | the projection's scratch (2 P complex, block 0)
    V *stw = sm + rows * g.rs;
    R *edge = reinterpret_cast<R *>(stw + P);
    for (int t = tid; t < P; t += nt) stw[t] = split_twiddle(g, a.tw, grp, t / Py, t % Py);
    V *rowp[2];
    rowp[0] = cl.map_shared_rank(sm, 0);
    rowp[1] = cl.map_shared_rank(sm, 1);
    R *edge0 = cl.map_shared_rank(edge, 0);
    __syncthreads();
    cluster_sync_relaxed();

    const int main = Py << lM, cnt = main + Py, hc = (cnt + 1) >> 1;
    const int e_end = (h + 1) * hc < cnt ? (h + 1) * hc : cnt;
    // ---- phase A: z-part inverse of this block's share of the (k_py, column) items ----
    {
        const V *X = reinterpret_cast<const V *>(a.in) + (size_t)field * g.nhalf;
        for (int e = h * hc + tid; e < e_end; e += nt) {
            int k, kpy;
            if (e < main) { k = e & (M - 1); kpy = e >> lM; }
            else { k = M; kpy = e - main; }
            V t[PZ];
#pragma unroll
            for (int zz = 0; zz < PZ; ++zz)
                t[zz] = ctw<+1>(__ldcg(&X[(size_t)((zz * Py + kpy) * g.QR + grp) * g.xs + k]), stw[zz * Py + kpy]);
            dft8<+1>(t);
#pragma unroll
            for (int zz = 0; zz < PZ; ++zz)
                rowp[zz / ZPB][((zz % ZPB) * Py + kpy) * g.rs + row_swz(k)] = t[zz];
        }
    }
    cl.sync();

    // ---- phase B: y-part inverse and c2r pre-processing of the block's own rows ----
    for (int e = tid; e < ZPB * hM; e += nt) {
        const int kk = e % hM, zl = e / hM, zg = h * ZPB + zl;
        const int npass = kk == 0 ? 2 : 1;
#pragma unroll 1
        for (int pp = 0; pp < npass; ++pp) {
            const bool k0 = kk == 0 && pp == 0;
            const int ca = pp ? hM : kk, cb = pp ? hM : (kk == 0 ? M : M - kk);
            V va[8], vb[8];
#pragma unroll
            for (int yy = 0; yy < 8; ++yy) {
                if (yy < Py) {
                    const int row = zl * Py + yy;
                    va[yy] = sm[row * g.rs + row_swz(ca)];
                    vb[yy] = sm[row * g.rs + row_swz(cb)];
                }
            }
            dft_small<+1>(va, Py);
            dft_small<+1>(vb, Py);
            const V w = __ldg(&a.tw[ca << (g.ltab - g.lnx)]);
#pragma unroll
            for (int yy = 0; yy < 8; ++yy) {
                if (yy < Py) {
                    const int row = zl * Py + yy;
                    if (k0) {
                        edge0[zg * Py + yy] = va[yy].x;
                        edge0[P + zg * Py + yy] = vb[yy].x;
                    }
                    V za, zb;
                    c2r_pre_pair<V, R>(va[yy], vb[yy], w, k0, za, zb);
                    sm[row * g.rs + row_swz(ca)] = za;
                    if (!k0 && cb != ca) sm[row * g.rs + row_swz(cb)] = zb;
                }
            }
        }
    }
    __syncthreads();

    // ---- row transforms and psi^3 on the block's rows ----
    {
        const int Tr = M >> 3;
        const int RB = nt / Tr;
        for (int rb = 0; rb < rows; rb += RB) {
            const int r = rb + tid / Tr, j = tid % Tr;
            const bool act = r < rows;
            const RowAddr ad{r * g.rs};
            V v[8];
            const RowBarrier rbar = Tr <= 32 ? RowBarrier{0, Tr} : RowBarrier{0, nt};
            fft_run_t<+1, LM>(v, sm, ad, j, act, false, true, a.st, rbar);
            cube_shifted(v, mean);
            fft_run_t<-1, LM>(v, sm, ad, j, act, true, false, a.st, rbar);
        }
    }
    __syncthreads();

    // ---- phase D: c2r post-processing and y-part forward, rows (z_p, k_py) of the block ----
    for (int e = tid; e < ZPB * hM; e += nt) {
        const int kk = e % hM, zl = e / hM;
        const int npass = kk == 0 ? 2 : 1;
#pragma unroll 1
        for (int pp = 0; pp < npass; ++pp) {
            const bool k0 = kk == 0 && pp == 0;
            const int ca = pp ? hM : kk, cb = pp ? hM : (kk == 0 ? M : M - kk);
            row_pair_d<R>(g, sm, nullptr, 0, grp, zl, ca, cb, k0, a.tw, stw, a.scale);
        }
    }
    cl.sync();

    // ---- phase E: z-part forward of this block's share of the items, twiddle, store C' ----
    {
        V *out = reinterpret_cast<V *>(a.out) + (size_t)field * g.nhalf;
        for (int e = h * hc + tid; e < e_end; e += nt) {
            int k, kpy;
            if (e < main) { k = e & (M - 1); kpy = e >> lM; }
            else { k = M; kpy = e - main; }
            V t[PZ];
#pragma unroll
            for (int zz = 0; zz < PZ; ++zz) t[zz] = rowp[zz / ZPB][((zz % ZPB) * Py + kpy) * g.rs + row_swz(k)];
            dft8<-1>(t);
#pragma unroll
            for (int zz = 0; zz < PZ; ++zz)
                __stcg(&out[(size_t)((zz * Py + kpy) * g.QR + grp) * g.xs + k],
                       cscale(cmul(t[zz], stw[zz * Py + kpy]), a.scale));
        }
    }
    // block 0 projects the edge columns (all 2 P edge values arrived before the cluster barrier
    // that follows phase D)
    if (h == 0 && a.proj) {
        V *xw = reinterpret_cast<V *>(a.proj) + (size_t)field * g.nhalf;
        project_edge_columns_par<R>(g, edge, grp, stw, xw, reinterpret_cast<V *>(edge + 2 * P));
    }
    cluster_sync_relaxed();
}

}  // namespace pfc
