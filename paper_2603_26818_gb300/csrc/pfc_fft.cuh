// Device FFT building blocks for the PFC passes (sm_103a).
//
// All transforms are power-of-two Stockham FFTs held in shared memory, with radix-8 stages
// (one radix-2 or radix-4 stage when log2 n is not a multiple of 3). A thread with index
// j in [0, n/8) always loads the eight elements j + m n/8 (m = 0..7) of its instance, in every
// stage; it stores them to the auto-sorted Stockham positions. In the last stage the stored
// positions are again j + m n/8, so a transform can end with its outputs in registers and a
// second transform can start from those registers: the row pass forms psi^3 between an
// inverse and a forward transform without touching shared memory.
//
// Stage twiddles come from per-stage tables (StageTw) generated on the host in FP64 (rounded once
// for the FP32 path); other twiddles from one table tw[i] = exp(-2 pi i * i / 2^ltab). The
// inverse transform uses the conjugate.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pfc {

template <typename R> struct VT;
template <> struct VT<float> { using V = float2; };
template <> struct VT<double> { using V = double2; };

// Two complex values of adjacent kx columns, moved and transformed together (one 16-byte access,
// one twiddle for both): the element type of the two-column line pass.
struct __align__(16) cf2 {
    float2 a, b;
};

// L2 eviction priority of the C' stream of a step: the psi^3 row pass writes C' with priority
// to stay in L2 (evict_last) for the update pass of the same step, which reads it for the last
// time (evict_first). PFC_L2_HINTS=0 at compile time gives plain .cg accesses (to compare).
#ifndef PFC_L2_HINTS
#define PFC_L2_HINTS 1
#endif
__device__ __forceinline__ void st_keep_l2(float2 *p, float2 v) {
#if PFC_L2_HINTS
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
#else
    __stcg(p, v);
#endif
}
__device__ __forceinline__ float4 ld_last_use_l2(const float4 *p) {
#if PFC_L2_HINTS
    unsigned long long pol;
    float4 r;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p), "l"(pol)
                 : "memory");
    return r;
#else
    return __ldcg(p);
#endif
}

// scalar type and twiddle (table element) type of a transform element type
template <typename V> struct ElemOf;
template <> struct ElemOf<float2> { using R = float; using Tw = float2; };
template <> struct ElemOf<double2> { using R = double; using Tw = double2; };
template <> struct ElemOf<cf2> { using R = float; using Tw = float2; };

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V> __device__ __forceinline__ V cconj(V a) { return V{a.x, -a.y}; }
template <typename V, typename R> __device__ __forceinline__ V cscale(V a, R s) { return V{a.x * s, a.y * s}; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * b for S = -1, a * conj(b) for S = +1 (b is a forward-table twiddle).
template <int S, typename V> __device__ __forceinline__ V ctw(V a, V b) {
    if (S < 0) return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
    return V{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// multiply by S*i
template <int S, typename V> __device__ __forceinline__ V cmul_i(V a) {
    if (S < 0) return V{a.y, -a.x};
    return V{-a.y, a.x};
}
// t W8 and t W8^3, W8 = exp(S 2 pi i / 8), h = 1/sqrt(2):
//   t W8 = (x - S y, y + S x) h;  t W8^3 = (-x - S y, S x - y) h
template <int S, typename V, typename R> __device__ __forceinline__ V w8_1(V t, R h) {
    return V{(t.x - S * t.y) * h, (t.y + S * t.x) * h};
}
template <int S, typename V, typename R> __device__ __forceinline__ V w8_3(V t, R h) {
    return V{(-t.x - S * t.y) * h, (S * t.x - t.y) * h};
}

// the same operations on two columns at once
__device__ __forceinline__ cf2 cadd(cf2 p, cf2 q) { return cf2{cadd(p.a, q.a), cadd(p.b, q.b)}; }
__device__ __forceinline__ cf2 csub(cf2 p, cf2 q) { return cf2{csub(p.a, q.a), csub(p.b, q.b)}; }
__device__ __forceinline__ cf2 cscale(cf2 p, float s) { return cf2{cscale(p.a, s), cscale(p.b, s)}; }
template <int S> __device__ __forceinline__ cf2 ctw(cf2 p, float2 w) { return cf2{ctw<S>(p.a, w), ctw<S>(p.b, w)}; }
template <int S> __device__ __forceinline__ cf2 cmul_i(cf2 p) { return cf2{cmul_i<S>(p.a), cmul_i<S>(p.b)}; }
template <int S> __device__ __forceinline__ cf2 w8_1(cf2 t, float h) { return cf2{w8_1<S>(t.a, h), w8_1<S>(t.b, h)}; }
template <int S> __device__ __forceinline__ cf2 w8_3(cf2 t, float h) { return cf2{w8_3<S>(t.a, h), w8_3<S>(t.b, h)}; }

// ------------------------------------------------------------------------------------------
// Small DFTs in registers: X[k] = sum_n x[n] exp(S 2 pi i n k / R), in natural order.
// ------------------------------------------------------------------------------------------
template <int S, typename V> __device__ __forceinline__ void dft2(V &a, V &b) {
    V t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int S, typename V> __device__ __forceinline__ void dft4(V &c0, V &c1, V &c2, V &c3) {
    V d0 = cadd(c0, c2), e0 = csub(c0, c2);
    V d1 = cadd(c1, c3), e1 = cmul_i<S>(csub(c1, c3));
    c0 = cadd(d0, d1);
    c2 = csub(d0, d1);
    c1 = cadd(e0, e1);
    c3 = csub(e0, e1);
}

// Decimation in frequency: even outputs from x[n] + x[n+4], odd outputs from
// (x[n] - x[n+4]) W8^n, each a DFT4.
template <int S, typename V> __device__ __forceinline__ void dft8(V (&v)[8]) {
    using R = typename ElemOf<V>::R;
    const R h = (R)0.70710678118654752440084436210484903928;
    V a0 = cadd(v[0], v[4]), a4 = csub(v[0], v[4]);
    V a1 = cadd(v[1], v[5]), t5 = csub(v[1], v[5]);
    V a2 = cadd(v[2], v[6]), a6 = cmul_i<S>(csub(v[2], v[6]));
    V a3 = cadd(v[3], v[7]), t7 = csub(v[3], v[7]);
    V a5 = w8_1<S>(t5, h);
    V a7 = w8_3<S>(t7, h);
    V b0 = cadd(a0, a2), b2 = csub(a0, a2);
    V b1 = cadd(a1, a3), b3 = cmul_i<S>(csub(a1, a3));
    V b4 = cadd(a4, a6), b6 = csub(a4, a6);
    V b5 = cadd(a5, a7), b7 = cmul_i<S>(csub(a5, a7));
    v[0] = cadd(b0, b1);
    v[4] = csub(b0, b1);
    v[2] = cadd(b2, b3);
    v[6] = csub(b2, b3);
    v[1] = cadd(b4, b5);
    v[5] = csub(b4, b5);
    v[3] = cadd(b6, b7);
    v[7] = csub(b6, b7);
}

// DFT of n in {1, 2, 4, 8} points held in t[0..n).
template <int S, typename V> __device__ __forceinline__ void dft_small(V (&t)[8], int n) {
    if (n == 8) dft8<S>(t);
    else if (n == 4) dft4<S>(t[0], t[1], t[2], t[3]);
    else if (n == 2) dft2<S>(t[0], t[1]);
}

// ------------------------------------------------------------------------------------------
// Shared-memory addressing of one transform instance: element i lives at at(i).
// ------------------------------------------------------------------------------------------
// One padding slot after every 8 elements (bank spreading of line tile rows, see PadTileAddr).
// For the index sets a transform touches (j + m n/8 with n/8 a multiple of 8, and the Stockham
// outputs o + r Ns with Ns a multiple of 8, or o a multiple of 8 when Ns = 1), the padded index
// is linear in m (or r) with the steps below.
__host__ __device__ __forceinline__ int row_pad(int i) { return i + (i >> 3); }
template <int N8> __host__ __device__ constexpr int pad_step() { return N8 >= 8 ? N8 + N8 / 8 : N8; }
template <int NS> __host__ __device__ constexpr int pad_ostep() { return NS >= 8 ? NS + NS / 8 : NS; }

// A row of a row buffer, starting at element base (a multiple of 16). Element i lives at
// base + row_swz(i), row_swz(i) = i ^ ((i >> 3) & 15): the XOR permutes each aligned block of 16
// elements, so rows need no padding, and each index set the transforms and the pair phases
// touch in one half-warp (16 consecutive elements, the stride-8 outputs of a first stage, the
// 8-element runs of a second stage) lands on 16 distinct bank groups. (A padding slot per 8
// elements leaves two-way conflicts on the consecutive sets.) When an index set has a stride
// that is a multiple of 128, the XOR term is the same for all of its members and the accessors
// add compile-time steps to one computed address.
__host__ __device__ __forceinline__ int row_swz(int i) { return i ^ ((i >> 3) & 15); }

struct RowAddr {
    int base;
    __device__ __forceinline__ int at(int i) const { return base + row_swz(i); }
};

// A column of an interleaved tile with a uniform stride: element i at off + i * stride.
struct TileAddr {
    int off, stride;
    __device__ __forceinline__ int at(int i) const { return off + i * stride; }
};

// A column of an interleaved tile whose rows of w elements get one padding row after every 8
// rows: element i at off + row_pad(i) w. For the transform index sets (see row_pad) the address
// is linear in m (or r) with steps pad_step * w, and with tile rows of at least 16 bytes
// every half-warp access of the transforms touches 16 distinct banks.
struct PadTileAddr {
    int off, w;
    __device__ __forceinline__ int at(int i) const { return off + row_pad(i) * w; }
};

// Per-stage twiddle tables, laid out [r][k] so that the threads of a warp (consecutive k) read
// consecutive addresses for every r:
//   t8: radix-8 stages with Ns = 8, 64, 512:  entry r Ns + k = W_{8 Ns}^{r k}, r = 0..7
//   t4: radix-4 last stages with Ns = 8, 64, 512:  r Ns + k = W_{4 Ns}^{r k}, r = 0..3
//   t2: radix-2 last stages with Ns = 8, 64, 512:  r Ns + k = W_{2 Ns}^{r k}, r = 0..1
// Tables of one kind are stored back to back; the block for Ns = 8^s starts at
// R (8^s - 8) / 7 entries. All entries are FP64-generated (rounded once for FP32).
struct BlockBarrier {
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct NamedBarrier {
    int id, n;
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
};
// The barrier of the n threads that transform one row: a warp barrier when the row lies within
// one warp (n <= 32, rows of n threads starting at multiples of n), else barrier id over n
// threads (id 0 with n = the block: __syncthreads).
struct RowBarrier {
    int id, n;
    __device__ __forceinline__ void sync() const {
        if (n <= 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

template <typename V> struct StageTw {
    const V *t8, *t4, *t2;
};

__host__ __device__ __forceinline__ int stage_tw_off(int R, int lNs) {
    const int ns = 1 << lNs;
    return R * (ns - 8) / 7;
}

template <int S, typename V>
__device__ __forceinline__ void stage_exec(V (&v)[8], int lR, int lNs, int j, int n8,
                                           const StageTw<typename ElemOf<V>::Tw> &tw) {
    const int Ns = 1 << lNs;
    if (lR == 3) {
        if (lNs > 0) {
            const int k = j & (Ns - 1);
            const auto *t = tw.t8 + stage_tw_off(8, lNs) + k;
#pragma unroll
            for (int r = 1; r < 8; ++r) v[r] = ctw<S>(v[r], __ldg(t + r * Ns));
        }
        dft8<S>(v);
    } else if (lR == 2) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            V c0 = v[u], c1 = v[u + 2], c2 = v[u + 4], c3 = v[u + 6];
            if (lNs > 0) {
                const int k = (j + u * n8) & (Ns - 1);
                const auto *t = tw.t4 + stage_tw_off(4, lNs) + k;
                c1 = ctw<S>(c1, __ldg(t + Ns));
                c2 = ctw<S>(c2, __ldg(t + 2 * Ns));
                c3 = ctw<S>(c3, __ldg(t + 3 * Ns));
            }
            dft4<S>(c0, c1, c2, c3);
            v[u] = c0; v[u + 2] = c1; v[u + 4] = c2; v[u + 6] = c3;
        }
    } else if (lR == 1) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            V c0 = v[u], c1 = v[u + 4];
            if (lNs > 0) {
                const int k = (j + u * n8) & (Ns - 1);
                c1 = ctw<S>(c1, __ldg(tw.t2 + stage_tw_off(2, lNs) + Ns + k));
            }
            dft2<S>(c0, c1);
            v[u] = c0; v[u + 4] = c1;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Transforms with a compile-time length n = 2^L: every stage unrolled, radix and Ns constant.
// ------------------------------------------------------------------------------------------
template <int N8, typename V>
__device__ __forceinline__ void load8_t(V (&v)[8], const V *sm, const RowAddr &ad, int j) {
    if (N8 % 128 == 0) {
        const int p = ad.at(j);
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = sm[p + m * N8];
    } else {
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = sm[ad.at(j + m * N8)];
    }
}
template <int N8, typename V>
__device__ __forceinline__ void load8_t(V (&v)[8], const V *sm, const PadTileAddr &ad, int j) {
    if (N8 >= 8) {
        const int p = ad.at(j), st = pad_step<N8>() * ad.w;
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = sm[p + m * st];
    } else {
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = sm[ad.at(j + m * N8)];
    }
}
template <int N8, typename V>
__device__ __forceinline__ void load8_t(V (&v)[8], const V *sm, const TileAddr &ad, int j) {
    const int p = ad.at(j), st = N8 * ad.stride;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = sm[p + m * st];
}

// Store the R outputs o + r Ns (r < R) of one butterfly.
template <int NS, int R, typename V>
__device__ __forceinline__ void store_group(const V *vals, V *sm, const RowAddr &ad, int o) {
    if (NS % 128 == 0) {
        const int p = ad.at(o);
#pragma unroll
        for (int r = 0; r < R; ++r) sm[p + r * NS] = vals[r];
    } else if (NS == 1 && R == 8) {
        // o = 8 j': row_swz(o + r) = row_swz(o) ^ r, and base is a multiple of 16
        const int p = ad.at(o);
#pragma unroll
        for (int r = 0; r < R; ++r) sm[p ^ r] = vals[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) sm[ad.at(o + r * NS)] = vals[r];
    }
}
template <int NS, int R, typename V>
__device__ __forceinline__ void store_group(const V *vals, V *sm, const PadTileAddr &ad, int o) {
    if (NS >= 8 || (NS == 1 && R == 8)) {
        const int p = ad.at(o), st = pad_ostep<NS>() * ad.w;
#pragma unroll
        for (int r = 0; r < R; ++r) sm[p + r * st] = vals[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) sm[ad.at(o + r * NS)] = vals[r];
    }
}
template <int NS, int R, typename V>
__device__ __forceinline__ void store_group(const V *vals, V *sm, const TileAddr &ad, int o) {
    const int p = ad.at(o), st = NS * ad.stride;
#pragma unroll
    for (int r = 0; r < R; ++r) sm[p + r * st] = vals[r];
}

template <int LR, int LNS, int N8, typename V, typename Addr>
__device__ __forceinline__ void stage_store_t(const V (&v)[8], V *sm, const Addr &ad, int j) {
    constexpr int Ns = 1 << LNS;
    if (LR == 3) {
        const int k = j & (Ns - 1);
        store_group<Ns, 8>(v, sm, ad, ((j - k) << 3) + k);
    } else if (LR == 2) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int b = j + u * N8, k = b & (Ns - 1);
            const V t[4] = {v[u], v[u + 2], v[u + 4], v[u + 6]};
            store_group<Ns, 4>(t, sm, ad, ((b - k) << 2) + k);
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = j + u * N8, k = b & (Ns - 1);
            const V t[2] = {v[u], v[u + 4]};
            store_group<Ns, 2>(t, sm, ad, ((b - k) << 1) + k);
        }
    }
}

template <int S, int L, int LR, int LNS, typename V, typename Addr, typename Bar>
__device__ __forceinline__ void stage_t(V (&v)[8], V *sm, const Addr &ad, int j, bool act,
                                        bool load, bool store, const StageTw<typename ElemOf<V>::Tw> &tw, const Bar &bar) {
    constexpr int N8 = 1 << (L - 3);
    if (act && load) load8_t<N8>(v, sm, ad, j);
    if (act) stage_exec<S>(v, LR, LNS, j, N8, tw);
    if (!store) return;
    bar.sync();
    if (act) stage_store_t<LR, LNS, N8>(v, sm, ad, j);
    bar.sync();
}

template <int S, int L, typename V, typename Addr, typename Bar>
__device__ __forceinline__ void fft_run_t(V (&v)[8], V *sm, const Addr &ad, int j, bool act,
                                          bool in_regs, bool out_regs, const StageTw<typename ElemOf<V>::Tw> &tw, const Bar &bar) {
    constexpr int NFULL = L / 3;
    constexpr int LLAST = L - 3 * NFULL;    // 0: all stages radix 8
    constexpr int NST = NFULL + (LLAST ? 1 : 0);
    // radix-8 stages s = 0 .. NFULL-1 with Ns = 8^s, then one radix 2^LLAST stage
    stage_t<S, L, 3, 0>(v, sm, ad, j, act, !in_regs, !(NST == 1 && out_regs), tw, bar);
    if (NFULL > 1) stage_t<S, L, 3, (NFULL > 1 ? 3 : 0)>(v, sm, ad, j, act, true, !(NST == 2 && out_regs), tw, bar);
    if (NFULL > 2) stage_t<S, L, 3, (NFULL > 2 ? 6 : 0)>(v, sm, ad, j, act, true, !(NST == 3 && out_regs), tw, bar);
    if (NFULL > 3) stage_t<S, L, 3, (NFULL > 3 ? 9 : 0)>(v, sm, ad, j, act, true, !(NST == 4 && out_regs), tw, bar);
    if (LLAST) stage_t<S, L, (LLAST ? LLAST : 1), 3 * NFULL>(v, sm, ad, j, act, true, !out_regs, tw, bar);
}

// Ping-pong stage: the inputs come from src, the outputs go to a different buffer dst, so one
// barrier (after the store) separates this stage's reads from the next stage's writes.
template <int S, int L, int LR, int LNS, typename V, typename Addr, typename Bar>
__device__ __forceinline__ void stage_pp_t(V (&v)[8], V *sm, const Addr &src, const Addr &dst, int j,
                                           bool act, bool load, bool store, const StageTw<typename ElemOf<V>::Tw> &tw,
                                           const Bar &bar) {
    constexpr int N8 = 1 << (L - 3);
    if (act && load) load8_t<N8>(v, sm, src, j);
    if (act) stage_exec<S>(v, LR, LNS, j, N8, tw);
    if (!store) return;
    if (act) stage_store_t<LR, LNS, N8>(v, sm, dst, j);
    bar.sync();
}

// The transform of fft_run_t with its stages alternating between buffer A and a scratch buffer B
// of the same shape: half the barriers of the in-place form. Exactly one of in_regs / out_regs:
//   out_regs: the input is in A; the stores alternate B, A, B, ...; the result is left in v.
//   in_regs:  the input is in v; the stores alternate so that the last one lands in A. A barrier
//             is issued first, so other threads may still be reading A or B.
template <int S, int L, typename V, typename Addr, typename Bar>
__device__ __forceinline__ void fft_run_pp_t(V (&v)[8], V *sm, const Addr &A, const Addr &B, int j,
                                             bool act, bool in_regs, bool out_regs,
                                             const StageTw<typename ElemOf<V>::Tw> &tw, const Bar &bar) {
    constexpr int NFULL = L / 3;
    constexpr int LLAST = L - 3 * NFULL;
    constexpr int NST = NFULL + (LLAST ? 1 : 0);
    const int nstore = NST - (out_regs ? 1 : 0);
    auto dst = [&](int k) -> Addr {
        const bool to_a = in_regs ? ((nstore - 1 - k) & 1) == 0 : (k & 1) != 0;
        return to_a ? A : B;
    };
    auto src = [&](int k) -> Addr { return k == 0 ? A : dst(k - 1); };
    if (in_regs) bar.sync();
    stage_pp_t<S, L, 3, 0>(v, sm, src(0), dst(0), j, act, !in_regs, !(NST == 1 && out_regs), tw, bar);
    if (NFULL > 1)
        stage_pp_t<S, L, 3, (NFULL > 1 ? 3 : 0)>(v, sm, src(1), dst(1), j, act, true, !(NST == 2 && out_regs), tw, bar);
    if (NFULL > 2)
        stage_pp_t<S, L, 3, (NFULL > 2 ? 6 : 0)>(v, sm, src(2), dst(2), j, act, true, !(NST == 3 && out_regs), tw, bar);
    if (NFULL > 3)
        stage_pp_t<S, L, 3, (NFULL > 3 ? 9 : 0)>(v, sm, src(3), dst(3), j, act, true, !(NST == 4 && out_regs), tw, bar);
    if (LLAST)
        stage_pp_t<S, L, (LLAST ? LLAST : 1), 3 * NFULL>(v, sm, src(NFULL), dst(NFULL), j, act, true, !out_regs, tw, bar);
}

template <int S, typename V, typename Addr, typename Bar = BlockBarrier>
__device__ __forceinline__ void fft_run_pp(V (&v)[8], V *sm, const Addr &A, const Addr &B, int L, int j,
                                           bool act, bool in_regs, bool out_regs,
                                           const StageTw<typename ElemOf<V>::Tw> &tw, const Bar &bar = Bar()) {
    switch (L) {
        case 3: fft_run_pp_t<S, 3>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
        case 4: fft_run_pp_t<S, 4>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
        case 5: fft_run_pp_t<S, 5>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
        case 6: fft_run_pp_t<S, 6>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
        case 7: fft_run_pp_t<S, 7>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
        case 8: fft_run_pp_t<S, 8>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
        case 9: fft_run_pp_t<S, 9>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
        case 10: fft_run_pp_t<S, 10>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
        case 11: fft_run_pp_t<S, 11>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
        default: fft_run_pp_t<S, 12>(v, sm, A, B, j, act, in_regs, out_regs, tw, bar); break;
    }
}

// One transform of n = 2^L points (3 <= L <= 12), run by every thread of the block (it contains
// __syncthreads); threads with act == false only take part in the barriers.
//   in_regs:  stage 0 takes its inputs from v (slot m = element j + m n/8) instead of smem.
//   out_regs: the last stage leaves its outputs in v (slot m = element j + m n/8) and is not
//             stored; otherwise the result is in smem in natural order and v is undefined.
// When in_regs is set, a barrier is issued before the first store, so other threads may still
// be reading smem that this call overwrites.
template <int S, typename V, typename Addr, typename Bar = BlockBarrier>
__device__ __forceinline__ void fft_run(V (&v)[8], V *sm, const Addr &ad, int L, int j, bool act,
                                        bool in_regs, bool out_regs, const StageTw<typename ElemOf<V>::Tw> &tw,
                                        const Bar &bar = Bar()) {
    switch (L) {
        case 3: fft_run_t<S, 3>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
        case 4: fft_run_t<S, 4>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
        case 5: fft_run_t<S, 5>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
        case 6: fft_run_t<S, 6>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
        case 7: fft_run_t<S, 7>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
        case 8: fft_run_t<S, 8>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
        case 9: fft_run_t<S, 9>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
        case 10: fft_run_t<S, 10>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
        case 11: fft_run_t<S, 11>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
        default: fft_run_t<S, 12>(v, sm, ad, j, act, in_regs, out_regs, tw, bar); break;
    }
}

}  // namespace pfc
