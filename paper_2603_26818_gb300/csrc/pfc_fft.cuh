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
// Twiddles come from one table tw[i] = exp(-2 pi i * i / 2^ltab), generated on the host in FP64
// (and rounded once for the FP32 path). The inverse transform uses the conjugate.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pfc {

template <typename R> struct VT;
template <> struct VT<float> { using V = float2; };
template <> struct VT<double> { using V = double2; };

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
    using R = decltype(v[0].x);
    const R h = (R)0.70710678118654752440084436210484903928;
    V a0 = cadd(v[0], v[4]), a4 = csub(v[0], v[4]);
    V a1 = cadd(v[1], v[5]), t5 = csub(v[1], v[5]);
    V a2 = cadd(v[2], v[6]), a6 = cmul_i<S>(csub(v[2], v[6]));
    V a3 = cadd(v[3], v[7]), t7 = csub(v[3], v[7]);
    // t5 * W8^1 = (x - S y, y + S x) / sqrt2 ; t7 * W8^3 = (-x - S y, S x - y) / sqrt2
    V a5 = V{(t5.x - S * t5.y) * h, (t5.y + S * t5.x) * h};
    V a7 = V{(-t7.x - S * t7.y) * h, (S * t7.x - t7.y) * h};
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
// Shared-memory addressing of one transform instance: element i lives at addr(i).
// ------------------------------------------------------------------------------------------
// A row of a row buffer: one padding slot after every 8 elements (bank spreading).
__host__ __device__ __forceinline__ int row_pad(int i) { return i + (i >> 3); }

struct RowAddr {
    int base;
    __device__ __forceinline__ int operator()(int i) const { return base + row_pad(i); }
};

// A column of an interleaved tile: flat e = off + i * stride, padded by e >> pshift.
struct TileAddr {
    int off, stride, pshift;
    __device__ __forceinline__ int operator()(int i) const {
        int e = off + i * stride;
        return e + (e >> pshift);
    }
};

// ------------------------------------------------------------------------------------------
// Stockham stage machinery. Stage s has radix R = 2^lR and Ns = 2^lNs (the product of the
// previous radices). Butterfly b has k = b mod Ns; it reads b + r n/R, multiplies input r by
// W_{Ns R}^{r k}, runs a DFT_R and writes output r to (b - k) R + k + r Ns.
// Thread j owns butterflies b = j + u n/8 (u < 8/R): its inputs are always j + m n/8 with
// slot m = u + (8/R) r.
// ------------------------------------------------------------------------------------------
template <typename V, typename Addr>
__device__ __forceinline__ void load8(V (&v)[8], const V *sm, const Addr &ad, int j, int n8) {
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = sm[ad(j + m * n8)];
}

template <int S, typename V>
__device__ __forceinline__ void stage_exec(V (&v)[8], int lR, int lNs, int j, int n8,
                                           const V *__restrict__ tw, int ltab) {
    const int Ns = 1 << lNs;
    const int sh = ltab - lNs - lR;  // W_{Ns R}^{x} = tw[x << sh]
    if (lR == 3) {
        const int k = j & (Ns - 1);
        if (lNs > 0) {
#pragma unroll
            for (int r = 1; r < 8; ++r) v[r] = ctw<S>(v[r], __ldg(&tw[(r * k) << sh]));
        }
        dft8<S>(v);
    } else if (lR == 2) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int k = (j + u * n8) & (Ns - 1);
            V c0 = v[u], c1 = v[u + 2], c2 = v[u + 4], c3 = v[u + 6];
            if (lNs > 0) {
                c1 = ctw<S>(c1, __ldg(&tw[k << sh]));
                c2 = ctw<S>(c2, __ldg(&tw[(2 * k) << sh]));
                c3 = ctw<S>(c3, __ldg(&tw[(3 * k) << sh]));
            }
            dft4<S>(c0, c1, c2, c3);
            v[u] = c0; v[u + 2] = c1; v[u + 4] = c2; v[u + 6] = c3;
        }
    } else if (lR == 1) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = (j + u * n8) & (Ns - 1);
            V c0 = v[u], c1 = v[u + 4];
            if (lNs > 0) c1 = ctw<S>(c1, __ldg(&tw[k << sh]));
            dft2<S>(c0, c1);
            v[u] = c0; v[u + 4] = c1;
        }
    }
}

template <typename V, typename Addr>
__device__ __forceinline__ void stage_store(const V (&v)[8], V *sm, const Addr &ad, int lR, int lNs,
                                            int j, int n8) {
    const int Ns = 1 << lNs;
    if (lR == 3) {
        const int k = j & (Ns - 1);
        const int o = ((j - k) << 3) + k;
#pragma unroll
        for (int r = 0; r < 8; ++r) sm[ad(o + r * Ns)] = v[r];
    } else if (lR == 2) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int b = j + u * n8, k = b & (Ns - 1);
            const int o = ((b - k) << 2) + k;
#pragma unroll
            for (int r = 0; r < 4; ++r) sm[ad(o + r * Ns)] = v[u + 2 * r];
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = j + u * n8, k = b & (Ns - 1);
            const int o = ((b - k) << 1) + k;
            sm[ad(o)] = v[u];
            sm[ad(o + Ns)] = v[u + 4];
        }
    }
}

// One transform of n = 2^L points (L >= 3), run by every thread of the block (it contains
// __syncthreads); threads with act == false only take part in the barriers.
//   in_regs:  stage 0 takes its inputs from v (slot m = element j + m n/8) instead of smem.
//   out_regs: the last stage leaves its outputs in v (slot m = element j + m n/8) and is not
//             stored; otherwise the result is in smem in natural order and v is undefined.
// When in_regs is set, the caller must not have other threads still reading smem that this
// call overwrites before its first barrier (a barrier is issued before the first store).
template <int S, typename V, typename Addr>
__device__ __forceinline__ void fft_run(V (&v)[8], V *sm, const Addr &ad, int L, int j, bool act,
                                        bool in_regs, bool out_regs, const V *__restrict__ tw,
                                        int ltab) {
    const int n8 = 1 << (L - 3);
    const int nst = (L + 2) / 3;
    const int nfull = L / 3;
    int lNs = 0;
    for (int s = 0; s < nst; ++s) {
        const int lR = (s < nfull) ? 3 : (L - 3 * nfull);
        if (act && !(s == 0 && in_regs)) load8(v, sm, ad, j, n8);
        if (act) stage_exec<S>(v, lR, lNs, j, n8, tw, ltab);
        if (s == nst - 1 && out_regs) break;
        __syncthreads();
        if (act) stage_store(v, sm, ad, lR, lNs, j, n8);
        __syncthreads();
        lNs += lR;
    }
}

// NJ transform instances (or NJ butterfly groups of one instance) per thread, all advanced
// stage by stage between the same barriers. Slot u uses addressing ad[u], thread index j[u]
// and is idle when act[u] is false. Results end in smem in natural order.
template <int S, int NJ, typename V, typename Addr>
__device__ __forceinline__ void fft_run_multi(V *sm, const Addr (&ad)[NJ], int L, const int (&j)[NJ],
                                              const bool (&act)[NJ], const V *__restrict__ tw,
                                              int ltab) {
    const int n8 = 1 << (L - 3);
    const int nst = (L + 2) / 3;
    const int nfull = L / 3;
    int lNs = 0;
    V v[NJ][8];
    for (int s = 0; s < nst; ++s) {
        const int lR = (s < nfull) ? 3 : (L - 3 * nfull);
#pragma unroll
        for (int u = 0; u < NJ; ++u) {
            if (act[u]) {
                load8(v[u], sm, ad[u], j[u], n8);
                stage_exec<S>(v[u], lR, lNs, j[u], n8, tw, ltab);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NJ; ++u)
            if (act[u]) stage_store(v[u], sm, ad[u], lR, lNs, j[u], n8);
        __syncthreads();
        lNs += lR;
    }
}

}  // namespace pfc
