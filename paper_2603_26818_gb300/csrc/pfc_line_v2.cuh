// Update pass (semi-implicit step) of FP32 plans whose line tiles have an even width W, with
// two adjacent kx columns per element (cf2, 16 bytes).
//
// The arithmetic is that of k_line<float, LINE_STEP> (pfc_pass.cuh): the forward Q-part of the
// y/z transforms of one C' and one X' tile, the update with the multipliers computed from k^2,
// the inverse Q-part. Here a thread carries the same 8 tile rows of two columns instead of one:
// every global and shared-memory access moves 16 bytes, the stage twiddles are loaded once for
// both columns, and a tile needs half the threads. With W = 2 (the 3D tiles of 64 x 64 rows) a
// warp-wide load then asks for 32 rows of 16 bytes instead of 16 rows twice, which is what keeps
// the load/store queue of the one-column form full.
//
// The kernel sees the tile through a geometry gv whose width is W / 2 elements (gv.W, gv.lW,
// gv.xs and gv.tsz in cf2 units); g is the plan's geometry (wavenumbers, strides of the grid).
#pragma once

#include "pfc_pass.cuh"

namespace pfc {

__device__ __forceinline__ cf2 ldcg2(const cf2 *p) {
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    return cf2{float2{v.x, v.y}, float2{v.z, v.w}};
}
__device__ __forceinline__ void stcg2(cf2 *p, cf2 v) {
    __stcg(reinterpret_cast<float4 *>(p), make_float4(v.a.x, v.a.y, v.b.x, v.b.y));
}

// psi_hat' = ca X - cb C for one column, with the multipliers of wavenumber (kx, ky, kz)
__device__ __forceinline__ float2 update1(const UpdR<float> &up, const OpR<float> &op, int kx, float fy2z2,
                                          bool zero, float2 x, float2 c) {
    const float fx = up.cx * (float)kx;
    const float k2 = fx * fx + fy2z2;
    const float lk = lin_symbol<float>(op, k2);
    const float inv = 1.0f / (1.0f + up.dt * k2 * lk);
    const float ca = inv * up.invQ, cb = up.dt * k2 * inv * up.inv_halfN;
    if (zero) return float2{0.0f, 0.0f};
    return float2{ca * x.x - cb * c.x, ca * x.y - cb * c.y};
}

// LY, LZ: as for k_line (compile-time transform lengths, 0 = the plan's)
template <int MAXT, int LY = 0, int LZ = 0>
__global__ void __launch_bounds__(MAXT, 1) k_line_v2(const Geom g, const Geom gv, const LineArgs<float> a) {
    using V = cf2;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const int cg = blockIdx.x, kp = blockIdx.y, field = blockIdx.z;
    V *T = sm;
    V *Cs = sm + gv.tsz;
    const LineMap mp = line_map(gv, threadIdx.x);
    const PadTileAddr ady = tile_y(gv, mp);
    const TileAddr adz = tile_z(gv, mp);
    const bool two_axes = LZ > 0 || (LY == 0 && gv.Qz > 1);
    int kpy, kpz;
    line_kp(g, kp, kpy, kpz);
    const int lsy = g.lPy + g.lRy, lsz = g.lPz + g.lRz;
    const size_t foff = (size_t)field * (size_t)(g.nhalf / 2);
    V vt[8];
    {
        // C' first, completely into shared memory (natural order)
        V vc[8];
        const V *C = reinterpret_cast<const V *>(a.c) + foff;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const float4 t = ld_last_use_l2(reinterpret_cast<const float4 *>(
                &C[xprime_index(gv, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)]));
            vc[m] = cf2{float2{t.x, t.y}, float2{t.z, t.w}};
        }
        line_yfft<-1, LY>(vc, Cs, ady, gv, mp.jy, true, false, a.st);
        if (two_axes) line_zfft<-1, LZ>(vc, Cs, adz, gv, mp.jz, false, false, a.st);
    }
    {
        const V *X = reinterpret_cast<const V *>(a.x) + foff;
#pragma unroll
        for (int m = 0; m < 8; ++m) vt[m] = ldcg2(&X[xprime_index(gv, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)]);
        line_yfft<-1, LY>(vt, T, ady, gv, mp.jy, true, !two_axes, a.st);
        if (two_axes) line_zfft<-1, LZ>(vt, T, adz, gv, mp.jz, false, true, a.st);
    }
    {
        OpR<float> op = a.up.op[field == 0 ? 0 : 1];
        if (a.rmem) op.r = a.rmem[field];
        const int kx0 = cg * g.W + 2 * mp.w;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const V c = Cs[tile_slot(mp, two_axes, ady, adz, m)];
            const int kqy = two_axes ? mp.yq : mp.jy + m * mp.ny8;
            const int kqz = two_axes ? mp.jz + m * mp.nz8 : 0;
            const int ky = kpy + (kqy << lsy), kz = kpz + (kqz << lsz);
            const int my = ky <= (g.ny >> 1) ? ky : ky - g.ny;
            const int mz = kz <= (g.nz >> 1) ? kz : kz - g.nz;
            const float fy = a.up.cy * (float)my, fz = a.up.cz * (float)mz;
            const float f2 = fy * fy + fz * fz;
            const bool k0 = ky == 0 && kz == 0;
            vt[m] = V{update1(a.up, op, kx0, f2, k0 && kx0 == 0, vt[m].a, c.a),
                      update1(a.up, op, kx0 + 1, f2, false, vt[m].b, c.b)};
        }
    }
    // inverse: the last forward axis first, from registers
    if (two_axes) {
        line_zfft<+1, LZ>(vt, T, adz, gv, mp.jz, true, false, a.st);
        line_yfft<+1, LY>(vt, T, ady, gv, mp.jy, false, true, a.st);
    } else {
        line_yfft<+1, LY>(vt, T, ady, gv, mp.jy, true, true, a.st);
    }
    V *Xo = reinterpret_cast<V *>(a.xout ? a.xout : a.x) + foff;
#pragma unroll
    for (int m = 0; m < 8; ++m) stcg2(&Xo[xprime_index(gv, kp, cg, mp.zq, mp.jy + m * mp.ny8, mp.w)], vt[m]);
}

// The element view of a plan geometry for k_line_v2 (W even).
__host__ __device__ inline Geom v2_view(const Geom &g) {
    Geom v = g;
    v.W = g.W / 2;
    v.lW = g.lW - 1;
    v.xs = g.xs / 2;
    v.tsz = (g.Q + g.Q / 8) * v.W;
    return v;
}

}  // namespace pfc
