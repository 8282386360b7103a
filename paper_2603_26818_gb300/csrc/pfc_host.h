// Host-side planning helpers shared by the plan API (pfc_api.cu) and the allocation-free
// entry point (pfc_noalloc.cu): FP64 twiddle generation, operator stability check and the
// tile planner. Header-only, host code.
#pragma once

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/pfc.h"
#include "pfc_launch.h"

namespace pfc {

// records the message returned by pfc_last_error() on this thread and passes s through
pfc_status set_error(pfc_status s, const std::string &msg);

inline int ilog2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}
inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// exp(-2 pi i t / n) in FP64 with the angle reduced to the first octant, so every entry is
// the correctly rounded cosine/sine of a small argument (or an exact symmetry of one).
inline void unit_root_fwd(int64_t t, int64_t n, double *re, double *im) {
    t %= n;
    const int64_t q = (4 * t) / n, rr = 4 * t - q * n;   // angle = (pi/2)(q + rr/n)
    double c, s;
    if (2 * rr <= n) {
        const double phi = (M_PI / 2) * (double)rr / (double)n;
        c = std::cos(phi);
        s = std::sin(phi);
    } else {
        const double phi = (M_PI / 2) * (double)(n - rr) / (double)n;
        c = std::sin(phi);
        s = std::cos(phi);
    }
    double cc, ss;   // rotate by q quarter turns
    switch (q) {
        case 0: cc = c; ss = s; break;
        case 1: cc = -s; ss = c; break;
        case 2: cc = -c; ss = -s; break;
        default: cc = s; ss = -c; break;
    }
    *re = cc;
    *im = -ss;
}

inline double lin_symbol_host(const pfc_op &op, double k2) {
    const double a = 1.0 - k2;
    if (op.kind == PFC_ONE_MODE) return op.r + a * a;
    const double b = op.q2 * op.q2 - k2;
    return op.r + a * a * (op.R1 + b * b);
}

// min over k^2 in [0, k2max] of the implicit matrix's smallest eigenvalue (sampled densely).
inline double min_implicit(const pfc_op *ops, int nfields, double alpha, double dt, double k2max) {
    double mn = 1e300;
    const int ns = 200000;
    for (int i = 0; i <= ns; ++i) {
        const double k2 = k2max * (double)i / ns;
        const double m11 = 1.0 + dt * k2 * lin_symbol_host(ops[0], k2);
        if (nfields == 1) {
            mn = std::min(mn, m11);
        } else {
            const double m22 = 1.0 + dt * k2 * lin_symbol_host(ops[1], k2);
            const double m12 = dt * k2 * alpha;
            const double tr = m11 + m22, det = m11 * m22 - m12 * m12;
            const double disc = std::sqrt(std::max(0.0, tr * tr / 4 - det));
            mn = std::min(mn, tr / 2 - disc);
        }
    }
    return mn;
}

inline OpDev to_dev(const pfc_op &o) { return OpDev{o.kind, o.r, o.R1, o.q2}; }

struct Tiles {
    Geom g;
    int nt_row, nt_line;
    size_t smem_row, smem_line;
    int row_cs = 0, nt_row_cs = 0;   // ROW_CUBE split over clusters of row_cs blocks (0: off)
    size_t smem_row_cs = 0;
};

// A tiling of a grid: the split of the y/z transforms between the passes (Py, Pz, and Ry, Rz
// for the middle pass of the three-pass schedule; Ry = Rz = 1 is the two-pass schedule), the
// line tile width W, and whether the psi^3 row pass may run on clusters where a cluster kernel
// exists for the grid (cluster = 0 keeps it on single blocks).
struct TileChoice {
    int Py = 0, Pz = 0, W = 0;
    int cluster = 1;
    int Ry = 1, Rz = 1;
};

// Which schedules tile_candidates may return: the two-pass ones, the three-pass ones, or the
// two-pass ones when the grid has any and the three-pass ones otherwise.
enum { SCHED_TWO = 2, SCHED_THREE = 3, SCHED_AUTO = 0 };

inline Geom grid_geom(int nx, int ny, int nz) {
    Geom g{};
    g.nx = nx; g.ny = ny; g.nz = nz; g.M = nx / 2;
    g.lnx = ilog2(nx); g.lny = ilog2(ny); g.lnz = ilog2(nz); g.lM = g.lnx - 1;
    g.ltab = std::max(g.lnx, std::max(g.lny, g.lnz));
    g.rs = (int)round_up(g.M + 1, 16);   // row_swz keeps each aligned block of 16
    g.Ry = g.Rz = g.R = 1;
    g.lRy = g.lRz = g.lR = 0;
    return g;
}

// Score of the tiling (Py, Pz, W) of grid g, or LONG_MIN when it breaks a kernel limit or does
// not fit shared memory:
//   row pass:  gpc groups of P = Py Pz rows of M + 1 elements (stride rounded up to 16)
//   line pass: ntile tiles of Q W complex values (Q = ny nz / P), W columns each, one padding
//              row after every 8 tile rows
// Preference: 32-byte tile rows (one DRAM sector per tile row), then line blocks of at most 512
// threads nearest to 2^lnt_target (several small blocks per SM interleave their load, transform
// and store phases), then the smallest P. At 4096^2 FP32, 32-byte rows in 256-thread blocks
// measured fastest, ahead of 64-byte rows or 512 threads. limit_w: tile rows of at most 64
// bytes (lifted for a width forced by PFC_TILE).
//
// Three-pass tilings (Ry Rz > 1; the middle pass takes the Ry x Rz-point sums, each at most 8):
// the line tile is Q = ny nz / (P R) long. They cost 9 sweeps a step instead of 5, so the planner
// takes them only for grids with no two-pass tiling; among them the same preferences apply,
// then the smallest R.
// max_w: the widest tile (16 for the per-pass launches; the persistent batch launch, whose line
// tiles must fill its fixed block size, allows up to 128 columns).
inline long tile_score(const Geom &g, int Py, int Pz, int W, size_t vb, int ntile, size_t smem_max,
                       bool limit_w, int lnt_target = 8, int Ry = 1, int Rz = 1, int max_w = 16) {
    const int max_threads = vb == 8 ? 1024 : 512;   // line pass blocks
    const int ny = g.ny, nz = g.nz;
    if (!is_pow2(Py) || Py > 8 || !is_pow2(Pz) || Pz > 8 || !is_pow2(W) || W > max_w) return LONG_MIN;
    if (!is_pow2(Ry) || Ry > 8 || !is_pow2(Rz) || Rz > 8 || (nz == 1 && Rz > 1)) return LONG_MIN;
    const int three = Ry * Rz > 1;
    if ((Py > 1 && ny / Py < 8) || ny % (Py * Ry)) return LONG_MIN;
    if ((nz == 1 && Pz > 1) || (Pz > 1 && nz / Pz < 8) || nz % (Pz * Rz)) return LONG_MIN;
    const int Qy = ny / (Py * Ry), Qz = nz / (Pz * Rz);
    if ((Qy < 8 && Qy != 1) || (Qz < 8 && Qz != 1)) return LONG_MIN;
    if (three && (Qy < 8 || (nz > 1 && Qz < 8))) return LONG_MIN;
    const int P = Py * Pz, Q = Qy * Qz;
    if ((size_t)P * ((size_t)g.rs * vb + vb) > smem_max) return LONG_MIN;
    if (limit_w && (size_t)W * vb > 64) return LONG_MIN;
    if (W > g.M + 1 && W > 1) return LONG_MIN;
    const int64_t QW = (int64_t)Q * W;
    if (QW < 8 || QW / 8 > max_threads) return LONG_MIN;
    const size_t tile = (size_t)(Q + Q / 8) * W;
    if ((size_t)ntile * tile * vb > smem_max) return LONG_MIN;
    const size_t wb = (size_t)W * vb;
    const long pref = wb == 32 ? 5 : wb == 64 ? 4 : wb == 16 ? 3 : wb == 128 ? 2 : 1;
    const int lnt = ilog2((int)(QW / 8));
    return pref * 1000000 - (QW / 8 > 512 ? 200000 : 0) - (long)std::abs(lnt - lnt_target) * 1000 -
           P - 100 * (Ry * Rz - 1);
}

// Line-block size the planner aims at (log2 threads). A grid alone: 256 threads. The members of
// a batch class (many grids stepped by the same launches, so parallelism comes from the members):
// 32 threads. On the 1024-domain ensemble ({64..512}^2, FP32) the autotuner's choices for the 16
// classes had line blocks of 8 to 64 threads, and timed 1.39x the step of the 256-thread rule.
inline int line_target(int instances) { return instances >= 8 ? 5 : 8; }

// Every valid tiling (Py, Pz, W) of the grid, best score first; ties keep the order Py, Pz
// ascending, W descending. force: fields > 0 are fixed (a forced W lifts the 64-byte limit).
// instances: as for plan_tiles_as (sets the line-block size aimed at).
// sched: SCHED_TWO, SCHED_THREE or SCHED_AUTO (a forced Ry or Rz > 1 selects SCHED_THREE).
inline std::vector<TileChoice> tile_candidates(int nx, int ny, int nz, size_t vb, int ntile, size_t smem_max,
                                               const TileChoice &force = TileChoice{}, int instances = 1,
                                               int sched = SCHED_AUTO) {
    const Geom g = grid_geom(nx, ny, nz);
    if (force.Ry > 1 || force.Rz > 1) sched = SCHED_THREE;
    auto collect = [&](bool three) {
        std::vector<std::pair<long, TileChoice>> all;
        for (int Py = 1; Py <= 8; Py *= 2) {
            if (force.Py > 0 && Py != force.Py) continue;
            for (int Pz = 1; Pz <= 8; Pz *= 2) {
                if (force.Pz > 0 && Pz != force.Pz) continue;
                for (int Ry = 1; Ry <= (three ? 8 : 1); Ry *= 2) {
                    if (three && force.Ry > 1 && Ry != force.Ry) continue;
                    for (int Rz = 1; Rz <= (three ? 8 : 1); Rz *= 2) {
                        if (three && force.Rz > 1 && Rz != force.Rz) continue;
                        if (three && Ry * Rz == 1) continue;
                        for (int W = 16; W >= 1; W /= 2) {
                            if (force.W > 0 && W != force.W) continue;
                            const long s = tile_score(g, Py, Pz, W, vb, ntile, smem_max, force.W <= 0,
                                                      line_target(instances), Ry, Rz);
                            if (s == LONG_MIN) continue;
                            TileChoice c;
                            c.Py = Py; c.Pz = Pz; c.W = W; c.cluster = force.cluster;
                            c.Ry = Ry; c.Rz = Rz;
                            all.push_back({s, c});
                        }
                    }
                }
            }
        }
        std::stable_sort(all.begin(), all.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
        std::vector<TileChoice> out;
        for (auto &e : all) out.push_back(e.second);
        return out;
    };
    if (sched == SCHED_THREE) return collect(true);
    std::vector<TileChoice> two = collect(false);
    if (sched == SCHED_TWO || !two.empty()) return two;
    return collect(true);
}

// The plan of one tiling (Py, Pz, W all set): derived sizes, row groups per CTA, block sizes,
// shared memory, and the clustered psi^3 row pass where one exists for the grid.
// instances: grids of this shape stepped by the same launches (the members of a batch class)
inline bool plan_tiles_as(Tiles &t, const TileChoice &c, int nx, int ny, int nz, size_t vb, int ntile,
                          size_t smem_max, int instances = 1, int max_w = 16) {
    Geom g = grid_geom(nx, ny, nz);
    const int Ry = std::max(c.Ry, 1), Rz = std::max(c.Rz, 1);
    if (tile_score(g, c.Py, c.Pz, c.W, vb, ntile, smem_max, false, 8, Ry, Rz, max_w) == LONG_MIN) return false;
    // row blocks of at most 512 threads: two blocks (64 registers a thread) fit an SM, so one
    // block's memory phases overlap the other's transforms (256^3 FP32 row pass 212 -> 162 us
    // against 1024-thread blocks)
    const int max_row_threads = 512;
    const size_t row_bytes = (size_t)g.rs * vb;
    g.Py = c.Py; g.Pz = c.Pz; g.Ry = Ry; g.Rz = Rz;
    g.Qy = ny / (c.Py * Ry); g.Qz = nz / (c.Pz * Rz); g.W = c.W;
    g.lPy = ilog2(g.Py); g.lPz = ilog2(g.Pz); g.lQy = ilog2(g.Qy); g.lQz = ilog2(g.Qz);
    g.lRy = ilog2(Ry); g.lRz = ilog2(Rz);
    g.P = g.Py * g.Pz; g.Q = g.Qy * g.Qz; g.lQ = ilog2(g.Q);
    g.R = Ry * Rz; g.lR = ilog2(g.R); g.QR = g.R * g.Q;
    g.lW = ilog2(g.W);
    g.tsz = (g.Q + g.Q / 8) * g.W;
    g.xs = (int)round_up(g.M + 1, std::max(g.W, 2));
    g.ncg = g.xs / g.W;
    // row groups per CTA: enough rows for >= 256 threads, within smem and dividing Q, while the
    // row pass keeps at least one block per SM (a small grid alone has few groups)
    const int Tr = g.M / 8;
    int gpc = 1;
    while (gpc * 2 <= g.QR && (size_t)(gpc * 2) * g.P * (row_bytes + vb) <= smem_max &&
           gpc * g.P * Tr < 256 && (int64_t)g.QR * instances / (gpc * 2) >= 152)
        gpc *= 2;
    g.gpc = gpc;
    g.nreal = (int64_t)nx * ny * nz;
    g.nhalf = (int64_t)g.P * g.QR * g.xs;
    g.nstd = (int64_t)ny * nz * (g.M + 1);
    const int rows = gpc * g.P;
    t.nt_row = std::min(max_row_threads, std::max(Tr, rows * Tr));
    if (t.nt_row < 32) t.nt_row = std::max(Tr, 32 / Tr * Tr);
    // rows, the split twiddles of the block's rows, then the saved real parts of the kx = 0
    // and nx/2 columns (2 gpc P reals)
    t.smem_row = (size_t)round_up((int64_t)rows * (row_bytes + vb) + 2 * gpc * g.P * (vb / 2), 16);
    t.g = g;
    const int64_t QW = (int64_t)g.Q * g.W;
    t.nt_line = (int)(QW / 8);
    t.smem_line = (size_t)ntile * (size_t)g.tsz * vb;
    // A group of FP32 rows too large for two blocks per SM is split over a cluster of two blocks:
    // 2D (Pz = 1, Py = 8) four rows per block, 3D (Pz = 8) four z_p rows of Py each
    // (PFC_ROW_CLUSTER=0 turns this off).
    t.row_cs = 0;
    t.nt_row_cs = 0;
    t.smem_row_cs = 0;
    const char *rc = std::getenv("PFC_ROW_CLUSTER");
    const bool rc_on = c.cluster != 0 && !(rc && rc[0] == '0');
    // (the cluster kernels are compiled for these row lengths only: M = 2048 in 2D, 256, 512 and
    // 1024 in 3D)
    if (rc_on && vb == 8 && g.Pz == 1 && g.Py == 8 && gpc == 1 && 2 * (size_t)rows * row_bytes > smem_max &&
        g.M == 2048) {
        // four rows and one scratch row per row in flight (two) for ping-pong transforms
        t.row_cs = 2;
        t.nt_row_cs = 2 * Tr;
        t.smem_row_cs = (size_t)round_up((int64_t)(4 + 2) * row_bytes + 8 * vb, 16);
    } else if (rc_on && vb == 8 && g.Pz == 8 && gpc == 1 && 2 * (size_t)rows * row_bytes > smem_max &&
               (g.M == 256 || g.M == 512 || g.M == 1024)) {
        // 3D: the group's 8 Py rows split by z_p halves over a cluster of two blocks
        t.row_cs = 2;
        t.nt_row_cs = std::min(512, 4 * g.Py * Tr);
        t.smem_row_cs = (size_t)round_up((int64_t)4 * g.Py * row_bytes + (int64_t)g.P * vb + g.P * vb +
                                             2 * (int64_t)g.P * vb, 16);
    }
    return true;
}

// The launch configuration of a tiling on a stream (the clustered row pass included).
inline LaunchCfg launch_cfg(const Tiles &t, cudaStream_t stream) {
    LaunchCfg c{t.g, t.nt_row, t.nt_line, t.smem_row, t.smem_line, stream};
    c.row_cs = t.row_cs;
    c.nt_row_cs = t.nt_row_cs;
    c.smem_row_cs = t.smem_row_cs;
    return c;
}

// The planner's tiling: the best-scoring candidate. PFC_TILE="Py,Pz,W" forces a tiling and
// "Py,Pz,W,Ry,Rz" a three-pass one (used to compare tilings and to test the three-pass
// schedule on small grids; rejected if it does not fit).
inline bool plan_tiles(Tiles &t, int nx, int ny, int nz, size_t vb, int ntile, size_t smem_max,
                       int instances = 1) {
    TileChoice force;
    if (const char *env = std::getenv("PFC_TILE"))
        std::sscanf(env, "%d,%d,%d,%d,%d", &force.Py, &force.Pz, &force.W, &force.Ry, &force.Rz);
    const std::vector<TileChoice> c = tile_candidates(nx, ny, nz, vb, ntile, smem_max, force, instances);
    return !c.empty() && plan_tiles_as(t, c[0], nx, ny, nz, vb, ntile, smem_max, instances);
}

// Autotune cache file: one JSON object per line,
//   {"key": "<nz>x<ny>x<nx> prec<p> fields<f> <device>", "Py": .., "Pz": .., "W": .., "cluster": ..,
//    "Ry": .., "Rz": .., "ms_per_step": ..}
// (entries without Ry and Rz are two-pass tilings). Lookup returns the last entry for the key;
// lines in any other form are skipped.
inline bool tune_cache_lookup(const char *path, const std::string &key, TileChoice &c, double &ms) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        char k[512];
        TileChoice t;
        double m = 0;
        const bool full = std::sscanf(line, "{\"key\": \"%511[^\"]\", \"Py\": %d, \"Pz\": %d, \"W\": %d, "
                                            "\"cluster\": %d, \"Ry\": %d, \"Rz\": %d, \"ms_per_step\": %lf}",
                                      k, &t.Py, &t.Pz, &t.W, &t.cluster, &t.Ry, &t.Rz, &m) == 8;
        bool ok = full;
        if (!full) {
            t = TileChoice{};
            ok = std::sscanf(line, "{\"key\": \"%511[^\"]\", \"Py\": %d, \"Pz\": %d, \"W\": %d, \"cluster\": %d, "
                                   "\"ms_per_step\": %lf}", k, &t.Py, &t.Pz, &t.W, &t.cluster, &m) == 6;
        }
        if (ok && key == k) {
            c = t;
            ms = m;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

inline void tune_cache_store(const char *path, const std::string &key, const TileChoice &c, double ms) {
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": \"%s\", \"Py\": %d, \"Pz\": %d, \"W\": %d, \"cluster\": %d, \"Ry\": %d, "
                    "\"Rz\": %d, \"ms_per_step\": %.6f}\n",
                 key.c_str(), c.Py, c.Pz, c.W, c.cluster, std::max(c.Ry, 1), std::max(c.Rz, 1), ms);
    std::fclose(f);
}

// A kernel's shared-memory limit is an attribute of the function, shared by every plan of the
// process: plans (and batches, and the allocation-free step) only ever raise it to the largest
// size any of them launches with, so a plan created later with smaller tiles cannot make an
// earlier plan's launches exceed the limit.
template <typename R> cudaError_t raise_smem_attrs(const LaunchCfg &c) {
    static std::mutex mu;
    static size_t row = 0, line = 0, cs2 = 0, cs3 = 0;
    std::lock_guard<std::mutex> lock(mu);
    LaunchCfg m = c;
    m.smem_row = row = std::max(row, c.smem_row);
    m.smem_line = line = std::max(line, c.smem_line);
    if (c.row_cs == 2) {
        size_t &cs = c.g.Pz == 1 ? cs2 : cs3;
        m.smem_row_cs = cs = std::max(cs, c.smem_row_cs);
    }
    return set_smem_attrs<R>(m);
}

// Per-stage twiddle tables (see StageTw): entries for R = 8, 4, 2 and Ns = 8, 64, 512.
constexpr int STW8 = 4672, STW4 = 2336, STW2 = 1168;
constexpr int STW_TOTAL = STW8 + STW4 + STW2;

// FP64 values (re, im interleaved) of the full table exp(-2 pi i t / ntab), t < ntab, and of
// the per-stage tables [r][k] = W_{R Ns}^{r k}.
inline void twiddle_tables(int64_t ntab, std::vector<double> &full, std::vector<double> &stage) {
    full.assign(2 * ntab, 0.0);
    for (int64_t i = 0; i < ntab; ++i) unit_root_fwd(i, ntab, &full[2 * i], &full[2 * i + 1]);
    stage.assign(2 * STW_TOTAL, 0.0);
    int64_t o = 0;
    for (int R : {8, 4, 2})
        for (int64_t ns = 8; ns <= 512; ns *= 8)
            for (int r = 0; r < R; ++r)
                for (int64_t k = 0; k < ns; ++k, ++o) unit_root_fwd(r * k, R * ns, &stage[2 * o], &stage[2 * o + 1]);
}

}  // namespace pfc
