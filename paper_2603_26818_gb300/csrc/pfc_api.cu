// Host side of libpfc.so: plans, tile planning, launches, CUDA graphs and the C ABI of pfc.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "../../include/pfc.h"
#include "pfc_host.h"

using namespace pfc;

namespace {

thread_local std::string g_last_error;

pfc_status fail(pfc_status s, const std::string &msg) { return set_error(s, msg); }

#define PFC_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

}  // namespace

struct pfc_plan {
    int ndim = 0;
    int nx = 0, ny = 0, nz = 0;
    double dx = 0, dt = 0;
    pfc_op ops[2] = {};
    int nfields = 1;
    double alpha = 0;
    int prec = PFC_FP64;
    cudaStream_t stream = nullptr;
    Tiles t{};
    void *X = nullptr, *C = nullptr, *tw = nullptr, *stw = nullptr;
    void *Y = nullptr;            // three-pass plans: the state in the row-pass form (P-part only)
    int scheme = PFC_SEMI_IMPLICIT;   // time integrator (pfc_set_integrator)
    double stab = 0.0;            // its stabilisation constant S
    void *X2 = nullptr, *C2 = nullptr;   // the second time level of the second-order scheme
    // mixed-radix plans (extents of 2, 3, 5, 7 that are not all powers of two): X holds S, Y the
    // row-space work array, C the cube's transform, E the projection columns
    bool mixed = false;
    MrGeom mg{};
    void *mtw = nullptr, *mtwx = nullptr, *E = nullptr;
    int mr_rows = 1;              // x pass: rows (warps) a block
    int mr_W[3] = {1, 1, 1};      // column passes: columns a block, per axis
    int mr_G = 2;                 // column passes: warps a column (capped per launch)
    bool mr_even_first = false;   // radix order of every axis: 8, 4, 2 before 7, 5, 3
    size_t mtw_cap = 0;           // bytes of the stage-twiddle table
    size_t mr_smem_col = 0;       // shared memory of the column passes' largest launch
    int mr_wE[3] = {1, 1, 1};     // the same for the two projection columns
    void *A = nullptr;            // third half spectrum, allocated by the first adjoint call
    double *d_adjpart = nullptr;  // adjoint line-pass partial sums (one per block)
    double *d_mean = nullptr, *d_part = nullptr, *d_out = nullptr;
    int *d_status = nullptr;
    size_t scratch = 0;
    size_t half_cap = 0;          // bytes allocated for each of X and C
    size_t y_cap = 0;             // bytes allocated for Y
    size_t lv_cap = 0;            // bytes allocated for each of X2 and C2
    size_t adj_bytes = 0;         // bytes of A and d_adjpart
    int ntile = 2;                // line-pass tiles (3 for a two-field plan)
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    bool destroyed = false;
};

namespace {

constexpr int GRAPH_CHUNK = 16;

size_t smem_optin();   // the device's opt-in shared memory per block (0 when the query fails)

size_t vbytes(const pfc_plan *p) { return p->prec == PFC_FP64 ? 16 : 8; }


template <typename R> StageTw<typename VT<R>::V> stage_tw(const pfc_plan *p) {
    using V = typename VT<R>::V;
    const V *b = reinterpret_cast<const V *>(p->stw);
    return StageTw<V>{b, b + STW8, b + STW8 + STW4};
}

template <typename R> RowArgs<R> row_args(const pfc_plan *p) {
    RowArgs<R> a{};
    a.tw = reinterpret_cast<const typename VT<R>::V *>(p->tw);
    a.st = stage_tw<R>(p);
    a.scale = (R)1;
    return a;
}

template <typename R> LineArgs<R> line_args(const pfc_plan *p) {
    LineArgs<R> a{};
    a.st = stage_tw<R>(p);
    a.scale = (R)1;
    const Geom &g = p->t.g;
    const double two_pi = 6.28318530717958647692528676655900576839;
    a.up.dt = (R)p->dt;
    a.up.cx = (R)(two_pi / (g.nx * p->dx));
    a.up.cy = (R)(two_pi / (g.ny * p->dx));
    a.up.cz = (R)(two_pi / (g.nz * p->dx));
    a.up.invQ = (R)(1.0 / g.Q);
    a.up.inv_halfN = (R)(2.0 / (double)g.nreal);
    for (int f = 0; f < 2; ++f) {
        const pfc_op &o = p->ops[f < p->nfields ? f : 0];
        a.up.op[f] = OpR<R>{o.kind, (R)o.r, (R)o.R1, (R)(o.q2 * o.q2)};
    }
    return a;
}

LaunchCfg cfg(const pfc_plan *p) { return launch_cfg(p->t, p->stream); }

template <typename R> void launch_row_m(const pfc_plan *p, int mode, const RowArgs<R> &a, int nf) {
    launch_row<R>(cfg(p), mode, a, nf);
}
// Middle pass of a three-pass plan: dir -1 forward (row-pass form -> line form), +1 inverse
// (unnormalised); edges: only the kx = 0 and nx/2 columns.
template <typename R>
void launch_mid_m(const pfc_plan *p, int dir, const void *in, void *out, double scale, bool edges) {
    MidArgs<R> a{};
    a.in = in;
    a.out = out;
    a.scale = (R)scale;
    a.tw = reinterpret_cast<const typename VT<R>::V *>(p->tw);
    a.edges = edges ? 1 : 0;
    launch_mid<R>(cfg(p), dir, a);
}
bool three_pass(const pfc_plan *p) { return p->t.g.R > 1; }

// ------------------------------------------------------------------------------------------
// Mixed-radix plans (pfc_mixed.cuh): one pass per axis
// ------------------------------------------------------------------------------------------
template <typename R> void launch_means(pfc_plan *p, const void *state);

template <typename R> MrArgs<R> mr_args(const pfc_plan *p) {
    MrArgs<R> a{};
    a.tw = reinterpret_cast<const typename VT<R>::V *>(p->mtw);
    a.twx = reinterpret_cast<const typename VT<R>::V *>(p->mtwx);
    a.scale = (R)1;
    const double two_pi = 6.28318530717958647692528676655900576839;
    const MrGeom &g = p->mg;
    a.up.dt = (R)p->dt;
    a.up.cx = (R)(two_pi / (g.nx * p->dx));
    a.up.cy = (R)(two_pi / (g.ny * p->dx));
    a.up.cz = (R)(two_pi / (g.nz * p->dx));
    a.up.inv_halfN = (R)(1.0 / ((double)g.ny * g.nz * g.M));
    a.up.op[0] = OpR<R>{p->ops[0].kind, (R)p->ops[0].r, (R)p->ops[0].R1, (R)(p->ops[0].q2 * p->ops[0].q2)};
    return a;
}
// column pass along axis (1 y, 2 z) of a half spectrum of M + 1 columns
template <typename R>
void mr_col(const pfc_plan *p, int mode, int axis, const void *in, void *out, double scale) {
    MrArgs<R> a = mr_args<R>(p);
    a.scale = (R)scale;
    launch_mr_col<R>(p->stream, mode, p->mg, a, axis, p->mr_W[axis], p->mg.M + 1, in, out,
                     mr_col_group(p->mr_W[axis], p->mr_G));
}
template <typename R>
void mr_row(const pfc_plan *p, int mode, const void *in, void *out, const double *mean, double scale) {
    MrArgs<R> a = mr_args<R>(p);
    a.scale = (R)scale;
    a.mean = mean;
    launch_mr_row<R>(p->stream, mode, p->mg, a, in, out, p->E, p->mr_rows);
}
// forward y (and z) of a half spectrum in place, the last pass scaled
template <typename R> void mr_fwd_yz(const pfc_plan *p, void *x, double scale) {
    const bool z = p->mg.nz > 1;
    mr_col<R>(p, MR_COL_FWD, 1, x, x, z ? 1.0 : scale);
    if (z) mr_col<R>(p, MR_COL_FWD, 2, x, x, scale);
}
// inverse z (and y) from in into out (unnormalised)
template <typename R> void mr_inv_yz(const pfc_plan *p, const void *in, void *out) {
    if (p->mg.nz > 1) {
        mr_col<R>(p, MR_COL_INV, 2, in, out, 1.0);
        mr_col<R>(p, MR_COL_INV, 1, out, out, 1.0);
    } else {
        mr_col<R>(p, MR_COL_INV, 1, in, out, 1.0);
    }
}
// The mixed-radix step sequence; mk(kind) is called before each group of launches (the kinds of
// pfc_profile_steps: 0 x pass, 1 y/z passes, 2 entry, 3 exit, 4 projection columns).
template <typename R, typename Mark>
void mixed_enqueue(pfc_plan *p, void *state, int64_t nsteps, Mark &&mk) {
    const MrGeom &g = p->mg;
    const double sc = 1.0 / ((double)g.ny * g.nz * g.M);
    mk(2);
    launch_means<R>(p, state);
    // entry: S = F(psi - mean) / (ny nz M)
    mr_row<R>(p, MR_ROW_FWD, state, p->X, p->d_mean, 1.0);
    mr_fwd_yz<R>(p, p->X, sc);
    // the projection columns E as a half spectrum of two columns
    MrGeom ge = g;
    ge.xs = 2;
    MrArgs<R> ea = mr_args<R>(p);
    for (int64_t s = 0; s < nsteps; ++s) {
        mk(1);
        mr_inv_yz<R>(p, p->X, p->Y);
        mk(0);
        mr_row<R>(p, MR_ROW_CUBE, p->Y, p->C, p->d_mean, 1.0);
        mk(1);
        if (g.nz > 1) mr_col<R>(p, MR_COL_FWD, 1, p->C, p->C, 1.0);
        mk(4);
        // Hermitian projection of the kx = 0 and nx/2 columns: F_yz of their real parts / (ny nz)
        ea.scale = (R)(g.nz > 1 ? 1.0 : 1.0 / g.ny);
        launch_mr_col<R>(p->stream, MR_COL_FWD, ge, ea, 1, p->mr_wE[1], 2, p->E, p->E, mr_col_group(p->mr_wE[1], p->mr_G));
        if (g.nz > 1) {
            ea.scale = (R)(1.0 / ((double)g.ny * g.nz));
            launch_mr_col<R>(p->stream, MR_COL_FWD, ge, ea, 2, p->mr_wE[2], 2, p->E, p->E,
                             mr_col_group(p->mr_wE[2], p->mr_G));
        }
        launch_mr_edges<R>(p->stream, g, p->E, p->X, 1.0);
        mk(1);
        mr_col<R>(p, MR_COL_UPDATE, g.nz > 1 ? 2 : 1, p->C, p->X, 1.0);
    }
    // exit
    mk(3);
    mr_inv_yz<R>(p, p->X, p->Y);
    mr_row<R>(p, MR_ROW_INV, p->Y, state, p->d_mean, 1.0);
}
// launches of mixed_enqueue
int64_t mixed_launches(const pfc_plan *p, int64_t nsteps) {
    const bool z = p->mg.nz > 1;
    return 3 + (z ? 2 : 1) + nsteps * (z ? 8 : 5) + (z ? 3 : 2);
}
template <typename R> pfc_status mixed_step_impl(pfc_plan *p, void *state, int64_t nsteps) {
    mixed_enqueue<R>(p, state, nsteps, [](int) {});
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}
template <typename R> pfc_status mixed_r2c_impl(pfc_plan *p, const void *in, void *out) {
    mr_row<R>(p, MR_ROW_FWD, in, out, nullptr, 1.0);
    mr_fwd_yz<R>(p, out, 1.0);
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}
template <typename R> pfc_status mixed_c2r_impl(pfc_plan *p, const void *in, void *out) {
    mr_inv_yz<R>(p, in, p->Y);
    mr_row<R>(p, MR_ROW_INV, p->Y, out, nullptr, 1.0 / ((double)p->mg.ny * p->mg.nz * p->mg.M));
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}

// radices of n, the odd ones first (7, 5, 3), then 8, 4, 2 (even_first: the other way round);
// false when n has another prime factor
bool mr_factor(int n, std::vector<int> &rad, bool even_first = false) {
    rad.clear();
    std::vector<int> odd, even;
    for (int r : {7, 5, 3})
        while (n % r == 0) { odd.push_back(r); n /= r; }
    while (n % 8 == 0) { even.push_back(8); n /= 8; }
    if (n % 4 == 0) { even.push_back(4); n /= 4; }
    if (n % 2 == 0) { even.push_back(2); n /= 2; }
    const std::vector<int> &a = even_first ? even : odd, &b = even_first ? odd : even;
    rad.insert(rad.end(), a.begin(), a.end());
    rad.insert(rad.end(), b.begin(), b.end());
    return n == 1 && (int)rad.size() <= MR_MAXST;
}

// The stage radices and twiddle offsets of the three axes of g (lengths already set) in the
// given radix order, and the stage twiddles W_{r Ns}^{m k} they index (FP64, re/im pairs).
void mr_axes(MrGeom &g, bool even_first, std::vector<double> &tw) {
    tw.clear();
    for (int a = 0; a < 3; ++a) {
        MrAxis &ax = g.ax[a];
        std::vector<int> rad;
        if (ax.n > 1) mr_factor(ax.n, rad, even_first);
        ax.nst = (int)rad.size();
        int Ns = 1;
        for (int s = 0; s < ax.nst; ++s) {
            ax.radix[s] = rad[s];
            ax.ns[s] = Ns;
            ax.twoff[s] = (int)(tw.size() / 2);
            for (int m = 0; m < rad[s]; ++m)
                for (int k = 0; k < Ns; ++k) {
                    double re, im;
                    unit_root_fwd((int64_t)m * k, (int64_t)rad[s] * Ns, &re, &im);
                    tw.push_back(re);
                    tw.push_back(im);
                }
            Ns *= rad[s];
        }
    }
}
bool mr_extent_ok(int64_t n) {
    std::vector<int> r;
    return n >= 8 && n <= 4096 && mr_factor((int)n, r);
}
template <typename R> void launch_line_m(const pfc_plan *p, int mode, const LineArgs<R> &a, int nf) {
    launch_line<R>(cfg(p), mode, a, nf);
}

// Mean of each field of a real array into d_mean[f] (FP64).
template <typename R> void launch_means(pfc_plan *p, const void *state) {
    const Geom &g = p->t.g;
    for (int f = 0; f < p->nfields; ++f) {
        const R *x = reinterpret_cast<const R *>(state) + (size_t)f * g.nreal;
        launch_reduce_real<R>(p->stream, RED_SUM, x, nullptr, g.nreal, p->d_part, p->d_status);
        launch_finish(p->stream, p->d_part, RED_BLOCKS, 1.0 / (double)g.nreal, p->d_mean + f);
    }
}

// The buffers of step s (0-based within one pfc_step call). The second-order scheme carries two
// time levels, X'/C' of step s - 1 and s: step s reads level s from lv[s % 2] and level s - 1 from
// lv[(s + 1) % 2], and writes level s + 1 over level s - 1. The other schemes work in place.
struct StepBufs {
    void *x, *c, *xprev, *cprev, *xout;
};
StepBufs step_bufs(const pfc_plan *p, int64_t s) {
    if (p->scheme != PFC_SBDF2) return StepBufs{p->X, p->C, nullptr, nullptr, p->X};
    void *xs[2] = {p->X, p->X2}, *cs[2] = {p->C, p->C2};
    const int cur = (int)(s & 1), oth = 1 - cur;
    return StepBufs{xs[cur], cs[cur], s > 0 ? xs[oth] : nullptr, s > 0 ? cs[oth] : nullptr, xs[oth]};
}
// where the carried state is after nsteps steps of a call
void *final_state(const pfc_plan *p, int64_t nsteps) {
    return p->scheme == PFC_SBDF2 && (nsteps & 1) ? p->X2 : p->X;
}

// The line pass of one step: per field, or the coupled 2x2 solve for a two-field plan; the
// alternative integrators (single field) on the LINE_SCHEME pass.
template <typename R> void launch_update(pfc_plan *p, const StepBufs &b) {
    LineArgs<R> la = line_args<R>(p);
    if (p->nfields == 2) {
        using V = typename VT<R>::V;
        const Geom &g = p->t.g;
        Step2Args<R> a2{};
        a2.x0 = p->X;
        a2.x1 = reinterpret_cast<V *>(p->X) + g.nhalf;
        a2.c0 = p->C;
        a2.c1 = reinterpret_cast<const V *>(p->C) + g.nhalf;
        a2.alpha = (R)p->alpha;
        a2.up = la.up;
        a2.st = la.st;
        launch_line_step2<R>(cfg(p), a2);
        return;
    }
    la.x = b.x;
    la.c = b.c;
    if (p->scheme == PFC_SEMI_IMPLICIT) {
        launch_line_m<R>(p, LINE_STEP, la, 1);
        return;
    }
    la.xout = b.xout;
    la.up.d0 = (R)1;
    la.up.d1 = (R)1;
    la.up.S = (R)0;
    la.up.xw0 = la.up.cw0 = (R)1;
    la.up.xw1 = la.up.cw1 = (R)0;
    if (p->scheme == PFC_STABILIZED) {
        la.up.S = (R)p->stab;
    } else if (b.xprev) {
        // (3 X^{n+1} - 4 X^n + X^{n-1}) / (2 dt) = -k^2 (Lk X^{n+1} + 2 N^n - N^{n-1})
        la.xprev = b.xprev;
        la.cprev = b.cprev;
        la.up.d0 = (R)3;
        la.up.d1 = (R)2;
        la.up.xw0 = (R)4;
        la.up.xw1 = (R)-1;
        la.up.cw0 = (R)2;
        la.up.cw1 = (R)-1;
    }   // else: the second-order scheme's first step, a semi-implicit step written to xout
    launch_line_m<R>(p, LINE_SCHEME, la, 1);
}

// The psi^3 row pass of one step on the carried state x, writing c. Two-pass plans: X' -> C',
// edge columns projected in X'. Three-pass plans carry X'' (P and R parts done): the middle
// pass takes it back to the row-pass form in Y, the row pass writes C' and projects Y's edge
// columns, and the middle pass takes C' forward in place and the projected edge columns of Y
// forward into X'' (scale 1/R, the scale of the carried state). Sweeps: 2 + 2 + 2 (+ the edge
// columns) before the line pass.
template <typename R> void enqueue_cube(pfc_plan *p, void *x, void *c, int mark_mid = -1, int mark_row = -1,
                                        const std::function<void(int)> &mark = nullptr) {
    const bool three = three_pass(p);
    if (three) {
        if (mark) mark(mark_mid);
        launch_mid_m<R>(p, +1, x, p->Y, 1.0, false);
    }
    RowArgs<R> ra = row_args<R>(p);
    ra.in = three ? p->Y : x;
    ra.out = c;
    ra.proj = three ? p->Y : x;
    ra.mean = p->d_mean;
    if (mark) mark(mark_row);
    launch_row_m<R>(p, ROW_CUBE, ra, p->nfields);
    if (three) {
        if (mark) mark(mark_mid);
        launch_mid_m<R>(p, -1, c, c, 1.0, false);
        launch_mid_m<R>(p, -1, p->Y, x, 1.0 / p->t.g.R, true);
    }
}

// Step s of a call (row pass (+ middle passes) + line pass).
template <typename R> void enqueue_step(pfc_plan *p, int64_t s, const std::function<void(int)> &mark = nullptr) {
    const StepBufs b = step_bufs(p, s);
    enqueue_cube<R>(p, b.x, b.c, 4, 0, mark);
    if (mark) mark(1);
    launch_update<R>(p, b);
}

// Entry: real state -> carried state (X' or, three-pass, X'' = middle forward of X' / R).
template <typename R> void enqueue_entry(pfc_plan *p, const void *state) {
    const Geom &g = p->t.g;
    launch_means<R>(p, state);
    RowArgs<R> ra = row_args<R>(p);
    ra.in = state;
    ra.out = p->X;
    ra.mean = p->d_mean;
    ra.scale = (R)(1.0 / ((double)g.P * (double)g.M));
    launch_row_m<R>(p, ROW_FWD, ra, p->nfields);
    if (three_pass(p)) launch_mid_m<R>(p, -1, p->X, p->X, 1.0 / g.R, false);
}

// Exit: carried state x -> real state.
template <typename R> void enqueue_exit(pfc_plan *p, void *x, void *state) {
    const bool three = three_pass(p);
    if (three) launch_mid_m<R>(p, +1, x, p->Y, 1.0, false);
    RowArgs<R> rb = row_args<R>(p);
    rb.in = three ? p->Y : x;
    rb.out = state;
    rb.mean = p->d_mean;
    launch_row_m<R>(p, ROW_INV, rb, p->nfields);
}

// nsteps steps: the second-order scheme's starting step directly, then chunks of GRAPH_CHUNK
// steps through one captured graph (an even chunk, so every chunk starts at the same parity of
// the time levels), then the remainder directly.
template <typename R> pfc_status run_steps(pfc_plan *p, int64_t nsteps) {
    int64_t done = 0;
    if (p->scheme == PFC_SBDF2) enqueue_step<R>(p, done++);
    if (nsteps - done >= GRAPH_CHUNK && !p->graph) {
        cudaStream_t cap;
        PFC_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaStream_t saved = p->stream;
        p->stream = cap;
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int s = 0; s < GRAPH_CHUNK; ++s) enqueue_step<R>(p, done + s);
            e = cudaStreamEndCapture(cap, &graph);
        }
        p->stream = saved;
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&p->graph, graph, 0);
            cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return fail(PFC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        p->graph_steps = GRAPH_CHUNK;
    }
    if (p->graph) {
        for (; done + p->graph_steps <= nsteps; done += p->graph_steps)
            PFC_CUDA(cudaGraphLaunch(p->graph, p->stream));
    }
    for (; done < nsteps; ++done) enqueue_step<R>(p, done);
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}

template <typename R> pfc_status step_impl(pfc_plan *p, void *state, int64_t nsteps) {
    if (p->mixed) return mixed_step_impl<R>(p, state, nsteps);
    enqueue_entry<R>(p, state);
    PFC_CUDA(cudaGetLastError());
    pfc_status s = run_steps<R>(p, nsteps);
    if (s != PFC_OK) return s;
    enqueue_exit<R>(p, final_state(p, nsteps), state);
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}

template <typename R> pfc_status r2c_impl(pfc_plan *p, const void *in, void *out) {
    if (p->mixed) return mixed_r2c_impl<R>(p, in, out);
    RowArgs<R> ra = row_args<R>(p);
    ra.in = in;
    ra.out = p->X;
    launch_row_m<R>(p, ROW_FWD, ra, p->nfields);
    if (three_pass(p)) launch_mid_m<R>(p, -1, p->X, p->X, 1.0, false);
    LineArgs<R> la = line_args<R>(p);
    la.x = p->X;
    la.std_out = out;
    launch_line_m<R>(p, LINE_FWD, la, p->nfields);
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}

template <typename R> pfc_status c2r_impl(pfc_plan *p, const void *in, void *out) {
    if (p->mixed) return mixed_c2r_impl<R>(p, in, out);
    const Geom &g = p->t.g;
    LineArgs<R> la = line_args<R>(p);
    la.x = p->X;
    la.std_in = in;
    la.scale = (R)(2.0 / (double)g.nreal);
    launch_line_m<R>(p, LINE_INV, la, p->nfields);
    if (three_pass(p)) launch_mid_m<R>(p, +1, p->X, p->X, 1.0, false);
    RowArgs<R> ra = row_args<R>(p);
    ra.in = p->X;
    ra.out = out;
    launch_row_m<R>(p, ROW_INV, ra, p->nfields);
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}

pfc_status read_status(pfc_plan *p) {
    int st = 0;
    PFC_CUDA(cudaMemcpyAsync(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    PFC_CUDA(cudaStreamSynchronize(p->stream));
    if (st) {
        PFC_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
        PFC_CUDA(cudaStreamSynchronize(p->stream));
        if (st & STATUS_TIMEOUT) return fail(PFC_ERR_TIMEOUT, "a bounded device wait gave up");
        if (st & STATUS_NONFINITE) return fail(PFC_ERR_NONFINITE, "the state holds NaN or Inf");
    }
    return PFC_OK;
}

template <typename R> pfc_status mass_impl(pfc_plan *p, const void *state, double *out) {
    launch_means<R>(p, state);
    PFC_CUDA(cudaGetLastError());
    std::vector<double> m(p->nfields);
    PFC_CUDA(cudaMemcpyAsync(m.data(), p->d_mean, sizeof(double) * p->nfields,
                             cudaMemcpyDeviceToHost, p->stream));
    pfc_status s = read_status(p);
    if (s != PFC_OK) return s;
    std::memcpy(out, m.data(), sizeof(double) * p->nfields);
    return PFC_OK;
}

template <typename R> pfc_status energy_impl(pfc_plan *p, const void *state, double *out) {
    const Geom &g = p->t.g;
    launch_means<R>(p, state);
    // slots in d_out: [0, nf) spectral sums, [nf, 2nf) sum psi^4, [2nf] cross term
    for (int f = 0; f < p->nfields; ++f) {
        const R *x = reinterpret_cast<const R *>(state) + (size_t)f * g.nreal;
        if (p->mixed) {
            mr_row<R>(p, MR_ROW_FWD, x, p->C, p->d_mean + f, 1.0);
            mr_fwd_yz<R>(p, p->C, 1.0);
        } else {
            RowArgs<R> ra = row_args<R>(p);
            ra.in = x;
            ra.out = p->X;
            ra.mean = p->d_mean + f;
            launch_row_m<R>(p, ROW_FWD, ra, 1);
            if (three_pass(p)) launch_mid_m<R>(p, -1, p->X, p->X, 1.0, false);
            LineArgs<R> la = line_args<R>(p);
            la.x = p->X;
            la.std_out = p->C;
            launch_line_m<R>(p, LINE_FWD, la, 1);
        }
        launch_reduce_spec<R>(p->stream, g, to_dev(p->ops[f]), p->dx, p->C, p->d_mean + f,
                              p->d_part, p->d_status);
        launch_finish(p->stream, p->d_part, RED_BLOCKS, 1.0, p->d_out + f);
        launch_reduce_real<R>(p->stream, RED_POW4, x, nullptr, g.nreal, p->d_part, p->d_status);
        launch_finish(p->stream, p->d_part, RED_BLOCKS, 1.0, p->d_out + p->nfields + f);
    }
    if (p->nfields == 2) {
        const R *x0 = reinterpret_cast<const R *>(state);
        launch_reduce_real<R>(p->stream, RED_DOT, x0, x0 + g.nreal, g.nreal, p->d_part, p->d_status);
        launch_finish(p->stream, p->d_part, RED_BLOCKS, 1.0, p->d_out + 4);
    }
    PFC_CUDA(cudaGetLastError());
    double h[5] = {0, 0, 0, 0, 0};
    PFC_CUDA(cudaMemcpyAsync(h, p->d_out, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
    pfc_status s = read_status(p);
    if (s != PFC_OK) return s;
    const double n = (double)g.nreal;
    double f = 0.0;
    for (int i = 0; i < p->nfields; ++i) f += 0.5 * h[i] / (n * n) + 0.25 * h[p->nfields + i] / n;
    if (p->nfields == 2) f += p->alpha * h[4] / n;
    *out = f;
    return PFC_OK;
}

bool plan_ok(const pfc_plan *p) { return p && !p->destroyed; }

}  // namespace

// The hydrodynamic PFC model on one grid: a single-field plan for the transforms and the
// work arrays of one step.
struct pfc_hydro {
    pfc_plan *p = nullptr;
    int ndim = 0;
    double rho = 1, gamma = 1, a0 = 0;
    void *Ps = nullptr, *Ns = nullptr, *Mu = nullptr, *Hw = nullptr, *Fh = nullptr, *Vh = nullptr;  // half spectra
    void *T1 = nullptr, *T2 = nullptr;   // real fields
};

namespace {

// One hydrodynamic step after another (the sequence of the oracle's hydro step): the density's
// transforms, derivatives and update with the old velocity, then each velocity component's
// update with the new density. 20 transforms of the grid a step in 3D (16 in 2D).
template <typename R> pfc_status hydro_impl(pfc_hydro *h, void *psi, void *v, int64_t nsteps) {
    pfc_plan *p = h->p;
    const Geom &g = p->t.g;
    const double two_pi = 6.28318530717958647692528676655900576839;
    HydArgs<R> a{};
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
    a.cx = (R)(two_pi / (g.nx * p->dx));
    a.cy = (R)(two_pi / (g.ny * p->dx));
    a.cz = (R)(two_pi / (g.nz * p->dx));
    a.dt = (R)p->dt;
    a.vf = (R)(std::isinf(h->rho) ? 0.0 : p->dt / h->rho);
    a.gamma = (R)h->gamma;
    a.a0sq = (R)(h->a0 * h->a0);
    a.op = OpR<R>{p->ops[0].kind, (R)p->ops[0].r, (R)p->ops[0].R1, (R)(p->ops[0].q2 * p->ops[0].q2)};
    const int64_t H = g.nstd, N = g.nreal;
    cudaStream_t s = p->stream;
    R *ps = reinterpret_cast<R *>(psi);
    R *t1 = reinterpret_cast<R *>(h->T1), *t2 = reinterpret_cast<R *>(h->T2);
    pfc_status st;
#define HYD_CALL(x) if ((st = (x)) != PFC_OK) return st
    for (int64_t k = 0; k < nsteps; ++k) {
        HYD_CALL(r2c_impl<R>(p, psi, h->Ps));
        launch_hyd_real<R>(s, HYD_CUBE, N, ps, nullptr, t1);
        HYD_CALL(r2c_impl<R>(p, t1, h->Ns));
        for (int j = 0; j < h->ndim; ++j) {   // advection v . grad psi into T1
            launch_hyd_spec<R>(s, HYD_DERIV, a, H, h->Hw, h->Ps, nullptr, j);
            HYD_CALL(c2r_impl<R>(p, h->Hw, t2));
            launch_hyd_real<R>(s, j == 0 ? HYD_MUL : HYD_FMA, N, reinterpret_cast<R *>(v) + (size_t)j * N, t2, t1);
        }
        HYD_CALL(r2c_impl<R>(p, t1, h->Fh));
        launch_hyd_spec<R>(s, HYD_PSI, a, H, h->Ps, h->Ns, h->Fh, 0);
        HYD_CALL(c2r_impl<R>(p, h->Ps, psi));
        launch_hyd_real<R>(s, HYD_CUBE, N, ps, nullptr, t1);
        HYD_CALL(r2c_impl<R>(p, t1, h->Ns));
        launch_hyd_spec<R>(s, HYD_MU, a, H, h->Mu, h->Ns, h->Ps, 0);
        for (int j = 0; j < h->ndim; ++j) {   // velocity component j
            R *vj = reinterpret_cast<R *>(v) + (size_t)j * N;
            launch_hyd_spec<R>(s, HYD_DERIV, a, H, h->Hw, h->Mu, nullptr, j);
            HYD_CALL(c2r_impl<R>(p, h->Hw, t2));
            launch_hyd_real<R>(s, HYD_MUL, N, ps, t2, t1);
            HYD_CALL(r2c_impl<R>(p, t1, h->Fh));
            HYD_CALL(r2c_impl<R>(p, vj, h->Vh));
            launch_hyd_spec<R>(s, HYD_VEL, a, H, h->Vh, h->Fh, nullptr, j);
            HYD_CALL(c2r_impl<R>(p, h->Vh, vj));
        }
    }
#undef HYD_CALL
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}

void hydro_free(pfc_hydro *h) {
    if (h->p) pfc_plan_destroy(h->p);
    cudaFree(h->Ps); cudaFree(h->Ns); cudaFree(h->Mu); cudaFree(h->Hw); cudaFree(h->Fh); cudaFree(h->Vh);
    cudaFree(h->T1); cudaFree(h->T2);
    delete h;
}

// Adjoint of one step: lam_out = A lam_next - 3 psi_n^2 B lam_next, *dr += <lam_next, d psi'/dr>.
// Three-pass plans run the same chain with the middle pass between the row-pass form (in Y) and
// the line form of each array.
template <typename R>
pfc_status adjoint_impl(pfc_plan *p, const void *psi_n, const void *lam_next, void *lam_out, double *dr) {
    const Geom &g = p->t.g;
    const bool three = three_pass(p);
    if (p->nfields != 1) return fail(PFC_ERR_UNSUPPORTED, "the adjoint step is built for single-field plans");
    if (p->scheme != PFC_SEMI_IMPLICIT)
        return fail(PFC_ERR_UNSUPPORTED, "the adjoint step is the adjoint of the semi-implicit step");
    if (p->t.nt_line > 512) return fail(PFC_ERR_UNSUPPORTED, "the adjoint line pass needs tiles of at most 512 threads");
    if (psi_n == lam_out) return fail(PFC_ERR_INVALID_ARG, "lam_out must not alias psi_n");
    const size_t half_bytes = (size_t)g.nhalf * vbytes(p);
    const int nblk = g.ncg * g.P * g.R;
    if (!p->A) {
        PFC_CUDA(cudaMalloc(&p->A, half_bytes));
        PFC_CUDA(cudaMemset(p->A, 0, half_bytes));
        PFC_CUDA(cudaMalloc(&p->d_adjpart, (size_t)nblk * sizeof(double)));
        p->adj_bytes = half_bytes + (size_t)nblk * sizeof(double);
        p->scratch += p->adj_bytes;
    }
    const R scale_x = (R)(1.0 / ((double)g.P * (double)g.M));
    const double inv_r = 1.0 / g.R;
    void *rowform = three ? p->Y : p->A;     // psi_n in the row-pass form
    RowArgs<R> f1 = row_args<R>(p);          // Psi' = X' form of psi_n
    f1.in = psi_n;
    f1.out = rowform;
    f1.scale = scale_x;
    launch_row_m<R>(p, ROW_FWD, f1, 1);
    RowArgs<R> f2 = row_args<R>(p);          // C' = F_p(psi_n^3)
    f2.in = rowform;
    f2.out = p->C;
    f2.proj = rowform;
    launch_row_m<R>(p, ROW_CUBE, f2, 1);
    if (three) {
        launch_mid_m<R>(p, -1, p->C, p->C, 1.0, false);
        launch_mid_m<R>(p, -1, p->Y, p->A, inv_r, false);
    }
    RowArgs<R> f3 = row_args<R>(p);          // Lam' = X' form of lam_next
    f3.in = lam_next;
    f3.out = p->X;
    f3.scale = scale_x;
    launch_row_m<R>(p, ROW_FWD, f3, 1);
    if (three) launch_mid_m<R>(p, -1, p->X, p->X, inv_r, false);
    AdjArgs<R> aa{};
    aa.lam = p->X;
    aa.psi = p->A;
    aa.c = p->C;
    aa.partials = p->d_adjpart;
    aa.up = line_args<R>(p).up;
    aa.PM = (R)((double)g.P * (double)g.M * (double)g.R);
    aa.st = stage_tw<R>(p);
    launch_line_adj<R>(cfg(p), aa);
    launch_finish(p->stream, p->d_adjpart, nblk, 1.0 / (2.0 * g.Q), dr, true);
    if (three) launch_mid_m<R>(p, +1, p->X, p->Y, 1.0, false);
    RowArgs<R> i1 = row_args<R>(p);          // lam_out = U
    i1.in = three ? p->Y : p->X;
    i1.out = lam_out;
    launch_row_m<R>(p, ROW_INV, i1, 1);
    if (three) launch_mid_m<R>(p, +1, p->A, p->Y, 1.0, false);
    RowArgs<R> i2 = row_args<R>(p);          // lam_out -= 3 psi_n^2 V
    i2.in = three ? p->Y : p->A;
    i2.out = lam_out;
    i2.aux = psi_n;
    launch_row_m<R>(p, ROW_ADJ_MIX, i2, 1);
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}

// ------------------------------------------------------------------------------------------
// Recorded segments and the fused adjoint (two-pass single-field semi-implicit plans)
// ------------------------------------------------------------------------------------------
// Record layout: a 256-byte header holding the FP64 mean, then the X' forms of the states of
// steps 0 .. n (n + 1 half spectra; slot k + 1 is the line pass's output of step k), then the
// C' forms F_p(psi_k^3) of steps 0 .. n - 1 (n half spectra).
constexpr size_t REC_HEAD = 256;
size_t record_bytes(const pfc_plan *p, int64_t n) {
    return REC_HEAD + (size_t)(2 * n + 1) * (size_t)p->t.g.nhalf * vbytes(p);
}

// The fused adjoint row pass's geometry: the plan's, with fewer row groups per block when its
// two row buffers need it; false when one group does not fit.
bool adj2_geom(const pfc_plan *p, Geom &g, int &nt, size_t &smem) {
    const size_t smax = smem_optin();
    g = p->t.g;
    while (g.gpc > 1 && row_adj2_smem(g, vbytes(p)) > smax) g.gpc /= 2;
    smem = row_adj2_smem(g, vbytes(p));
    const int Tr = g.M / 8, rows = g.gpc * g.P;
    nt = std::min(512, std::max(Tr, rows * Tr));
    if (nt < 32) nt = std::max(Tr, 32 / Tr * Tr);
    return smem <= smax;
}

pfc_status segment_supported(const pfc_plan *p) {
    if (p->mixed) return fail(PFC_ERR_UNSUPPORTED, "recorded segments are built for power-of-two grids");
    if (p->nfields != 1) return fail(PFC_ERR_UNSUPPORTED, "recorded segments are built for single-field plans");
    if (p->scheme != PFC_SEMI_IMPLICIT) return fail(PFC_ERR_UNSUPPORTED, "recorded segments follow the semi-implicit step");
    if (three_pass(p)) return fail(PFC_ERR_UNSUPPORTED, "recorded segments are built for two-pass plans");
    if (p->t.nt_line > 512) return fail(PFC_ERR_UNSUPPORTED, "the adjoint line pass needs tiles of at most 512 threads");
    Geom g;
    int nt;
    size_t smem;
    if (!adj2_geom(p, g, nt, smem)) return fail(PFC_ERR_UNSUPPORTED, "the fused adjoint row pass does not fit shared memory");
    return PFC_OK;
}

template <typename R> pfc_status record_impl(pfc_plan *p, void *state, int64_t n, void *rec) {
    using V = typename VT<R>::V;
    const Geom &g = p->t.g;
    V *slot = reinterpret_cast<V *>(static_cast<unsigned char *>(rec) + REC_HEAD);
    V *cslot = slot + (size_t)(n + 1) * g.nhalf;
    launch_means<R>(p, state);
    RowArgs<R> ra = row_args<R>(p);
    ra.in = state;
    ra.out = slot;
    ra.mean = p->d_mean;
    ra.scale = (R)(1.0 / ((double)g.P * (double)g.M));
    launch_row_m<R>(p, ROW_FWD, ra, 1);
    for (int64_t k = 0; k < n; ++k) {
        V *xk = slot + (size_t)k * g.nhalf;
        RowArgs<R> rc = row_args<R>(p);
        rc.in = xk;
        rc.out = cslot + (size_t)k * g.nhalf;
        rc.proj = xk;
        rc.mean = p->d_mean;
        launch_row_m<R>(p, ROW_CUBE, rc, 1);
        LineArgs<R> la = line_args<R>(p);
        la.x = xk;
        la.c = rc.out;
        la.xout = xk + g.nhalf;
        launch_line_m<R>(p, LINE_STEP, la, 1);
    }
    RowArgs<R> rb = row_args<R>(p);
    rb.in = slot + (size_t)n * g.nhalf;
    rb.out = state;
    rb.mean = p->d_mean;
    launch_row_m<R>(p, ROW_INV, rb, 1);
    PFC_CUDA(cudaMemcpyAsync(rec, p->d_mean, sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}

template <typename R> pfc_status segment_impl(pfc_plan *p, const void *rec, int64_t n, void *lam, double *dr) {
    using V = typename VT<R>::V;
    const Geom &g = p->t.g;
    const size_t half_bytes = (size_t)g.nhalf * vbytes(p);
    const int nblk = g.ncg * g.P * g.R;
    if (!p->A) {
        PFC_CUDA(cudaMalloc(&p->A, half_bytes));
        PFC_CUDA(cudaMemset(p->A, 0, half_bytes));
        PFC_CUDA(cudaMalloc(&p->d_adjpart, (size_t)nblk * sizeof(double)));
        p->adj_bytes = half_bytes + (size_t)nblk * sizeof(double);
        p->scratch += p->adj_bytes;
    }
    Geom g2;
    int nt2;
    size_t smem2;
    adj2_geom(p, g2, nt2, smem2);
    PFC_CUDA(set_smem_adj2<R>(smem2));
    const V *slot = reinterpret_cast<const V *>(static_cast<const unsigned char *>(rec) + REC_HEAD);
    const V *cslot = slot + (size_t)(n + 1) * g.nhalf;
    const double *mean = static_cast<const double *>(rec);
    RowArgs<R> f = row_args<R>(p);          // Lam' = X' form of lam (no mean)
    f.in = lam;
    f.out = p->X;
    f.scale = (R)(1.0 / ((double)g.P * (double)g.M));
    launch_row_m<R>(p, ROW_FWD, f, 1);
    AdjArgs<R> aa{};
    aa.lam = p->X;
    aa.vout = p->A;
    aa.partials = p->d_adjpart;
    aa.up = line_args<R>(p).up;
    aa.PM = (R)((double)g.P * (double)g.M);
    aa.st = stage_tw<R>(p);
    RowArgs<R> rr = row_args<R>(p);
    rr.in = p->X;
    rr.aux2 = p->A;
    rr.out = p->X;
    rr.mean = mean;
    rr.scale = (R)(1.0 / ((double)g.P * (double)g.M));
    for (int64_t k = n - 1; k >= 0; --k) {
        aa.psi = const_cast<V *>(slot + (size_t)k * g.nhalf);
        aa.c = cslot + (size_t)k * g.nhalf;
        launch_line_adj<R>(cfg(p), aa);
        launch_finish(p->stream, p->d_adjpart, nblk, 1.0 / (2.0 * g.Q), dr, true);
        rr.aux3 = aa.psi;
        launch_row_adj2<R>(p->stream, g2, nt2, smem2, rr);
    }
    RowArgs<R> i1 = row_args<R>(p);
    i1.in = p->X;
    i1.out = lam;
    launch_row_m<R>(p, ROW_INV, i1, 1);
    PFC_CUDA(cudaGetLastError());
    return PFC_OK;
}

// pfc_step with an event between consecutive launches; kinds: 0 row, 1 line, 2 entry, 3 exit,
// 4 middle passes.
template <typename R>
pfc_status profile_impl(pfc_plan *p, void *state, int64_t nsteps, double *ms, int64_t *launches) {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    auto mark = [&](int k) -> cudaError_t {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        ev.push_back(e);
        kind.push_back(k);
        return cudaEventRecord(e, p->stream);
    };
    int64_t nl = 0;
    const bool three = three_pass(p);
    cudaError_t err = cudaSuccess;
    if (p->mixed) {
        mixed_enqueue<R>(p, state, nsteps, [&](int k) {
            if (err == cudaSuccess) err = mark(k);
        });
        nl = mixed_launches(p, nsteps);
    } else {
        err = mark(2);
        enqueue_entry<R>(p, state);
        nl += 2 * p->nfields + 1 + (three ? 1 : 0);
        auto mk = [&](int k) {
            if (err == cudaSuccess) err = mark(k);
        };
        for (int64_t s = 0; s < nsteps && err == cudaSuccess; ++s) {
            enqueue_step<R>(p, s, mk);
            nl += 2 + (three ? 3 : 0);
        }
        mk(3);
        enqueue_exit<R>(p, final_state(p, nsteps), state);
        nl += 1 + (three ? 1 : 0);
    }
    if (err == cudaSuccess) err = mark(-1);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
    double acc[5] = {0, 0, 0, 0, 0};
    for (size_t i = 0; err == cudaSuccess && i + 1 < ev.size(); ++i) {
        float t = 0.f;
        err = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
        if (kind[i] >= 0) acc[kind[i]] += t;
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (err != cudaSuccess) return fail(PFC_ERR_CUDA, std::string("profile: ") + cudaGetErrorString(err));
    std::memcpy(ms, acc, sizeof(acc));
    *launches = nl;
    return PFC_OK;
}

// Switch a plan to the tiling t: X' and C' grow when t pads kx further (contents cleared),
// the adjoint's arrays are released (its next call allocates them for t), kernel shared-memory
// limits are raised, and the captured graph is dropped.
pfc_status apply_tiles(pfc_plan *p, const Tiles &t) {
    const size_t need = (size_t)t.g.nhalf * p->nfields * vbytes(p);
    PFC_CUDA(cudaStreamSynchronize(p->stream));
    if (t.g.R > 1 && !p->Y) {
        // a three-pass tiling needs the row-pass form of the state as well (allocated on demand)
        PFC_CUDA(cudaMalloc(&p->Y, std::max(need, p->half_cap)));
        p->scratch += std::max(need, p->half_cap);
        p->y_cap = std::max(need, p->half_cap);
    }
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    if (p->A) {
        cudaFree(p->A);
        cudaFree(p->d_adjpart);
        p->A = nullptr;
        p->d_adjpart = nullptr;
        p->scratch -= p->adj_bytes;
        p->adj_bytes = 0;
    }
    if (need > p->half_cap) {
        // the new arrays first: on failure the plan keeps its arrays and tiling
        void *x = nullptr, *c = nullptr;
        PFC_CUDA(cudaMalloc(&x, need));
        if (cudaError_t e = cudaMalloc(&c, need); e != cudaSuccess) {
            cudaFree(x);
            return fail(e == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA,
                        std::string("autotune scratch: ") + cudaGetErrorString(e));
        }
        cudaFree(p->X);
        cudaFree(p->C);
        p->X = x;
        p->C = c;
        p->scratch += 2 * (need - p->half_cap);
        p->half_cap = need;
    }
    if (p->X2 && p->lv_cap < p->half_cap) {
        void *x = nullptr, *c = nullptr;
        PFC_CUDA(cudaMalloc(&x, p->half_cap));
        if (cudaError_t e = cudaMalloc(&c, p->half_cap); e != cudaSuccess) {
            cudaFree(x);
            return fail(e == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA,
                        std::string("time levels: ") + cudaGetErrorString(e));
        }
        cudaFree(p->X2);
        cudaFree(p->C2);
        p->X2 = x;
        p->C2 = c;
        p->scratch += 2 * (p->half_cap - p->lv_cap);
        p->lv_cap = p->half_cap;
    }
    if (p->Y && p->y_cap < p->half_cap) {
        void *y = nullptr;
        PFC_CUDA(cudaMalloc(&y, p->half_cap));
        cudaFree(p->Y);
        p->Y = y;
        p->scratch += p->half_cap - p->y_cap;
        p->y_cap = p->half_cap;
    }
    PFC_CUDA(cudaMemsetAsync(p->X, 0, p->half_cap, p->stream));
    PFC_CUDA(cudaMemsetAsync(p->C, 0, p->half_cap, p->stream));
    p->t = t;
    PFC_CUDA(p->prec == PFC_FP64 ? raise_smem_attrs<double>(cfg(p)) : raise_smem_attrs<float>(cfg(p)));
    return PFC_OK;
}

// ms per step of pfc_step(state, nsteps) on the current tiling: one untimed call (which also
// captures the graph), then the faster of two timed calls.
pfc_status time_steps(pfc_plan *p, void *state, int nsteps, double *ms) {
    cudaEvent_t e0, e1;
    PFC_CUDA(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(PFC_ERR_CUDA, std::string("autotune events: ") + cudaGetErrorString(err));
    }
    pfc_status st = pfc_step(p, state, nsteps);
    double best = 1e300;
    for (int rep = 0; rep < 2 && st == PFC_OK; ++rep) {
        float t = 0.f;
        if ((err = cudaEventRecord(e0, p->stream)) != cudaSuccess) break;
        if ((st = pfc_step(p, state, nsteps)) != PFC_OK) break;
        if ((err = cudaEventRecord(e1, p->stream)) != cudaSuccess) break;
        if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
        if ((err = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
        best = std::min(best, (double)t / nsteps);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PFC_OK) return st;
    if (err != cudaSuccess) return fail(PFC_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(err));
    *ms = best;
    return PFC_OK;
}

// Key of an autotune cache entry: the grid, precision, field count and device.
std::string tune_key(const pfc_plan *p) {
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        std::snprintf(prop.name, sizeof(prop.name), "unknown");
    for (char *c = prop.name; *c; ++c)
        if (*c == ' ' || *c == '"') *c = '_';
    char buf[384];
    std::snprintf(buf, sizeof(buf), "%dx%dx%d prec%d fields%d %s", p->nz, p->ny, p->nx, p->prec, p->nfields,
                  prop.name);
    return buf;
}

size_t smem_optin() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return (size_t)optin;
}

// A mixed-radix plan (single field, the semi-implicit step): tables, work arrays, launch shapes.
pfc_status mixed_plan_create(pfc_plan **out, int ndim, const int64_t d[3], double dx, double dt,
                             const pfc_op *ops, int precision, void *stream) {
    pfc_plan *p = new pfc_plan();
    p->ndim = ndim;
    p->nz = (int)d[0]; p->ny = (int)d[1]; p->nx = (int)d[2];
    p->dx = dx; p->dt = dt;
    p->ops[0] = ops[0];
    p->nfields = 1;
    p->prec = precision;
    p->stream = reinterpret_cast<cudaStream_t>(stream);
    p->mixed = true;
    MrGeom &g = p->mg;
    g.nx = p->nx; g.ny = p->ny; g.nz = p->nz; g.M = p->nx / 2; g.xs = g.M + 1; g.ndim = ndim;
    g.nstd = (int64_t)g.ny * g.nz * g.xs;
    g.nreal = (int64_t)g.nx * g.ny * g.nz;
    // the plan geometry's fields the shared kernels (reductions) read
    Geom &pg = p->t.g;
    pg = Geom{};
    pg.nx = g.nx; pg.ny = g.ny; pg.nz = g.nz; pg.M = g.M; pg.nreal = g.nreal; pg.nstd = g.nstd;
    pg.Ry = pg.Rz = pg.R = 1;
    const size_t vb = vbytes(p);
    // tables: per axis the stage twiddles
    std::vector<double> tw;
    const int lens[3] = {g.M, g.ny, g.nz};
    int optin = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        delete p;
        return fail(PFC_ERR_CUDA, "device query failed");
    }
    // a block's shared memory: up to 100 KB (two blocks an SM), more only for one long line
    const size_t budget = 100 * 1024;
    size_t smem_col = 0;
    for (int a = 0; a < 3; ++a) g.ax[a].n = lens[a];
    mr_axes(g, false, tw);
    for (int a = 0; a < 3; ++a) {
        const MrAxis &ax = g.ax[a];
        // launch shapes: one warp a line; as many lines a block as the budget holds (rows of
        // 128 bytes in the column passes: 16 FP32 or 8 FP64 columns)
        if (a == 0) {
            int rows = 8;
            while (rows > 1 && mr_row_smem(ax.n, rows, vb) > budget) rows /= 2;
            p->mr_rows = rows;
        } else if (ax.n > 1) {
            int W = vb == 8 ? 16 : 8;
            while (W > 1 && mr_col_smem(ax.n, W, vb) > budget) W /= 2;
            p->mr_W[a] = W;
            p->mr_wE[a] = mr_col_smem(ax.n, 2, vb) <= budget ? 2 : 1;
            smem_col = std::max(smem_col, mr_col_smem(ax.n, std::max(W, p->mr_wE[a]), vb));
        }
    }
    if (smem_col > (size_t)optin || mr_row_smem(g.M, p->mr_rows, vb) > (size_t)optin) {
        delete p;
        return fail(PFC_ERR_UNSUPPORTED, "a line of this grid does not fit shared memory");
    }
    std::vector<double> twx(2 * (size_t)g.nx);
    for (int t = 0; t < g.nx; ++t) unit_root_fwd(t, g.nx, &twx[2 * t], &twx[2 * t + 1]);
    auto cleanup = [&](cudaError_t err) {
        pfc_plan_destroy(p);
        return fail(err == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA,
                    std::string("plan allocation: ") + cudaGetErrorString(err));
    };
    const size_t half = (size_t)g.nstd * vb;
    cudaError_t e;
    if ((e = cudaMalloc(&p->X, half)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->C, half)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->Y, half)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->E, 2 * (size_t)g.ny * g.nz * vb)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->mtw, tw.size() / 2 * vb)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->mtwx, twx.size() / 2 * vb)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->d_mean, 8 * sizeof(double))) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->d_part, RED_BLOCKS * sizeof(double))) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->d_out, 8 * sizeof(double))) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->d_status, sizeof(int))) != cudaSuccess) return cleanup(e);
    p->half_cap = p->y_cap = half;
    p->scratch = 3 * half + 2 * (size_t)g.ny * g.nz * vb + (tw.size() + twx.size()) / 2 * vb +
                 (16 + RED_BLOCKS) * sizeof(double) + sizeof(int);
    auto upload = [&](void *dst, const std::vector<double> &src) {
        if (p->prec == PFC_FP64) return cudaMemcpy(dst, src.data(), src.size() * 8, cudaMemcpyHostToDevice);
        std::vector<float> f(src.begin(), src.end());
        return cudaMemcpy(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
    };
    if ((e = upload(p->mtw, tw)) != cudaSuccess) return cleanup(e);
    if ((e = upload(p->mtwx, twx)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess) return cleanup(e);
    if ((e = cudaMemset(p->d_mean, 0, 8 * sizeof(double))) != cudaSuccess) return cleanup(e);
    const size_t smem_row = mr_row_smem(g.M, p->mr_rows, vb);
    e = p->prec == PFC_FP64 ? set_smem_mr<double>(smem_row, smem_col) : set_smem_mr<float>(smem_row, smem_col);
    if (e != cudaSuccess) return cleanup(e);
    p->mtw_cap = tw.size() / 2 * vb;
    p->mr_smem_col = smem_col;
    *out = p;
    return PFC_OK;
}

// A launch shape of a mixed-radix plan: the radix order of the axes, warps a column of the
// column passes, rows a block of the x pass.
struct MrShape {
    bool even_first;
    int G, rows;
};

// Switch a mixed-radix plan to shape c (its twiddle table rebuilt for the radix order).
template <typename R> pfc_status mr_apply(pfc_plan *p, const MrShape &c) {
    const size_t vb = vbytes(p);
    MrGeom g = p->mg;
    std::vector<double> tw;
    mr_axes(g, c.even_first, tw);
    const size_t need = tw.size() / 2 * vb;
    PFC_CUDA(cudaStreamSynchronize(p->stream));
    if (need > p->mtw_cap) {
        void *t = nullptr;
        PFC_CUDA(cudaMalloc(&t, need));
        cudaFree(p->mtw);
        p->mtw = t;
        p->mtw_cap = need;
    }
    if (sizeof(R) == 8) {
        PFC_CUDA(cudaMemcpy(p->mtw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(tw.begin(), tw.end());
        PFC_CUDA(cudaMemcpy(p->mtw, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    }
    PFC_CUDA(set_smem_mr<R>(mr_row_smem(g.M, c.rows, vb), p->mr_smem_col));
    p->mg = g;
    p->mr_even_first = c.even_first;
    p->mr_G = c.G;
    p->mr_rows = c.rows;
    return PFC_OK;
}

// The autotuner of mixed-radix plans: the radix order (odd radices first or last), one or two
// warps a column in the column passes, and the x pass' rows a block, each timed on trial_steps
// steps of a zero field (a fixed point of the step); the fastest is kept.
template <typename R> pfc_status mr_autotune(pfc_plan *p, int max_candidates, int trial_steps, double *best_ms_out) {
    const size_t vb = vbytes(p);
    const MrShape cur{p->mr_even_first, p->mr_G, p->mr_rows};
    std::vector<MrShape> cand{cur};
    bool mixed_order = false;   // some axis has both odd and even radices
    for (int a = 0; a < 3; ++a) {
        bool odd = false, even = false;
        for (int s = 0; s < p->mg.ax[a].nst; ++s) (p->mg.ax[a].radix[s] & 1 ? odd : even) = true;
        mixed_order = mixed_order || (odd && even);
    }
    const size_t optin = smem_optin();
    for (int ef = 0; ef < (mixed_order ? 2 : 1); ++ef)
        for (int G : {2, 1})
            for (int rows : {cur.rows, cur.rows / 2, cur.rows * 2}) {
                // (the x pass runs at most 256 threads a block: its launch bounds)
                if (rows < 1 || rows > 8 || mr_row_smem(p->mg.M, rows, vb) > optin) continue;
                const MrShape c{ef != 0, G, rows};
                bool dup = false;
                for (const MrShape &d : cand) dup = dup || (d.even_first == c.even_first && d.G == c.G && d.rows == c.rows);
                if (!dup) cand.push_back(c);
            }
    if ((int)cand.size() > max_candidates) cand.resize(max_candidates);
    void *tmp = nullptr;
    const size_t bytes = (size_t)p->mg.nreal * sizeof(R);
    PFC_CUDA(cudaMalloc(&tmp, bytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(tmp, 0, bytes, p->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int best = 0;
    double best_ms = 1e300;
    pfc_status st = PFC_OK;
    for (size_t i = 0; i < cand.size() && e == cudaSuccess && st == PFC_OK; ++i) {
        if ((st = mr_apply<R>(p, cand[i])) != PFC_OK) break;
        mixed_enqueue<R>(p, tmp, 1, [](int) {});
        float ms = 0.f;
        e = cudaEventRecord(e0, p->stream);
        if (e == cudaSuccess) mixed_enqueue<R>(p, tmp, trial_steps, [](int) {});
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms / trial_steps < best_ms) {
            best_ms = ms / trial_steps;
            best = (int)i;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(p->stream);
    cudaFree(tmp);
    if (st != PFC_OK) return st;
    if (e != cudaSuccess) return fail(PFC_ERR_CUDA, std::string("mixed-radix autotune: ") + cudaGetErrorString(e));
    if ((st = mr_apply<R>(p, cand[best])) != PFC_OK) return st;
    if (best_ms_out) *best_ms_out = best_ms;
    return PFC_OK;
}

}  // namespace

pfc_status pfc::set_error(pfc_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

// ============================================================================================
// C ABI
// ============================================================================================
extern "C" {

const char *pfc_status_string(pfc_status s) {
    switch (s) {
        case PFC_OK: return "PFC_OK";
        case PFC_ERR_INVALID_ARG: return "PFC_ERR_INVALID_ARG";
        case PFC_ERR_UNSUPPORTED: return "PFC_ERR_UNSUPPORTED";
        case PFC_ERR_UNSTABLE_OPERATOR: return "PFC_ERR_UNSTABLE_OPERATOR";
        case PFC_ERR_OUT_OF_MEMORY: return "PFC_ERR_OUT_OF_MEMORY";
        case PFC_ERR_CUDA: return "PFC_ERR_CUDA";
        case PFC_ERR_NONFINITE: return "PFC_ERR_NONFINITE";
        case PFC_ERR_TIMEOUT: return "PFC_ERR_TIMEOUT";
    }
    return "PFC_ERR_UNKNOWN";
}

const char *pfc_last_error(void) { return g_last_error.c_str(); }

pfc_status pfc_plan_create(pfc_plan **out, int ndim, const int64_t *dims, double dx, double dt,
                           const pfc_op *ops, int nfields, const double *coupling, int precision,
                           void *stream) {
    if (!out || !dims || !ops) return fail(PFC_ERR_INVALID_ARG, "null pointer argument");
    if (ndim != 2 && ndim != 3) return fail(PFC_ERR_INVALID_ARG, "ndim must be 2 or 3");
    if (!(dx > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dt))
        return fail(PFC_ERR_INVALID_ARG, "dx and dt must be finite and > 0");
    if (nfields < 1 || nfields > 2) return fail(PFC_ERR_UNSUPPORTED, "nfields must be 1 or 2");
    if (precision != PFC_FP64 && precision != PFC_FP32_MIXED)
        return fail(PFC_ERR_INVALID_ARG, "unknown precision");
    for (int f = 0; f < nfields; ++f) {
        if (ops[f].kind != PFC_ONE_MODE && ops[f].kind != PFC_TWO_MODE)
            return fail(PFC_ERR_INVALID_ARG, "unknown operator kind");
        if (!std::isfinite(ops[f].r) || !std::isfinite(ops[f].R1) || !std::isfinite(ops[f].q2))
            return fail(PFC_ERR_INVALID_ARG, "operator coefficients must be finite");
    }
    int64_t d[3] = {1, 1, 1};   // (nz, ny, nx)
    for (int i = 0; i < ndim; ++i) d[3 - ndim + i] = dims[i];
    bool all_pow2 = true, mixed_ok = d[2] % 2 == 0 && mr_extent_ok(d[2] / 2);
    for (int i = 3 - ndim; i < 3; ++i) {
        if (d[i] <= 0) return fail(PFC_ERR_INVALID_ARG, "dims must be positive");
        all_pow2 = all_pow2 && is_pow2(d[i]) && d[i] >= 16 && d[i] <= 4096;
        mixed_ok = mixed_ok && mr_extent_ok(d[i]);
    }
    if (!all_pow2 && !mixed_ok)
        return fail(PFC_ERR_UNSUPPORTED, "extents must be powers of two in [16, 4096], or products of 2, 3, 5 "
                                         "and 7 in [8, 4096] with nx / 2 one too");
    if (!all_pow2 && nfields != 1)
        return fail(PFC_ERR_UNSUPPORTED, "two-field plans need power-of-two extents");
    double alpha = 0.0;
    if (nfields == 2 && coupling) alpha = coupling[1];
    const double kmax = M_PI / dx;
    const double k2max = kmax * kmax * ndim;
    if (min_implicit(ops, nfields, alpha, dt, k2max) <= 0.0)
        return fail(PFC_ERR_UNSTABLE_OPERATOR, "1 + dt k^2 Lk(k) is not positive on the grid");

    if (!all_pow2) return mixed_plan_create(out, ndim, d, dx, dt, ops, precision, stream);
    pfc_plan *p = new pfc_plan();
    p->ndim = ndim;
    p->nz = (int)d[0]; p->ny = (int)d[1]; p->nx = (int)d[2];
    p->dx = dx; p->dt = dt;
    for (int f = 0; f < nfields; ++f) p->ops[f] = ops[f];
    p->nfields = nfields;
    p->alpha = alpha;
    p->prec = precision;
    p->stream = reinterpret_cast<cudaStream_t>(stream);

    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) { delete p; return fail(PFC_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e)); }
    const size_t smem_max = (size_t)optin;
    // the line pass holds two tiles, a two-field plan's three (see k_line_step2)
    if (!plan_tiles(p->t, p->nx, p->ny, p->nz, vbytes(p), nfields == 2 ? 3 : 2, smem_max) ||
        (nfields == 2 && (p->t.nt_line > 512 || p->t.g.R > 1))) {
        delete p;
        return fail(PFC_ERR_UNSUPPORTED, "no pass tiling fits shared memory for this grid and precision");
    }
    const Geom &g = p->t.g;
    e = p->prec == PFC_FP64 ? raise_smem_attrs<double>(cfg(p)) : raise_smem_attrs<float>(cfg(p));
    if (e != cudaSuccess) { delete p; return fail(PFC_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e)); }

    const size_t half_bytes = (size_t)g.nhalf * nfields * vbytes(p);
    const int64_t ntab = int64_t(1) << g.ltab;
    auto cleanup = [&](cudaError_t err) {
        pfc_plan_destroy(p);
        return fail(err == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA,
                    std::string("plan allocation: ") + cudaGetErrorString(err));
    };
    if ((e = cudaMalloc(&p->X, half_bytes)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->C, half_bytes)) != cudaSuccess) return cleanup(e);
    if (g.R > 1) {
        if ((e = cudaMalloc(&p->Y, half_bytes)) != cudaSuccess) return cleanup(e);
        p->y_cap = half_bytes;
    }
    if ((e = cudaMalloc(&p->tw, ntab * vbytes(p))) != cudaSuccess) return cleanup(e);
    const int64_t nst = STW_TOTAL;
    if ((e = cudaMalloc(&p->stw, nst * vbytes(p))) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->d_mean, 8 * sizeof(double))) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->d_part, RED_BLOCKS * sizeof(double))) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->d_out, 8 * sizeof(double))) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->d_status, sizeof(int))) != cudaSuccess) return cleanup(e);
    p->half_cap = half_bytes;
    p->ntile = nfields == 2 ? 3 : 2;
    p->scratch = (g.R > 1 ? 3 : 2) * half_bytes + (ntab + nst) * vbytes(p) + (16 + RED_BLOCKS) * sizeof(double) +
                 sizeof(int);

    std::vector<double> tw, st;
    twiddle_tables(ntab, tw, st);
    auto upload = [&](void *dst, const std::vector<double> &src) {
        if (p->prec == PFC_FP64) return cudaMemcpy(dst, src.data(), src.size() * 8, cudaMemcpyHostToDevice);
        std::vector<float> f(src.size());
        for (size_t i = 0; i < src.size(); ++i) f[i] = (float)src[i];
        return cudaMemcpy(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
    };
    if ((e = upload(p->tw, tw)) != cudaSuccess) return cleanup(e);
    if ((e = upload(p->stw, st)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMemset(p->X, 0, half_bytes)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMemset(p->C, 0, half_bytes)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMemset(p->d_mean, 0, 8 * sizeof(double))) != cudaSuccess) return cleanup(e);
    if ((e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess) return cleanup(e);
    *out = p;
    return PFC_OK;
}

pfc_status pfc_plan_destroy(pfc_plan *p) {
    if (!p) return PFC_OK;
    if (!p->destroyed && p->mixed) {
        cudaStreamSynchronize(p->stream);
        cudaFree(p->mtw); cudaFree(p->mtwx); cudaFree(p->E);
        p->mtw = p->mtwx = p->E = nullptr;
    }
    if (p->destroyed) return fail(PFC_ERR_INVALID_ARG, "plan already destroyed");
    cudaStreamSynchronize(p->stream);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    cudaFree(p->X); cudaFree(p->C); cudaFree(p->Y); cudaFree(p->X2); cudaFree(p->C2); cudaFree(p->tw); cudaFree(p->stw);
    cudaFree(p->A); cudaFree(p->d_adjpart);
    cudaFree(p->d_mean); cudaFree(p->d_part); cudaFree(p->d_out); cudaFree(p->d_status);
    p->destroyed = true;
    delete p;
    return PFC_OK;
}

pfc_status pfc_step(pfc_plan *p, void *state, int64_t nsteps) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (!state) return fail(PFC_ERR_INVALID_ARG, "null state");
    if (nsteps < 0) return fail(PFC_ERR_INVALID_ARG, "nsteps must be >= 0");
    if ((reinterpret_cast<uintptr_t>(state) & 15) != 0) return fail(PFC_ERR_INVALID_ARG, "state must be 16-byte aligned");
    if (nsteps == 0) return PFC_OK;
    return p->prec == PFC_FP64 ? step_impl<double>(p, state, nsteps) : step_impl<float>(p, state, nsteps);
}

pfc_status pfc_fft_r2c(pfc_plan *p, const void *in, void *out) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (!in || !out) return fail(PFC_ERR_INVALID_ARG, "null array");
    return p->prec == PFC_FP64 ? r2c_impl<double>(p, in, out) : r2c_impl<float>(p, in, out);
}

pfc_status pfc_fft_c2r(pfc_plan *p, const void *in, void *out) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (!in || !out) return fail(PFC_ERR_INVALID_ARG, "null array");
    return p->prec == PFC_FP64 ? c2r_impl<double>(p, in, out) : c2r_impl<float>(p, in, out);
}

pfc_status pfc_mass(pfc_plan *p, const void *state, double *out) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (!state || !out) return fail(PFC_ERR_INVALID_ARG, "null pointer");
    return p->prec == PFC_FP64 ? mass_impl<double>(p, state, out) : mass_impl<float>(p, state, out);
}

pfc_status pfc_energy(pfc_plan *p, const void *state, double *out) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (!state || !out) return fail(PFC_ERR_INVALID_ARG, "null pointer");
    return p->prec == PFC_FP64 ? energy_impl<double>(p, state, out) : energy_impl<float>(p, state, out);
}

pfc_status pfc_step_adjoint(pfc_plan *p, const void *psi_n, const void *lam_next, void *lam_out,
                            double *dr) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (!psi_n || !lam_next || !lam_out || !dr) return fail(PFC_ERR_INVALID_ARG, "null pointer");
    if (p->mixed) return fail(PFC_ERR_UNSUPPORTED, "the adjoint step is built for power-of-two grids");
    return p->prec == PFC_FP64 ? adjoint_impl<double>(p, psi_n, lam_next, lam_out, dr)
                               : adjoint_impl<float>(p, psi_n, lam_next, lam_out, dr);
}

pfc_status pfc_profile_steps(pfc_plan *p, void *state, int64_t nsteps, double *ms_out,
                             int64_t *launches) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (!state || !ms_out || !launches) return fail(PFC_ERR_INVALID_ARG, "null pointer");
    if (nsteps < 0) return fail(PFC_ERR_INVALID_ARG, "nsteps must be >= 0");
    return p->prec == PFC_FP64 ? profile_impl<double>(p, state, nsteps, ms_out, launches)
                               : profile_impl<float>(p, state, nsteps, ms_out, launches);
}

pfc_status pfc_set_r(pfc_plan *p, int field, double r) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (field < 0 || field >= p->nfields) return fail(PFC_ERR_INVALID_ARG, "field out of range");
    if (!std::isfinite(r)) return fail(PFC_ERR_INVALID_ARG, "r must be finite");
    pfc_op ops[2] = {p->ops[0], p->ops[1]};
    ops[field].r = r;
    const double kmax = M_PI / p->dx;
    if (min_implicit(ops, p->nfields, p->alpha, p->dt, kmax * kmax * p->ndim) <= 0.0)
        return fail(PFC_ERR_UNSTABLE_OPERATOR, "1 + dt k^2 Lk(k) is not positive on the grid");
    cudaStreamSynchronize(p->stream);
    p->ops[field].r = r;
    if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
    return PFC_OK;
}

pfc_status pfc_set_integrator(pfc_plan *p, int scheme, double S) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (scheme != PFC_SEMI_IMPLICIT && scheme != PFC_STABILIZED && scheme != PFC_SBDF2)
        return fail(PFC_ERR_INVALID_ARG, "unknown integrator");
    if (!std::isfinite(S) || S < 0) return fail(PFC_ERR_INVALID_ARG, "S must be finite and >= 0");
    if (scheme != PFC_SEMI_IMPLICIT && p->mixed)
        return fail(PFC_ERR_UNSUPPORTED, "mixed-radix grids step with the semi-implicit scheme");
    if (scheme != PFC_SEMI_IMPLICIT && p->nfields != 1)
        return fail(PFC_ERR_UNSUPPORTED, "the alternative integrators are built for single-field plans");
    // the implicit factor of the scheme must stay positive: 1 + dt k^2 (Lk + S) (stabilised, Lk
    // shifted by S), 3 + 2 dt k^2 Lk (second order, the semi-implicit factor at dt 2/3)
    pfc_op op = p->ops[0];
    double dt = p->dt;
    if (scheme == PFC_STABILIZED) op.r += S;
    if (scheme == PFC_SBDF2) dt = 2.0 * p->dt / 3.0;
    const double kmax = M_PI / p->dx;
    if (min_implicit(&op, 1, 0.0, dt, kmax * kmax * p->ndim) <= 0.0 ||
        (scheme == PFC_SBDF2 && min_implicit(p->ops, 1, 0.0, p->dt, kmax * kmax * p->ndim) <= 0.0))
        return fail(PFC_ERR_UNSTABLE_OPERATOR, "the scheme's implicit factor is not positive on the grid");
    PFC_CUDA(cudaStreamSynchronize(p->stream));
    if (scheme == PFC_SBDF2 && !p->X2) {
        PFC_CUDA(cudaMalloc(&p->X2, p->half_cap));
        if (cudaError_t e = cudaMalloc(&p->C2, p->half_cap); e != cudaSuccess) {
            cudaFree(p->X2);
            p->X2 = nullptr;
            return fail(e == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA,
                        std::string("time levels: ") + cudaGetErrorString(e));
        }
        PFC_CUDA(cudaMemset(p->X2, 0, p->half_cap));
        PFC_CUDA(cudaMemset(p->C2, 0, p->half_cap));
        p->lv_cap = p->half_cap;
        p->scratch += 2 * p->half_cap;
    }
    p->scheme = scheme;
    p->stab = scheme == PFC_STABILIZED ? S : 0.0;
    if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
    return PFC_OK;
}

pfc_status pfc_record_bytes(pfc_plan *p, int64_t nsteps, int64_t *bytes_out) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (nsteps < 1 || !bytes_out) return fail(PFC_ERR_INVALID_ARG, "nsteps must be >= 1 and bytes_out non-null");
    pfc_status s = segment_supported(p);
    if (s != PFC_OK) return s;
    *bytes_out = (int64_t)record_bytes(p, nsteps);
    return PFC_OK;
}

pfc_status pfc_step_record(pfc_plan *p, void *state, int64_t nsteps, void *record) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (!state || !record || nsteps < 1) return fail(PFC_ERR_INVALID_ARG, "null array or nsteps < 1");
    if ((reinterpret_cast<uintptr_t>(state) & 15) != 0 || (reinterpret_cast<uintptr_t>(record) & 255) != 0)
        return fail(PFC_ERR_INVALID_ARG, "state must be 16-byte and record 256-byte aligned");
    pfc_status s = segment_supported(p);
    if (s != PFC_OK) return s;
    return p->prec == PFC_FP64 ? record_impl<double>(p, state, nsteps, record)
                               : record_impl<float>(p, state, nsteps, record);
}

pfc_status pfc_adjoint_segment(pfc_plan *p, const void *record, int64_t nsteps, void *lam, double *dr) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (!record || !lam || !dr || nsteps < 1) return fail(PFC_ERR_INVALID_ARG, "null pointer or nsteps < 1");
    if ((reinterpret_cast<uintptr_t>(lam) & 15) != 0 || (reinterpret_cast<uintptr_t>(record) & 255) != 0)
        return fail(PFC_ERR_INVALID_ARG, "lam must be 16-byte and record 256-byte aligned");
    pfc_status s = segment_supported(p);
    if (s != PFC_OK) return s;
    return p->prec == PFC_FP64 ? segment_impl<double>(p, record, nsteps, lam, dr)
                               : segment_impl<float>(p, record, nsteps, lam, dr);
}

pfc_status pfc_hydro_create(pfc_hydro **out, int ndim, const int64_t *dims, double dx, double dt,
                            const pfc_op *op, double rho, double gamma, double a0, int precision, void *stream) {
    if (!out || !op) return fail(PFC_ERR_INVALID_ARG, "null pointer argument");
    if (!(rho > 0) || std::isnan(rho)) return fail(PFC_ERR_INVALID_ARG, "rho must be > 0 (inf allowed)");
    if (!(gamma >= 0) || !std::isfinite(gamma) || !(a0 >= 0) || !std::isfinite(a0))
        return fail(PFC_ERR_INVALID_ARG, "gamma and a0 must be finite and >= 0");
    pfc_plan *p = nullptr;
    pfc_status st = pfc_plan_create(&p, ndim, dims, dx, dt, op, 1, nullptr, precision, stream);
    if (st != PFC_OK) return st;
    pfc_hydro *h = new pfc_hydro();
    h->p = p;
    h->ndim = ndim;
    h->rho = rho;
    h->gamma = gamma;
    h->a0 = a0;
    const Geom &g = p->t.g;
    const size_t hb = (size_t)g.nstd * vbytes(p), rb = (size_t)g.nreal * vbytes(p) / 2;
    void **halves[6] = {&h->Ps, &h->Ns, &h->Mu, &h->Hw, &h->Fh, &h->Vh};
    cudaError_t e = cudaSuccess;
    for (void **b : halves)
        if (e == cudaSuccess) e = cudaMalloc(b, hb);
    if (e == cudaSuccess) e = cudaMalloc(&h->T1, rb);
    if (e == cudaSuccess) e = cudaMalloc(&h->T2, rb);
    if (e != cudaSuccess) {
        hydro_free(h);
        return fail(e == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA,
                    std::string("hydro allocation: ") + cudaGetErrorString(e));
    }
    *out = h;
    return PFC_OK;
}

pfc_status pfc_hydro_step(pfc_hydro *h, void *psi, void *v, int64_t nsteps) {
    if (!h || !plan_ok(h->p)) return fail(PFC_ERR_INVALID_ARG, "invalid hydro object");
    if (!psi || !v) return fail(PFC_ERR_INVALID_ARG, "null array");
    if (nsteps < 0) return fail(PFC_ERR_INVALID_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return PFC_OK;
    return h->p->prec == PFC_FP64 ? hydro_impl<double>(h, psi, v, nsteps) : hydro_impl<float>(h, psi, v, nsteps);
}

pfc_status pfc_hydro_destroy(pfc_hydro *h) {
    if (!h) return PFC_OK;
    if (h->p) cudaStreamSynchronize(h->p->stream);
    hydro_free(h);
    return PFC_OK;
}

pfc_status pfc_sync(pfc_plan *p) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    return read_status(p);
}

pfc_status pfc_plan_info(pfc_plan *p, int32_t *tiles, int64_t *scratch_bytes) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    const Geom &g = p->t.g;
    if (tiles && p->mixed) {
        // one pass per axis: Py = Pz = 0, W = the y pass' columns a block, gpc = the x pass' rows a block
        const int32_t v[11] = {0, 0, 0, 0, p->mr_W[1], p->mr_rows, 32 * p->mr_rows, 32 * p->mr_W[1], 0, 1, 1};
        std::memcpy(tiles, v, sizeof(v));
    } else if (tiles) {
        const int32_t v[11] = {g.Py, g.Pz, g.Qy, g.Qz, g.W, g.gpc, p->t.nt_row, p->t.nt_line, p->t.row_cs,
                               g.Ry, g.Rz};
        std::memcpy(tiles, v, sizeof(v));
    }
    if (scratch_bytes) *scratch_bytes = (int64_t)p->scratch;
    return PFC_OK;
}

pfc_status pfc_plan_autotune(pfc_plan *p, int max_candidates, int trial_steps, const char *cache_path,
                             double *best_ms_out) {
    if (!plan_ok(p)) return fail(PFC_ERR_INVALID_ARG, "invalid plan");
    if (max_candidates < 1 || trial_steps < 1) return fail(PFC_ERR_INVALID_ARG, "max_candidates and trial_steps must be >= 1");
    if (p->mixed)
        return p->prec == PFC_FP64 ? mr_autotune<double>(p, max_candidates, trial_steps, best_ms_out)
                                   : mr_autotune<float>(p, max_candidates, trial_steps, best_ms_out);
    const size_t smem_max = smem_optin();
    if (!smem_max) return fail(PFC_ERR_CUDA, "device query failed");
    const std::string key = tune_key(p);
    const Tiles before = p->t;
    if (!cache_path) cache_path = std::getenv("PFC_AUTOTUNE_CACHE");
    if (cache_path && !cache_path[0]) cache_path = nullptr;
    if (cache_path) {
        TileChoice c;
        double ms = 0;
        Tiles t;
        if (tune_cache_lookup(cache_path, key, c, ms) &&
            plan_tiles_as(t, c, p->nx, p->ny, p->nz, vbytes(p), p->ntile, smem_max) &&
            (p->nfields == 1 || t.nt_line <= 512)) {
            pfc_status st = apply_tiles(p, t);
            if (st != PFC_OK) return st;
            if (best_ms_out) *best_ms_out = ms;
            return PFC_OK;
        }
    }
    // candidates in the planner's order (its own choice first), each also without the clustered
    // row pass where it has one; line blocks no larger than the planner's (or 512 threads), so
    // that every call the plan supported (the adjoint, the coupled pass) stays supported
    const int max_line = std::max(512, before.nt_line);
    std::vector<std::pair<TileChoice, Tiles>> cand;
    // the pass schedule is a choice too: two-pass tilings first (5 sweeps a step), then, for
    // single-field plans, up to two three-pass tilings (9 sweeps, but line tiles R times shorter)
    std::vector<TileChoice> choices = tile_candidates(p->nx, p->ny, p->nz, vbytes(p), p->ntile, smem_max);
    if (p->nfields == 1 && before.g.R == 1) {
        std::vector<TileChoice> three =
            tile_candidates(p->nx, p->ny, p->nz, vbytes(p), p->ntile, smem_max, TileChoice{}, 1, SCHED_THREE);
        const int keep = std::min<int>(2, (int)three.size());
        const int room = std::max(0, max_candidates - keep);
        if ((int)choices.size() > room) choices.resize(room);
        choices.insert(choices.end(), three.begin(), three.begin() + keep);
    }
    for (const TileChoice &c0 : choices) {
        for (int cl = 1; cl >= 0 && (int)cand.size() < max_candidates; --cl) {
            TileChoice c = c0;
            c.cluster = cl;
            Tiles t;
            if (!plan_tiles_as(t, c, p->nx, p->ny, p->nz, vbytes(p), p->ntile, smem_max)) break;
            if (t.nt_line > max_line || (p->nfields == 2 && t.nt_line > 512)) break;
            cand.push_back({c, t});
            if (t.row_cs == 0) break;   // no clustered variant to compare against
        }
        if ((int)cand.size() >= max_candidates) break;
    }
    if (cand.empty()) return fail(PFC_ERR_UNSUPPORTED, "no tiling to try");
    const size_t rbytes = p->prec == PFC_FP64 ? 8 : 4;
    void *tmp = nullptr;
    PFC_CUDA(cudaMalloc(&tmp, (size_t)p->t.g.nreal * p->nfields * rbytes));
    // a zero field is a fixed point of the step: the timed work is the real work on finite data
    cudaError_t e = cudaMemsetAsync(tmp, 0, (size_t)p->t.g.nreal * p->nfields * rbytes, p->stream);
    if (e != cudaSuccess) {
        cudaFree(tmp);
        return fail(PFC_ERR_CUDA, std::string("autotune state: ") + cudaGetErrorString(e));
    }
    int best = -1;
    double best_ms = 1e300;
    pfc_status st = PFC_OK;
    for (size_t i = 0; i < cand.size(); ++i) {
        if ((st = apply_tiles(p, cand[i].second)) != PFC_OK) break;
        double ms = 0;
        if ((st = time_steps(p, tmp, trial_steps, &ms)) != PFC_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = (int)i;
        }
    }
    cudaFree(tmp);
    if (st != PFC_OK) {
        const std::string msg = pfc_last_error();
        apply_tiles(p, before);
        return fail(st, "autotune: " + msg);
    }
    if ((st = apply_tiles(p, cand[best].second)) != PFC_OK) return st;
    if (cache_path) tune_cache_store(cache_path, key, cand[best].first, best_ms);
    if (best_ms_out) *best_ms_out = best_ms;
    return PFC_OK;
}

}  // extern "C"
