// Batched ensemble of independent 2D one-mode domains of uneven sizes (pfc_batch_* of pfc.h).
//
// Domains are grouped by size class (ny, nx). Within a class a domain is one member of each
// launch (the member index is blockIdx.y of the row pass and blockIdx.z of the line pass), with
// its r and its FP64 mean read from device arrays and its place in the caller's packed state
// from an offset table. The nsteps loop runs as a CUDA graph captured once per batch: every
// size class gets its own branch (a forked stream), so classes proceed concurrently and each
// class carries its own chain of row and line passes.
//
// Classes small enough for one block's shared memory (both extents <= 128, two half spectra in
// the opt-in limit) are on-chip classes instead: one launch per call, one block per member, all
// nsteps steps in shared memory (k_onchip, pfc_onchip.cuh), on the class's own stream beside the
// graph. PFC_ONCHIP=0 keeps every class on the two-pass path (to compare the two).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>

#include "pfc_host.h"

using namespace pfc;

namespace {

constexpr int BATCH_GRAPH_CHUNK = 16;
constexpr int BATCH_LTAB = 9;   // tables for 512 points serve every class

struct BatchClass {
    int ny = 0, nx = 0;
    Tiles t{};
    std::vector<int> members;   // domain indices, in class order
    int cbase = 0;              // first class-major slot of this class
    void *X = nullptr, *C = nullptr, *r = nullptr;
    int64_t *moff = nullptr;    // device: member offsets into the packed state
    cudaStream_t s = nullptr;
    size_t cap = 0;             // bytes allocated for each of X and C
    bool onchip = false;        // stepped in shared memory by k_onchip (no X, C)
    size_t smem_oc = 0;         // its shared memory per block
    // persistent schedule: the class's tiling there (line tiles of the launch's block size) or
    // on-chip stepping inside the launch
    Tiles tp{};
    bool p_onchip = false;
};


}  // namespace

struct pfc_batch {
    int nd = 0, prec = PFC_FP32_MIXED;
    double dx = 0, dt = 0;
    cudaStream_t stream = nullptr;
    std::vector<BatchClass> cls;
    std::vector<int> slot_of;       // domain -> class-major slot
    int64_t *d_off = nullptr, *d_n = nullptr;   // class-major offsets and sizes
    double *d_mean = nullptr;       // class-major means
    int *d_status = nullptr;
    void *tw = nullptr, *stw = nullptr;
    size_t smem_row = 0, smem_line = 0;
    size_t smem_oc = 0;             // shared memory of the on-chip classes' launches (largest)
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    bool destroyed = false;
    // persistent schedule (pfc_batch_set_schedule)
    int sched = PFC_BATCH_GRAPH;
    int p_nt = 128;                  // threads a block
    size_t p_oc_max = 0;             // largest on-chip shared memory allowed in the launch
    double p_oc_share = -1.0;        // share of the blocks for on-chip members (< 0: by points)
    bool p_ready = false;            // tilings, items and arrays prepared
    int p_grid = 0, p_oc_blocks = 0;
    size_t p_smem = 0;
    int n_mean = 0, n_row = 0, n_line = 0, n_oc = 0;
    int2 *d_mean_items = nullptr, *d_oc_items = nullptr;
    int4 *d_row_items = nullptr, *d_line_items = nullptr;
    unsigned *d_sync = nullptr;
    long long p_budget = 0;          // clock64 cycles a barrier wait may take
    int p_extra = 0;
    void *p_args = nullptr;          // PbArgs<R> of the launch (host copy)
    cudaGraph_t p_graph = nullptr;
    cudaGraphExec_t p_exec = nullptr;
    const void *p_state = nullptr;   // the state and step count the graph was captured for
    int64_t p_nsteps = -1;
    bool p_graph_ok = true;          // false once capturing the launch failed (launched directly)
    cudaStream_t p_cap = nullptr;
    const void *p_pair_state = nullptr;
    // an attached coupled pair (pfc_batch_attach_pair), stepped inside the persistent launch
    bool has_pair = false;
    int pair_ndim = 0;
    int pair_n[3] = {1, 1, 1};       // nx, ny, nz
    pfc_op pair_ops[2]{};
    double pair_alpha = 0;
    Tiles pair_t{};
    void *pair_X = nullptr, *pair_C = nullptr;
    size_t pair_cap = 0;
    int64_t *pair_moff = nullptr;    // device {0, N}: the fields' offsets in the pair's state
    double *pair_mean = nullptr;     // device: the fields' FP64 means
};

namespace {

#define PFC_BCUDA(call)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return set_error(e_ == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA, \
                             std::string(#call) + ": " + cudaGetErrorString(e_));                \
    } while (0)

// each class launches with its own shared-memory size (the kernels' attribute is the maximum)
LaunchCfg bcfg(const pfc_batch *, const BatchClass &c, cudaStream_t s) {
    return LaunchCfg{c.t.g, c.t.nt_row, c.t.nt_line, c.t.smem_row, c.t.smem_line, s};
}

template <typename R> StageTw<typename VT<R>::V> bstage(const pfc_batch *b) {
    using V = typename VT<R>::V;
    const V *p = reinterpret_cast<const V *>(b->stw);
    return StageTw<V>{p, p + STW8, p + STW8 + STW4};
}

template <typename R> RowArgs<R> brow(const pfc_batch *b, const BatchClass &c) {
    RowArgs<R> a{};
    a.tw = reinterpret_cast<const typename VT<R>::V *>(b->tw);
    a.st = bstage<R>(b);
    a.scale = (R)1;
    a.mean = b->d_mean + c.cbase;
    a.moff = c.moff;
    return a;
}

template <typename R> void enqueue_class_step(const pfc_batch *b, const BatchClass &c, cudaStream_t s) {
    const Geom &g = c.t.g;
    const int nm = (int)c.members.size();
    RowArgs<R> ra = brow<R>(b, c);
    ra.in = c.X;
    ra.out = c.C;
    ra.proj = c.X;
    launch_row<R>(bcfg(b, c, s), ROW_CUBE, ra, nm);
    LineArgs<R> la{};
    la.x = c.X;
    la.c = c.C;
    la.scale = (R)1;
    la.st = bstage<R>(b);
    const double two_pi = 6.28318530717958647692528676655900576839;
    la.up.dt = (R)b->dt;
    la.up.cx = (R)(two_pi / (g.nx * b->dx));
    la.up.cy = (R)(two_pi / (g.ny * b->dx));
    la.up.cz = (R)(two_pi / (g.nz * b->dx));
    la.up.invQ = (R)(1.0 / g.Q);
    la.up.inv_halfN = (R)(2.0 / (double)g.nreal);
    la.up.op[0] = la.up.op[1] = OpR<R>{PFC_ONE_MODE, (R)0, (R)0, (R)0};
    la.rmem = reinterpret_cast<const R *>(c.r);
    launch_line<R>(bcfg(b, c, s), LINE_STEP, la, nm);
}

// nsteps steps of every class, each class on its own stream forked from `origin` and joined
// back into it (used both while capturing the graph and for the remainder steps).
template <typename R> pfc_status enqueue_steps(pfc_batch *b, cudaStream_t origin, int64_t nsteps) {
    PFC_BCUDA(cudaEventRecord(b->ev_fork, origin));
    for (size_t i = 0; i < b->cls.size(); ++i) {
        BatchClass &c = b->cls[i];
        if (c.onchip) continue;
        PFC_BCUDA(cudaStreamWaitEvent(c.s, b->ev_fork, 0));
        for (int64_t k = 0; k < nsteps; ++k) enqueue_class_step<R>(b, c, c.s);
        PFC_BCUDA(cudaEventRecord(b->ev_join[i], c.s));
        PFC_BCUDA(cudaStreamWaitEvent(origin, b->ev_join[i], 0));
    }
    PFC_BCUDA(cudaGetLastError());
    return PFC_OK;
}

template <typename R> pfc_status persist_step(pfc_batch *b, void *state, int64_t nsteps, void *pair_state);

template <typename R> pfc_status batch_step_impl(pfc_batch *b, void *state, int64_t nsteps) {
    if (b->sched == PFC_BATCH_PERSISTENT) return persist_step<R>(b, state, nsteps, nullptr);
    launch_batch_mean<R>(b->stream, reinterpret_cast<const R *>(state), b->d_off, b->d_n, b->nd,
                         b->d_mean, b->d_status);
    for (BatchClass &c : b->cls) {
        if (c.onchip) continue;
        RowArgs<R> ra = brow<R>(b, c);
        ra.in = state;
        ra.out = c.X;
        ra.scale = (R)(1.0 / ((double)c.t.g.P * (double)c.t.g.M));
        launch_row<R>(bcfg(b, c, b->stream), ROW_FWD, ra, (int)c.members.size());
    }
    PFC_BCUDA(cudaGetLastError());
    // on-chip classes: every step of the call in one launch per class, on the class's stream
    bool any_onchip = false;
    PFC_BCUDA(cudaEventRecord(b->ev_fork, b->stream));
    for (size_t i = 0; i < b->cls.size(); ++i) {
        BatchClass &c = b->cls[i];
        if (!c.onchip) continue;
        any_onchip = true;
        PFC_BCUDA(cudaStreamWaitEvent(c.s, b->ev_fork, 0));
        OnchipArgs<R> oa{};
        oa.state = state;
        oa.moff = c.moff;
        oa.mean = b->d_mean + c.cbase;
        oa.r = reinterpret_cast<const R *>(c.r);
        oa.nsteps = nsteps;
        const Geom &g = c.t.g;
        const double two_pi = 6.28318530717958647692528676655900576839;
        oa.up.dt = (R)b->dt;
        oa.up.cx = (R)(two_pi / (g.nx * b->dx));
        oa.up.cy = (R)(two_pi / (g.ny * b->dx));
        oa.up.inv_halfN = (R)(2.0 / (double)g.nreal);
        oa.up.op[0] = OpR<R>{PFC_ONE_MODE, (R)0, (R)0, (R)0};
        oa.tw = reinterpret_cast<const typename VT<R>::V *>(b->tw);
        oa.st = bstage<R>(b);
        launch_onchip<R>(c.s, g, oa, (int)c.members.size(), c.smem_oc);
        PFC_BCUDA(cudaGetLastError());
        PFC_BCUDA(cudaEventRecord(b->ev_join[i], c.s));
    }
    if (nsteps >= BATCH_GRAPH_CHUNK && !b->graph) {
        cudaStream_t cap;
        PFC_BCUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        pfc_status st = PFC_OK;
        if (e == cudaSuccess) {
            st = enqueue_steps<R>(b, cap, BATCH_GRAPH_CHUNK);
            e = cudaStreamEndCapture(cap, &graph);
        }
        if (e == cudaSuccess && st == PFC_OK) {
            e = cudaGraphInstantiate(&b->graph, graph, 0);
            cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cap);
        if (st != PFC_OK) return st;
        if (e != cudaSuccess) return set_error(PFC_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    int64_t done = 0;
    if (b->graph)
        for (; done + BATCH_GRAPH_CHUNK <= nsteps; done += BATCH_GRAPH_CHUNK)
            PFC_BCUDA(cudaGraphLaunch(b->graph, b->stream));
    if (done < nsteps) {
        pfc_status st = enqueue_steps<R>(b, b->stream, nsteps - done);
        if (st != PFC_OK) return st;
    }
    for (BatchClass &c : b->cls) {
        if (c.onchip) continue;
        RowArgs<R> ra = brow<R>(b, c);
        ra.in = c.X;
        ra.out = state;
        launch_row<R>(bcfg(b, c, b->stream), ROW_INV, ra, (int)c.members.size());
    }
    if (any_onchip)
        for (size_t i = 0; i < b->cls.size(); ++i)
            if (b->cls[i].onchip) PFC_BCUDA(cudaStreamWaitEvent(b->stream, b->ev_join[i], 0));
    PFC_BCUDA(cudaGetLastError());
    return PFC_OK;
}

// Autotune one class: time up to max_candidates tilings (the planner's order, its own choice
// first) on trial_steps class steps of zero fields (a fixed point of the step), keep the fastest.
template <typename R> void free_persist(pfc_batch *b);

template <typename R>
pfc_status tune_class(pfc_batch *b, BatchClass &c, int max_candidates, int trial_steps, size_t smem_max,
                      double *ms_out) {
    const size_t vb = sizeof(R) * 2;
    const int nm = (int)c.members.size();
    std::vector<Tiles> cand;
    for (const TileChoice &tc : tile_candidates(c.nx, c.ny, 1, vb, 2, smem_max, TileChoice{}, nm)) {
        Tiles t;
        if (!plan_tiles_as(t, tc, c.nx, c.ny, 1, vb, 2, smem_max, nm) || t.nt_line > 512) continue;
        t.g.ltab = BATCH_LTAB;
        cand.push_back(t);
        if ((int)cand.size() >= max_candidates) break;
    }
    if (cand.empty()) return set_error(PFC_ERR_UNSUPPORTED, "no tiling to try for a domain size");
    cudaEvent_t e0, e1;
    PFC_BCUDA(cudaEventCreate(&e0));
    if (cudaError_t e1err = cudaEventCreate(&e1); e1err != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(PFC_ERR_CUDA, std::string("batch autotune events: ") + cudaGetErrorString(e1err));
    }
    // switch the class to tiling t; on failure the class keeps its arrays and tiling
    auto use = [&](const Tiles &t) -> cudaError_t {
        const size_t need = (size_t)t.g.nhalf * vb * nm;
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e == cudaSuccess && need > c.cap) {
            void *x = nullptr, *y = nullptr;
            if ((e = cudaMalloc(&x, need)) != cudaSuccess) return e;
            if ((e = cudaMalloc(&y, need)) != cudaSuccess) {
                cudaFree(x);
                return e;
            }
            cudaFree(c.X);
            cudaFree(c.C);
            c.X = x;
            c.C = y;
            c.cap = need;
            free_persist<R>(b);   // its launch arguments held the old arrays
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(c.X, 0, c.cap, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c.C, 0, c.cap, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_mean + c.cbase, 0, nm * sizeof(double), b->stream);
        const LaunchCfg lc{t.g, t.nt_row, t.nt_line, t.smem_row, t.smem_line, b->stream};
        if (e == cudaSuccess) e = raise_smem_attrs<R>(lc);
        if (e == cudaSuccess) c.t = t;
        return e;
    };
    cudaError_t e = cudaSuccess;
    int best = -1;
    double best_ms = 1e300;
    for (size_t i = 0; i < cand.size() && e == cudaSuccess; ++i) {
        if ((e = use(cand[i])) != cudaSuccess) break;
        for (int k = 0; k < trial_steps; ++k) enqueue_class_step<R>(b, c, b->stream);
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            float t = 0.f;
            e = cudaEventRecord(e0, b->stream);
            for (int k = 0; k < trial_steps; ++k) enqueue_class_step<R>(b, c, b->stream);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && (double)t / trial_steps < best_ms) {
                best_ms = (double)t / trial_steps;
                best = (int)i;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = use(cand[best]);
    if (e != cudaSuccess) return set_error(PFC_ERR_CUDA, std::string("batch autotune: ") + cudaGetErrorString(e));
    *ms_out = best_ms;
    return PFC_OK;
}

// ---- persistent schedule ----

// Line tiles of exactly nt threads (Q W = 8 nt) for a class of the persistent launch: the
// candidate the planner scores best among them (one-axis tiles, up to 128 columns).
// ntile: line tiles in shared memory (2; 3 for the coupled pair's update). Among the tilings,
// those whose shared memory (the larger of the row and line pass) fits smem_pref come first,
// then the planner's score: the launch's blocks all take the largest shared memory of any
// class, so one greedy class would lower the blocks an SM holds for every class.
bool persist_tiles(Tiles &t, int nx, int ny, int nz, size_t vb, int nt, size_t smem_max, int members,
                   int ntile, int ltab, size_t smem_pref) {
    const Geom g0 = grid_geom(nx, ny, nz);
    bool found = false, best_fit = false;
    long best = LONG_MIN;
    for (int Py = 1; Py <= 8; Py *= 2)
        for (int Pz = 1; Pz <= (nz > 1 ? 8 : 1); Pz *= 2)
            for (int W = 1; W <= 128; W *= 2) {
                if (ny % Py || nz % Pz || (int64_t)(ny / Py) * (nz / Pz) * W != 8 * (int64_t)nt) continue;
                const long sc = tile_score(g0, Py, Pz, W, vb, ntile, smem_max, false, ilog2(nt), 1, 1, 128);
                if (sc == LONG_MIN) continue;
                TileChoice c;
                c.Py = Py;
                c.Pz = Pz;
                c.W = W;
                c.cluster = 0;
                Tiles tc;
                if (!plan_tiles_as(tc, c, nx, ny, nz, vb, ntile, smem_max, members, 128) || tc.nt_line != nt) continue;
                const bool fit = std::max(tc.smem_row, tc.smem_line) <= smem_pref;
                if (!found || (fit && !best_fit) || (fit == best_fit && sc > best)) {
                    found = true;
                    best_fit = fit;
                    best = sc;
                    t = tc;
                }
            }
    if (!found) return false;
    t.g.ltab = ltab;
    return true;
}

template <typename R> void free_persist(pfc_batch *b) {
    if (b->p_exec) cudaGraphExecDestroy(b->p_exec);
    if (b->p_graph) cudaGraphDestroy(b->p_graph);
    b->p_exec = nullptr;
    b->p_graph = nullptr;
    b->p_state = nullptr;
    b->p_nsteps = -1;
    cudaFree(b->d_mean_items); cudaFree(b->d_oc_items); cudaFree(b->d_row_items); cudaFree(b->d_line_items);
    b->d_mean_items = b->d_oc_items = nullptr;
    b->d_row_items = b->d_line_items = nullptr;
    delete reinterpret_cast<PbArgs<R> *>(b->p_args);
    b->p_args = nullptr;
    b->p_ready = false;
}

template <typename R> cudaError_t persist_occ(int nt, size_t smem, int *bps) {
    return nt == 512   ? persist_occupancy<R, 512>(smem, bps)
           : nt == 256 ? persist_occupancy<R, 256>(smem, bps)
                       : persist_occupancy<R, 128>(smem, bps);
}

template <typename R> cudaError_t persist_launch(const pfc_batch *b, const PbArgs<R> &a, cudaStream_t s) {
    return b->p_nt == 512   ? launch_batch_persist<R, 512>(a, b->p_grid, b->p_smem, s)
           : b->p_nt == 256 ? launch_batch_persist<R, 256>(a, b->p_grid, b->p_smem, s)
                            : launch_batch_persist<R, 128>(a, b->p_grid, b->p_smem, s);
}

// Tilings, class arrays, work items and launch shape of the persistent schedule.
template <typename R> pfc_status persist_prepare(pfc_batch *b) {
    using V = typename VT<R>::V;
    free_persist<R>(b);
    const size_t vb = sizeof(V);
    int dev = 0, optin = 0, nsm = 0, clk_khz = 0;
    PFC_BCUDA(cudaGetDevice(&dev));
    PFC_BCUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    PFC_BCUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev) != cudaSuccess || clk_khz <= 0) clk_khz = 2000000;
    // a barrier wait may take two seconds (a phase takes well under a millisecond)
    if (b->p_budget <= 0) b->p_budget = (long long)clk_khz * 2000;
    if (b->cls.size() > (size_t)PB_MAXC) return set_error(PFC_ERR_UNSUPPORTED, "too many size classes for one persistent launch");
    const int nt = b->p_nt;
    // shared memory a block may take while four blocks fit an SM (the pass bodies' 16 named
    // barriers a block allow at most four)
    int smem_sm = 0;
    PFC_BCUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    // (1 KB a block is reserved by the hardware, 8 B are the kernel's static shared memory)
    const size_t smem_pref = (size_t)smem_sm / 4 > 1032 ? (size_t)smem_sm / 4 - 1032 : 0;
    // Which classes run on chip: those with no tiling of the block size (both extents <= 128),
    // and, when oc_max > 0, those whose two half spectra fit oc_max. (Inside this launch the
    // on-chip body runs at the launch's register budget of 64 a thread, far below the 214 of its
    // own kernel, and its spills make it slower than the two-pass items: on the 1024-domain
    // ensemble, putting the 64 x 64 class on chip lowered the rate from 4.1e10 to 3.4e10.)
    const size_t nclass = b->cls.size();
    std::vector<Tiles> tl(nclass);
    std::vector<char> tp_ok(nclass), oc_able(nclass);
    std::vector<size_t> oc_smem(nclass);
    size_t smem = 0;
    for (size_t i = 0; i < nclass; ++i) {
        BatchClass &c = b->cls[i];
        oc_smem[i] = onchip_smem(c.ny, c.nx, vb);
        oc_able[i] = c.ny <= ONCHIP_MAX && c.nx <= ONCHIP_MAX && oc_smem[i] <= (size_t)optin;
        tp_ok[i] = persist_tiles(tl[i], c.nx, c.ny, 1, vb, nt, (size_t)optin, (int)c.members.size(), 2, BATCH_LTAB,
                                 smem_pref);
        if (!tp_ok[i] && !oc_able[i])
            return set_error(PFC_ERR_UNSUPPORTED, "no tiling of a domain size fills the persistent launch's blocks");
        c.p_onchip = !tp_ok[i];
        smem = std::max(smem, c.p_onchip ? oc_smem[i] : std::max(tl[i].smem_row, tl[i].smem_line));
    }
    if (b->p_oc_max > 0) {
        const size_t oc_max = std::min(b->p_oc_max, (size_t)optin);
        for (size_t i = 0; i < nclass; ++i)
            if (oc_able[i] && tp_ok[i] && oc_smem[i] <= oc_max) {
                b->cls[i].p_onchip = true;
                smem = std::max(smem, oc_smem[i]);
            }
    }
    double pts_oc = 0, pts_tp = 0;
    for (size_t i = 0; i < nclass; ++i) {
        BatchClass &c = b->cls[i];
        const int nm = (int)c.members.size();
        if (c.p_onchip) {
            pts_oc += (double)c.ny * c.nx * nm;
            continue;
        }
        const Tiles &t = tl[i];
        c.tp = t;
        pts_tp += (double)c.ny * c.nx * nm;
        const size_t need = (size_t)t.g.nhalf * vb * nm;
        if (need > c.cap) {
            void *x = nullptr, *y = nullptr;
            PFC_BCUDA(cudaStreamSynchronize(b->stream));
            PFC_BCUDA(cudaMalloc(&x, need));
            if (cudaError_t e = cudaMalloc(&y, need); e != cudaSuccess) {
                cudaFree(x);
                return set_error(PFC_ERR_OUT_OF_MEMORY, std::string("persistent batch arrays: ") + cudaGetErrorString(e));
            }
            cudaFree(c.X);
            cudaFree(c.C);
            c.X = x;
            c.C = y;
            c.cap = need;
            // the graph schedule's captured graph held the old arrays: captured again when used
            if (b->graph) {
                cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
            }
        }
    }
    // an attached coupled pair: its tiling (three line tiles for the 2x2 update) and arrays
    if (b->has_pair) {
        if (nclass + 1 > (size_t)PB_MAXC)
            return set_error(PFC_ERR_UNSUPPORTED, "too many size classes for one persistent launch");
        Tiles t;
        if (!persist_tiles(t, b->pair_n[0], b->pair_n[1], b->pair_n[2], vb, nt, (size_t)optin, 2, 3, BATCH_LTAB,
                           smem_pref))
            return set_error(PFC_ERR_UNSUPPORTED, "no tiling of the coupled pair's grid fills the persistent launch's blocks");
        b->pair_t = t;
        smem = std::max(smem, std::max(t.smem_row, t.smem_line));
        pts_tp += 2.0 * (double)t.g.nreal;
        const size_t need = 2 * (size_t)t.g.nhalf * vb;
        if (need > b->pair_cap) {
            PFC_BCUDA(cudaStreamSynchronize(b->stream));
            cudaFree(b->pair_X);
            cudaFree(b->pair_C);
            b->pair_X = b->pair_C = nullptr;
            b->pair_cap = 0;
            PFC_BCUDA(cudaMalloc(&b->pair_X, need));
            PFC_BCUDA(cudaMalloc(&b->pair_C, need));
            b->pair_cap = need;
        }
        const int64_t moff[2] = {0, t.g.nreal};
        PFC_BCUDA(cudaMemcpy(b->pair_moff, moff, sizeof(moff), cudaMemcpyHostToDevice));
    }
    smem = std::max(smem, (size_t)nt * sizeof(double));   // the mean reduction's buffer
    int bps = 0;
    PFC_BCUDA(persist_occ<R>(nt, smem, &bps));
    if (bps < 1) return set_error(PFC_ERR_UNSUPPORTED, "the persistent kernel does not fit an SM with this shared memory");

    // classes and work items
    auto *pa = new PbArgs<R>();
    b->p_args = pa;
    std::vector<std::pair<int64_t, int2>> mi, oi;
    std::vector<std::pair<int64_t, int4>> ri, li;
    const double two_pi = 6.28318530717958647692528676655900576839;
    const V *tw = reinterpret_cast<const V *>(b->tw);
    for (size_t ci = 0; ci < b->cls.size(); ++ci) {
        BatchClass &c = b->cls[ci];
        PbClass<R> &pc = pa->cls[ci];
        const int nm = (int)c.members.size();
        Geom g;
        if (c.p_onchip) {
            g = grid_geom(c.nx, c.ny, 1);
            g.nreal = (int64_t)c.nx * c.ny;
            g.ltab = BATCH_LTAB;
        } else {
            g = c.tp.g;
        }
        pc.g = g;
        RowArgs<R> ra{};
        ra.tw = tw;
        ra.st = bstage<R>(b);
        ra.mean = b->d_mean + c.cbase;
        ra.moff = c.moff;
        pc.fwd = pc.cube = pc.inv = ra;
        pc.fwd.scale = (R)(1.0 / ((double)g.P * (double)g.M));
        pc.cube.scale = pc.inv.scale = (R)1;
        LineArgs<R> la{};
        la.scale = (R)1;
        la.st = bstage<R>(b);
        la.up.dt = (R)b->dt;
        la.up.cx = (R)(two_pi / (g.nx * b->dx));
        la.up.cy = (R)(two_pi / (g.ny * b->dx));
        la.up.cz = (R)(two_pi / (g.nz * b->dx));
        la.up.inv_halfN = (R)(2.0 / (double)g.nreal);
        la.up.op[0] = la.up.op[1] = OpR<R>{PFC_ONE_MODE, (R)0, (R)0, (R)0};
        la.rmem = reinterpret_cast<const R *>(c.r);
        if (c.p_onchip) {
            pc.line = la;
            for (int m = 0; m < nm; ++m) oi.push_back({(int64_t)c.ny * c.nx, int2{(int)ci, m}});
            continue;
        }
        la.up.invQ = (R)(1.0 / g.Q);
        la.x = c.X;
        la.c = c.C;
        pc.line = la;
        pc.fwd.out = c.X;
        pc.cube.in = c.X;
        pc.cube.out = c.C;
        pc.cube.proj = c.X;
        pc.inv.in = c.X;
        const int64_t rcost = (int64_t)g.gpc * g.P * (g.M + 1), lcost = (int64_t)g.Q * g.W;
        for (int m = 0; m < nm; ++m) {
            mi.push_back({g.nreal, int2{(int)ci, m}});
            for (int bx = 0; bx < g.QR / g.gpc; ++bx) ri.push_back({rcost, int4{(int)ci, m, bx, 0}});
            for (int kp = 0; kp < g.P * g.R; ++kp)
                for (int cg = 0; cg < g.ncg; ++cg) li.push_back({lcost, int4{(int)ci, m, cg, kp}});
        }
    }
    pa->pair_ci = -1;
    if (b->has_pair) {
        const int pci = (int)b->cls.size();
        const Geom &g = b->pair_t.g;
        PbClass<R> &pc = pa->cls[pci];
        pc.g = g;
        RowArgs<R> ra{};
        ra.tw = tw;
        ra.st = bstage<R>(b);
        ra.mean = b->pair_mean;
        ra.moff = b->pair_moff;
        pc.fwd = pc.cube = pc.inv = ra;
        pc.fwd.scale = (R)(1.0 / ((double)g.P * (double)g.M));
        pc.cube.scale = pc.inv.scale = (R)1;
        pc.fwd.out = b->pair_X;
        pc.cube.in = b->pair_X;
        pc.cube.out = b->pair_C;
        pc.cube.proj = b->pair_X;
        pc.inv.in = b->pair_X;
        Step2Args<R> a2{};
        a2.x0 = b->pair_X;
        a2.x1 = reinterpret_cast<V *>(b->pair_X) + g.nhalf;
        a2.c0 = b->pair_C;
        a2.c1 = reinterpret_cast<const V *>(b->pair_C) + g.nhalf;
        a2.alpha = (R)b->pair_alpha;
        a2.up.dt = (R)b->dt;
        a2.up.cx = (R)(two_pi / (g.nx * b->dx));
        a2.up.cy = (R)(two_pi / (g.ny * b->dx));
        a2.up.cz = (R)(two_pi / (g.nz * b->dx));
        a2.up.invQ = (R)(1.0 / g.Q);
        a2.up.inv_halfN = (R)(2.0 / (double)g.nreal);
        for (int f = 0; f < 2; ++f) {
            const pfc_op &o = b->pair_ops[f];
            a2.up.op[f] = OpR<R>{o.kind, (R)o.r, (R)o.R1, (R)(o.q2 * o.q2)};
        }
        a2.st = bstage<R>(b);
        pa->pair = a2;
        pa->pair_ci = pci;
        const int64_t rcost = (int64_t)g.gpc * g.P * (g.M + 1), lcost = 2 * (int64_t)g.Q * g.W;
        for (int f = 0; f < 2; ++f) {
            mi.push_back({g.nreal, int2{pci, f}});
            for (int bx = 0; bx < g.QR / g.gpc; ++bx) ri.push_back({rcost, int4{pci, f, bx, 0}});
        }
        for (int kp = 0; kp < g.P * g.R; ++kp)
            for (int cg = 0; cg < g.ncg; ++cg) li.push_back({lcost, int4{pci, 0, cg, kp}});
    }
    // largest first; equal costs keep class, member and block order
    auto by_cost = [](const auto &x, const auto &y) { return x.first > y.first; };
    std::stable_sort(mi.begin(), mi.end(), by_cost);
    std::stable_sort(oi.begin(), oi.end(), by_cost);
    std::stable_sort(ri.begin(), ri.end(), by_cost);
    std::stable_sort(li.begin(), li.end(), by_cost);
    auto upload = [&](auto &vec, auto *&dptr) -> cudaError_t {
        using T = typename std::decay_t<decltype(vec)>::value_type::second_type;
        std::vector<T> h;
        for (auto &e : vec) h.push_back(e.second);
        if (h.empty()) return cudaSuccess;
        cudaError_t e = cudaMalloc(&dptr, h.size() * sizeof(T));
        if (e == cudaSuccess) e = cudaMemcpy(dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        return e;
    };
    PFC_BCUDA(upload(mi, b->d_mean_items));
    PFC_BCUDA(upload(oi, b->d_oc_items));
    PFC_BCUDA(upload(ri, b->d_row_items));
    PFC_BCUDA(upload(li, b->d_line_items));
    if (!b->d_sync) PFC_BCUDA(cudaMalloc(&b->d_sync, PB_NSYNC * sizeof(unsigned)));
    b->n_mean = (int)mi.size();
    b->n_oc = (int)oi.size();
    b->n_row = (int)ri.size();
    b->n_line = (int)li.size();
    b->p_smem = smem;
    b->p_grid = nsm * bps;
    int ocb = 0;
    if (b->n_oc > 0) {
        if (b->n_row == 0) {
            ocb = std::min(b->p_grid, b->n_oc);
        } else {
            const double share = b->p_oc_share >= 0 ? b->p_oc_share : pts_oc / (pts_oc + pts_tp);
            ocb = (int)std::lround(share * b->p_grid);
            ocb = std::max(1, std::min(ocb, std::min(b->n_oc, b->p_grid - 1)));
        }
    }
    b->p_oc_blocks = ocb;
    pa->mean_items = b->d_mean_items;
    pa->oc_items = b->d_oc_items;
    pa->row_items = b->d_row_items;
    pa->line_items = b->d_line_items;
    pa->n_mean = b->n_mean;
    pa->n_oc = b->n_oc;
    pa->n_row = b->n_row;
    pa->n_line = b->n_line;
    pa->n_oc_blocks = ocb;
    pa->sync = b->d_sync;
    pa->status = b->d_status;
    b->p_ready = true;
    return PFC_OK;
}

// One pfc_batch_step on the persistent schedule: the sync words cleared, then the launch, as a
// graph of those two nodes captured for this state and step count (replayed while they stay the
// same), or directly when the launch could not be captured.
template <typename R> pfc_status persist_step(pfc_batch *b, void *state, int64_t nsteps, void *pair_state) {
    if (!b->p_ready) {
        pfc_status st = persist_prepare<R>(b);
        if (st != PFC_OK) return st;
    }
    PbArgs<R> &pa = *reinterpret_cast<PbArgs<R> *>(b->p_args);
    pa.state = state;
    for (size_t ci = 0; ci < b->cls.size(); ++ci) {
        pa.cls[ci].fwd.in = state;    // entry: the real state in, X' out
        pa.cls[ci].inv.out = state;   // exit: X' in, the real state out
    }
    if (pa.pair_ci >= 0) {
        pa.cls[pa.pair_ci].fwd.in = pair_state;
        pa.cls[pa.pair_ci].inv.out = pair_state;
    }
    pa.nsteps = nsteps;
    pa.budget = b->p_budget;
    pa.extra = b->p_extra;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    PFC_BCUDA(cudaStreamIsCapturing(b->stream, &cs));
    const bool direct = !b->p_graph_ok || cs != cudaStreamCaptureStatusNone;
    if (!direct && (b->p_state != state || b->p_pair_state != pair_state || b->p_nsteps != nsteps || !b->p_exec)) {
        if (b->p_exec) cudaGraphExecDestroy(b->p_exec);
        if (b->p_graph) cudaGraphDestroy(b->p_graph);
        b->p_exec = nullptr;
        b->p_graph = nullptr;
        if (!b->p_cap) PFC_BCUDA(cudaStreamCreateWithFlags(&b->p_cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(b->p_cap, cudaStreamCaptureModeThreadLocal);
        cudaError_t el = cudaSuccess;
        if (e == cudaSuccess) {
            el = cudaMemsetAsync(b->d_sync, 0, PB_NSYNC * sizeof(unsigned), b->p_cap);
            if (el == cudaSuccess) el = persist_launch<R>(b, pa, b->p_cap);
            e = cudaStreamEndCapture(b->p_cap, &b->p_graph);
        }
        if (e == cudaSuccess && el == cudaSuccess) e = cudaGraphInstantiate(&b->p_exec, b->p_graph, 0);
        if (e != cudaSuccess || el != cudaSuccess) {
            // not capturable here: launch directly from now on
            cudaGetLastError();
            if (b->p_graph) cudaGraphDestroy(b->p_graph);
            b->p_graph = nullptr;
            b->p_exec = nullptr;
            b->p_graph_ok = false;
        } else {
            b->p_state = state;
            b->p_pair_state = pair_state;
            b->p_nsteps = nsteps;
        }
    }
    if (b->p_graph_ok && !direct) {
        PFC_BCUDA(cudaGraphLaunch(b->p_exec, b->stream));
    } else {
        PFC_BCUDA(cudaMemsetAsync(b->d_sync, 0, PB_NSYNC * sizeof(unsigned), b->stream));
        PFC_BCUDA(persist_launch<R>(b, pa, b->stream));
    }
    return PFC_OK;
}

// The schedule of pfc_batch_step chosen by measurement: whole calls of trial_steps (at least 20)
// steps on a zero state (a fixed point of the step) with the graph schedule and the persistent one at
// 256, 128 and 512 threads a block; the fastest is kept.
template <typename R> pfc_status tune_schedule(pfc_batch *b, int trial_steps) {
    trial_steps = std::max(trial_steps, 20);   // the graph schedule replays its graph from 16 steps
    int64_t total = 0;
    for (const BatchClass &c : b->cls) total += (int64_t)c.ny * c.nx * (int64_t)c.members.size();
    const int64_t ptotal = b->has_pair ? 2 * (int64_t)b->pair_n[0] * b->pair_n[1] * b->pair_n[2] : 0;
    void *tmp = nullptr;
    PFC_BCUDA(cudaMalloc(&tmp, (size_t)(total + ptotal) * sizeof(R)));
    void *ptmp = b->has_pair ? reinterpret_cast<R *>(tmp) + total : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(tmp, 0, (size_t)(total + ptotal) * sizeof(R), b->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int cand[4][2] = {{PFC_BATCH_GRAPH, 0}, {PFC_BATCH_PERSISTENT, 256}, {PFC_BATCH_PERSISTENT, 128},
                            {PFC_BATCH_PERSISTENT, 512}};
    int best = -1;
    double best_ms = 1e300;
    pfc_status st = PFC_OK;
    // a call of the chosen schedule (a coupled pair attached: the persistent one only)
    auto call = [&]() {
        return b->sched == PFC_BATCH_PERSISTENT ? persist_step<R>(b, tmp, trial_steps, ptmp)
                                                : batch_step_impl<R>(b, tmp, trial_steps);
    };
    for (int i = b->has_pair ? 1 : 0; i < 4 && e == cudaSuccess && st == PFC_OK; ++i) {
        b->sched = cand[i][0];
        if (b->sched == PFC_BATCH_PERSISTENT) {
            b->p_nt = cand[i][1];
            b->p_oc_max = 0;
            b->p_oc_share = -1.0;
            if (persist_prepare<R>(b) != PFC_OK) continue;   // this block size cannot step the batch
        }
        if ((st = call()) != PFC_OK) break;
        float ms = 0.f;
        e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess && (st = call()) != PFC_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = i;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (st != PFC_OK) return st;
    if (e != cudaSuccess) return set_error(PFC_ERR_CUDA, std::string("batch schedule autotune: ") + cudaGetErrorString(e));
    if (best < 0) return set_error(PFC_ERR_UNSUPPORTED, "no persistent block size can step the batch");
    b->sched = cand[best][0];
    if (b->sched == PFC_BATCH_PERSISTENT) {
        b->p_nt = cand[best][1];
        return persist_prepare<R>(b);
    }
    return PFC_OK;
}

void free_batch(pfc_batch *b) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (BatchClass &c : b->cls) {
        cudaFree(c.X); cudaFree(c.C); cudaFree(c.r); cudaFree(c.moff);
        if (c.s) cudaStreamDestroy(c.s);
    }
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    cudaFree(b->d_off); cudaFree(b->d_n); cudaFree(b->d_mean); cudaFree(b->d_status);
    cudaFree(b->tw); cudaFree(b->stw);
    if (b->prec == PFC_FP64) free_persist<double>(b);
    else free_persist<float>(b);
    cudaFree(b->d_sync);
    if (b->p_cap) cudaStreamDestroy(b->p_cap);
    cudaFree(b->pair_X); cudaFree(b->pair_C); cudaFree(b->pair_moff); cudaFree(b->pair_mean);
    delete b;
}

}  // namespace

extern "C" {

pfc_status pfc_batch_create(pfc_batch **out, int nd, const int64_t *dims_host, const double *r_host,
                            double dx, double dt, int precision, void *stream) {
    if (!out || !dims_host || !r_host) return set_error(PFC_ERR_INVALID_ARG, "null pointer argument");
    if (nd < 1) return set_error(PFC_ERR_INVALID_ARG, "ndomains must be >= 1");
    if (!(dx > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dt))
        return set_error(PFC_ERR_INVALID_ARG, "dx and dt must be finite and > 0");
    if (precision != PFC_FP64 && precision != PFC_FP32_MIXED)
        return set_error(PFC_ERR_INVALID_ARG, "unknown precision");
    const double kmax = M_PI / dx;
    std::map<std::pair<int, int>, std::vector<int>> groups;
    const char *oc_env = std::getenv("PFC_ONCHIP");
    const bool onchip_on = !(oc_env && oc_env[0] == '0');
    for (int d = 0; d < nd; ++d) {
        const int64_t ny = dims_host[2 * d], nx = dims_host[2 * d + 1];
        if (!is_pow2(ny) || !is_pow2(nx) || ny < 16 || nx < 16 || ny > 512 || nx > 512)
            return set_error(PFC_ERR_UNSUPPORTED, "domain extents must be powers of two in [16, 512]");
        if (!std::isfinite(r_host[d])) return set_error(PFC_ERR_INVALID_ARG, "r must be finite");
        const pfc_op op{PFC_ONE_MODE, r_host[d], 0.0, 0.0};
        if (min_implicit(&op, 1, 0.0, dt, 2 * kmax * kmax) <= 0.0)
            return set_error(PFC_ERR_UNSTABLE_OPERATOR, "1 + dt k^2 Lk(k) is not positive for domain " + std::to_string(d));
        groups[{(int)ny, (int)nx}].push_back(d);
    }
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return set_error(PFC_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));

    pfc_batch *b = new pfc_batch();
    b->nd = nd;
    b->prec = precision;
    b->dx = dx;
    b->dt = dt;
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    b->slot_of.assign(nd, 0);
    const size_t vb = precision == PFC_FP64 ? 16 : 8;
    std::vector<int64_t> off_idx(nd + 1, 0);
    for (int d = 0; d < nd; ++d) off_idx[d + 1] = off_idx[d] + dims_host[2 * d] * dims_host[2 * d + 1];
    std::vector<int64_t> off_cm, n_cm;
    auto bail = [&](pfc_status s, const std::string &msg) {
        free_batch(b);
        return set_error(s, msg);
    };
    int slot = 0;
    for (auto &kv : groups) {
        BatchClass c;
        c.ny = kv.first.first;
        c.nx = kv.first.second;
        c.members = kv.second;
        c.cbase = slot;
        c.onchip = onchip_on && c.ny <= ONCHIP_MAX && c.nx <= ONCHIP_MAX &&
                   onchip_smem(c.ny, c.nx, vb) <= (size_t)optin;
        if (c.onchip) {
            c.t = Tiles{};
            c.t.g = grid_geom(c.nx, c.ny, 1);
            c.t.g.nreal = (int64_t)c.nx * c.ny;
            c.smem_oc = onchip_smem(c.ny, c.nx, vb);
            b->smem_oc = std::max(b->smem_oc, c.smem_oc);
        } else if (!plan_tiles(c.t, c.nx, c.ny, 1, vb, 2, (size_t)optin, (int)c.members.size())) {
            return bail(PFC_ERR_UNSUPPORTED, "no pass tiling fits shared memory for a domain size");
        }
        c.t.g.ltab = BATCH_LTAB;
        std::vector<int64_t> moff;
        std::vector<double> rr;
        for (int d : c.members) {
            b->slot_of[d] = slot++;
            off_cm.push_back(off_idx[d]);
            n_cm.push_back(off_idx[d + 1] - off_idx[d]);
            moff.push_back(off_idx[d]);
            rr.push_back(r_host[d]);
        }
        const size_t nm = c.members.size();
        const size_t half = c.onchip ? 0 : (size_t)c.t.g.nhalf * vb * nm;
        b->cls.push_back(c);
        BatchClass &cc = b->cls.back();
        cc.cap = half;
        if ((!cc.onchip && ((e = cudaMalloc(&cc.X, half)) != cudaSuccess || (e = cudaMalloc(&cc.C, half)) != cudaSuccess ||
                            (e = cudaMemset(cc.X, 0, half)) != cudaSuccess || (e = cudaMemset(cc.C, 0, half)) != cudaSuccess)) ||
            (e = cudaMalloc(&cc.moff, nm * sizeof(int64_t))) != cudaSuccess ||
            (e = cudaMemcpy(cc.moff, moff.data(), nm * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMalloc(&cc.r, nm * (vb / 2))) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&cc.s, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(e == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA,
                        std::string("batch allocation: ") + cudaGetErrorString(e));
        if (precision == PFC_FP64) {
            e = cudaMemcpy(cc.r, rr.data(), nm * 8, cudaMemcpyHostToDevice);
        } else {
            std::vector<float> rf(rr.begin(), rr.end());
            e = cudaMemcpy(cc.r, rf.data(), nm * 4, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return bail(PFC_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
        b->smem_row = std::max(b->smem_row, cc.t.smem_row);
        b->smem_line = std::max(b->smem_line, cc.t.smem_line);
    }
    if (b->smem_oc) {
        e = precision == PFC_FP64 ? set_smem_onchip<double>(b->smem_oc) : set_smem_onchip<float>(b->smem_oc);
        if (e != cudaSuccess) return bail(PFC_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
    }
    if ((e = cudaMalloc(&b->d_off, nd * sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_n, nd * sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMemcpy(b->d_off, off_cm.data(), nd * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_n, n_cm.data(), nd * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_mean, nd * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_status, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(b->d_status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess)
        return bail(PFC_ERR_CUDA, std::string("batch allocation: ") + cudaGetErrorString(e));
    b->ev_join.assign(b->cls.size(), nullptr);
    for (auto &ev : b->ev_join)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return bail(PFC_ERR_CUDA, std::string("batch events: ") + cudaGetErrorString(e));
    std::vector<double> full, stage;
    twiddle_tables(int64_t(1) << BATCH_LTAB, full, stage);
    if ((e = cudaMalloc(&b->tw, full.size() / 2 * vb)) != cudaSuccess ||
        (e = cudaMalloc(&b->stw, stage.size() / 2 * vb)) != cudaSuccess)
        return bail(PFC_ERR_OUT_OF_MEMORY, std::string("batch tables: ") + cudaGetErrorString(e));
    if (precision == PFC_FP64) {
        if ((e = cudaMemcpy(b->tw, full.data(), full.size() * 8, cudaMemcpyHostToDevice)) == cudaSuccess)
            e = cudaMemcpy(b->stw, stage.data(), stage.size() * 8, cudaMemcpyHostToDevice);
    } else {
        std::vector<float> f(full.begin(), full.end()), s2(stage.begin(), stage.end());
        if ((e = cudaMemcpy(b->tw, f.data(), f.size() * 4, cudaMemcpyHostToDevice)) == cudaSuccess)
            e = cudaMemcpy(b->stw, s2.data(), s2.size() * 4, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return bail(PFC_ERR_CUDA, std::string("batch tables: ") + cudaGetErrorString(e));
    const LaunchCfg mx{b->cls[0].t.g, 0, 0, b->smem_row, b->smem_line, b->stream};
    e = precision == PFC_FP64 ? raise_smem_attrs<double>(mx) : raise_smem_attrs<float>(mx);
    if (e != cudaSuccess) return bail(PFC_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
    *out = b;
    return PFC_OK;
}

pfc_status pfc_batch_destroy(pfc_batch *b) {
    if (!b) return PFC_OK;
    free_batch(b);
    return PFC_OK;
}

pfc_status pfc_batch_step(pfc_batch *b, void *packed_state, int64_t nsteps) {
    if (!b) return set_error(PFC_ERR_INVALID_ARG, "invalid batch");
    if (!packed_state) return set_error(PFC_ERR_INVALID_ARG, "null state");
    if (nsteps < 0) return set_error(PFC_ERR_INVALID_ARG, "nsteps must be >= 0");
    if ((reinterpret_cast<uintptr_t>(packed_state) & 15) != 0)
        return set_error(PFC_ERR_INVALID_ARG, "state must be 16-byte aligned");
    if (b->has_pair) return set_error(PFC_ERR_INVALID_ARG, "the batch has a coupled pair: pfc_batch_step_with_pair");
    if (nsteps == 0) return PFC_OK;
    return b->prec == PFC_FP64 ? batch_step_impl<double>(b, packed_state, nsteps)
                               : batch_step_impl<float>(b, packed_state, nsteps);
}

pfc_status pfc_batch_attach_pair(pfc_batch *b, int ndim, const int64_t *dims, const pfc_op *ops, double alpha) {
    if (!b || !dims || !ops) return set_error(PFC_ERR_INVALID_ARG, "null pointer argument");
    if (b->has_pair) return set_error(PFC_ERR_INVALID_ARG, "the batch already has a coupled pair");
    if (ndim != 2 && ndim != 3) return set_error(PFC_ERR_INVALID_ARG, "ndim must be 2 or 3");
    int n[3] = {1, 1, 1};   // nx, ny, nz
    for (int d = 0; d < ndim; ++d) {
        const int64_t v = dims[ndim - 1 - d];
        if (!is_pow2(v) || v < 16 || v > 512)
            return set_error(PFC_ERR_UNSUPPORTED, "the pair's extents must be powers of two in [16, 512]");
        n[d] = (int)v;
    }
    for (int f = 0; f < 2; ++f)
        if ((ops[f].kind != PFC_ONE_MODE && ops[f].kind != PFC_TWO_MODE) || !std::isfinite(ops[f].r) ||
            !std::isfinite(ops[f].R1) || !std::isfinite(ops[f].q2))
            return set_error(PFC_ERR_INVALID_ARG, "bad operator");
    if (!std::isfinite(alpha)) return set_error(PFC_ERR_INVALID_ARG, "alpha must be finite");
    const double kmax = M_PI / b->dx;
    if (min_implicit(ops, 2, alpha, b->dt, ndim * kmax * kmax) <= 0.0)
        return set_error(PFC_ERR_UNSTABLE_OPERATOR, "the coupled implicit system is not positive definite for some k");
    PFC_BCUDA(cudaStreamSynchronize(b->stream));
    if (!b->pair_moff) PFC_BCUDA(cudaMalloc(&b->pair_moff, 2 * sizeof(int64_t)));
    if (!b->pair_mean) PFC_BCUDA(cudaMalloc(&b->pair_mean, 2 * sizeof(double)));
    b->has_pair = true;
    b->pair_ndim = ndim;
    for (int d = 0; d < 3; ++d) b->pair_n[d] = n[d];
    b->pair_ops[0] = ops[0];
    b->pair_ops[1] = ops[1];
    b->pair_alpha = alpha;
    const pfc_status st = b->prec == PFC_FP64 ? persist_prepare<double>(b) : persist_prepare<float>(b);
    if (st != PFC_OK) {
        b->has_pair = false;
        return st;
    }
    b->sched = PFC_BATCH_PERSISTENT;
    return PFC_OK;
}

pfc_status pfc_batch_step_with_pair(pfc_batch *b, void *packed_state, void *pair_state, int64_t nsteps) {
    if (!b) return set_error(PFC_ERR_INVALID_ARG, "invalid batch");
    if (!b->has_pair) return set_error(PFC_ERR_INVALID_ARG, "the batch has no coupled pair");
    if (!packed_state || !pair_state) return set_error(PFC_ERR_INVALID_ARG, "null state");
    if (nsteps < 0) return set_error(PFC_ERR_INVALID_ARG, "nsteps must be >= 0");
    if ((reinterpret_cast<uintptr_t>(packed_state) & 15) != 0 || (reinterpret_cast<uintptr_t>(pair_state) & 15) != 0)
        return set_error(PFC_ERR_INVALID_ARG, "states must be 16-byte aligned");
    if (nsteps == 0) return PFC_OK;
    return b->prec == PFC_FP64 ? persist_step<double>(b, packed_state, nsteps, pair_state)
                               : persist_step<float>(b, packed_state, nsteps, pair_state);
}

pfc_status pfc_batch_autotune(pfc_batch *b, int max_candidates, int trial_steps, double *best_ms_out) {
    if (!b) return set_error(PFC_ERR_INVALID_ARG, "invalid batch");
    if (max_candidates < 1 || trial_steps < 1)
        return set_error(PFC_ERR_INVALID_ARG, "max_candidates and trial_steps must be >= 1");
    int dev = 0, optin = 0;
    PFC_BCUDA(cudaGetDevice(&dev));
    PFC_BCUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    PFC_BCUDA(cudaStreamSynchronize(b->stream));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    double total = 0;
    b->smem_row = b->smem_line = 0;
    for (BatchClass &c : b->cls) {
        if (c.onchip) continue;   // no tiling: stepped in shared memory
        double ms = 0;
        pfc_status st = b->prec == PFC_FP64 ? tune_class<double>(b, c, max_candidates, trial_steps, (size_t)optin, &ms)
                                            : tune_class<float>(b, c, max_candidates, trial_steps, (size_t)optin, &ms);
        if (st != PFC_OK) return st;
        total += ms;
        b->smem_row = std::max(b->smem_row, c.t.smem_row);
        b->smem_line = std::max(b->smem_line, c.t.smem_line);
    }
    PFC_BCUDA(cudaStreamSynchronize(b->stream));
    pfc_status st = b->prec == PFC_FP64 ? tune_schedule<double>(b, trial_steps) : tune_schedule<float>(b, trial_steps);
    if (st != PFC_OK) return st;
    if (best_ms_out) *best_ms_out = total;
    return PFC_OK;
}

pfc_status pfc_batch_info(pfc_batch *b, int32_t *classes_out, int max_classes, int32_t *nclasses) {
    if (!b || !nclasses) return set_error(PFC_ERR_INVALID_ARG, "null pointer argument");
    if (max_classes < 0 || (max_classes > 0 && !classes_out)) return set_error(PFC_ERR_INVALID_ARG, "bad class buffer");
    *nclasses = (int32_t)b->cls.size();
    for (int i = 0; i < (int)b->cls.size() && i < max_classes; ++i) {
        const BatchClass &c = b->cls[i];
        const int32_t v[9] = {c.ny, c.nx, (int32_t)c.members.size(), c.onchip ? 0 : c.t.g.Py,
                              c.onchip ? 0 : c.t.g.W, c.onchip ? 0 : c.t.g.gpc,
                              c.onchip ? ONCHIP_THREADS : c.t.nt_row, c.onchip ? 0 : c.t.nt_line,
                              c.onchip ? 0 : c.t.g.Qy};
        std::memcpy(classes_out + 9 * i, v, sizeof(v));
    }
    return PFC_OK;
}

pfc_status pfc_batch_set_schedule(pfc_batch *b, int schedule, int threads, int64_t onchip_smem_max,
                                  double onchip_block_share) {
    if (!b) return set_error(PFC_ERR_INVALID_ARG, "invalid batch");
    if (schedule != PFC_BATCH_GRAPH && schedule != PFC_BATCH_PERSISTENT)
        return set_error(PFC_ERR_INVALID_ARG, "unknown batch schedule");
    if (schedule == PFC_BATCH_PERSISTENT && threads != 128 && threads != 256 && threads != 512)
        return set_error(PFC_ERR_INVALID_ARG, "persistent blocks have 128, 256 or 512 threads");
    if (onchip_smem_max < 0 || !(onchip_block_share <= 1.0) || std::isnan(onchip_block_share))
        return set_error(PFC_ERR_INVALID_ARG, "bad on-chip limit or block share");
    PFC_BCUDA(cudaStreamSynchronize(b->stream));
    if (schedule == PFC_BATCH_GRAPH) {
        if (b->has_pair) return set_error(PFC_ERR_INVALID_ARG, "a batch with a coupled pair runs the persistent schedule");
        b->sched = schedule;
        return PFC_OK;
    }
    b->p_nt = threads;
    b->p_oc_max = (size_t)onchip_smem_max;
    b->p_oc_share = onchip_block_share;
    const pfc_status st = b->prec == PFC_FP64 ? persist_prepare<double>(b) : persist_prepare<float>(b);
    if (st == PFC_OK) b->sched = schedule;   // on failure the batch keeps its schedule
    return st;
}

pfc_status pfc_batch_schedule_info(pfc_batch *b, int64_t *info_out) {
    if (!b || !info_out) return set_error(PFC_ERR_INVALID_ARG, "null pointer argument");
    const int64_t v[10] = {b->sched, b->p_nt, b->p_grid, b->p_oc_blocks, (int64_t)b->p_smem,
                           b->p_graph_ok ? 1 : 0, b->n_row, b->n_line, b->n_oc, b->n_mean};
    std::memcpy(info_out, v, sizeof(v));
    return PFC_OK;
}

pfc_status pfc_batch_set_wait_limit(pfc_batch *b, double seconds, int extra_arrivals) {
    if (!b) return set_error(PFC_ERR_INVALID_ARG, "invalid batch");
    if (!(seconds > 0) || !(seconds <= 60) || extra_arrivals < 0 || extra_arrivals > 1024)
        return set_error(PFC_ERR_INVALID_ARG, "wait limit must be in (0, 60] s and extra arrivals in [0, 1024]");
    int dev = 0, clk_khz = 0;
    PFC_BCUDA(cudaGetDevice(&dev));
    if (cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev) != cudaSuccess || clk_khz <= 0) clk_khz = 2000000;
    PFC_BCUDA(cudaStreamSynchronize(b->stream));
    b->p_budget = (long long)((double)clk_khz * 1000.0 * seconds);
    b->p_extra = extra_arrivals;
    return PFC_OK;
}

pfc_status pfc_batch_sync(pfc_batch *b) {
    if (!b) return set_error(PFC_ERR_INVALID_ARG, "invalid batch");
    int st = 0;
    PFC_BCUDA(cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    PFC_BCUDA(cudaStreamSynchronize(b->stream));
    if (st) PFC_BCUDA(cudaMemset(b->d_status, 0, sizeof(int)));
    if (st & STATUS_TIMEOUT) return set_error(PFC_ERR_TIMEOUT, "a grid barrier of the persistent batch launch ran out of time");
    if (st & STATUS_NONFINITE) return set_error(PFC_ERR_NONFINITE, "the state holds NaN or Inf");
    return PFC_OK;
}

pfc_status pfc_batch_mass(pfc_batch *b, const void *packed_state, double *out_host) {
    if (!b || !packed_state || !out_host) return set_error(PFC_ERR_INVALID_ARG, "null pointer argument");
    if (b->prec == PFC_FP64)
        launch_batch_mean<double>(b->stream, reinterpret_cast<const double *>(packed_state), b->d_off,
                                  b->d_n, b->nd, b->d_mean, b->d_status);
    else
        launch_batch_mean<float>(b->stream, reinterpret_cast<const float *>(packed_state), b->d_off,
                                 b->d_n, b->nd, b->d_mean, b->d_status);
    std::vector<double> cm(b->nd);
    int st = 0;
    PFC_BCUDA(cudaMemcpyAsync(cm.data(), b->d_mean, b->nd * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    PFC_BCUDA(cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    PFC_BCUDA(cudaStreamSynchronize(b->stream));
    if (st) {
        PFC_BCUDA(cudaMemset(b->d_status, 0, sizeof(int)));
        return set_error(PFC_ERR_NONFINITE, "the state holds NaN or Inf");
    }
    for (int d = 0; d < b->nd; ++d) out_host[d] = cm[b->slot_of[d]];
    return PFC_OK;
}

}  // extern "C"
