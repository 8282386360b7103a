// The persistent schedule of a batch (pfc_batch_* of pfc.h): one launch runs a whole
// pfc_batch_step call, every size class and every step.
//
// The launch is cooperative (all blocks resident at once) with NT threads a block. It splits its
// blocks in two:
//   blocks [0, n_oc_blocks): the on-chip members (classes small enough for one block's shared
//     memory). A block takes one member at a time from a queue, computes its FP64 mean, then runs
//     all nsteps steps of that member in shared memory (onchip_body). These blocks never wait on
//     any other block.
//   blocks [n_oc_blocks, grid): the two-pass members of every other class (and the two fields
//     of an attached coupled pair, whose line items take both fields of a tile), phase by phase:
//     the FP64 means; the entry row pass (real state -> X'); nsteps times the psi^3 row pass and
//     the update line pass (the two passes of the single-grid plans); the exit row pass (X' ->
//     real state). Within a phase a block takes work items from the phase's queue (an atomic
//     counter): one item is one row-pass block or one line-pass tile of one member of one
//     class, exactly the work of one block of the per-class launches. Items are sorted by cost,
//     largest first, so the queue drains longest-first.
// Between two phases the two-pass blocks meet at a grid barrier: an arrival counter and a
// generation word in global memory. The last block to arrive resets the counter and the queue
// of the phase after next, then publishes the next generation with a release store; the others
// spin on acquire loads (with nanosleep) until it changes, for at most `budget` SM clock cycles.
// A block whose wait runs out sets STATUS_TIMEOUT in the status word and returns; every other
// block then runs out at its next barrier (or sees the flag), so the launch always ends. The
// host reads the word (pfc_batch_sync). `extra` adds arrivals the barrier waits for beyond the
// blocks that exist (0 in normal use; a test sets it to make every wait run out).
//
// Memory ordering: a phase's results are written with plain or .cg stores and read in a later
// phase with .cg loads (X', C') or plain loads (means, the real state); the arrival is preceded
// by a device-scope fence and the wait is an acquire load followed by a fence, so every write
// of a phase is visible to every block in the phases after the barrier.
#pragma once

#include "pfc_coupled.cuh"
#include "pfc_onchip.cuh"
#include "pfc_pass.cuh"

namespace pfc {

constexpr int PB_MAXC = 36;   // size classes: extents 16 .. 512 in each of two axes

// sync words of a persistent launch (zeroed by the host before each launch)
enum { PB_ARRIVE = 0, PB_GEN = 1, PB_Q0 = 2, PB_QOC = 5, PB_NSYNC = 8 };

// One size class: its geometry and the arguments of its passes. On-chip classes use g (their
// on-chip geometry), fwd.moff / fwd.mean / fwd.tw / fwd.st, line.up and line.rmem.
template <typename R> struct PbClass {
    Geom g;
    RowArgs<R> fwd, cube, inv;   // entry (real -> X'), psi^3 and exit (X' -> real) row passes
    LineArgs<R> line;            // update pass
};

template <typename R> struct PbArgs {
    PbClass<R> cls[PB_MAXC];
    const int2 *mean_items;      // (class, member) of the two-pass members
    const int4 *row_items;       // (class, member, row block, 0)
    const int4 *line_items;      // (class, member, column group, split index)
    const int2 *oc_items;        // (class, member) of the on-chip members
    int n_mean, n_row, n_line, n_oc;
    int n_oc_blocks;
    int extra;
    int64_t nsteps;
    void *state;                 // packed real state of the batch (in/out)
    int pair_ci;                 // class index of an attached coupled pair (-1: none); its
    Step2Args<R> pair;           // members are its two fields, its line items the 2x2 update
    unsigned *sync;              // PB_NSYNC words
    int *status;
    long long budget;            // clock64 cycles a barrier wait may take
};

__device__ __forceinline__ unsigned pb_ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void pb_st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier of the two-pass blocks (nb arrivals expected); qreset: the queue word the last
// arrival clears. False when the wait ran out here or in another block.
template <typename R>
__device__ __forceinline__ bool pb_barrier(const PbArgs<R> &a, unsigned nb, unsigned &gen, int qreset,
                                           int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = gen + 1;
        __threadfence();
        const unsigned t = atomicAdd(&a.sync[PB_ARRIVE], 1u);
        if (t == nb - 1) {
            atomicExch(&a.sync[PB_ARRIVE], 0u);
            atomicExch(&a.sync[qreset], 0u);
            __threadfence();
            pb_st_release(&a.sync[PB_GEN], target);
        } else {
            const long long t0 = clock64();
            int polls = 0;
            while (pb_ld_acquire(&a.sync[PB_GEN]) != target) {
                if (clock64() - t0 > a.budget ||
                    ((++polls & 63) == 0 && (*(volatile int *)a.status & STATUS_TIMEOUT))) {
                    ok = 0;
                    atomicOr(a.status, STATUS_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        gen = target;
        *s_flag = ok;
    }
    __syncthreads();
    const int ok = *s_flag;
    __syncthreads();
    return ok != 0;
}

// Next item of queue q for the whole block (or a value >= n when the queue is empty).
__device__ __forceinline__ int pb_take(unsigned *q, int *s_item) {
    if (threadIdx.x == 0) *s_item = (int)atomicAdd(q, 1u);
    __syncthreads();
    const int it = *s_item;
    __syncthreads();
    return it;
}

// FP64 mean of member m of class c (n = g.nreal values at its offset in the packed state), in a
// fixed order; sets STATUS_NONFINITE on NaN or Inf.
template <typename R, int NT>
__device__ __forceinline__ void pb_mean(const PbClass<R> &c, int m, const PbArgs<R> &a, double *sh) {
    const R *x = reinterpret_cast<const R *>(c.fwd.in) + c.fwd.moff[m];
    const int64_t n = c.g.nreal;
    double acc = 0.0;
    bool bad = false;
    for (int64_t i = threadIdx.x; i < n; i += NT) {
        const double v = (double)x[i];
        if (!isfinite(v)) bad = true;
        acc += v;
    }
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
    sh[threadIdx.x] = acc;
    __syncthreads();
#pragma unroll
    for (int s = NT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) const_cast<double *>(c.fwd.mean)[m] = sh[0] / (double)n;
    __syncthreads();
}

// The work items call the pass bodies through functions that are not inlined: each body then
// gets the register allocation of its own kernel (at most 64 registers a thread), instead of one
// allocation for the union of all bodies (which spilled heavily).

// A psi^3 row-pass item: the row length fixed at compile time for M = 2^5 .. 2^8, and for the
// FP32 2D classes (Pz = 1) Py too (as the per-class launches do).
template <typename R, int LM, int PY = 0>
__device__ __noinline__ void pb_row_cube_t(const PbClass<R> &c, int bx, int m) {
    row_body<R, ROW_CUBE, LM, PY>(c.g, c.cube, bx, m);
}
template <typename R, int LM>
__device__ __forceinline__ void pb_row_cube_py(const PbClass<R> &c, int bx, int m) {
    if constexpr (sizeof(R) == 4) {
        if (c.g.Pz == 1) {
            switch (c.g.Py) {
            case 1: pb_row_cube_t<R, LM, 1>(c, bx, m); return;
            case 2: pb_row_cube_t<R, LM, 2>(c, bx, m); return;
            case 4: pb_row_cube_t<R, LM, 4>(c, bx, m); return;
            case 8: pb_row_cube_t<R, LM, 8>(c, bx, m); return;
            default: break;
            }
        }
    }
    pb_row_cube_t<R, LM>(c, bx, m);
}
template <typename R>
__device__ __forceinline__ void pb_row_cube(const PbClass<R> &c, int bx, int m) {
    switch (c.g.lM) {
    case 5: pb_row_cube_py<R, 5>(c, bx, m); return;
    case 6: pb_row_cube_py<R, 6>(c, bx, m); return;
    case 7: pb_row_cube_py<R, 7>(c, bx, m); return;
    case 8: pb_row_cube_py<R, 8>(c, bx, m); return;
    default: pb_row_cube_t<R, 0>(c, bx, m); return;
    }
}

// An update-pass item: the tile length fixed at compile time for Qy = 2^6 .. 2^9.
template <typename R, int LY>
__device__ __noinline__ void pb_line_t(const PbClass<R> &c, int cg, int kp, int m) {
    line_body<R, LINE_STEP, LY, 0>(c.g, c.line, cg, kp, m);
}
template <typename R>
__device__ __forceinline__ void pb_line(const PbClass<R> &c, int cg, int kp, int m) {
    switch (c.g.lQy) {
    case 6: pb_line_t<R, 6>(c, cg, kp, m); return;
    case 7: pb_line_t<R, 7>(c, cg, kp, m); return;
    case 8: pb_line_t<R, 8>(c, cg, kp, m); return;
    case 9: pb_line_t<R, 9>(c, cg, kp, m); return;
    default: pb_line_t<R, 0>(c, cg, kp, m); return;
    }
}

// an update item of an attached coupled pair: both fields of one tile
template <typename R>
__device__ __noinline__ void pb_line_pair(const PbClass<R> &c, const Step2Args<R> &a, int cg, int kp) {
    line_step2_body<R>(c.g, a, cg, kp);
}

// entry and exit row passes
template <typename R, int MODE>
__device__ __noinline__ void pb_row_io(const PbClass<R> &c, int bx, int m) {
    row_body<R, MODE, 0>(c.g, MODE == ROW_FWD ? c.fwd : c.inv, bx, m);
}

// all the steps of one on-chip member
template <typename R>
__device__ __noinline__ void pb_onchip(const PbClass<R> &c, int m, void *state, int64_t nsteps) {
    OnchipArgs<R> oa;
    oa.state = state;
    oa.moff = c.fwd.moff;
    oa.mean = c.fwd.mean;
    oa.r = c.line.rmem;
    oa.nsteps = nsteps;
    oa.up = c.line.up;
    oa.tw = c.fwd.tw;
    oa.st = c.fwd.st;
    onchip_body<R>(c.g, oa, m);
}

// resident threads an SM the register allocation is sized for
#ifndef PFC_PB_THREADS_PER_SM
#define PFC_PB_THREADS_PER_SM 1024
#endif

template <typename R, int NT>
__global__ void __launch_bounds__(NT, PFC_PB_THREADS_PER_SM / NT) k_batch_persist(const __grid_constant__ PbArgs<R> a) {
    __shared__ int s_item;
    __shared__ int s_flag;
    // the mean reduction runs between work items: it takes the start of the dynamic shared
    // memory (at least NT doubles: every item's tiles are larger), so the kernel's static shared
    // memory stays at two words and four blocks of up to 55 KB fit an SM
    extern __shared__ __align__(16) unsigned char smraw[];
    double *s_red = reinterpret_cast<double *>(smraw);

    if ((int)blockIdx.x < a.n_oc_blocks) {
        for (;;) {
            const int it = pb_take(&a.sync[PB_QOC], &s_item);
            if (it >= a.n_oc) return;
            const int2 w = a.oc_items[it];
            const PbClass<R> &c = a.cls[w.x];
            pb_mean<R, NT>(c, w.y, a, s_red);
            pb_onchip<R>(c, w.y, a.state, a.nsteps);
            __syncthreads();
        }
    }

    const unsigned nb = gridDim.x - (unsigned)a.n_oc_blocks + (unsigned)a.extra;
    unsigned gen = 0;
    int phase = 0;
    // the barrier that ends `phase` clears the queue of phase + 2 (the one phase - 1 used)
    auto next_phase = [&]() -> bool {
        const bool ok = pb_barrier(a, nb, gen, PB_Q0 + (phase + 2) % 3, &s_flag);
        ++phase;
        return ok;
    };
    unsigned *const q = a.sync + PB_Q0;

    // means of the two-pass members
    for (;;) {
        const int it = pb_take(&q[phase % 3], &s_item);
        if (it >= a.n_mean) break;
        const int2 w = a.mean_items[it];
        pb_mean<R, NT>(a.cls[w.x], w.y, a, s_red);
    }
    if (!next_phase()) return;
    // entry: X' = the row-pass forward transform of psi - mean
    for (;;) {
        const int it = pb_take(&q[phase % 3], &s_item);
        if (it >= a.n_row) break;
        const int4 w = a.row_items[it];
        pb_row_io<R, ROW_FWD>(a.cls[w.x], w.z, w.y);
        __syncthreads();
    }
    if (!next_phase()) return;
    for (int64_t s = 0; s < a.nsteps; ++s) {
        for (;;) {
            const int it = pb_take(&q[phase % 3], &s_item);
            if (it >= a.n_row) break;
            const int4 w = a.row_items[it];
            pb_row_cube<R>(a.cls[w.x], w.z, w.y);
            __syncthreads();
        }
        if (!next_phase()) return;
        for (;;) {
            const int it = pb_take(&q[phase % 3], &s_item);
            if (it >= a.n_line) break;
            const int4 w = a.line_items[it];
            if (w.x == a.pair_ci) pb_line_pair<R>(a.cls[w.x], a.pair, w.z, w.w);
            else pb_line<R>(a.cls[w.x], w.z, w.w, w.y);
            __syncthreads();
        }
        if (!next_phase()) return;
    }
    // exit: the real state from X'
    for (;;) {
        const int it = pb_take(&q[phase % 3], &s_item);
        if (it >= a.n_row) break;
        const int4 w = a.row_items[it];
        pb_row_io<R, ROW_INV>(a.cls[w.x], w.z, w.y);
        __syncthreads();
    }
}

}  // namespace pfc
