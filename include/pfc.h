/*
 * pfc.h - C ABI of the GB300 (sm_103a) semi-implicit Fourier pseudo-spectral
 * phase-field-crystal (PFC) library, libpfc.so.
 *
 * The method (paper: "Multi-GPU fast Fourier transforms in MATLAB for large-scale phase-field
 * crystal simulations"): a periodic field psi on an equispaced grid evolves by the conserved
 * PFC dynamics of Eq. (6), d_t psi = lap((eps + L) psi + psi^3), discretised pseudo-spectrally
 * (Eqs. (1)-(4)) with semi-implicit time integration (the update of Listing 1):
 *
 *     psi_hat <- (psi_hat - dt k^2 FFT(psi^3)) / (1 + dt k^2 Lk(k)),
 *
 * Lk(k) = eps + L(k). One-mode: Lk = r + (1 - k^2)^2. Two-mode (tenth-order PDE, the paper's
 * FCC operator of Eq. (5) when R1 = 0 and q2^2 = 4/3): Lk = r + (1 - k^2)^2 (R1 + (q2^2 - k^2)^2).
 *
 * Conventions shared by every call:
 *   - dims are given slowest first, like a C array or a torch/numpy shape: 2D (ny, nx),
 *     3D (nz, ny, nx); x is contiguous. Every extent is a power of two in [16, 4096], or
 *     the grid is a mixed-radix one: every extent a product of 2, 3, 5 and 7 in [8, 4096],
 *     nx even and nx / 2 such a product too (the paper's 750^3, 900^3, 1400^3); otherwise
 *     PFC_ERR_UNSUPPORTED.
 *   - Box length per axis is n dx; k = 2 pi m / (n dx) with m in FFT order.
 *   - Real arrays hold nfields fields back to back, each nz*ny*nx values; complex arrays
 *     are interleaved (re, im) with the half-spectrum shape (nz, ny, nx/2 + 1).
 *   - Element type: double for PFC_FP64, float for PFC_FP32_MIXED (complex: double2 / float2).
 *   - All array pointers are DEVICE pointers (16-byte aligned) owned by the caller, unless a
 *     parameter says "host". The plan owns its scratch, tables, status word and graphs.
 *   - Calls are asynchronous and stream-ordered on the plan's stream, except pfc_mass,
 *     pfc_energy and pfc_sync, which synchronise that stream.
 *   - A plan is not thread-safe. Out-parameters are written only on PFC_OK.
 *   - No C++ exception crosses the ABI. After a non-OK status, pfc_last_error() returns a
 *     one-line description (thread-local, valid until the next call on the same thread).
 */
#ifndef PFC_H
#define PFC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PFC_OK = 0,
    PFC_ERR_INVALID_ARG = 1,        /* null pointer, bad count, non-positive dx or dt, ... */
    PFC_ERR_UNSUPPORTED = 2,        /* a size or option this build does not implement */
    PFC_ERR_UNSTABLE_OPERATOR = 3,  /* min_k (1 + dt k^2 Lk) <= 0 (or a coupled det <= 0) */
    PFC_ERR_OUT_OF_MEMORY = 4,      /* device allocation failed */
    PFC_ERR_CUDA = 5,               /* a CUDA runtime call failed */
    PFC_ERR_NONFINITE = 6,          /* a reduction met NaN or Inf in the state */
    PFC_ERR_TIMEOUT = 7             /* a bounded device-side wait gave up */
} pfc_status;

typedef enum { PFC_FP64 = 0, PFC_FP32_MIXED = 1 } pfc_precision;

typedef enum { PFC_ONE_MODE = 0, PFC_TWO_MODE = 1 } pfc_op_kind;

/* Time integrators of pfc_set_integrator. */
typedef enum { PFC_SEMI_IMPLICIT = 0, PFC_STABILIZED = 1, PFC_SBDF2 = 2 } pfc_integrator;

/* Linear PFC symbol Lk(k) (Eq. (5)-(6)); kind is a pfc_op_kind. R1 and q2 are read only for
 * PFC_TWO_MODE. */
typedef struct {
    int kind;
    double r;
    double R1;
    double q2;
} pfc_op;

typedef struct pfc_plan pfc_plan;

/* Create a plan for nfields coupled fields on one grid.
 *   ndim      2 or 3; dims[ndim] slowest first.
 *   dx, dt    grid spacing and time step, > 0.
 *   ops       nfields operators (host array).
 *   nfields   1, or 2 for the density/composition pair. With 2 fields both are conserved
 *             and the linear coupling alpha psi c enters both chemical potentials; the
 *             per-mode 2x2 implicit system is solved exactly.
 *   coupling  host nfields*nfields symmetric matrix, only the off-diagonal read; NULL = 0.
 *   precision PFC_FP64 (all FP64) or PFC_FP32_MIXED (FP32 data and butterflies, twiddles
 *             generated in FP64 and rounded, FP64 reductions, the k = 0 mode carried in FP64).
 *   stream    cudaStream_t the plan issues all its work on (NULL = legacy default stream).
 * Pass schedule: a step is a row pass (x transforms, psi^3, the first part of the y/z
 * transforms) and a line pass (the rest of the y/z transforms and the update), 5 sweeps of a
 * half spectrum, when a group of rows and two line tiles fit one SM's shared memory. Larger
 * grids (FP64 512^3, 3D grids from 1024^3 up) take the three-pass schedule: a middle pass takes
 * over a third part of the y/z transforms (9 sweeps a step). Two-field plans need the two-pass
 * schedule (UNSUPPORTED otherwise).
 * Mixed-radix grids (extents not all powers of two) take one pass per axis instead, each line
 * a Stockham transform of radices 2, 3, 4, 5, 7, 8 in shared memory (11 sweeps a step in 3D,
 * 7 in 2D). They support one field and the semi-implicit step: pfc_step, the transforms,
 * pfc_mass, pfc_energy, pfc_set_r, pfc_profile_steps, pfc_plan_autotune (radix order and
 * launch shapes) and the hydrodynamic model; the adjoint, recorded segments and the other
 * integrators return UNSUPPORTED.
 * Allocates the plan's device scratch with cudaMalloc: 2 * nfields half spectra, and a third
 * for a three-pass or mixed-radix plan.
 * Errors: INVALID_ARG, UNSUPPORTED, UNSTABLE_OPERATOR, OUT_OF_MEMORY, CUDA. */
pfc_status pfc_plan_create(pfc_plan **out, int ndim, const int64_t *dims, double dx, double dt,
                           const pfc_op *ops, int nfields, const double *coupling,
                           int precision, void *stream);

/* Release the plan and its device memory (synchronises its stream first). NULL is a no-op. */
pfc_status pfc_plan_destroy(pfc_plan *plan);

/* Advance state (device, real, nfields fields) by nsteps >= 0 semi-implicit steps, in place.
 * One step is psi -> IFFT[(FFT psi - dt k^2 FFT psi^3) / (1 + dt k^2 Lk)] (Listing 1 update,
 * Eq. (6)). The mean of each field (mass, the k = 0 mode) is held in FP64 across the call and
 * is conserved exactly. nsteps = 0 leaves state untouched. */
pfc_status pfc_step(pfc_plan *plan, void *state, int64_t nsteps);

/* Forward real-to-complex transform of each field, unnormalised (Eq. (4), MATLAB fft):
 * in_real (device, real) -> out_half (device, complex half spectrum). in_real is not modified;
 * the arrays must not overlap. */
pfc_status pfc_fft_r2c(pfc_plan *plan, const void *in_real, void *out_half);

/* Inverse complex-to-real transform with the 1/N factor (MATLAB ifft); the imaginary parts
 * of the kx = 0 and kx = nx/2 bins are ignored. in_half is not modified. */
pfc_status pfc_fft_c2r(pfc_plan *plan, const void *in_half, void *out_real);

/* Mass: the mean density of each field, out_host[nfields] (host), FP64 accumulation; the
 * k = 0 Fourier coefficient divided by N. Eq. (6) puts the whole right-hand side under a
 * Laplacian, so the k = 0 mode is multiplied by k^2 = 0 in the update of Listing 1 and the mass
 * of each field is a constant of the motion (pfc_step carries it exactly in FP64).
 * Synchronises. Errors: NONFINITE if the state holds NaN or Inf. */
pfc_status pfc_mass(pfc_plan *plan, const void *state, double *out_host);

/* Energy density F/|Omega| of Eq. (5), summed over the plan's fields, out_host (host, one
 * double): mean over points of psi Lk psi / 2 + psi^4 / 4 (+ alpha psi c for two fields),
 * the quadratic part evaluated in Fourier space by Parseval, FP64 accumulation. Synchronises. */
pfc_status pfc_energy(pfc_plan *plan, const void *state, double *out_host);

/* Adjoint of one step (single-field plans). With psi_{n+1} = A psi_n - B psi_n^3,
 * A = IFFT (1/D) FFT, B = IFFT (dt k^2/D) FFT, D = 1 + dt k^2 Lk:
 *     lam_out = A lam_next - 3 psi_n^2 (B lam_next)
 *     *dr_accum_dev += < lam_next, d psi_{n+1} / d r >,  d psi_{n+1}/dr = IFFT(-(dt k^2/D) psi_hat_{n+1})
 * psi_n, lam_next, lam_out: device real arrays (lam_out may alias lam_next, not psi_n).
 * dr_accum_dev: one device double, accumulated in FP64 (stream ordered, not synchronised).
 * The first call allocates a third half spectrum in the plan. Single-field plans only. */
pfc_status pfc_step_adjoint(pfc_plan *plan, const void *psi_n, const void *lam_next,
                            void *lam_out, double *dr_accum_dev);

/* Recorded segments: the adjoint over several steps without leaving the plan's internal form.
 * pfc_step_record advances state by nsteps >= 1 semi-implicit steps exactly like pfc_step and
 * keeps, in the caller's device buffer record (pfc_record_bytes bytes, 256-byte aligned), the
 * FP64 mean and each step's state and F(psi^3) in the plan's internal transformed layout.
 * pfc_adjoint_segment then applies the adjoint of those nsteps steps, last to first (the same
 * per-step adjoint as pfc_step_adjoint):
 *     lam (device real array, in: dL/dpsi at the segment's end, out: dL/dpsi at its start),
 *     *dr_accum_dev += sum over the steps of < lam_{n+1}, d psi_{n+1} / dr >.
 * lam stays in the internal layout between the steps, and the state, its cube and the adjoint
 * products are read from the record: 9 sweeps of a half spectrum per adjoint step instead of
 * the 17 of a pfc_step_adjoint call. A record is valid for the plan's tiling and operator at the
 * time it was written (pfc_plan_autotune and pfc_set_r invalidate it).
 * Single-field two-pass plans with the semi-implicit integrator whose fused adjoint row pass
 * fits shared memory (UNSUPPORTED otherwise, e.g. FP64 256^3: use pfc_step_adjoint).
 * Stream ordered, not synchronised. Errors: INVALID_ARG, UNSUPPORTED, OUT_OF_MEMORY, CUDA. */
pfc_status pfc_record_bytes(pfc_plan *plan, int64_t nsteps, int64_t *bytes_out);
pfc_status pfc_step_record(pfc_plan *plan, void *state, int64_t nsteps, void *record);
pfc_status pfc_adjoint_segment(pfc_plan *plan, const void *record, int64_t nsteps, void *lam,
                               double *dr_accum_dev);

/* Change r of field `field` (0-based); re-checks operator stability. */
pfc_status pfc_set_r(pfc_plan *plan, int field, double r);

/* Time integrator of pfc_step (single-field plans; a new plan uses PFC_SEMI_IMPLICIT). The paper
 * integrates with the semi-implicit scheme (Listing 1) and notes that other time-integration
 * schemes can be used; in Fourier space each mode obeys d/dt psi_hat = -k^2 (Lk psi_hat + N_hat),
 * N = psi^3 (Eq. (6)), and one step is
 *   PFC_SEMI_IMPLICIT  psi_hat <- (psi_hat - dt k^2 N_hat) / (1 + dt k^2 Lk)              (S unused)
 *   PFC_STABILIZED     psi_hat <- ((1 + dt k^2 S) psi_hat - dt k^2 N_hat) / (1 + dt k^2 (Lk + S)):
 *                      S psi moved from the explicit to the implicit part (S >= 0; S = 0 is the
 *                      semi-implicit step); first order
 *   PFC_SBDF2          (3 psi_hat^{n+1} - 4 psi_hat^n + psi_hat^{n-1}) / (2 dt)
 *                          = -k^2 (Lk psi_hat^{n+1} + 2 N_hat^n - N_hat^{n-1}):
 *                      second-order backward differentiation with the nonlinear term extrapolated
 *                      (S unused). It carries two time levels inside one pfc_step call, whose
 *                      first step is a semi-implicit step: a call of nsteps steps is one run
 *                      (the levels do not persist between calls). Allocates two more half spectra.
 * Passes: the same two (or three) passes per step; PFC_SBDF2's line pass reads the previous
 * level's X' and C' too (7 sweeps a step in the two-pass schedule). Re-checks that the scheme's
 * implicit factor is positive. pfc_step_adjoint stays the adjoint of the semi-implicit step
 * (UNSUPPORTED under another scheme). Errors: INVALID_ARG, UNSUPPORTED (two-field plans),
 * UNSTABLE_OPERATOR, OUT_OF_MEMORY, CUDA. */
pfc_status pfc_set_integrator(pfc_plan *plan, int scheme, double S);

/* Synchronise the plan's stream and return the latched device status (TIMEOUT, NONFINITE),
 * clearing it. */
pfc_status pfc_sync(pfc_plan *plan);

/* Tile choice and memory of a plan (host out-params).
 *   tiles[11] = {Py, Pz, Qy, Qz, W, row_groups_per_cta, threads_row, threads_line,
 *                row_cluster, Ry, Rz}
 *     row_cluster: blocks per cluster of the psi^3 row pass, 0 = none.
 *     Ry, Rz: the middle pass of the three-pass schedule (1, 1 = the two-pass schedule); the
 *     y length is Py Ry Qy and the z length Pz Rz Qz.
 *     A mixed-radix plan reports Py = Pz = Qy = Qz = 0, W = the y pass' columns a block,
 *     row_groups_per_cta = the x pass' rows a block, and the threads of those blocks.
 *   scratch_bytes = device bytes the plan owns. */
pfc_status pfc_plan_info(pfc_plan *plan, int32_t *tiles, int64_t *scratch_bytes);

/* Autotuner: choose the plan's tiling by measurement. The candidates are the valid tilings of
 * the grid (the split of the y/z transforms between the row and line passes, the line tile
 * width, and, where the grid has one, the clustered psi^3 row pass on or off), in the
 * planner's order with its own choice first; at most max_candidates (>= 1) of them are timed,
 * each on pfc_step of trial_steps (>= 1) steps of a zero field (a fixed point of the step) in
 * a scratch array, and the fastest is kept. The results of later calls do not depend on the
 * tiling beyond rounding; pfc_plan_info reports the choice. Line blocks stay within the
 * planner's limits, so every call the plan supported stays supported.
 *   cache_path  a text file of one JSON object per line, keyed by grid, precision, field
 *               count and device name: an entry for this plan is applied without timing (the
 *               last one wins); otherwise the choice is appended to the file. NULL: the file
 *               named by the environment variable PFC_AUTOTUNE_CACHE, or no cache if unset.
 *   best_ms_out host, may be NULL: ms per step of the chosen tiling (from the cache entry
 *               when one was applied).
 * Synchronises. Allocates a real array of the grid for the duration of the call, and larger
 * plan scratch when the chosen tiling pads kx further; the adjoint's third half spectrum is
 * released (the next pfc_step_adjoint allocates it again). Errors: INVALID_ARG,
 * OUT_OF_MEMORY, CUDA; on an error the planner's tiling is restored.
 * Mixed-radix plans: the candidates are the radix order of every axis (7, 5, 3 before 8, 4, 2,
 * or after), one or two warps a line in the column passes and the x pass' rows a block (the
 * current shape, half and twice), timed on the plan's step sequence of trial_steps steps of a
 * zero field; cache_path is not used. The twiddle table is rebuilt for the radix order. */
pfc_status pfc_plan_autotune(pfc_plan *plan, int max_candidates, int trial_steps,
                             const char *cache_path, double *best_ms_out);

/* Measurement support. Runs exactly the work of pfc_step(plan, state, nsteps) but records a
 * CUDA event on the plan's stream between consecutive kernel launches (no CUDA graph), then
 * synchronises and returns the summed event time per kernel kind in ms_out[5] (host):
 *   {row pass forming psi^3, line pass with the update, entry conversion, exit conversion,
 *    middle passes of a three-pass plan (0 for two-pass plans)};
 * on a mixed-radix plan {x pass forming psi^3, the y and z passes, entry, exit, the transforms
 *    of the projection columns}
 * and the number of kernel launches in *launches (host). */
pfc_status pfc_profile_steps(pfc_plan *plan, void *state, int64_t nsteps, double *ms_out,
                             int64_t *launches);

/* The step for callers that must not allocate device memory. The paper has no counterpart:
 * it exists for callers that cannot call cudaMalloc, such as a process whose device memory is
 * already held by another allocator (a framework's caching allocator, a fixed budget) or a
 * latency-sensitive loop that cannot afford the device-wide synchronisation of cudaMalloc and
 * cudaFree. Same arithmetic as pfc_step on a single field (the same kernels and tiling as a
 * plan of the grid); no plan is needed and nothing is allocated: the work arrays live in one
 * file-scope device array of 24 MiB that every GPU loading libpfc.so holds until the process
 * exits.
 *   ndim, dims, dx, dt, op, precision  as for pfc_plan_create (one field).
 *   state   device real array, advanced in place by nsteps steps (stream ordered on stream).
 *   stream  cudaStream_t (NULL = legacy default stream).
 * The call synchronises stream once, after the FP64 mean of the input state, to read the
 * status word: a state holding NaN or Inf returns PFC_ERR_NONFINITE and is left unchanged.
 * The steps that follow are stream ordered (not synchronised).
 * Limit: the two padded half spectra of the grid must fit the array beside its 0.3 MiB of
 * tables, e.g. 2D 1024x1024 in FP64 or 1024x2048 in FP32-mixed, 3D 128^3 in FP32-mixed or
 * 64^3 in FP64 (2048^2 FP32-mixed and 128^3 FP64 do not fit); a larger grid returns
 * PFC_ERR_UNSUPPORTED before any device work (use pfc_plan_create).
 * The first call on a device (and the first after a device reset) writes the array's twiddle
 * tables with synchronous copies. The host-side checks of a problem (stability, tiling, size)
 * are done on its first call and remembered. All calls share the array and find the previous
 * call's contents there: each call clears what must start at zero, and calls that overlap on
 * the GPU (other streams or threads) race. */
pfc_status pfc_step_noalloc(int ndim, const int64_t *dims, double dx, double dt, const pfc_op *op,
                            int precision, void *state, int64_t nsteps, void *stream);

/* ---------------------------------------------------------------------------------- */
/* Hydrodynamic PFC: the paper's multiphysics example (Eq. (hpfc)), a density psi and a     */
/* mesoscopic velocity v on one grid:                                                    */
/*     d_t psi = lap(mu) - v . grad psi,      rho d_t v = Gamma lap v - < psi grad mu >,  */
/*     mu = Lk psi + psi^3,  < . > the Gaussian average of width a0 (exp(-a0^2 k^2 / 2)).  */
/* One step (the paper's multi-field listing): psi semi-implicit as in pfc_step with the    */
/* advection term explicit (old velocity); then each velocity component implicit in the    */
/* viscosity, forced by the averaged psi' d_j mu' of the new density. Spatial derivatives   */
/* are spectral (i k_j, zero at the axis' Nyquist index).                                  */
/* ---------------------------------------------------------------------------------- */
typedef struct pfc_hydro pfc_hydro;

/* ndim, dims, dx, dt, op, precision, stream as for pfc_plan_create (one field); rho > 0 (+inf:
 * the velocity never changes), Gamma >= 0, a0 >= 0. Allocates a plan and six half spectra and
 * two real fields of work arrays. Errors as pfc_plan_create. */
pfc_status pfc_hydro_create(pfc_hydro **out, int ndim, const int64_t *dims, double dx, double dt,
                            const pfc_op *op, double rho, double gamma, double a0, int precision,
                            void *stream);
/* Advance psi (device real field) and v (device, ndim real fields back to back, x component
 * first) by nsteps steps, in place, stream ordered. The mean of psi is not carried separately
 * (the advection term changes it where div v != 0). */
pfc_status pfc_hydro_step(pfc_hydro *h, void *psi, void *v, int64_t nsteps);
pfc_status pfc_hydro_destroy(pfc_hydro *h);

/* ---------------------------------------------------------------------------------- */
/* Amplitude-expansion PFC: the density psi = psibar + sum_j [eta_j exp(i k_j.r) + c.c.] */
/* carried as namp complex amplitude fields. The paper names this model (multiphysics  */
/* section) as a workload of tens of complex fields; its equations here are the        */
/* projection of Eq. (6) with the energy of Eq. (5) onto the modes k_j.                */
/* ---------------------------------------------------------------------------------- */
typedef struct pfc_apfc pfc_apfc;

/* ndim 2 or 3, dims slowest first (each in [8, 4096], prime factors 2, 3, 5, 7); dx, dt > 0;
 * op the PFC operator L of Eq. (5); namp in [1, 16] amplitudes with reciprocal-lattice
 * vectors kvecs[namp * ndim] (host, components x first); psibar the mean density (fixed).
 * One step per amplitude j, every grid wavevector q (FFT order; the middle bin of an even axis
 * is -n/2):
 *   eta_hat_j <- (eta_hat_j - dt Q N_hat_j) / (1 + dt Q L(Q)),  Q = |k_j + q|^2,
 * the update of Listing 1 at the shifted wavevector, with N_j the component of psi^3 at k_j:
 * 3 psibar^2 eta_j plus the products of two (times 3 psibar) and three signed amplitudes whose
 * vectors sum to k_j (found on the host, exact to 1e-9 relative; eta_{-m} = conj(eta_m)).
 * Transforms are complex mixed-radix passes, one warp a line; a step is 7 sweeps of the
 * amplitude fields in 2D, 11 in 3D. Allocates two copies of the amplitude fields and tables.
 * Errors: INVALID_ARG, UNSUPPORTED, UNSTABLE_OPERATOR (1 + dt Q L(Q) <= 0 for some Q on the
 * grid), OUT_OF_MEMORY, CUDA. */
pfc_status pfc_apfc_create(pfc_apfc **out, int ndim, const int64_t *dims, double dx, double dt,
                           const pfc_op *op, int namp, const double *kvecs, double psibar,
                           int precision, void *stream);
/* Advance eta (device, namp complex fields [amp][z][y][x], interleaved re/im in the
 * precision's real type, 16-byte aligned) by nsteps, in place, stream ordered. */
pfc_status pfc_apfc_step(pfc_apfc *h, void *eta, int64_t nsteps);
/* *count_out (host) = the number of resonance terms over all amplitudes. Synchronises. */
pfc_status pfc_apfc_resonances(pfc_apfc *h, int32_t *count_out);
pfc_status pfc_apfc_destroy(pfc_apfc *h);

/* Names of a status code and of the last error on this thread. Never NULL. */
const char *pfc_status_string(pfc_status status);
const char *pfc_last_error(void);

/* ---------------------------------------------------------------------------------- */
/* Batched ensemble: many independent 2D one-mode domains of uneven sizes. Domains of    */
/* one size form a class stepped by one launch per pass (a member index per block);      */
/* every class is a branch of a CUDA graph captured once and replayed; or the whole call */
/* runs as one persistent launch (pfc_batch_set_schedule).                               */
/* ---------------------------------------------------------------------------------- */
typedef struct pfc_batch pfc_batch;

/* ndomains >= 1 domains; dims_host[2*d] = ny, dims_host[2*d+1] = nx of domain d (powers of two
 * in [16, 512]); r_host[d] its one-mode r. All share dx, dt and the precision. The packed state
 * holds the domains back to back in index order, domain d at element offset
 * sum_{e<d} ny_e nx_e. Domains are grouped by size; each size class runs as one branch of a
 * CUDA graph captured at the first pfc_batch_step with nsteps >= 16 (replayed afterwards), so
 * classes run concurrently. Allocates two half spectra per domain. */
pfc_status pfc_batch_create(pfc_batch **out, int ndomains, const int64_t *dims_host,
                            const double *r_host, double dx, double dt, int precision,
                            void *stream);
pfc_status pfc_batch_destroy(pfc_batch *batch);

/* Advance every domain of the packed device state by nsteps. */
pfc_status pfc_batch_step(pfc_batch *batch, void *packed_state, int64_t nsteps);

/* Autotune the tiling of every size class as pfc_plan_autotune does, each class timed alone on
 * trial_steps of its steps on zero fields; *best_ms_out (host, may be NULL) = the sum over
 * classes of the chosen ms per step. Then the schedule (pfc_batch_set_schedule): whole calls of
 * trial_steps steps on a zero state with the graph schedule and the persistent one at 256,
 * 128 and 512 threads a block (the persistent one only when a coupled pair is attached), the
 * fastest kept (pfc_batch_schedule_info reports it). The step graph is
 * captured again at the next pfc_batch_step. Synchronises. Errors: INVALID_ARG, UNSUPPORTED,
 * CUDA. */
pfc_status pfc_batch_autotune(pfc_batch *batch, int max_candidates, int trial_steps,
                              double *best_ms_out);

/* Size classes of the batch and their tiles (host out-params): *nclasses = number of classes;
 * for class i < max_classes, classes_out[9 i .. 9 i + 8] = {ny, nx, members, Py, W,
 * row_groups_per_cta, threads_row, threads_line, Qy}. classes_out may be NULL when
 * max_classes is 0. */
pfc_status pfc_batch_info(pfc_batch *batch, int32_t *classes_out, int max_classes, int32_t *nclasses);

/* Per-domain mass (mean), out_host[ndomains]. Synchronises. */
pfc_status pfc_batch_mass(pfc_batch *batch, const void *packed_state, double *out_host);

/* Schedules of pfc_batch_step.
 * PFC_BATCH_GRAPH: per size class one launch per pass, the classes as branches of a CUDA
 *   graph (above).
 * PFC_BATCH_PERSISTENT: the whole call in one cooperative launch (all blocks resident),
 *   replayed as a CUDA graph of that launch while the state pointer and nsteps stay the same.
 *   The launch's blocks of `threads` (128, 256 or 512) threads split in two groups. Blocks of the
 *   first group take on-chip members one at a time and run all their steps in shared memory:
 *   classes with both extents <= 128 that have no tiling of the block size, and (when
 *   onchip_smem_max > 0) those whose two half spectra take at most onchip_smem_max bytes. onchip_block_share in [0, 1] is the share of blocks in that group (< 0: the on-chip
 *   members' share of grid points). The other blocks take the two-pass members' work items
 *   (one row-pass block or one line-pass tile of one member each, the per-class launches'
 *   block work) from one queue per phase, meeting at a grid barrier between the phases: the
 *   means, the entry pass, nsteps x (psi^3 row pass, update pass), the exit pass. The shared
 *   memory of every block is the largest the classes need, so fewer blocks fit an SM when an
 *   on-chip class needs much. Every barrier wait is bounded (pfc_batch_set_wait_limit); a wait
 *   that runs out ends the launch with PFC_ERR_TIMEOUT latched for pfc_batch_sync, and the
 *   state is then undefined. The arithmetic per member is that of the plans (Eq. (6) and the
 *   update of Listing 1 in the two-pass form), so both schedules agree to rounding.
 * Setting a schedule synchronises the batch's stream and allocates what it needs; when it
 * fails the batch keeps its schedule.
 * Errors: INVALID_ARG, UNSUPPORTED (more than 36 size classes, or a class the launch cannot
 * step), OUT_OF_MEMORY, CUDA. */
enum { PFC_BATCH_GRAPH = 0, PFC_BATCH_PERSISTENT = 1 };
pfc_status pfc_batch_set_schedule(pfc_batch *batch, int schedule, int threads,
                                  int64_t onchip_smem_max, double onchip_block_share);

/* info_out[10] (host) = {schedule, threads, blocks, on-chip blocks, shared memory bytes a block,
 * captured as a graph (1) or launched directly (0), row items, line items, on-chip items,
 * mean items} of the persistent schedule (zeros before it is first set up). */
pfc_status pfc_batch_schedule_info(pfc_batch *batch, int64_t *info_out);

/* Bound of every grid-barrier wait of the persistent launch, in seconds of SM clock (default
 * 2 s; a phase takes well under a millisecond). extra_arrivals (normally 0) makes every
 * barrier wait for that many blocks beyond those that exist, so that every wait runs out:
 * an aid to test the timeout path without a device fault. Synchronises. */
pfc_status pfc_batch_set_wait_limit(pfc_batch *batch, double seconds, int extra_arrivals);

/* Attach a coupled density/composition pair (two conserved fields, the 2x2 per-mode implicit
 * update of pfc_plan_create with nfields = 2) to the batch: it is stepped inside the batch's
 * persistent launch, its row-pass items beside the domains' and its line items (both fields of
 * a tile) beside theirs, with the batch's dx, dt and precision. ndim 2 or 3, dims slowest
 * first, powers of two in [16, 512]; ops[2] the fields' operators; alpha the linear coupling.
 * Sets the persistent schedule (with its current block size). After this, pfc_batch_step
 * returns INVALID_ARG: use pfc_batch_step_with_pair. Synchronises and allocates two half
 * spectra per field. Errors: INVALID_ARG (a pair already attached), UNSUPPORTED,
 * UNSTABLE_OPERATOR, OUT_OF_MEMORY, CUDA. */
pfc_status pfc_batch_attach_pair(pfc_batch *batch, int ndim, const int64_t *dims, const pfc_op *ops,
                                 double alpha);

/* Advance the domains (packed_state) and the attached pair (pair_state: device, real,
 * [field][z][y][x], in place) by nsteps in one persistent launch. */
pfc_status pfc_batch_step_with_pair(pfc_batch *batch, void *packed_state, void *pair_state,
                                    int64_t nsteps);

/* Synchronises the batch's stream and returns the latched device status (cleared on read):
 * PFC_ERR_TIMEOUT when a persistent launch's barrier wait ran out, PFC_ERR_NONFINITE when a
 * mean reduction met NaN or Inf, else PFC_OK. */
pfc_status pfc_batch_sync(pfc_batch *batch);

#ifdef __cplusplus
}
#endif

#endif /* PFC_H */
