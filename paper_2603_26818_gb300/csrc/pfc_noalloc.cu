// pfc_step_noalloc: the semi-implicit step for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is already reserved by
// another allocator (a framework's caching allocator that holds the whole GPU, a fixed memory
// budget), or a latency-sensitive host loop that cannot afford the device-wide
// synchronisation that cudaMalloc and cudaFree imply. pfc_plan_create allocates the plan's
// scratch; this entry point instead uses one file-scope device array of fixed size,
// g_noalloc_scratch (24 MiB), which every GPU that loads libpfc.so holds until the process
// exits. It calls no cudaMalloc, cudaFree or allocating library routine.
//
// Layout of the array: twiddle tables for FP64 and FP32 (written once per device), a small
// area for the mean, the reduction partials and the status word, then the two half-spectrum
// work arrays X' and C' of the call.
//
// In host code the array's name only stands in for the device object, so the address passed
// to kernels comes from cudaGetSymbolAddress, taken once per device (with that device
// current) by the first call on that device. That first call also writes the tables with
// synchronous copies, so it must come before any stream capture. Every call shares the one
// array and finds the previous call's contents in it: the status word and the work arrays are
// cleared at the start of each call, and calls that overlap on the GPU (on different streams,
// or from different host threads) race on the array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "pfc_host.h"

namespace {

using namespace pfc;

constexpr size_t NOALLOC_BYTES = size_t(24) << 20;
constexpr int64_t NTAB = 4096;                           // largest extent; tables at 2^12 points
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t OFF_TW64 = 0;
constexpr size_t OFF_TW32 = align256(OFF_TW64 + NTAB * 16);
constexpr size_t OFF_ST64 = align256(OFF_TW32 + NTAB * 8);
constexpr size_t OFF_ST32 = align256(OFF_ST64 + STW_TOTAL * 16);
constexpr size_t OFF_MEAN = align256(OFF_ST32 + STW_TOTAL * 8);
constexpr size_t OFF_PART = align256(OFF_MEAN + 8 * sizeof(double));
constexpr size_t OFF_STATUS = align256(OFF_PART + RED_BLOCKS * sizeof(double));
constexpr size_t OFF_WORK = align256(OFF_STATUS + sizeof(int));

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_base[MAX_DEVICES] = {};

// Once per device, with that device current: the array's device address, and the tables.
pfc_status device_setup(int dev, unsigned char **base) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_base[dev]) {
        *base = g_base[dev];
        return PFC_OK;
    }
    unsigned char *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return set_error(PFC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    std::vector<double> full, stage;
    twiddle_tables(NTAB, full, stage);
    std::vector<float> full32(full.begin(), full.end()), stage32(stage.begin(), stage.end());
    if ((e = cudaMemcpy(ptr + OFF_TW64, full.data(), full.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ptr + OFF_TW32, full32.data(), full32.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ptr + OFF_ST64, stage.data(), stage.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ptr + OFF_ST32, stage32.data(), stage32.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return set_error(PFC_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
    g_base[dev] = ptr;
    *base = ptr;
    return PFC_OK;
}

template <typename R>
pfc_status run(const LaunchCfg &c, unsigned char *base, const pfc_op &op, double dx, double dt,
               void *state, int64_t nsteps) {
    using V = typename VT<R>::V;
    const Geom &g = c.g;
    const size_t vb = sizeof(V);
    V *X = reinterpret_cast<V *>(base + OFF_WORK);
    V *C = reinterpret_cast<V *>(base + OFF_WORK + align256(g.nhalf * vb));
    double *mean = reinterpret_cast<double *>(base + OFF_MEAN);
    double *part = reinterpret_cast<double *>(base + OFF_PART);
    int *status = reinterpret_cast<int *>(base + OFF_STATUS);
    const V *tw = reinterpret_cast<const V *>(base + (sizeof(R) == 8 ? OFF_TW64 : OFF_TW32));
    const V *st = reinterpret_cast<const V *>(base + (sizeof(R) == 8 ? OFF_ST64 : OFF_ST32));
    const StageTw<V> stw{st, st + STW8, st + STW8 + STW4};

    // the previous call's contents: clear the status word and both work arrays
    cudaError_t e;
    if ((e = cudaMemsetAsync(status, 0, sizeof(int), c.stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + OFF_WORK, 0, 2 * align256(g.nhalf * vb), c.stream)) != cudaSuccess)
        return set_error(PFC_ERR_CUDA, std::string("clear: ") + cudaGetErrorString(e));

    launch_reduce_real<R>(c.stream, RED_SUM, reinterpret_cast<const R *>(state), nullptr, g.nreal, part, status);
    launch_finish(c.stream, part, RED_BLOCKS, 1.0 / (double)g.nreal, mean);

    RowArgs<R> ra{};
    ra.tw = tw;
    ra.st = stw;
    ra.mean = mean;
    ra.in = state;
    ra.out = X;
    ra.scale = (R)(1.0 / ((double)g.P * (double)g.M));
    launch_row<R>(c, ROW_FWD, ra, 1);

    RowArgs<R> rc = ra;
    rc.in = X;
    rc.out = C;
    rc.proj = X;
    rc.scale = (R)1;
    LineArgs<R> la{};
    la.x = X;
    la.c = C;
    la.scale = (R)1;
    la.st = stw;
    const double two_pi = 6.28318530717958647692528676655900576839;
    la.up.dt = (R)dt;
    la.up.cx = (R)(two_pi / (g.nx * dx));
    la.up.cy = (R)(two_pi / (g.ny * dx));
    la.up.cz = (R)(two_pi / (g.nz * dx));
    la.up.invQ = (R)(1.0 / g.Q);
    la.up.inv_halfN = (R)(2.0 / (double)g.nreal);
    la.up.op[0] = la.up.op[1] = OpR<R>{op.kind, (R)op.r, (R)op.R1, (R)(op.q2 * op.q2)};
    for (int64_t s = 0; s < nsteps; ++s) {
        launch_row<R>(c, ROW_CUBE, rc, 1);
        launch_line<R>(c, LINE_STEP, la, 1);
    }

    RowArgs<R> rb = ra;
    rb.in = X;
    rb.out = state;
    rb.scale = (R)1;
    launch_row<R>(c, ROW_INV, rb, 1);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return set_error(PFC_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return PFC_OK;
}

}  // namespace

extern "C" pfc_status pfc_step_noalloc(int ndim, const int64_t *dims, double dx, double dt,
                                       const pfc_op *op, int precision, void *state,
                                       int64_t nsteps, void *stream) {
    if (!dims || !op || !state) return set_error(PFC_ERR_INVALID_ARG, "null pointer argument");
    if (ndim != 2 && ndim != 3) return set_error(PFC_ERR_INVALID_ARG, "ndim must be 2 or 3");
    if (!(dx > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dt))
        return set_error(PFC_ERR_INVALID_ARG, "dx and dt must be finite and > 0");
    if (precision != PFC_FP64 && precision != PFC_FP32_MIXED)
        return set_error(PFC_ERR_INVALID_ARG, "unknown precision");
    if (op->kind != PFC_ONE_MODE && op->kind != PFC_TWO_MODE)
        return set_error(PFC_ERR_INVALID_ARG, "unknown operator kind");
    if (nsteps < 0) return set_error(PFC_ERR_INVALID_ARG, "nsteps must be >= 0");
    if ((reinterpret_cast<uintptr_t>(state) & 15) != 0)
        return set_error(PFC_ERR_INVALID_ARG, "state must be 16-byte aligned");
    int64_t d[3] = {1, 1, 1};
    for (int i = 0; i < ndim; ++i) d[3 - ndim + i] = dims[i];
    for (int i = 3 - ndim; i < 3; ++i)
        if (!is_pow2(d[i]) || d[i] < 16 || d[i] > 4096)
            return set_error(PFC_ERR_UNSUPPORTED, "every extent must be a power of two in [16, 4096]");
    const double kmax = M_PI / dx;
    if (min_implicit(op, 1, 0.0, dt, kmax * kmax * ndim) <= 0.0)
        return set_error(PFC_ERR_UNSTABLE_OPERATOR, "1 + dt k^2 Lk(k) is not positive on the grid");
    if (nsteps == 0) return PFC_OK;

    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return set_error(PFC_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    if (dev >= MAX_DEVICES) return set_error(PFC_ERR_UNSUPPORTED, "device index beyond 63");
    const size_t vb = precision == PFC_FP64 ? 16 : 8;
    Tiles t{};
    if (!plan_tiles(t, (int)d[2], (int)d[1], (int)d[0], vb, 2, (size_t)optin))
        return set_error(PFC_ERR_UNSUPPORTED, "no pass tiling fits shared memory for this grid");
    t.g.ltab = 12;   // the tables hold 4096 points; every index shift is taken from 2^12
    const size_t need = OFF_WORK + 2 * align256(t.g.nhalf * vb);
    if (need > NOALLOC_BYTES)
        return set_error(PFC_ERR_UNSUPPORTED,
                         "grid too large for the 24 MiB static scratch of pfc_step_noalloc (needs " +
                             std::to_string(need) + " bytes); use pfc_plan_create");
    unsigned char *base = nullptr;
    pfc_status s = device_setup(dev, &base);
    if (s != PFC_OK) return s;
    const LaunchCfg c{t.g, t.nt_row, t.nt_line, t.smem_row, t.smem_line, reinterpret_cast<cudaStream_t>(stream)};
    e = precision == PFC_FP64 ? raise_smem_attrs<double>(c) : raise_smem_attrs<float>(c);
    if (e != cudaSuccess) return set_error(PFC_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
    return precision == PFC_FP64 ? run<double>(c, base, *op, dx, dt, state, nsteps)
                                 : run<float>(c, base, *op, dx, dt, state, nsteps);
}
