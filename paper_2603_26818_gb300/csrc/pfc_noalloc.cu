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
// Layout of the array: twiddle tables for FP64 and FP32, a small area for the mean, the
// reduction partials, the status word and a marker that says the tables are present, then the
// two half-spectrum work arrays X' and C' of the call.
//
// In host code the array's name only stands in for the device object, so the address passed
// to kernels comes from cudaGetSymbolAddress, taken on every call with the calling device
// current. Each call synchronises its stream once, after the FP64 mean of the input state: it
// reads back the status word (a NaN or Inf in the state returns PFC_ERR_NONFINITE and leaves
// the state untouched) together with the marker. On the first call on a device, and after a
// device reset has wiped the array, the marker is missing and the call writes the tables with
// synchronous copies. Every call shares the one array and finds the previous call's contents
// in it: the status word and the work arrays are cleared at the start of each call, and calls
// that overlap on the GPU (on different streams, or from different host threads) race on the
// array.
//
// The host-side checks of a grid (operator stability over the grid's wavenumbers, the tiling,
// the size limit) and the kernels' shared-memory limits are settled once per (device, grid, dx,
// dt, operator, precision) and kept in a small table in this file, so repeated calls on the
// same problem skip them. The launches are those of a plan of the same grid (the clustered
// psi^3 row pass included), so the arithmetic is pfc_step's.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

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
constexpr size_t OFF_STATUS = align256(OFF_PART + RED_BLOCKS * sizeof(double));   // int, then marker
constexpr size_t OFF_MARK = OFF_STATUS + 8;
constexpr size_t OFF_WORK = align256(OFF_STATUS + 16);
constexpr unsigned long long TABLES_MARK = 0x7066635f74616273ull;   // written after the tables

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

cudaError_t raise_attrs(const LaunchCfg &c, int precision) {
    return precision == PFC_FP64 ? raise_smem_attrs<double>(c) : raise_smem_attrs<float>(c);
}

// Validated host-side facts of one problem: its tiling (or the reason it is rejected).
struct Prepared {
    pfc_status status = PFC_OK;
    std::string msg;
    Tiles t{};
};
using Key = std::tuple<int, int64_t, int64_t, int64_t, double, double, int, double, double, double, int>;
std::mutex g_mu;
std::map<Key, Prepared> g_prepared;

Prepared prepare(int dev, const int64_t d[3], int ndim, double dx, double dt, const pfc_op &op, int precision) {
    Prepared p;
    const double kmax = M_PI / dx;
    if (min_implicit(&op, 1, 0.0, dt, kmax * kmax * ndim) <= 0.0) {
        p.status = PFC_ERR_UNSTABLE_OPERATOR;
        p.msg = "1 + dt k^2 Lk(k) is not positive on the grid";
        return p;
    }
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) {
        p.status = PFC_ERR_CUDA;
        p.msg = std::string("device query: ") + cudaGetErrorString(e);
        return p;
    }
    const size_t vb = precision == PFC_FP64 ? 16 : 8;
    if (!plan_tiles(p.t, (int)d[2], (int)d[1], (int)d[0], vb, 2, (size_t)optin)) {
        p.status = PFC_ERR_UNSUPPORTED;
        p.msg = "no pass tiling fits shared memory for this grid";
        return p;
    }
    p.t.g.ltab = 12;   // the tables hold 4096 points; every index shift is taken from 2^12
    const size_t need = OFF_WORK + 2 * align256(p.t.g.nhalf * vb);
    if (need > NOALLOC_BYTES) {
        p.status = PFC_ERR_UNSUPPORTED;
        p.msg = "grid too large for the 24 MiB static scratch of pfc_step_noalloc (needs " +
                std::to_string(need) + " bytes); use pfc_plan_create";
        return p;
    }
    if ((e = raise_attrs(launch_cfg(p.t, nullptr), precision)) != cudaSuccess) {
        p.status = PFC_ERR_CUDA;
        p.msg = std::string("smem attribute: ") + cudaGetErrorString(e);
    }
    return p;
}

// Write the twiddle tables and then the marker (synchronous copies).
cudaError_t upload_tables(unsigned char *ptr) {
    std::vector<double> full, stage;
    twiddle_tables(NTAB, full, stage);
    std::vector<float> full32(full.begin(), full.end()), stage32(stage.begin(), stage.end());
    const unsigned long long mark = TABLES_MARK;
    cudaError_t e;
    if ((e = cudaMemcpy(ptr + OFF_TW64, full.data(), full.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ptr + OFF_TW32, full32.data(), full32.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ptr + OFF_ST64, stage.data(), stage.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ptr + OFF_ST32, stage32.data(), stage32.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    return cudaMemcpy(ptr + OFF_MARK, &mark, sizeof(mark), cudaMemcpyHostToDevice);
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

    // the previous call's contents: clear the status word, then the FP64 mean of the state
    cudaError_t e;
    if ((e = cudaMemsetAsync(status, 0, sizeof(int), c.stream)) != cudaSuccess)
        return set_error(PFC_ERR_CUDA, std::string("clear: ") + cudaGetErrorString(e));
    launch_reduce_real<R>(c.stream, RED_SUM, reinterpret_cast<const R *>(state), nullptr, g.nreal, part, status);
    launch_finish(c.stream, part, RED_BLOCKS, 1.0 / (double)g.nreal, mean);
    // status word and table marker, read back once per call
    struct {
        int status, pad;
        unsigned long long mark;
    } hdr{};
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&hdr, base + OFF_STATUS, sizeof(hdr), cudaMemcpyDeviceToHost, c.stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c.stream)) != cudaSuccess)
        return set_error(PFC_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (hdr.mark != TABLES_MARK) {
        // first call on this device, or the array was wiped by a device reset
        if ((e = upload_tables(base)) != cudaSuccess)
            return set_error(PFC_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
        // a reset also dropped the kernels' shared-memory limits
        if ((e = raise_attrs(c, sizeof(R) == 8 ? PFC_FP64 : PFC_FP32_MIXED)) != cudaSuccess)
            return set_error(PFC_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
    }
    if (hdr.status & STATUS_NONFINITE)
        return set_error(PFC_ERR_NONFINITE, "the state holds NaN or Inf (left unchanged)");
    if ((e = cudaMemsetAsync(base + OFF_WORK, 0, 2 * align256(g.nhalf * vb), c.stream)) != cudaSuccess)
        return set_error(PFC_ERR_CUDA, std::string("clear: ") + cudaGetErrorString(e));

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
    if (!std::isfinite(op->r) || !std::isfinite(op->R1) || !std::isfinite(op->q2))
        return set_error(PFC_ERR_INVALID_ARG, "operator coefficients must be finite");
    if (nsteps < 0) return set_error(PFC_ERR_INVALID_ARG, "nsteps must be >= 0");
    if ((reinterpret_cast<uintptr_t>(state) & 15) != 0)
        return set_error(PFC_ERR_INVALID_ARG, "state must be 16-byte aligned");
    int64_t d[3] = {1, 1, 1};
    for (int i = 0; i < ndim; ++i) d[3 - ndim + i] = dims[i];
    for (int i = 3 - ndim; i < 3; ++i)
        if (!is_pow2(d[i]) || d[i] < 16 || d[i] > 4096)
            return set_error(PFC_ERR_UNSUPPORTED, "every extent must be a power of two in [16, 4096]");
    // the two unpadded half spectra are a lower bound of the work arrays: reject on the host
    // before any device query when even they do not fit
    const size_t vb = precision == PFC_FP64 ? 16 : 8;
    const size_t half_min = (size_t)(d[0] * d[1] * (d[2] / 2 + 1)) * vb;
    if (OFF_WORK + 2 * align256(half_min) > NOALLOC_BYTES)
        return set_error(PFC_ERR_UNSUPPORTED,
                         "grid too large for the 24 MiB static scratch of pfc_step_noalloc (needs at least " +
                             std::to_string(OFF_WORK + 2 * align256(half_min)) + " bytes); use pfc_plan_create");
    if (nsteps == 0) return PFC_OK;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(PFC_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    const Key key{dev, d[0], d[1], d[2], dx, dt, op->kind, op->r, op->R1, op->q2, precision};
    Prepared prep;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_prepared.find(key);
        if (it == g_prepared.end()) it = g_prepared.emplace(key, prepare(dev, d, ndim, dx, dt, *op, precision)).first;
        prep = it->second;
    }
    if (prep.status != PFC_OK) return set_error(prep.status, prep.msg);
    unsigned char *base = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&base, g_noalloc_scratch)) != cudaSuccess)
        return set_error(PFC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    const LaunchCfg c = launch_cfg(prep.t, reinterpret_cast<cudaStream_t>(stream));
    return precision == PFC_FP64 ? run<double>(c, base, *op, dx, dt, state, nsteps)
                                 : run<float>(c, base, *op, dx, dt, state, nsteps);
}
