// Amplitude-expansion PFC (pfc_apfc_* of pfc.h): host logic and the kernels' instantiations.
// The model, its passes and their sweeps are described in pfc_apfc.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

#include "pfc_apfc.cuh"
#include "pfc_host.h"

using namespace pfc;

struct pfc_apfc {
    int ndim = 2, namp = 0, prec = PFC_FP32_MIXED;
    int n[3] = {1, 1, 1};      // nx, ny, nz
    double dx = 0, dt = 0, psibar = 0;
    pfc_op op{};
    std::vector<double> kv;    // namp x 3 (x, y, z)
    ApGeom g{};
    void *S = nullptr, *T = nullptr;   // carried spectra and the work array, namp fields each
    void *tw = nullptr;
    int *term_beg = nullptr;
    int4 *terms = nullptr;
    void *coef = nullptr;
    int rows_nl = 1;           // rows a block of the x pass of a step
    int colW[3] = {0, 0, 0};   // columns a block of the y and z passes
    size_t smem_nl = 0, smem_io = 0, smem_col = 0;
    cudaStream_t stream = nullptr;
};

namespace {

constexpr int AP_IO_LINES = 8;   // lines a block of the entry and exit x passes

// radices of a complex line of n points: 7, 5, 3 first, then 8, 4, 2 (false for another prime)
bool ap_factor(int n, std::vector<int> &rad) {
    rad.clear();
    for (int r : {7, 5, 3})
        while (n % r == 0) { rad.push_back(r); n /= r; }
    while (n % 8 == 0) { rad.push_back(8); n /= 8; }
    if (n % 4 == 0) { rad.push_back(4); n /= 4; }
    if (n % 2 == 0) { rad.push_back(2); n /= 2; }
    return n == 1 && (int)rad.size() <= MR_MAXST;
}

// The resonances of amplitude j: signed modes (a, b) with k_a + k_b = k_j and (a, b, c) with
// k_a + k_b + k_c = k_j, each unordered combination once with the number of ordered tuples it
// stands for. A match is exact to 1e-9 of the largest component.
struct Term {
    int a, b, c;   // c = 0: quadratic
    int count;
};
std::vector<std::vector<Term>> resonance_terms(const std::vector<double> &kv, int namp) {
    double scale = 1.0;
    for (double v : kv) scale = std::max(scale, std::fabs(v));
    const double tol = 1e-9 * scale;
    auto comp = [&](int s, int d) { return kv[3 * (std::abs(s) - 1) + d] * (s > 0 ? 1.0 : -1.0); };
    std::vector<int> modes;
    for (int i = 1; i <= namp; ++i) {
        modes.push_back(i);
        modes.push_back(-i);
    }
    std::vector<std::vector<Term>> out(namp);
    for (int j = 0; j < namp; ++j) {
        std::map<std::tuple<int, int, int>, int> cnt;
        for (int a : modes)
            for (int b : modes) {
                bool ok = true;
                for (int d = 0; d < 3 && ok; ++d) ok = std::fabs(comp(a, d) + comp(b, d) - kv[3 * j + d]) <= tol;
                if (ok) ++cnt[std::make_tuple(std::min(a, b), std::max(a, b), 0)];
                for (int c : modes) {
                    bool ok3 = true;
                    for (int d = 0; d < 3 && ok3; ++d)
                        ok3 = std::fabs(comp(a, d) + comp(b, d) + comp(c, d) - kv[3 * j + d]) <= tol;
                    if (!ok3) continue;
                    int s[3] = {a, b, c};
                    std::sort(s, s + 3);
                    ++cnt[std::make_tuple(s[0], s[1], s[2])];
                }
            }
        for (auto &kvp : cnt)
            out[j].push_back(Term{std::get<0>(kvp.first), std::get<1>(kvp.first), std::get<2>(kvp.first), kvp.second});
    }
    return out;
}

template <typename R> ApArgs<R> ap_args(const pfc_apfc *h) {
    ApArgs<R> a{};
    a.tw = reinterpret_cast<const typename VT<R>::V *>(h->tw);
    a.scale = (R)(1.0 / (double)h->g.npts);
    a.dt = (R)h->dt;
    a.inv_n = (R)(1.0 / (double)h->g.npts);
    const double two_pi = 6.28318530717958647692528676655900576839;
    a.cx = (R)(two_pi / (h->n[0] * h->dx));
    a.cy = (R)(two_pi / (h->n[1] * h->dx));
    a.cz = (R)(two_pi / (h->n[2] * h->dx));
    for (int j = 0; j < h->namp; ++j) {
        a.kx[j] = (R)h->kv[3 * j];
        a.ky[j] = (R)h->kv[3 * j + 1];
        a.kz[j] = (R)h->kv[3 * j + 2];
    }
    a.op = OpR<R>{h->op.kind, (R)h->op.r, (R)h->op.R1, (R)(h->op.q2 * h->op.q2)};
    a.c1 = (R)(3.0 * h->psibar * h->psibar);
    a.term_beg = h->term_beg;
    a.terms = h->terms;
    a.coef = reinterpret_cast<const R *>(h->coef);
    return a;
}

template <typename R> void launch_col(const pfc_apfc *h, const ApArgs<R> &a, int mode, int axis, const void *in,
                                      void *out) {
    const int W = h->colW[axis];
    const dim3 grid((h->n[0] + W - 1) / W, axis == 1 ? h->n[2] : h->n[1], h->namp);
    const size_t smem = mr_col_smem(h->g.ax[axis].n, W, sizeof(R) * 2);
    if (mode == AP_COL_FWD) k_ap_col<R, AP_COL_FWD><<<grid, 32 * W, smem, h->stream>>>(h->g, a, axis, in, out);
    else if (mode == AP_COL_INV) k_ap_col<R, AP_COL_INV><<<grid, 32 * W, smem, h->stream>>>(h->g, a, axis, in, out);
    else k_ap_col<R, AP_COL_UPDATE><<<grid, 32 * W, smem, h->stream>>>(h->g, a, axis, in, out);
}

template <typename R> void launch_row_io(const pfc_apfc *h, const ApArgs<R> &a, int mode, const void *in, void *out) {
    const int64_t lines = (int64_t)h->n[1] * h->n[2] * h->namp;
    const dim3 grid((unsigned)((lines + AP_IO_LINES - 1) / AP_IO_LINES));
    if (mode == AP_ROW_FWD) k_ap_row_io<R, AP_ROW_FWD><<<grid, 32 * AP_IO_LINES, h->smem_io, h->stream>>>(h->g, a, in, out);
    else k_ap_row_io<R, AP_ROW_INV><<<grid, 32 * AP_IO_LINES, h->smem_io, h->stream>>>(h->g, a, in, out);
}

template <typename R> void launch_row_nl(const pfc_apfc *h, const ApArgs<R> &a) {
    const int64_t rows = (int64_t)h->n[1] * h->n[2];
    const dim3 grid((unsigned)((rows + h->rows_nl - 1) / h->rows_nl));
    k_ap_row_nl<R><<<grid, 32 * h->namp * h->rows_nl, h->smem_nl, h->stream>>>(h->g, a, h->T, h->rows_nl);
}

template <typename R> cudaError_t set_attrs(const pfc_apfc *h) {
    cudaError_t e = cudaSuccess;
    auto raise = [&](const void *fn, size_t bytes) {
        if (e != cudaSuccess) return;
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, fn);
        if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < bytes)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    raise(reinterpret_cast<const void *>(k_ap_col<R, AP_COL_FWD>), h->smem_col);
    raise(reinterpret_cast<const void *>(k_ap_col<R, AP_COL_INV>), h->smem_col);
    raise(reinterpret_cast<const void *>(k_ap_col<R, AP_COL_UPDATE>), h->smem_col);
    raise(reinterpret_cast<const void *>(k_ap_row_io<R, AP_ROW_FWD>), h->smem_io);
    raise(reinterpret_cast<const void *>(k_ap_row_io<R, AP_ROW_INV>), h->smem_io);
    raise(reinterpret_cast<const void *>(k_ap_row_nl<R>), h->smem_nl);
    return e;
}

// nsteps steps of the amplitudes in eta (real space, [amp][z][y][x] complex), in place.
template <typename R> pfc_status apfc_step_impl(pfc_apfc *h, void *eta, int64_t nsteps) {
    const ApArgs<R> a = ap_args<R>(h);
    ApArgs<R> a1 = a;          // the inner forward pass of 3D grids: unscaled
    a1.scale = (R)1;
    const int last = h->ndim == 3 ? 2 : 1;
    // entry: S = F(eta) / N
    launch_row_io<R>(h, a, AP_ROW_FWD, eta, h->T);
    if (h->ndim == 3) launch_col<R>(h, a1, AP_COL_FWD, 1, h->T, h->T);
    launch_col<R>(h, a, AP_COL_FWD, last, h->T, h->S);
    for (int64_t s = 0; s < nsteps; ++s) {
        launch_col<R>(h, a, AP_COL_INV, last, h->S, h->T);
        if (h->ndim == 3) launch_col<R>(h, a, AP_COL_INV, 1, h->T, h->T);
        launch_row_nl<R>(h, a);
        if (h->ndim == 3) launch_col<R>(h, a1, AP_COL_FWD, 1, h->T, h->T);
        launch_col<R>(h, a, AP_COL_UPDATE, last, h->T, h->S);
    }
    // exit: eta = F^-1(S)
    launch_col<R>(h, a, AP_COL_INV, last, h->S, h->T);
    if (h->ndim == 3) launch_col<R>(h, a, AP_COL_INV, 1, h->T, h->T);
    launch_row_io<R>(h, a, AP_ROW_INV, h->T, eta);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PFC_ERR_CUDA, std::string("apfc launch: ") + cudaGetErrorString(e));
    return PFC_OK;
}

}  // namespace

namespace {

void free_apfc(pfc_apfc *h) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->S); cudaFree(h->T); cudaFree(h->tw);
    cudaFree(h->term_beg); cudaFree(h->terms); cudaFree(h->coef);
    delete h;
}

}  // namespace

extern "C" {

pfc_status pfc_apfc_create(pfc_apfc **out, int ndim, const int64_t *dims, double dx, double dt, const pfc_op *op,
                           int namp, const double *kvecs, double psibar, int precision, void *stream) {
    if (!out || !dims || !op || !kvecs) return set_error(PFC_ERR_INVALID_ARG, "null pointer argument");
    if (ndim != 2 && ndim != 3) return set_error(PFC_ERR_INVALID_ARG, "ndim must be 2 or 3");
    if (namp < 1 || namp > AP_MAXAMP) return set_error(PFC_ERR_INVALID_ARG, "namp must be in [1, 16]");
    if (!(dx > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dt) || !std::isfinite(psibar))
        return set_error(PFC_ERR_INVALID_ARG, "dx and dt must be finite and > 0, psibar finite");
    if (precision != PFC_FP64 && precision != PFC_FP32_MIXED) return set_error(PFC_ERR_INVALID_ARG, "unknown precision");
    if ((op->kind != PFC_ONE_MODE && op->kind != PFC_TWO_MODE) || !std::isfinite(op->r) || !std::isfinite(op->R1) ||
        !std::isfinite(op->q2))
        return set_error(PFC_ERR_INVALID_ARG, "bad operator");
    int n[3] = {1, 1, 1};
    for (int d = 0; d < ndim; ++d) {
        const int64_t v = dims[ndim - 1 - d];
        std::vector<int> rad;
        if (v < 8 || v > 4096 || !ap_factor((int)v, rad))
            return set_error(PFC_ERR_UNSUPPORTED, "extents must be in [8, 4096] with prime factors 2, 3, 5, 7");
        n[d] = (int)v;
    }
    std::vector<double> kv(3 * namp, 0.0);
    double kmax = 0.0;
    for (int j = 0; j < namp; ++j) {
        double k2 = 0;
        for (int d = 0; d < ndim; ++d) {
            const double v = kvecs[ndim * j + d];
            if (!std::isfinite(v)) return set_error(PFC_ERR_INVALID_ARG, "k vectors must be finite");
            kv[3 * j + d] = v;
            k2 += v * v;
        }
        kmax = std::max(kmax, std::sqrt(k2));
    }
    // 1 + dt Q L(Q) > 0 for every Q = |k_j + q|^2 on the grid
    double qmax2 = 0;
    for (int d = 0; d < ndim; ++d) qmax2 += (M_PI / dx) * (M_PI / dx);
    const double Qmax = (kmax + std::sqrt(qmax2)) * (kmax + std::sqrt(qmax2));
    if (min_implicit(op, 1, 0.0, dt, Qmax) <= 0.0)
        return set_error(PFC_ERR_UNSTABLE_OPERATOR, "1 + dt Q L(Q) is not positive for some shifted wavevector");

    pfc_apfc *h = new pfc_apfc();
    h->ndim = ndim;
    h->namp = namp;
    h->prec = precision;
    for (int d = 0; d < 3; ++d) h->n[d] = n[d];
    h->dx = dx;
    h->dt = dt;
    h->psibar = psibar;
    h->op = *op;
    h->kv = kv;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    ApGeom &g = h->g;
    g.nx = n[0]; g.ny = n[1]; g.nz = n[2]; g.ndim = ndim; g.namp = namp;
    g.npts = (int64_t)n[0] * n[1] * n[2];
    const size_t vb = precision == PFC_FP64 ? 16 : 8;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        delete h;
        return set_error(PFC_ERR_CUDA, "device query failed");
    }
    // stage twiddles of the three axes
    std::vector<double> tw;
    for (int a = 0; a < 3; ++a) {
        MrAxis &ax = g.ax[a];
        ax.n = n[a];
        std::vector<int> rad;
        if (ax.n > 1) ap_factor(ax.n, rad);
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
    // launch shapes: up to 100 KB of shared memory a block (two blocks an SM)
    const size_t budget = 100 * 1024;
    int rows = 1;
    while (rows * 2 * namp <= 16 && ap_row_smem(n[0], rows * 2 * namp, vb) <= budget) rows *= 2;
    h->rows_nl = rows;
    h->smem_nl = ap_row_smem(n[0], rows * namp, vb);
    h->smem_io = ap_row_smem(n[0], AP_IO_LINES, vb);
    for (int a = 1; a < ndim; ++a) {
        int W = vb == 8 ? 16 : 8;
        while (W > 1 && mr_col_smem(n[a], W, vb) > budget) W /= 2;
        h->colW[a] = W;
        h->smem_col = std::max(h->smem_col, mr_col_smem(n[a], W, vb));
    }
    if (h->smem_nl > (size_t)optin || h->smem_io > (size_t)optin || h->smem_col > (size_t)optin) {
        delete h;
        return set_error(PFC_ERR_UNSUPPORTED, "a line of this grid does not fit shared memory");
    }
    // resonance terms and their coefficients
    const std::vector<std::vector<Term>> terms = resonance_terms(kv, namp);
    std::vector<int> beg(namp + 1, 0);
    std::vector<int4> tv;
    std::vector<double> cv;
    for (int j = 0; j < namp; ++j) {
        for (const Term &t : terms[j]) {
            tv.push_back(int4{t.a, t.b, t.c, 0});
            cv.push_back(t.c == 0 ? 3.0 * psibar * t.count : (double)t.count);
        }
        beg[j + 1] = (int)tv.size();
    }
    if (tv.empty()) {
        tv.push_back(int4{1, 1, 0, 0});   // a placeholder so the arrays exist (never read)
        cv.push_back(0.0);
    }
    const size_t field = (size_t)g.npts * vb * namp;
    cudaError_t e;
    auto bail = [&](cudaError_t err) {
        free_apfc(h);
        return set_error(err == cudaErrorMemoryAllocation ? PFC_ERR_OUT_OF_MEMORY : PFC_ERR_CUDA,
                         std::string("apfc allocation: ") + cudaGetErrorString(err));
    };
    if ((e = cudaMalloc(&h->S, field)) != cudaSuccess || (e = cudaMalloc(&h->T, field)) != cudaSuccess ||
        (e = cudaMalloc(&h->tw, std::max<size_t>(tw.size(), 2) / 2 * vb)) != cudaSuccess ||
        (e = cudaMalloc(&h->term_beg, beg.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&h->terms, tv.size() * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc(&h->coef, cv.size() * (vb / 2))) != cudaSuccess)
        return bail(e);
    if ((e = cudaMemcpy(h->term_beg, beg.data(), beg.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->terms, tv.data(), tv.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e);
    if (precision == PFC_FP64) {
        if (!tw.empty() && (e = cudaMemcpy(h->tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e);
        if ((e = cudaMemcpy(h->coef, cv.data(), cv.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e);
        e = set_attrs<double>(h);
    } else {
        std::vector<float> t32(tw.begin(), tw.end()), c32(cv.begin(), cv.end());
        if (!t32.empty() && (e = cudaMemcpy(h->tw, t32.data(), t32.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e);
        if ((e = cudaMemcpy(h->coef, c32.data(), c32.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e);
        e = set_attrs<float>(h);
    }
    if (e != cudaSuccess) return bail(e);
    *out = h;
    return PFC_OK;
}

pfc_status pfc_apfc_step(pfc_apfc *h, void *eta, int64_t nsteps) {
    if (!h) return set_error(PFC_ERR_INVALID_ARG, "invalid apfc handle");
    if (!eta) return set_error(PFC_ERR_INVALID_ARG, "null amplitudes");
    if (nsteps < 0) return set_error(PFC_ERR_INVALID_ARG, "nsteps must be >= 0");
    if ((reinterpret_cast<uintptr_t>(eta) & 15) != 0) return set_error(PFC_ERR_INVALID_ARG, "amplitudes must be 16-byte aligned");
    if (nsteps == 0) return PFC_OK;
    return h->prec == PFC_FP64 ? apfc_step_impl<double>(h, eta, nsteps) : apfc_step_impl<float>(h, eta, nsteps);
}

pfc_status pfc_apfc_resonances(pfc_apfc *h, int32_t *count_out) {
    if (!h || !count_out) return set_error(PFC_ERR_INVALID_ARG, "null pointer argument");
    std::vector<int> beg(h->namp + 1);
    if (cudaMemcpy(beg.data(), h->term_beg, beg.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_error(PFC_ERR_CUDA, "apfc table read");
    *count_out = beg[h->namp];
    return PFC_OK;
}

pfc_status pfc_apfc_destroy(pfc_apfc *h) {
    if (!h) return PFC_OK;
    free_apfc(h);
    return PFC_OK;
}

}  // extern "C"
