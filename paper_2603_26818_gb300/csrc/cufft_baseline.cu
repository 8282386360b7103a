// Baseline only: the plain semi-implicit PFC step written the straightforward way with vendor
// cuFFT (D2Z/Z2D in FP64, R2C/C2R in FP32) and two elementwise kernels:
//   psi_hat = FFT(psi); c = psi^3; N_hat = FFT(c);
//   psi_hat = (psi_hat - dt k^2 N_hat) / ((1 + dt k^2 Lk) N);  psi = IFFT(psi_hat).
// It is timed beside the fused kernels of libpfc.so; the product library does not use it.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <cstdint>

namespace {

template <typename R> struct CT;
template <> struct CT<double> { using C = cufftDoubleComplex; };
template <> struct CT<float> { using C = cufftComplex; };

template <typename R> __global__ void k_cube(const R *__restrict__ x, R *__restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R v = x[i];
        y[i] = v * v * v;
    }
}

template <typename R>
__global__ void k_update(typename CT<R>::C *__restrict__ ph, const typename CT<R>::C *__restrict__ nh,
                         int nz, int ny, int nxh, int nx, double dx, double dt, int kind, double r,
                         double R1, double q2, double invN) {
    const int64_t h = (int64_t)nz * ny * nxh;
    const R two_pi = (R)6.28318530717958647692528676655900576839;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < h; i += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % nxh);
        const int64_t row = i / nxh;
        const int ky = (int)(row % ny), kz = (int)(row / ny);
        const int my = ky <= ny / 2 ? ky : ky - ny, mz = kz <= nz / 2 ? kz : kz - nz;
        const R fx = two_pi * kx / (R)(nx * dx), fy = two_pi * my / (R)(ny * dx), fz = two_pi * mz / (R)(nz * dx);
        const R k2 = fx * fx + fy * fy + fz * fz;
        const R a = (R)1 - k2;
        R lk;
        if (kind == 0) lk = (R)r + a * a;
        else { const R b = (R)(q2 * q2) - k2; lk = (R)r + a * a * ((R)R1 + b * b); }
        const R inv = (R)invN / ((R)1 + (R)dt * k2 * lk);
        const R cb = (R)dt * k2;
        typename CT<R>::C p = ph[i];
        const typename CT<R>::C q = nh[i];
        p.x = (p.x - cb * q.x) * inv;
        p.y = (p.y - cb * q.y) * inv;
        ph[i] = p;
    }
}

struct Base {
    int prec;  // 0 fp64, 1 fp32
    int nz, ny, nx;
    double dx, dt;
    int kind;
    double r, R1, q2;
    cudaStream_t stream;
    cufftHandle fwd, inv;
    void *ph, *nh, *cube;
};

}  // namespace

extern "C" {

int pfcb_create(void **out, int ndim, const int64_t *dims, double dx, double dt, int kind, double r,
                double R1, double q2, int precision, void *stream) {
    Base *b = new Base();
    b->prec = precision;
    b->nz = ndim == 3 ? (int)dims[0] : 1;
    b->ny = (int)dims[ndim - 2];
    b->nx = (int)dims[ndim - 1];
    b->dx = dx; b->dt = dt; b->kind = kind; b->r = r; b->R1 = R1; b->q2 = q2;
    b->stream = (cudaStream_t)stream;
    int n[3] = {b->nz, b->ny, b->nx};
    int *nn = ndim == 3 ? n : n + 1;
    const bool f64 = precision == 0;
    if (cufftPlanMany(&b->fwd, ndim, nn, nullptr, 1, 0, nullptr, 1, 0, f64 ? CUFFT_D2Z : CUFFT_R2C, 1) != CUFFT_SUCCESS) return 5;
    if (cufftPlanMany(&b->inv, ndim, nn, nullptr, 1, 0, nullptr, 1, 0, f64 ? CUFFT_Z2D : CUFFT_C2R, 1) != CUFFT_SUCCESS) return 5;
    cufftSetStream(b->fwd, b->stream);
    cufftSetStream(b->inv, b->stream);
    const size_t rb = f64 ? 8 : 4;
    const size_t h = (size_t)b->nz * b->ny * (b->nx / 2 + 1);
    if (cudaMalloc(&b->ph, h * 2 * rb) != cudaSuccess) return 4;
    if (cudaMalloc(&b->nh, h * 2 * rb) != cudaSuccess) return 4;
    if (cudaMalloc(&b->cube, (size_t)b->nz * b->ny * b->nx * rb) != cudaSuccess) return 4;
    *out = b;
    return 0;
}

int pfcb_step(void *h, void *state, int64_t nsteps) {
    Base *b = (Base *)h;
    const int64_t n = (int64_t)b->nz * b->ny * b->nx;
    const int nxh = b->nx / 2 + 1;
    const int64_t hh = (int64_t)b->nz * b->ny * nxh;
    const double invN = 1.0 / (double)n;
    for (int64_t s = 0; s < nsteps; ++s) {
        if (b->prec == 0) {
            double *x = (double *)state;
            if (cufftExecD2Z(b->fwd, x, (cufftDoubleComplex *)b->ph) != CUFFT_SUCCESS) return 5;
            k_cube<double><<<1216, 256, 0, b->stream>>>(x, (double *)b->cube, n);
            if (cufftExecD2Z(b->fwd, (double *)b->cube, (cufftDoubleComplex *)b->nh) != CUFFT_SUCCESS) return 5;
            k_update<double><<<1216, 256, 0, b->stream>>>((cufftDoubleComplex *)b->ph, (const cufftDoubleComplex *)b->nh,
                                                          b->nz, b->ny, nxh, b->nx, b->dx, b->dt, b->kind, b->r, b->R1, b->q2, invN);
            if (cufftExecZ2D(b->inv, (cufftDoubleComplex *)b->ph, x) != CUFFT_SUCCESS) return 5;
        } else {
            float *x = (float *)state;
            if (cufftExecR2C(b->fwd, x, (cufftComplex *)b->ph) != CUFFT_SUCCESS) return 5;
            k_cube<float><<<1216, 256, 0, b->stream>>>(x, (float *)b->cube, n);
            if (cufftExecR2C(b->fwd, (float *)b->cube, (cufftComplex *)b->nh) != CUFFT_SUCCESS) return 5;
            k_update<float><<<1216, 256, 0, b->stream>>>((cufftComplex *)b->ph, (const cufftComplex *)b->nh,
                                                         b->nz, b->ny, nxh, b->nx, b->dx, b->dt, b->kind, b->r, b->R1, b->q2, invN);
            if (cufftExecC2R(b->inv, (cufftComplex *)b->ph, x) != CUFFT_SUCCESS) return 5;
        }
    }
    (void)hh;
    return cudaGetLastError() == cudaSuccess ? 0 : 5;
}

int pfcb_destroy(void *h) {
    Base *b = (Base *)h;
    if (!b) return 0;
    cudaStreamSynchronize(b->stream);
    cufftDestroy(b->fwd);
    cufftDestroy(b->inv);
    cudaFree(b->ph);
    cudaFree(b->nh);
    cudaFree(b->cube);
    delete b;
    return 0;
}

}  // extern "C"
