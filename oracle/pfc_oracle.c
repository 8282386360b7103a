/*
 * Oracle: semi-implicit Fourier pseudo-spectral phase-field-crystal (PFC) step, FP64, CPU.
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously-correct restatement of what
 * the method computes. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg load it. The GPU library never links it, calls it or shares a line with it: the two
 * sides have separate headers, tables, FFTs and helpers.
 *
 * What is computed, with the paper's equation numbers:
 *   - Pseudo-spectral method (Section "Fourier pseudo-spectral method", Eqs. (1)-(4)):
 *     the field is held on an equispaced periodic grid; linear operators act in Fourier space
 *     as polynomials in k via (d/dx)^n -> (ik)^n; the polynomial nonlinearity is evaluated
 *     pointwise in real space and transformed.
 *   - PFC free energy Eq. (5): F = integral of psi/2 (eps + L) psi + psi^4/4, and the
 *     conserved dynamics Eq. (6): d_t psi = lap( (eps + L) psi + psi^3 ).
 *   - Semi-implicit time integration (the update of Listing 1): the linear part implicit,
 *     psi^3 explicit:
 *         psi_hat <- (psi_hat - dt k^2 FFT(psi^3)) / (1 + dt k^2 Lk(k)),
 *     with Lk(k) = eps + L evaluated at |k|.  One-mode form: Lk = r + (1-k^2)^2.
 *     Two-mode (tenth-order) form: Lk = r + (1-k^2)^2 (R1 + (q2^2-k^2)^2); the paper's
 *     FCC operator (1+lap)^2 (4/3+lap)^2 is R1 = 0, q2^2 = 4/3.
 *
 * Conventions (readings of the paper, each also listed in the design notes):
 *   - Arrays are row-major (nz, ny, nx), x fastest. 2D uses nz = 1.
 *   - Box length per axis is n*dx; k_m = 2 pi m~ / (n dx) with m~ in FFT order
 *     {0..n/2, -n/2+1..-1}.  Only k^2 enters the method, so the Nyquist sign is irrelevant.
 *   - Forward transforms are unnormalised, the inverse carries 1/N (MATLAB fft/ifft).
 *   - The real-to-complex transform keeps kx in [0, nx/2]; the complex-to-real transform
 *     ignores the imaginary parts of the kx = 0 and kx = nx/2 bins.
 *   - No de-aliasing of psi^3 (the paper applies none).
 *
 * Everything is FP64.  FFTs: an iterative radix-2 Cooley-Tukey for powers of two, a recursive
 * mixed-radix Cooley-Tukey (smallest prime factor first, naive DFT for the prime leaves)
 * for other lengths, and a naive O(n^2) DFT kept for the pins.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double TWO_PI = 6.28318530717958647692528676655900576839;

/* exp(sign * 2 pi i * num / den), with num reduced modulo den first. */
static cplx unit_root(int64_t num, int64_t den, int sign)
{
    int64_t m = num % den;
    if (m < 0) m += den;
    double ang = TWO_PI * (double)m / (double)den;
    return cos(ang) + (double)sign * sin(ang) * I;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* 1D transforms                                                                          */
/* ------------------------------------------------------------------------------------ */

/* Naive DFT from the definition: out[k] = sum_j in[j] exp(sign 2 pi i j k / n). */
void orc_dft(int64_t n, const cplx *in, cplx *out, int sign)
{
    for (int64_t k = 0; k < n; ++k) {
        cplx acc = 0;
        for (int64_t j = 0; j < n; ++j) acc += in[j] * unit_root(j * k, n, sign);
        out[k] = acc;
    }
}

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* Iterative radix-2 decimation-in-time FFT, in place. n must be a power of two. */
void orc_fft_radix2(int64_t n, cplx *x, int sign)
{
    for (int64_t i = 1, j = 0; i < n; ++i) {           /* bit-reversal permutation */
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len / 2;
        for (int64_t k = 0; k < half; ++k) {
            cplx w = unit_root(k, len, sign);
            for (int64_t s = 0; s < n; s += len) {
                cplx u = x[s + k], v = x[s + k + half] * w;
                x[s + k] = u + v;
                x[s + k + half] = u - v;
            }
        }
    }
}

static int64_t smallest_factor(int64_t n)
{
    for (int64_t p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* Recursive mixed-radix Cooley-Tukey: n = p m with p the smallest prime factor.
 * Y_r = DFT_m of the subsequence in[r], in[r+p], ...; X[k + m q] = sum_r W_n^{r(k+mq)} Y_r[k]. */
static void fft_mixed_rec(int64_t n, const cplx *in, int64_t stride, cplx *out, int sign)
{
    if (n == 1) { out[0] = in[0]; return; }
    int64_t p = smallest_factor(n), m = n / p;
    if (p == n) {                                       /* prime length: the definition */
        for (int64_t k = 0; k < n; ++k) {
            cplx acc = 0;
            for (int64_t j = 0; j < n; ++j) acc += in[j * stride] * unit_root(j * k, n, sign);
            out[k] = acc;
        }
        return;
    }
    cplx *y = malloc(sizeof(cplx) * n);
    for (int64_t r = 0; r < p; ++r) fft_mixed_rec(m, in + r * stride, stride * p, y + r * m, sign);
    for (int64_t k = 0; k < m; ++k)
        for (int64_t q = 0; q < p; ++q) {
            cplx acc = 0;
            for (int64_t r = 0; r < p; ++r) acc += y[r * m + k] * unit_root(r * (k + m * q), n, sign);
            out[k + m * q] = acc;
        }
    free(y);
}

void orc_fft_mixed(int64_t n, cplx *x, int sign)
{
    cplx *tmp = malloc(sizeof(cplx) * n);
    fft_mixed_rec(n, x, 1, tmp, sign);
    memcpy(x, tmp, sizeof(cplx) * n);
    free(tmp);
}

/* Unnormalised complex FFT of length n: radix-2 for powers of two, mixed radix otherwise. */
void orc_fft(int64_t n, cplx *x, int sign)
{
    if (n <= 1) return;
    if (is_pow2(n)) orc_fft_radix2(n, x, sign);
    else orc_fft_mixed(n, x, sign);
}

/* ------------------------------------------------------------------------------------ */
/* Multi-dimensional transforms on row-major (n0, n1, n2) arrays, axis by axis            */
/* ------------------------------------------------------------------------------------ */

/* Complex FFT along one axis of a (d0, d1, d2) complex array. */
static void fft_axis(cplx *a, int64_t d0, int64_t d1, int64_t d2, int axis, int sign)
{
    int64_t len = axis == 0 ? d0 : (axis == 1 ? d1 : d2);
    if (len <= 1) return;
    int64_t stride = axis == 0 ? d1 * d2 : (axis == 1 ? d2 : 1);
    int64_t nlines = d0 * d1 * d2 / len;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * len);
#pragma omp for schedule(static)
        for (int64_t l = 0; l < nlines; ++l) {
            /* line l -> base offset: the two non-axis indices in row-major order */
            int64_t base;
            if (axis == 2) base = l * d2;
            else if (axis == 1) base = (l / d2) * d1 * d2 + (l % d2);
            else base = l;
            for (int64_t j = 0; j < len; ++j) buf[j] = a[base + j * stride];
            orc_fft(len, buf, sign);
            for (int64_t j = 0; j < len; ++j) a[base + j * stride] = buf[j];
        }
        free(buf);
    }
}

/* Real-to-complex forward transform, unnormalised.
 * in: real (nz, ny, nx); out: complex (nz, ny, nx/2+1). */
void orc_rfftn(int64_t nz, int64_t ny, int64_t nx, const double *in, cplx *out)
{
    int64_t nxh = nx / 2 + 1;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * nx);
#pragma omp for schedule(static)
        for (int64_t row = 0; row < nz * ny; ++row) {
            for (int64_t x = 0; x < nx; ++x) buf[x] = in[row * nx + x];
            orc_fft(nx, buf, -1);
            for (int64_t k = 0; k < nxh; ++k) out[row * nxh + k] = buf[k];
        }
        free(buf);
    }
    fft_axis(out, nz, ny, nxh, 1, -1);
    fft_axis(out, nz, ny, nxh, 0, -1);
}

/* Complex-to-real inverse transform with the 1/N factor.
 * in: complex (nz, ny, nx/2+1), not modified; out: real (nz, ny, nx). */
void orc_irfftn(int64_t nz, int64_t ny, int64_t nx, const cplx *in, double *out)
{
    int64_t nxh = nx / 2 + 1, n = nz * ny * nx;
    cplx *work = malloc(sizeof(cplx) * nz * ny * nxh);
    memcpy(work, in, sizeof(cplx) * nz * ny * nxh);
    fft_axis(work, nz, ny, nxh, 0, +1);
    fft_axis(work, nz, ny, nxh, 1, +1);
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * nx);
#pragma omp for schedule(static)
        for (int64_t row = 0; row < nz * ny; ++row) {
            const cplx *h = work + row * nxh;
            for (int64_t k = 0; k < nx; ++k) {
                if (k < nxh) {
                    cplx v = h[k];
                    if (k == 0 || 2 * k == nx) v = creal(v);   /* imaginary part ignored */
                    buf[k] = v;
                } else {
                    buf[k] = conj(h[nx - k]);
                }
            }
            orc_fft(nx, buf, +1);
            for (int64_t x = 0; x < nx; ++x) out[row * nx + x] = creal(buf[x]) / (double)n;
        }
        free(buf);
    }
    free(work);
}

/* ------------------------------------------------------------------------------------ */
/* PFC model                                                                              */
/* ------------------------------------------------------------------------------------ */

/* Wavenumber of FFT index m on an axis of n points and spacing dx (box length n dx). */
static double wavenumber(int64_t m, int64_t n, double dx)
{
    int64_t mt = (m <= n / 2) ? m : m - n;
    return TWO_PI * (double)mt / ((double)n * dx);
}

/* |k|^2 at half-spectrum index (iz, iy, ikx). */
static double ksq(int64_t iz, int64_t iy, int64_t ikx, int64_t nz, int64_t ny, int64_t nx, double dx)
{
    double kx = wavenumber(ikx, nx, dx), ky = wavenumber(iy, ny, dx), kz = wavenumber(iz, nz, dx);
    return kx * kx + ky * ky + kz * kz;
}

/* Linear PFC symbol Lk(k^2) = eps + L: kind 0 one-mode, kind 1 two-mode (tenth order). */
double orc_lin_op(int kind, double r, double R1, double q2, double k2)
{
    double a = 1.0 - k2;
    if (kind == 0) return r + a * a;
    double b = q2 * q2 - k2;
    return r + a * a * (R1 + b * b);
}

/* One or more semi-implicit steps, in place on the real field psi (nz, ny, nx):
 *   psi_hat = FFT(psi), N_hat = FFT(psi^3),
 *   psi_hat <- (psi_hat - dt k^2 N_hat) / (1 + dt k^2 Lk(k)),  psi = IFFT(psi_hat). */
void orc_step(int64_t nz, int64_t ny, int64_t nx, double dx, double dt,
              int kind, double r, double R1, double q2, double *psi, int64_t nsteps)
{
    int64_t n = nz * ny * nx, nxh = nx / 2 + 1, h = nz * ny * nxh;
    cplx *ph = malloc(sizeof(cplx) * h), *nh = malloc(sizeof(cplx) * h);
    double *cube = malloc(sizeof(double) * n);
    for (int64_t s = 0; s < nsteps; ++s) {
        orc_rfftn(nz, ny, nx, psi, ph);
        for (int64_t j = 0; j < n; ++j) cube[j] = psi[j] * psi[j] * psi[j];
        orc_rfftn(nz, ny, nx, cube, nh);
        for (int64_t iz = 0; iz < nz; ++iz)
            for (int64_t iy = 0; iy < ny; ++iy)
                for (int64_t ik = 0; ik < nxh; ++ik) {
                    int64_t idx = (iz * ny + iy) * nxh + ik;
                    double k2 = ksq(iz, iy, ik, nz, ny, nx, dx);
                    double lk = orc_lin_op(kind, r, R1, q2, k2);
                    ph[idx] = (ph[idx] - dt * k2 * nh[idx]) / (1.0 + dt * k2 * lk);
                }
        orc_irfftn(nz, ny, nx, ph, psi);
    }
    free(ph); free(nh); free(cube);
}

/* Alternative time integrators of the same spectral system. The paper integrates with the
 * semi-implicit scheme above and notes that other time-integration schemes can be used. Each
 * Fourier mode obeys d/dt psi_hat = -k^2 (Lk psi_hat + N_hat), N = psi^3 (Eq. (6)); one step of
 *   scheme 0  semi-implicit Euler (orc_step);
 *   scheme 1  stabilised semi-implicit Euler with a constant S: S psi is added to the implicit
 *             linear part and taken away from the explicit part,
 *               psi_hat <- ((1 + dt k^2 S) psi_hat - dt k^2 N_hat) / (1 + dt k^2 (Lk + S));
 *   scheme 2  second-order semi-implicit backward differentiation: BDF2 for the linear part
 *             and the nonlinear part extrapolated to t_{n+1} from t_n and t_{n-1},
 *               (3 psi_hat^{n+1} - 4 psi_hat^n + psi_hat^{n-1}) / (2 dt)
 *                   = -k^2 (Lk psi_hat^{n+1} + 2 N_hat^n - N_hat^{n-1}),
 *             the first step of a call being one step of scheme 0 (the call's nsteps steps are
 *             one run: the two previous levels are carried inside the call only). */
void orc_step_scheme(int64_t nz, int64_t ny, int64_t nx, double dx, double dt, int kind, double r,
                     double R1, double q2, int scheme, double S, double *psi, int64_t nsteps)
{
    int64_t n = nz * ny * nx, nxh = nx / 2 + 1, h = nz * ny * nxh;
    cplx *ph = malloc(sizeof(cplx) * h), *nh = malloc(sizeof(cplx) * h);
    cplx *ph_old = malloc(sizeof(cplx) * h), *nh_old = malloc(sizeof(cplx) * h);
    double *cube = malloc(sizeof(double) * n);
    for (int64_t s = 0; s < nsteps; ++s) {
        orc_rfftn(nz, ny, nx, psi, ph);
        for (int64_t j = 0; j < n; ++j) cube[j] = psi[j] * psi[j] * psi[j];
        orc_rfftn(nz, ny, nx, cube, nh);
        for (int64_t iz = 0; iz < nz; ++iz)
            for (int64_t iy = 0; iy < ny; ++iy)
                for (int64_t ik = 0; ik < nxh; ++ik) {
                    int64_t idx = (iz * ny + iy) * nxh + ik;
                    double k2 = ksq(iz, iy, ik, nz, ny, nx, dx);
                    double lk = orc_lin_op(kind, r, R1, q2, k2);
                    cplx next;
                    if (scheme == 1)
                        next = ((1.0 + dt * k2 * S) * ph[idx] - dt * k2 * nh[idx]) / (1.0 + dt * k2 * (lk + S));
                    else if (scheme == 2 && s > 0)
                        next = (4.0 * ph[idx] - ph_old[idx] - 2.0 * dt * k2 * (2.0 * nh[idx] - nh_old[idx])) /
                               (3.0 + 2.0 * dt * k2 * lk);
                    else
                        next = (ph[idx] - dt * k2 * nh[idx]) / (1.0 + dt * k2 * lk);
                    ph_old[idx] = ph[idx];
                    nh_old[idx] = nh[idx];
                    ph[idx] = next;
                }
        orc_irfftn(nz, ny, nx, ph, psi);
    }
    free(ph); free(nh); free(ph_old); free(nh_old); free(cube);
}

/* ------------------------------------------------------------------------------------ */
/* Hydrodynamic PFC (the paper's multiphysics example, Eq. (hpfc))                          */
/* ------------------------------------------------------------------------------------ */

/* i k_j of half-spectrum index (iz, iy, ikx) along axis j (0 x, 1 y, 2 z), zero at the Nyquist
 * index of that axis (spectral first derivative of a real field). */
static cplx deriv_mult(int j, int64_t iz, int64_t iy, int64_t ikx, int64_t nz, int64_t ny, int64_t nx, double dx)
{
    int64_t m = j == 0 ? ikx : (j == 1 ? iy : iz), n = j == 0 ? nx : (j == 1 ? ny : nz);
    if (n > 1 && 2 * m == n) return 0;
    return I * wavenumber(m, n, dx);
}

/* One or more steps of the hydrodynamic PFC model
 *     d_t psi = lap(mu) - v . grad psi,      rho d_t v = Gamma lap v - < psi grad mu >,
 *     mu = Lk psi + psi^3 (the variational derivative of the PFC energy, Eq. (5)),
 * < . > the convolution with the normalised Gaussian of width a0, a multiplication by
 * exp(-a0^2 k^2 / 2) in Fourier space. The update follows the paper's multi-field listing:
 *     psi_hat' = (psi_hat - dt k^2 FFT(psi^3) - dt FFT(v . grad psi)) / (1 + dt k^2 Lk)
 *     psi' = IFFT(psi_hat'),   mu_hat' = FFT(psi'^3) + Lk psi_hat'
 *     v_hat_j' = (v_hat_j - (dt/rho) G FFT(psi' d_j mu')) / (1 + (dt/rho) Gamma k^2)
 * (the density first, with the old velocity; the velocity with the new density). grad and d_j
 * are spectral derivatives (deriv_mult). psi: real (nz, ny, nx); v: ndim real fields back to back
 * (ndim = 2 when nz = 1, else 3), x component first. rho may be +inf (the velocity then stays
 * put). */
void orc_hydro_step(int64_t nz, int64_t ny, int64_t nx, double dx, double dt, int kind, double r,
                    double R1, double q2, double rho, double gamma, double a0, double *psi, double *v,
                    int64_t nsteps)
{
    int64_t n = nz * ny * nx, nxh = nx / 2 + 1, h = nz * ny * nxh;
    int nd = nz > 1 ? 3 : 2;
    cplx *ph = malloc(sizeof(cplx) * h), *nh = malloc(sizeof(cplx) * h), *wk = malloc(sizeof(cplx) * h);
    cplx *mu = malloc(sizeof(cplx) * h), *fh = malloc(sizeof(cplx) * h);
    double *t1 = malloc(sizeof(double) * n), *t2 = malloc(sizeof(double) * n);
    double vf = dt / rho;
    for (int64_t s = 0; s < nsteps; ++s) {
        orc_rfftn(nz, ny, nx, psi, ph);
        for (int64_t i = 0; i < n; ++i) t1[i] = psi[i] * psi[i] * psi[i];
        orc_rfftn(nz, ny, nx, t1, nh);
        /* advection v . grad psi */
        for (int64_t i = 0; i < n; ++i) t2[i] = 0;
        for (int j = 0; j < nd; ++j) {
            for (int64_t iz = 0; iz < nz; ++iz)
                for (int64_t iy = 0; iy < ny; ++iy)
                    for (int64_t ik = 0; ik < nxh; ++ik) {
                        int64_t idx = (iz * ny + iy) * nxh + ik;
                        wk[idx] = deriv_mult(j, iz, iy, ik, nz, ny, nx, dx) * ph[idx];
                    }
            orc_irfftn(nz, ny, nx, wk, t1);
            for (int64_t i = 0; i < n; ++i) t2[i] += v[j * n + i] * t1[i];
        }
        orc_rfftn(nz, ny, nx, t2, fh);
        for (int64_t iz = 0; iz < nz; ++iz)
            for (int64_t iy = 0; iy < ny; ++iy)
                for (int64_t ik = 0; ik < nxh; ++ik) {
                    int64_t idx = (iz * ny + iy) * nxh + ik;
                    double k2 = ksq(iz, iy, ik, nz, ny, nx, dx);
                    double lk = orc_lin_op(kind, r, R1, q2, k2);
                    ph[idx] = (ph[idx] - dt * k2 * nh[idx] - dt * fh[idx]) / (1.0 + dt * k2 * lk);
                }
        orc_irfftn(nz, ny, nx, ph, psi);
        /* chemical potential of the new density */
        for (int64_t i = 0; i < n; ++i) t1[i] = psi[i] * psi[i] * psi[i];
        orc_rfftn(nz, ny, nx, t1, nh);
        for (int64_t iz = 0; iz < nz; ++iz)
            for (int64_t iy = 0; iy < ny; ++iy)
                for (int64_t ik = 0; ik < nxh; ++ik) {
                    int64_t idx = (iz * ny + iy) * nxh + ik;
                    double k2 = ksq(iz, iy, ik, nz, ny, nx, dx);
                    mu[idx] = nh[idx] + orc_lin_op(kind, r, R1, q2, k2) * ph[idx];
                }
        for (int j = 0; j < nd; ++j) {
            for (int64_t iz = 0; iz < nz; ++iz)
                for (int64_t iy = 0; iy < ny; ++iy)
                    for (int64_t ik = 0; ik < nxh; ++ik) {
                        int64_t idx = (iz * ny + iy) * nxh + ik;
                        wk[idx] = deriv_mult(j, iz, iy, ik, nz, ny, nx, dx) * mu[idx];
                    }
            orc_irfftn(nz, ny, nx, wk, t1);
            for (int64_t i = 0; i < n; ++i) t1[i] *= psi[i];
            orc_rfftn(nz, ny, nx, t1, fh);
            orc_rfftn(nz, ny, nx, v + j * n, wk);
            for (int64_t iz = 0; iz < nz; ++iz)
                for (int64_t iy = 0; iy < ny; ++iy)
                    for (int64_t ik = 0; ik < nxh; ++ik) {
                        int64_t idx = (iz * ny + iy) * nxh + ik;
                        double k2 = ksq(iz, iy, ik, nz, ny, nx, dx);
                        double g = exp(-0.5 * a0 * a0 * k2);
                        wk[idx] = (wk[idx] - vf * g * fh[idx]) / (1.0 + vf * gamma * k2);
                    }
            orc_irfftn(nz, ny, nx, wk, v + j * n);
        }
    }
    free(ph); free(nh); free(wk); free(mu); free(fh); free(t1); free(t2);
}

/* Mass: the mean density (1/N) sum_j psi_j, i.e. psi_hat(k=0)/N. */
double orc_mass(int64_t n, const double *psi)
{
    double s = 0;
    for (int64_t j = 0; j < n; ++j) s += psi[j];
    return s / (double)n;
}

/* (Lk psi) in real space: IFFT(Lk(k) FFT(psi)). */
static void apply_lin(int64_t nz, int64_t ny, int64_t nx, double dx, int kind, double r, double R1,
                      double q2, const double *psi, double *out)
{
    int64_t nxh = nx / 2 + 1, h = nz * ny * nxh;
    cplx *ph = malloc(sizeof(cplx) * h);
    orc_rfftn(nz, ny, nx, psi, ph);
    for (int64_t iz = 0; iz < nz; ++iz)
        for (int64_t iy = 0; iy < ny; ++iy)
            for (int64_t ik = 0; ik < nxh; ++ik) {
                int64_t idx = (iz * ny + iy) * nxh + ik;
                ph[idx] *= orc_lin_op(kind, r, R1, q2, ksq(iz, iy, ik, nz, ny, nx, dx));
            }
    orc_irfftn(nz, ny, nx, ph, out);
    free(ph);
}

/* Energy density F/|Omega| of Eq. (5) on the grid: mean over points of psi (Lk psi)/2 + psi^4/4. */
double orc_energy(int64_t nz, int64_t ny, int64_t nx, double dx, int kind, double r, double R1,
                  double q2, const double *psi)
{
    int64_t n = nz * ny * nx;
    double *lp = malloc(sizeof(double) * n);
    apply_lin(nz, ny, nx, dx, kind, r, R1, q2, psi, lp);
    double f = 0;
    for (int64_t j = 0; j < n; ++j) {
        double p2 = psi[j] * psi[j];
        f += 0.5 * psi[j] * lp[j] + 0.25 * p2 * p2;
    }
    free(lp);
    return f / (double)n;
}

/* ------------------------------------------------------------------------------------ */
/* Two coupled conserved fields (density psi, composition c)                              */
/* ------------------------------------------------------------------------------------ */
/* mu_psi = Lk_psi psi + psi^3 + alpha c,  mu_c = Lk_c c + c^3 + alpha psi,
 * d_t psi = lap mu_psi, d_t c = lap mu_c.  Semi-implicit: the linear terms (both Lk and the
 * alpha coupling) implicit, the cubes explicit, i.e. per mode the 2x2 system
 *   [1 + dt k^2 Lk_psi,  dt k^2 alpha    ] [psi_hat']   [psi_hat - dt k^2 N_psi]
 *   [dt k^2 alpha,       1 + dt k^2 Lk_c ] [c_hat'  ] = [c_hat   - dt k^2 N_c  ]
 * solved by Cramer's rule. */
void orc_step2(int64_t nz, int64_t ny, int64_t nx, double dx, double dt,
               int kind_p, double r_p, double R1_p, double q2_p,
               int kind_c, double r_c, double R1_c, double q2_c, double alpha,
               double *psi, double *c, int64_t nsteps)
{
    int64_t n = nz * ny * nx, nxh = nx / 2 + 1, h = nz * ny * nxh;
    cplx *ph = malloc(sizeof(cplx) * h), *nph = malloc(sizeof(cplx) * h);
    cplx *ch = malloc(sizeof(cplx) * h), *nch = malloc(sizeof(cplx) * h);
    double *cube = malloc(sizeof(double) * n);
    for (int64_t s = 0; s < nsteps; ++s) {
        orc_rfftn(nz, ny, nx, psi, ph);
        orc_rfftn(nz, ny, nx, c, ch);
        for (int64_t j = 0; j < n; ++j) cube[j] = psi[j] * psi[j] * psi[j];
        orc_rfftn(nz, ny, nx, cube, nph);
        for (int64_t j = 0; j < n; ++j) cube[j] = c[j] * c[j] * c[j];
        orc_rfftn(nz, ny, nx, cube, nch);
        for (int64_t iz = 0; iz < nz; ++iz)
            for (int64_t iy = 0; iy < ny; ++iy)
                for (int64_t ik = 0; ik < nxh; ++ik) {
                    int64_t idx = (iz * ny + iy) * nxh + ik;
                    double k2 = ksq(iz, iy, ik, nz, ny, nx, dx);
                    double m11 = 1.0 + dt * k2 * orc_lin_op(kind_p, r_p, R1_p, q2_p, k2);
                    double m22 = 1.0 + dt * k2 * orc_lin_op(kind_c, r_c, R1_c, q2_c, k2);
                    double m12 = dt * k2 * alpha;
                    cplx b1 = ph[idx] - dt * k2 * nph[idx];
                    cplx b2 = ch[idx] - dt * k2 * nch[idx];
                    double det = m11 * m22 - m12 * m12;
                    ph[idx] = (m22 * b1 - m12 * b2) / det;
                    ch[idx] = (m11 * b2 - m12 * b1) / det;
                }
        orc_irfftn(nz, ny, nx, ph, psi);
        orc_irfftn(nz, ny, nx, ch, c);
    }
    free(ph); free(nph); free(ch); free(nch); free(cube);
}

/* Energy density of the coupled pair: mean of psi Lk_psi psi/2 + psi^4/4 + c Lk_c c/2 + c^4/4
 * + alpha psi c (the free energy whose variational derivatives are mu_psi and mu_c above). */
double orc_energy2(int64_t nz, int64_t ny, int64_t nx, double dx,
                   int kind_p, double r_p, double R1_p, double q2_p,
                   int kind_c, double r_c, double R1_c, double q2_c, double alpha,
                   const double *psi, const double *c)
{
    int64_t n = nz * ny * nx;
    double *lp = malloc(sizeof(double) * n), *lc = malloc(sizeof(double) * n);
    apply_lin(nz, ny, nx, dx, kind_p, r_p, R1_p, q2_p, psi, lp);
    apply_lin(nz, ny, nx, dx, kind_c, r_c, R1_c, q2_c, c, lc);
    double f = 0;
    for (int64_t j = 0; j < n; ++j) {
        double p2 = psi[j] * psi[j], c2 = c[j] * c[j];
        f += 0.5 * psi[j] * lp[j] + 0.25 * p2 * p2 + 0.5 * c[j] * lc[j] + 0.25 * c2 * c2
             + alpha * psi[j] * c[j];
    }
    free(lp); free(lc);
    return f / (double)n;
}

/* ------------------------------------------------------------------------------------ */
/* Tangent-linear and adjoint of one step                                                 */
/* ------------------------------------------------------------------------------------ */
/* One step is psi' = A psi - B (psi^3) with A = IFFT a(k) FFT, B = IFFT b(k) FFT,
 * a = 1/D, b = dt k^2 / D, D = 1 + dt k^2 Lk(k).  Both A and B are real and symmetric
 * (a, b are real and even in k), so for J = A - B diag(3 psi^2):
 *   tangent: dpsi' = A dpsi - B (3 psi^2 dpsi)
 *   adjoint: lam   = A lam' - 3 psi^2 (B lam')
 * and, with dD/dr = dt k^2,  d psi'/dr = IFFT( -(dt k^2 / D) psi_hat' ). */

/* mode 0: out = IFFT(a * FFT(x)); mode 1: out = IFFT(b * FFT(x)); mode 2: out = IFFT(-b * FFT(x)) */
static void apply_mult(int64_t nz, int64_t ny, int64_t nx, double dx, double dt, int kind, double r,
                       double R1, double q2, int mode, const double *x, double *out)
{
    int64_t nxh = nx / 2 + 1, h = nz * ny * nxh;
    cplx *xh = malloc(sizeof(cplx) * h);
    orc_rfftn(nz, ny, nx, x, xh);
    for (int64_t iz = 0; iz < nz; ++iz)
        for (int64_t iy = 0; iy < ny; ++iy)
            for (int64_t ik = 0; ik < nxh; ++ik) {
                int64_t idx = (iz * ny + iy) * nxh + ik;
                double k2 = ksq(iz, iy, ik, nz, ny, nx, dx);
                double d = 1.0 + dt * k2 * orc_lin_op(kind, r, R1, q2, k2);
                double m = mode == 0 ? 1.0 / d : (mode == 1 ? dt * k2 / d : -dt * k2 / d);
                xh[idx] *= m;
            }
    orc_irfftn(nz, ny, nx, xh, out);
    free(xh);
}

/* Tangent-linear step: dpsi_out = A dpsi - B (3 psi_n^2 dpsi). */
void orc_step_tangent(int64_t nz, int64_t ny, int64_t nx, double dx, double dt, int kind, double r,
                      double R1, double q2, const double *psi_n, const double *dpsi, double *dpsi_out)
{
    int64_t n = nz * ny * nx;
    double *q = malloc(sizeof(double) * n), *u = malloc(sizeof(double) * n);
    for (int64_t j = 0; j < n; ++j) q[j] = 3.0 * psi_n[j] * psi_n[j] * dpsi[j];
    apply_mult(nz, ny, nx, dx, dt, kind, r, R1, q2, 0, dpsi, u);
    apply_mult(nz, ny, nx, dx, dt, kind, r, R1, q2, 1, q, dpsi_out);
    for (int64_t j = 0; j < n; ++j) dpsi_out[j] = u[j] - dpsi_out[j];
    free(q); free(u);
}

/* Adjoint step: lam_out = A lam_next - 3 psi_n^2 (B lam_next);
 * *dr += < lam_next, d psi_{n+1}/dr > with psi_{n+1} the forward step of psi_n. */
void orc_step_adjoint(int64_t nz, int64_t ny, int64_t nx, double dx, double dt, int kind, double r,
                      double R1, double q2, const double *psi_n, const double *lam_next,
                      double *lam_out, double *dr)
{
    int64_t n = nz * ny * nx;
    double *next = malloc(sizeof(double) * n), *g = malloc(sizeof(double) * n);
    double *u = malloc(sizeof(double) * n), *v = malloc(sizeof(double) * n);
    memcpy(next, psi_n, sizeof(double) * n);
    orc_step(nz, ny, nx, dx, dt, kind, r, R1, q2, next, 1);
    apply_mult(nz, ny, nx, dx, dt, kind, r, R1, q2, 2, next, g);
    double acc = 0;
    for (int64_t j = 0; j < n; ++j) acc += lam_next[j] * g[j];
    *dr += acc;
    apply_mult(nz, ny, nx, dx, dt, kind, r, R1, q2, 0, lam_next, u);
    apply_mult(nz, ny, nx, dx, dt, kind, r, R1, q2, 1, lam_next, v);
    for (int64_t j = 0; j < n; ++j) lam_out[j] = u[j] - 3.0 * psi_n[j] * psi_n[j] * v[j];
    free(next); free(g); free(u); free(v);
}

/* Loss 0.5 ||psi_T - target||^2 after nsteps from psi0, and its gradients with respect to
 * psi0 and r by the adjoint recursion over the stored trajectory (no checkpointing). */
double orc_adjoint_run(int64_t nz, int64_t ny, int64_t nx, double dx, double dt, int kind, double r,
                       double R1, double q2, const double *psi0, int64_t nsteps,
                       const double *target, double *grad_psi0, double *grad_r)
{
    int64_t n = nz * ny * nx;
    double *traj = malloc(sizeof(double) * n * (nsteps + 1));
    memcpy(traj, psi0, sizeof(double) * n);
    for (int64_t s = 0; s < nsteps; ++s) {
        memcpy(traj + (s + 1) * n, traj + s * n, sizeof(double) * n);
        orc_step(nz, ny, nx, dx, dt, kind, r, R1, q2, traj + (s + 1) * n, 1);
    }
    double loss = 0;
    double *lam = malloc(sizeof(double) * n), *lam2 = malloc(sizeof(double) * n);
    for (int64_t j = 0; j < n; ++j) {
        double d = traj[nsteps * n + j] - target[j];
        loss += 0.5 * d * d;
        lam[j] = d;
    }
    double dr = 0;
    for (int64_t s = nsteps - 1; s >= 0; --s) {
        orc_step_adjoint(nz, ny, nx, dx, dt, kind, r, R1, q2, traj + s * n, lam, lam2, &dr);
        double *t = lam; lam = lam2; lam2 = t;
    }
    memcpy(grad_psi0, lam, sizeof(double) * n);
    *grad_r = dr;
    free(traj); free(lam); free(lam2);
    return loss;
}
