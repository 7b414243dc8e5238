/*
 * evx oracle: plain FP64 CPU routines used ONLY as test infrastructure.
 *
 * This file is test infrastructure. Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg may load it. It shares no code,
 * header, table or helper with the CUDA library; it is written to be read
 * against the mathematics, not to be fast.
 *
 * Contents
 *   orc_fft3d      textbook mixed-radix (recursive Cooley-Tukey, any prime
 *                  factor handled by a direct DFT of that size) complex FFT,
 *                  applied along each axis of a C-order nx*ny*nz array.
 *                  Forward uses exp(-i...), inverse exp(+i...), both
 *                  unnormalised. This is the "F{.}" of the paper's appendix
 *                  (section "Semi-implicit timestepping").
 *   orc_dft_modes  direct O(V) evaluation of sum_x f(c(x)) exp(-i k.x) at a
 *                  list of wave vectors, with f = identity or f(c) = c^3 - c
 *                  (the pointwise chemical-potential term of the
 *                  Cahn-Hilliard right-hand side). Used to check single
 *                  Fourier modes of a large grid one by one.
 *   orc_vm_rhs_modes  the same sums of the variable-mobility finite-
 *                  difference right-hand side, formed plane by plane.
 *
 * Twiddle factors are evaluated with libm cos/sin in FP64.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

/* smallest prime factor of n (n >= 2) */
static int smallest_prime_factor(int n)
{
    for (int p = 2; (long)p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* table w[e] = exp(sign * 2 pi i e / n), e = 0..n-1 */
static cplx *make_roots(int n, int sign)
{
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int e = 0; e < n; ++e) {
        double ang = sign * TWO_PI * (double)e / (double)n;
        w[e] = cos(ang) + I * sin(ang);
    }
    return w;
}

/*
 * Recursive decimation in time.
 *   out[k] = sum_{j<n} in[j*stride] * w_n^{j k},  w_n = exp(sign 2 pi i / n)
 * Split n = p*m with p the smallest prime factor: the p interleaved
 * subsequences in[(p j + r) stride] are transformed (length m) into
 * out[r m .. r m + m), then combined
 *   X[k + m q] = sum_r w_n^{r (k + m q)} Y_r[k].
 * roots holds the N-th roots of unity of the top-level length N; a level of
 * length n uses every (N/n)-th entry.
 */
static void fft_rec(const cplx *in, long stride, cplx *out, int n,
                    const cplx *roots, int N, cplx *tmp)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_prime_factor(n);
    int m = n / p;
    for (int r = 0; r < p; ++r)
        fft_rec(in + r * stride, stride * p, out + (long)r * m, m, roots, N, tmp);
    long step = N / n;
    for (int k = 0; k < m; ++k) {
        for (int r = 0; r < p; ++r) tmp[r] = out[(long)r * m + k];
        for (int q = 0; q < p; ++q) {
            cplx s = 0;
            for (int r = 0; r < p; ++r) {
                long e = ((long)r * (k + (long)m * q)) % n;
                s += tmp[r] * roots[e * step];
            }
            out[(long)q * m + k] = s;
        }
    }
}

/* in-place 1D transform of a contiguous array using a caller-made root table */
static void fft1d_with(cplx *x, int n, const cplx *roots, cplx *buf, cplx *tmp)
{
    memcpy(buf, x, sizeof(cplx) * (size_t)n);
    fft_rec(buf, 1, x, n, roots, n, tmp);
}

/* 1D transform, in place, of n interleaved (re, im) doubles. sign = -1 forward, +1 inverse. */
void orc_fft1d(double *data, int n, int sign)
{
    cplx *x = (cplx *)data;
    cplx *roots = make_roots(n, sign);
    cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    fft1d_with(x, n, roots, buf, tmp);
    free(tmp);
    free(buf);
    free(roots);
}

/*
 * One axis of a C-order nx*ny*nz complex array. axis 0 = x (stride ny*nz),
 * 1 = y (stride nz), 2 = z (stride 1). Pencils are gathered into a contiguous
 * buffer, transformed and scattered back; the loop over pencils is shared
 * among OpenMP threads (each pencil is independent).
 */
static void fft_axis(cplx *a, int nx, int ny, int nz, int axis, int sign)
{
    int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    long stride = axis == 0 ? (long)ny * nz : (axis == 1 ? (long)nz : 1);
    long npencil = (long)nx * ny * nz / n;
    cplx *roots = make_roots(n, sign);
#pragma omp parallel
    {
        cplx *pen = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(static)
        for (long q = 0; q < npencil; ++q) {
            /* base offset of pencil q */
            long base;
            if (axis == 2) {
                base = q * nz;
            } else if (axis == 1) {
                long x = q / nz, z = q % nz;
                base = x * (long)ny * nz + z;
            } else {
                base = q; /* q enumerates (y, z) */
            }
            for (int i = 0; i < n; ++i) pen[i] = a[base + i * stride];
            fft1d_with(pen, n, roots, buf, tmp);
            for (int i = 0; i < n; ++i) a[base + i * stride] = pen[i];
        }
        free(tmp);
        free(buf);
        free(pen);
    }
    free(roots);
}

/* Unnormalised 3D transform in place (interleaved re/im doubles). */
void orc_fft3d(double *data, int nx, int ny, int nz, int sign)
{
    cplx *a = (cplx *)data;
    fft_axis(a, nx, ny, nz, 2, sign);
    fft_axis(a, nx, ny, nz, 1, sign);
    fft_axis(a, nx, ny, nz, 0, sign);
}

/*
 * Direct sums  F_f(k) = sum_{x,y,z} f(c[x,y,z]) exp(-2 pi i (mx x/nx + my y/ny + mz z/nz))
 * for nmodes integer wave vectors (mx, my, mz) given in modes[3*i..3*i+2].
 * which = 0: f(c) = c;  which = 1: f(c) = c^3 - c.
 * The sum is separable: an inner sum over z for each (x, y), then y, then x.
 * Per-x partial sums are stored and added in order, so the result does not
 * depend on the number of threads.
 */
void orc_dft_modes(const float *c, int nx, int ny, int nz, int nmodes,
                   const int *modes, int which, double *out_re, double *out_im)
{
    cplx *ex = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes * nx);
    cplx *ey = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes * ny);
    cplx *ez = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes * nz);
    for (int m = 0; m < nmodes; ++m) {
        for (int x = 0; x < nx; ++x) {
            double ang = -TWO_PI * (double)(((long)modes[3 * m] * x) % nx) / nx;
            ex[(long)m * nx + x] = cos(ang) + I * sin(ang);
        }
        for (int y = 0; y < ny; ++y) {
            double ang = -TWO_PI * (double)(((long)modes[3 * m + 1] * y) % ny) / ny;
            ey[(long)m * ny + y] = cos(ang) + I * sin(ang);
        }
        for (int z = 0; z < nz; ++z) {
            double ang = -TWO_PI * (double)(((long)modes[3 * m + 2] * z) % nz) / nz;
            ez[(long)m * nz + z] = cos(ang) + I * sin(ang);
        }
    }
    cplx *partial = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes * nx);
#pragma omp parallel
    {
        cplx *sz = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes);
        cplx *sy = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes);
#pragma omp for schedule(static)
        for (int x = 0; x < nx; ++x) {
            for (int m = 0; m < nmodes; ++m) sy[m] = 0;
            for (int y = 0; y < ny; ++y) {
                const float *row = c + ((long)x * ny + y) * nz;
                for (int m = 0; m < nmodes; ++m) sz[m] = 0;
                for (int z = 0; z < nz; ++z) {
                    double v = (double)row[z];
                    double f = which ? (v * v * v - v) : v;
                    for (int m = 0; m < nmodes; ++m) sz[m] += f * ez[(long)m * nz + z];
                }
                for (int m = 0; m < nmodes; ++m) sy[m] += sz[m] * ey[(long)m * ny + y];
            }
            for (int m = 0; m < nmodes; ++m) partial[(long)m * nx + x] = sy[m] * ex[(long)m * nx + x];
        }
        free(sy);
        free(sz);
    }
    for (int m = 0; m < nmodes; ++m) {
        cplx s = 0;
        for (int x = 0; x < nx; ++x) s += partial[(long)m * nx + x];
        out_re[m] = creal(s);
        out_im[m] = cimag(s);
    }
    free(partial);
    free(ez);
    free(ey);
    free(ex);
}

/*
 * Variable-mobility right-hand side on one x-plane and its Fourier modes.
 * The general form of "Semi-implicit timestepping" with the mobility of Eq.
 * (cahn-hilliard) read as M(c) = M max(1 - c^2, 0):
 *   mu  = c^3 - c - kappa lap_h c,  lap_h the periodic 7-point Laplacian / h^2,
 *   rhs = (1/h^2) sum_d [ (M_x + M_{x+e_d})/2 (mu_{x+e_d} - mu_x)
 *                         - (M_{x-e_d} + M_x)/2 (mu_x - mu_{x-e_d}) ].
 * orc_vm_rhs_modes returns the direct sums sum_x rhs(x) exp(-i k.x) at the
 * given integer wave vectors. Each x-plane of rhs is formed on its own from
 * the c planes x-2 .. x+2 (mu and M on planes x-1, x, x+1), then summed like
 * orc_dft_modes; per-x partial sums are added in order.
 */
static long wrap(long i, long n) { return ((i % n) + n) % n; }

static void vm_mu_plane(const float *c, int nx, int ny, int nz, long p, double kappa, double h, double *out)
{
    const long x = wrap(p, nx), xm = wrap(p - 1, nx), xp = wrap(p + 1, nx);
    for (long y = 0; y < ny; ++y) {
        const long ym = wrap(y - 1, ny), yp = wrap(y + 1, ny);
        for (long z = 0; z < nz; ++z) {
            const long zm = wrap(z - 1, nz), zp = wrap(z + 1, nz);
            const double v = c[(x * ny + y) * nz + z];
            const double lap = ((double)c[(xp * ny + y) * nz + z] + (double)c[(xm * ny + y) * nz + z]
                                + (double)c[(x * ny + yp) * nz + z] + (double)c[(x * ny + ym) * nz + z]
                                + (double)c[(x * ny + y) * nz + zp] + (double)c[(x * ny + y) * nz + zm]
                                - 6.0 * v) / (h * h);
            out[y * nz + z] = v * v * v - v - kappa * lap;
        }
    }
}

static void vm_mob_plane(const float *c, int nx, int ny, int nz, long p, double M, double *out)
{
    const long x = wrap(p, nx);
    for (long i = 0; i < (long)ny * nz; ++i) {
        const double v = c[x * ny * nz + i];
        const double m = 1.0 - v * v;
        out[i] = M * (m > 0.0 ? m : 0.0);
    }
}

void orc_vm_rhs_modes(const float *c, int nx, int ny, int nz, double M, double kappa, double h,
                      int nmodes, const int *modes, double *out_re, double *out_im)
{
    cplx *ex = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes * nx);
    cplx *ey = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes * ny);
    cplx *ez = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes * nz);
    for (int m = 0; m < nmodes; ++m) {
        for (int x = 0; x < nx; ++x)
            ex[(long)m * nx + x] = cexp(-I * TWO_PI * (double)(((long)modes[3 * m] * x) % nx) / nx);
        for (int y = 0; y < ny; ++y)
            ey[(long)m * ny + y] = cexp(-I * TWO_PI * (double)(((long)modes[3 * m + 1] * y) % ny) / ny);
        for (int z = 0; z < nz; ++z)
            ez[(long)m * nz + z] = cexp(-I * TWO_PI * (double)(((long)modes[3 * m + 2] * z) % nz) / nz);
    }
    cplx *partial = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes * nx);
    const long P = (long)ny * nz;
#pragma omp parallel
    {
        double *mu = (double *)malloc(sizeof(double) * 3 * P);   /* planes x-1, x, x+1 */
        double *mob = (double *)malloc(sizeof(double) * 3 * P);
        double *rhs = (double *)malloc(sizeof(double) * P);
        cplx *sz = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes);
        cplx *sy = (cplx *)malloc(sizeof(cplx) * (size_t)nmodes);
#pragma omp for schedule(static)
        for (int x = 0; x < nx; ++x) {
            for (int j = 0; j < 3; ++j) {
                vm_mu_plane(c, nx, ny, nz, x - 1 + j, kappa, h, mu + j * P);
                vm_mob_plane(c, nx, ny, nz, x - 1 + j, M, mob + j * P);
            }
            const double *u0 = mu + P, *m0 = mob + P;
            for (long y = 0; y < ny; ++y) {
                const long ym = wrap(y - 1, ny), yp = wrap(y + 1, ny);
                for (long z = 0; z < nz; ++z) {
                    const long zm = wrap(z - 1, nz), zp = wrap(z + 1, nz);
                    const long i = y * nz + z;
                    /* neighbour indices within the three planes: -x, +x, -y, +y, -z, +z */
                    const double un[6] = {mu[i], mu[2 * P + i], u0[ym * nz + z], u0[yp * nz + z], u0[y * nz + zm],
                                          u0[y * nz + zp]};
                    const double mn[6] = {mob[i], mob[2 * P + i], m0[ym * nz + z], m0[yp * nz + z], m0[y * nz + zm],
                                          m0[y * nz + zp]};
                    double acc = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        const double fp = 0.5 * (m0[i] + mn[2 * d + 1]) * (un[2 * d + 1] - u0[i]);
                        const double fm = 0.5 * (mn[2 * d] + m0[i]) * (u0[i] - un[2 * d]);
                        acc += fp - fm;
                    }
                    rhs[i] = acc / (h * h);
                }
            }
            for (int m = 0; m < nmodes; ++m) sy[m] = 0;
            for (long y = 0; y < ny; ++y) {
                for (int m = 0; m < nmodes; ++m) sz[m] = 0;
                for (long z = 0; z < nz; ++z) {
                    const double f = rhs[y * nz + z];
                    for (int m = 0; m < nmodes; ++m) sz[m] += f * ez[(long)m * nz + z];
                }
                for (int m = 0; m < nmodes; ++m) sy[m] += sz[m] * ey[(long)m * ny + y];
            }
            for (int m = 0; m < nmodes; ++m) partial[(long)m * nx + x] = sy[m] * ex[(long)m * nx + x];
        }
        free(sy);
        free(sz);
        free(rhs);
        free(mob);
        free(mu);
    }
    for (int m = 0; m < nmodes; ++m) {
        cplx s = 0;
        for (int x = 0; x < nx; ++x) s += partial[(long)m * nx + x];
        out_re[m] = creal(s);
        out_im[m] = cimag(s);
    }
    free(partial);
    free(ez);
    free(ey);
    free(ex);
}

/* Number of OpenMP threads the routines above will use (for reporting). */
int orc_num_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
