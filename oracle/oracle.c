/*
 * oracle.c -- FP64 CPU oracle for the 3-D discrete Fourier transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls this file;
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (AccFFT, Section 2, first paragraphs): the 3-D DFT of an
 * N0 x N1 x N2 array, which the paper describes as a dense matrix-vector
 * product that Cooley-Tukey reduces to O(N log N) work.  Written out:
 *
 *   forward  X[k0,k1,k2] = sum_j x[j0,j1,j2] * exp(-2 pi i (j0k0/N0 + j1k1/N1 + j2k2/N2))
 *   backward x[j]        = (1/N) sum_k X[k] * exp(+2 pi i (...))
 *
 * The sign convention is not printed in the paper; the one above is the one of
 * the libraries it builds on (FFTW, cuFFT).  The 1/N on the backward transform
 * follows footnote 2 of Section 2 ("full normalization" on the inverse).
 *
 * The 3-D transform is applied axis by axis in the order of Algorithm 1
 * (left column): contiguous axis N2 first, then N1, then N0; the backward
 * transform runs N0, N1, N2 (Algorithm 1, right column).  The DFT is
 * separable, so this equals the dense definition exactly up to rounding.
 *
 * Two independent 1-D engines:
 *   method 0 "naive": the O(n^2) sum of the definition, with the phase index
 *            (j*k) mod n taken in 64-bit integers and the unit roots and the
 *            accumulation in long double.
 *   method 1 "fft":   recursive mixed-radix decimation-in-time Cooley-Tukey
 *            (radices 2, 3, 5; any other prime factor falls back to the naive
 *            sum), in double, with unit roots from the same long-double table.
 *
 * Complex data is interleaved (re, im) real_t (double unless built with
 * -DORC_REAL=float), row-major [n0][n1][n2] with n2
 * contiguous.  Half-spectrum (r2c) arrays are [n0][n1][n2/2+1].
 *
 * Pins (tests/test_oracle_pins.py): impulse, shift theorem, plane waves, real
 * cosines, Parseval, linearity, round trip, Hermitian symmetry, exact integer
 * results for n in {1,2,4} (DFT matrices with entries in {1,-1,i,-i}),
 * brute-force agreement of the two engines, and numpy.fft as a third opinion.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The arithmetic type: double (the oracle).  The same source compiled with
 * -DORC_REAL=float is the FP32 build that the benchmark times as the CPU
 * baseline of FP32 transforms; it is never used as a parity reference. */
#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real_t;
typedef struct { real_t re, im; } cplx;

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NOMEM 2

static const long double ORC_TWO_PI = 6.283185307179586476925286766559005768L;

/* Unit roots w[m] = exp(sign * 2 pi i m / n), m = 0..n-1, long double argument. */
static void unit_roots_ld(int64_t n, int sign, long double *wr, long double *wi)
{
    for (int64_t m = 0; m < n; ++m) {
        long double a = ORC_TWO_PI * (long double)m / (long double)n;
        wr[m] = cosl(a);
        wi[m] = (long double)sign * sinl(a);
    }
}

/* ---------------------------------------------------------------- naive --- */

/* One line of the O(n^2) DFT: X[k] = sum_j x[j] w^(j k mod n). */
static void dft_line_naive(const cplx *x, cplx *X, int64_t n,
                           const long double *wr, const long double *wi)
{
    for (int64_t k = 0; k < n; ++k) {
        long double sr = 0.0L, si = 0.0L;
        for (int64_t j = 0; j < n; ++j) {
            int64_t m = (int64_t)(((__int128)j * k) % n);
            long double xr = x[j].re, xi = x[j].im;
            sr += xr * wr[m] - xi * wi[m];
            si += xr * wi[m] + xi * wr[m];
        }
        X[k].re = (real_t)sr;
        X[k].im = (real_t)si;
    }
}

/* ------------------------------------------------------------------ fft --- */

static int64_t smallest_factor(int64_t n)
{
    if (n % 2 == 0) return 2;
    if (n % 3 == 0) return 3;
    if (n % 5 == 0) return 5;
    return n; /* no small factor: the whole length is treated as one prime */
}

/*
 * Decimation-in-time Cooley-Tukey, written from the textbook identity
 *   n = p m,  X[k + m s] = sum_{q<p} W_n^{q (k + m s)} Y_q[k],
 *   Y_q = DFT_m of the subsequence x[q], x[q+p], x[q+2p], ...
 * for k < m, s < p.  W_n^e is looked up as wroot[(e mod n) * (ntab / n)] in
 * the table of ntab-th roots (n divides ntab).
 *
 * x is read with stride `stride`; X receives n contiguous outputs.
 */
static void fft_rec(const cplx *x, int64_t stride, cplx *X, int64_t n,
                    const cplx *wroot, int64_t ntab)
{
    if (n == 1) { X[0] = x[0]; return; }
    int64_t p = smallest_factor(n);
    int64_t m = n / p;
    int64_t step = ntab / n;
    if (p == n) {
        /* prime length without a small factor: the definition itself */
        for (int64_t k = 0; k < n; ++k) {
            real_t sr = 0.0, si = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                const cplx w = wroot[((j * k) % n) * step];
                const cplx v = x[j * stride];
                sr += v.re * w.re - v.im * w.im;
                si += v.re * w.im + v.im * w.re;
            }
            X[k].re = sr; X[k].im = si;
        }
        return;
    }
    /* sub-transforms Y_q land in X[q*m .. q*m+m-1] */
    for (int64_t q = 0; q < p; ++q)
        fft_rec(x + q * stride, stride * p, X + q * m, m, wroot, ntab);
    /* combine: the p outputs {k + m s} occupy the same slots as {q m + k} */
    cplx t[5], y[5];
    for (int64_t k = 0; k < m; ++k) {
        for (int64_t q = 0; q < p; ++q) t[q] = X[q * m + k];
        for (int64_t s = 0; s < p; ++s) {
            real_t sr = 0.0, si = 0.0;
            for (int64_t q = 0; q < p; ++q) {
                int64_t e = (q * (k + m * s)) % n;
                const cplx w = wroot[e * step];
                sr += t[q].re * w.re - t[q].im * w.im;
                si += t[q].re * w.im + t[q].im * w.re;
            }
            y[s].re = sr; y[s].im = si;
        }
        for (int64_t s = 0; s < p; ++s) X[k + m * s] = y[s];
    }
}

/* --------------------------------------------------------- axis driver --- */

/*
 * Transform every line along one axis of a complex array viewed as
 * [outer][n][inner] (the axis has length n and element stride `inner`).
 * sign = -1 forward, +1 backward (unscaled).  method 0 naive, 1 fft.
 */
int orc_dft_axis(real_t *data, int64_t outer, int64_t n, int64_t inner,
                 int sign, int method, int nthreads)
{
    if (!data || outer < 0 || n < 1 || inner < 0 || (sign != 1 && sign != -1) ||
        (method != 0 && method != 1))
        return ORC_ERR_ARG;
    if (outer == 0 || inner == 0) return ORC_OK;
    cplx *a = (cplx *)data;

    long double *wr = (long double *)malloc(sizeof(long double) * (size_t)n);
    long double *wi = (long double *)malloc(sizeof(long double) * (size_t)n);
    cplx *wd = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!wr || !wi || !wd) { free(wr); free(wi); free(wd); return ORC_ERR_NOMEM; }
    unit_roots_ld(n, sign, wr, wi);
    for (int64_t m = 0; m < n; ++m) { wd[m].re = (real_t)wr[m]; wd[m].im = (real_t)wi[m]; }

    const int64_t lines = outer * inner;
    int status = ORC_OK;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
#endif
    {
        cplx *in = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        if (!in || !out) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            status = ORC_ERR_NOMEM;
        }
        /* every thread reaches the worksharing loop, even without buffers */
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t l = 0; l < lines; ++l) {
            if (!in || !out) continue;
            const int64_t o = l / inner, i = l % inner;
            cplx *base = a + o * n * inner + i;
            for (int64_t j = 0; j < n; ++j) in[j] = base[j * inner];
            if (method == 0) dft_line_naive(in, out, n, wr, wi);
            else fft_rec(in, 1, out, n, wd, n);
            for (int64_t j = 0; j < n; ++j) base[j * inner] = out[j];
        }
        free(in); free(out);
    }
    free(wr); free(wi); free(wd);
    return status;
}

static int bad_dims(int64_t n0, int64_t n1, int64_t n2)
{
    return n0 < 1 || n1 < 1 || n2 < 1;
}

/*
 * 3-D c2c.  direction -1: forward, unscaled, axes 2,1,0 (Algorithm 1 left).
 * direction +1: backward, axes 0,1,2 (Algorithm 1 right), then x 1/N
 * (Section 2, footnote 2).  in and out may alias.
 */
int orc_c2c_3d(const real_t *in, real_t *out, int64_t n0, int64_t n1, int64_t n2,
               int direction, int method, int nthreads)
{
    if (!in || !out || bad_dims(n0, n1, n2) || (direction != 1 && direction != -1))
        return ORC_ERR_ARG;
    const int64_t N = n0 * n1 * n2;
    if (in != out) memmove(out, in, sizeof(cplx) * (size_t)N);
    int s;
    if (direction < 0) {
        if ((s = orc_dft_axis(out, n0 * n1, n2, 1, -1, method, nthreads))) return s;
        if ((s = orc_dft_axis(out, n0, n1, n2, -1, method, nthreads))) return s;
        if ((s = orc_dft_axis(out, 1, n0, n1 * n2, -1, method, nthreads))) return s;
    } else {
        if ((s = orc_dft_axis(out, 1, n0, n1 * n2, 1, method, nthreads))) return s;
        if ((s = orc_dft_axis(out, n0, n1, n2, 1, method, nthreads))) return s;
        if ((s = orc_dft_axis(out, n0 * n1, n2, 1, 1, method, nthreads))) return s;
        const real_t inv = 1.0 / (real_t)N;
        for (int64_t i = 0; i < 2 * N; ++i) out[i] *= inv;
    }
    return ORC_OK;
}

/*
 * r2c forward (AccFFT R2C, Section 1 feature list): the c2c forward transform
 * of the real input, keeping k2 = 0 .. floor(n2/2).  Computed as the axis-2
 * DFT of the real lines promoted to complex, the half kept, then axes 1 and 0
 * on the half array -- the same numbers as slicing the full 3-D spectrum,
 * since the transforms along axes 0 and 1 act on each k2 column separately.
 * in: n0*n1*n2 doubles.  out: n0*n1*(n2/2+1) interleaved complex.
 */
int orc_r2c_3d(const real_t *in, real_t *out, int64_t n0, int64_t n1, int64_t n2,
               int method, int nthreads)
{
    if (!in || !out || bad_dims(n0, n1, n2)) return ORC_ERR_ARG;
    const int64_t nh = n2 / 2 + 1;
    cplx *full = (cplx *)malloc(sizeof(cplx) * (size_t)(n0 * n1 * n2));
    if (!full) return ORC_ERR_NOMEM;
    for (int64_t i = 0; i < n0 * n1 * n2; ++i) { full[i].re = in[i]; full[i].im = 0.0; }
    int s = orc_dft_axis((real_t *)full, n0 * n1, n2, 1, -1, method, nthreads);
    if (s) { free(full); return s; }
    cplx *h = (cplx *)out;
    for (int64_t l = 0; l < n0 * n1; ++l)
        for (int64_t k = 0; k < nh; ++k) h[l * nh + k] = full[l * n2 + k];
    free(full);
    if ((s = orc_dft_axis(out, n0, n1, nh, -1, method, nthreads))) return s;
    return orc_dft_axis(out, 1, n0, n1 * nh, -1, method, nthreads);
}

/*
 * c2r backward: the inverse of r2c on Hermitian-consistent input.  Axes 0 and
 * 1 are inverted on a copy of the half array, then each axis-2 line is
 * extended to length n2 by Hermitian symmetry, Y[n2-k] = conj(Y[k]), with
 * the imaginary parts of bin 0 and (even n2) bin n2/2 dropped, inverted, and
 * its real part kept; finally x 1/N.  `in` is not modified.
 * in: n0*n1*(n2/2+1) interleaved complex.  out: n0*n1*n2 doubles.
 */
int orc_c2r_3d(const real_t *in, real_t *out, int64_t n0, int64_t n1, int64_t n2,
               int method, int nthreads)
{
    if (!in || !out || bad_dims(n0, n1, n2)) return ORC_ERR_ARG;
    const int64_t nh = n2 / 2 + 1;
    const int64_t lines = n0 * n1;
    cplx *h = (cplx *)malloc(sizeof(cplx) * (size_t)(lines * nh));
    cplx *full = (cplx *)malloc(sizeof(cplx) * (size_t)(lines * n2));
    if (!h || !full) { free(h); free(full); return ORC_ERR_NOMEM; }
    memcpy(h, in, sizeof(cplx) * (size_t)(lines * nh));
    int s;
    if ((s = orc_dft_axis((real_t *)h, 1, n0, n1 * nh, 1, method, nthreads)) ||
        (s = orc_dft_axis((real_t *)h, n0, n1, nh, 1, method, nthreads))) {
        free(h); free(full); return s;
    }
    for (int64_t l = 0; l < lines; ++l) {
        const cplx *src = h + l * nh;
        cplx *dst = full + l * n2;
        dst[0].re = src[0].re; dst[0].im = 0.0;
        for (int64_t k = 1; k < n2; ++k) {
            if (2 * k < n2) {
                dst[k] = src[k];
            } else if (2 * k == n2) {
                dst[k].re = src[k].re; dst[k].im = 0.0;
            } else {
                dst[k].re = src[n2 - k].re; dst[k].im = -src[n2 - k].im;
            }
        }
    }
    free(h);
    s = orc_dft_axis((real_t *)full, lines, n2, 1, 1, method, nthreads);
    if (s) { free(full); return s; }
    const real_t inv = 1.0 / (real_t)(n0 * n1 * n2);
    for (int64_t i = 0; i < lines * n2; ++i) out[i] = full[i].re * inv;
    free(full);
    return ORC_OK;
}

/*
 * Selected bins of the forward 3-D DFT straight from the definition, for
 * arrays too large to transform whole on the CPU:
 *   X[k] = sum_{j0} w0^{j0 k0} sum_{j1} w1^{j1 k1} sum_{j2} w2^{j2 k2} x[j0,j1,j2]
 * (the same sum, grouped by axis; each unit root is looked up by its exact
 * integer phase (j k) mod n).  in: complex (is_real = 0) or real (is_real = 1)
 * [n0][n1][n2]; ks: nk triples (k0, k1, k2) with 0 <= ki < ni; out: nk complex.
 */
int orc_dft_bins(const real_t *in, int is_real, int64_t n0, int64_t n1, int64_t n2,
                 const int64_t *ks, int64_t nk, real_t *out, int nthreads)
{
    if (!in || !ks || !out || bad_dims(n0, n1, n2) || nk < 0) return ORC_ERR_ARG;
    for (int64_t b = 0; b < nk; ++b)
        if (ks[3 * b] < 0 || ks[3 * b] >= n0 || ks[3 * b + 1] < 0 || ks[3 * b + 1] >= n1 ||
            ks[3 * b + 2] < 0 || ks[3 * b + 2] >= n2)
            return ORC_ERR_ARG;
    for (int64_t b = 0; b < nk; ++b) {
        const int64_t k0 = ks[3 * b], k1 = ks[3 * b + 1], k2 = ks[3 * b + 2];
        cplx *w0 = (cplx *)malloc(sizeof(cplx) * (size_t)n0);
        cplx *w1 = (cplx *)malloc(sizeof(cplx) * (size_t)n1);
        cplx *w2 = (cplx *)malloc(sizeof(cplx) * (size_t)n2);
        if (!w0 || !w1 || !w2) { free(w0); free(w1); free(w2); return ORC_ERR_NOMEM; }
        for (int64_t j = 0; j < n0; ++j) {
            long double a = ORC_TWO_PI * (long double)((j * k0) % n0) / (long double)n0;
            w0[j].re = (real_t)cosl(a); w0[j].im = -(real_t)sinl(a);
        }
        for (int64_t j = 0; j < n1; ++j) {
            long double a = ORC_TWO_PI * (long double)((j * k1) % n1) / (long double)n1;
            w1[j].re = (real_t)cosl(a); w1[j].im = -(real_t)sinl(a);
        }
        for (int64_t j = 0; j < n2; ++j) {
            long double a = ORC_TWO_PI * (long double)((j * k2) % n2) / (long double)n2;
            w2[j].re = (real_t)cosl(a); w2[j].im = -(real_t)sinl(a);
        }
        real_t sr = 0.0, si = 0.0;
#ifdef _OPENMP
        if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) reduction(+ : sr, si) schedule(static)
#endif
        for (int64_t j0 = 0; j0 < n0; ++j0) {
            real_t ar = 0.0, ai = 0.0;
            for (int64_t j1 = 0; j1 < n1; ++j1) {
                real_t br = 0.0, bi = 0.0;
                const int64_t base = (j0 * n1 + j1) * n2;
                if (is_real) {
                    const real_t *x = in + base;
                    for (int64_t j2 = 0; j2 < n2; ++j2) {
                        br += x[j2] * w2[j2].re;
                        bi += x[j2] * w2[j2].im;
                    }
                } else {
                    const cplx *x = (const cplx *)in + base;
                    for (int64_t j2 = 0; j2 < n2; ++j2) {
                        br += x[j2].re * w2[j2].re - x[j2].im * w2[j2].im;
                        bi += x[j2].re * w2[j2].im + x[j2].im * w2[j2].re;
                    }
                }
                ar += br * w1[j1].re - bi * w1[j1].im;
                ai += br * w1[j1].im + bi * w1[j1].re;
            }
            sr += ar * w0[j0].re - ai * w0[j0].im;
            si += ar * w0[j0].im + ai * w0[j0].re;
        }
        out[2 * b] = sr;
        out[2 * b + 1] = si;
        free(w0); free(w1); free(w2);
    }
    return ORC_OK;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
