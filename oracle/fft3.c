/*
 * Plain FP64 discrete Fourier transforms for the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the oracle: the slow,
 * obviously correct CPU statement of what the GPU library computes.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never does.
 *
 * What it computes (JDFTx paper, Sec. 2.1: the operators I and J move a field
 * between reciprocal and real space "using Fast Fourier Transforms"):
 *
 *     y[m] = sum_{t=0}^{n-1} x[t] * exp(sign * 2*pi*i * t*m / n)
 *
 * unnormalised, sign = +1 (reciprocal -> real, operator I) or -1 (real ->
 * reciprocal, operator J before its 1/N factor).  A 3-D transform applies the
 * 1-D transform along each axis of an S0 x S1 x S2 box stored with axis 2
 * fastest (linear index j2 + S2*(j1 + S1*j0)).
 *
 * Three routines, each pinned against the others in tests:
 *   oracle_dft1d   direct O(n^2) sum, the definition itself;
 *   oracle_fft1d   textbook recursive decimation-in-time Cooley-Tukey: split
 *                  by the smallest prime factor p of n into p interleaved
 *                  subsequences, transform each, combine with twiddles;
 *   oracle_dft3d_direct  O(N^2) sum over the whole box (tiny boxes only).
 * The per-axis loops may run on several OpenMP threads; the arithmetic of each
 * line does not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

/* exp(sign * 2 pi i * e / n) with e reduced mod n first, so the angle stays small. */
static cplx root_of_unity(long e, long n, int sign)
{
    long r = e % n;
    if (r < 0) r += n;
    double a = TWO_PI * (double)r / (double)n;
    cplx w = { cos(a), sign * sin(a) };
    return w;
}

void oracle_dft1d(const cplx* x, cplx* y, int n, int sign)
{
    for (int m = 0; m < n; ++m) {
        double sr = 0.0, si = 0.0;
        for (int t = 0; t < n; ++t) {
            cplx w = root_of_unity((long)t * m, n, sign);
            sr += x[t].re * w.re - x[t].im * w.im;
            si += x[t].re * w.im + x[t].im * w.re;
        }
        y[m].re = sr;
        y[m].im = si;
    }
}

static int smallest_prime_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* Recursive step: transform x[0], x[stride], ..., x[(n-1)*stride] into y[0..n-1].
 * work must hold n elements. */
static void fft_rec(const cplx* x, long stride, cplx* y, int n, int sign, cplx* work)
{
    if (n == 1) { y[0] = x[0]; return; }
    int p = smallest_prime_factor(n);
    if (p == n) {                 /* prime length: the definition */
        for (int m = 0; m < n; ++m) {
            double sr = 0.0, si = 0.0;
            for (int t = 0; t < n; ++t) {
                cplx w = root_of_unity((long)t * m, n, sign);
                cplx v = x[(long)t * stride];
                sr += v.re * w.re - v.im * w.im;
                si += v.re * w.im + v.im * w.re;
            }
            y[m].re = sr; y[m].im = si;
        }
        return;
    }
    int m = n / p;
    /* Subsequence r = x[r], x[r+p], ... has length m; its transform Y_r goes
     * to work[r*m .. r*m+m-1]. */
    for (int r = 0; r < p; ++r)
        fft_rec(x + (long)r * stride, stride * p, work + (long)r * m, m, sign, y);
    /* X[k + q*m] = sum_r w_n^{r (k + q m)} Y_r[k]. */
    for (int q = 0; q < p; ++q) {
        for (int k = 0; k < m; ++k) {
            int out = k + q * m;
            double sr = 0.0, si = 0.0;
            for (int r = 0; r < p; ++r) {
                cplx w = root_of_unity((long)r * out, n, sign);
                cplx v = work[(long)r * m + k];
                sr += v.re * w.re - v.im * w.im;
                si += v.re * w.im + v.im * w.re;
            }
            y[out].re = sr; y[out].im = si;
        }
    }
}

void oracle_fft1d(const cplx* x, cplx* y, int n, int sign)
{
    cplx* work = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    fft_rec(x, 1, y, n, sign, work);
    free(work);
}

/* Transform every line of the box along one axis, in place. */
static void fft_axis(cplx* a, int S0, int S1, int S2, int axis, int sign)
{
    int S[3] = { S0, S1, S2 };
    long strideof[3] = { (long)S1 * S2, S2, 1 };
    int n = S[axis];
    long stride = strideof[axis];
    /* Lines are indexed by the two other axes. */
    int oa = (axis == 0) ? 1 : 0, ob = (axis == 2) ? 1 : 2;
    long nlines = (long)S[oa] * S[ob];
    #pragma omp parallel
    {
        cplx* line = (cplx*)malloc(sizeof(cplx) * (size_t)n);
        cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)n);
        cplx* work = (cplx*)malloc(sizeof(cplx) * (size_t)n);
        #pragma omp for schedule(static)
        for (long L = 0; L < nlines; ++L) {
            long ia = L / S[ob], ib = L % S[ob];
            long base = ia * strideof[oa] + ib * strideof[ob];
            for (int t = 0; t < n; ++t) line[t] = a[base + t * stride];
            fft_rec(line, 1, out, n, sign, work);
            for (int t = 0; t < n; ++t) a[base + t * stride] = out[t];
        }
        free(line); free(out); free(work);
    }
}

/* In-place unnormalised 3-D transform of `count` boxes stored back to back. */
void oracle_fft3d(cplx* a, int S0, int S1, int S2, int count, int sign)
{
    long N = (long)S0 * S1 * S2;
    for (int c = 0; c < count; ++c) {
        cplx* box = a + (long)c * N;
        fft_axis(box, S0, S1, S2, 2, sign);
        fft_axis(box, S0, S1, S2, 1, sign);
        fft_axis(box, S0, S1, S2, 0, sign);
    }
}

/* Direct O(N^2) 3-D sum, the definition with no factorisation: for tiny boxes. */
void oracle_dft3d_direct(const cplx* x, cplx* y, int S0, int S1, int S2, int sign)
{
    long N = (long)S0 * S1 * S2;
    #pragma omp parallel for schedule(static)
    for (long m = 0; m < N; ++m) {
        long m0 = m / ((long)S1 * S2), m1 = (m / S2) % S1, m2 = m % S2;
        double sr = 0.0, si = 0.0;
        for (long t = 0; t < N; ++t) {
            long t0 = t / ((long)S1 * S2), t1 = (t / S2) % S1, t2 = t % S2;
            /* phase = (t0 m0 / S0 + t1 m1 / S1 + t2 m2 / S2) turns */
            double turns = (double)((t0 * m0) % S0) / S0 + (double)((t1 * m1) % S1) / S1
                         + (double)((t2 * m2) % S2) / S2;
            double ang = TWO_PI * turns;
            double wr = cos(ang), wi = sign * sin(ang);
            sr += x[t].re * wr - x[t].im * wi;
            si += x[t].re * wi + x[t].im * wr;
        }
        y[m].re = sr; y[m].im = si;
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
