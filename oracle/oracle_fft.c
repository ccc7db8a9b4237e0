/*
 * oracle_fft.c -- plain, slow, obviously-correct FP64 CPU discrete Fourier
 * transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA path against an
 * independent computation.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What is computed (the paper, Sec. 3.3 / Sec. 5.1(a): the "Fourier transform"
 * function block of a C application that is swapped for a device library; the
 * paper prints no formula, so the textbook definition of the complex DFT is
 * used):
 *
 *     X[k] = c * sum_{n=0}^{N-1} x[n] * exp(s * 2*pi*i * n*k / N),  k = 0..N-1
 *
 * with exponent sign s in {-1, +1} (s = -1 is called "forward"), c = 1, or
 * c = 1/N when the caller asks for the inverse-scaled form.  A multi-dimensional
 * transform of dims N_0..N_{r-1} (row-major, last index fastest) is the same sum
 * over the multi-index with phase sum_d n_d*k_d/N_d, i.e. 1-D transforms along
 * every axis (separability); c = 1/prod(N_d) when scaled.  Batches are
 * independent transforms stored one after another.
 *
 * Two routines compute the 1-D sum:
 *   oracle_dft_naive  -- the definition written out, O(N^2), long double
 *                        accumulation; used on tiny sizes to pin the other.
 *   oracle_fft_1d     -- textbook recursive decimation-in-time Cooley-Tukey:
 *                        N = p*M with p the smallest prime factor of N,
 *                        Y_q = DFT_M of the stride-p subsequence starting at q,
 *                        X[k] = sum_q exp(s*2*pi*i*q*k/N) * Y_q[k mod M];
 *                        a prime length is summed directly.
 * Twiddles exp(s*2*pi*i*m/D) use exact integer reduction of m modulo D and
 * long double cos/sin, rounded once to double.
 *
 * Complex data is interleaved (re, im) doubles.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double re, im;
} cplx;

static const long double TWO_PI_L = 6.283185307179586476925286766559005768394L;

/* exp(s * 2*pi*i * m / D) with the integer m reduced modulo D first. */
static cplx twiddle(long long m, long long D, int sign)
{
    long long r = m % D;
    if (r < 0) r += D;
    long double ang = TWO_PI_L * (long double)r / (long double)D;
    cplx w;
    w.re = (double)cosl(ang);
    w.im = (double)((long double)sign * sinl(ang));
    return w;
}

static long long smallest_prime_factor(long long n)
{
    if (n % 2 == 0) return 2;
    for (long long p = 3; p * p <= n; p += 2)
        if (n % p == 0) return p;
    return n;
}

/* ------------------------------------------------------------------------ */
/* Naive O(N^2) DFT: the definition, accumulated in long double.            */
/* ------------------------------------------------------------------------ */
int oracle_dft_naive(const double* in, double* out, long long n, int sign)
{
    if (n <= 0 || (sign != 1 && sign != -1) || !in || !out) return -1;
    for (long long k = 0; k < n; ++k) {
        long double sr = 0.0L, si = 0.0L;
        for (long long j = 0; j < n; ++j) {
            long long m = (j % n) * (k % n) % n;
            long double ang = TWO_PI_L * (long double)m / (long double)n;
            long double c = cosl(ang);
            long double s = (long double)sign * sinl(ang);
            long double xr = in[2 * j], xi = in[2 * j + 1];
            sr += xr * c - xi * s;
            si += xr * s + xi * c;
        }
        out[2 * k] = (double)sr;
        out[2 * k + 1] = (double)si;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Recursive mixed-radix Cooley-Tukey (decimation in time).                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    const cplx* tab; /* tab[m] = exp(sign*2*pi*i*m/Ntop), m in [0, Ntop) */
    long long Ntop;
} ct_ctx;

/* x: input with element stride `stride`; X: N contiguous outputs;
 * work: scratch of at least N elements (only used after the sub-calls). */
static void ct_rec(const ct_ctx* c, const cplx* x, long long stride, cplx* X,
                   long long N, cplx* work)
{
    if (N == 1) {
        X[0] = x[0];
        return;
    }
    const long long p = smallest_prime_factor(N);
    const long long tstep = c->Ntop / N; /* w_N^m = tab[m * tstep] */
    if (p == N) {
        /* prime length: the definition, summed directly */
        for (long long k = 0; k < N; ++k) {
            double ar = 0.0, ai = 0.0;
            for (long long q = 0; q < N; ++q) {
                const cplx w = c->tab[((q * k) % N) * tstep];
                const cplx v = x[q * stride];
                ar += v.re * w.re - v.im * w.im;
                ai += v.re * w.im + v.im * w.re;
            }
            X[k].re = ar;
            X[k].im = ai;
        }
        return;
    }
    const long long M = N / p;
    /* Y_q = DFT_M(x[q], x[q+p], x[q+2p], ...) stored at X[q*M .. q*M+M-1] */
    for (long long q = 0; q < p; ++q)
        ct_rec(c, x + q * stride, stride * p, X + q * M, M, work);
    /* X[k] = sum_q w_N^{q*k} * Y_q[k mod M] */
    for (long long k = 0; k < N; ++k) {
        double ar = 0.0, ai = 0.0;
        const long long km = k % M;
        for (long long q = 0; q < p; ++q) {
            const cplx w = c->tab[((q * k) % N) * tstep];
            const cplx y = X[q * M + km];
            ar += y.re * w.re - y.im * w.im;
            ai += y.re * w.im + y.im * w.re;
        }
        work[k].re = ar;
        work[k].im = ai;
    }
    memcpy(X, work, (size_t)N * sizeof(cplx));
}

static cplx* make_table(long long n, int sign)
{
    cplx* tab = (cplx*)malloc((size_t)n * sizeof(cplx));
    if (!tab) return NULL;
    for (long long m = 0; m < n; ++m) tab[m] = twiddle(m, n, sign);
    return tab;
}

int oracle_fft_1d(const double* in, double* out, long long n, int sign)
{
    if (n <= 0 || (sign != 1 && sign != -1) || !in || !out) return -1;
    cplx* tab = make_table(n, sign);
    cplx* X = (cplx*)malloc((size_t)n * sizeof(cplx));
    cplx* work = (cplx*)malloc((size_t)n * sizeof(cplx));
    if (!tab || !X || !work) {
        free(tab), free(X), free(work);
        return -2;
    }
    ct_ctx c = {tab, n};
    ct_rec(&c, (const cplx*)in, 1, X, n, work);
    memcpy(out, X, (size_t)n * sizeof(cplx));
    free(tab), free(X), free(work);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Multi-dimensional, batched: 1-D transforms along every axis in turn.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    cplx* data;       /* whole batch, transformed in place */
    const cplx* tab;  /* table for this axis length */
    long long L;      /* axis length */
    long long S;      /* element stride along the axis (product of later dims) */
    long long O;      /* product of earlier dims */
    long long N;      /* elements per transform */
    long long lines;  /* batch * O * S */
    long long first, last; /* line range [first, last) for this worker */
    int status;
} axis_job;

static void* axis_worker(void* arg)
{
    axis_job* j = (axis_job*)arg;
    cplx* line = (cplx*)malloc((size_t)j->L * sizeof(cplx));
    cplx* X = (cplx*)malloc((size_t)j->L * sizeof(cplx));
    cplx* work = (cplx*)malloc((size_t)j->L * sizeof(cplx));
    if (!line || !X || !work) {
        j->status = -2;
        free(line), free(X), free(work);
        return NULL;
    }
    ct_ctx c = {j->tab, j->L};
    for (long long ln = j->first; ln < j->last; ++ln) {
        /* line index -> (batch b, outer o, inner s) */
        const long long s = ln % j->S;
        const long long o = (ln / j->S) % j->O;
        const long long b = ln / (j->S * j->O);
        cplx* base = j->data + b * j->N + o * j->L * j->S + s;
        for (long long n = 0; n < j->L; ++n) line[n] = base[n * j->S];
        ct_rec(&c, line, 1, X, j->L, work);
        for (long long n = 0; n < j->L; ++n) base[n * j->S] = X[n];
    }
    free(line), free(X), free(work);
    j->status = 0;
    return NULL;
}

/*
 * in/out: batch * prod(dims) interleaved complex doubles (may alias).
 * scale != 0 multiplies the result by 1/prod(dims).
 * nthreads >= 1 worker threads split the lines of each axis.
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_fft_nd(const double* in, double* out, int rank, const long long* dims,
                  long long batch, int sign, int scale, int nthreads)
{
    if (rank < 1 || rank > 8 || !dims || batch < 0 || !in || !out) return -1;
    if (sign != 1 && sign != -1) return -1;
    if (nthreads < 1) nthreads = 1;
    long long N = 1;
    for (int d = 0; d < rank; ++d) {
        if (dims[d] < 1) return -1;
        N *= dims[d];
    }
    if (batch == 0) return 0;
    cplx* data = (cplx*)out;
    if (out != in) memcpy(out, in, (size_t)(N * batch) * sizeof(cplx));

    for (int d = rank - 1; d >= 0; --d) {
        const long long L = dims[d];
        if (L == 1) continue;
        long long S = 1, O = 1;
        for (int e = d + 1; e < rank; ++e) S *= dims[e];
        for (int e = 0; e < d; ++e) O *= dims[e];
        cplx* tab = make_table(L, sign);
        if (!tab) return -2;
        const long long lines = batch * O * S;
        int nt = nthreads;
        if ((long long)nt > lines) nt = (int)lines;
        axis_job* jobs = (axis_job*)calloc((size_t)nt, sizeof(axis_job));
        pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
        if (!jobs || !th) {
            free(tab), free(jobs), free(th);
            return -2;
        }
        for (int t = 0; t < nt; ++t) {
            jobs[t].data = data;
            jobs[t].tab = tab;
            jobs[t].L = L;
            jobs[t].S = S;
            jobs[t].O = O;
            jobs[t].N = N;
            jobs[t].lines = lines;
            jobs[t].first = lines * t / nt;
            jobs[t].last = lines * (t + 1) / nt;
            jobs[t].status = -3;
        }
        int status = 0;
        if (nt == 1) {
            axis_worker(&jobs[0]);
        } else {
            for (int t = 0; t < nt; ++t)
                if (pthread_create(&th[t], NULL, axis_worker, &jobs[t]) != 0) {
                    axis_worker(&jobs[t]); /* run inline if no thread */
                    th[t] = 0;
                }
            for (int t = 0; t < nt; ++t)
                if (th[t]) pthread_join(th[t], NULL);
        }
        for (int t = 0; t < nt; ++t)
            if (jobs[t].status != 0) status = jobs[t].status;
        free(tab), free(jobs), free(th);
        if (status != 0) return status;
    }
    if (scale) {
        const double inv = 1.0 / (double)N;
        for (long long i = 0; i < N * batch; ++i) {
            data[i].re *= inv;
            data[i].im *= inv;
        }
    }
    return 0;
}

/* Reference twiddle exp(s*2*pi*i*m/D) in double (long double evaluation),
 * exported so tests can check device-built twiddle tables. */
void oracle_twiddle(long long m, long long D, int sign, double* re, double* im)
{
    cplx w = twiddle(m, D, sign);
    *re = w.re;
    *im = w.im;
}
