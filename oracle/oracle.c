/*
 * oracle.c -- plain CPU reference for the PACO hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or table with the CUDA path.
 *
 * What PACO computes is, exactly up to rounding order, the canonical DFT of
 * Sect. 2 of the paper ("Model and Main Result"):
 *
 *     y = Omega_N x,   (Omega_N)_{k,j} = w_N^{-kj},   w_N = exp(2*pi*i/N),
 *
 * and Theorem 3 (end-to-end correctness) states that the factor-swapped
 * output view Y[k2,k1] equals y[k1 + k2*N1].  The oracle is therefore that
 * definition written out, evaluated three independent ways:
 *
 *   oracle_dft_direct  O(n^2) sum in long double over exact residues
 *                      r = (k*j) mod n (Sect. 2 definition, verbatim);
 *   oracle_fft         textbook recursive radix-2 decimation-in-time FFT in
 *                      FP64 (even/odd split), twiddles w_N^{dir*r} from exact
 *                      integer residues, evaluated in long double;
 *   oracle_dft_at      the definition at selected output indices only, in
 *                      FP64 with exact residues and pairwise summation, for
 *                      sizes too large for the direct sum.
 *
 * `dir` selects the exponent sign: dir = -1 is the paper's forward transform
 * (w^{-kj}); dir = +1 is the unnormalised conjugate transform (w^{+kj}), which
 * the paper does not define (it is the adjoint, used for the inverse and for
 * the gradient).
 *
 * oracle_digit_reverse is the base-b digit reversal pi_ell of Sect. 3.2 /
 * App. A.1, computed from an explicit digit array (most significant digit
 * first), with no bit tricks.
 *
 * Complex data are interleaved (re, im) doubles.  Every function returns 0 on
 * success and a negative value on a bad argument.
 *
 * ORACLE_PLANT (a compile-time integer, unset in every normal build) plants
 * one deliberate mistake so that the tests can show that the pins catch it:
 *   1 conjugated twiddle in the FFT combine    2 direct sum drops its last term
 *   3 FFT combine ignores the twiddle stride    4 digit reversal reverses bits
 *   5 sampled sum uses index k+1               6 FFT swaps the butterfly outputs
 */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI_L 3.141592653589793238462643383279502884L

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* exp(dir * 2*pi*i * r / n) for an exact residue 0 <= r < n, in long double. */
static void unit_root_ld(int64_t r, int64_t n, int dir, long double *c, long double *s)
{
    long double ang = 2.0L * ORACLE_PI_L * (long double)r / (long double)n;
    *c = cosl(ang);
    *s = (long double)dir * sinl(ang);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Direct DFT: y[k] = sum_j x[j] * w_n^{dir*k*j}  (Sect. 2 definition).    */
/* ---------------------------------------------------------------------- */
int oracle_dft_direct(int64_t n, const double *x, double *y, int dir)
{
    if (n <= 0 || (dir != -1 && dir != 1) || n > (1LL << 20)) return -1;
    long double *tc = (long double *)malloc(sizeof(long double) * (size_t)n);
    long double *ts = (long double *)malloc(sizeof(long double) * (size_t)n);
    if (!tc || !ts) { free(tc); free(ts); return -2; }
    for (int64_t r = 0; r < n; ++r) unit_root_ld(r, n, dir, &tc[r], &ts[r]);
    for (int64_t k = 0; k < n; ++k) {
        long double are = 0.0L, aim = 0.0L;
        for (int64_t j = 0; j < (ORACLE_PLANT == 2 ? n - 1 : n); ++j) {
            int64_t r = (k * j) % n;          /* exact residue */
            long double xr = x[2 * j], xi = x[2 * j + 1];
            are += xr * tc[r] - xi * ts[r];
            aim += xr * ts[r] + xi * tc[r];
        }
        y[2 * k] = (double)are;
        y[2 * k + 1] = (double)aim;
    }
    free(tc);
    free(ts);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Recursive radix-2 decimation-in-time FFT (textbook Cooley-Tukey).       */
/* ---------------------------------------------------------------------- */
/* The butterflies of one combine step, k in [k0, k1): y[k], y[k+h] from the
 * half-length DFTs of the evens (y[0..h)) and the odds (y[h..n)).
 * tw[r] = w_N^{dir*r} for r < N/2; at size n = 2h the root w_n^{dir*k}
 * is tw[k * tw_step] with tw_step = N/n.                                  */
static void combine(int64_t h, double *y, const double *tw, int64_t tw_step, int64_t k0, int64_t k1)
{
    for (int64_t k = k0; k < k1; ++k) {
        int64_t ti_ = (ORACLE_PLANT == 3) ? k : k * tw_step;
        double wr = tw[2 * ti_], wi = tw[2 * ti_ + 1];
        if (ORACLE_PLANT == 1) wi = -wi;
        double orr = y[2 * (k + h)], oi = y[2 * (k + h) + 1];
        double tr = wr * orr - wi * oi;
        double ti = wr * oi + wi * orr;
        double er = y[2 * k], ei = y[2 * k + 1];
        if (ORACLE_PLANT == 6 && k == 1) { tr = -tr; ti = -ti; }
        y[2 * k] = er + tr;
        y[2 * k + 1] = ei + ti;
        y[2 * (k + h)] = er - tr;
        y[2 * (k + h) + 1] = ei - ti;
    }
}

/* y[0..n) = DFT_n of x[0], x[stride], ..., x[(n-1)*stride].               */
static void fft_rec(int64_t n, const double *x, int64_t stride, double *y,
                    const double *tw, int64_t tw_step)
{
    if (n == 1) {
        y[0] = x[0];
        y[1] = x[1];
        return;
    }
    int64_t h = n / 2;
    fft_rec(h, x, 2 * stride, y, tw, 2 * tw_step);                /* evens */
    fft_rec(h, x + 2 * stride, 2 * stride, y + 2 * h, tw, 2 * tw_step); /* odds */
    combine(h, y, tw, tw_step, 0, h);
}

/* The same recursion with its top `depth` levels spread over OpenMP tasks:
 * the two halves of a level run as two tasks, and its combine step is cut
 * into independent ranges of k.  Every output is produced by the same
 * butterflies, on the same operands, as in fft_rec, so the result is
 * bit-identical to the serial one for any thread count.  Called from inside
 * a parallel region.                                                      */
static void fft_rec_tasks(int64_t n, const double *x, int64_t stride, double *y,
                          const double *tw, int64_t tw_step, int depth)
{
    if (depth <= 0 || n < ((int64_t)1 << 15)) {
        fft_rec(n, x, stride, y, tw, tw_step);
        return;
    }
    int64_t h = n / 2;
#ifdef _OPENMP
#pragma omp task
#endif
    fft_rec_tasks(h, x, 2 * stride, y, tw, 2 * tw_step, depth - 1);
#ifdef _OPENMP
#pragma omp task
#endif
    fft_rec_tasks(h, x + 2 * stride, 2 * stride, y + 2 * h, tw, 2 * tw_step, depth - 1);
#ifdef _OPENMP
#pragma omp taskwait
#endif
    const int64_t chunk = (int64_t)1 << 14;
    for (int64_t k0 = 0; k0 < h; k0 += chunk) {
        int64_t k1 = k0 + chunk < h ? k0 + chunk : h;
#ifdef _OPENMP
#pragma omp task firstprivate(k0, k1)
#endif
        combine(h, y, tw, tw_step, k0, k1);
    }
#ifdef _OPENMP
#pragma omp taskwait
#endif
}

static double *make_half_table(int64_t n, int dir)
{
    int64_t h = n > 1 ? n / 2 : 1;
    double *tw = (double *)malloc(sizeof(double) * 2 * (size_t)h);
    if (!tw) return NULL;
    /* each entry depends on r alone: the loop may run on any thread count */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (h >= 65536)
#endif
    for (int64_t r = 0; r < h; ++r) {
        long double c, s;
        unit_root_ld(r, n, dir, &c, &s);
        tw[2 * r] = (double)c;
        tw[2 * r + 1] = (double)s;
    }
    return tw;
}

/* Batched recursive FFT: `batch` contiguous transforms of length n, on up
 * to `threads` OpenMP threads (threads <= 0: the runtime default).  With at
 * least as many transforms as threads, whole transforms run in parallel;
 * otherwise each transform's top recursion levels run as tasks
 * (fft_rec_tasks).  Either way each output comes from the same arithmetic
 * as the one-thread recursion.                                            */
int oracle_fft(int64_t n, int64_t batch, const double *x, double *y, int dir, int threads)
{
    if (!is_pow2(n) || batch < 0 || (dir != -1 && dir != 1)) return -1;
    if (batch == 0) return 0;
    double *tw = make_half_table(n, dir);
    if (!tw) return -2;
#ifdef _OPENMP
    int nt = threads > 0 ? threads : omp_get_max_threads();
    if (batch >= nt || nt == 1) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) if (batch > 1)
        for (int64_t t = 0; t < batch; ++t)
            fft_rec(n, x + 2 * t * n, 1, y + 2 * t * n, tw, 1);
    } else {
        int depth = 0;
        while ((1 << depth) < 4 * nt) ++depth;     /* about four tasks per thread */
        for (int64_t t = 0; t < batch; ++t) {
#pragma omp parallel num_threads(nt)
#pragma omp single
            fft_rec_tasks(n, x + 2 * t * n, 1, y + 2 * t * n, tw, 1, depth);
        }
    }
#else
    for (int64_t t = 0; t < batch; ++t)
        fft_rec(n, x + 2 * t * n, 1, y + 2 * t * n, tw, 1);
#endif
    (void)threads;
    free(tw);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* The definition at selected outputs: y[k] = sum_j x[j] w_n^{dir*k*j}.    */
/* FP64, exact residues r = k*j mod n, roots from two long-double-derived  */
/* tables w^{r} = hi[r >> hb] * lo[r & (2^hb - 1)], pairwise summation.     */
/* ---------------------------------------------------------------------- */
static void pairwise_acc(const double *x, int64_t j0, int64_t len, int64_t k, int64_t n,
                         const double *lo, const double *hi, int hb, double *sre, double *sim)
{
    if (len <= 256) {
        double ar = 0.0, ai = 0.0;
        uint64_t mask = ((uint64_t)1 << hb) - 1;
        for (int64_t j = j0; j < j0 + len; ++j) {
            uint64_t r = (uint64_t)(((__int128)(ORACLE_PLANT == 5 ? k + 1 : k) * j) % n);
            const double *a = lo + 2 * (r & mask), *b = hi + 2 * (r >> hb);
            double wr = a[0] * b[0] - a[1] * b[1];
            double wi = a[0] * b[1] + a[1] * b[0];
            double xr = x[2 * j], xi = x[2 * j + 1];
            ar += xr * wr - xi * wi;
            ai += xr * wi + xi * wr;
        }
        *sre = ar;
        *sim = ai;
        return;
    }
    int64_t h = len / 2;
    double r1, i1, r2, i2;
    pairwise_acc(x, j0, h, k, n, lo, hi, hb, &r1, &i1);
    pairwise_acc(x, j0 + h, len - h, k, n, lo, hi, hb, &r2, &i2);
    *sre = r1 + r2;
    *sim = i1 + i2;
}

int oracle_dft_at(int64_t n, const double *x, int64_t count, const int64_t *ks,
                  double *out, int dir, int threads)
{
    if (n <= 0 || count < 0 || (dir != -1 && dir != 1)) return -1;
    int hb = 0;
    while (((int64_t)1 << (2 * hb)) < n) ++hb;          /* 2^hb >= sqrt(n) */
    int64_t nlo = (int64_t)1 << hb, nhi = (n + nlo - 1) / nlo;
    double *lo = (double *)malloc(sizeof(double) * 2 * (size_t)nlo);
    double *hi = (double *)malloc(sizeof(double) * 2 * (size_t)nhi);
    if (!lo || !hi) { free(lo); free(hi); return -2; }
    for (int64_t r = 0; r < nlo; ++r) {
        long double c, s;
        unit_root_ld(r % n, n, dir, &c, &s);
        lo[2 * r] = (double)c;
        lo[2 * r + 1] = (double)s;
    }
    for (int64_t r = 0; r < nhi; ++r) {
        long double c, s;
        unit_root_ld((r * nlo) % n, n, dir, &c, &s);
        hi[2 * r] = (double)c;
        hi[2 * r + 1] = (double)s;
    }
    for (int64_t i = 0; i < count; ++i)
        if (ks[i] < 0 || ks[i] >= n) { free(lo); free(hi); return -1; }
#ifdef _OPENMP
    int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t i = 0; i < count; ++i)
        pairwise_acc(x, 0, n, ks[i], n, lo, hi, hb, &out[2 * i], &out[2 * i + 1]);
    (void)threads;
    free(lo);
    free(hi);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Base-b digit reversal pi_ell (Sect. 3.2; App. A.1): the ell-digit       */
/* base-b string d_{ell-1} ... d_0 of u maps to d_0 ... d_{ell-1}.         */
/* ---------------------------------------------------------------------- */
int64_t oracle_digit_reverse(int64_t u, int64_t b, int ell)
{
    if (b < 2 || ell < 0 || ell > 62 || u < 0) return -1;
    if (ORACLE_PLANT == 4) {                 /* planted: bit reversal */
        int t = 0;
        while (((int64_t)1 << t) < b) ++t;
        b = 2;
        ell *= t;
    }
    int64_t digits[64];
    int64_t v = u;
    for (int i = 0; i < ell; ++i) {        /* digits[i] = d_i, least significant first */
        digits[i] = v % b;
        v /= b;
    }
    if (v != 0) return -1;                 /* u has more than ell digits */
    int64_t out = 0;
    for (int i = 0; i < ell; ++i)          /* d_0 becomes the most significant digit */
        out = out * b + digits[i];
    return out;
}

/* pi_ell applied to every u in [0, b^ell): out[u] = pi_ell(u). */
int oracle_digit_reverse_table(int64_t b, int ell, int64_t *out)
{
    if (b < 2 || ell < 0) return -1;
    int64_t n = 1;
    for (int i = 0; i < ell; ++i) n *= b;
    for (int64_t u = 0; u < n; ++u) out[u] = oracle_digit_reverse(u, b, ell);
    return 0;
}
