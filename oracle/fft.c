/*
 * Oracle: a plain FP64 discrete Fourier transform of its own.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the plain FP64 CPU oracle.  It is
 * built and called by the tests, by __graft_entry__.smoke() and by the CPU-baseline
 * leg of bench.py, never by the library's solve path, and it shares no code with it.
 *
 * Sec. 2 evaluates the Gaussian-sum convolution by the convolution theorem on the
 * zero-padded grid, and Sec. 3 counts the cost of those transforms (size 8 N_tot).  The
 * transform is the unnormalised DFT along one axis,
 *
 *     X[k] = sum_{j=0}^{n-1} x[j] exp(sign * 2 pi i j k / n),   sign = -1 forward, +1 inverse,
 *
 * computed by the recursive decimation-in-time Cooley-Tukey split n = p m: the p
 * interleaved subsequences x[p j + r] (r = 0..p-1) are transformed (length m), and
 *
 *     X[k + m s] = sum_{r=0}^{p-1} W_n^{r k} W_p^{r s} Y_r[k],   W_n = exp(sign 2 pi i / n),
 *
 * for k < m, s < p.  The radices are 5, 3 and 2 (and, for a length with another prime
 * factor, that prime), each p-point step a direct O(p^2) sum.  No pruning, no
 * reordering beyond the split: every transform is the full complex one.
 *
 * Twiddles W_n^e are cos and sin of 2 pi e / n with the angle reduced to [0, pi/4] by
 * the octant symmetries, so that values tied by symmetry are exactly equal.
 *
 * Arrays are complex128 (re, im interleaved) in C order with shape (n0, n1, n2); the
 * transform runs along one axis over every line of the other two, lines in parallel
 * (OpenMP).
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cplx;

#define MAXF 64

typedef struct {
    int n;            /* transform length */
    int nf;           /* number of factors */
    int fac[MAXF];    /* radices, outermost first */
    cplx *w;          /* w[e] = exp(-2 pi i e / n), e = 0..n-1 */
} plan1d;

/* exp(-2 pi i e / n) with the angle reduced to an octant: 8 e = o n + r, 0 <= r < n. */
static cplx twiddle(long e, long n)
{
    e %= n;
    if (e < 0) e += n;
    long t = 8 * e;
    long o = t / n, r = t - o * n;
    const double q = M_PI / 4.0;
    double phi = q * (double)r / (double)n;          /* theta = q o + phi        */
    double psi = q * (double)(n - r) / (double)n;    /* theta = q (o + 1) - psi  */
    double c, s;                                     /* cos theta, sin theta     */
    switch (o) {
    case 0: c = cos(phi); s = sin(phi); break;
    case 1: c = sin(psi); s = cos(psi); break;
    case 2: c = -sin(phi); s = cos(phi); break;
    case 3: c = -cos(psi); s = sin(psi); break;
    case 4: c = -cos(phi); s = -sin(phi); break;
    case 5: c = -sin(psi); s = -cos(psi); break;
    case 6: c = sin(phi); s = -cos(phi); break;
    default: c = cos(psi); s = -sin(psi); break;
    }
    cplx w = {c, -s};
    return w;
}

static int factorise(int n, int *fac)
{
    int nf = 0;
    static const int small[3] = {5, 3, 2};
    for (int i = 0; i < 3; ++i)
        while (n % small[i] == 0 && nf < MAXF) { fac[nf++] = small[i]; n /= small[i]; }
    for (int p = 7; n > 1 && nf < MAXF; p += 2)
        while (n % p == 0) { fac[nf++] = p; n /= p; }
    return n == 1 ? nf : -1;
}

static int plan_init(plan1d *P, int n)
{
    P->n = n;
    P->nf = factorise(n, P->fac);
    if (P->nf < 0) return -1;
    P->w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!P->w) return -1;
    for (int e = 0; e < n; ++e) P->w[e] = twiddle(e, n);
    return 0;
}

/* W_N^e (0 <= e < N) for the plan's length N, conjugated for the inverse transform. */
static inline cplx W(const plan1d *P, long e, int sign)
{
    cplx w = P->w[e];
    if (sign > 0) w.im = -w.im;
    return w;
}

static inline cplx cmul(cplx a, cplx b)
{
    cplx c = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return c;
}

/*
 * y[0..n) = DFT_n of x[0], x[xs], x[2 xs], ...  (out of place; level indexes P->fac).
 * Length n = P->n / (product of the factors above this level).  tmp holds at least 2 p
 * values; a level uses it only after its sub-transforms have returned.
 */
static void dft_rec(const cplx *x, long xs, cplx *y, int n, int level, const plan1d *P, int sign,
                    cplx *tmp)
{
    const int p = P->fac[level];
    const int m = n / p;
    if (m > 1)
        for (int r = 0; r < p; ++r)
            dft_rec(x + r * xs, xs * p, y + (long)r * m, m, level + 1, P, sign, tmp);
    /* W_n^e = W_N^{e N/n}, W_p^e = W_N^{e N/p}. */
    const long sn = P->n / n, sp = P->n / p;
    cplx *t = tmp, *wp = tmp + p;
    for (int e = 0; e < p; ++e) wp[e] = W(P, e * sp, sign);
    for (int k = 0; k < m; ++k) {
        if (m > 1) {
            t[0] = y[k];
            for (int r = 1; r < p; ++r) t[r] = cmul(y[(long)r * m + k], W(P, (long)r * k * sn, sign));
        } else {
            for (int r = 0; r < p; ++r) t[r] = x[r * xs];
        }
        for (int s = 0; s < p; ++s) {
            cplx acc = t[0];
            int e = 0;                                   /* e = r s mod p */
            for (int r = 1; r < p; ++r) {
                e += s;
                if (e >= p) e -= p;
                cplx v = cmul(t[r], wp[e]);
                acc.re += v.re;
                acc.im += v.im;
            }
            y[(long)s * m + k] = acc;
        }
    }
}

#define BLOCK 8   /* lines gathered together along the contiguous axis */

/*
 * Transform every line along `axis` (0, 1 or 2) of the complex array data[n0][n1][n2],
 * in place.  sign = -1: forward, +1: inverse; neither is normalised.  threads: OpenMP
 * threads (0: the OpenMP default).  Returns 0, or -1 on a bad argument or a failed
 * allocation.
 */
int oracle_fft_axis(double *data, long n0, long n1, long n2, int axis, int sign, int threads)
{
    if (!data || n0 < 1 || n1 < 1 || n2 < 1 || axis < 0 || axis > 2 || (sign != 1 && sign != -1))
        return -1;
    const long dims[3] = {n0, n1, n2};
    const long n = dims[axis];
    if (n == 1) return 0;
    if (n > (1L << 30)) return -1;
    const long stride = axis == 0 ? n1 * n2 : axis == 1 ? n2 : 1;
    /* Lines come in groups: for axis 2 one line each; for the other axes up to BLOCK
     * lines adjacent along the contiguous axis (their elements sit side by side). */
    const long width = axis == 2 ? 1 : BLOCK;
    const long per_row = axis == 2 ? 1 : (n2 + width - 1) / width;
    const long rows = axis == 2 ? n0 * n1 : (axis == 1 ? n0 : n1);
    const long groups = rows * per_row;
    plan1d P;
    if (plan_init(&P, (int)n) != 0) return -1;
    cplx *base = (cplx *)data;
    int failed = 0;
    const int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel num_threads(nt) reduction(| : failed)
    {
        cplx *in = (cplx *)malloc(sizeof(cplx) * (size_t)(n * width));
        cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)(2 * n + 16));
        if (!in || !out || !tmp) {
            failed = 1;
        } else {
#pragma omp for schedule(static)
            for (long g = 0; g < groups; ++g) {
                long off, cnt;
                if (axis == 2) {
                    off = g * n2;
                    cnt = 1;
                } else {
                    const long row = g / per_row, i2 = (g % per_row) * width;
                    off = (axis == 1 ? row * n1 * n2 : row * n2) + i2;
                    cnt = n2 - i2 < width ? n2 - i2 : width;
                }
                for (long j = 0; j < n; ++j)
                    for (long b = 0; b < cnt; ++b) in[b * n + j] = base[off + j * stride + b];
                for (long b = 0; b < cnt; ++b) {
                    dft_rec(in + b * n, 1, out, (int)n, 0, &P, sign, tmp);
                    memcpy(in + b * n, out, sizeof(cplx) * (size_t)n);
                }
                for (long j = 0; j < n; ++j)
                    for (long b = 0; b < cnt; ++b) base[off + j * stride + b] = in[b * n + j];
            }
        }
        free(in);
        free(out);
        free(tmp);
    }
    free(P.w);
    return failed ? -1 : 0;
}

/* The radices the transform of length n uses, outermost first (for the tests). */
int oracle_fft_factors(int n, int *fac, int cap)
{
    int f[MAXF];
    int nf = factorise(n, f);
    if (nf < 0) return -1;
    for (int i = 0; i < nf && i < cap; ++i) fac[i] = f[i];
    return nf;
}
