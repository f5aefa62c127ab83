/*
 * Oracle: per-axis factors of the G-tensor by adaptive Gauss-Kronrod quadrature.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the plain FP64 CPU oracle.  It is
 * built and called by the tests, by __graft_entry__.smoke() and by the CPU-baseline
 * leg of bench.py, never by the library's solve path, and it shares no code with it.
 *
 * Sec. 2 (the G-tensor formula) writes the symbol of the Gaussian-sum kernel as a
 * product over the axes of one-dimensional integrals and says they are computed by
 * one-dimensional adaptive Gauss-Kronrod quadrature.  For a cube (l_q = 1) the
 * factor of term j at integer frequency k is
 *
 *     A_j(k) = 2 * integral_0^2 exp(-tau_j^2 t^2) cos(pi k t / 2) dt .
 *
 * The rule pair is the 7-point Gauss / 15-point Kronrod pair.  Each (j, k) integral is
 * refined by recursive bisection: a panel is accepted when the Kronrod-minus-Gauss
 * difference on it is below atol * (panel length / 2), so the summed error estimate is
 * below atol over [0, 2].  atol is relative to the scale min(4, sqrt(pi)/tau_j) of the
 * integral, which is A_j(0) up to a factor erf(2 tau_j) in [0.99, 1] for tau_j >= 1.
 */
#include <math.h>
#include <stddef.h>

/* Kronrod abscissae on [-1, 1] (positive half, decreasing; the last one is 0). */
static const double XK[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
/* Kronrod weights for XK. */
static const double WK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
/* Gauss weights for the Gauss abscissae XK[1], XK[3], XK[5] and the centre XK[7]. */
static const double WG[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static inline double integrand(double tau2, double kap, double t) {
    return exp(-tau2 * t * t) * cos(kap * t);
}

/* One G7/K15 panel.  The error estimate is the one of QUADPACK's 15-point rule
 * (Piessens et al., 1983): the Kronrod-Gauss difference is rescaled by the integral of
 * |f - mean| over the panel.  *floor_ is 50 ulp of the integral of |f|: an estimate
 * at or below it is round-off, and the panel is accepted whatever the tolerance. */
static void gk15(double tau2, double kap, double a, double b, double *res, double *err,
                 double *floor_) {
    double c = 0.5 * (a + b), hw = 0.5 * (b - a);
    double f[15];
    f[7] = integrand(tau2, kap, c);
    for (int i = 0; i < 7; ++i) {
        double dx = hw * XK[i];
        f[i] = integrand(tau2, kap, c - dx);
        f[14 - i] = integrand(tau2, kap, c + dx);
    }
    double rk = WK[7] * f[7], rg = WG[3] * f[7], rabs = WK[7] * fabs(f[7]);
    for (int i = 0; i < 7; ++i) {
        double s = f[i] + f[14 - i];
        rk += WK[i] * s;
        rabs += WK[i] * (fabs(f[i]) + fabs(f[14 - i]));
        if (i & 1) rg += WG[i >> 1] * s;
    }
    double mean = 0.5 * rk, rasc = WK[7] * fabs(f[7] - mean);
    for (int i = 0; i < 7; ++i) rasc += WK[i] * (fabs(f[i] - mean) + fabs(f[14 - i] - mean));
    double e = fabs((rk - rg) * hw);
    rasc *= hw;
    rabs *= hw;
    if (rasc != 0.0 && e != 0.0) {
        double q = pow(200.0 * e / rasc, 1.5);
        e = rasc * (q < 1.0 ? q : 1.0);
    }
    *floor_ = 50.0 * 2.220446049250313e-16 * rabs;
    *res = rk * hw;
    *err = e;
}

/* Recursive bisection; returns the integral over [a, b].  *npanel counts accepted panels. */
static double adapt(double tau2, double kap, double a, double b, double atol, int depth,
                    long *npanel) {
    double res, err, fl;
    gk15(tau2, kap, a, b, &res, &err, &fl);
    if (err <= atol * 0.5 * (b - a) || err <= fl || depth >= 30) {
        ++*npanel;
        return res;
    }
    double m = 0.5 * (a + b);
    return adapt(tau2, kap, a, m, atol, depth + 1, npanel) +
           adapt(tau2, kap, m, b, atol, depth + 1, npanel);
}

/* Test hook: the raw Kronrod and Gauss sums of t^p over one panel [a, b], so the tests
 * can check the stored abscissae and weights by their exactness on monomials. */
void oracle_gk15_monomial(int p, double a, double b, double *kron, double *gauss) {
    double c = 0.5 * (a + b), hw = 0.5 * (b - a);
    double rk = WK[7] * pow(c, p), rg = WG[3] * pow(c, p);
    for (int i = 0; i < 7; ++i) {
        double dx = hw * XK[i];
        double s = pow(c - dx, p) + pow(c + dx, p);
        rk += WK[i] * s;
        if (i & 1) rg += WG[i >> 1] * s;
    }
    *kron = rk * hw;
    *gauss = rg * hw;
}

/*
 * A[j * (kmax + 1) + k] = A_j(k) for j < nterms, 0 <= k <= kmax.
 * rtol: acceptance tolerance relative to min(4, sqrt(pi)/tau_j).
 * Returns the total number of accepted panels.
 */
long oracle_a_table(const double *tau, int nterms, int kmax, double rtol, double *A) {
    long total = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
    for (int j = 0; j < nterms; ++j) {
        double tj = tau[j];
        double scale = sqrt(M_PI) / tj;
        if (scale > 4.0) scale = 4.0;
        double atol = rtol * scale;
        for (int k = 0; k <= kmax; ++k) {
            long np = 0;
            double kap = 0.5 * M_PI * (double)k;
            /* Break points.  (1) t = 8 / tau: for large tau the integrand is a spike at
             * t = 0 narrower than the node spacing of a panel on [0, 2], which the rule
             * would miss.  (2) One panel per period 4 / k of cos(pi k t / 2): a panel
             * spanning many periods can alias to a smooth-looking sample and pass the
             * Kronrod-Gauss test with a wrong value. */
            double tb = 8.0 / tj;
            double tend = (tb < 2.0) ? tb : 2.0;
            int np0 = (k + 1) / 2;
            if (np0 < 1) np0 = 1;
            double v = 0.0;
            for (int p = 0; p < np0; ++p) {
                double a = 2.0 * p / np0, b = 2.0 * (p + 1) / np0;
                if (a >= tend) break;
                if (b > tend) b = tend;
                v += adapt(tj * tj, kap, a, b, atol, 0, &np);
            }
            if (tend < 2.0) v += adapt(tj * tj, kap, tend, 2.0, atol, 0, &np);
            A[(size_t)j * (size_t)(kmax + 1) + (size_t)k] = 2.0 * v;
            total += np;
        }
    }
    return total;
}
