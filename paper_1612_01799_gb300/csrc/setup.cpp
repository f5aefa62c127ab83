// Host-side FP64 setup of a solve plan: delta, Gaussian sum, per-axis G-tensor
// factors, near-zone constants, twiddles.  Exl, arXiv:1612.01799, Sec. 2 and Sec. 3.
#include "setup.h"

#include <algorithm>
#include <cmath>
#include <thread>

#include "../../include/poisson.h"

namespace gsp {

static const double kPi = 3.141592653589793238462643383279502884;

double eps_for_tol(double tol) { return std::min(std::max(0.1 * tol, 1e-14), 1e-7); }

double delta_for_cube(double L, int N) {
    // Sec. 3: delta := min_q (b_q - a_q) / (50 n_q), with delta >= 1e-3.  The number is
    // used as is in the scaled coordinates of the box [-1, 1]^3.
    return std::max(2.0 * L / (50.0 * N), 1e-3);
}

double erfc_inverse(double y) {
    // erfc is strictly decreasing: bisection to the last bit, then one Newton step.
    double lo = -10.0, hi = 30.0;
    for (int it = 0; it < 200 && hi - lo > 0; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (std::erfc(mid) > y) lo = mid; else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    double d = -2.0 / std::sqrt(kPi) * std::exp(-x * x);
    if (d != 0.0) x -= (std::erfc(x) - y) / d;
    return x;
}

bool build_gauss_sum(double eps, double delta, double r_max, std::vector<double> &tau,
                     std::vector<double> &w, double &h, double &err) {
    // 1/(4 pi r) = 1/(2 pi^{3/2}) int_R exp(-r^2 e^{2s} + s) ds, trapezoid rule on the
    // grid s_j = j h.  Tails: dropping t = e^s < t_lo changes 4 pi r U by at most
    // erf(r t_lo) <= 2 r t_lo / sqrt(pi) (eps/4 at r_max); dropping t > t_hi by at most
    // erfc(delta t_hi) = eps/4.  Step: the largest h = 2/m whose measured maximum
    // relative error over 4096 log-spaced radii in [delta, r_max] is <= eps.
    const int nfit = 4096;
    const double t_lo = eps * std::sqrt(kPi) / (8.0 * r_max);
    const double t_hi = erfc_inverse(0.25 * eps) / delta;
    const double s_lo = std::log(t_lo), s_hi = std::log(t_hi);
    std::vector<double> r(nfit);
    const double lr0 = std::log(delta), lr1 = std::log(r_max);
    for (int i = 0; i < nfit; ++i) r[i] = std::exp(lr0 + (lr1 - lr0) * i / (nfit - 1));
    r[0] = delta;
    r[nfit - 1] = r_max;
    const double norm = 1.0 / (2.0 * std::pow(kPi, 1.5));
    // The sum and its error for h = 2/m.
    auto candidate = [&](int m, std::vector<double> &tt, std::vector<double> &ww) {
        const double hh = 2.0 / m;
        const long j0 = (long)std::floor(s_lo / hh), j1 = (long)std::ceil(s_hi / hh);
        tt.clear();
        ww.clear();
        for (long j = j0; j <= j1; ++j) {
            double s = (double)j * hh;
            tt.push_back(std::exp(s));
            ww.push_back(hh * std::exp(s) * norm);
        }
        double e = 0.0;
        for (int i = 0; i < nfit; ++i) {
            double acc = 0.0;
            for (size_t j = 0; j < tt.size(); ++j) {
                double a = r[i] * tt[j];
                acc += ww[j] * std::exp(-a * a);
            }
            e = std::max(e, std::fabs(4.0 * kPi * r[i] * acc - 1.0));
        }
        return e;
    };
    // The first m (smallest, i.e. the largest step) whose error is <= eps, found by
    // evaluating batches of consecutive m on the host's threads: the same m as a scan.
    const int batch = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    for (int m0 = 2; m0 < 4000; m0 += batch) {
        const int nb = std::min(batch, 4000 - m0);
        std::vector<std::vector<double>> tt(nb), ww(nb);
        std::vector<double> e(nb);
        std::vector<std::thread> th;
        for (int b = 0; b < nb; ++b) th.emplace_back([&, b]() { e[b] = candidate(m0 + b, tt[b], ww[b]); });
        for (auto &x : th) x.join();
        for (int b = 0; b < nb; ++b)
            if (e[b] <= eps) {
                tau.swap(tt[b]);
                w.swap(ww[b]);
                h = 2.0 / (m0 + b);
                err = e[b];
                return true;
            }
    }
    return false;
}

// Gauss-Legendre nodes and weights of order n on [-1, 1] by Newton's method on P_n.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &wt) {
    x.assign(n, 0.0);
    wt.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        wt[i] = wt[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

template <class F>
static void parallel_for(int n, F f) {
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 4 || nt == 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            for (int i = (int)t; i < n; i += (int)nt) f(i);
        });
    for (auto &x : th) x.join();
}

void build_axis_table(const std::vector<double> &tau, int N, std::vector<double> &A) {
    // tau >= 3: the Gaussian has decayed below erfc(6) ~ 2e-17 of its mass by t = 2,
    // so the factor is the full-line integral (sqrt(pi)/tau) exp(-kappa^2/(4 tau^2)).
    // tau < 3: composite 16-point Gauss-Legendre on [0, 2] with at least N/2 equal
    // panels, so one panel spans at most one period of cos(pi N t / 2).
    const int K = N + 1;
    const int S = (int)tau.size();
    A.assign((size_t)S * K, 0.0);
    const int order = 16;
    std::vector<double> gx, gw;
    gauss_legendre(order, gx, gw);
    const int P = axis_table_panels(N);
    const int T = P * order;
    std::vector<double> t(T), wt(T);
    for (int p = 0; p < P; ++p) {
        double a = 2.0 * p / P, b = 2.0 * (p + 1) / P;
        for (int i = 0; i < order; ++i) {
            t[p * order + i] = 0.5 * (a + b) + 0.5 * (b - a) * gx[i];
            wt[p * order + i] = 0.5 * (b - a) * gw[i];
        }
    }
    std::vector<int> small;
    for (int j = 0; j < S; ++j) {
        if (tau[j] >= 3.0) {
            for (int k = 0; k < K; ++k) {
                double kap = 0.5 * kPi * k;
                A[(size_t)j * K + k] =
                    std::sqrt(kPi) / tau[j] * std::exp(-kap * kap / (4.0 * tau[j] * tau[j]));
            }
        } else {
            small.push_back(j);
        }
    }
    if (small.empty()) return;
    std::vector<double> cosk((size_t)K * T);
    parallel_for(K, [&](int k) {
        double kap = 0.5 * kPi * k;
        for (int n = 0; n < T; ++n) cosk[(size_t)k * T + n] = std::cos(kap * t[n]);
    });
    parallel_for((int)small.size(), [&](int ii) {
        int j = small[ii];
        std::vector<double> g(T);
        double t2 = tau[j] * tau[j];
        for (int n = 0; n < T; ++n) g[n] = wt[n] * std::exp(-t2 * t[n] * t[n]);
        for (int k = 0; k < K; ++k) {
            // Compensated (Neumaier) summation: thousands of node terms of size ~1/P.
            const double *c = &cosk[(size_t)k * T];
            double acc = 0.0, comp = 0.0;
            for (int n = 0; n < T; ++n) {
                const double term = g[n] * c[n];
                const double t = acc + term;
                comp += (std::fabs(acc) >= std::fabs(term)) ? (acc - t) + term : (term - t) + acc;
                acc = t;
            }
            A[(size_t)j * K + k] = 2.0 * (acc + comp);
        }
    });
}

// int_0^d r^p exp(-tau^2 r^2) dr for p = 2, 4: closed forms through erf, or the power
// series sum_n (-tau^2)^n d^{2n+p+1} / (n! (2n+p+1)) when tau d < 1/2.
static double radial_moment(int p, double tau, double d) {
    double x = tau * d;
    if (x < 0.5) {
        double total = 0.0, fact = 1.0, t2n = 1.0;
        for (int n = 0; n < 80; ++n) {
            if (n > 0) {
                fact *= n;
                t2n *= -tau * tau;
            }
            double term = t2n * std::pow(d, 2 * n + p + 1) / (fact * (2 * n + p + 1));
            total += term;
            if (std::fabs(term) <= 1e-20 * std::fabs(total)) break;
        }
        return total;
    }
    double e = std::exp(-x * x), er = std::erf(x);
    if (p == 2) return std::sqrt(kPi) * er / (4.0 * tau * tau * tau) - d * e / (2.0 * tau * tau);
    return 3.0 * std::sqrt(kPi) * er / (8.0 * std::pow(tau, 5)) -
           e * (d * d * d / (2.0 * tau * tau) + 3.0 * d / (4.0 * std::pow(tau, 4)));
}

void near_zone_constants(const std::vector<double> &tau, const std::vector<double> &w,
                         double delta, double &C0, double &C2) {
    // I_delta = int_{B_delta} (U - U_GS)(y) rho(x - y) dy with the third-order Taylor
    // polynomial of rho: the odd orders and the mixed second derivatives integrate to
    // zero over the ball, and int y_q^2 f(|y|) = (1/3) int |y|^2 f(|y|), so
    // I_delta = C0 rho + C2 Laplace(rho) with C0 = int_{B_delta}(U - U_GS) and
    // C2 = (1/6) int_{B_delta} (U - U_GS) |y|^2; int_{B_delta} U = delta^2/2 and
    // int_{B_delta} U |y|^2 = delta^4/4.
    double s2 = 0.0, s4 = 0.0;
    for (size_t j = 0; j < tau.size(); ++j) {
        s2 += w[j] * radial_moment(2, tau[j], delta);
        s4 += w[j] * radial_moment(4, tau[j], delta);
    }
    C0 = 0.5 * delta * delta - 4.0 * kPi * s2;
    C2 = (0.25 * std::pow(delta, 4) - 4.0 * kPi * s4) / 6.0;
}

int axis_table_panels(int N) { return std::max(16, (N + 1) / 2); }

void gauss_legendre16(double *x, double *w) {
    std::vector<double> gx, gw;
    gauss_legendre(16, gx, gw);
    for (int i = 0; i < 16; ++i) x[i] = gx[i], w[i] = gw[i];
}

int build_host_tables(int N, double L, double tol, HostTables &o) {
    const int rc = build_host_scalars(N, L, tol, o);
    if (rc != POISSON_OK) return rc;
    build_axis_table(o.tau, N, o.A);
    return POISSON_OK;
}

int build_host_scalars(int N, double L, double tol, HostTables &o) {
    if (N < 4 || N > 1024 || (N & 1) || !(L > 0.0) || !(tol > 0.0) || !std::isfinite(L) ||
        !std::isfinite(tol))
        return POISSON_ERR_ARG;
    o.N = N;
    o.L = L;
    o.tol = tol;
    o.lambda = L;
    o.delta = delta_for_cube(L, N);
    if (!(o.delta < 1.0)) return POISSON_ERR_ARG;  // Sec. 3: delta < min_q l_q = 1
    o.eps = eps_for_tol(tol);
    o.r_max = 2.0 * std::sqrt(3.0);
    if (!build_gauss_sum(o.eps, o.delta, o.r_max, o.tau, o.w, o.h, o.gs_err))
        return POISSON_ERR_NUMERIC;
    near_zone_constants(o.tau, o.w, o.delta, o.C0, o.C2);
    return POISSON_OK;
}

int build_host_scalars_box(const int *n3, const double *L3, double tol, HostTables &o) {
    if (!n3 || !L3 || !(tol > 0.0) || !std::isfinite(tol)) return POISSON_ERR_ARG;
    for (int q = 0; q < 3; ++q)
        if (n3[q] < 4 || n3[q] > 1024 || (n3[q] & 1)) return POISSON_ERR_ARG;
    const int N = n3[0];
    double lam = 0.0, lmin = 0.0;
    for (int q = 0; q < 3; ++q) {
        if (!(L3[q] > 0.0) || !std::isfinite(L3[q])) return POISSON_ERR_ARG;
        lam = std::max(lam, L3[q]);
    }
    o.N = N;
    o.L = lam;
    o.tol = tol;
    o.lambda = lam;
    o.box = true;
    double l2 = 0.0;
    lmin = 1.0;
    for (int q = 0; q < 3; ++q) {
        o.l[q] = L3[q] / lam;
        l2 += o.l[q] * o.l[q];
        lmin = std::min(lmin, o.l[q]);
    }
    // Sec. 3: min_q (b_q - a_q) / (50 n_q), at least 1e-3, used as is in the scaled box.
    o.delta = std::max(std::min({2.0 * L3[0] / (50.0 * n3[0]), 2.0 * L3[1] / (50.0 * n3[1]),
                                 2.0 * L3[2] / (50.0 * n3[2])}),
                       1e-3);
    if (!(o.delta < lmin)) return POISSON_ERR_ARG;  // Sec. 3: delta < min_q l_q
    o.eps = eps_for_tol(tol);
    o.r_max = 2.0 * std::sqrt(l2);
    if (!build_gauss_sum(o.eps, o.delta, o.r_max, o.tau, o.w, o.h, o.gs_err))
        return POISSON_ERR_NUMERIC;
    near_zone_constants(o.tau, o.w, o.delta, o.C0, o.C2);
    return POISSON_OK;
}

void twiddles(int n, std::vector<double> &re_im) {
    re_im.resize(2 * (size_t)n);
    const long double two_pi = 2.0L * std::acos(-1.0L);
    for (int e = 0; e < n; ++e) {
        long double a = two_pi * (long double)e / (long double)n;
        re_im[2 * (size_t)e] = (double)std::cos(a);
        re_im[2 * (size_t)e + 1] = (double)-std::sin(a);
    }
}

}  // namespace gsp
