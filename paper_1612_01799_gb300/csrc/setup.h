// Host-side FP64 setup of a solve plan (Sec. 2 and Sec. 3 of Exl, arXiv:1612.01799).
#pragma once
#include <cstddef>
#include <vector>

namespace gsp {

struct HostTables {
    int N = 0;
    double L = 0, tol = 0;
    double lambda = 0;   // box scale, = L for the cube [-L, L]^3
    double delta = 0;    // near-zone radius (scaled coordinates)
    double eps = 0;      // Gaussian-sum accuracy
    double r_max = 0;    // fit range upper end, 2 |l| = 2 sqrt(3)
    double h = 0;        // sinc-quadrature step
    double gs_err = 0;   // measured max relative error of U_GS on the fit grid
    std::vector<double> tau, w;   // Gaussian sum, S+1 terms
    std::vector<double> A;        // (S+1) x (N+1): A_j(k), row-major (the x axis of a box)
    double C0 = 0, C2 = 0;        // near-zone Taylor constants
    // Box [-L_x, L_x] x [-L_y, L_y] x [-L_z, L_z] (Sec. 2 standardised form): half-lengths
    // l_q = L_q / lambda of the scaled box; all 1 for the cube.
    bool box = false;
    double l[3] = {1.0, 1.0, 1.0};
    std::vector<double> A3;       // box: the three axes' tables l_q A_j(tau_j l_q), x, y, z
};

// eps = clamp(tol/10, 1e-14, 1e-7).
double eps_for_tol(double tol);
// Sec. 3 heuristic for a cube: 2L/(50 N), at least 1e-3.
double delta_for_cube(double L, int N);
// Inverse of the complementary error function on (0, 2).
double erfc_inverse(double y);

// Sinc quadrature of 1/(4 pi r) on [delta, r_max] to max relative error eps.
// Returns false if no step on the ladder reaches eps.
bool build_gauss_sum(double eps, double delta, double r_max, std::vector<double> &tau,
                     std::vector<double> &w, double &h, double &err);

// A[j*(N+1)+k] = 2 int_0^2 exp(-tau_j^2 t^2) cos(pi k t / 2) dt, k = 0..N.
void build_axis_table(const std::vector<double> &tau, int N, std::vector<double> &A);

// Panels of the composite Gauss-Legendre rule of the axis table: max(16, (N + 1) / 2).
int axis_table_panels(int N);

// The 16-point Gauss-Legendre nodes x[16] and weights w[16] on [-1, 1].
void gauss_legendre16(double *x, double *w);

// C0 and C2 of I_delta = C0 rho + C2 Laplace(rho).
void near_zone_constants(const std::vector<double> &tau, const std::vector<double> &w,
                         double delta, double &C0, double &C2);

// Everything above for the cube [-L, L]^3 with N points per axis.  Returns 0 or a
// POISSON_ERR_* code.
int build_host_tables(int N, double L, double tol, HostTables &out);

// The same without the axis table (out.A left empty), for a setup that builds the table
// on the device.
int build_host_scalars(int N, double L, double tol, HostTables &out);

// The scalars for the box [-L3[0], L3[0]] x [-L3[1], L3[1]] x [-L3[2], L3[2]] with n3[q]
// points on axis q: lambda = max_q L_q, l_q = L_q / lambda, delta = max(min_q 2 L_q /
// (50 n_q), 1e-3) below min_q l_q, the Gaussian sum fitted on [delta, 2 |l|].
int build_host_scalars_box(const int *n3, const double *L3, double tol, HostTables &out);

// tw[e] = exp(-2 pi i e / n), e in [0, n), as (re, im) pairs, accurate to FP64 rounding.
void twiddles(int n, std::vector<double> &re_im);

}  // namespace gsp
