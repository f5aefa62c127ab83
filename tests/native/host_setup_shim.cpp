// Test shim: exposes the library's host-side plan setup (csrc/setup.cpp) to the CPU
// tests, so its tables can be compared with the oracle's without a GPU.
#include <algorithm>
#include <cstring>

#include "setup.h"

extern "C" int shim_host_tables(int N, double L, double tol, int cap_terms, int *n_terms,
                                double *tau, double *w, double *A, double *scalars) {
    gsp::HostTables t;
    int rc = gsp::build_host_tables(N, L, tol, t);
    if (rc) return rc;
    *n_terms = (int)t.tau.size();
    if ((int)t.tau.size() > cap_terms) return -100;
    std::copy(t.tau.begin(), t.tau.end(), tau);
    std::copy(t.w.begin(), t.w.end(), w);
    std::copy(t.A.begin(), t.A.end(), A);
    scalars[0] = t.delta;
    scalars[1] = t.eps;
    scalars[2] = t.C0;
    scalars[3] = t.C2;
    scalars[4] = t.h;
    scalars[5] = t.gs_err;
    return 0;
}

extern "C" void shim_twiddles(int n, double *out) {
    std::vector<double> v;
    gsp::twiddles(n, v);
    std::memcpy(out, v.data(), v.size() * sizeof(double));
}

// Box scalars (n3[q] points on axis q): out = {lambda, l_x, l_y, l_z, delta, eps, C0, C2, r_max}.
extern "C" int shim_box_scalars(const int *n3, const double *L3, double tol, int cap_terms, int *n_terms,
                                double *tau, double *w, double *out) {
    gsp::HostTables t;
    int rc = gsp::build_host_scalars_box(n3, L3, tol, t);
    if (rc) return rc;
    *n_terms = (int)t.tau.size();
    if ((int)t.tau.size() > cap_terms) return -100;
    std::copy(t.tau.begin(), t.tau.end(), tau);
    std::copy(t.w.begin(), t.w.end(), w);
    const double v[9] = {t.lambda, t.l[0], t.l[1], t.l[2], t.delta, t.eps, t.C0, t.C2, t.r_max};
    std::copy(v, v + 9, out);
    return 0;
}
