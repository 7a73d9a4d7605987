// Host numerics of the solver: finite-difference weights (Fornberg's
// recursion), the leapfrog stability limit and the default absorbing-layer
// profile. Double precision on the host; the kernels receive FP32 copies.
#include <cmath>
#include <cstddef>
#include <vector>

#include "fd_internal.h"

namespace fdgb {

// Weights of the centred second derivative of accuracy order k = 2r on the
// unit-spaced nodes -r..r (Listing 1: space_order; Listing 2 shows k = 2 with
// taps 1, -2, 1 per axis). Computed with Fornberg's recursion for
// finite-difference weights on arbitrary nodes (B. Fornberg, Math. Comp. 51,
// 1988): weights for derivative orders 0..2 are built up one node at a time.
// Output c[j] is the weight of nodes +-j, j = 0..r.
bool fornberg_second_derivative(int space_order, double *c) {
    if (space_order < 2 || space_order % 2 != 0 || space_order > 2 * kMaxRadiusHost) return false;
    const int r = space_order / 2;
    const int n_nodes = 2 * r + 1;
    constexpr int M = 2;  // highest derivative order carried
    // fixed-size arrays: no heap use, so the allocation-free entry point can call it too
    double node[2 * kMaxRadiusHost + 1];
    for (int i = 0; i < n_nodes; ++i) node[i] = double(i - r);
    const double x0 = 0.0;
    // w[m][nu]: weight of node nu for derivative m, using the nodes seen so far
    double w[M + 1][2 * kMaxRadiusHost + 1] = {};
    w[0][0] = 1.0;
    double prod_prev = 1.0;
    double dist_last = node[0] - x0;
    for (int n = 1; n < n_nodes; ++n) {
        double prod = 1.0;
        const double dist_prev = dist_last;
        dist_last = node[n] - x0;
        const int mmax = n < M ? n : M;
        for (int nu = 0; nu < n; ++nu) {
            const double gap = node[n] - node[nu];
            prod *= gap;
            if (nu == n - 1) {
                // weights of the new node from the previous node's old weights
                for (int m = mmax; m >= 0; --m) {
                    const double lower = m > 0 ? w[m - 1][n - 1] : 0.0;
                    w[m][n] = prod_prev * (double(m) * lower - dist_prev * w[m][n - 1]) / prod;
                }
            }
            for (int m = mmax; m >= 0; --m) {
                const double lower = m > 0 ? w[m - 1][nu] : 0.0;
                w[m][nu] = (dist_last * w[m][nu] - double(m) * lower) / gap;
            }
        }
        prod_prev = prod;
    }
    for (int j = 0; j <= r; ++j) c[j] = w[2][r + j];
    return true;
}

double stability_limit(int space_order, double h, double vmax) {
    double c[kMaxRadiusHost + 1];
    if (!fornberg_second_derivative(space_order, c) || !(h > 0) || !(vmax > 0)) return -1.0;
    double s = std::fabs(c[0]);
    for (int j = 1; j <= space_order / 2; ++j) s += 2.0 * std::fabs(c[j]);
    // -L peaks at the Nyquist mode with 3 s / h^2; leapfrog needs dt^2 v^2 peak <= 4
    return 2.0 * h / (vmax * std::sqrt(3.0 * s));
}

// Default damping eta = m * sum_a d_max (l_a / nbl)^2 with l_a the depth in
// cells into the layer along axis a and d_max = 3 v_max ln(1000) / (2 nbl h).
void default_damping(const float *m, float *eta, int Nx, int Ny, int Nz, int nbl, double h,
                     double vmax) {
    const size_t plane = size_t(Ny) * size_t(Nz);
    if (nbl <= 0) {
        for (size_t i = 0; i < size_t(Nx) * plane; ++i) eta[i] = 0.0f;
        return;
    }
    const double dmax = 3.0 * vmax * std::log(1000.0) / (2.0 * double(nbl) * h);
    auto frac2 = [nbl](int i, int N) {
        int lo = nbl - i, hi = i - (N - 1 - nbl);
        int d = lo > hi ? lo : hi;
        if (d < 0) d = 0;
        double f = double(d) / double(nbl);
        return f * f;
    };
    std::vector<double> fy(Ny), fz(Nz);
    for (int y = 0; y < Ny; ++y) fy[y] = frac2(y, Ny);
    for (int z = 0; z < Nz; ++z) fz[z] = frac2(z, Nz);
    for (int x = 0; x < Nx; ++x) {
        const double fx = frac2(x, Nx);
        for (int y = 0; y < Ny; ++y) {
            const size_t row = size_t(x) * plane + size_t(y) * size_t(Nz);
            for (int z = 0; z < Nz; ++z) {
                const double d = dmax * (fx + fy[y] + fz[z]);
                eta[row + z] = float(double(m[row + z]) * d);
            }
        }
    }
}

}  // namespace fdgb
