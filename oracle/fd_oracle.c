/*
 * FP64 CPU oracle for the explicit time step of the 3D acoustic isotropic wave
 * equation with absorbing-layer damping and point-source injection
 * (arXiv 1912.00695, Sec. 2.1 Eq. 1; the damped update as printed in Listing 2).
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY. Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may call it. It
 * shares no code, header or constant with the CUDA path.
 *
 * It is the plain definition of the scheme, written out loop by loop in
 * double precision, with no blocking, fusion or reordering:
 *
 *   m (u^{n+1} - 2u^n + u^{n-1}) / dt^2 - L u^n + eta (u^{n+1} - u^{n-1}) / (2 dt) = q^n
 *
 * solved for u^{n+1} (Eq. 1 plus the damping term of Listing 2), where L is the
 * central finite-difference Laplacian of accuracy order k ("space_order",
 * Listing 1) on an isotropic grid of spacing h.
 *
 * Grid convention: arrays are C-order [x][y][z] (z fastest) over the whole
 * computational domain (interior plus absorbing layer), the order Listing 2
 * indexes u[t][x][y][z]. Outside the domain the field is zero (Dirichlet), or
 * wraps around when `periodic` is set (periodic mode exists for the pins:
 * plane waves and energy conservation).
 *
 * Pins (tests/test_oracle_*.py): weights against an exact rational Vandermonde
 * solve and polynomial exactness; the Laplacian against the closed-form plane
 * wave symbol and symmetry; the step against u^{n+1} solved from the damped
 * Eq. 1 at k=2, h=1 (damping sign and r0 denominator as in Listing 2), a
 * dense-matrix brute force, the exact discrete plane-wave
 * solution and discrete energy conservation; dt_max against power iteration;
 * off-grid sampling against a library interpolator and affine exactness,
 * off-grid spreading against integer-node sources combined by linearity and a
 * dense brute force, and reciprocity between off-grid points.
 * The default damping profile is a convention the paper does not give
 * (parity unpinned as a formula; pinned only by its invariants).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_RADIUS 12

static size_t idx3(long x, long y, long z, long ny, long nz) {
    return ((size_t)x * (size_t)ny + (size_t)y) * (size_t)nz + (size_t)z;
}

/* Number of OpenMP threads the oracle will use (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Weights c_0..c_r of the centred second derivative of accuracy order k = 2r
 * (Listing 1's space_order; Listing 2 shows k=2: c_1 = 1, c_0 = -2 per axis).
 * Closed form: c_j = 2 (-1)^{j+1} (r!)^2 / (j^2 (r-j)! (r+j)!), j = 1..r, and
 * c_0 = -2 sum_j c_j (the weights annihilate constants).
 * Returns 0, or -1 if k is odd, < 2 or above 2*ORACLE_MAX_RADIUS.
 */
int oracle_fd_weights(int k, double *c) {
    if (k < 2 || (k % 2) != 0 || k > 2 * ORACLE_MAX_RADIUS) return -1;
    int r = k / 2;
    double sum = 0.0;
    for (int j = 1; j <= r; ++j) {
        /* (r!)^2 / ((r-j)! (r+j)!) = prod_{i=r-j+1..r} i / prod_{i=r+1..r+j} i */
        double num = 1.0, den = 1.0;
        for (int i = r - j + 1; i <= r; ++i) num *= (double)i;
        for (int i = r + 1; i <= r + j; ++i) den *= (double)i;
        double sign = (j % 2 == 1) ? 1.0 : -1.0;
        c[j] = 2.0 * sign * num / (den * (double)j * (double)j);
        sum += c[j];
    }
    c[0] = -2.0 * sum;
    return 0;
}

/* u at (x,y,z), zero outside the domain, or wrapped when periodic. */
static double sample(const double *u, long x, long y, long z, long nx, long ny, long nz,
                     int periodic) {
    if (periodic) {
        x = ((x % nx) + nx) % nx;
        y = ((y % ny) + ny) % ny;
        z = ((z % nz) + nz) % nz;
    } else if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) {
        return 0.0;
    }
    return u[idx3(x, y, z, ny, nz)];
}

/*
 * L u at every point: (1/h^2) sum over the three axes a of
 * sum_{j=-r..r} c_|j| u(p + j e_a)   (Listing 1's u.laplace; Listing 2 for k=2).
 */
int oracle_laplacian(const double *u, double *lap, long nx, long ny, long nz, int k, double h,
                     int periodic) {
    double c[ORACLE_MAX_RADIUS + 1];
    if (oracle_fd_weights(k, c) != 0) return -1;
    int r = k / 2;
    double inv_h2 = 1.0 / (h * h);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < nx; ++x)
        for (long y = 0; y < ny; ++y)
            for (long z = 0; z < nz; ++z) {
                double s = 0.0;
                for (int j = -r; j <= r; ++j) {
                    double w = c[j < 0 ? -j : j];
                    s += w * sample(u, x + j, y, z, nx, ny, nz, periodic);
                    s += w * sample(u, x, y + j, z, nx, ny, nz, periodic);
                    s += w * sample(u, x, y, z + j, nx, ny, nz, periodic);
                }
                lap[idx3(x, y, z, ny, nz)] = s * inv_h2;
            }
    return 0;
}

/*
 * One time step without sources: u_next from u (level n) and u_prev (level n-1),
 *   u_next = (dt^2 L u + m (2u - u_prev) + dt/2 eta u_prev) / (m + dt/2 eta),
 * the algebraic solution of the damped leapfrog equation above. eta may be NULL
 * (no damping). u_next must not alias u or u_prev.
 */
int oracle_step(const double *u, const double *u_prev, double *u_next, const double *m,
                const double *eta, long nx, long ny, long nz, int k, double h, double dt,
                int periodic) {
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    double *lap = (double *)malloc(n * sizeof(double));
    if (!lap) return -2;
    if (oracle_laplacian(u, lap, nx, ny, nz, k, h, periodic) != 0) {
        free(lap);
        return -1;
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)n; ++i) {
        double e = eta ? eta[i] : 0.0;
        double num = dt * dt * lap[i] + m[i] * (2.0 * u[i] - u_prev[i]) + 0.5 * dt * e * u_prev[i];
        u_next[i] = num / (m[i] + 0.5 * dt * e);
    }
    free(lap);
    return 0;
}

/*
 * Advance nt steps from global step step0 (Eq. 1 with sources, Sec. 2.1).
 * On entry u = u^{step0}, u_prev = u^{step0-1}; on return u = u^{step0+nt},
 * u_prev = u^{step0+nt-1}.
 * Sources: ns point sources at domain nodes (sx[s], sy[s], sz[s]); source s
 * contributes q = wavelet[s*ld + n] at step n (zero once n >= ld), entering the
 * equation as the right-hand side q at that node, i.e.
 *   u^{n+1}[s] += dt^2 q / (m[s] + dt/2 eta[s]).
 * Returns 0, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_forward(double *u, double *u_prev, const double *m, const double *eta, long nx,
                   long ny, long nz, int k, double h, double dt, int periodic, int ns,
                   const int *sx, const int *sy, const int *sz, const double *wavelet, long ld,
                   long step0, long nt) {
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    for (int s = 0; s < ns; ++s)
        if (sx[s] < 0 || sx[s] >= nx || sy[s] < 0 || sy[s] >= ny || sz[s] < 0 || sz[s] >= nz)
            return -1;
    double *next = (double *)malloc(n * sizeof(double));
    if (!next) return -2;
    for (long it = 0; it < nt; ++it) {
        long step = step0 + it;
        int rc = oracle_step(u, u_prev, next, m, eta, nx, ny, nz, k, h, dt, periodic);
        if (rc != 0) {
            free(next);
            return rc;
        }
        for (int s = 0; s < ns; ++s) {
            double q = (step >= 0 && step < ld) ? wavelet[(size_t)s * (size_t)ld + (size_t)step] : 0.0;
            size_t p = idx3(sx[s], sy[s], sz[s], ny, nz);
            double e = eta ? eta[p] : 0.0;
            next[p] += dt * dt * q / (m[p] + 0.5 * dt * e);
        }
        /* rotate levels: u_prev <- u, u <- next */
        memcpy(u_prev, u, n * sizeof(double));
        memcpy(u, next, n * sizeof(double));
    }
    free(next);
    return 0;
}

/*
 * Off-grid points (sources and receivers between nodes). The paper names
 * receivers and off-grid sources as the next step of the workflow (Sec. 5) but
 * gives no formula; the reading taken is multilinear (trilinear)
 * interpolation in the computational-domain index space, node (i, j, l) at
 * coordinates (i, j, l):
 *
 *   sampling:  v(p) = sum over the 8 nodes c of the cell holding p of W_c u[c],
 *   spreading: a source q at p adds W_c q to the right-hand side at node c,
 *   W_c = prod over axes a of (1 - |p_a - c_a|),
 *
 * so spreading is the adjoint (transpose) of sampling. The cell of a
 * coordinate t on an axis of n nodes is [i0, i0 + 1] with
 * i0 = min(floor(t), n - 2), so t = n - 1 lies in the last cell with weight 1 on
 * its upper node. Coordinates must lie in [0, n - 1] on every axis.
 *
 * Writes the 8 nodes (x, y, z triples, x slowest over the 2x2x2 corners) and
 * weights; returns 0, or -1 if the point lies outside the domain or an axis
 * has fewer than 2 nodes.
 */
int oracle_trilinear(double x, double y, double z, long nx, long ny, long nz, long *nodes,
                     double *w) {
    const double p[3] = {x, y, z};
    const long n[3] = {nx, ny, nz};
    long i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 2 || !(p[a] >= 0.0) || !(p[a] <= (double)(n[a] - 1))) return -1;
        long i = (long)floor(p[a]);
        if (i > n[a] - 2) i = n[a] - 2;
        i0[a] = i;
        f[a] = p[a] - (double)i;
    }
    int c = 0;
    for (int dx = 0; dx < 2; ++dx)
        for (int dy = 0; dy < 2; ++dy)
            for (int dz = 0; dz < 2; ++dz, ++c) {
                nodes[3 * c] = i0[0] + dx;
                nodes[3 * c + 1] = i0[1] + dy;
                nodes[3 * c + 2] = i0[2] + dz;
                w[c] = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
            }
    return 0;
}

/*
 * oracle_forward with off-grid sources and receivers. Source s sits at the
 * continuous domain coordinates src[3s..3s+2] and is spread onto its 8 nodes:
 *   u^{n+1}[c] += W_c dt^2 q / (m[c] + dt/2 eta[c]),  q = wavelet[s*ld + n];
 * receiver r at rec[3r..3r+2] records, after each step (sources included),
 *   traces[r*nt + it] = sum_c W_c u^{step0+it+1}[c].
 * Returns 0, -1 on bad arguments (a point outside the domain), -2 on
 * allocation failure.
 */
int oracle_forward_offgrid(double *u, double *u_prev, const double *m, const double *eta, long nx,
                           long ny, long nz, int k, double h, double dt, int periodic, int ns,
                           const double *src, const double *wavelet, long ld, int nr,
                           const double *rec, double *traces, long step0, long nt) {
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    long *snodes = (long *)malloc(sizeof(long) * 24 * (size_t)(ns > 0 ? ns : 1));
    double *sw = (double *)malloc(sizeof(double) * 8 * (size_t)(ns > 0 ? ns : 1));
    long *rnodes = (long *)malloc(sizeof(long) * 24 * (size_t)(nr > 0 ? nr : 1));
    double *rw = (double *)malloc(sizeof(double) * 8 * (size_t)(nr > 0 ? nr : 1));
    double *next = (double *)malloc(n * sizeof(double));
    int rc = 0;
    if (!snodes || !sw || !rnodes || !rw || !next) rc = -2;
    for (int s = 0; s < ns && rc == 0; ++s)
        if (oracle_trilinear(src[3 * s], src[3 * s + 1], src[3 * s + 2], nx, ny, nz, snodes + 24 * s,
                             sw + 8 * s) != 0)
            rc = -1;
    for (int r = 0; r < nr && rc == 0; ++r)
        if (oracle_trilinear(rec[3 * r], rec[3 * r + 1], rec[3 * r + 2], nx, ny, nz, rnodes + 24 * r,
                             rw + 8 * r) != 0)
            rc = -1;
    for (long it = 0; it < nt && rc == 0; ++it) {
        long step = step0 + it;
        rc = oracle_step(u, u_prev, next, m, eta, nx, ny, nz, k, h, dt, periodic);
        if (rc != 0) break;
        for (int s = 0; s < ns; ++s) {
            double q = (step >= 0 && step < ld) ? wavelet[(size_t)s * (size_t)ld + (size_t)step] : 0.0;
            for (int c = 0; c < 8; ++c) {
                const long *nd = snodes + 24 * s + 3 * c;
                size_t p = idx3(nd[0], nd[1], nd[2], ny, nz);
                double e = eta ? eta[p] : 0.0;
                next[p] += sw[8 * s + c] * dt * dt * q / (m[p] + 0.5 * dt * e);
            }
        }
        for (int r = 0; r < nr; ++r) {
            double v = 0.0;
            for (int c = 0; c < 8; ++c) {
                const long *nd = rnodes + 24 * r + 3 * c;
                v += rw[8 * r + c] * next[idx3(nd[0], nd[1], nd[2], ny, nz)];
            }
            traces[(size_t)r * (size_t)nt + (size_t)it] = v;
        }
        memcpy(u_prev, u, n * sizeof(double));
        memcpy(u, next, n * sizeof(double));
    }
    free(snodes);
    free(sw);
    free(rnodes);
    free(rw);
    free(next);
    return rc;
}

/*
 * Adjoint propagation and the FWI gradient (the paper's motivating workloads,
 * Sec. 1 and Sec. 5; not formulated there). The forward map of one shot is the
 * block lower-triangular system, for n = 0..nt-1 (u^0 = u^{-1} = 0),
 *   A u^{n+1} - (dt^2 L + 2M) u^n + (M - dt/2 E) u^{n-1} = dt^2 S q^n,
 *   A = M + dt/2 E (M = diag m, E = diag eta, S the source spreading),
 * with traces d^n = R u^{n+1} (R the receivers' sampling). L, M, E and A are
 * symmetric, so the transposed system is solved backward in time:
 *   A w^{n+1} = (dt^2 L + 2M) w^{n+2} - (M - dt/2 E) w^{n+3} + R^T r^n,
 * n = nt-1..0, w^{nt+1} = w^{nt+2} = 0, for the data-space vector r. For the
 * misfit J(m) = 1/2 sum_{r,n} (d^n - d_obs^n)^2, r = d - d_obs and, since only
 * the system matrix depends on m (dA/dm = dM/dm = I),
 *   dJ/dm = - sum_{n=0}^{nt-1} w^{n+1} * (u^{n+1} - 2u^n + u^{n-1})   (pointwise).
 * The adjoint of q -> d is (F^T r)^n = dt^2 S^T w^{n+1}.
 *
 * oracle_fwi_gradient: forward run keeping every level, traces, misfit, the
 * backward recursion written out as above, the gradient. src/rec: continuous
 * domain coordinates (trilinear spreading/sampling as oracle_forward_offgrid).
 * Outputs: grad[nx*ny*nz], syn[nr*nt] (synthetic traces), *misfit; adj_src
 * (if not NULL) receives (F^T d_obs)^n at each source, [ns*nt] (with r = d_obs).
 * Returns 0, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_fwi_gradient(const double *m, const double *eta, long nx, long ny, long nz, int k, double h,
                        double dt, int ns, const double *src, const double *wavelet, long ld, int nr,
                        const double *rec, const double *d_obs, long nt, double *grad, double *syn,
                        double *misfit, double *adj_src) {
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    if (nt < 1 || nr < 1) return -1;
    double *hist = (double *)calloc(n * (size_t)(nt + 2), sizeof(double)); /* u^{-1}, u^0, ..., u^nt */
    double *u = (double *)calloc(n, sizeof(double));
    double *up = (double *)calloc(n, sizeof(double));
    double *w1 = (double *)calloc(n, sizeof(double)); /* w^{j+1} */
    double *w2 = (double *)calloc(n, sizeof(double)); /* w^{j+2} */
    double *lap = (double *)malloc(n * sizeof(double));
    double *wn = (double *)malloc(n * sizeof(double));
    long *rnodes = (long *)malloc(sizeof(long) * 24 * (size_t)nr);
    double *rw = (double *)malloc(sizeof(double) * 8 * (size_t)nr);
    long *snodes = (long *)malloc(sizeof(long) * 24 * (size_t)(ns > 0 ? ns : 1));
    double *sw = (double *)malloc(sizeof(double) * 8 * (size_t)(ns > 0 ? ns : 1));
    int rc = 0;
    if (!hist || !u || !up || !w1 || !w2 || !lap || !wn || !rnodes || !rw || !snodes || !sw) rc = -2;
    for (int r = 0; r < nr && rc == 0; ++r)
        if (oracle_trilinear(rec[3 * r], rec[3 * r + 1], rec[3 * r + 2], nx, ny, nz, rnodes + 24 * r, rw + 8 * r))
            rc = -1;
    for (int s = 0; s < ns && rc == 0; ++s)
        if (oracle_trilinear(src[3 * s], src[3 * s + 1], src[3 * s + 2], nx, ny, nz, snodes + 24 * s, sw + 8 * s))
            rc = -1;
    /* forward one step at a time, every level kept: hist slot j + 1 holds u^j */
    for (long it = 0; it < nt && rc == 0; ++it) {
        rc = oracle_forward_offgrid(u, up, m, eta, nx, ny, nz, k, h, dt, 0, ns, src, wavelet, ld, 0, rec, NULL,
                                    it, 1);
        if (rc == 0) memcpy(hist + n * (size_t)(it + 2), u, n * sizeof(double));
    }
    /* traces d^n = R u^{n+1} and the misfit */
    double J = 0.0;
    for (int r = 0; r < nr && rc == 0; ++r)
        for (long it = 0; it < nt; ++it) {
            const double *un = hist + n * (size_t)(it + 2);
            double v = 0.0;
            for (int c = 0; c < 8; ++c) {
                const long *nd = rnodes + 24 * r + 3 * c;
                v += rw[8 * r + c] * un[idx3(nd[0], nd[1], nd[2], ny, nz)];
            }
            syn[(size_t)r * (size_t)nt + (size_t)it] = v;
            const double res = v - d_obs[(size_t)r * (size_t)nt + (size_t)it];
            J += 0.5 * res * res;
        }
    if (rc == 0) *misfit = J;
    /* backward recursion for r = syn - d_obs, and the gradient */
    if (rc == 0) {
        memset(grad, 0, n * sizeof(double));
        if (adj_src) memset(adj_src, 0, sizeof(double) * (size_t)(ns > 0 ? ns : 0) * (size_t)nt);
    }
    for (long it = nt - 1; it >= 0 && rc == 0; --it) {
        /* w^{it+1} from w1 = w^{it+2}, w2 = w^{it+3} */
        rc = oracle_laplacian(w1, lap, nx, ny, nz, k, h, 0);
        if (rc != 0) break;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)n; ++i) {
            double e = eta ? eta[i] : 0.0;
            wn[i] = dt * dt * lap[i] + 2.0 * m[i] * w1[i] - (m[i] - 0.5 * dt * e) * w2[i];
        }
        for (int r = 0; r < nr; ++r) {
            const double res = syn[(size_t)r * (size_t)nt + (size_t)it] - d_obs[(size_t)r * (size_t)nt + (size_t)it];
            for (int c = 0; c < 8; ++c) {
                const long *nd = rnodes + 24 * r + 3 * c;
                wn[idx3(nd[0], nd[1], nd[2], ny, nz)] += rw[8 * r + c] * res;
            }
        }
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)n; ++i) {
            double e = eta ? eta[i] : 0.0;
            wn[i] /= m[i] + 0.5 * dt * e;
        }
        /* gradient term n = it: - w^{it+1} (u^{it+1} - 2u^{it} + u^{it-1}) */
        const double *a = hist + n * (size_t)(it + 2), *b = hist + n * (size_t)(it + 1), *c0 = hist + n * (size_t)it;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)n; ++i) grad[i] -= wn[i] * (a[i] - 2.0 * b[i] + c0[i]);
        memcpy(w2, w1, n * sizeof(double));
        memcpy(w1, wn, n * sizeof(double));
    }
    /* adjoint of q -> d applied to d_obs: a second backward sweep with r = d_obs */
    if (rc == 0 && adj_src && ns > 0) {
        memset(w1, 0, n * sizeof(double));
        memset(w2, 0, n * sizeof(double));
        for (long it = nt - 1; it >= 0 && rc == 0; --it) {
            rc = oracle_laplacian(w1, lap, nx, ny, nz, k, h, 0);
            if (rc != 0) break;
#pragma omp parallel for schedule(static)
            for (long i = 0; i < (long)n; ++i) {
                double e = eta ? eta[i] : 0.0;
                wn[i] = dt * dt * lap[i] + 2.0 * m[i] * w1[i] - (m[i] - 0.5 * dt * e) * w2[i];
            }
            for (int r = 0; r < nr; ++r)
                for (int c = 0; c < 8; ++c) {
                    const long *nd = rnodes + 24 * r + 3 * c;
                    wn[idx3(nd[0], nd[1], nd[2], ny, nz)] += rw[8 * r + c] * d_obs[(size_t)r * (size_t)nt + (size_t)it];
                }
            for (long i = 0; i < (long)n; ++i) {
                double e = eta ? eta[i] : 0.0;
                wn[i] /= m[i] + 0.5 * dt * e;
            }
            for (int s = 0; s < ns; ++s) {
                double v = 0.0;
                for (int c = 0; c < 8; ++c) {
                    const long *nd = snodes + 24 * s + 3 * c;
                    v += sw[8 * s + c] * wn[idx3(nd[0], nd[1], nd[2], ny, nz)];
                }
                adj_src[(size_t)s * (size_t)nt + (size_t)it] = dt * dt * v;
            }
            memcpy(w2, w1, n * sizeof(double));
            memcpy(w1, wn, n * sizeof(double));
        }
    }
    free(hist);
    free(u);
    free(up);
    free(w1);
    free(w2);
    free(lap);
    free(wn);
    free(rnodes);
    free(rw);
    free(snodes);
    free(sw);
    return rc;
}

/*
 * Discrete energy between levels n and n+1 of the undamped, source-free scheme:
 *   E^{n+1/2} = sum m ((u^{n+1} - u^n)/dt)^2 - sum u^{n+1} (L u^n).
 * Multiplying the scheme by (u^{n+1} - u^{n-1}) and using the symmetry of L
 * shows E is invariant when eta = 0 and q = 0, and non-increasing when eta >= 0.
 * Returns NAN on bad arguments.
 */
double oracle_energy(const double *u_new, const double *u_old, const double *m, long nx, long ny,
                     long nz, int k, double h, double dt, int periodic) {
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    double *lap = (double *)malloc(n * sizeof(double));
    if (!lap) return NAN;
    if (oracle_laplacian(u_old, lap, nx, ny, nz, k, h, periodic) != 0) {
        free(lap);
        return NAN;
    }
    double kin = 0.0, pot = 0.0;
    for (size_t i = 0; i < n; ++i) {
        double d = (u_new[i] - u_old[i]) / dt;
        kin += m[i] * d * d;
        pot += u_new[i] * lap[i];
    }
    free(lap);
    return kin - pot;
}

/*
 * Largest stable dt of the 3D leapfrog scheme (von Neumann): the symbol of -L
 * peaks at the Nyquist mode with value 3 sum_{j=-r..r} |c_j| / h^2, and the
 * leapfrog is stable while dt^2 v^2 * peak <= 4, so
 *   dt_max = 2 h / (v_max sqrt(3 sum |c_j|)).
 * Returns -1 on bad arguments.
 */
double oracle_dt_max(int k, double h, double vmax) {
    double c[ORACLE_MAX_RADIUS + 1];
    if (h <= 0.0 || vmax <= 0.0 || oracle_fd_weights(k, c) != 0) return -1.0;
    double s = fabs(c[0]);
    for (int j = 1; j <= k / 2; ++j) s += 2.0 * fabs(c[j]);
    return 2.0 * h / (vmax * sqrt(3.0 * s));
}

/*
 * Default absorbing-layer damping (a convention: the paper names absorbing
 * boundaries, Sec. 4, but gives no profile):
 *   eta = m * d,   d = sum over axes of d_max (l_a / L)^2,
 * with l_a the depth into the layer along axis a in cells (0 in the interior,
 * nbl at the outermost node), L = nbl, and d_max = 3 v_max ln(1/R) / (2 nbl h),
 * R = 1e-3, v_max = 1 / sqrt(min m). nbl = 0 gives eta = 0.
 */
int oracle_default_damping(double *eta, const double *m, long nx, long ny, long nz, int nbl,
                           double h) {
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    if (nbl < 0 || h <= 0.0) return -1;
    if (nbl == 0) {
        for (size_t i = 0; i < n; ++i) eta[i] = 0.0;
        return 0;
    }
    double mmin = INFINITY;
    for (size_t i = 0; i < n; ++i) mmin = m[i] < mmin ? m[i] : mmin;
    double vmax = 1.0 / sqrt(mmin);
    double dmax = 3.0 * vmax * log(1.0 / 1e-3) / (2.0 * (double)nbl * h);
    long dims[3] = {nx, ny, nz};
    for (long x = 0; x < nx; ++x)
        for (long y = 0; y < ny; ++y)
            for (long z = 0; z < nz; ++z) {
                long pos[3] = {x, y, z};
                double d = 0.0;
                for (int a = 0; a < 3; ++a) {
                    long lo = nbl - pos[a];                    /* depth below the low side */
                    long hi = pos[a] - (dims[a] - 1 - nbl);    /* depth past the high side */
                    long depth = lo > hi ? lo : hi;
                    if (depth < 0) depth = 0;
                    double f = (double)depth / (double)nbl;
                    d += dmax * f * f;
                }
                size_t p = idx3(x, y, z, ny, nz);
                eta[p] = m[p] * d;
            }
    return 0;
}
