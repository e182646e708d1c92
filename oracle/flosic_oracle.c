/*
 * Plain FP64 CPU oracle for the real-space FLO-SIC orbital-SIC step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this
 * code; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * This file holds the grid-sized loops that are too slow in Python: the
 * finite-difference Laplacian, the multipole boundary values, the Poisson
 * solve by plain conjugate gradients, tricubic interpolation at the
 * Fermi-orbital descriptors (FODs), the grid gradient of the paper's force
 * scheme, and the pointwise fully polarised LSDA functional.  The small
 * dense algebra (Fermi orbitals, overlap, Loewdin) lives in flosic.py.
 *
 * Conventions (shared by every function here):
 *   - a grid is nx*ny*nz interior points r_ijk = origin + h*(i,j,k),
 *     0 <= i < nx etc.; element index g = (k*ny + j)*nx + i (x fastest);
 *   - orbitals (and every field that is not a potential) are zero at every
 *     point outside the interior (zero Dirichlet, Sec. II.A, M-SPARC);
 *   - integrals are dV * sum_g with dV = h^3 (trapezoid rule on a uniform
 *     grid whose end values vanish, Sec. II.A);
 *   - the multipole centre c is the box centre origin + h*(n-1)/2;
 *   - extended systems (the *_bc variants): a mask per, bit d set = periodic
 *     along direction d (x = bit 0), replaces the zero outside values along
 *     those directions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_M 6            /* half-width of the 12th-order stencil */
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Finite-difference weights (Sec. II.A: high-order centred FD).       */
/* ------------------------------------------------------------------ */

static double orc_fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* Centred second-derivative weights of order 2M on a unit grid:
 *   w_k = 2 (-1)^{k+1} (M!)^2 / (k^2 (M-k)! (M+k)!),  k = 1..M
 *   w_0 = -2 sum_{k=1}^{M} 1/k^2
 * so that u''(x) ~ (1/h^2) [w_0 u(x) + sum_k w_k (u(x+kh) + u(x-kh))]. */
void orc_fd_weights(int M, double* w) {
    double mf = orc_fact(M);
    double w0 = 0.0;
    for (int k = 1; k <= M; ++k) {
        double sgn = (k % 2 == 1) ? 1.0 : -1.0;
        w[k] = 2.0 * sgn * mf * mf /
               ((double)k * (double)k * orc_fact(M - k) * orc_fact(M + k));
        w0 -= 2.0 / ((double)k * (double)k);
    }
    w[0] = w0;
}

/* 3-D Laplacian Delta_h u at every interior point, with u = 0 outside
 * the interior.  out[g] = (1/h^2) sum_d [w_0 u_g + sum_k w_k (u_{g+k e_d} +
 * u_{g-k e_d})].  Plain loop with a bounds test on every tap. */
/* Delta_h u.  per: bit d set = periodic along direction d (taps wrap
 * around the box, Sec. II.A's conditions for extended directions); clear =
 * zero outside the interior. */
void orc_laplacian_bc(int nx, int ny, int nz, double h, int per, const double* u,
                      double* out) {
    double w[ORC_M + 1];
    orc_fd_weights(ORC_M, w);
    const double ih2 = 1.0 / (h * h);
    const int n[3] = {nx, ny, nz};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t g = ((int64_t)k * ny + j) * nx + i;
                int p[3] = {i, j, k};
                double acc = 3.0 * w[0] * u[g];
                for (int d = 0; d < 3; ++d)
                    for (int m = 1; m <= ORC_M; ++m)
                        for (int s = -1; s <= 1; s += 2) {
                            int q[3] = {p[0], p[1], p[2]};
                            q[d] += s * m;
                            if (q[d] < 0 || q[d] >= n[d]) {
                                if (!((per >> d) & 1)) continue;
                                q[d] = ((q[d] % n[d]) + n[d]) % n[d];
                            }
                            int64_t gq = ((int64_t)q[2] * ny + q[1]) * nx + q[0];
                            acc += w[m] * u[gq];
                        }
                out[g] = acc * ih2;
            }
}

/* Delta_h u with zero values outside the interior (isolated systems). */
void orc_laplacian(int nx, int ny, int nz, double h, const double* u,
                   double* out) {
    orc_laplacian_bc(nx, ny, nz, h, 0, u, out);
}

/* ------------------------------------------------------------------ */
/* Multipole boundary values (Sec. II.A: Dirichlet values of the        */
/* electrostatic potential from a multipole expansion, isolated case).  */
/* ------------------------------------------------------------------ */

/* Moments about c, l <= 2, of a density on the grid:
 *   mom[0]   = Q  = dV sum rho
 *   mom[1..3]= p  = dV sum rho R
 *   mom[4..9]= Theta_{xx,yy,zz,xy,xz,yz} = dV sum rho (3 R_j R_k - |R|^2 d_jk)
 * with R = r - c. */
void orc_multipole_moments(int nx, int ny, int nz, double h,
                           const double* origin, const double* rho,
                           double* mom) {
    double c[3] = {origin[0] + 0.5 * h * (nx - 1), origin[1] + 0.5 * h * (ny - 1),
                   origin[2] + 0.5 * h * (nz - 1)};
    double dV = h * h * h;
    for (int m = 0; m < 10; ++m) mom[m] = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t g = ((int64_t)k * ny + j) * nx + i;
                double q = rho[g] * dV;
                double R[3] = {origin[0] + h * i - c[0], origin[1] + h * j - c[1],
                               origin[2] + h * k - c[2]};
                double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
                mom[0] += q;
                mom[1] += q * R[0];
                mom[2] += q * R[1];
                mom[3] += q * R[2];
                mom[4] += q * (3.0 * R[0] * R[0] - r2);
                mom[5] += q * (3.0 * R[1] * R[1] - r2);
                mom[6] += q * (3.0 * R[2] * R[2] - r2);
                mom[7] += q * 3.0 * R[0] * R[1];
                mom[8] += q * 3.0 * R[0] * R[2];
                mom[9] += q * 3.0 * R[1] * R[2];
            }
}

/* Multipole potential at offset R from c:
 *   V_b = Q/|R| + p.R/|R|^3 + (1/2) sum_jk Theta_jk R_j R_k / |R|^5. */
double orc_multipole_value(const double* mom, const double* R) {
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    double r = sqrt(r2);
    double r3 = r2 * r, r5 = r3 * r2;
    double v = mom[0] / r;
    v += (mom[1] * R[0] + mom[2] * R[1] + mom[3] * R[2]) / r3;
    double quad = mom[4] * R[0] * R[0] + mom[5] * R[1] * R[1] + mom[6] * R[2] * R[2] +
                  2.0 * (mom[7] * R[0] * R[1] + mom[8] * R[0] * R[2] + mom[9] * R[1] * R[2]);
    v += 0.5 * quad / r5;
    return v;
}

/* Boundary part of the Poisson right-hand side.  -Delta_h V = 4 pi rho at
 * interior points with V = V_b on the ghost points (up to 6 layers outside
 * the interior) becomes A V = 4 pi rho + bc, A = -Delta_h with zero ghosts,
 * bc[g] = (1/h^2) sum over the taps of g that land outside of w_m V_b. */
void orc_bc_rhs(int nx, int ny, int nz, double h, const double* origin,
                const double* mom, double* bc) {
    double w[ORC_M + 1];
    orc_fd_weights(ORC_M, w);
    double c[3] = {origin[0] + 0.5 * h * (nx - 1), origin[1] + 0.5 * h * (ny - 1),
                   origin[2] + 0.5 * h * (nz - 1)};
    const int n[3] = {nx, ny, nz};
    const double ih2 = 1.0 / (h * h);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t g = ((int64_t)k * ny + j) * nx + i;
                int p[3] = {i, j, k};
                double acc = 0.0;
                for (int d = 0; d < 3; ++d)
                    for (int m = 1; m <= ORC_M; ++m)
                        for (int s = -1; s <= 1; s += 2) {
                            int q[3] = {p[0], p[1], p[2]};
                            q[d] += s * m;
                            if (q[d] >= 0 && q[d] < n[d]) continue;
                            double R[3] = {origin[0] + h * q[0] - c[0],
                                           origin[1] + h * q[1] - c[1],
                                           origin[2] + h * q[2] - c[2]};
                            acc += w[m] * orc_multipole_value(mom, R);
                        }
                bc[g] = acc * ih2;
            }
}

/* Adjoint of the linear map rho -> bc (moments, then boundary values, then
 * the ghost taps): out = M^T C^T y, where C^T y collects, for each moment,
 * sum_g y_g (1/h^2) sum_ghost-taps w_m basis(R_tap), and M^T spreads the ten
 * coefficients back over the grid with the moment weights dV*{1, R, 3RR-R^2}.
 * Used only for the exact (non-self-adjoint) Poisson adjoint. */
void orc_bc_rhs_adjoint(int nx, int ny, int nz, double h, const double* origin,
                        const double* y, double* out) {
    double w[ORC_M + 1];
    orc_fd_weights(ORC_M, w);
    double c[3] = {origin[0] + 0.5 * h * (nx - 1), origin[1] + 0.5 * h * (ny - 1),
                   origin[2] + 0.5 * h * (nz - 1)};
    const int n[3] = {nx, ny, nz};
    const double ih2 = 1.0 / (h * h);
    double coef[10];
    for (int m = 0; m < 10; ++m) coef[m] = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t g = ((int64_t)k * ny + j) * nx + i;
                int p[3] = {i, j, k};
                for (int d = 0; d < 3; ++d)
                    for (int m = 1; m <= ORC_M; ++m)
                        for (int s = -1; s <= 1; s += 2) {
                            int q[3] = {p[0], p[1], p[2]};
                            q[d] += s * m;
                            if (q[d] >= 0 && q[d] < n[d]) continue;
                            double R[3] = {origin[0] + h * q[0] - c[0],
                                           origin[1] + h * q[1] - c[1],
                                           origin[2] + h * q[2] - c[2]};
                            /* d V_b / d mom_m at R, one unit moment at a time */
                            for (int mm = 0; mm < 10; ++mm) {
                                double e[10] = {0};
                                e[mm] = 1.0;
                                coef[mm] += y[g] * ih2 * w[m] * orc_multipole_value(e, R);
                            }
                        }
            }
    double dV = h * h * h;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t g = ((int64_t)k * ny + j) * nx + i;
                double R[3] = {origin[0] + h * i - c[0], origin[1] + h * j - c[1],
                               origin[2] + h * k - c[2]};
                double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
                double basis[10] = {1.0, R[0], R[1], R[2],
                                    3.0 * R[0] * R[0] - r2, 3.0 * R[1] * R[1] - r2,
                                    3.0 * R[2] * R[2] - r2, 3.0 * R[0] * R[1],
                                    3.0 * R[0] * R[2], 3.0 * R[1] * R[2]};
                double acc = 0.0;
                for (int m = 0; m < 10; ++m) acc += coef[m] * basis[m];
                out[g] = dV * acc;
            }
}

/* ------------------------------------------------------------------ */
/* Poisson solve (Sec. II.A: electrostatics from a Poisson equation).   */
/* ------------------------------------------------------------------ */

static double orc_dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Plain (unpreconditioned) conjugate gradients on A x = b, A = -Delta_h
 * with the boundary mask per of orc_laplacian_bc (zero ghosts along the
 * other directions).  A is symmetric positive definite, or, when every
 * direction is periodic, semidefinite with the constants as null space; b
 * must then have zero sum, and from a zero-sum start every iterate keeps a
 * zero sum (the minimum-norm solution).  x holds the start vector on entry
 * and the solution on exit.  Stops when ||r|| <= tol ||b||.  Returns the
 * iteration count, or -1 if max_iter was reached first. */
int orc_cg_bc(int nx, int ny, int nz, double h, int per, const double* b, double* x,
              double tol, int max_iter) {
    int64_t G = (int64_t)nx * ny * nz;
    double* r = (double*)malloc(sizeof(double) * G);
    double* p = (double*)malloc(sizeof(double) * G);
    double* q = (double*)malloc(sizeof(double) * G);
    orc_laplacian_bc(nx, ny, nz, h, per, x, q);
    for (int64_t g = 0; g < G; ++g) {
        r[g] = b[g] + q[g];  /* b - A x = b + Delta_h x */
        p[g] = r[g];
    }
    double bb = orc_dot(G, b, b);
    double rr = orc_dot(G, r, r);
    int it = 0, result = -1;
    if (bb == 0.0) {
        for (int64_t g = 0; g < G; ++g) x[g] = 0.0;
        result = 0;
    }
    while (result < 0) {
        if (rr <= tol * tol * bb) { result = it; break; }
        if (it >= max_iter) break;
        orc_laplacian_bc(nx, ny, nz, h, per, p, q);
        for (int64_t g = 0; g < G; ++g) q[g] = -q[g];  /* q = A p */
        double alpha = rr / orc_dot(G, p, q);
        for (int64_t g = 0; g < G; ++g) {
            x[g] += alpha * p[g];
            r[g] -= alpha * q[g];
        }
        double rr_new = orc_dot(G, r, r);
        double beta = rr_new / rr;
        rr = rr_new;
        for (int64_t g = 0; g < G; ++g) p[g] = r[g] + beta * p[g];
        ++it;
    }
    free(r);
    free(p);
    free(q);
    return result;
}

/* Conjugate gradients with zero ghosts in every direction. */
int orc_cg(int nx, int ny, int nz, double h, const double* b, double* x,
           double tol, int max_iter) {
    return orc_cg_bc(nx, ny, nz, h, 0, b, x, tol, max_iter);
}

/* One orbital: solve -Delta_h V = 4 pi rho with multipole (l <= 2) Dirichlet
 * values on the ghost shell.  V must hold the start vector (zeros, or a warm
 * start).  Returns the CG iteration count (-1 if not converged). */
int orc_poisson(int nx, int ny, int nz, double h, const double* origin,
                const double* rho, double* V, double tol, int max_iter) {
    int64_t G = (int64_t)nx * ny * nz;
    double mom[10];
    orc_multipole_moments(nx, ny, nz, h, origin, rho, mom);
    double* b = (double*)malloc(sizeof(double) * G);
    orc_bc_rhs(nx, ny, nz, h, origin, mom, b);
    for (int64_t g = 0; g < G; ++g) b[g] += 4.0 * ORC_PI * rho[g];
    int it = orc_cg(nx, ny, nz, h, b, V, tol, max_iter);
    free(b);
    return it;
}

/* Many orbitals on one grid, independent problems; parallel over orbitals
 * when built with OpenMP.  rho and V are [norb][G]. */
void orc_poisson_batch(int norb, int nx, int ny, int nz, double h,
                       const double* origin, const double* rho, double* V,
                       double tol, int max_iter, int* iters) {
    int64_t G = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1)
    for (int o = 0; o < norb; ++o)
        iters[o] = orc_poisson(nx, ny, nz, h, origin, rho + (int64_t)o * G,
                               V + (int64_t)o * G, tol, max_iter);
}

/* Zero-boundary solves A x = b for many right-hand sides ([nrhs][G]). */
void orc_cg_batch(int nrhs, int nx, int ny, int nz, double h, const double* b,
                  double* x, double tol, int max_iter, int* iters) {
    int64_t G = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1)
    for (int o = 0; o < nrhs; ++o)
        iters[o] = orc_cg(nx, ny, nz, h, b + (int64_t)o * G, x + (int64_t)o * G,
                          tol, max_iter);
}

/* Solves A x = b (A with boundary mask per) for many right-hand sides. */
void orc_cg_batch_bc(int nrhs, int nx, int ny, int nz, double h, int per,
                     const double* b, double* x, double tol, int max_iter,
                     int* iters) {
    int64_t G = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1)
    for (int o = 0; o < nrhs; ++o)
        iters[o] = orc_cg_bc(nx, ny, nz, h, per, b + (int64_t)o * G,
                             x + (int64_t)o * G, tol, max_iter);
}

/* Slab (periodic along x and y, finite along z; Sec. II.A: Dirichlet values
 * from a dipole correction for surfaces).  The ghost planes along z carry
 * the potential of the planar average of rho, which depends on its charge Q
 * and dipole p_z = sum rho (z - c_z) dV only:
 *   V_b(z) = -(2 pi / A) (Q |z - c_z| - sgn(z - c_z) p_z),  A = nx ny h^2,
 * i.e. the 1-D field of charged sheets, -2 pi |z - z'| / A per unit charge.
 * Adds (1/h^2) sum over the z-taps of g that leave the box of w_m V_b to
 * out[g] (points within 6 planes of a z face). */
void orc_slab_bc_rhs(int nx, int ny, int nz, double h, const double* origin,
                     double Q, double pz, double* out) {
    double w[ORC_M + 1];
    orc_fd_weights(ORC_M, w);
    const double ih2 = 1.0 / (h * h);
    const double area = (double)nx * ny * h * h;
    const double cz = origin[2] + 0.5 * h * (nz - 1);
    for (int k = 0; k < nz; ++k) {
        double acc = 0.0;
        for (int m = 1; m <= ORC_M; ++m)
            for (int s = -1; s <= 1; s += 2) {
                int q = k + s * m;
                if (q >= 0 && q < nz) continue;
                double Z = origin[2] + h * q - cz;
                double sg = (Z > 0.0) ? 1.0 : -1.0;
                acc += w[m] * (-2.0 * ORC_PI / area) * (Q * fabs(Z) - sg * pz);
            }
        if (acc == 0.0) continue;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) out[((int64_t)k * ny + j) * nx + i] += acc * ih2;
    }
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Cubic interpolation at FODs (Sec. II.B).                            */
/* ------------------------------------------------------------------ */

/* 4-point Lagrange basis on nodes -1,0,1,2 at t in [0,1), and d/dt. */
static void orc_lagrange4(double t, double* L, double* dL) {
    double n[4] = {-1.0, 0.0, 1.0, 2.0};
    for (int a = 0; a < 4; ++a) {
        double num = 1.0, den = 1.0;
        for (int b = 0; b < 4; ++b) {
            if (b == a) continue;
            num *= (t - n[b]);
            den *= (n[a] - n[b]);
        }
        L[a] = num / den;
        /* derivative: sum over the dropped factor */
        double d = 0.0;
        for (int c = 0; c < 4; ++c) {
            if (c == a) continue;
            double prod = 1.0;
            for (int b = 0; b < 4; ++b) {
                if (b == a || b == c) continue;
                prod *= (t - n[b]);
            }
            d += prod;
        }
        dL[a] = d / den;
    }
}

/* Locate the cell of coordinate u (grid units): i0 = floor(u), t = u - i0.
 * Along a periodic direction of n points u is first reduced to [0, n). */
static void orc_cell(double u, int n, int periodic, int* i0, double* t) {
    if (periodic) u -= n * floor(u / n);
    double f = floor(u);
    *i0 = (int)f;
    *t = u - f;
}

/* Node index q along a direction of n points: wrapped when periodic, else
 * -1 when outside (the node counts as zero). */
static int orc_node(int q, int n, int periodic) {
    if (q >= 0 && q < n) return q;
    if (!periodic) return -1;
    return ((q % n) + n) % n;
}

/* Tricubic tensor-product Lagrange interpolant of nfield fields ([nfield][G])
 * at point a: val[f] and grad[f][3] (exact derivative of the interpolant, in
 * 1/bohr).  Along a direction whose bit of per is set the field is periodic
 * (nodes wrap); along the others nodes outside the interior count as zero. */
void orc_interp_bc(int nx, int ny, int nz, double h, const double* origin, int per,
                   int nfield, const double* u, const double* a, double* val,
                   double* grad) {
    int64_t G = (int64_t)nx * ny * nz;
    int i0[3];
    double t[3], L[3][4], dL[3][4];
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        orc_cell((a[d] - origin[d]) / h, n[d], (per >> d) & 1, &i0[d], &t[d]);
        orc_lagrange4(t[d], L[d], dL[d]);
    }
    for (int f = 0; f < nfield; ++f) {
        double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b)
                for (int e = 0; e < 4; ++e) {
                    int q[3] = {i0[0] - 1 + e, i0[1] - 1 + b, i0[2] - 1 + c};
                    int skip = 0;
                    for (int d = 0; d < 3; ++d) {
                        q[d] = orc_node(q[d], n[d], (per >> d) & 1);
                        if (q[d] < 0) skip = 1;
                    }
                    if (skip) continue;
                    double uv = u[(int64_t)f * G + ((int64_t)q[2] * ny + q[1]) * nx + q[0]];
                    v += L[0][e] * L[1][b] * L[2][c] * uv;
                    gx += dL[0][e] * L[1][b] * L[2][c] * uv;
                    gy += L[0][e] * dL[1][b] * L[2][c] * uv;
                    gz += L[0][e] * L[1][b] * dL[2][c] * uv;
                }
        val[f] = v;
        if (grad) {
            grad[3 * f + 0] = gx / h;
            grad[3 * f + 1] = gy / h;
            grad[3 * f + 2] = gz / h;
        }
    }
}

void orc_interp(int nx, int ny, int nz, double h, const double* origin,
                int nfield, const double* u, const double* a, double* val,
                double* grad) {
    orc_interp_bc(nx, ny, nz, h, origin, 0, nfield, u, a, val, grad);
}

/* Adjoint of orc_interp_bc's value map for one field: out[node] += coef *
 * weight(node) over the 64 nodes of the cell of a (wrapped along periodic
 * directions, skipped outside along the others). */
void orc_interp_scatter_bc(int nx, int ny, int nz, double h, const double* origin, int per,
                           const double* a, double coef, double* out) {
    int i0[3];
    double t[3], L[3][4], dL[3][4];
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        orc_cell((a[d] - origin[d]) / h, n[d], (per >> d) & 1, &i0[d], &t[d]);
        orc_lagrange4(t[d], L[d], dL[d]);
    }
    for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b)
            for (int e = 0; e < 4; ++e) {
                int q[3] = {i0[0] - 1 + e, i0[1] - 1 + b, i0[2] - 1 + c};
                int skip = 0;
                for (int d = 0; d < 3; ++d) {
                    q[d] = orc_node(q[d], n[d], (per >> d) & 1);
                    if (q[d] < 0) skip = 1;
                }
                if (skip) continue;
                out[((int64_t)q[2] * ny + q[1]) * nx + q[0]] +=
                    coef * L[0][e] * L[1][b] * L[2][c];
            }
}

void orc_interp_scatter(int nx, int ny, int nz, double h, const double* origin,
                        const double* a, double coef, double* out) {
    orc_interp_scatter_bc(nx, ny, nz, h, origin, 0, a, coef, out);
}

/* Grid gradient of the paper's force scheme (Sec. II.B): central difference
 * (u_{+1} - u_{-1})/(2h) at inner points, forward (u_1 - u_0)/h at the first
 * point and backward (u_{n-1} - u_{n-2})/h at the last point of each line.
 * out is [3][G]. */
void orc_grad_central(int nx, int ny, int nz, double h, const double* u,
                      double* out) {
    int64_t G = (int64_t)nx * ny * nz;
    const int n[3] = {nx, ny, nz};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t g = ((int64_t)k * ny + j) * nx + i;
                int p[3] = {i, j, k};
                int64_t stride[3] = {1, nx, (int64_t)nx * ny};
                for (int d = 0; d < 3; ++d) {
                    double v;
                    if (n[d] == 1) v = 0.0;
                    else if (p[d] == 0) v = (u[g + stride[d]] - u[g]) / h;
                    else if (p[d] == n[d] - 1) v = (u[g] - u[g - stride[d]]) / h;
                    else v = (u[g + stride[d]] - u[g - stride[d]]) / (2.0 * h);
                    out[(int64_t)d * G + g] = v;
                }
            }
}

/* ------------------------------------------------------------------ */
/* Fully polarised LSDA (Eq. 1 uses E_xc[rho_i, 0]; Sec. III: LSDA      */
/* exchange + PW92 correlation).                                        */
/* ------------------------------------------------------------------ */

/* PW92 correlation of the fully polarised gas (zeta = 1), where the spin
 * interpolation reduces exactly to the ferromagnetic fit
 *   G(rs) = -2A(1 + a1 rs) ln[1 + 1/(2A(b1 rs^1/2 + b2 rs + b3 rs^3/2 + b4 rs^2))]
 * Constants: the epsilon_c(rs, zeta=1) fit parameters of Perdew & Wang,
 * Phys. Rev. B 45, 13244 (1992); A is the tabulated 0.015545, not the exact
 * high-density coefficient (1 - ln 2)/(2 pi^2) = 0.0155454... */
#define PW92_A 0.015545
#define PW92_A1 0.20548
#define PW92_B1 14.1189
#define PW92_B2 6.1977
#define PW92_B3 3.3662
#define PW92_B4 0.62517

void orc_pw92_ferro(double rs, double* ec, double* dec_drs) {
    double s = sqrt(rs);
    double q0 = -2.0 * PW92_A * (1.0 + PW92_A1 * rs);
    double q1 = 2.0 * PW92_A * (PW92_B1 * s + PW92_B2 * rs + PW92_B3 * rs * s +
                                PW92_B4 * rs * rs);
    double dq1 = PW92_A * (PW92_B1 / s + 2.0 * PW92_B2 + 3.0 * PW92_B3 * s +
                           4.0 * PW92_B4 * rs);
    double lg = log(1.0 + 1.0 / q1);
    *ec = q0 * lg;
    *dec_drs = -2.0 * PW92_A * PW92_A1 * lg - q0 * dq1 / (q1 * q1 + q1);
}

/* Energy per particle eps_xc and potential v_xc of the up channel for the
 * spin densities (n, 0).  Exchange by spin scaling of the Slater/Dirac form:
 *   eps_x = -(3/4)(6 n/pi)^{1/3},  v_x = -(6 n/pi)^{1/3}.
 * Correlation: v_c = eps_c - (rs/3) d eps_c/d rs (the zeta term vanishes at
 * zeta = 1).  Below rho_min both are zero. */
void orc_lsda_pol(double n, double rho_min, double* eps, double* v) {
    if (!(n > rho_min)) {
        *eps = 0.0;
        *v = 0.0;
        return;
    }
    double kx = cbrt(6.0 * n / ORC_PI);
    double ex = -0.75 * kx;
    double vx = -kx;
    double rs = cbrt(3.0 / (4.0 * ORC_PI * n));
    double ec, dec;
    orc_pw92_ferro(rs, &ec, &dec);
    double vc = ec - rs / 3.0 * dec;
    *eps = ex + ec;
    *v = vx + vc;
}

/* The same pointwise over G values; eps_x and eps_c split out for tests. */
void orc_lsda_pol_grid(int64_t G, const double* n, double rho_min, double* eps,
                       double* v) {
    for (int64_t g = 0; g < G; ++g) orc_lsda_pol(n[g], rho_min, &eps[g], &v[g]);
}
