/*
 * FP64 CPU oracle for the conservative diffuse interface (CDI) phase-field
 * step of Mirjalili, Ivey & Mani (arXiv 1803.01262).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg load this code.  It shares nothing with the CUDA
 * library: no headers, no helpers, no constants.
 *
 * It is deliberately plain: whole-array passes with nested loops over
 * periodic indices, one pass per step of the paper's recipe (Section 2.2):
 *   1. normal vectors at cell centres from central differences,
 *   2. sharpening term phi(1-phi) n at cell centres, then averaged onto faces,
 *   3. diffusive flux on faces,
 *   4. advective flux on faces with phi averaged onto the face,
 *   5. flux divergence and explicit Euler update (Eq. 11 in 1D).
 * Flux on the face between cells L and R along axis d (the conservative form
 * of Eq. 1, whose right-hand side is div[gamma(eps grad phi - phi(1-phi) n)]):
 *   F = u_f (phi_L + phi_R)/2 - gamma eps (phi_R - phi_L)/dx
 *       + gamma (s_L + s_R)/2,          s = phi (1 - phi) n_d.
 *   phi^{k+1}_c = phi^k_c + dt * ( -(1/dx) sum_d (F_{c+1/2} - F_{c-1/2}) ).
 * Readings of the paper taken here:
 *   - the sign in the sharpening term of Eq. 11 is read as
 *     ((phi_{i-1})^2 - phi_{i-1}) n_{i-1}, as Eq. 13 and Eq. 16 require;
 *   - the normal is 0 where the central-difference gradient is exactly 0
 *     (the paper divides by |grad phi| without a guard);
 *   - a non-default face-product sharpening (oracle_rhs_face / oracle_step_face):
 *     the flux term gamma phi_f (1 - phi_f) n_f with phi_f = (phi_L + phi_R)/2
 *     and n_f = (n_L + n_R)/2, the cell-centre normals interpolated to the
 *     face; Eq. 13 and Eq. 19 do not hold for it (Section 2.2 forms the
 *     product at cell centres), and the boundedness proof does not cover it;
 *   - every entry point takes a floor tiny >= 0 under the root,
 *     n = g / sqrt(|g|^2 + tiny) for g != 0: tiny = 0 is the paper's
 *     unit normal, tiny = the smallest normal number of a working precision
 *     is the regularised normal a finite-precision step divides by (it only
 *     matters where |g|^2 falls to that number);
 *   - the 1/(2dx) of the central gradient cancels in n = g/|g|, so g is the
 *     plain difference phi_{c+e} - phi_{c-e};
 *   - velocities are face values u[k][j][i] = u_{i+1/2,j,k} (right face),
 *     multiplied by vel_scale (the time factor of a time-periodic field).
 *
 * The discrete adjoint (oracle_adjoint) is the reverse-mode derivative of
 * exactly these passes, taken in reverse order.
 *
 * Layout: arrays are [k][j][i] with i fastest, n = nx*ny*nz, periodic.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_API __attribute__((visibility("default")))

static long wrap(long a, long n) { long r = a % n; return r < 0 ? r + n : r; }

static long at(long i, long j, long k, long nx, long ny, long nz)
{
    return (wrap(k, nz) * ny + wrap(j, ny)) * nx + wrap(i, nx);
}

/* Index of the neighbour of cell (i,j,k) displaced by s along axis d. */
static long nb(long i, long j, long k, int d, long s, long nx, long ny, long nz)
{
    if (d == 0) return at(i + s, j, k, nx, ny, nz);
    if (d == 1) return at(i, j + s, k, nx, ny, nz);
    return at(i, j, k + s, nx, ny, nz);
}

/* Step 1: cell-centre normals n = g/m, m = sqrt(|g|^2 + tiny),
 * g_d = phi_{c+e_d} - phi_{c-e_d}; n = 0 where g = 0.  Also returns m (needed
 * by the adjoint; 0 where g = 0). */
static void normals(long nx, long ny, long nz, const double *phi, double tiny,
                    double *n0, double *n1, double *n2, double *gmag)
{
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                long c = at(i, j, k, nx, ny, nz);
                double g[3];
                for (int d = 0; d < 3; d++)
                    g[d] = phi[nb(i, j, k, d, +1, nx, ny, nz)] - phi[nb(i, j, k, d, -1, nx, ny, nz)];
                double g2 = g[0] * g[0];
                g2 = g2 + g[1] * g[1];
                g2 = g2 + g[2] * g[2];
                double m = g2 > 0.0 ? sqrt(g2 + tiny) : 0.0;
                gmag[c] = m;
                if (m > 0.0) {
                    n0[c] = g[0] / m; n1[c] = g[1] / m; n2[c] = g[2] / m;
                } else {
                    n0[c] = 0.0; n1[c] = 0.0; n2[c] = 0.0;
                }
            }
}

/* Steps 1-4: face fluxes F_d[c] on the face c + 1/2 e_d for every cell c. */
static void face_fluxes(long nx, long ny, long nz, double dx, const double *phi,
                        const double *u, const double *v, const double *w,
                        double eps, double gamma, double vel_scale, double tiny, int face,
                        double *F0, double *F1, double *F2)
{
    long n = nx * ny * nz;
    double *nrm[3], *s[3], *gm;
    for (int d = 0; d < 3; d++) {
        nrm[d] = (double *)malloc(sizeof(double) * n);
        s[d] = (double *)malloc(sizeof(double) * n);
    }
    gm = (double *)malloc(sizeof(double) * n);
    normals(nx, ny, nz, phi, tiny, nrm[0], nrm[1], nrm[2], gm);

    /* Step 2a: sharpening term at cell centres. */
    for (long c = 0; c < n; c++)
        for (int d = 0; d < 3; d++)
            s[d][c] = phi[c] * (1.0 - phi[c]) * nrm[d][c];

    const double *vel[3] = {u, v, w};
    double *F[3] = {F0, F1, F2};
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                long L = at(i, j, k, nx, ny, nz);
                for (int d = 0; d < 3; d++) {
                    long R = nb(i, j, k, d, +1, nx, ny, nz);
                    /* Step 2b: sharpening interpolated (averaged) to the face; or, in
                     * the face-product form, phi_f (1 - phi_f) times the averaged normal. */
                    double sharp_f;
                    if (face) {
                        double pf = 0.5 * (phi[L] + phi[R]);
                        sharp_f = pf * (1.0 - pf) * 0.5 * (nrm[d][L] + nrm[d][R]);
                    } else {
                        sharp_f = 0.5 * (s[d][L] + s[d][R]);
                    }
                    /* Step 3: diffusive flux, eps * dphi/dx on the face. */
                    double diff_f = eps * (phi[R] - phi[L]) / dx;
                    /* Step 4: advective flux, u_f times phi averaged to the face. */
                    double phi_f = 0.5 * (phi[L] + phi[R]);
                    double adv_f = (vel_scale * vel[d][L]) * phi_f;
                    F[d][L] = adv_f - gamma * (diff_f - sharp_f);
                }
            }
    for (int d = 0; d < 3; d++) { free(nrm[d]); free(s[d]); }
    free(gm);
}

/* d phi / dt = -(1/dx) sum_d (F_{c+1/2 e_d} - F_{c-1/2 e_d})  (Step 5, divergence). */
static int rhs_impl(int nx, int ny, int nz, double dx, const double *phi,
                    const double *u, const double *v, const double *w,
                    double eps, double gamma, double vel_scale, double tiny, int face,
                    double *rhs)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0.0) || !(tiny >= 0.0)) return -1;
    long n = (long)nx * ny * nz;
    double *F[3];
    for (int d = 0; d < 3; d++) F[d] = (double *)malloc(sizeof(double) * n);
    face_fluxes(nx, ny, nz, dx, phi, u, v, w, eps, gamma, vel_scale, tiny, face, F[0], F[1], F[2]);
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                long c = at(i, j, k, nx, ny, nz);
                double div = 0.0;
                for (int d = 0; d < 3; d++)
                    div += F[d][c] - F[d][nb(i, j, k, d, -1, nx, ny, nz)];
                rhs[c] = -div / dx;
            }
    for (int d = 0; d < 3; d++) free(F[d]);
    return 0;
}

ORACLE_API int oracle_rhs(int nx, int ny, int nz, double dx, const double *phi,
                          const double *u, const double *v, const double *w,
                          double eps, double gamma, double vel_scale, double tiny,
                          double *rhs)
{
    return rhs_impl(nx, ny, nz, dx, phi, u, v, w, eps, gamma, vel_scale, tiny, 0, rhs);
}

ORACLE_API int oracle_rhs_face(int nx, int ny, int nz, double dx, const double *phi,
                               const double *u, const double *v, const double *w,
                               double eps, double gamma, double vel_scale, double tiny,
                               double *rhs)
{
    return rhs_impl(nx, ny, nz, dx, phi, u, v, w, eps, gamma, vel_scale, tiny, 1, rhs);
}

/* One explicit Euler step phi_out = phi + dt * rhs(phi)  (Eq. 11, Step 5). */
static int step_impl(int nx, int ny, int nz, double dx, const double *phi,
                     const double *u, const double *v, const double *w,
                     double dt, double eps, double gamma, double vel_scale,
                     double tiny, int face, double *phi_out)
{
    long n = (long)nx * ny * nz;
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    double *r = (double *)malloc(sizeof(double) * n);
    int rc = rhs_impl(nx, ny, nz, dx, phi, u, v, w, eps, gamma, vel_scale, tiny, face, r);
    if (rc == 0)
        for (long c = 0; c < n; c++) phi_out[c] = phi[c] + dt * r[c];
    free(r);
    return rc;
}

ORACLE_API int oracle_step(int nx, int ny, int nz, double dx, const double *phi,
                           const double *u, const double *v, const double *w,
                           double dt, double eps, double gamma, double vel_scale,
                           double tiny, double *phi_out)
{
    return step_impl(nx, ny, nz, dx, phi, u, v, w, dt, eps, gamma, vel_scale, tiny, 0, phi_out);
}

ORACLE_API int oracle_step_face(int nx, int ny, int nz, double dx, const double *phi,
                                const double *u, const double *v, const double *w,
                                double dt, double eps, double gamma, double vel_scale,
                                double tiny, double *phi_out)
{
    return step_impl(nx, ny, nz, dx, phi, u, v, w, dt, eps, gamma, vel_scale, tiny, 1, phi_out);
}

/* Mass and bounds of a field: out = {mass, sum, min, max, n_strict, n_tol}
 * with mass = dV * sum, n_strict = #(phi < 0 or phi > 1) and
 * n_tol = #(phi < -tol or phi > 1 + tol). */
ORACLE_API int oracle_stats(long n, const double *phi, double dV, double tol,
                            double *out4, long long *counts2)
{
    double sum = 0.0, mn = INFINITY, mx = -INFINITY;
    long long ns = 0, nt = 0;
    for (long c = 0; c < n; c++) {
        double p = phi[c];
        sum += p;
        if (p < mn) mn = p;
        if (p > mx) mx = p;
        if (p < 0.0 || p > 1.0) ns++;
        if (p < -tol || p > 1.0 + tol) nt++;
    }
    out4[0] = dV * sum; out4[1] = sum; out4[2] = mn; out4[3] = mx;
    counts2[0] = ns; counts2[1] = nt;
    return 0;
}

/*
 * Discrete adjoint of one Euler step (reverse mode through Steps 5..1).
 *   lam_out = (d phi^{k+1} / d phi^k)^T lam_next
 * If gu/gv/gw are non-NULL the velocity gradient (d phi^{k+1}/d u_f)^T lam_next
 * is ADDED to them.  Derivation, face f = c + 1/2 e_d between L = c, R = c+e_d:
 *   Fbar_f = (dt/dx)(lam_R - lam_L)            (Step 5 transposed)
 *   phibar_L += Fbar (us/2 + gamma eps/dx)    (Steps 3-4)
 *   phibar_R += Fbar (us/2 - gamma eps/dx)
 *   sbar_d[L] += gamma Fbar / 2, sbar_d[R] += gamma Fbar / 2   (Step 2b)
 *   ubar_f += Fbar vel_scale (phi_L + phi_R)/2
 *   phibar_c += sum_d sbar_d (1 - 2 phi_c) n_d                 (Step 2a)
 *   nbar_d = sbar_d phi_c (1 - phi_c)
 *   gbar = (nbar - n (n . nbar)) / m   (0 where g = 0)          (Step 1)
 *     the derivative of n = g / m, m = sqrt(|g|^2 + tiny): dn/dg = (I - n n^T)/m
 *   phibar_{c+e_d} += gbar_d, phibar_{c-e_d} -= gbar_d
 *   lam_out = lam_next + phibar.
 */
ORACLE_API int oracle_adjoint(int nx, int ny, int nz, double dx, const double *phi,
                              const double *u, const double *v, const double *w,
                              const double *lam_next, double dt, double eps,
                              double gamma, double vel_scale, double tiny, double *lam_out,
                              double *gu, double *gv, double *gw)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0.0) || !(tiny >= 0.0)) return -1;
    long n = (long)nx * ny * nz;
    double *nrm[3], *sbar[3], *gm, *pbar;
    for (int d = 0; d < 3; d++) {
        nrm[d] = (double *)malloc(sizeof(double) * n);
        sbar[d] = (double *)calloc(n, sizeof(double));
    }
    gm = (double *)malloc(sizeof(double) * n);
    pbar = (double *)calloc(n, sizeof(double));
    normals(nx, ny, nz, phi, tiny, nrm[0], nrm[1], nrm[2], gm);

    const double *vel[3] = {u, v, w};
    double *gvel[3] = {gu, gv, gw};
    /* Steps 5..2b transposed, face by face. */
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                long L = at(i, j, k, nx, ny, nz);
                for (int d = 0; d < 3; d++) {
                    long R = nb(i, j, k, d, +1, nx, ny, nz);
                    double Fbar = (dt / dx) * (lam_next[R] - lam_next[L]);
                    double us = vel_scale * vel[d][L];
                    pbar[L] += Fbar * (0.5 * us + gamma * eps / dx);
                    pbar[R] += Fbar * (0.5 * us - gamma * eps / dx);
                    sbar[d][L] += 0.5 * gamma * Fbar;
                    sbar[d][R] += 0.5 * gamma * Fbar;
                    if (gvel[d]) gvel[d][L] += Fbar * vel_scale * 0.5 * (phi[L] + phi[R]);
                }
            }
    /* Steps 2a and 1 transposed, cell by cell. */
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                long c = at(i, j, k, nx, ny, nz);
                double p = phi[c];
                double nbar[3], ndot = 0.0;
                for (int d = 0; d < 3; d++) {
                    pbar[c] += sbar[d][c] * (1.0 - 2.0 * p) * nrm[d][c];
                    nbar[d] = sbar[d][c] * p * (1.0 - p);
                    ndot += nrm[d][c] * nbar[d];
                }
                if (gm[c] > 0.0) {
                    for (int d = 0; d < 3; d++) {
                        double gbar = (nbar[d] - nrm[d][c] * ndot) / gm[c];
                        pbar[nb(i, j, k, d, +1, nx, ny, nz)] += gbar;
                        pbar[nb(i, j, k, d, -1, nx, ny, nz)] -= gbar;
                    }
                }
            }
    for (long c = 0; c < n; c++) lam_out[c] = lam_next[c] + pbar[c];
    for (int d = 0; d < 3; d++) { free(nrm[d]); free(sbar[d]); }
    free(gm); free(pbar);
    return 0;
}
