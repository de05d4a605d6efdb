/* Drives every oracle entry point over odd shapes (extents 1 and 2, ragged sizes), with and
 * without a floor under |g|^2 and with NULL velocity gradients, on exact-size heap arrays:
 * built with AddressSanitizer and UBSan by tests/test_oracle_memory.py (test infrastructure). */
#include <stdio.h>
#include <stdlib.h>
int oracle_rhs(int, int, int, double, const double *, const double *, const double *, const double *, double, double, double, double, double *);
int oracle_rhs_face(int, int, int, double, const double *, const double *, const double *, const double *, double, double, double, double, double *);
int oracle_step(int, int, int, double, const double *, const double *, const double *, const double *, double, double, double, double, double, double *);
int oracle_step_face(int, int, int, double, const double *, const double *, const double *, const double *, double, double, double, double, double, double *);
int oracle_stats(long, const double *, double, double, double *, long long *);
int oracle_adjoint(int, int, int, double, const double *, const double *, const double *, const double *, const double *, double, double, double, double, double, double *, double *, double *, double *);
static double *arr(long n, unsigned *s) {
    double *a = malloc(sizeof(double) * n);
    for (long i = 0; i < n; i++) { *s = *s * 1664525u + 1013904223u; a[i] = (*s >> 8) / 16777216.0; }
    return a;
}
int main(void) {
    int shapes[][3] = {{1,1,1},{2,1,1},{1,2,1},{1,1,2},{2,2,2},{3,1,1},{1,3,5},{7,1,3},{4,5,6},{2,3,1},{17,2,3},{1,1,29}};
    unsigned s = 12345;
    int bad = 0;
    for (unsigned k = 0; k < sizeof shapes / sizeof shapes[0]; k++) {
        int nx = shapes[k][0], ny = shapes[k][1], nz = shapes[k][2];
        long n = (long)nx * ny * nz;
        double *phi = arr(n, &s), *u = arr(n, &s), *v = arr(n, &s), *w = arr(n, &s), *lam = arr(n, &s);
        double *o = malloc(sizeof(double) * n), *gu = malloc(sizeof(double) * n), *gv = malloc(sizeof(double) * n), *gw = malloc(sizeof(double) * n);
        for (long i = 0; i < n; i++) gu[i] = gv[i] = gw[i] = 0.0;
        for (int t = 0; t < 2; t++) {
            double tiny = t ? 1e-20 : 0.0;
            bad |= oracle_rhs(nx, ny, nz, 0.1, phi, u, v, w, 0.1, 1.0, 0.7, tiny, o) != 0;
            bad |= oracle_rhs_face(nx, ny, nz, 0.1, phi, u, v, w, 0.1, 1.0, 0.7, tiny, o) != 0;
            bad |= oracle_step(nx, ny, nz, 0.1, phi, u, v, w, 1e-3, 0.1, 1.0, 0.7, tiny, o) != 0;
            bad |= oracle_step_face(nx, ny, nz, 0.1, phi, u, v, w, 1e-3, 0.1, 1.0, 0.7, tiny, o) != 0;
            bad |= oracle_adjoint(nx, ny, nz, 0.1, phi, u, v, w, lam, 1e-3, 0.1, 1.0, 0.7, tiny, o, gu, gv, gw) != 0;
            bad |= oracle_adjoint(nx, ny, nz, 0.1, phi, u, v, w, lam, 1e-3, 0.1, 1.0, 0.7, tiny, o, NULL, NULL, NULL) != 0;
        }
        double out4[4]; long long c2[2];
        bad |= oracle_stats(n, phi, 1e-3, 2.2e-16, out4, c2) != 0;
        free(phi); free(u); free(v); free(w); free(lam); free(o); free(gu); free(gv); free(gw);
    }
    printf("done, nonzero returns: %d\n", bad);
    return 0;
}
