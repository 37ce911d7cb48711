/*
 * oracle_cs.c -- reference gradient of w^T tau by the complex-step method.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle_real.c).
 *
 * The inverse-dynamics recursion of dyn_body.h is compiled here with
 * `real` = double complex. For an input x_j perturbed by i*h,
 *     d(w^T tau)/dx_j = Im(w^T tau(x + i h e_j)) / h + O(h^2),
 * with no subtractive cancellation (Squire & Trapp 1998; Martins et al.
 * 2003), so h = 1e-20 gives the derivative to rounding. The recursion uses
 * only +, *, sin and cos, which are analytic, so the method applies.
 * Cost: 3n complex evaluations per instance.
 */
#include <complex.h>
#include <math.h>

typedef double complex real;
#define RSIN csin
#define RCOS ccos
#define PREFIX(x) cs_##x
#include "dyn_body.h"

static const double cs_default_base[18] = {0, 0, 0, 0, 0, 0, 0, 0, 9.81, 0, 0, 0,
                                           0, 0, 0, 0, 0, 0};

void oracle_rnea_grad_cs(int n, const double *M, const double *S, const double *inertia,
                         int B, const double *q, const double *qd, const double *qdd,
                         const double *w, const double *base, double *gq, double *gqd,
                         double *gqdd)
{
    const double h = 1e-20;
    const double *bc = base ? base : cs_default_base;
    real *in[3], *tau;
    for (int k = 0; k < 3; ++k) in[k] = malloc(sizeof(real) * (size_t)n);
    tau = malloc(sizeof(real) * (size_t)n);
    const double *src[3] = {q, qd, qdd};
    double *dst[3] = {gq, gqd, gqdd};
    for (int b = 0; b < B; ++b) {
        size_t o = (size_t)b * n;
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < n; ++i) in[k][i] = src[k][o + i];
        for (int k = 0; k < 3; ++k) {
            for (int j = 0; j < n; ++j) {
                in[k][j] = src[k][o + j] + I * h;
                cs_rnea_one(n, M, S, inertia, in[0], in[1], in[2], bc, tau, NULL, NULL, NULL);
                in[k][j] = src[k][o + j];
                double g = 0;
                for (int i = 0; i < n; ++i) g += w[o + i] * cimag(tau[i]);
                dst[k][o + j] = g / h;
            }
        }
    }
    for (int k = 0; k < 3; ++k) free(in[k]);
    free(tau);
}
