/*
 * dyn_body.h -- scalar-generic part of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may include, link or
 * call this code; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA path against a plain,
 * sequential restatement of the paper's recursions.
 *
 * This file is included twice: once with `real` = double (oracle_real.c) and
 * once with `real` = double complex (oracle_cs.c), so that the same
 * recursion can be differentiated by the complex-step method.  Everything is
 * written with explicit dense 6x6 matrices, in the order the equations are
 * printed, with no fusion:
 *
 *   Sec. II-A, Eq. (id-forward):   f_{i-1,i} = M_i exp(S_i q_i)
 *                                  V_i  = Ad_{f^-1} V_{i-1} + S_i qd_i
 *                                  dV_i = S_i qdd_i + Ad_{f^-1} dV_{i-1}
 *                                         - ad_{S_i qd_i} Ad_{f^-1} V_{i-1}
 *   Sec. II-A, Eq. (id-backward):  F_i  = Ad^T_{f_{i,i+1}^-1} F_{i+1}
 *                                         + J_i dV_i - ad^T_{V_i}(J_i V_i)
 *                                  tau_i = S_i^T F_i
 *
 * Conventions (readings of points the paper leaves open):
 *   twist  V = (v, w), linear part first; wrench F = (f, n), pairing F^T V;
 *   Ad_{(R,p)} = [[R, [p]R], [0, R]],  ad_{(v,w)} = [[[w], [v]], [0, [w]]];
 *   f_{i-1,i} maps frame-i coordinates to frame i-1, M_i = f_{i-1,i}(q=0),
 *   S_i is expressed in frame i;
 *   exp of a unit-axis twist: R = I + sin(t)[w] + (1-cos t)[w]^2,
 *   p = (I t + (1-cos t)[w] + (t - sin t)[w]^2) v  (Lynch & Park, Prop. 3.25);
 *   F_{n+1} is expressed in frame n (the transform f_{n,n+1} is the identity).
 */
#include <stdlib.h>
#include <string.h>

typedef real mat3[3][3];
typedef real mat6[6][6];

static void PREFIX(hat3)(const real w[3], mat3 W)
{
    W[0][0] = 0;     W[0][1] = -w[2]; W[0][2] = w[1];
    W[1][0] = w[2];  W[1][1] = 0;     W[1][2] = -w[0];
    W[2][0] = -w[1]; W[2][1] = w[0];  W[2][2] = 0;
}

static void PREFIX(mat3_mul)(const mat3 A, const mat3 B, mat3 C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real s = 0;
            for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

static void PREFIX(mat3_vec)(const mat3 A, const real x[3], real y[3])
{
    for (int i = 0; i < 3; ++i) {
        real s = 0;
        for (int k = 0; k < 3; ++k) s += A[i][k] * x[k];
        y[i] = s;
    }
}

static void PREFIX(mat6_vec)(const mat6 A, const real x[6], real y[6])
{
    for (int i = 0; i < 6; ++i) {
        real s = 0;
        for (int k = 0; k < 6; ++k) s += A[i][k] * x[k];
        y[i] = s;
    }
}

/* y = A^T x */
static void PREFIX(mat6T_vec)(const mat6 A, const real x[6], real y[6])
{
    for (int i = 0; i < 6; ++i) {
        real s = 0;
        for (int k = 0; k < 6; ++k) s += A[k][i] * x[k];
        y[i] = s;
    }
}

/* exp([S] t) for a twist S = (v, w) with |w| = 1, as (R, p). */
static void PREFIX(twist_exp)(const double S[6], real t, mat3 R, real p[3])
{
    real w[3] = {S[3], S[4], S[5]};
    real v[3] = {S[0], S[1], S[2]};
    mat3 W, W2;
    PREFIX(hat3)(w, W);
    PREFIX(mat3_mul)(W, W, W2);
    real st = RSIN(t), ct = RCOS(t);
    mat3 G;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real Id = (i == j) ? 1.0 : 0.0;
            R[i][j] = Id + st * W[i][j] + (1.0 - ct) * W2[i][j];
            G[i][j] = Id * t + (1.0 - ct) * W[i][j] + (t - st) * W2[i][j];
        }
    PREFIX(mat3_vec)(G, v, p);
}

/* f_{i-1,i} = M_i exp([S_i] q_i), with M_i given as 12 doubles (R row-major, p). */
static void PREFIX(link_transform)(const double Mi[12], const double Si[6], real qi,
                                   mat3 R, real p[3])
{
    mat3 RM, Re;
    real pM[3] = {Mi[9], Mi[10], Mi[11]};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) RM[i][j] = Mi[3 * i + j];
    real pe[3];
    PREFIX(twist_exp)(Si, qi, Re, pe);
    PREFIX(mat3_mul)(RM, Re, R);
    PREFIX(mat3_vec)(RM, pe, p);
    for (int i = 0; i < 3; ++i) p[i] += pM[i];
}

/* (R, p)^-1 = (R^T, -R^T p) */
static void PREFIX(se3_inverse)(const mat3 R, const real p[3], mat3 Ri, real pi[3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ri[i][j] = R[j][i];
    real t[3];
    PREFIX(mat3_vec)(Ri, p, t);
    for (int i = 0; i < 3; ++i) pi[i] = -t[i];
}

/* Ad_{(R,p)} = [[R, [p]R], [0, R]] */
static void PREFIX(Ad_matrix)(const mat3 R, const real p[3], mat6 A)
{
    mat3 P, PR;
    PREFIX(hat3)(p, P);
    PREFIX(mat3_mul)(P, R, PR);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) A[i][j] = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i][j] = R[i][j];
            A[i][3 + j] = PR[i][j];
            A[3 + i][3 + j] = R[i][j];
        }
}

/* ad_{(v,w)} = [[[w], [v]], [0, [w]]] */
static void PREFIX(ad_matrix)(const real xi[6], mat6 A)
{
    mat3 Vh, Wh;
    PREFIX(hat3)(xi, Vh);
    PREFIX(hat3)(xi + 3, Wh);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) A[i][j] = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i][j] = Wh[i][j];
            A[i][3 + j] = Vh[i][j];
            A[3 + i][3 + j] = Wh[i][j];
        }
}

/* Spatial inertia about the frame origin from (m, c, I_c):
 * J = [[m I, -m[c]], [m[c], I_c - m[c][c]]]. */
static void PREFIX(spatial_inertia)(const double in[10], mat6 J)
{
    real m = in[0];
    real c[3] = {in[1], in[2], in[3]};
    mat3 Ic = {{in[4], in[7], in[8]}, {in[7], in[5], in[9]}, {in[8], in[9], in[6]}};
    mat3 C, CC;
    PREFIX(hat3)(c, C);
    PREFIX(mat3_mul)(C, C, CC);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            J[i][j] = (i == j) ? m : 0.0;
            J[i][3 + j] = -m * C[i][j];
            J[3 + i][j] = m * C[i][j];
            J[3 + i][3 + j] = Ic[i][j] - m * CC[i][j];
        }
}

/*
 * One inverse-dynamics evaluation (Sec. II-A, Eqs. id-forward / id-backward).
 * base = {V_0[6], dV_0[6], F_{n+1}[6]} (real doubles).
 * Optional trace outputs (n*6 each, may be NULL): V, dV, F.
 */
void PREFIX(rnea_one)(int n, const double *M, const double *S, const double *inertia,
                      const real *q, const real *qd, const real *qdd, const double *base,
                      real *tau, real *Vout, real *dVout, real *Fout)
{
    mat6 *Adinv = (mat6 *)malloc(sizeof(mat6) * (size_t)n); /* Ad_{f_{i-1,i}^-1} */
    real (*V)[6] = malloc(sizeof(real[6]) * (size_t)n);
    real (*dV)[6] = malloc(sizeof(real[6]) * (size_t)n);
    real Vprev[6], dVprev[6];
    for (int k = 0; k < 6; ++k) {
        Vprev[k] = base[k];
        dVprev[k] = base[6 + k];
    }

    /* forward propagation, base toward tip: i = 1..n */
    for (int i = 0; i < n; ++i) {
        mat3 R, Ri;
        real p[3], pi[3];
        PREFIX(link_transform)(M + 12 * i, S + 6 * i, q[i], R, p);
        PREFIX(se3_inverse)(R, p, Ri, pi);
        PREFIX(Ad_matrix)(Ri, pi, Adinv[i]);

        real Sqd[6], Sqdd[6];
        for (int k = 0; k < 6; ++k) {
            Sqd[k] = S[6 * i + k] * qd[i];
            Sqdd[k] = S[6 * i + k] * qdd[i];
        }
        real AV[6], AdV[6], corr[6];
        mat6 adS;
        PREFIX(mat6_vec)(Adinv[i], Vprev, AV);
        PREFIX(mat6_vec)(Adinv[i], dVprev, AdV);
        PREFIX(ad_matrix)(Sqd, adS);
        PREFIX(mat6_vec)(adS, AV, corr);
        for (int k = 0; k < 6; ++k) {
            V[i][k] = AV[k] + Sqd[k];
            dV[i][k] = Sqdd[k] + AdV[k] - corr[k];
        }
        for (int k = 0; k < 6; ++k) {
            Vprev[k] = V[i][k];
            dVprev[k] = dV[i][k];
        }
    }

    /* backward propagation, tip toward base: i = n..1 */
    real Fnext[6];
    for (int k = 0; k < 6; ++k) Fnext[k] = base[12 + k];
    for (int i = n - 1; i >= 0; --i) {
        mat6 J, adV;
        real JV[6], JdV[6], adT[6], carried[6], F[6];
        PREFIX(spatial_inertia)(inertia + 10 * i, J);
        PREFIX(mat6_vec)(J, V[i], JV);
        PREFIX(mat6_vec)(J, dV[i], JdV);
        PREFIX(ad_matrix)(V[i], adV);
        PREFIX(mat6T_vec)(adV, JV, adT);
        if (i == n - 1) {
            for (int k = 0; k < 6; ++k) carried[k] = Fnext[k];
        } else {
            PREFIX(mat6T_vec)(Adinv[i + 1], Fnext, carried);
        }
        for (int k = 0; k < 6; ++k) F[k] = carried[k] + JdV[k] - adT[k];
        real t = 0;
        for (int k = 0; k < 6; ++k) t += S[6 * i + k] * F[k];
        tau[i] = t;
        for (int k = 0; k < 6; ++k) Fnext[k] = F[k];
        if (Vout)
            for (int k = 0; k < 6; ++k) Vout[6 * i + k] = V[i][k];
        if (dVout)
            for (int k = 0; k < 6; ++k) dVout[6 * i + k] = dV[i][k];
        if (Fout)
            for (int k = 0; k < 6; ++k) Fout[6 * i + k] = F[k];
    }
    free(Adinv);
    free(V);
    free(dV);
}
