/*
 * oracle_real.c -- FP64 CPU oracle: inverse dynamics, joint-space inertia,
 * and forward dynamics two ways.
 *
 * TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU
 * baseline). The product path never links or calls it, and it shares no
 * code, header or constant with the CUDA sources.
 *
 * Compiled with -ffp-contract=off: every product and sum is rounded as
 * written, round to nearest.
 *
 * Exported functions (plain C ABI, host pointers, row-major arrays):
 *   oracle_rnea         tau = ID(q, qd, qdd, V0, dV0, F_{n+1})     Sec. II-A
 *   oracle_rnea_trace   same, also returning V_i, dV_i, F_i
 *   oracle_mass_matrix  M(q) column j = ID(q, 0, delta_j, 0, 0, 0) Sec. III-C
 *   oracle_fd_jsiia     qdd = M^-1 (tau - tau_bias), Cholesky      Eqs. tau-bias, JSIinv
 *   oracle_fd_aba       qdd by the articulated-body recursion      Eqs. abi, recursive-fd
 *   oracle_rnea_grad_cs d(w^T tau)/d(q, qd, qdd) by complex step (oracle_cs.c)
 */
#include <math.h>

typedef double real;
#define RSIN sin
#define RCOS cos
#define PREFIX(x) x
#include "dyn_body.h"

static const double default_base[18] = {0, 0, 0, 0, 0, 0, 0, 0, 9.81, 0, 0, 0,
                                        0, 0, 0, 0, 0, 0};

static const double *pick_base(const double *base)
{
    return base ? base : default_base;
}

void oracle_rnea(int n, const double *M, const double *S, const double *inertia, int B,
                 const double *q, const double *qd, const double *qdd,
                 const double *base, double *tau)
{
    const double *bc = pick_base(base);
    for (int b = 0; b < B; ++b) {
        size_t o = (size_t)b * (size_t)n;
        rnea_one(n, M, S, inertia, q + o, qd + o, qdd + o, bc, tau + o, NULL, NULL, NULL);
    }
}

void oracle_rnea_trace(int n, const double *M, const double *S, const double *inertia,
                       const double *q, const double *qd, const double *qdd,
                       const double *base, double *tau, double *V, double *dV, double *F)
{
    rnea_one(n, M, S, inertia, q, qd, qdd, pick_base(base), tau, V, dV, F);
}

/* Joint-space inertia, one column per unit joint acceleration (Sec. III-C):
 * M_{.,j}(q) = ID(q, 0, delta_j, 0, 0, 0). Output [B, n, n], row-major. */
void oracle_mass_matrix(int n, const double *M, const double *S, const double *inertia,
                        int B, const double *q, double *Mq)
{
    static const double zero_base[18] = {0};
    double *zeros = calloc((size_t)n, sizeof(double));
    double *e = calloc((size_t)n, sizeof(double));
    double *col = malloc(sizeof(double) * (size_t)n);
    for (int b = 0; b < B; ++b) {
        const double *qb = q + (size_t)b * n;
        double *Mb = Mq + (size_t)b * n * n;
        for (int j = 0; j < n; ++j) {
            e[j] = 1.0;
            rnea_one(n, M, S, inertia, qb, zeros, e, zero_base, col, NULL, NULL, NULL);
            e[j] = 0.0;
            for (int i = 0; i < n; ++i) Mb[(size_t)i * n + j] = col[i];
        }
    }
    free(zeros);
    free(e);
    free(col);
}

/* In-place Cholesky A = L L^T (lower triangle). Returns 0, or -1 if a pivot
 * is not positive. */
static int cholesky(int n, double *A)
{
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) return -1;
        double ljj = sqrt(d);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = s / ljj;
        }
    }
    return 0;
}

/* Forward dynamics by joint-space-inertia inversion (Eqs. tau-bias, JSIinv;
 * Algorithm 2): tau_bias = ID(q, qd, 0, base), M(q) by unit columns, then a
 * Cholesky solve of M qdd = tau - tau_bias. status[b] = 0, or -1 when M is
 * not positive definite. */
void oracle_fd_jsiia(int n, const double *M, const double *S, const double *inertia,
                     int B, const double *q, const double *qd, const double *tau,
                     const double *base, double *qdd, int *status)
{
    const double *bc = pick_base(base);
    double *zeros = calloc((size_t)n, sizeof(double));
    double *bias = malloc(sizeof(double) * (size_t)n);
    double *Mq = malloc(sizeof(double) * (size_t)n * n);
    double *y = malloc(sizeof(double) * (size_t)n);
    for (int b = 0; b < B; ++b) {
        size_t o = (size_t)b * n;
        rnea_one(n, M, S, inertia, q + o, qd + o, zeros, bc, bias, NULL, NULL, NULL);
        oracle_mass_matrix(n, M, S, inertia, 1, q + o, Mq);
        int st = cholesky(n, Mq);
        if (status) status[b] = st;
        if (st != 0) {
            for (int i = 0; i < n; ++i) qdd[o + i] = NAN;
            continue;
        }
        /* L y = tau - bias; L^T x = y */
        for (int i = 0; i < n; ++i) {
            double s = tau[o + i] - bias[i];
            for (int k = 0; k < i; ++k) s -= Mq[(size_t)i * n + k] * y[k];
            y[i] = s / Mq[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < n; ++k) s -= Mq[(size_t)k * n + i] * qdd[o + k];
            qdd[o + i] = s / Mq[(size_t)i * n + i];
        }
    }
    free(zeros);
    free(bias);
    free(Mq);
    free(y);
}

/* 6x6 helpers used only by the articulated-body oracle. */
static void mat6_mul(const mat6 A, const mat6 Bm, mat6 C)
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s = 0;
            for (int k = 0; k < 6; ++k) s += A[i][k] * Bm[k][j];
            C[i][j] = s;
        }
}

static void mat6_transpose(const mat6 A, mat6 T)
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) T[i][j] = A[j][i];
}

/*
 * Forward dynamics by the articulated-body inertia algorithm, in the
 * paper's notation (Sec. II-B):
 *   tau_bias = ID(q, qd, 0, V0, dV0, F_{n+1}),  hat tau = tau - tau_bias
 *   Eq. (abi), i = n..1:
 *     hat J_n = J_n,
 *     hat J_i = J_i + X^T hat J_{i+1} X
 *               - X^T hat J_{i+1} S_{i+1} S_{i+1}^T hat J_{i+1} X / Omega_{i+1},
 *     X = Ad_{f_{i,i+1}^-1},  Omega_i = S_i^T hat J_i S_i
 *   Y_{i,i+1}  = X^T (I - hat J_{i+1} S_{i+1} S_{i+1}^T / Omega_{i+1})
 *   Pi_{i,i+1} = X^T hat J_{i+1} S_{i+1} / Omega_{i+1}
 *   Eq. (recursive-fd), backward, i = n..1 (hat z_n = 0):
 *     hat z_i = Y_{i,i+1} hat z_{i+1} + Pi_{i,i+1} hat tau_{i+1}
 *     c_i = hat tau_i - S_i^T hat z_i,   hat c_i = c_i / Omega_i
 *   forward, i = 1..n (lambda_0 = 0):
 *     lambda_i = Y_{i-1,i}^T lambda_{i-1} + S_i hat c_i
 *     qdd_i    = hat c_i - Pi_{i-1,i}^T lambda_{i-1}
 * Boundary reading: hat J_n = J_n and hat z_n = 0 (no link n+1); the base
 * acceleration and external wrench enter only through tau_bias.
 */
static void fd_aba_one(int n, const double *M, const double *S, const double *inertia,
                       const double *q, const double *qd, const double *tau,
                       const double *base, double *qdd)
{
    if (n <= 0) return;
    double *zeros = calloc((size_t)n, sizeof(double));
    double *bias = malloc(sizeof(double) * (size_t)n);
    double *htau = malloc(sizeof(double) * (size_t)n);
    mat6 *X = malloc(sizeof(mat6) * (size_t)n);      /* X[i] = Ad_{f_{i-1,i}^-1} */
    mat6 *Jh = malloc(sizeof(mat6) * (size_t)n);     /* hat J_i */
    mat6 *Y = malloc(sizeof(mat6) * (size_t)n);      /* Y[i] = Y_{i-1,i} (i >= 1) */
    double (*Pi)[6] = malloc(sizeof(double[6]) * (size_t)n); /* Pi[i] = Pi_{i-1,i} */
    double *Om = malloc(sizeof(double) * (size_t)n);
    double (*zh)[6] = malloc(sizeof(double[6]) * (size_t)n);
    double *ch = malloc(sizeof(double) * (size_t)n);

    rnea_one(n, M, S, inertia, q, qd, zeros, base, bias, NULL, NULL, NULL);
    for (int i = 0; i < n; ++i) htau[i] = tau[i] - bias[i];

    for (int i = 0; i < n; ++i) {
        mat3 R, Ri;
        double p[3], pi[3];
        link_transform(M + 12 * i, S + 6 * i, q[i], R, p);
        se3_inverse(R, p, Ri, pi);
        Ad_matrix(Ri, pi, X[i]);
    }

    /* Eq. (abi): articulated-body inertias, tip to base */
    spatial_inertia(inertia + 10 * (n - 1), Jh[n - 1]);
    for (int i = n - 2; i >= 0; --i) {
        const double *Sn = S + 6 * (i + 1);
        mat6 J, XT, T1, T2, XTJX;
        spatial_inertia(inertia + 10 * i, J);
        mat6_transpose(X[i + 1], XT);
        mat6_mul(XT, Jh[i + 1], T1);    /* X^T hat J */
        mat6_mul(T1, X[i + 1], XTJX);   /* X^T hat J X */
        double JS[6], Om1 = 0;
        mat6_vec(Jh[i + 1], Sn, JS);    /* hat J S */
        for (int k = 0; k < 6; ++k) Om1 += Sn[k] * JS[k];
        double u[6];                    /* X^T hat J S */
        mat6T_vec(X[i + 1], JS, u);
        for (int a = 0; a < 6; ++a)
            for (int b2 = 0; b2 < 6; ++b2) T2[a][b2] = u[a] * u[b2] / Om1;
        for (int a = 0; a < 6; ++a)
            for (int b2 = 0; b2 < 6; ++b2) Jh[i][a][b2] = J[a][b2] + XTJX[a][b2] - T2[a][b2];
    }

    for (int i = 0; i < n; ++i) {
        const double *Si = S + 6 * i;
        double JS[6], s = 0;
        mat6_vec(Jh[i], Si, JS);
        for (int k = 0; k < 6; ++k) s += Si[k] * JS[k];
        Om[i] = s;
    }

    /* Y_{i-1,i} and Pi_{i-1,i} for i = 1..n-1 (0-based: the pair (i-1, i)) */
    for (int i = 1; i < n; ++i) {
        const double *Si = S + 6 * i;
        double JS[6];
        mat6_vec(Jh[i], Si, JS);
        mat6 Pmat, XT;
        for (int a = 0; a < 6; ++a)
            for (int b2 = 0; b2 < 6; ++b2)
                Pmat[a][b2] = ((a == b2) ? 1.0 : 0.0) - JS[a] * Si[b2] / Om[i];
        mat6_transpose(X[i], XT);
        mat6_mul(XT, Pmat, Y[i]);
        double t[6];
        mat6T_vec(X[i], JS, t);
        for (int k = 0; k < 6; ++k) Pi[i][k] = t[k] / Om[i];
    }

    /* backward recursion: hat z, hat c */
    for (int k = 0; k < 6; ++k) zh[n - 1][k] = 0.0;
    for (int i = n - 2; i >= 0; --i) {
        double yz[6];
        mat6_vec(Y[i + 1], zh[i + 1], yz);
        for (int k = 0; k < 6; ++k) zh[i][k] = yz[k] + Pi[i + 1][k] * htau[i + 1];
    }
    for (int i = 0; i < n; ++i) {
        double sz = 0;
        for (int k = 0; k < 6; ++k) sz += S[6 * i + k] * zh[i][k];
        double c = htau[i] - sz;
        ch[i] = c / Om[i];
    }

    /* forward recursion: lambda, qdd */
    double lam[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
        double lnew[6], pl = 0;
        if (i == 0) {
            for (int k = 0; k < 6; ++k) lnew[k] = 0.0;
        } else {
            mat6T_vec(Y[i], lam, lnew);
            for (int k = 0; k < 6; ++k) pl += Pi[i][k] * lam[k];
        }
        qdd[i] = ch[i] - pl;
        for (int k = 0; k < 6; ++k) lam[k] = lnew[k] + S[6 * i + k] * ch[i];
    }

    free(zeros); free(bias); free(htau); free(X); free(Jh); free(Y);
    free(Pi); free(Om); free(zh); free(ch);
}

void oracle_fd_aba(int n, const double *M, const double *S, const double *inertia, int B,
                   const double *q, const double *qd, const double *tau,
                   const double *base, double *qdd)
{
    const double *bc = pick_base(base);
    for (int b = 0; b < B; ++b) {
        size_t o = (size_t)b * n;
        fd_aba_one(n, M, S, inertia, q + o, qd + o, tau + o, bc, qdd + o);
    }
}

/* Articulated-body inertias and Omega_i for one state (test access to the
 * intermediate quantities of Eq. (abi)). Jhat: [n, 36], Omega: [n]. */
void oracle_abi_trace(int n, const double *M, const double *S, const double *inertia,
                      const double *q, double *Jhat, double *Omega)
{
    if (n <= 0) return;
    mat6 *X = malloc(sizeof(mat6) * (size_t)n);
    mat6 *Jh = malloc(sizeof(mat6) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        mat3 R, Ri;
        double p[3], pi[3];
        link_transform(M + 12 * i, S + 6 * i, q[i], R, p);
        se3_inverse(R, p, Ri, pi);
        Ad_matrix(Ri, pi, X[i]);
    }
    spatial_inertia(inertia + 10 * (n - 1), Jh[n - 1]);
    for (int i = n - 2; i >= 0; --i) {
        const double *Sn = S + 6 * (i + 1);
        mat6 J, XT, T1, XTJX;
        spatial_inertia(inertia + 10 * i, J);
        mat6_transpose(X[i + 1], XT);
        mat6_mul(XT, Jh[i + 1], T1);
        mat6_mul(T1, X[i + 1], XTJX);
        double JS[6], Om1 = 0, u[6];
        mat6_vec(Jh[i + 1], Sn, JS);
        for (int k = 0; k < 6; ++k) Om1 += Sn[k] * JS[k];
        mat6T_vec(X[i + 1], JS, u);
        for (int a = 0; a < 6; ++a)
            for (int b2 = 0; b2 < 6; ++b2)
                Jh[i][a][b2] = J[a][b2] + XTJX[a][b2] - u[a] * u[b2] / Om1;
    }
    for (int i = 0; i < n; ++i) {
        double JS[6], s = 0;
        mat6_vec(Jh[i], S + 6 * i, JS);
        for (int k = 0; k < 6; ++k) s += S[6 * i + k] * JS[k];
        Omega[i] = s;
        for (int a = 0; a < 6; ++a)
            for (int b2 = 0; b2 < 6; ++b2) Jhat[(size_t)i * 36 + 6 * a + b2] = Jh[i][a][b2];
    }
    free(X);
    free(Jh);
}
