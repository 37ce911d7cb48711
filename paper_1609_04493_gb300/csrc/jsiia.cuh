// jsiia.cuh -- forward dynamics by joint-space-inertia inversion (Sec. III-C,
// Eqs. tau-bias and JSIinv; Algorithm 2), one warp per instance, n <= 32.
//
//   columns   lane j evaluates M_{.,j}(q) = ID(q, 0, delta_j, 0, 0, 0): with qd = 0
//             and no base motion the velocities vanish, dV is zero below link j,
//             dV_j = S_j, dV_i = Ad_{f_i^-1} dV_{i-1} above, F_hat_i = J_i dV_i,
//             and the backward recursion gives M_ij = S_i^T F_i. The backward
//             sweep re-derives dV_{i-1} = Ad_{f_i} dV_i instead of storing it.
//   bias      tau_bias = ID(q, qd, 0, V_0, dV_0, F_{n+1}) on lane n (n < 32, in
//             parallel with the columns) or on lane 0 after its column (n = 32).
//   solve     M = L L^T by a Cholesky factorisation with one row per lane, then
//             L y = tau - tau_bias and L^T qdd = y: FP64, in shared memory.
// Columns and bias run in T. Link rotations R_i = A_i Rz(q_i) are formed once per
// instance (lane i) and shared. A non-positive pivot sets RD_WARN_SINGULAR.
#pragma once
#include "../../include/rdyn.h"
#include "rnea_serial.cuh"

namespace rdyn {

template <typename T>
struct JsiiaSmem {
    double L[32][33];  // M, then its Cholesky factor (padded rows)
    T R[32][9];        // link rotations
    T bias[32];
};

template <typename T>
__device__ __forceinline__ Rot<T> jsiia_rot(const JsiiaSmem<T> &sm, int i)
{
    Rot<T> R;
#pragma unroll
    for (int k = 0; k < 9; ++k) R.r[k] = sm.R[i][k];
    return R;
}

// Column j of M(q) into sm.L[.][j].
template <typename T>
__device__ __forceinline__ void jsiia_column(const T *sc, JsiiaSmem<T> &sm, int n, int j)
{
    V3<T> a = mk3(T(0), T(0), T(0)), al = mk3(T(0), T(0), T(0));
    for (int i = j; i < n; ++i) {
        if (i == j) {
            al.z = T(1);  // dV_j = S_j
        } else {
            const Rot<T> R = jsiia_rot(sm, i);
            const T *L = sc + i * kLinkConsts;
            a = mulAT(R.r, cross_add(al, mk3(L[9], L[10], L[11]), a));
            al = mulAT(R.r, al);
        }
    }
    Wrench<T> F;
    F.f = F.n = mk3(T(0), T(0), T(0));
    for (int i = n - 1; i >= 0; --i) {
        const T *L = sc + i * kLinkConsts;
        if (i >= j) {
            // F_hat = J dV: f = m (a + al x c), n = c x f + I_c al
            const V3<T> cm = mk3(L[13], L[14], L[15]);
            const V3<T> f = scale3(L[12], cross_add(al, cm, a));
            F.f = add3(F.f, f);
            F.n = add3(F.n, cross_add(cm, f, sym_mul(L + 16, al)));
        }
        sm.L[i][j] = (double)F.n.z;
        if (i > 0) {
            const Rot<T> R = jsiia_rot(sm, i);
            const V3<T> bi = mk3(L[9], L[10], L[11]);
            // F_{i-1} part carried from link i: Ad^T_{f_i^-1} F_i
            const V3<T> rf = mulA(R.r, F.f);
            F.n = cross_add(bi, rf, mulA(R.r, F.n));
            F.f = rf;
            if (i > j) {  // dV_{i-1} = Ad_{f_i} dV_i
                const V3<T> pal = mulA(R.r, al);
                a = cross_add(bi, pal, mulA(R.r, a));
                al = pal;
            }
        }
    }
}

// tau_bias with qdd = 0 (the motion re-derived in the backward sweep).
template <typename T>
__device__ __forceinline__ void jsiia_bias(const T *sc, JsiiaSmem<T> &sm, int n,
                                           const T *__restrict__ qdr, const BaseParams<T> &base)
{
    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);
    for (int i = 0; i < n; ++i) {
        const T *L = sc + i * kLinkConsts;
        x = forward_step_R(jsiia_rot(sm, i), mk3(L[9], L[10], L[11]), __ldg(qdr + i), T(0), x);
    }
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    for (int i = n - 1; i >= 0; --i) {
        const T *L = sc + i * kLinkConsts;
        const Wrench<T> Fh = bias_wrench(L[12], mk3(L[13], L[14], L[15]), L + 16, x);
        if (i == n - 1) {
            F.f = add3(F.f, Fh.f);
            F.n = add3(F.n, Fh.n);
        } else {
            const T *Ln = sc + (i + 1) * kLinkConsts;
            F = carry_wrench_R(jsiia_rot(sm, i + 1), mk3(Ln[9], Ln[10], Ln[11]), F, Fh);
        }
        sm.bias[i] = F.n.z;
        if (i > 0)
            x = backward_recover_R(jsiia_rot(sm, i), mk3(L[9], L[10], L[11]), __ldg(qdr + i), T(0), x);
    }
}

template <typename T, int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
jsiia_kernel(const T *__restrict__ consts, int n, int B, const T *__restrict__ q,
             const T *__restrict__ qd, const T *__restrict__ tau, T *__restrict__ qdd,
             int *__restrict__ status, BaseParams<T> base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *sc = reinterpret_cast<T *>(smem);
    const int nc = n * kLinkConsts;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) sc[k] = consts[k];
    const size_t cbytes = (((size_t)nc * sizeof(T)) + 15) & ~(size_t)15;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    JsiiaSmem<T> &sm = reinterpret_cast<JsiiaSmem<T> *>(smem + cbytes)[warp];
    __syncthreads();

    const int b = blockIdx.x * WARPS + warp;
    if (b >= B) return;  // whole warps leave together
    const size_t row = (size_t)b * (size_t)n;

    if (lane < n) {
        T s, c;
        sincos_t(__ldg(q + row + lane), &s, &c);
        const Rot<T> R = make_rot(sc + lane * kLinkConsts, c, s);
#pragma unroll
        for (int k = 0; k < 9; ++k) sm.R[lane][k] = R.r[k];
    }
    __syncwarp();
    if (lane < n) jsiia_column(sc, sm, n, lane);
    else if (lane == n) jsiia_bias(sc, sm, n, qd + row, base);
    __syncwarp();
    if (n == 32 && lane == 0) jsiia_bias(sc, sm, n, qd + row, base);
    __syncwarp();

    // Cholesky, lane i owns row i (lower triangle of sm.L)
    int bad = 0;
    for (int k = 0; k < n; ++k) {
        if (lane == k) {
            double d = sm.L[k][k];
            for (int p = 0; p < k; ++p) d -= sm.L[k][p] * sm.L[k][p];
            if (!(d > 0.0)) {
                bad = 1;
                d = 1e-300;
            }
            sm.L[k][k] = sqrt(d);
        }
        __syncwarp();
        if (lane > k && lane < n) {
            double s = sm.L[lane][k];
            for (int p = 0; p < k; ++p) s -= sm.L[lane][p] * sm.L[k][p];
            sm.L[lane][k] = s / sm.L[k][k];
        }
        __syncwarp();
    }

    // L y = tau - tau_bias, then L^T x = y (lane i holds entry i)
    double r = lane < n ? (double)__ldg(tau + row + lane) - (double)sm.bias[lane] : 0.0;
    for (int k = 0; k < n; ++k) {
        const double yk = __shfl_sync(0xffffffffu, r / sm.L[k][k], k);
        if (lane == k) r = yk;
        else if (lane > k && lane < n) r -= sm.L[lane][k] * yk;
    }
    for (int k = n - 1; k >= 0; --k) {
        const double xk = __shfl_sync(0xffffffffu, r / sm.L[k][k], k);
        if (lane == k) r = xk;
        else if (lane < k) r -= sm.L[k][lane] * xk;
    }
    if (lane < n) {
        qdd[row + lane] = (T)r;
        if (!(r == r)) bad = 1;
    }
    bad = __any_sync(0xffffffffu, bad);
    if (status && lane == 0) status[b] = bad ? RD_WARN_SINGULAR : 0;
}

template <typename T, int WARPS>
__host__ __device__ constexpr size_t jsiia_smem_bytes(int n)
{
    return ((((size_t)n * kLinkConsts * sizeof(T)) + 15) & ~(size_t)15) +
           (size_t)WARPS * sizeof(JsiiaSmem<T>);
}

}  // namespace rdyn
