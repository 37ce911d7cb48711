// aba_tri.cuh -- forward dynamics (aba_dh.cuh) with three warps per 32
// instances: warp Z of aba_pair.cuh, and the articulated-inertia recursion of
// its warp J split over two warps by block.
//
// With J_hat = [[A, Bm], [Bm^T, C]] the update J_hat_i = J_i + X^T P X of
// aba_dh.cuh (P = J_hat_{i+1} - U U^T / Omega) falls into two parts:
//   warp JA: P.A and P.C, their rotations, the shift terms of A ([b] A_r, its
//     transpose PT, and -[b] A_r [b]), A' and C'; then Omega_i = C'_zz, its
//     reciprocal and U_w = C' e_z;
//   warp JB: P.Bm, its rotation B_r, the shift term Nr = [b] B_r, and
//     Bm' = B_r + PT + [m c]; then U_v = Bm' e_z.
// Per link JA needs Nr (for C') and, for P.A, the U_v of the link before; JB
// needs PT (for Bm') and, for P.Bm, (U_w, 1 / Omega) of the link before. Each
// value goes through a two-slot ring per lane in shared memory and is announced
// by a per-lane counter (the link its producer has reached, counting down);
// the producer publishes PT (or Nr) before it waits for the other's, so the
// two never wait on each other at the same point. A slot is written again only
// after its reader has announced a later step that follows the read, so two
// slots suffice. Warp Z waits for both halves of U_i (counters JA-U and JB-U).
//
// The arithmetic is that of aba_dh_update, operation by operation, so the
// results agree with the two-warp and one-thread kernels to rounding. Every
// wait is bounded as in aba_pair.cuh; a role that times out flags
// RD_WARN_TIMEOUT through its flag word and waits no more.
#pragma once
#include "aba_pair.cuh"

namespace rdyn {

// Per-block exchange state of the three-warp kernel (32 instances).
template <typename D>
struct AbaTriShared {
    D pt[2][9][32];  // JA -> JB: PT of link i in slot i & 1
    D nr[2][9][32];  // JB -> JA: Nr
    D ua[2][3][32];  // JA -> JB: U_w x, U_w y, 1 / Omega
    D ub[2][3][32];  // JB -> JA: U_v
    int cnt[4][32];  // per lane: JA's PT, JA's U, JB's Nr, JB's U
    int flags[2][32];
};

enum { kTriPT = 0, kTriUA = 1, kTriNR = 2, kTriUB = 3 };

// Warp JA's share of one instance (lane `lane` of the block's exchange state).
template <typename T, typename D, typename TB, int TRIG>
__device__ __forceinline__ void aba_tri_ja(const T *__restrict__ sc, const D *__restrict__ sd,
                                           const DF *__restrict__ sdf, int n,
                                           const T *__restrict__ qr, D *__restrict__ wsz, int B,
                                           int b, AbaTriShared<D> &sh, int lane)
{
    volatile int *cnt = &sh.cnt[0][0];
    int bad = 0, timeout = 0;
    Sym3<D> A, C;
    D Uw[3], invOm = D(0);
#pragma unroll 1
    for (int i = n - 1; i >= 0; --i) {
        const D *ri = sd + i * kAbaDh64;
        if (i > 0) {
            prefetch_l1(sd + (i - 1) * kAbaDh64);
            prefetch_l1(sd + (i - 1) * kAbaDh64 + kAbaDh64 / 2);
        }
        if (i == n - 1) {
            const D m = ri[6], zero = D(0);
            A = Sym3<D>{m, m, m, zero, zero, zero};
            C = Sym3<D>{ri[19], ri[20], ri[21], ri[22], ri[23], ri[24]};
        } else {
            TB s1, c1;
            aba_trig_tb<T, TB, TRIG>(sc, sdf, qr, i + 1, s1, c1);
            const D c = dcvt<D>(c1), s = dcvt<D>(s1);
            const D *r = sd + (i + 1) * kAbaDh64;
            // P.C from this warp's own U_w and 1 / Omega of link i+1
            const D wx = Uw[0] * invOm, wy = Uw[1] * invOm;
            const D Pcxx = fma(-wx, Uw[0], C.xx), Pcyy = fma(-wy, Uw[1], C.yy);
            const D Pcxy = fma(-wx, Uw[1], C.xy);
            // P.A needs JB's U_v of link i+1
            aba_wait2(cnt + kTriUB * 32 + lane, cnt + kTriUB * 32 + lane, i + 1, timeout);
            const int so = (i + 1) & 1;
            const D Uv[3] = {sh.ub[so][0][lane], sh.ub[so][1][lane], sh.ub[so][2][lane]};
            const D ux = Uv[0] * invOm, uy = Uv[1] * invOm, uz = Uv[2] * invOm;
            const Sym3<D> PA = {fma(-ux, Uv[0], A.xx), fma(-uy, Uv[1], A.yy),
                                fma(-uz, Uv[2], A.zz), fma(-ux, Uv[1], A.xy),
                                fma(-ux, Uv[2], A.xz), fma(-uy, Uv[2], A.yz)};
            // rotations (aba_dh_update's order)
            const D ca = r[0], sa = r[1];
            const D ca2 = r[25], sa2 = r[26], casa = r[27], c2a = r[28], s2a = r[29];
            const D c2 = fma(c, c, -s * s), s2 = dtwice(c * s);
            Sym3<D> MA = rotz_sym(PA, c, s, c2, s2);
            const D hc = dhalf(Pcxx + Pcyy), dc = dhalf(Pcxx - Pcyy);
            const D tc = fma(dc, c2, -Pcxy * s2);
            const D Cxx = hc + tc, Cyy = hc - tc, Cxy = fma(dc, s2, Pcxy * c2);
            MA = rotx_sym(MA, ca, sa, c2a, s2a);
            const Sym3<D> MC = {Cxx, ca2 * Cyy, sa2 * Cyy, ca * Cxy, sa * Cxy, casa * Cyy};
            // shift terms of A: PT = ([b] A_r)^T, published for JB
            const D bv[3] = {r[2], r[3], r[4]};
            D Ar[9], Pm[9], PT[9];
            sym_to_full(MA, Ar);
            hat_mul(bv, Ar, Pm);
#pragma unroll
            for (int u = 0; u < 3; ++u)
#pragma unroll
                for (int v = 0; v < 3; ++v) PT[3 * u + v] = Pm[3 * v + u];
            const int si = i & 1;
#pragma unroll
            for (int k = 0; k < 9; ++k) sh.pt[si][k][lane] = PT[k];
            __threadfence_block();
            cnt[kTriPT * 32 + lane] = i;
            const D q00 = fma(bv[1], PT[6], -bv[2] * PT[3]);
            const D q01 = fma(bv[1], PT[7], -bv[2] * PT[4]);
            const D q02 = fma(bv[1], PT[8], -bv[2] * PT[5]);
            const D q11 = fma(bv[2], PT[1], -bv[0] * PT[7]);
            const D q12 = fma(bv[2], PT[2], -bv[0] * PT[8]);
            const D q22 = fma(bv[0], PT[5], -bv[1] * PT[2]);
            const D m = ri[6];
            A = Sym3<D>{MA.xx + m, MA.yy + m, MA.zz + m, MA.xy, MA.xz, MA.yz};
            // C' needs JB's Nr of link i
            aba_wait2(cnt + kTriNR * 32 + lane, cnt + kTriNR * 32 + lane, i, timeout);
            D Nr[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) Nr[k] = sh.nr[si][k][lane];
            C.xx = dtwice_add(Nr[0], MC.xx) + q00 + ri[19];
            C.yy = dtwice_add(Nr[4], MC.yy) + q11 + ri[20];
            C.zz = dtwice_add(Nr[8], MC.zz) + q22 + ri[21];
            C.xy = MC.xy + Nr[1] + Nr[3] + q01 + ri[22];
            C.xz = MC.xz + Nr[2] + Nr[6] + q02 + ri[23];
            C.yz = MC.yz + Nr[5] + Nr[7] + q12 + ri[24];
        }
        Uw[0] = C.xz;
        Uw[1] = C.yz;
        Uw[2] = C.zz;
        const D Om = C.zz;
        if (!dpositive(Om)) bad = 1;
        invOm = drecip(Om);
#pragma unroll
        for (int k = 0; k < 3; ++k) aba_zput(wsz, B, b, i, 3 + k, Uw[k]);
        aba_zput(wsz, B, b, i, 7, invOm);
        const int si = i & 1;
        sh.ua[si][0][lane] = Uw[0];
        sh.ua[si][1][lane] = Uw[1];
        sh.ua[si][2][lane] = invOm;
        if (i == 0) sh.flags[0][lane] = bad | (timeout << 1);
        __threadfence_block();
        cnt[kTriUA * 32 + lane] = i;
    }
}

// Warp JB's share of one instance.
template <typename T, typename D, typename TB, int TRIG>
__device__ __forceinline__ void aba_tri_jb(const T *__restrict__ sc, const D *__restrict__ sd,
                                           const DF *__restrict__ sdf, int n,
                                           const T *__restrict__ qr, D *__restrict__ wsz, int B,
                                           int b, AbaTriShared<D> &sh, int lane)
{
    volatile int *cnt = &sh.cnt[0][0];
    int timeout = 0;
    D Bm[9], Uv[3];
#pragma unroll 1
    for (int i = n - 1; i >= 0; --i) {
        const D *ri = sd + i * kAbaDh64;
        if (i > 0) {
            prefetch_l1(sd + (i - 1) * kAbaDh64);
            prefetch_l1(sd + (i - 1) * kAbaDh64 + kAbaDh64 / 2);
        }
        if (i == n - 1) {
            const D zero = D(0);
            Bm[0] = zero;    Bm[1] = ri[18];  Bm[2] = -ri[17];
            Bm[3] = -ri[18]; Bm[4] = zero;    Bm[5] = ri[16];
            Bm[6] = ri[17];  Bm[7] = -ri[16]; Bm[8] = zero;
        } else {
            TB s1, c1;
            aba_trig_tb<T, TB, TRIG>(sc, sdf, qr, i + 1, s1, c1);
            const D c = dcvt<D>(c1), s = dcvt<D>(s1);
            const D *r = sd + (i + 1) * kAbaDh64;
            // P.Bm needs JA's U_w and 1 / Omega of link i+1
            aba_wait2(cnt + kTriUA * 32 + lane, cnt + kTriUA * 32 + lane, i + 1, timeout);
            const int so = (i + 1) & 1;
            const D uw0 = sh.ua[so][0][lane], uw1 = sh.ua[so][1][lane];
            const D iom = sh.ua[so][2][lane];
            const D wx = uw0 * iom, wy = uw1 * iom;
            D PB[9];
#pragma unroll
            for (int rr = 0; rr < 3; ++rr) {
                PB[3 * rr] = fma(-Uv[rr], wx, Bm[3 * rr]);
                PB[3 * rr + 1] = fma(-Uv[rr], wy, Bm[3 * rr + 1]);
                PB[3 * rr + 2] = D(0);
            }
            // rotations (aba_dh_update's order)
            const D ca = r[0], sa = r[1];
            D B1[6];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                B1[k] = fma(c, PB[k], -s * PB[3 + k]);
                B1[2 + k] = fma(s, PB[k], c * PB[3 + k]);
                B1[4 + k] = PB[6 + k];
            }
            D B2[6];
#pragma unroll
            for (int rr = 0; rr < 3; ++rr) {
                B2[2 * rr] = fma(c, B1[2 * rr], -s * B1[2 * rr + 1]);
                B2[2 * rr + 1] = fma(s, B1[2 * rr], c * B1[2 * rr + 1]);
            }
            D Br[9];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const D y = B2[2 + k], z = B2[4 + k];
                Br[k] = B2[k];
                Br[3 + k] = fma(ca, y, -sa * z);
                Br[6 + k] = fma(sa, y, ca * z);
            }
#pragma unroll
            for (int rr = 0; rr < 3; ++rr) {
                const D col1 = Br[3 * rr + 1];
                Br[3 * rr + 1] = ca * col1;
                Br[3 * rr + 2] = sa * col1;
            }
            // Nr = [b] B_r, published for JA
            const D bv[3] = {r[2], r[3], r[4]};
            D Nr[9];
            hat_mul(bv, Br, Nr);
            const int si = i & 1;
#pragma unroll
            for (int k = 0; k < 9; ++k) sh.nr[si][k][lane] = Nr[k];
            __threadfence_block();
            cnt[kTriNR * 32 + lane] = i;
            // Bm' needs JA's PT of link i
            aba_wait2(cnt + kTriPT * 32 + lane, cnt + kTriPT * 32 + lane, i, timeout);
            D PT[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) PT[k] = sh.pt[si][k][lane];
            const D mcx = ri[16], mcy = ri[17], mcz = ri[18];
            Bm[0] = Br[0] + PT[0];
            Bm[1] = Br[1] + PT[1] + mcz;
            Bm[2] = Br[2] + PT[2] - mcy;
            Bm[3] = Br[3] + PT[3] - mcz;
            Bm[4] = Br[4] + PT[4];
            Bm[5] = Br[5] + PT[5] + mcx;
            Bm[6] = Br[6] + PT[6] + mcy;
            Bm[7] = Br[7] + PT[7] - mcx;
            Bm[8] = Br[8] + PT[8];
        }
        Uv[0] = Bm[2];
        Uv[1] = Bm[5];
        Uv[2] = Bm[8];
#pragma unroll
        for (int k = 0; k < 3; ++k) aba_zput(wsz, B, b, i, k, Uv[k]);
        const int si = i & 1;
#pragma unroll
        for (int k = 0; k < 3; ++k) sh.ub[si][k][lane] = Uv[k];
        if (i == 0) sh.flags[1][lane] = timeout << 1;
        __threadfence_block();
        cnt[kTriUB * 32 + lane] = i;
    }
}

// Three warps per 32 instances: warp 0 JA, warp 1 JB, warp 2 Z (aba_pair.cuh).
// Arguments as aba_pair_kernel.
template <typename T, typename D, typename TB, int TRIG>
__global__ void __launch_bounds__(96)
aba_tri_kernel(const T *__restrict__ sc, const D *__restrict__ sd, const DF *__restrict__ sdf,
               int n, int B, const T *__restrict__ q, const T *__restrict__ qd,
               const T *__restrict__ tau, T *__restrict__ qdd_out, int *__restrict__ status,
               T *__restrict__ ws, D *__restrict__ wsz, BaseParams<T> base)
{
    __shared__ AbaTriShared<D> sh;
    const int role = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * 32 + lane;
    if (role == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sh.cnt[k][lane] = n;
        sh.flags[0][lane] = 0;
        sh.flags[1][lane] = 0;
    }
    __syncthreads();
    if (b >= B) return;  // all three lanes of an idle instance; nothing waits on them
    const size_t row = (size_t)b * (size_t)n;
    if (role == 0) {
        aba_tri_ja<T, D, TB, TRIG>(sc, sd, sdf, n, q + row, wsz, B, b, sh, lane);
    } else if (role == 1) {
        aba_tri_jb<T, D, TB, TRIG>(sc, sd, sdf, n, q + row, wsz, B, b, sh, lane);
    } else {
        const volatile int *cnt = &sh.cnt[0][0];
        const int st = aba_pair_z<T, D, TB, TRIG>(
            sc, sd, sdf, n, q + row, qd + row, tau + row, qdd_out + row, ws, wsz, B, b, base,
            cnt + kTriUA * 32 + lane, cnt + kTriUB * 32 + lane, &sh.flags[0][lane],
            &sh.flags[1][lane]);
        if (status) status[b] = st;
    }
}

}  // namespace rdyn
