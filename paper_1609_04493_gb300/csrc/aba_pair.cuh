// aba_pair.cuh -- forward dynamics (aba_dh.cuh) with two warps per 32
// instances: one runs the articulated-inertia recursion, the other everything
// else, concurrently.
//
// In the articulated-body algorithm (Sec. II-B) the nonlinear recursion of
// Eq. (abi) depends on the joint angles only, not on qd or tau, so it can run
// beside the bias sweeps instead of after them:
//   warp J (lane = instance): tip to base, J_hat_i from J_hat_{i+1} (the
//     structured update of aba_dh.cuh), U_i = J_hat_i S_i and 1 / Omega_i into
//     the workspace, then the lane's progress counter in shared memory;
//   warp Z (the same instances): sweep 1 (bias motion and wrenches), then tip
//     to base the wrench carry, tau_hat, and for each link, once warp J has
//     published it, c_hat_i and z_hat (Eq. recursive-fd); then sweep 3.
// Warp J never waits; warp Z waits on the counter with a bounded spin (about
// a second) and flags RD_WARN_TIMEOUT if it ever runs out. The split pays most
// where the bias sweeps are long: beyond 64 links they run in double-float
// (RD_ABA_EXTENDED_BIAS), and then the two warps carry similar loads.
// Constants and records in global memory; any n <= RD_MAX_LINKS, element loads.
// The workspace is that of aba_dh.cuh (sweep-1 state, then U, c_hat, 1/Omega).
#pragma once
#include <type_traits>

#include "aba_dh.cuh"

namespace rdyn {

// Spin bound of warp Z's wait: 2^22 polls with a 64 ns pause, a quarter of a
// second or more. After one timeout a lane waits no more (its result is
// flagged RD_WARN_TIMEOUT), so one instance never spins longer than that.
constexpr int kAbaPairSpinLimit = 1 << 22;

// Bounded wait of one lane until both counters have reached link i or below
// (pu == pv for a single producer), then the fence that orders the producer's
// stores before this lane's loads. After one timeout a lane waits no more.
__device__ __forceinline__ void aba_wait2(const volatile int *pu, const volatile int *pv, int i,
                                          int &timeout)
{
    for (int it = 0; !timeout && (*pu > i || *pv > i); ++it) {
        if (it >= kAbaPairSpinLimit) {
            timeout = 1;
            break;
        }
        __nanosleep(64);
    }
    __threadfence_block();
}

// sin / cos of link i in the bias precision TB, as sweep 1 forms them
template <typename T, typename TB, int TRIG>
__device__ __forceinline__ void aba_trig_tb(const T *__restrict__ sc, const DF *__restrict__ sdf,
                                            const T *__restrict__ qr, int i, TB &s, TB &c)
{
    if constexpr (!std::is_same<TB, T>::value)
        df_sincos((double)__ldg(qr + i) + df_to_double(sdf[i * kAbaDh64 + 5]), &s, &c);
    else
        dh_trig<T, TRIG>(__ldg(qr + i) + sc[i * kDhConsts + 5], &s, &c);
}

// Warp J's share of one instance: the articulated inertias, tip to base; U_i
// and 1 / Omega_i into the workspace slots (wsz, B, b), then *progress = i.
// *jbad: 1 if some Omega_i was not positive, written before the last
// publication.
template <typename T, typename D, typename TB, int TRIG>
__device__ __forceinline__ void aba_pair_j(const T *__restrict__ sc, const D *__restrict__ sd,
                                           const DF *__restrict__ sdf, int n,
                                           const T *__restrict__ qr, D *__restrict__ wsz, int B,
                                           int b, volatile int *progress, int *jbad)
{
    auto trig_tb = [&](int i, TB &s, TB &c) { aba_trig_tb<T, TB, TRIG>(sc, sdf, qr, i, s, c); };
    // ---- warp J: the articulated inertias, tip to base
    int bad = 0;
    AbiT<D> Jh;
    D Uv[3], Uw[3], invOm = D(0);
#pragma unroll 1
    for (int i = n - 1; i >= 0; --i) {
        const D *ri = sd + i * kAbaDh64;
        if (i > 0) {
            prefetch_l1(sd + (i - 1) * kAbaDh64);
            prefetch_l1(sd + (i - 1) * kAbaDh64 + kAbaDh64 / 2);
        }
        if (i == n - 1) {
            const D m = ri[6], zero = D(0);
            Jh.A = Sym3<D>{m, m, m, zero, zero, zero};
            Jh.Bm[0] = zero;    Jh.Bm[1] = ri[18];  Jh.Bm[2] = -ri[17];
            Jh.Bm[3] = -ri[18]; Jh.Bm[4] = zero;    Jh.Bm[5] = ri[16];
            Jh.Bm[6] = ri[17];  Jh.Bm[7] = -ri[16]; Jh.Bm[8] = zero;
            Jh.C = Sym3<D>{ri[19], ri[20], ri[21], ri[22], ri[23], ri[24]};
        } else {
            AbiT<D> P;
            const D ux = Uv[0] * invOm, uy = Uv[1] * invOm, uz = Uv[2] * invOm;
            const D wx = Uw[0] * invOm, wy = Uw[1] * invOm;
            P.A = Sym3<D>{fma(-ux, Uv[0], Jh.A.xx), fma(-uy, Uv[1], Jh.A.yy),
                          fma(-uz, Uv[2], Jh.A.zz), fma(-ux, Uv[1], Jh.A.xy),
                          fma(-ux, Uv[2], Jh.A.xz), fma(-uy, Uv[2], Jh.A.yz)};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                P.Bm[3 * r] = fma(-Uv[r], wx, Jh.Bm[3 * r]);
                P.Bm[3 * r + 1] = fma(-Uv[r], wy, Jh.Bm[3 * r + 1]);
                P.Bm[3 * r + 2] = D(0);
            }
            P.C = Sym3<D>{fma(-wx, Uw[0], Jh.C.xx), fma(-wy, Uw[1], Jh.C.yy), D(0),
                          fma(-wx, Uw[1], Jh.C.xy), D(0), D(0)};
            TB s1, c1;
            trig_tb(i + 1, s1, c1);
            Jh = aba_dh_update(P, dcvt<D>(c1), dcvt<D>(s1), sd + (i + 1) * kAbaDh64, ri);
        }
        Uv[0] = Jh.Bm[2]; Uv[1] = Jh.Bm[5]; Uv[2] = Jh.Bm[8];
        Uw[0] = Jh.C.xz;  Uw[1] = Jh.C.yz;  Uw[2] = Jh.C.zz;
        const D Om = Jh.C.zz;
        if (!dpositive(Om)) bad = 1;
        invOm = drecip(Om);
        {
            const D vals[6] = {Uv[0], Uv[1], Uv[2], Uw[0], Uw[1], Uw[2]};
#pragma unroll
            for (int k = 0; k < 6; ++k) aba_zput(wsz, B, b, i, k, vals[k]);
            aba_zput(wsz, B, b, i, 7, invOm);
        }
        if (i == 0) *jbad = bad;
        __threadfence_block();
        *progress = i;
    }
}

// Warp Z's share of one instance: sweep 1, then sweep 2's wrench carry and
// z_hat / c_hat as U_i and 1 / Omega_i arrive (both counters pu, pv at i or
// below), then sweep 3. jbu, jbv: the producers' flag words (bit 0: a
// non-positive Omega_i, bit 1: a producer timed out). Returns the status word.
template <typename T, typename D, typename TB, int TRIG>
__device__ __forceinline__ int aba_pair_z(const T *__restrict__ sc, const D *__restrict__ sd,
                                          const DF *__restrict__ sdf, int n,
                                          const T *__restrict__ qr, const T *__restrict__ qdr,
                                          const T *__restrict__ taur, T *__restrict__ qddr,
                                          T *__restrict__ ws, D *__restrict__ wsz, int B, int b,
                                          const BaseParams<T> &base, const volatile int *pu,
                                          const volatile int *pv, const int *jbu, const int *jbv)
{
    constexpr bool kExt = !std::is_same<TB, T>::value;
    auto trig_tb = [&](int i, TB &s, TB &c) { aba_trig_tb<T, TB, TRIG>(sc, sdf, qr, i, s, c); };


    // ---- warp Z. Sweep 1: bias motion (qdd = 0) and bias wrenches, base to tip
    Motion<TB> x;
    x.v = mk3(dcvt<TB>(base.V0[0]), dcvt<TB>(base.V0[1]), dcvt<TB>(base.V0[2]));
    x.w = mk3(dcvt<TB>(base.V0[3]), dcvt<TB>(base.V0[4]), dcvt<TB>(base.V0[5]));
    x.a = mk3(dcvt<TB>(base.dV0[0]), dcvt<TB>(base.dV0[1]), dcvt<TB>(base.dV0[2]));
    x.al = mk3(dcvt<TB>(base.dV0[3]), dcvt<TB>(base.dV0[4]), dcvt<TB>(base.dV0[5]));
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        TB s, c;
        trig_tb(i, s, c);
        Wrench<TB> Fh;
        if constexpr (kExt) {
            const DF *r = sdf + i * kAbaDh64;
            if (i + 1 < n) {
                prefetch_l1(r + kAbaDh64);
                prefetch_l1(r + kAbaDh64 + kAbaDh64 / 2);
            }
            x = dh_forward(dh_rot(r[0], r[1], c, s), mk3(r[2], r[3], r[4]),
                           DF(__ldg(qdr + i)), DF(0.0f), x);
            Fh = bias_wrench(r[6], mk3(r[7], r[8], r[9]), r + 10, x);
        } else {
            if (i + 1 < n) prefetch_l1(sc + (i + 1) * kDhConsts);
            DhLink<T> L;
            load_dh(sc + i * kDhConsts, L);
            x = dh_forward(dh_rot(L.ca, L.sa, c, s), L.b, __ldg(qdr + i), T(0), x);
            Fh = bias_wrench(L.m, L.c, L.I, x);
        }
        {
            const TB vals[8] = {Fh.f.x, Fh.f.y, Fh.f.z, Fh.n.x, Fh.n.y, Fh.n.z, c, s};
#pragma unroll
            for (int k = 0; k < 8; ++k) bias_put<TB>(ws, B, b, i, k, vals[k]);
        }
    }

    // Sweep 2 (warp Z's part): wrench carry, tau_hat, c_hat, z_hat, tip to base
    int timeout = 0;
    Wrench<TB> F;
    F.f = mk3(dcvt<TB>(base.Fn[0]), dcvt<TB>(base.Fn[1]), dcvt<TB>(base.Fn[2]));
    F.n = mk3(dcvt<TB>(base.Fn[3]), dcvt<TB>(base.Fn[4]), dcvt<TB>(base.Fn[5]));
    Wrench<D> z;
    z.f = z.n = mk3(D(0), D(0), D(0));
    DhRot<TB> Rn = dh_rot(dcvt<TB>(T(1)), dcvt<TB>(T(0)), dcvt<TB>(T(1)), dcvt<TB>(T(0)));
    V3<TB> bn = mk3(dcvt<TB>(T(0)), dcvt<TB>(T(0)), dcvt<TB>(T(0)));
    DhRot<D> RnZ = dh_rot(D(1), D(0), D(1), D(0));
    V3<D> bnZ = mk3(D(0), D(0), D(0));
    D Up[6] = {D(0), D(0), D(0), D(0), D(0), D(0)}, chat_up = D(0);
    // warp J's values, ordered after its progress store by the fences (the
    // message-passing pattern at block scope)
    auto ldz = [&](int i, int k) -> D { return aba_zget(wsz, B, b, i, k); };
#pragma unroll 1
    for (int i = n - 1; i >= 0; --i) {
        Wrench<TB> Fh;
        Fh.f = mk3(bias_get<TB>(ws, B, b, i, 0), bias_get<TB>(ws, B, b, i, 1),
                   bias_get<TB>(ws, B, b, i, 2));
        Fh.n = mk3(bias_get<TB>(ws, B, b, i, 3), bias_get<TB>(ws, B, b, i, 4),
                   bias_get<TB>(ws, B, b, i, 5));
        const TB c = bias_get<TB>(ws, B, b, i, 6), s = bias_get<TB>(ws, B, b, i, 7);
        if (i == n - 1) {
            F.f = add3(F.f, Fh.f);
            F.n = add3(F.n, Fh.n);
        } else {
            F = dh_carry(Rn, bn, F, Fh);
            // z_hat_i = X^T (z_hat_{i+1} + U_{i+1} c_hat_{i+1})
            Wrench<D> zz;
            zz.f = mk3(fma(Up[0], chat_up, z.f.x), fma(Up[1], chat_up, z.f.y),
                       fma(Up[2], chat_up, z.f.z));
            zz.n = mk3(fma(Up[3], chat_up, z.n.x), fma(Up[4], chat_up, z.n.y),
                       fma(Up[5], chat_up, z.n.z));
            z.f = dh_mul(RnZ, zz.f);
            z.n = cross_add(bnZ, z.f, dh_mul(RnZ, zz.n));
        }
        D tau_hat;
        if constexpr (kExt) tau_hat = dcvt<D>(DF(__ldg(taur + i)) - F.n.z);
        else tau_hat = dsub_exact<D>(__ldg(taur + i), F.n.z);
        // U_i and 1 / Omega_i from warp J
        aba_wait2(pu, pv, i, timeout);
#pragma unroll
        for (int k = 0; k < 6; ++k) Up[k] = ldz(i, k);
        const D invOm = ldz(i, 7);
        chat_up = (tau_hat - z.n.z) * invOm;
        aba_zput(wsz, B, b, i, 6, chat_up);
        const D *ri = sd + i * kAbaDh64;
        if constexpr (kExt) {
            const DF *rf = sdf + i * kAbaDh64;
            Rn = dh_rot(rf[0], rf[1], c, s);
            bn = mk3(rf[2], rf[3], rf[4]);
        } else {
            const T *Lt = sc + i * kDhConsts;
            Rn = dh_rot(Lt[0], Lt[1], c, s);
            bn = mk3(Lt[2], Lt[3], Lt[4]);
        }
        RnZ = dh_rot(ri[0], ri[1], dcvt<D>(c), dcvt<D>(s));
        bnZ = mk3(ri[2], ri[3], ri[4]);
    }

    // Sweep 3: lambda and qdd, base to tip
    const int jb = *jbu | *jbv;
    int bad = jb & 1;
    timeout |= (jb >> 1) & 1;
    V3<D> lv = mk3(D(0), D(0), D(0)), lw = mk3(D(0), D(0), D(0));
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        const TB c = bias_get<TB>(ws, B, b, i, 6), s = bias_get<TB>(ws, B, b, i, 7);
        const D *ri = sd + i * kAbaDh64;
        const DhRot<D> R = dh_rot(ri[0], ri[1], dcvt<D>(c), dcvt<D>(s));
        const V3<D> bi = mk3(ri[2], ri[3], ri[4]);
        V3<D> av = dh_mulT(R, cross_add(lw, bi, lv)), aw = dh_mulT(R, lw);
        D ua = ldz(i, 0) * av.x;
        ua = fma(ldz(i, 1), av.y, ua);
        ua = fma(ldz(i, 2), av.z, ua);
        ua = fma(ldz(i, 3), aw.x, ua);
        ua = fma(ldz(i, 4), aw.y, ua);
        ua = fma(ldz(i, 5), aw.z, ua);
        const D qdd_i = fma(-ldz(i, 7), ua, ldz(i, 6));
        aw.z = aw.z + qdd_i;
        lv = av;
        lw = aw;
        if (disnan(qdd_i)) bad = 1;
        qddr[i] = dcvt<T>(qdd_i);
    }
    return (bad ? RD_WARN_SINGULAR : 0) | (timeout ? RD_WARN_TIMEOUT : 0);
}

// One instance's share of the work for one of the two warps (role 0: J, role
// 1: Z). The caller sets *progress to n or more (nothing published) and *jbad
// to 0, and makes both visible to the pair, before either role starts. qr, qdr,
// taur, qddr: the instance's rows; ws / wsz with (B, b): its workspace slots.
// Role Z returns the status word, role J 0. The body synchronises with nothing
// but its partner lane's progress counter: callers may run it on any subset of
// a warp's lanes (fleets mix request kinds within a warp).
template <typename T, typename D, typename TB, int TRIG>
__device__ __forceinline__ int aba_pair_role(int role, const T *__restrict__ sc,
                                             const D *__restrict__ sd,
                                             const DF *__restrict__ sdf, int n,
                                             const T *__restrict__ qr, const T *__restrict__ qdr,
                                             const T *__restrict__ taur, T *__restrict__ qddr,
                                             T *__restrict__ ws, D *__restrict__ wsz, int B,
                                             int b, const BaseParams<T> &base,
                                             volatile int *progress, int *jbad)
{
    if (role == 0) {
        aba_pair_j<T, D, TB, TRIG>(sc, sd, sdf, n, qr, wsz, B, b, progress, jbad);
        return 0;
    }
    return aba_pair_z<T, D, TB, TRIG>(sc, sd, sdf, n, qr, qdr, taur, qddr, ws, wsz, B, b, base,
                                      progress, progress, jbad, jbad);
}

// withhold (a test hook, RD_ABA_TEST_WITHHOLD): warp J publishes into a counter
// that warp Z does not read, so every wait of warp Z runs out and reports
// RD_WARN_TIMEOUT.
template <typename T, typename D, typename TB, int TRIG>
__global__ void __launch_bounds__(64)
aba_pair_kernel(const T *__restrict__ sc, const D *__restrict__ sd, const DF *__restrict__ sdf,
                int n, int B, const T *__restrict__ q, const T *__restrict__ qd,
                const T *__restrict__ tau, T *__restrict__ qdd_out, int *__restrict__ status,
                T *__restrict__ ws, D *__restrict__ wsz, BaseParams<T> base, int withhold)
{
    __shared__ volatile int progress[32];
    __shared__ volatile int withheld[32];
    __shared__ int jbad[32];
    const int role = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * 32 + lane;
    if (role == 0) {
        progress[lane] = n;
        jbad[lane] = 0;
    }
    __syncthreads();
    if (b >= B) return;  // both lanes of an idle instance; nothing waits on them
    const size_t row = (size_t)b * (size_t)n;
    const int st = aba_pair_role<T, D, TB, TRIG>(role, sc, sd, sdf, n, q + row, qd + row, tau + row,
                                                 qdd_out + row, ws, wsz, B, b, base,
                                                 (role == 0 && withhold) ? &withheld[lane]
                                                                         : &progress[lane],
                                                 &jbad[lane]);
    if (role == 1 && status) status[b] = st;
}

}  // namespace rdyn
