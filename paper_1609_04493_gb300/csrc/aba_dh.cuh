// aba_dh.cuh -- forward dynamics by the articulated-body algorithm (aba.cuh:
// Sec. II-B, Eqs. abi and recursive-fd) in the common-normal frames of
// spatial_dh.cuh. aba_dh_kernel takes the link constants as a __grid_constant__
// kernel parameter (n % 4 == 0, n <= NMAX, 16-byte aligned rows);
// aba_dhg_kernel reads them from global memory (any n, any rows); fleets call
// the same per-instance body.
//
// The sweeps and the precision split are those of aba.cuh. What changes is the
// articulated-inertia update
//     J_hat_i = J_i + X^T P X,   P = J_hat_{i+1} - U U^T / Omega_{i+1},
//     X = Ad_{f_{i+1}^-1},  f = (Rx(alpha) Rz(theta), b):
// * P S = U - U (U^T S) / Omega = 0 for S = e_z (angular), so P has a zero w_z
//   row and column: of its lower-right block only the xy part is nonzero and
//   the last column of its off-diagonal block vanishes. Only the nonzero
//   entries are formed.
// * The rotation R = Rx(alpha) Rz(theta) is applied as two plane rotations. A
//   plane rotation of a symmetric block needs its 2x2 part in double-angle form
//   (cos 2 theta, sin 2 theta) and the two couplings; the rotation about z keeps
//   P's zeros, and the one about x acts on an angular block that has only its
//   xy part.
// * Then the shift by b, as in aba.cuh.
// J_i about the frame origin is precomputed on the host (FP64 record below).
//
// The scalar D of the inertia update and the solves is double, or for FP32
// data (the default there) the double-float pair of df.cuh (about 48 bits,
// computed on the FP32 pipe): the records then hold each FP64 constant split
// into a pair on the host, and the z_hat / lambda recursions run in D too.
#pragma once
#include <type_traits>

#include "aba.cuh"
#include "df.cuh"
#include "df_trig.cuh"
#include "rnea_dhp.cuh"

namespace rdyn {

// Hint: bring the 128-byte line holding p into L1 ahead of its use. Only for
// addresses in global memory (not kernel parameters).
__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.L1 [%0];" ::"l"(p));
}

// FP64 record of a link: the 16 common-normal constants (spatial_dh.cuh), then
// m c (3), the rotational inertia about the frame origin C_o = I_c + m (|c|^2 -
// c c^T) (xx, yy, zz, xy, xz, yz), and cos^2 alpha, sin^2 alpha, cos alpha sin
// alpha, cos 2 alpha, sin 2 alpha; 2 pad.
constexpr int kAbaDh64 = 32;

// D: double, or DF (df.cuh) for the double-float variant
template <typename T, typename D, int NMAX>
struct AbaDhConsts {
    T c[NMAX * kDhConsts];    // in the data precision, for the FP32 (or FP64) sweeps
    D d[NMAX * kAbaDh64];
};

// S' = Rz S Rz^T for symmetric S (double angle c2 = cos 2t, s2 = sin 2t)
template <typename D>
__device__ __forceinline__ Sym3<D> rotz_sym(const Sym3<D> &S, D c, D s, D c2, D s2)
{
    const D h = dhalf(S.xx + S.yy), d = dhalf(S.xx - S.yy);
    const D t = fma(d, c2, -S.xy * s2);
    return Sym3<D>{h + t, h - t, S.zz, fma(d, s2, S.xy * c2), fma(c, S.xz, -s * S.yz),
                   fma(s, S.xz, c * S.yz)};
}

// S' = Rx S Rx^T for symmetric S: the (y, z) plane
template <typename D>
__device__ __forceinline__ Sym3<D> rotx_sym(const Sym3<D> &S, D ca, D sa, D c2, D s2)
{
    const D h = dhalf(S.yy + S.zz), d = dhalf(S.yy - S.zz);
    const D t = fma(d, c2, -S.yz * s2);
    return Sym3<D>{S.xx, h + t, h - t, fma(ca, S.xy, -sa * S.xz), fma(sa, S.xy, ca * S.xz),
                   fma(d, s2, S.yz * c2)};
}

// X^T P X + J_i for the projected articulated inertia P of link i+1 (zero w_z
// row and column) and the transform of link i+1 (cos/sin of theta, record r).
template <typename D>
__device__ __forceinline__ AbiT<D> aba_dh_update(const AbiT<D> &P, D c, D s, const D *r,
                                                 const D *ri)
{
    const D ca = r[0], sa = r[1];
    const D ca2 = r[25], sa2 = r[26], casa = r[27], c2a = r[28], s2a = r[29];
    const D c2 = fma(c, c, -s * s), s2 = dtwice(c * s);
    // rotation about z: A full, Bm with a zero last column, C with its xy part only
    AbiT<D> M;
    M.A = rotz_sym(P.A, c, s, c2, s2);
    D B1[6];  // rows 0..2, columns 0..1 of Rz Bm (rows mixed)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        B1[k] = fma(c, P.Bm[k], -s * P.Bm[3 + k]);
        B1[2 + k] = fma(s, P.Bm[k], c * P.Bm[3 + k]);
        B1[4 + k] = P.Bm[6 + k];
    }
    D B2[6];  // then columns mixed (Bm Rz^T)
#pragma unroll
    for (int rr = 0; rr < 3; ++rr) {
        B2[2 * rr] = fma(c, B1[2 * rr], -s * B1[2 * rr + 1]);
        B2[2 * rr + 1] = fma(s, B1[2 * rr], c * B1[2 * rr + 1]);
    }
    const D hc = dhalf(P.C.xx + P.C.yy), dc = dhalf(P.C.xx - P.C.yy);
    const D tc = fma(dc, c2, -P.C.xy * s2);
    const D Cxx = hc + tc, Cyy = hc - tc, Cxy = fma(dc, s2, P.C.xy * c2);
    // rotation about x
    M.A = rotx_sym(M.A, ca, sa, c2a, s2a);
    // Bm: rows 1, 2 mixed (columns 0, 1), then columns: col1 -> ca col1, col2 = sa col1
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
    M.C = Sym3<D>{Cxx, ca2 * Cyy, sa2 * Cyy, ca * Cxy, sa * Cxy, casa * Cyy};
#pragma unroll
    for (int k = 0; k < 9; ++k) M.Bm[k] = Br[k];
    // shift by b (aba.cuh): A' = A_r, B' = B_r - A_r [b],
    // C' = C_r + [b]B_r - B_r^T[b] - [b]A_r[b]; then + J_i (A = m I, Bm = -[m c], C = C_o)
    const D b[3] = {r[2], r[3], r[4]};
    D Ar[9], Pm[9], PT[9], Nr[9];
    sym_to_full(M.A, Ar);
    hat_mul(b, Ar, Pm);  // [b] A_r; its transpose is -A_r [b]
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) PT[3 * i + j] = Pm[3 * j + i];
    hat_mul(b, M.Bm, Nr);  // [b] B_r
    // -[b] A_r [b] = [b] PT is symmetric: only its upper triangle is formed
    // (row 0 of [b] X: b1 X_2j - b2 X_1j; row 1: b2 X_0j - b0 X_2j; row 2:
    // b0 X_1j - b1 X_0j)
    const D q00 = fma(b[1], PT[6], -b[2] * PT[3]);
    const D q01 = fma(b[1], PT[7], -b[2] * PT[4]);
    const D q02 = fma(b[1], PT[8], -b[2] * PT[5]);
    const D q11 = fma(b[2], PT[1], -b[0] * PT[7]);
    const D q12 = fma(b[2], PT[2], -b[0] * PT[8]);
    const D q22 = fma(b[0], PT[5], -b[1] * PT[2]);
    const D m = ri[6], mcx = ri[16], mcy = ri[17], mcz = ri[18];
    AbiT<D> o;
    o.A = Sym3<D>{M.A.xx + m, M.A.yy + m, M.A.zz + m, M.A.xy, M.A.xz, M.A.yz};
    o.Bm[0] = M.Bm[0] + PT[0];
    o.Bm[1] = M.Bm[1] + PT[1] + mcz;
    o.Bm[2] = M.Bm[2] + PT[2] - mcy;
    o.Bm[3] = M.Bm[3] + PT[3] - mcz;
    o.Bm[4] = M.Bm[4] + PT[4];
    o.Bm[5] = M.Bm[5] + PT[5] + mcx;
    o.Bm[6] = M.Bm[6] + PT[6] + mcy;
    o.Bm[7] = M.Bm[7] + PT[7] - mcx;
    o.Bm[8] = M.Bm[8] + PT[8];
    o.C.xx = dtwice_add(Nr[0], M.C.xx) + q00 + ri[19];
    o.C.yy = dtwice_add(Nr[4], M.C.yy) + q11 + ri[20];
    o.C.zz = dtwice_add(Nr[8], M.C.zz) + q22 + ri[21];
    o.C.xy = M.C.xy + Nr[1] + Nr[3] + q01 + ri[22];
    o.C.xz = M.C.xz + Nr[2] + Nr[6] + q02 + ri[23];
    o.C.yz = M.C.yz + Nr[5] + Nr[7] + q12 + ri[24];
    return o;
}

// Sweep-1 state of a link, F_hat (6) then cos, sin, in the bias precision TB:
// for TB = T the slots 0..5, 8, 9 of the kAbaStateScalars-wide layout; for TB
// = DF eight pairs per link, [link][8][instance], in the same workspace
// (aba_bias_ws_scalars floats per link and instance).
constexpr int kAbaBiasPairs = 8;

template <typename T, typename TB>
__host__ __device__ constexpr int aba_bias_ws_scalars()
{
    return std::is_same<TB, T>::value ? kAbaStateScalars : 2 * kAbaBiasPairs;
}

template <typename TB, typename T>
__device__ __forceinline__ void bias_put(T *ws, int B, int b, int i, int k, TB v)
{
    if constexpr (std::is_same<TB, T>::value) {
        aba_put(ws, B, b, i, k < 6 ? k : k + 2, v);
    } else {
        TB *w = reinterpret_cast<TB *>(ws);
        w[((size_t)i * kAbaBiasPairs + k) * (size_t)B + b] = v;
    }
}

template <typename TB, typename T>
__device__ __forceinline__ TB bias_get(const T *ws, int B, int b, int i, int k)
{
    if constexpr (std::is_same<TB, T>::value) {
        return aba_get(ws, B, b, i, k < 6 ? k : k + 2);
    } else {
        const TB *w = reinterpret_cast<const TB *>(ws);
        return w[((size_t)i * kAbaBiasPairs + k) * (size_t)B + b];
    }
}

// One forward-dynamics instance in common-normal frames. sc: the chain's 16
// constants per link in T; sd: its records in D (FP64, or split into
// double-float pairs); qr, qdr, taur, qddr: its joint rows (VEC: n % 4 == 0 and
// 16-byte aligned, else element loads); ws / wsz and (B, b): its workspace
// (aba_put; Z is the type of the solve state and of the z_hat / lambda
// recursions: D, or T). PF: constants, records and workspace live in global
// memory (fleets), and each sweep prefetches the next link's into L1 while it
// computes the current one. TB: precision of the bias sweeps (the motion and
// bias wrenches of sweep 1, the wrench carry and tau_hat of sweep 2) and of the
// joint sin/cos: T, or DF for long chains, whose bias torques grow far above
// tau so that FP32 rounding there sets the error of qdd; with TB = DF they run
// on sdf, the chain's records as double-float pairs, with the sin/cos of
// df_trig.cuh. Returns 1 when an Omega_i <= 0 or a non-finite qdd appeared.
template <typename T, typename D, typename Z, int TRIG, bool VEC, bool PF = false,
          typename TB = T>
__device__ __forceinline__ int aba_dh_instance(const T *sc, const D *sd, int n,
                                               const T *__restrict__ qr, const T *__restrict__ qdr,
                                               const T *__restrict__ taur, T *__restrict__ qddr,
                                               T *__restrict__ ws, Z *__restrict__ wsz, int B, int b,
                                               const BaseParams<T> &base,
                                               const DF *__restrict__ sdf = nullptr)
{
    constexpr bool kExt = !std::is_same<TB, T>::value;
    static_assert(!kExt || (std::is_same<TB, DF>::value && sizeof(T) == 4),
                  "extended bias sweeps: double-float, FP32 data");
    int bad = 0;

    // ---- sweep 1: bias motion (qdd = 0) and bias wrenches
    Motion<TB> x;
    x.v = mk3(dcvt<TB>(base.V0[0]), dcvt<TB>(base.V0[1]), dcvt<TB>(base.V0[2]));
    x.w = mk3(dcvt<TB>(base.V0[3]), dcvt<TB>(base.V0[4]), dcvt<TB>(base.V0[5]));
    x.a = mk3(dcvt<TB>(base.dV0[0]), dcvt<TB>(base.dV0[1]), dcvt<TB>(base.dV0[2]));
    x.al = mk3(dcvt<TB>(base.dV0[3]), dcvt<TB>(base.dV0[4]), dcvt<TB>(base.dV0[5]));
    const int nchunks = (n + 3) / 4;
    for (int kc = 0; kc < nchunks; ++kc) {
        const int i0 = 4 * kc;
        const Chunk<T> cq = ld_chunk<T, VEC>(qr, i0, n), cqd = ld_chunk<T, VEC>(qdr, i0, n);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            if (VEC || i < n) {
                TB s, c;
                Wrench<TB> Fh;
                if constexpr (kExt) {
                    const DF *r = sdf + i * kAbaDh64;
                    if (PF && i + 1 < n) {
                        prefetch_l1(r + kAbaDh64);
                        prefetch_l1(r + kAbaDh64 + kAbaDh64 / 2);
                    }
                    df_sincos((double)cq.v[j] + df_to_double(r[5]), &s, &c);
                    x = dh_forward(dh_rot(r[0], r[1], c, s), mk3(r[2], r[3], r[4]),
                                   DF(cqd.v[j]), DF(0.0f), x);
                    Fh = bias_wrench(r[6], mk3(r[7], r[8], r[9]), r + 10, x);
                } else {
                    if (PF && i + 1 < n) prefetch_l1(sc + (i + 1) * kDhConsts);
                    DhLink<T> L;
                    load_dh(sc + i * kDhConsts, L);
                    dh_trig<T, TRIG>(cq.v[j] + L.th0, &s, &c);
                    x = dh_forward(dh_rot(L.ca, L.sa, c, s), L.b, cqd.v[j], T(0), x);
                    Fh = bias_wrench(L.m, L.c, L.I, x);
                }
                const TB vals[8] = {Fh.f.x, Fh.f.y, Fh.f.z, Fh.n.x, Fh.n.y, Fh.n.z, c, s};
#pragma unroll
                for (int k = 0; k < 8; ++k) bias_put<TB>(ws, B, b, i, k, vals[k]);
            }
        }
    }

    // ---- sweep 2: tau_hat, articulated inertias (D), z_hat, c_hat
    // (Z = D: the transform of the z_hat step comes from the D records)
    constexpr bool kZrec = std::is_same<Z, D>::value;
    // The double-float body is about ten times the FP64 one in instructions:
    // unrolled four links deep it no longer fits the instruction cache, and
    // at one warp per scheduler every miss stalls issue. Its sweeps run one
    // link per iteration.
    constexpr bool kRolled = std::is_same<D, DF>::value;
    Wrench<TB> F;
    F.f = mk3(dcvt<TB>(base.Fn[0]), dcvt<TB>(base.Fn[1]), dcvt<TB>(base.Fn[2]));
    F.n = mk3(dcvt<TB>(base.Fn[3]), dcvt<TB>(base.Fn[4]), dcvt<TB>(base.Fn[5]));
    Wrench<Z> z;
    z.f = z.n = mk3(Z(0), Z(0), Z(0));
    AbiT<D> Jh;
    D Uv[3] = {D(0), D(0), D(0)}, Uw[3] = {D(0), D(0), D(0)}, invOm = D(0), chat = D(0);
    DhRot<TB> Rn = dh_rot(dcvt<TB>(T(1)), dcvt<TB>(T(0)), dcvt<TB>(T(1)), dcvt<TB>(T(0)));
    V3<TB> bn = mk3(dcvt<TB>(T(0)), dcvt<TB>(T(0)), dcvt<TB>(T(0)));
    DhRot<Z> RnZ = dh_rot(Z(1), Z(0), Z(1), Z(0));
    V3<Z> bnZ = mk3(Z(0), Z(0), Z(0));
    D cn = D(1), sn = D(0);  // cos, sin of link i+1 in D
    // one link of the sweep, given tau_i
    auto step2 = [&](int i, T tau_i) {
        if (PF && i > 0) {  // link i-1: records, constants, workspace
            const D *rp = sd + (i - 1) * kAbaDh64;
            prefetch_l1(rp);
            prefetch_l1(rp + kAbaDh64 / 2);
            prefetch_l1(sc + (i - 1) * kDhConsts);
            if constexpr (kExt) {
                prefetch_l1(sdf + (i - 1) * kAbaDh64);
                prefetch_l1(reinterpret_cast<const DF *>(ws) +
                            (size_t)(i - 1) * kAbaBiasPairs * B + b);
            } else {
                prefetch_l1(&ws[(size_t)(i - 1) * kAbaStateScalars * B + b]);
            }
        }
        Wrench<TB> Fh;
        Fh.f = mk3(bias_get<TB>(ws, B, b, i, 0), bias_get<TB>(ws, B, b, i, 1),
                   bias_get<TB>(ws, B, b, i, 2));
        Fh.n = mk3(bias_get<TB>(ws, B, b, i, 3), bias_get<TB>(ws, B, b, i, 4),
                   bias_get<TB>(ws, B, b, i, 5));
        const TB c = bias_get<TB>(ws, B, b, i, 6), s = bias_get<TB>(ws, B, b, i, 7);
        const D *ri = sd + i * kAbaDh64;
        if (i == n - 1) {
            F.f = add3(F.f, Fh.f);
            F.n = add3(F.n, Fh.n);
            const D m = ri[6], zero = D(0);
            Jh.A = Sym3<D>{m, m, m, zero, zero, zero};
            Jh.Bm[0] = zero;    Jh.Bm[1] = ri[18];  Jh.Bm[2] = -ri[17];
            Jh.Bm[3] = -ri[18]; Jh.Bm[4] = zero;    Jh.Bm[5] = ri[16];
            Jh.Bm[6] = ri[17];  Jh.Bm[7] = -ri[16]; Jh.Bm[8] = zero;
            Jh.C = Sym3<D>{ri[19], ri[20], ri[21], ri[22], ri[23], ri[24]};
        } else {
            F = dh_carry(Rn, bn, F, Fh);
            // P = J_hat_{i+1} - U U^T / Omega: its w_z row and column vanish
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
            Jh = aba_dh_update(P, cn, sn, sd + (i + 1) * kAbaDh64, ri);
            // z_hat_i = X^T (z_hat_{i+1} + U_{i+1} c_hat_{i+1})
            Wrench<Z> zz;
            if constexpr (kZrec) {  // one fused multiply-add per component
                zz.f = mk3(fma(Uv[0], chat, z.f.x), fma(Uv[1], chat, z.f.y),
                           fma(Uv[2], chat, z.f.z));
                zz.n = mk3(fma(Uw[0], chat, z.n.x), fma(Uw[1], chat, z.n.y),
                           fma(Uw[2], chat, z.n.z));
            } else {
                zz.f = mk3(z.f.x + dcvt<Z>(Uv[0] * chat), z.f.y + dcvt<Z>(Uv[1] * chat),
                           z.f.z + dcvt<Z>(Uv[2] * chat));
                zz.n = mk3(z.n.x + dcvt<Z>(Uw[0] * chat), z.n.y + dcvt<Z>(Uw[1] * chat),
                           z.n.z + dcvt<Z>(Uw[2] * chat));
            }
            // z_hat_i = Ad^T zz: the carry of spatial_dh.cuh without a wrench to add
            // (adding zeros is not an identity in IEEE arithmetic, so it would run)
            z.f = dh_mul(RnZ, zz.f);
            z.n = cross_add(bnZ, z.f, dh_mul(RnZ, zz.n));
        }
        D tau_hat;
        if constexpr (kExt) tau_hat = dcvt<D>(DF(tau_i) - F.n.z);
        else tau_hat = dsub_exact<D>(tau_i, F.n.z);
        Uv[0] = Jh.Bm[2]; Uv[1] = Jh.Bm[5]; Uv[2] = Jh.Bm[8];
        Uw[0] = Jh.C.xz; Uw[1] = Jh.C.yz; Uw[2] = Jh.C.zz;
        const D Om = Jh.C.zz;
        if (!dpositive(Om)) bad = 1;
        invOm = drecip(Om);
        chat = (tau_hat - dcvt<D>(z.n.z)) * invOm;
        const Z vals[8] = {dcvt<Z>(Uv[0]), dcvt<Z>(Uv[1]), dcvt<Z>(Uv[2]), dcvt<Z>(Uw[0]),
                           dcvt<Z>(Uw[1]), dcvt<Z>(Uw[2]), dcvt<Z>(chat), dcvt<Z>(invOm)};
#pragma unroll
        for (int k = 0; k < 8; ++k) aba_zput(wsz, B, b, i, k, vals[k]);
        // transform of link i, for the step to link i-1
        const T *Lt = sc + i * kDhConsts;
        if constexpr (kExt) {
            const DF *rf = sdf + i * kAbaDh64;
            Rn = dh_rot(rf[0], rf[1], c, s);
            bn = mk3(rf[2], rf[3], rf[4]);
        } else {
            Rn = dh_rot(Lt[0], Lt[1], c, s);
            bn = mk3(Lt[2], Lt[3], Lt[4]);
        }
        cn = dcvt<D>(c);
        sn = dcvt<D>(s);
        if constexpr (kZrec) {
            RnZ = dh_rot(ri[0], ri[1], cn, sn);
            bnZ = mk3(ri[2], ri[3], ri[4]);
        } else {
            RnZ = dh_rot(dcvt<Z>(Lt[0]), dcvt<Z>(Lt[1]), dcvt<Z>(c), dcvt<Z>(s));
            bnZ = mk3(dcvt<Z>(Lt[2]), dcvt<Z>(Lt[3]), dcvt<Z>(Lt[4]));
        }
    };
    if constexpr (kRolled) {
#pragma unroll 1
        for (int i = n - 1; i >= 0; --i) step2(i, taur[i]);
    } else {
        for (int i0 = ((n - 1) / 4) * 4; i0 >= 0; i0 -= 4) {
            const Chunk<T> ct = ld_chunk<T, VEC>(taur, i0, n);
#pragma unroll
            for (int j = 3; j >= 0; --j)
                if (VEC || i0 + j < n) step2(i0 + j, ct.v[j]);
        }
    }

    // ---- sweep 3: lambda and qdd
    V3<Z> lv = mk3(Z(0), Z(0), Z(0)), lw = mk3(Z(0), Z(0), Z(0));
    // one link of the sweep; returns qdd_i
    auto step3 = [&](int i) -> T {
        if (PF && i + 1 < n) {  // link i+1: records, solve state
            const D *rp = sd + (i + 1) * kAbaDh64;
            prefetch_l1(rp);
            prefetch_l1(rp + kAbaDh64 / 2);
            prefetch_l1(&wsz[(size_t)(i + 1) * kAbaSolveScalars * B + b]);
        }
        const TB c = bias_get<TB>(ws, B, b, i, 6), s = bias_get<TB>(ws, B, b, i, 7);
        DhRot<Z> R;
        V3<Z> bi;
        if constexpr (kZrec) {
            const D *ri = sd + i * kAbaDh64;
            R = dh_rot(ri[0], ri[1], dcvt<D>(c), dcvt<D>(s));
            bi = mk3(ri[2], ri[3], ri[4]);
        } else {
            const T *Lt = sc + i * kDhConsts;
            R = dh_rot(dcvt<Z>(Lt[0]), dcvt<Z>(Lt[1]), dcvt<Z>(c), dcvt<Z>(s));
            bi = mk3(dcvt<Z>(Lt[2]), dcvt<Z>(Lt[3]), dcvt<Z>(Lt[4]));
        }
        // a = Ad_{f^-1} lambda
        V3<Z> av = dh_mulT(R, cross_add(lw, bi, lv)), aw = dh_mulT(R, lw);
        const V3<Z> uv = mk3(aba_zget(wsz, B, b, i, 0), aba_zget(wsz, B, b, i, 1), aba_zget(wsz, B, b, i, 2));
        const V3<Z> uw = mk3(aba_zget(wsz, B, b, i, 3), aba_zget(wsz, B, b, i, 4), aba_zget(wsz, B, b, i, 5));
        const Z ch = aba_zget(wsz, B, b, i, 6), iom = aba_zget(wsz, B, b, i, 7);
        D ua = dcvt<D>(uv.x) * dcvt<D>(av.x);
        ua = fma(dcvt<D>(uv.y), dcvt<D>(av.y), ua);
        ua = fma(dcvt<D>(uv.z), dcvt<D>(av.z), ua);
        ua = fma(dcvt<D>(uw.x), dcvt<D>(aw.x), ua);
        ua = fma(dcvt<D>(uw.y), dcvt<D>(aw.y), ua);
        ua = fma(dcvt<D>(uw.z), dcvt<D>(aw.z), ua);
        const D qdd_i = fma(-dcvt<D>(iom), ua, dcvt<D>(ch));
        aw.z = aw.z + dcvt<Z>(qdd_i);
        lv = av;
        lw = aw;
        if (disnan(qdd_i)) bad = 1;
        return dcvt<T>(qdd_i);
    };
    if constexpr (kRolled) {
#pragma unroll 1
        for (int i = 0; i < n; ++i) qddr[i] = step3(i);
    } else {
        for (int kc = 0; kc < nchunks; ++kc) {
            const int i0 = 4 * kc;
            Chunk<T> out;
#pragma unroll
            for (int j = 0; j < 4; ++j) out.v[j] = (VEC || i0 + j < n) ? step3(i0 + j) : T(0);
            st_chunk<T, VEC>(qddr, i0, n, out);
        }
    }
    return bad;
}

// Minimum resident threads per SM the launch bounds ask for (they cap the
// registers per thread at 65536 / this).
#ifndef RD_ABA_MIN_THREADS_PER_SM
#define RD_ABA_MIN_THREADS_PER_SM 512
#endif
#ifndef RD_ABA_DHG_MIN_THREADS_PER_SM
#define RD_ABA_DHG_MIN_THREADS_PER_SM 384
#endif

template <typename T, typename D, typename Z, int NMAX, int BLOCK, int TRIG>
__global__ void __launch_bounds__(BLOCK, RD_ABA_MIN_THREADS_PER_SM / BLOCK)
aba_dh_kernel(const __grid_constant__ AbaDhConsts<T, D, NMAX> pc, int n, int B,
              const T *__restrict__ q, const T *__restrict__ qd, const T *__restrict__ tau,
              T *__restrict__ qdd_out, int *__restrict__ status, T *__restrict__ ws,
              Z *__restrict__ wsz, BaseParams<T> base)
{
    const int b = blockIdx.x * BLOCK + threadIdx.x;
    if (b >= B) return;
    const size_t row = (size_t)b * (size_t)n;
    const int bad = aba_dh_instance<T, D, Z, TRIG, true>(pc.c, pc.d, n, q + row, qd + row,
                                                         tau + row, qdd_out + row, ws, wsz, B, b,
                                                         base);
    if (status) status[b] = bad ? RD_WARN_SINGULAR : 0;
}

// Forward dynamics with the constants and the records (FP64, or double-float
// pairs) in global memory, for what the parameter space does not take: chains
// longer than 64 links, lengths not a multiple of 4, unaligned rows
// (VEC = false). The sweeps prefetch each next link's constants, records and
// workspace into L1. TB: precision of the bias sweeps (T, or DF on sdf, the
// records as double-float pairs).
template <typename T, typename D, typename Z, int BLOCK, bool VEC, typename TB = T>
__global__ void __launch_bounds__(BLOCK, (sizeof(T) == 8 ? 256 : RD_ABA_DHG_MIN_THREADS_PER_SM) / BLOCK)
aba_dhg_kernel(const T *__restrict__ sc, const D *__restrict__ sd, int n, int B,
               const T *__restrict__ q, const T *__restrict__ qd, const T *__restrict__ tau,
               T *__restrict__ qdd_out, int *__restrict__ status, T *__restrict__ ws,
               Z *__restrict__ wsz, BaseParams<T> base, const DF *__restrict__ sdf)
{
    const int b = blockIdx.x * BLOCK + threadIdx.x;
    if (b >= B) return;
    const size_t row = (size_t)b * (size_t)n;
    const int bad = aba_dh_instance<T, D, Z, kTrigPoly, VEC, true, TB>(
        sc, sd, n, q + row, qd + row, tau + row, qdd_out + row, ws, wsz, B, b, base, sdf);
    if (status) status[b] = bad ? RD_WARN_SINGULAR : 0;
}

}  // namespace rdyn
