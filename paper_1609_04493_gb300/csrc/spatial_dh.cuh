// spatial_dh.cuh -- register-level spatial algebra in common-normal frames.
//
// A refinement of the joint frames of spatial.cuh. Frame D_i of link i has
// its z axis on joint axis i, its origin on that axis, and its x axis along
// the common normal of axes i and i+1 (any normal direction for the last link
// and for parallel axes). Because x_{i-1} is then perpendicular to both
// z_{i-1} and z_i, the rotation between consecutive frames is a rotation
// about x followed by one about z (the Denavit-Hartenberg structure), and the
// link transform of Sec. II-A becomes
//     f_{i-1,i} = (R_i, b_i),   R_i = Rx(alpha_i) Rz(theta0_i + q_i),
// with b_i the origin of D_i in D_{i-1} (a general 3-vector: origins stay at
// the points nearest the user's frames, so no offset grows when two axes are
// close to parallel). Link 0 rotates about the z axis of a base frame D_{-1}
// equal to D_0 at q_0 = 0: alpha_0 = theta0_0 = 0, b_0 = 0. The torques are
// the z moments of the wrenches, exactly as in the joint frames.
//
// Compared with a general constant rotation A_i, applying R_i^T or R_i to a
// vector takes 8 multiply-adds instead of 9 after 4 products per link
// instead of the 12 that form A_i Rz(q_i), and a link needs 16 constants
// instead of 24.
#pragma once
#include "spatial.cuh"

namespace rdyn {

// Constants of link i in frame D_i, 16 scalars (four 16-byte pieces in FP32):
//   [0] cos alpha  [1] sin alpha  [2..4] b  [5] theta0
//   [6] m  [7..9] centre of mass  [10..15] I about the centre of mass
//   (xx, yy, zz, xy, xz, yz).
constexpr int kDhConsts = 16;

template <typename T>
struct DhLink {
    T ca, sa;
    V3<T> b;
    T th0;
    T m;
    V3<T> c;
    T I[6];
};

// The part of a link the motion recursion and the backward carry need.
template <typename T>
struct DhXf {
    T ca, sa;
    V3<T> b;
    T th0;
};

template <typename T>
__device__ __forceinline__ void load_dh(const T *p, DhLink<T> &L)
{
    T v[16];
    if constexpr (sizeof(T) == 4) {
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 t = p4[k];
            v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
        }
    } else {
        const double2 *p2 = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            double2 t = p2[k];
            v[2 * k] = t.x; v[2 * k + 1] = t.y;
        }
    }
    L.ca = v[0]; L.sa = v[1];
    L.b = mk3(v[2], v[3], v[4]);
    L.th0 = v[5];
    L.m = v[6];
    L.c = mk3(v[7], v[8], v[9]);
#pragma unroll
    for (int k = 0; k < 6; ++k) L.I[k] = v[10 + k];
}

template <typename T>
__device__ __forceinline__ void load_dh_xf(const T *p, DhXf<T> &X)
{
    T v[8];
    if constexpr (sizeof(T) == 4) {
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
        float4 a = p4[0], b = p4[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
        const double2 *p2 = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double2 t = p2[k];
            v[2 * k] = t.x; v[2 * k + 1] = t.y;
        }
    }
    X.ca = v[0]; X.sa = v[1];
    X.b = mk3(v[2], v[3], v[4]);
    X.th0 = v[5];
}

// R = Rx(alpha) Rz(theta) = [[c, -s, 0], [ca s, ca c, -sa], [sa s, sa c, ca]]
// with its four products of the two angles' sines and cosines.
template <typename T>
struct DhRot {
    T c, s, ca, sa;
    T sca, cca, ssa, csa;
};

template <typename T>
__device__ __forceinline__ DhRot<T> dh_rot(T ca, T sa, T c, T s)
{
    return DhRot<T>{c, s, ca, sa, s * ca, c * ca, s * sa, c * sa};
}

// R^T u
template <typename T>
__device__ __forceinline__ V3<T> dh_mulT(const DhRot<T> &R, V3<T> u)
{
    return V3<T>{fma(R.c, u.x, fma(R.sca, u.y, R.ssa * u.z)),
                 fma(-R.s, u.x, fma(R.cca, u.y, R.csa * u.z)),
                 fma(-R.sa, u.y, R.ca * u.z)};
}

// acc + R u (the accumulator folded into the multiply-add chains)
template <typename T>
__device__ __forceinline__ V3<T> dh_mul_add(const DhRot<T> &R, V3<T> u, V3<T> acc)
{
    return V3<T>{fma(R.c, u.x, fma(-R.s, u.y, acc.x)),
                 fma(R.sca, u.x, fma(R.cca, u.y, fma(-R.sa, u.z, acc.y))),
                 fma(R.ssa, u.x, fma(R.csa, u.y, fma(R.ca, u.z, acc.z)))};
}

// R u
template <typename T>
__device__ __forceinline__ V3<T> dh_mul(const DhRot<T> &R, V3<T> u)
{
    return V3<T>{fma(R.c, u.x, -R.s * u.y),
                 fma(R.sca, u.x, fma(R.cca, u.y, -R.sa * u.z)),
                 fma(R.ssa, u.x, fma(R.csa, u.y, R.ca * u.z))};
}

// Forward step of Eq. (id-forward) in frames D:
//   V_i  = Ad_{f^-1} V_{i-1} + S qd,
//   dV_i = S qdd + Ad_{f^-1} dV_{i-1} - ad_{S qd} Ad_{f^-1} V_{i-1},
// Ad_{f^-1}(x_v, x_w) = (R^T (x_v + x_w x b), R^T x_w), S = e_z (angular).
template <typename T>
__device__ __forceinline__ Motion<T> dh_forward(const DhRot<T> &R, V3<T> b, T qd, T qdd,
                                                const Motion<T> &p)
{
    Motion<T> o;
    o.v = dh_mulT(R, cross_add(p.w, b, p.v));
    o.w = dh_mulT(R, p.w);
    o.a = dh_mulT(R, cross_add(p.al, b, p.a));
    o.al = dh_mulT(R, p.al);
    o.w.z += qd;
    o.al.z += qdd;
    o.a.x = fma(qd, o.v.y, o.a.x);
    o.a.y = fma(-qd, o.v.x, o.a.y);
    o.al.x = fma(qd, o.w.y, o.al.x);
    o.al.y = fma(-qd, o.w.x, o.al.y);
    return o;
}

// Inverse of dh_forward: (V_{i-1}, dV_{i-1}) from (V_i, dV_i), using
// Ad_f(x_v, x_w) = (R x_v + b x (R x_w), R x_w).
template <typename T>
__device__ __forceinline__ Motion<T> dh_recover(const DhRot<T> &R, V3<T> b, T qd, T qdd,
                                                const Motion<T> &o)
{
    V3<T> w = o.w;
    w.z -= qd;
    V3<T> al = o.al;
    al.z -= qdd;
    V3<T> a = o.a;
    a.x = fma(-qd, o.v.y, a.x);
    a.y = fma(qd, o.v.x, a.y);
    al.x = fma(-qd, o.w.y, al.x);
    al.y = fma(qd, o.w.x, al.y);
    Motion<T> p;
    p.w = dh_mul(R, w);
    p.al = dh_mul(R, al);
    p.v = cross_add(b, p.w, dh_mul(R, o.v));
    p.a = cross_add(b, p.al, dh_mul(R, a));
    return p;
}

// Backward step of Eq. (id-backward) with the transform of link i+1:
//   F_i = Ad^T_{f_{i,i+1}^-1} F_{i+1} + F_hat_i
//       = (R f + F_hat.f, b x (R f) + R n + F_hat.n).
template <typename T>
__device__ __forceinline__ Wrench<T> dh_carry(const DhRot<T> &R, V3<T> b, const Wrench<T> &Fn,
                                              const Wrench<T> &Fh)
{
    Wrench<T> F;
    const V3<T> rf = dh_mul(R, Fn.f);
    F.f = add3(rf, Fh.f);
    F.n = cross_add(b, rf, dh_mul_add(R, Fn.n, Fh.n));
    return F;
}

}  // namespace rdyn
