// spatial.cuh -- register-level spatial algebra for the RNEA kernels.
//
// All link quantities live in "joint frames": frame i' of link i has its z
// axis on the joint axis and its origin on that axis, so the joint twist is
// S = (0, 0, 0, 0, 0, 1) and the link transform is
//     f_{i-1,i} = M'_i Rz(q_i),   M'_i = (A_i, b_i)
// (the host re-expresses the user's model in these frames once, at model
// creation). With that, Ad_{f^-1} and Ad^T_{f^-1} of Sec. II-A reduce to a
// constant 3x3 rotation, a planar rotation by q_i and one cross product, and
// tau_i = S_i^T F_i is the z moment of F_i.
#pragma once
#include <cuda_runtime.h>

namespace rdyn {

template <typename T>
struct V3 {
    T x, y, z;
};

template <typename T>
__device__ __forceinline__ V3<T> mk3(T x, T y, T z)
{
    return V3<T>{x, y, z};
}

template <typename T>
__device__ __forceinline__ V3<T> add3(V3<T> a, V3<T> b)
{
    return V3<T>{a.x + b.x, a.y + b.y, a.z + b.z};
}

template <typename T>
__device__ __forceinline__ V3<T> sub3(V3<T> a, V3<T> b)
{
    return V3<T>{a.x - b.x, a.y - b.y, a.z - b.z};
}

template <typename T>
__device__ __forceinline__ V3<T> scale3(T s, V3<T> a)
{
    return V3<T>{s * a.x, s * a.y, s * a.z};
}

// acc + a x b
template <typename T>
__device__ __forceinline__ V3<T> cross_add(V3<T> a, V3<T> b, V3<T> acc)
{
    return V3<T>{fma(a.y, b.z, fma(-a.z, b.y, acc.x)),
                 fma(a.z, b.x, fma(-a.x, b.z, acc.y)),
                 fma(a.x, b.y, fma(-a.y, b.x, acc.z))};
}

template <typename T>
__device__ __forceinline__ V3<T> cross3(V3<T> a, V3<T> b)
{
    return V3<T>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Link constants in the joint frame, 24 scalars (padded for 16-byte loads):
//   A[9] rotation of M'_i (row-major), b[3] translation of M'_i,
//   m, c[3] centre of mass, I[6] = (xx, yy, zz, xy, xz, yz) about the centre
//   of mass, 2 pad.
constexpr int kLinkConsts = 24;

template <typename T>
struct LinkC {
    T A[9];
    T b[3];
    T m;
    T c[3];
    T I[6];
};

// A^T x
template <typename T>
__device__ __forceinline__ V3<T> mulAT(const T *A, V3<T> x)
{
    return V3<T>{fma(A[0], x.x, fma(A[3], x.y, A[6] * x.z)),
                 fma(A[1], x.x, fma(A[4], x.y, A[7] * x.z)),
                 fma(A[2], x.x, fma(A[5], x.y, A[8] * x.z))};
}

// A x
template <typename T>
__device__ __forceinline__ V3<T> mulA(const T *A, V3<T> x)
{
    return V3<T>{fma(A[0], x.x, fma(A[1], x.y, A[2] * x.z)),
                 fma(A[3], x.x, fma(A[4], x.y, A[5] * x.z)),
                 fma(A[6], x.x, fma(A[7], x.y, A[8] * x.z))};
}

// Rz(q)^T u with (c, s) = (cos q, sin q)
template <typename T>
__device__ __forceinline__ V3<T> rzT(T c, T s, V3<T> u)
{
    return V3<T>{fma(c, u.x, s * u.y), fma(c, u.y, -s * u.x), u.z};
}

// Rz(q) u
template <typename T>
__device__ __forceinline__ V3<T> rz(T c, T s, V3<T> u)
{
    return V3<T>{fma(c, u.x, -s * u.y), fma(s, u.x, c * u.y), u.z};
}

// symmetric 3x3 (xx, yy, zz, xy, xz, yz) times x
template <typename T>
__device__ __forceinline__ V3<T> sym_mul(const T *I, V3<T> x)
{
    return V3<T>{fma(I[0], x.x, fma(I[3], x.y, I[4] * x.z)),
                 fma(I[3], x.x, fma(I[1], x.y, I[5] * x.z)),
                 fma(I[4], x.x, fma(I[5], x.y, I[2] * x.z))};
}

// Link rotation R = A Rz(q), formed once per link and applied to several
// vectors (12 operations to form, 9 per product instead of 13).
template <typename T>
struct Rot {
    T r[9];  // row-major
};

template <typename T>
__device__ __forceinline__ Rot<T> make_rot(const T *A, T c, T s)
{
    Rot<T> R;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R.r[3 * k + 0] = fma(c, A[3 * k + 0], s * A[3 * k + 1]);
        R.r[3 * k + 1] = fma(c, A[3 * k + 1], -s * A[3 * k + 0]);
        R.r[3 * k + 2] = A[3 * k + 2];
    }
    return R;
}

// Twist (v, w) and its time derivative (a, al) of one link.
template <typename T>
struct Motion {
    V3<T> v, w, a, al;
};

template <typename T>
struct Wrench {
    V3<T> f, n;
};

// Forward step, Sec. II-A Eq. (id-forward), in joint frames:
//   V_i  = Ad_{f^-1} V_{i-1} + S qd
//   dV_i = S qdd + Ad_{f^-1} dV_{i-1} - ad_{S qd} Ad_{f^-1} V_{i-1}
// with Ad_{f^-1}(x_v, x_w) = (R^T (x_v + x_w x b), R^T x_w), R = A Rz(q).
template <typename T>
__device__ __forceinline__ Motion<T> forward_step(const T *A, V3<T> b, T c, T s, T qd, T qdd,
                                                  const Motion<T> &p)
{
    Motion<T> o;
    V3<T> t = cross_add(p.w, b, p.v);
    V3<T> ta = cross_add(p.al, b, p.a);
    o.v = rzT(c, s, mulAT(A, t));
    o.w = rzT(c, s, mulAT(A, p.w));
    o.a = rzT(c, s, mulAT(A, ta));
    o.al = rzT(c, s, mulAT(A, p.al));
    o.w.z += qd;
    o.al.z += qdd;
    // -ad_{S qd}(x) = -qd (e_z x x_v, e_z x x_w); e_z x x = (-x.y, x.x, 0)
    o.a.x = fma(qd, o.v.y, o.a.x);
    o.a.y = fma(-qd, o.v.x, o.a.y);
    o.al.x = fma(qd, o.w.y, o.al.x);
    o.al.y = fma(-qd, o.w.x, o.al.y);
    return o;
}

// Inverse of forward_step: (V_{i-1}, dV_{i-1}) from (V_i, dV_i).
//   Ad_f(x_v, x_w) = (R x_v + b x (R x_w), R x_w)
template <typename T>
__device__ __forceinline__ Motion<T> backward_recover(const T *A, V3<T> b, T c, T s, T qd,
                                                      T qdd, const Motion<T> &o)
{
    // undo the S qd / S qdd / ad terms in the joint frame first
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
    p.w = mulA(A, rz(c, s, w));
    p.al = mulA(A, rz(c, s, al));
    V3<T> rv = mulA(A, rz(c, s, o.v));
    V3<T> ra = mulA(A, rz(c, s, a));
    p.v = cross_add(b, p.w, rv);
    p.a = cross_add(b, p.al, ra);
    return p;
}

// forward_step with the link rotation already formed.
template <typename T>
__device__ __forceinline__ Motion<T> forward_step_R(const Rot<T> &R, V3<T> b, T qd, T qdd,
                                                    const Motion<T> &p)
{
    Motion<T> o;
    V3<T> t = cross_add(p.w, b, p.v);
    V3<T> ta = cross_add(p.al, b, p.a);
    o.v = mulAT(R.r, t);
    o.w = mulAT(R.r, p.w);
    o.a = mulAT(R.r, ta);
    o.al = mulAT(R.r, p.al);
    o.w.z += qd;
    o.al.z += qdd;
    o.a.x = fma(qd, o.v.y, o.a.x);
    o.a.y = fma(-qd, o.v.x, o.a.y);
    o.al.x = fma(qd, o.w.y, o.al.x);
    o.al.y = fma(-qd, o.w.x, o.al.y);
    return o;
}

// backward_recover with the link rotation already formed.
template <typename T>
__device__ __forceinline__ Motion<T> backward_recover_R(const Rot<T> &R, V3<T> b, T qd, T qdd,
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
    p.w = mulA(R.r, w);
    p.al = mulA(R.r, al);
    p.v = cross_add(b, p.w, mulA(R.r, o.v));
    p.a = cross_add(b, p.al, mulA(R.r, a));
    return p;
}

// carry_wrench with the rotation of link i+1 already formed.
template <typename T>
__device__ __forceinline__ Wrench<T> carry_wrench_R(const Rot<T> &R, V3<T> b,
                                                    const Wrench<T> &Fn, const Wrench<T> &Fh)
{
    Wrench<T> F;
    V3<T> rf = mulA(R.r, Fn.f);
    V3<T> rn = mulA(R.r, Fn.n);
    F.f = add3(rf, Fh.f);
    F.n = cross_add(b, rf, add3(rn, Fh.n));
    return F;
}

// Bias wrench F_hat = J dV - ad^T_V (J V) (Sec. III-C), written with the
// centre of mass c:
//   a_c = a + w x v + al x c + w x (w x c) = a + al x c + w x (v + w x c),
//   f = m a_c,   n = c x f + I_c al + w x (I_c w).
template <typename T>
__device__ __forceinline__ Wrench<T> bias_wrench(T m, V3<T> c, const T *I, const Motion<T> &x)
{
    const V3<T> vc = cross_add(x.w, c, x.v);  // velocity of the centre of mass
    V3<T> ac = cross_add(x.al, c, x.a);
    ac = cross_add(x.w, vc, ac);
    Wrench<T> F;
    F.f = scale3(m, ac);
    V3<T> Iw = sym_mul(I, x.w);
    V3<T> n = sym_mul(I, x.al);
    n = cross_add(c, F.f, n);
    F.n = cross_add(x.w, Iw, n);
    return F;
}

// Backward step, Sec. II-A Eq. (id-backward):
//   F_i = Ad^T_{f_{i,i+1}^-1} F_{i+1} + F_hat_i,
//   Ad^T_{f^-1}(f, n) = (R f, b x (R f) + R n), R = A Rz(q_{i+1}).
template <typename T>
__device__ __forceinline__ Wrench<T> carry_wrench(const T *A, V3<T> b, T c, T s,
                                                  const Wrench<T> &Fn, const Wrench<T> &Fh)
{
    Wrench<T> F;
    V3<T> rf = mulA(A, rz(c, s, Fn.f));
    V3<T> rn = mulA(A, rz(c, s, Fn.n));
    F.f = add3(rf, Fh.f);
    F.n = cross_add(b, rf, add3(rn, Fh.n));
    return F;
}

}  // namespace rdyn
