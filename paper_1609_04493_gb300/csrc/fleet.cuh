// fleet.cuh -- mixed inverse / forward dynamics requests over many chains of
// different lengths in one launch.
//
// Every request r names a robot (its own constants, n_r links) and a kind:
// inverse dynamics (tau from q, qd, qdd; Sec. II-A) or forward dynamics (qdd
// from q, qd, tau; Sec. II-B). Joint vectors are ragged: request r's values
// sit at [off_r, off_r + n_r) of every data array. One thread evaluates one
// request with the per-instance bodies of the single-chain kernels (the
// re-derive-in-the-backward-sweep RNEA, and the articulated-body algorithm
// with FP64 inertia updates and solves), reading its robot's constants from
// global memory since no two requests need share them.
//
// Scheduling: the host sorts requests (forward dynamics first, then by
// decreasing n) so that the 32 requests a warp takes are alike.
//   persistent: a grid of resident CTAs; each warp takes the next 32 sorted
//               requests with one atomicAdd on a counter that the call resets
//               (stream-ordered memset) before the launch. No thread ever waits
//               on another.
//   per-group:  one ordinary launch per run of equal (kind, n) in the sorted
//               order -- the "one launch per request size" comparison.
#pragma once
#include "aba.cuh"
#include "rnea_serial.cuh"

namespace rdyn {

template <typename T>
struct FleetArgs {
    const T *consts;          // [total links][24]
    const double *consts64;   // [total links][24]
    const int *robot_n;       // [robots]
    const int *robot_link;    // [robots] first constant row
    const T *robot_tn;        // [robots][12] joint frame of the last link: R (9), r (3)
    const int *order;         // [R] sorted request indices
    const int *req_robot;     // [R]
    const int *req_kind;      // [R] 0 = inverse, 1 = forward dynamics
    const long long *req_off; // [R] offset of the joint values
    const long long *req_ws;  // [R] workspace offset in bytes (forward dynamics)
    int R;
    const T *q, *qd, *in2;    // in2: qdd (inverse) or tau (forward)
    T *out;                   // tau (inverse) or qdd (forward)
    int *status;              // [R] or null
    unsigned char *ws;
    int *counter;
    BaseParams<T> base;       // F_{n+1} in the frame of each robot's last link
};

// Inverse dynamics of one instance, backward sweep re-deriving the motion
// (rnea_serial_kernel<kRecompute> without the block-level staging).
template <typename T>
__device__ __forceinline__ void rnea_instance_recompute(const T *__restrict__ sc, int n,
                                                        const T *__restrict__ qr,
                                                        const T *__restrict__ qdr,
                                                        const T *__restrict__ qddr,
                                                        T *__restrict__ taur,
                                                        const BaseParams<T> &base)
{
    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);
    for (int i = 0; i < n; ++i) {
        LinkXf<T> X;
        load_xf(sc + i * kLinkConsts, X);
        T s, c;
        sincos_t(__ldg(qr + i), &s, &c);
        const Rot<T> R = make_rot(X.A, c, s);
        x = forward_step_R(R, mk3(X.b[0], X.b[1], X.b[2]), __ldg(qdr + i), __ldg(qddr + i), x);
    }
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    Rot<T> Rn;
    V3<T> bn = mk3(T(0), T(0), T(0));
    for (int i = n - 1; i >= 0; --i) {
        LinkC<T> L;
        load_link(sc + i * kLinkConsts, L);
        T s, c;
        sincos_t(__ldg(qr + i), &s, &c);
        const Rot<T> R = make_rot(L.A, c, s);
        const V3<T> bi = mk3(L.b[0], L.b[1], L.b[2]);
        const Wrench<T> Fh = bias_wrench(L.m, mk3(L.c[0], L.c[1], L.c[2]), L.I, x);
        if (i == n - 1) {
            F.f = add3(F.f, Fh.f);
            F.n = add3(F.n, Fh.n);
        } else {
            F = carry_wrench_R(Rn, bn, F, Fh);
        }
        taur[i] = F.n.z;
        if (i > 0) x = backward_recover_R(R, bi, __ldg(qdr + i), __ldg(qddr + i), x);
        Rn = R;
        bn = bi;
    }
}

template <typename T>
__device__ __forceinline__ void fleet_request(const FleetArgs<T> &a, int r)
{
    const int robot = a.req_robot[r];
    const int n = a.robot_n[robot];
    const long long lo = a.robot_link[robot];
    const long long off = a.req_off[r];
    // F_{n+1} from the robot's frame n to its joint frame n': (R^T f, R^T (n - r x f))
    BaseParams<T> bp = a.base;
    {
        const T *tn = a.robot_tn + (size_t)robot * 12;
        const V3<T> f = mk3(a.base.Fn[0], a.base.Fn[1], a.base.Fn[2]);
        const V3<T> nn = mk3(a.base.Fn[3], a.base.Fn[4], a.base.Fn[5]);
        const V3<T> rr = mk3(tn[9], tn[10], tn[11]);
        const V3<T> fp = mulAT(tn, f);
        const V3<T> np = mulAT(tn, sub3(nn, cross3(rr, f)));
        bp.Fn[0] = fp.x; bp.Fn[1] = fp.y; bp.Fn[2] = fp.z;
        bp.Fn[3] = np.x; bp.Fn[4] = np.y; bp.Fn[5] = np.z;
    }
    const T *sc = a.consts + lo * kLinkConsts;
    if (a.req_kind[r] == 0) {
        rnea_instance_recompute<T>(sc, n, a.q + off, a.qd + off, a.in2 + off, a.out + off, bp);
    } else {
        unsigned char *w = a.ws + a.req_ws[r];
        T *wt = reinterpret_cast<T *>(w);
        double *wz = reinterpret_cast<double *>(
            w + (((size_t)n * kAbaStateScalars * sizeof(T) + 15) & ~(size_t)15));
        const int bad = aba_instance<T, double, false>(sc, a.consts64 + lo * kLinkConsts, n,
                                                       a.q + off, a.qd + off, a.in2 + off,
                                                       a.out + off, wt, wz, 1, 0, bp);
        if (a.status) a.status[r] = bad ? 1 : 0;
    }
}

// Persistent: warps take 32 sorted requests at a time until none are left.
template <typename T>
__global__ void fleet_persistent_kernel(FleetArgs<T> a)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int start = 0;
        if (lane == 0) start = atomicAdd(a.counter, 32);
        start = __shfl_sync(0xffffffffu, start, 0);
        if (start >= a.R) break;
        const int k = start + lane;
        if (k < a.R) fleet_request(a, a.order[k]);
    }
}

// One ordinary launch over sorted positions [begin, end).
template <typename T>
__global__ void fleet_range_kernel(FleetArgs<T> a, int begin, int end)
{
    const int k = begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (k < end) fleet_request(a, a.order[k]);
}

}  // namespace rdyn
