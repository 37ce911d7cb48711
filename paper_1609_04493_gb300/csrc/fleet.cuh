// fleet.cuh -- mixed inverse / forward dynamics requests over many chains of
// different lengths in one launch.
//
// Every request r names a robot (its own constants, n_r links) and a kind:
// inverse dynamics (tau from q, qd, qdd; Sec. II-A) or forward dynamics (qdd
// from q, qd, tau; Sec. II-B). Joint vectors are ragged: request r's values
// sit at [off_r, off_r + n_r) of every data array. One thread evaluates one
// request with the per-instance bodies of the single-chain kernels (the
// re-derive-in-the-backward-sweep RNEA, and the articulated-body algorithm
// with its inertia updates and solves in double-float arithmetic for FP32
// data unless FP64 is asked for, FP64 for FP64 data) in the common-normal
// frames of spatial_dh.cuh,
// reading its robot's constants from global memory since no two requests need
// share them; each link prefetches the next link's constants (and, in forward
// dynamics, records and workspace) into L1 while it computes.
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
#include <climits>

#include "aba_dh.cuh"
#include "aba_pair.cuh"
#include "aba_tri.cuh"
#include "rnea_dhp.cuh"

namespace rdyn {

// T: data type; D: scalar of the forward-dynamics inertia updates and solves
// (double-float for FP32 data by default, else double)
template <typename T, typename D>
struct FleetArgs {
    const T *consts;          // [total links][16] common-normal constants
    const D *records;         // [total links][32] forward-dynamics records
    const int *robot_n;       // [robots]
    const int *robot_link;    // [robots] first constant row
    const T *robot_gb;        // [robots][12] base frame D_{-1} in frame 0: R (9), p (3)
    const T *robot_tn;        // [robots][12] frame D_{n-1} in frame n: R (9), r (3)
    const int *order;         // [R] sorted request indices
    const int *req_robot;     // [R]
    const int *req_kind;      // [R] 0 = inverse, 1 = forward dynamics
    const long long *req_off; // [R] offset of the joint values
    // forward-dynamics workspace of the 32 sorted positions [32 g, 32 g + 32):
    // byte offsets of its T part ([link][10][lane]) and its solve part
    // ([link][8][lane])
    const long long *group_ws, *group_wz;
    // the records as double-float pairs, and the number of leading groups of
    // 32 whose forward-dynamics requests run the bias sweeps on them in
    // double-float (FP32 data, chains beyond RD_ABA_EXTENDED_BIAS_LINKS)
    const DF *records_df;
    int ext_groups;
    // two- or three-warp forward dynamics (fleet_pair_kernel,
    // fleet_tri_kernel): the first pair_groups groups of 32 sorted requests,
    // taken through pair_counter
    int pair_groups;
    int *pair_counter;
    int R;
    const T *q, *qd, *in2;    // in2: qdd (inverse) or tau (forward)
    T *out;                   // tau (inverse) or qdd (forward)
    int *status;              // [R] or null
    unsigned char *ws;
    int *counter;
    BaseParams<T> base;       // V_0, dV_0 in frame 0; F_{n+1} in frame n
};

// Inverse dynamics of one instance in common-normal frames, backward sweep
// re-deriving the motion (the stateless rnea_dhp_kernel without staging; rows
// of any length and alignment, constants read from global memory).
template <typename T, int TRIG>
__device__ __forceinline__ void rnea_dh_instance(const T *__restrict__ sc, int n,
                                                 const T *__restrict__ qr,
                                                 const T *__restrict__ qdr,
                                                 const T *__restrict__ qddr, T *__restrict__ taur,
                                                 const BaseParams<T> &base)
{
    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);
    for (int i = 0; i < n; ++i) {
        if (i + 1 < n) prefetch_l1(sc + (i + 1) * kDhConsts);
        DhXf<T> X;
        load_dh_xf(sc + i * kDhConsts, X);
        T s, c;
        dh_trig<T, TRIG>(__ldg(qr + i) + X.th0, &s, &c);
        x = dh_forward(dh_rot(X.ca, X.sa, c, s), X.b, __ldg(qdr + i), __ldg(qddr + i), x);
    }
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    DhRot<T> Rn = dh_rot(T(1), T(0), T(1), T(0));
    V3<T> bn = mk3(T(0), T(0), T(0));
    for (int i = n - 1; i >= 0; --i) {
        if (i > 0) prefetch_l1(sc + (i - 1) * kDhConsts);
        DhLink<T> L;
        load_dh(sc + i * kDhConsts, L);
        T s, c;
        dh_trig<T, TRIG>(__ldg(qr + i) + L.th0, &s, &c);
        const DhRot<T> R = dh_rot(L.ca, L.sa, c, s);
        const Wrench<T> Fh = bias_wrench(L.m, L.c, L.I, x);
        if (i == n - 1) {
            F.f = add3(F.f, Fh.f);
            F.n = add3(F.n, Fh.n);
        } else {
            F = dh_carry(Rn, bn, F, Fh);
        }
        taur[i] = F.n.z;
        if (i > 0) x = dh_recover(R, L.b, __ldg(qdr + i), __ldg(qddr + i), x);
        Rn = R;
        bn = L.b;
    }
}

// Boundary terms in a robot's frames: V_0, dV_0 to D_{-1} (Ad_{G^-1}:
// (R^T (v + w x p), R^T w)); F_{n+1} from frame n to D_{n-1}:
// (R^T f, R^T (n - r x f)).
template <typename T, typename D>
__device__ __forceinline__ void fleet_base(const FleetArgs<T, D> &a, int robot, BaseParams<T> &bp)
{
    const T *g = a.robot_gb + (size_t)robot * 12;
    const V3<T> p = mk3(g[9], g[10], g[11]);
    const V3<T> v0 = mk3(a.base.V0[0], a.base.V0[1], a.base.V0[2]);
    const V3<T> w0 = mk3(a.base.V0[3], a.base.V0[4], a.base.V0[5]);
    const V3<T> a0 = mk3(a.base.dV0[0], a.base.dV0[1], a.base.dV0[2]);
    const V3<T> al0 = mk3(a.base.dV0[3], a.base.dV0[4], a.base.dV0[5]);
    const V3<T> vv = mulAT(g, cross_add(w0, p, v0)), ww = mulAT(g, w0);
    const V3<T> aa = mulAT(g, cross_add(al0, p, a0)), al = mulAT(g, al0);
    bp.V0[0] = vv.x; bp.V0[1] = vv.y; bp.V0[2] = vv.z;
    bp.V0[3] = ww.x; bp.V0[4] = ww.y; bp.V0[5] = ww.z;
    bp.dV0[0] = aa.x; bp.dV0[1] = aa.y; bp.dV0[2] = aa.z;
    bp.dV0[3] = al.x; bp.dV0[4] = al.y; bp.dV0[5] = al.z;
    const T *tn = a.robot_tn + (size_t)robot * 12;
    const V3<T> f = mk3(a.base.Fn[0], a.base.Fn[1], a.base.Fn[2]);
    const V3<T> nn = mk3(a.base.Fn[3], a.base.Fn[4], a.base.Fn[5]);
    const V3<T> rr = mk3(tn[9], tn[10], tn[11]);
    const V3<T> fp = mulAT(tn, f);
    const V3<T> np = mulAT(tn, sub3(nn, cross3(rr, f)));
    bp.Fn[0] = fp.x; bp.Fn[1] = fp.y; bp.Fn[2] = fp.z;
    bp.Fn[3] = np.x; bp.Fn[4] = np.y; bp.Fn[5] = np.z;
}

// The request at sorted position k.
template <typename T, typename D>
__device__ __forceinline__ void fleet_request(const FleetArgs<T, D> &a, int k)
{
    const int r = a.order[k];
    const int robot = a.req_robot[r];
    const int n = a.robot_n[robot];
    const long long lo = a.robot_link[robot];
    const long long off = a.req_off[r];
    BaseParams<T> bp;
    fleet_base(a, robot, bp);
    const T *sc = a.consts + lo * kDhConsts;
    if (a.req_kind[r] == 0) {
        rnea_dh_instance<T, kTrigPoly>(sc, n, a.q + off, a.qd + off, a.in2 + off, a.out + off, bp);
    } else {
        static_assert(sizeof(D) == sizeof(double), "solve-state slots are 8 bytes");
        const int g = k >> 5;
        T *wt = reinterpret_cast<T *>(a.ws + a.group_ws[g]);
        D *wz = reinterpret_cast<D *>(a.ws + a.group_wz[g]);
        int bad = -1;
        if constexpr (sizeof(T) == 4) {
            if (g < a.ext_groups)
                bad = aba_dh_instance<T, D, D, kTrigPoly, false, true, DF>(
                    sc, a.records + lo * kAbaDh64, n, a.q + off, a.qd + off, a.in2 + off,
                    a.out + off, wt, wz, 32, k & 31, bp, a.records_df + lo * kAbaDh64);
        }
        if (bad < 0)
            bad = aba_dh_instance<T, D, D, kTrigPoly, false, true>(
                sc, a.records + lo * kAbaDh64, n, a.q + off, a.qd + off, a.in2 + off,
                a.out + off, wt, wz, 32, k & 31, bp);
        if (a.status) a.status[r] = bad ? 1 : 0;
    }
}

// The request at sorted position k for one warp of a pair (role 0: the
// articulated inertias; role 1: the rest of forward dynamics; aba_pair.cuh).
// An inverse-dynamics request in a pair group runs on role 0 alone.
template <typename T, typename D>
__device__ __forceinline__ void fleet_request_pair(const FleetArgs<T, D> &a, int k, int role,
                                                   volatile int *progress, int *jbad)
{
    const int r = a.order[k];
    const int robot = a.req_robot[r];
    const int n = a.robot_n[robot];
    const long long lo = a.robot_link[robot];
    const long long off = a.req_off[r];
    if (a.req_kind[r] == 0) {
        if (role == 0) fleet_request(a, k);
        return;
    }
    BaseParams<T> bp;
    fleet_base(a, robot, bp);
    const T *sc = a.consts + lo * kDhConsts;
    const int g = k >> 5;
    T *wt = reinterpret_cast<T *>(a.ws + a.group_ws[g]);
    D *wz = reinterpret_cast<D *>(a.ws + a.group_wz[g]);
    int st = 0;
    if constexpr (sizeof(T) == 4) {
        if (g < a.ext_groups)
            st = aba_pair_role<T, D, DF, kTrigPoly>(role, sc, a.records + lo * kAbaDh64,
                                                    a.records_df + lo * kAbaDh64, n, a.q + off,
                                                    a.qd + off, a.in2 + off, a.out + off, wt, wz,
                                                    32, k & 31, bp, progress, jbad);
        else
            st = aba_pair_role<T, D, T, kTrigPoly>(role, sc, a.records + lo * kAbaDh64,
                                                   a.records_df + lo * kAbaDh64, n, a.q + off,
                                                   a.qd + off, a.in2 + off, a.out + off, wt, wz, 32,
                                                   k & 31, bp, progress, jbad);
    } else {
        st = aba_pair_role<T, D, T, kTrigPoly>(role, sc, a.records + lo * kAbaDh64, nullptr, n,
                                               a.q + off, a.qd + off, a.in2 + off, a.out + off,
                                               wt, wz, 32, k & 31, bp, progress, jbad);
    }
    if (role == 1 && a.status) a.status[r] = st ? 1 : 0;
}

__device__ __forceinline__ void pair_barrier(int id)
{
    asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

__device__ __forceinline__ void triple_barrier(int id)
{
    asm volatile("bar.sync %0, 96;" ::"r"(id) : "memory");
}

// The request at sorted position k for one warp of a triple (role 0: JA, 1: JB,
// 2: Z; aba_tri.cuh). An inverse-dynamics request runs on role 0 alone.
template <typename T, typename D>
__device__ __forceinline__ void fleet_request_tri(const FleetArgs<T, D> &a, int k, int role,
                                                  AbaTriShared<D> &sh, int lane)
{
    const int r = a.order[k];
    const int robot = a.req_robot[r];
    const int n = a.robot_n[robot];
    const long long lo = a.robot_link[robot];
    const long long off = a.req_off[r];
    if (a.req_kind[r] == 0) {
        if (role == 0) fleet_request(a, k);
        return;
    }
    const T *sc = a.consts + lo * kDhConsts;
    const D *sd = a.records + lo * kAbaDh64;
    const DF *sdf = a.records_df ? a.records_df + lo * kAbaDh64 : nullptr;
    const int g = k >> 5;
    T *wt = reinterpret_cast<T *>(a.ws + a.group_ws[g]);
    D *wz = reinterpret_cast<D *>(a.ws + a.group_wz[g]);
    const int b = k & 31;
    auto body = [&](auto tb_tag) {
        using TB = decltype(tb_tag);
        if (role == 0) {
            aba_tri_ja<T, D, TB, kTrigPoly>(sc, sd, sdf, n, a.q + off, wz, 32, b, sh, lane);
        } else if (role == 1) {
            aba_tri_jb<T, D, TB, kTrigPoly>(sc, sd, sdf, n, a.q + off, wz, 32, b, sh, lane);
        } else {
            BaseParams<T> bp;
            fleet_base(a, robot, bp);
            const volatile int *cnt = &sh.cnt[0][0];
            const int st = aba_pair_z<T, D, TB, kTrigPoly>(
                sc, sd, sdf, n, a.q + off, a.qd + off, a.in2 + off, a.out + off, wt, wz, 32, b, bp,
                cnt + kTriUA * 32 + lane, cnt + kTriUB * 32 + lane, &sh.flags[0][lane],
                &sh.flags[1][lane]);
            if (a.status) a.status[r] = st ? 1 : 0;
        }
    };
    if constexpr (sizeof(T) == 4) {
        if (g < a.ext_groups) {
            body(DF{});
            return;
        }
    }
    body(T{});
}

// Persistent with three-warp forward dynamics: as fleet_pair_kernel with warp
// triples (JA, JB, Z) per group of 32 sorted requests, at most two triples per
// block (96 or 192 threads; named barriers 1..4; 13 KB of exchange state per
// triple), then every warp on the remaining requests.
template <typename T, typename D>
__global__ void fleet_tri_kernel(FleetArgs<T, D> a)
{
    __shared__ AbaTriShared<D> sh[2];
    __shared__ volatile int grp[2];
    const int tri = threadIdx.x / 96;
    const int role = (threadIdx.x >> 5) % 3;
    const int lane = threadIdx.x & 31;
    for (;;) {
        if (role == 0) {
            if (lane == 0) grp[tri] = atomicAdd(a.pair_counter, 1);
#pragma unroll
            for (int c = 0; c < 4; ++c) sh[tri].cnt[c][lane] = INT_MAX;
            sh[tri].flags[0][lane] = 0;
            sh[tri].flags[1][lane] = 0;
        }
        __syncwarp();
        triple_barrier(1 + 2 * tri);
        const int g = grp[tri];
        if (g >= a.pair_groups) break;
        const int k = 32 * g + lane;
        if (k < a.R) fleet_request_tri(a, k, role, sh[tri], lane);
        __syncwarp();
        triple_barrier(2 + 2 * tri);
    }
    const int base = 32 * a.pair_groups;
    for (;;) {
        int start = 0;
        if (lane == 0) start = base + atomicAdd(a.counter, 32);
        start = __shfl_sync(0xffffffffu, start, 0);
        if (start >= a.R) break;
        const int k = start + lane;
        if (k < a.R) fleet_request(a, k);
    }
}

// Persistent with two-warp forward dynamics. Warps 2p and 2p + 1 of a block form
// a pair: first the pairs take the leading a.pair_groups groups of 32 sorted
// requests (forward dynamics with long chains, sorted first), both warps on the
// same group through one atomicAdd and a named barrier per step; then every
// warp takes 32 of the remaining requests at a time, as fleet_persistent_kernel.
// At most 7 pairs per block (named barriers 1..14).
template <typename T, typename D>
__global__ void fleet_pair_kernel(FleetArgs<T, D> a)
{
    __shared__ volatile int prog[7][32];
    __shared__ int jbad[7][32];
    __shared__ volatile int grp[7];
    const int pair = threadIdx.x >> 6;
    const int role = (threadIdx.x >> 5) & 1;
    const int lane = threadIdx.x & 31;
    for (;;) {
        if (role == 0) {
            if (lane == 0) grp[pair] = atomicAdd(a.pair_counter, 1);
            prog[pair][lane] = INT_MAX;
            jbad[pair][lane] = 0;
        }
        __syncwarp();
        pair_barrier(1 + 2 * pair);
        const int g = grp[pair];
        if (g >= a.pair_groups) break;
        const int k = 32 * g + lane;
        if (k < a.R) fleet_request_pair(a, k, role, &prog[pair][lane], &jbad[pair][lane]);
        __syncwarp();
        pair_barrier(2 + 2 * pair);
    }
    const int base = 32 * a.pair_groups;
    for (;;) {
        int start = 0;
        if (lane == 0) start = base + atomicAdd(a.counter, 32);
        start = __shfl_sync(0xffffffffu, start, 0);
        if (start >= a.R) break;
        const int k = start + lane;
        if (k < a.R) fleet_request(a, k);
    }
}

// Persistent: warps take 32 sorted requests at a time until none are left.
template <typename T, typename D>
__global__ void fleet_persistent_kernel(FleetArgs<T, D> a)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int start = 0;
        if (lane == 0) start = atomicAdd(a.counter, 32);
        start = __shfl_sync(0xffffffffu, start, 0);
        if (start >= a.R) break;
        const int k = start + lane;
        if (k < a.R) fleet_request(a, k);
    }
}

// One ordinary launch over sorted positions [begin, end).
template <typename T, typename D>
__global__ void fleet_range_kernel(FleetArgs<T, D> a, int begin, int end)
{
    const int k = begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (k < end) fleet_request(a, k);
}

}  // namespace rdyn
