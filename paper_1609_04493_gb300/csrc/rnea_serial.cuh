// rnea_serial.cuh -- one thread per instance: the two propagations of
// Sec. II-A (Eqs. id-forward, id-backward) run as a serial recursion over the
// links inside each thread, which is the work-efficient form of the two scans
// of Sec. III when the batch alone fills the GPU.
//
// Two ways to carry what the backward sweep needs from the forward sweep:
//   kStore     -- F_hat_i and (cos q_i, sin q_i) of every link go to shared
//                 memory (8 scalars per link per thread);
//   kRecompute -- nothing is stored: the backward sweep re-derives
//                 (V_{i-1}, dV_{i-1}) from (V_i, dV_i) by inverting the forward
//                 step (the operands of the forward scan form a group, Sec.
//                 III-B, so each step is invertible) and recomputes F_hat_i.
#pragma once
#include "spatial.cuh"

namespace rdyn {

template <typename T>
struct BaseParams {
    T V0[6];
    T dV0[6];
    T Fn[6];  // F_{n+1} in the joint frame of link n
};

enum StateMode { kStore = 0, kRecompute = 1 };

__device__ __forceinline__ void sincos_t(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double *s, double *c) { sincos(x, s, c); }

// Link constants from shared memory with 16-byte loads.
template <typename T>
__device__ __forceinline__ void load_link(const T *p, LinkC<T> &L);

template <>
__device__ __forceinline__ void load_link<float>(const float *p, LinkC<float> &L)
{
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
    float4 a = p4[0], b = p4[1], c = p4[2], d = p4[3], e = p4[4], f = p4[5];
    L.A[0] = a.x; L.A[1] = a.y; L.A[2] = a.z; L.A[3] = a.w;
    L.A[4] = b.x; L.A[5] = b.y; L.A[6] = b.z; L.A[7] = b.w;
    L.A[8] = c.x; L.b[0] = c.y; L.b[1] = c.z; L.b[2] = c.w;
    L.m = d.x; L.c[0] = d.y; L.c[1] = d.z; L.c[2] = d.w;
    L.I[0] = e.x; L.I[1] = e.y; L.I[2] = e.z; L.I[3] = e.w;
    L.I[4] = f.x; L.I[5] = f.y;
}

template <>
__device__ __forceinline__ void load_link<double>(const double *p, LinkC<double> &L)
{
    const double2 *p2 = reinterpret_cast<const double2 *>(p);
    double v[22];
#pragma unroll
    for (int k = 0; k < 11; ++k) {
        double2 t = p2[k];
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) L.A[k] = v[k];
    L.b[0] = v[9]; L.b[1] = v[10]; L.b[2] = v[11];
    L.m = v[12]; L.c[0] = v[13]; L.c[1] = v[14]; L.c[2] = v[15];
#pragma unroll
    for (int k = 0; k < 6; ++k) L.I[k] = v[16 + k];
}

// Per-thread backward-sweep state of one link: F_hat (6), cos, sin.
template <typename T>
struct LinkState {
    Wrench<T> Fh;
    T c, s;
};

template <typename T>
__device__ __forceinline__ void put_state(unsigned char *base, int i, int tid, int block,
                                          const LinkState<T> &x);
template <typename T>
__device__ __forceinline__ void get_state(const unsigned char *base, int i, int tid, int block,
                                          LinkState<T> &x);

template <>
__device__ __forceinline__ void put_state<float>(unsigned char *base, int i, int tid, int block,
                                                 const LinkState<float> &x)
{
    float4 *s = reinterpret_cast<float4 *>(base);
    s[(2 * i + 0) * block + tid] = make_float4(x.Fh.f.x, x.Fh.f.y, x.Fh.f.z, x.Fh.n.x);
    s[(2 * i + 1) * block + tid] = make_float4(x.Fh.n.y, x.Fh.n.z, x.c, x.s);
}

template <>
__device__ __forceinline__ void get_state<float>(const unsigned char *base, int i, int tid,
                                                 int block, LinkState<float> &x)
{
    const float4 *s = reinterpret_cast<const float4 *>(base);
    float4 u = s[(2 * i + 0) * block + tid];
    float4 v = s[(2 * i + 1) * block + tid];
    x.Fh.f = mk3(u.x, u.y, u.z);
    x.Fh.n = mk3(u.w, v.x, v.y);
    x.c = v.z;
    x.s = v.w;
}

template <>
__device__ __forceinline__ void put_state<double>(unsigned char *base, int i, int tid,
                                                  int block, const LinkState<double> &x)
{
    double2 *s = reinterpret_cast<double2 *>(base);
    s[(4 * i + 0) * block + tid] = make_double2(x.Fh.f.x, x.Fh.f.y);
    s[(4 * i + 1) * block + tid] = make_double2(x.Fh.f.z, x.Fh.n.x);
    s[(4 * i + 2) * block + tid] = make_double2(x.Fh.n.y, x.Fh.n.z);
    s[(4 * i + 3) * block + tid] = make_double2(x.c, x.s);
}

template <>
__device__ __forceinline__ void get_state<double>(const unsigned char *base, int i, int tid,
                                                  int block, LinkState<double> &x)
{
    const double2 *s = reinterpret_cast<const double2 *>(base);
    double2 a = s[(4 * i + 0) * block + tid];
    double2 b = s[(4 * i + 1) * block + tid];
    double2 c = s[(4 * i + 2) * block + tid];
    double2 d = s[(4 * i + 3) * block + tid];
    x.Fh.f = mk3(a.x, a.y, b.x);
    x.Fh.n = mk3(b.y, c.x, c.y);
    x.c = d.x;
    x.s = d.y;
}

template <typename T>
__host__ __device__ constexpr int state_bytes_per_link()
{
    return 8 * (int)sizeof(T);
}

// Shared memory: n * 24 link constants, then (kStore) n * 8 scalars per thread.
template <typename T, int BLOCK, int MODE>
__global__ void __launch_bounds__(BLOCK)
rnea_serial_kernel(const T *__restrict__ consts, int n, int B, const T *__restrict__ q,
                   const T *__restrict__ qd, const T *__restrict__ qdd, T *__restrict__ tau,
                   BaseParams<T> base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *sc = reinterpret_cast<T *>(smem);
    const int nc = n * kLinkConsts;
    for (int k = threadIdx.x; k < nc; k += BLOCK) sc[k] = consts[k];
    unsigned char *st = smem + (size_t)nc * sizeof(T);
    __syncthreads();

    const int tid = threadIdx.x;
    const int b = blockIdx.x * BLOCK + tid;
    if (b >= B) return;
    const size_t row = (size_t)b * (size_t)n;

    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);

    // forward sweep: base -> tip
    for (int i = 0; i < n; ++i) {
        LinkC<T> L;
        load_link(sc + i * kLinkConsts, L);
        T qi = __ldg(q + row + i), qdi = __ldg(qd + row + i), qddi = __ldg(qdd + row + i);
        T s, c;
        sincos_t(qi, &s, &c);
        x = forward_step(L.A, mk3(L.b[0], L.b[1], L.b[2]), c, s, qdi, qddi, x);
        if (MODE == kStore) {
            LinkState<T> ls;
            ls.Fh = bias_wrench(L.m, mk3(L.c[0], L.c[1], L.c[2]), L.I, x);
            ls.c = c;
            ls.s = s;
            put_state<T>(st, i, tid, BLOCK, ls);
        }
    }

    // backward sweep: tip -> base
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    T cn = T(1), sn = T(0);
    int inext = -1;
    for (int i = n - 1; i >= 0; --i) {
        LinkState<T> ls;
        LinkC<T> L;
        load_link(sc + i * kLinkConsts, L);
        if (MODE == kStore) {
            get_state<T>(st, i, tid, BLOCK, ls);
        } else {
            T qi = __ldg(q + row + i);
            sincos_t(qi, &ls.s, &ls.c);
            ls.Fh = bias_wrench(L.m, mk3(L.c[0], L.c[1], L.c[2]), L.I, x);
        }
        if (inext < 0) {
            F.f = add3(F.f, ls.Fh.f);
            F.n = add3(F.n, ls.Fh.n);
        } else {
            LinkC<T> Ln;
            load_link(sc + inext * kLinkConsts, Ln);
            F = carry_wrench(Ln.A, mk3(Ln.b[0], Ln.b[1], Ln.b[2]), cn, sn, F, ls.Fh);
        }
        tau[row + i] = F.n.z;
        if (MODE == kRecompute && i > 0) {
            T qdi = __ldg(qd + row + i), qddi = __ldg(qdd + row + i);
            x = backward_recover(L.A, mk3(L.b[0], L.b[1], L.b[2]), ls.c, ls.s, qdi, qddi, x);
        }
        cn = ls.c;
        sn = ls.s;
        inext = i;
    }
}

}  // namespace rdyn
