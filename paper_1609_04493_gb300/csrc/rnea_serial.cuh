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
//                 III-B, so each step is invertible) and recomputes F_hat_i;
//   kRecomputeCS -- as kRecompute, but (cos q_i, sin q_i) go to shared memory
//                 (2 scalars per link per thread) instead of being re-evaluated.
#pragma once
#include <cuda_pipeline_primitives.h>

#include "spatial.cuh"

namespace rdyn {

template <typename T>
struct BaseParams {
    T V0[6];
    T dV0[6];
    T Fn[6];  // F_{n+1} in the joint frame of link n
};

enum StateMode { kStore = 0, kRecompute = 1, kRecomputeCS = 2 };

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
__host__ __device__ constexpr int state_bytes_per_link(int mode)
{
    return (mode == kStore ? 8 : mode == kRecomputeCS ? 2 : 0) * (int)sizeof(T);
}

template <typename T>
__device__ __forceinline__ void put_cs(unsigned char *base, int i, int tid, int block, T c, T s)
{
    if constexpr (sizeof(T) == 4)
        reinterpret_cast<float2 *>(base)[i * block + tid] = make_float2(c, s);
    else
        reinterpret_cast<double2 *>(base)[i * block + tid] = make_double2(c, s);
}

template <typename T>
__device__ __forceinline__ void get_cs(const unsigned char *base, int i, int tid, int block,
                                       T &c, T &s)
{
    if constexpr (sizeof(T) == 4) {
        float2 v = reinterpret_cast<const float2 *>(base)[i * block + tid];
        c = v.x;
        s = v.y;
    } else {
        double2 v = reinterpret_cast<const double2 *>(base)[i * block + tid];
        c = v.x;
        s = v.y;
    }
}

// FP32 sine/cosine for the fast path: Cody & Waite's additive range reduction
// by 2*pi split into a float head and tail (r = x - k*2pi, |r| <= pi), then
// the SFU approximations, whose absolute error on [-pi, pi] is ~4e-7.
__device__ __forceinline__ void sincos_fast(float x, float *s, float *c)
{
    const float k = rintf(x * 0.159154943091895336f);
    float r = fmaf(-k, 6.28318548202514648f, x);
    r = fmaf(-k, -1.74845553146951715e-7f, r);
    __sincosf(r, s, c);
}

template <typename T, bool FAST>
__device__ __forceinline__ void joint_trig(T x, T *s, T *c)
{
    if constexpr (FAST && sizeof(T) == 4) sincos_fast(x, s, c);
    else sincos_t(x, s, c);
}

// Four consecutive joint values of one row.
template <typename T>
struct Chunk {
    T v[4];
};

// VEC: n % 4 == 0 and 16-byte aligned rows, whole chunks with vector loads;
// otherwise element loads with a bound check.
template <typename T, bool VEC>
__device__ __forceinline__ Chunk<T> ld_chunk(const T *__restrict__ p, int i0, int n)
{
    Chunk<T> c;
    if constexpr (VEC) {
        if constexpr (sizeof(T) == 4) {
            float4 t = __ldg(reinterpret_cast<const float4 *>(p + i0));
            c.v[0] = t.x; c.v[1] = t.y; c.v[2] = t.z; c.v[3] = t.w;
        } else {
            double2 a = __ldg(reinterpret_cast<const double2 *>(p + i0));
            double2 b = __ldg(reinterpret_cast<const double2 *>(p + i0 + 2));
            c.v[0] = a.x; c.v[1] = a.y; c.v[2] = b.x; c.v[3] = b.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) c.v[j] = (i0 + j < n) ? __ldg(p + i0 + j) : T(0);
    }
    return c;
}

template <typename T, bool VEC>
__device__ __forceinline__ void st_chunk(T *__restrict__ p, int i0, int n, const Chunk<T> &c)
{
    if constexpr (VEC) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(p + i0) = make_float4(c.v[0], c.v[1], c.v[2], c.v[3]);
        } else {
            *reinterpret_cast<double2 *>(p + i0) = make_double2(c.v[0], c.v[1]);
            *reinterpret_cast<double2 *>(p + i0 + 2) = make_double2(c.v[2], c.v[3]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (i0 + j < n) p[i0 + j] = c.v[j];
    }
}

// Rotation A and offset b of a link (the part the backward carry needs).
template <typename T>
struct LinkXf {
    T A[9];
    T b[3];
};

template <typename T>
__device__ __forceinline__ void load_xf(const T *p, LinkXf<T> &X)
{
    if constexpr (sizeof(T) == 4) {
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
        float4 a = p4[0], b = p4[1], c = p4[2];
        X.A[0] = a.x; X.A[1] = a.y; X.A[2] = a.z; X.A[3] = a.w;
        X.A[4] = b.x; X.A[5] = b.y; X.A[6] = b.z; X.A[7] = b.w;
        X.A[8] = c.x; X.b[0] = c.y; X.b[1] = c.z; X.b[2] = c.w;
    } else {
        const double2 *p2 = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double2 t = p2[k];
            if (2 * k < 9) X.A[2 * k] = t.x; else X.b[2 * k - 9] = t.x;
            if (2 * k + 1 < 9) X.A[2 * k + 1] = t.y; else X.b[2 * k + 1 - 9] = t.y;
        }
    }
}

// Asynchronous staging of the joint values (VEC path): every thread copies its
// own row's next chunks (4 links of q, qd, qdd) into a private slot of a
// kStages-deep ring in shared memory with cp.async, kStages - 1 chunks ahead
// of the chunk it is working on, so the loads are in flight without holding
// registers. A thread only ever reads what it copied itself, so no block
// barrier is involved: cp.async.wait_group orders each thread's own copies.
constexpr int kStages = 3;

template <typename T>
__host__ __device__ constexpr int vec16_per_chunk()
{
    return (4 * (int)sizeof(T)) / 16;  // 16-byte pieces in 4 joint values
}

template <typename T>
__host__ __device__ constexpr int stage_bytes_per_thread()
{
    return kStages * 3 * 4 * (int)sizeof(T);
}

// 16 bytes from global into shared memory asynchronously, cached in L2 only:
// the joint values are streamed once, so they need no L1 lines (the copy
// joins the same commit groups as __pipeline_memcpy_async)
__device__ __forceinline__ void cp_async16_cg(void *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}

template <typename T, int BLOCK>
__device__ __forceinline__ void stage_chunk(unsigned char *ring, int slot, int tid,
                                            const T *qr, const T *qdr, const T *qddr, int i0)
{
    constexpr int P = vec16_per_chunk<T>();
    float4 *r = reinterpret_cast<float4 *>(ring);
    const T *src[3] = {qr, qdr, qddr};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int h = 0; h < P; ++h)
            cp_async16_cg(&r[((slot * 3 + a) * P + h) * BLOCK + tid],
                          src[a] + i0 + h * (16 / (int)sizeof(T)));
}

template <typename T, int BLOCK>
__device__ __forceinline__ void read_chunk(const unsigned char *ring, int slot, int tid,
                                           Chunk<T> &cq, Chunk<T> &cqd, Chunk<T> &cqdd)
{
    constexpr int P = vec16_per_chunk<T>();
    const float4 *r = reinterpret_cast<const float4 *>(ring);
    Chunk<T> *dst[3] = {&cq, &cqd, &cqdd};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int h = 0; h < P; ++h) {
            float4 v = r[((slot * 3 + a) * P + h) * BLOCK + tid];
            if constexpr (sizeof(T) == 4) {
                dst[a]->v[0] = v.x; dst[a]->v[1] = v.y; dst[a]->v[2] = v.z; dst[a]->v[3] = v.w;
            } else {
                double2 d = *reinterpret_cast<double2 *>(&v);
                dst[a]->v[2 * h] = d.x;
                dst[a]->v[2 * h + 1] = d.y;
            }
        }
}

// Shared memory: n * 24 link constants, then (VEC) the staging ring, then
// the per-link state of the mode. Thread b of the grid evaluates instance b:
// forward sweep base -> tip, then backward sweep tip -> base, tau_i = z moment
// of F_i in joint frame i'.
template <typename T, int BLOCK, int MODE, bool VEC, bool FAST>
__global__ void __launch_bounds__(BLOCK)
rnea_serial_kernel(const T *__restrict__ consts, int n, int B, const T *__restrict__ q,
                   const T *__restrict__ qd, const T *__restrict__ qdd, T *__restrict__ tau,
                   BaseParams<T> base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *sc = reinterpret_cast<T *>(smem);
    const int nc = n * kLinkConsts;
    for (int k = threadIdx.x; k < nc; k += BLOCK) sc[k] = consts[k];
    unsigned char *ring = smem + (size_t)nc * sizeof(T);
    unsigned char *st = ring + (VEC ? (size_t)stage_bytes_per_thread<T>() * BLOCK : 0);
    __syncthreads();

    const int tid = threadIdx.x;
    const int b = blockIdx.x * BLOCK + tid;
    if (b >= B) return;
    const size_t row = (size_t)b * (size_t)n;
    const T *qr = q + row, *qdr = qd + row, *qddr = qdd + row;
    T *taur = tau + row;

    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);

    // ---- forward sweep: base -> tip, joint values staged ahead of use
    const int nchunks = (n + 3) / 4;
    Chunk<T> cq = {}, cqd = {}, cqdd = {};
    if constexpr (VEC) {
#pragma unroll
        for (int k = 0; k < kStages - 1; ++k) {
            if (k < nchunks) stage_chunk<T, BLOCK>(ring, k, tid, qr, qdr, qddr, 4 * k);
            __pipeline_commit();
        }
    } else {
        cq = ld_chunk<T, VEC>(qr, 0, n);
        cqd = ld_chunk<T, VEC>(qdr, 0, n);
        cqdd = ld_chunk<T, VEC>(qddr, 0, n);
    }
    for (int kc = 0; kc < nchunks; ++kc) {
        const int i0 = 4 * kc;
        Chunk<T> nq = cq, nqd = cqd, nqdd = cqdd;
        if constexpr (VEC) {
            const int ahead = kc + kStages - 1;
            if (ahead < nchunks) stage_chunk<T, BLOCK>(ring, ahead % kStages, tid, qr, qdr, qddr, 4 * ahead);
            __pipeline_commit();
            __pipeline_wait_prior(kStages - 1);
            read_chunk<T, BLOCK>(ring, kc % kStages, tid, cq, cqd, cqdd);
        } else {
            nq = cq; nqd = cqd; nqdd = cqdd;
            if (i0 + 4 < n) {
                nq = ld_chunk<T, VEC>(qr, i0 + 4, n);
                nqd = ld_chunk<T, VEC>(qdr, i0 + 4, n);
                nqdd = ld_chunk<T, VEC>(qddr, i0 + 4, n);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            if (VEC || i < n) {
                LinkC<T> L;
                load_link(sc + i * kLinkConsts, L);
                T s, c;
                joint_trig<T, FAST>(cq.v[j], &s, &c);
                const Rot<T> R = make_rot(L.A, c, s);
                x = forward_step_R(R, mk3(L.b[0], L.b[1], L.b[2]), cqd.v[j], cqdd.v[j], x);
                if constexpr (MODE == kStore) {
                    LinkState<T> ls;
                    ls.Fh = bias_wrench(L.m, mk3(L.c[0], L.c[1], L.c[2]), L.I, x);
                    ls.c = c;
                    ls.s = s;
                    put_state<T>(st, i, tid, BLOCK, ls);
                } else if constexpr (MODE == kRecomputeCS) {
                    put_cs<T>(st, i, tid, BLOCK, c, s);
                }
            }
        }
        if constexpr (!VEC) {
            cq = nq;
            cqd = nqd;
            cqdd = nqdd;
        }
    }

    // ---- backward sweep: tip -> base
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    constexpr bool kNeedJoints = MODE != kStore;
    LinkXf<T> Xn;  // kStore: A, b of link i+1 (with cn, sn)
    T cn = T(1), sn = T(0);
    Rot<T> Rn;     // recompute modes: rotation of link i+1
    V3<T> bn = mk3(T(0), T(0), T(0));
    const int last0 = ((n - 1) / 4) * 4;
    if (kNeedJoints) {
        if constexpr (VEC) {
#pragma unroll
            for (int k = 0; k < kStages - 1; ++k) {
                const int c = nchunks - 1 - k;
                if (c >= 0) stage_chunk<T, BLOCK>(ring, k, tid, qr, qdr, qddr, 4 * c);
                __pipeline_commit();
            }
        } else {
            cq = ld_chunk<T, VEC>(qr, last0, n);
            cqd = ld_chunk<T, VEC>(qdr, last0, n);
            cqdd = ld_chunk<T, VEC>(qddr, last0, n);
        }
    }
    for (int kb = 0; kb < nchunks; ++kb) {
        const int i0 = last0 - 4 * kb;
        Chunk<T> nq = cq, nqd = cqd, nqdd = cqdd;
        if (kNeedJoints) {
            if constexpr (VEC) {
                const int ahead = kb + kStages - 1;
                if (ahead < nchunks)
                    stage_chunk<T, BLOCK>(ring, ahead % kStages, tid, qr, qdr, qddr,
                                          last0 - 4 * ahead);
                __pipeline_commit();
                __pipeline_wait_prior(kStages - 1);
                read_chunk<T, BLOCK>(ring, kb % kStages, tid, cq, cqd, cqdd);
            } else {
                nq = cq; nqd = cqd; nqdd = cqdd;
                if (i0 > 0) {
                    nq = ld_chunk<T, VEC>(qr, i0 - 4, n);
                    nqd = ld_chunk<T, VEC>(qdr, i0 - 4, n);
                    nqdd = ld_chunk<T, VEC>(qddr, i0 - 4, n);
                }
            }
        }
        Chunk<T> ct;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            ct.v[j] = T(0);
            if (VEC || i < n) {
                if constexpr (MODE == kStore) {
                    LinkState<T> ls;
                    get_state<T>(st, i, tid, BLOCK, ls);
                    if (i == n - 1) {
                        F.f = add3(F.f, ls.Fh.f);
                        F.n = add3(F.n, ls.Fh.n);
                    } else {
                        F = carry_wrench(Xn.A, mk3(Xn.b[0], Xn.b[1], Xn.b[2]), cn, sn, F, ls.Fh);
                    }
                    load_xf(sc + i * kLinkConsts, Xn);
                    cn = ls.c;
                    sn = ls.s;
                } else {
                    LinkC<T> L;
                    load_link(sc + i * kLinkConsts, L);
                    T s, c;
                    if constexpr (MODE == kRecomputeCS) get_cs<T>(st, i, tid, BLOCK, c, s);
                    else joint_trig<T, FAST>(cq.v[j], &s, &c);
                    const Rot<T> R = make_rot(L.A, c, s);
                    const V3<T> bi = mk3(L.b[0], L.b[1], L.b[2]);
                    const Wrench<T> Fh = bias_wrench(L.m, mk3(L.c[0], L.c[1], L.c[2]), L.I, x);
                    if (i == n - 1) {
                        F.f = add3(F.f, Fh.f);
                        F.n = add3(F.n, Fh.n);
                    } else {
                        F = carry_wrench_R(Rn, bn, F, Fh);
                    }
                    if (i > 0) x = backward_recover_R(R, bi, cqd.v[j], cqdd.v[j], x);
                    Rn = R;
                    bn = bi;
                }
                ct.v[j] = F.n.z;
            }
        }
        st_chunk<T, VEC>(taur, i0, n, ct);
        if (kNeedJoints && !VEC) {
            cq = nq;
            cqd = nqd;
            cqdd = nqdd;
        }
    }
}

}  // namespace rdyn
