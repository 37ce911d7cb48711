// rnea_dhp.cuh -- the common-normal-frame RNEA of rnea_dh.cuh with the link
// constants passed as a __grid_constant__ kernel parameter, and a per-link
// backward-sweep state that is full for the first K links only.
//
// * Constants. Their index is the same for every thread of a warp, so they are
//   read through the uniform data path and take no slot in the per-thread
//   memory pipeline, which then carries only the joint values (a cp.async ring,
//   two chunks ahead) and the state.
// * State. Links 0..K-1 keep F_hat_i, cos and sin (8 scalars); links K..n-1
//   keep cos and sin only (2 scalars), and the backward sweep re-derives their
//   motion by inverting the forward step (the forward operands form a group,
//   Sec. III-B) and recomputes F_hat_i. K trades shared memory, and with it the
//   number of resident warps, against arithmetic; K = n is the plain stored
//   sweep, K = 0 the stateless one.
// * Trigonometry (FP32). The default evaluates sin/cos of q_i + theta0_i with
//   the FMA-pipe polynomials of trig_poly.cuh (error under one ulp); TRIG = 1
//   selects the special-function-unit approximation (RD_FLAG_FAST_TRIG). FP64
//   uses the library's sincos.
// For chains of at most NMAX links, n % 4 == 0 and 16-byte aligned rows.
#pragma once
#include "rnea_dh.cuh"
#include "trig_poly.cuh"

namespace rdyn {

template <typename T, int NMAX>
struct DhParamConsts {
    T c[NMAX * kDhConsts];
};

enum DhTrig { kTrigPoly = 0, kTrigSfu = 1 };

template <typename T, int TRIG>
__device__ __forceinline__ void dh_trig(T x, T *s, T *c)
{
    if constexpr (sizeof(T) == 8) sincos(x, s, c);
    else if constexpr (TRIG == kTrigSfu) sincos_fast(x, s, c);
    else sincos_poly(x, s, c);
}

// Four joint values of a row (16-byte aligned) into registers.
template <typename T>
__device__ __forceinline__ void ld_row_chunk(const T *__restrict__ p, int i0, Chunk<T> &c)
{
    if constexpr (sizeof(T) == 4) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p + i0));
        c.v[0] = t.x; c.v[1] = t.y; c.v[2] = t.z; c.v[3] = t.w;
    } else {
        double2 a = __ldg(reinterpret_cast<const double2 *>(p + i0));
        double2 b = __ldg(reinterpret_cast<const double2 *>(p + i0 + 2));
        c.v[0] = a.x; c.v[1] = a.y; c.v[2] = b.x; c.v[3] = b.y;
    }
}

// The backward sweep needs qd and qdd only; they sit at positions 1 and 2 of
// the forward ring's slots.
template <typename T, int BLOCK>
__device__ __forceinline__ void stage_chunk2(unsigned char *ring, int slot, int tid,
                                             const T *qdr, const T *qddr, int i0)
{
    constexpr int P = vec16_per_chunk<T>();
    float4 *r = reinterpret_cast<float4 *>(ring);
    const T *src[2] = {qdr, qddr};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int h = 0; h < P; ++h)
            cp_async16_cg(&r[((slot * 3 + a + 1) * P + h) * BLOCK + tid],
                          src[a] + i0 + h * (16 / (int)sizeof(T)));
}

template <typename T, int BLOCK>
__device__ __forceinline__ void read_chunk2(const unsigned char *ring, int slot, int tid,
                                            Chunk<T> &cqd, Chunk<T> &cqdd)
{
    constexpr int P = vec16_per_chunk<T>();
    const float4 *r = reinterpret_cast<const float4 *>(ring);
    Chunk<T> *dst[2] = {&cqd, &cqdd};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int h = 0; h < P; ++h) {
            float4 v = r[((slot * 3 + a + 1) * P + h) * BLOCK + tid];
            if constexpr (sizeof(T) == 4) {
                dst[a]->v[0] = v.x; dst[a]->v[1] = v.y; dst[a]->v[2] = v.z; dst[a]->v[3] = v.w;
            } else {
                double2 d = *reinterpret_cast<double2 *>(&v);
                dst[a]->v[2 * h] = d.x;
                dst[a]->v[2 * h + 1] = d.y;
            }
        }
}

// RL: how many of the K stored links (the first ones) keep their state in
// registers instead of shared memory
// STG: depth of the joint-value staging ring (3, or 2 to save shared memory)
template <typename T>
__host__ __device__ constexpr size_t dhp_smem_per_thread(int n, int K, int RL = 0, int STG = kStages)
{
    return (size_t)STG * 3 * 4 * sizeof(T) + (size_t)(K - RL) * 8 * sizeof(T) +
           (size_t)(n - K) * 2 * sizeof(T);
}

// Shared memory: the staging ring, then links RL..K-1 x 8 scalars, then
// (n - K) links x 2 scalars, each interleaved over the block's threads. The
// state of links 0..RL-1 (RL a multiple of 4, K >= RL) stays in registers: the
// chunks that hold them run as unrolled copies of the loop body, first in the
// forward sweep and last in the backward sweep, so every register index is a
// compile-time constant. With less shared memory per block more blocks are
// resident.
template <typename T, int NMAX, int BLOCK, int TRIG, int RL = 0, int STG = kStages>
__global__ void __launch_bounds__(BLOCK)
rnea_dhp_kernel(const __grid_constant__ DhParamConsts<T, NMAX> pc, int n, int K, int B,
                const T *__restrict__ q, const T *__restrict__ qd, const T *__restrict__ qdd,
                T *__restrict__ tau, BaseParams<T> base)
{
    static_assert(RL % 4 == 0 && RL >= 0 && RL <= 16, "register links: 0, 4, 8, 12 or 16");
    static_assert(STG == 2 || STG == 3, "staging ring of 2 or 3 chunks");
    constexpr int kRegChunks = RL / 4;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *ring = smem;
    unsigned char *stf = ring + (size_t)STG * 3 * 4 * sizeof(T) * BLOCK;
    unsigned char *stc = stf + (size_t)(K - RL) * 8 * sizeof(T) * BLOCK;
    LinkState<T> rs[kRegChunks > 0 ? RL : 1];
    const T *sc = pc.c;

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

    // ---- forward sweep: base -> tip
    const int nchunks = n / 4, kchunks = K / 4;
    Chunk<T> cq, cqd, cqdd;
#pragma unroll
    for (int k = 0; k < STG - 1; ++k) {
        if (k < nchunks) stage_chunk<T, BLOCK>(ring, k, tid, qr, qdr, qddr, 4 * k);
        __pipeline_commit();
    }
    // one stored link of the forward sweep: motion, bias wrench, cos, sin
    auto forward_stored = [&](int i, T qi, T qdi, T qddi) -> LinkState<T> {
        DhLink<T> L;
        load_dh(sc + i * kDhConsts, L);
        T s, c;
        dh_trig<T, TRIG>(qi + L.th0, &s, &c);
        x = dh_forward(dh_rot(L.ca, L.sa, c, s), L.b, qdi, qddi, x);
        LinkState<T> ls;
        ls.Fh = bias_wrench(L.m, L.c, L.I, x);
        ls.c = c;
        ls.s = s;
        return ls;
    };
    // the chunks whose state stays in registers
#pragma unroll
    for (int kc = 0; kc < kRegChunks; ++kc) {
        const int ahead = kc + STG - 1;
        if (ahead < nchunks) stage_chunk<T, BLOCK>(ring, ahead % STG, tid, qr, qdr, qddr, 4 * ahead);
        __pipeline_commit();
        __pipeline_wait_prior(STG - 1);
        read_chunk<T, BLOCK>(ring, kc % STG, tid, cq, cqd, cqdd);
#pragma unroll
        for (int j = 0; j < 4; ++j) rs[4 * kc + j] = forward_stored(4 * kc + j, cq.v[j], cqd.v[j], cqdd.v[j]);
    }
    for (int kc = kRegChunks; kc < nchunks; ++kc) {
        const int i0 = 4 * kc;
        const int ahead = kc + STG - 1;
        if (ahead < nchunks) stage_chunk<T, BLOCK>(ring, ahead % STG, tid, qr, qdr, qddr, 4 * ahead);
        __pipeline_commit();
        __pipeline_wait_prior(STG - 1);
        read_chunk<T, BLOCK>(ring, kc % STG, tid, cq, cqd, cqdd);
        if (kc < kchunks) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = i0 + j;
                put_state<T>(stf, i - RL, tid, BLOCK, forward_stored(i, cq.v[j], cqd.v[j], cqdd.v[j]));
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = i0 + j;
                DhXf<T> X;
                load_dh_xf(sc + i * kDhConsts, X);
                T s, c;
                dh_trig<T, TRIG>(cq.v[j] + X.th0, &s, &c);
                x = dh_forward(dh_rot(X.ca, X.sa, c, s), X.b, cqd.v[j], cqdd.v[j], x);
                put_cs<T>(stc, i - K, tid, BLOCK, c, s);
            }
        }
    }

    // ---- backward sweep: tip -> base; first the links without full state
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    DhRot<T> Rn = dh_rot(T(1), T(0), T(1), T(0));  // rotation of link i+1
    V3<T> bn = mk3(T(0), T(0), T(0));
    const int last0 = n - 4;
    const int nrc = nchunks - kchunks;
    // Forward chunk c was staged in slot c % STG and is only overwritten by
    // chunk c + STG, so the ring still holds the last STG chunks: the
    // backward sweep reads those in place and stages older ones STG - 1
    // steps ahead, each into the slot of the chunk read one step before.
    for (int kb = 0; kb < nrc; ++kb) {
        const int i0 = last0 - 4 * kb;
        const int ahead = kb + STG - 1;
        if (ahead >= STG && ahead < nrc) {
            const int c = nchunks - 1 - ahead;
            stage_chunk2<T, BLOCK>(ring, c % STG, tid, qdr, qddr, 4 * c);
        }
        __pipeline_commit();
        __pipeline_wait_prior(STG - 1);
        read_chunk2<T, BLOCK>(ring, (nchunks - 1 - kb) % STG, tid, cqd, cqdd);
        Chunk<T> ct;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            DhLink<T> L;
            load_dh(sc + i * kDhConsts, L);
            T s, c;
            get_cs<T>(stc, i - K, tid, BLOCK, c, s);
            const DhRot<T> R = dh_rot(L.ca, L.sa, c, s);
            const Wrench<T> Fh = bias_wrench(L.m, L.c, L.I, x);
            if (i == n - 1) {
                F.f = add3(F.f, Fh.f);
                F.n = add3(F.n, Fh.n);
            } else {
                F = dh_carry(Rn, bn, F, Fh);
            }
            if (i > K) x = dh_recover(R, L.b, cqd.v[j], cqdd.v[j], x);
            Rn = R;
            bn = L.b;
            ct.v[j] = F.n.z;
        }
        st_chunk<T, true>(taur, i0, n, ct);
    }
    // ---- then the links with full state: shared memory, then registers
    auto backward_stored = [&](int i, const LinkState<T> &ls) -> T {
        if (i == n - 1) {
            F.f = add3(F.f, ls.Fh.f);
            F.n = add3(F.n, ls.Fh.n);
        } else {
            F = dh_carry(Rn, bn, F, ls.Fh);
        }
        DhXf<T> X;
        load_dh_xf(sc + i * kDhConsts, X);
        Rn = dh_rot(X.ca, X.sa, ls.c, ls.s);
        bn = X.b;
        return F.n.z;
    };
    for (int kb = nrc; kb < nchunks - kRegChunks; ++kb) {
        const int i0 = last0 - 4 * kb;
        Chunk<T> ct;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            LinkState<T> ls;
            get_state<T>(stf, i - RL, tid, BLOCK, ls);
            ct.v[j] = backward_stored(i, ls);
        }
        st_chunk<T, true>(taur, i0, n, ct);
    }
#pragma unroll
    for (int kc = kRegChunks - 1; kc >= 0; --kc) {
        Chunk<T> ct;
#pragma unroll
        for (int j = 3; j >= 0; --j) ct.v[j] = backward_stored(4 * kc + j, rs[4 * kc + j]);
        st_chunk<T, true>(taur, 4 * kc, n, ct);
    }
}

}  // namespace rdyn
