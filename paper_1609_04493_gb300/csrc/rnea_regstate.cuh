// rnea_regstate.cuh -- one thread per instance, per-link backward-sweep state
// split between registers and shared memory.
//
// The shared-memory-state kernel (rnea_serial_kernel<kStore>) needs 32 bytes of
// state per link per thread, which caps it at a few warps per SM while most of
// the register file is unused. Here the state (F_hat_i, cos q_i, sin q_i) of
// the first RL links lives in registers -- those links are processed by fully
// unrolled code, so every access has a compile-time index -- and only links
// RL..n-1 go to shared memory. Same arithmetic as the serial kernel
// (Sec. II-A, Eqs. id-forward and id-backward, in joint frames).
#pragma once
#include "rnea_serial.cuh"

namespace rdyn {

template <typename T, int BLOCK>
struct RegStateCtx {
    const T *sc;
    unsigned char *ring;
    unsigned char *st;
    const T *qr, *qdr, *qddr;
    T *taur;
    int n, nchunks, tid;
};

// Prefetch for chunk kc (kStages - 1 ahead) and read chunk kc from the ring.
template <typename T, int BLOCK>
__device__ __forceinline__ void regstate_fetch(const RegStateCtx<T, BLOCK> &c, int kc,
                                               Chunk<T> &cq, Chunk<T> &cqd, Chunk<T> &cqdd)
{
    const int ahead = kc + kStages - 1;
    if (ahead < c.nchunks) stage_chunk<T, BLOCK>(c.ring, ahead % kStages, c.tid, c.qr, c.qdr, c.qddr, 4 * ahead);
    __pipeline_commit();
    __pipeline_wait_prior(kStages - 1);
    read_chunk<T, BLOCK>(c.ring, kc % kStages, c.tid, cq, cqd, cqdd);
}

// Forward step of link i: motion update and its state (F_hat, cos, sin).
template <typename T>
__device__ __forceinline__ void regstate_forward_link(const T *sc, int i, T q, T qd, T qdd,
                                                      Motion<T> &x, LinkState<T> &ls)
{
    LinkC<T> L;
    load_link(sc + i * kLinkConsts, L);
    T s, c;
    sincos_t(q, &s, &c);
    const Rot<T> R = make_rot(L.A, c, s);
    x = forward_step_R(R, mk3(L.b[0], L.b[1], L.b[2]), qd, qdd, x);
    ls.Fh = bias_wrench(L.m, mk3(L.c[0], L.c[1], L.c[2]), L.I, x);
    ls.c = c;
    ls.s = s;
}

// Backward step of link i given its state; Xn, cn, sn: transform of link i+1.
template <typename T>
__device__ __forceinline__ T regstate_backward_link(const T *sc, int i, int n, const LinkState<T> &ls,
                                                    Wrench<T> &F, LinkXf<T> &Xn, T &cn, T &sn)
{
    if (i == n - 1) {
        F.f = add3(F.f, ls.Fh.f);
        F.n = add3(F.n, ls.Fh.n);
    } else {
        F = carry_wrench(Xn.A, mk3(Xn.b[0], Xn.b[1], Xn.b[2]), cn, sn, F, ls.Fh);
    }
    load_xf(sc + i * kLinkConsts, Xn);
    cn = ls.c;
    sn = ls.s;
    return F.n.z;
}

// Requires n % 4 == 0 and 16-byte aligned rows (vector chunks). RL % 4 == 0.
// Shared memory: n * 24 constants, the cp.async ring, then (n - RL) * 8
// scalars of state per thread.
template <typename T, int BLOCK, int RL>
__global__ void __launch_bounds__(BLOCK)
rnea_regstate_kernel(const T *__restrict__ consts, int n, int B, const T *__restrict__ q,
                     const T *__restrict__ qd, const T *__restrict__ qdd, T *__restrict__ tau,
                     BaseParams<T> base)
{
    static_assert(RL % 4 == 0, "register links come in chunks of 4");
    extern __shared__ __align__(16) unsigned char smem[];
    T *sc = reinterpret_cast<T *>(smem);
    const int nc = n * kLinkConsts;
    for (int k = threadIdx.x; k < nc; k += BLOCK) sc[k] = consts[k];
    unsigned char *ring = smem + (size_t)nc * sizeof(T);
    unsigned char *st = ring + (size_t)stage_bytes_per_thread<T>() * BLOCK;
    __syncthreads();

    const int tid = threadIdx.x;
    const int b = blockIdx.x * BLOCK + tid;
    if (b >= B) return;
    const size_t row = (size_t)b * (size_t)n;
    RegStateCtx<T, BLOCK> ctx{sc, ring, st, q + row, qd + row, qdd + row, tau + row, n,
                              n / 4, tid};

    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);

#pragma unroll
    for (int k = 0; k < kStages - 1; ++k) {
        if (k < ctx.nchunks) stage_chunk<T, BLOCK>(ring, k, tid, ctx.qr, ctx.qdr, ctx.qddr, 4 * k);
        __pipeline_commit();
    }

    // ---- forward: links 0..RL-1 with register state (unrolled)
    LinkState<T> rs[RL > 0 ? RL : 1];
#pragma unroll
    for (int kc = 0; kc < RL / 4; ++kc) {
        if (4 * kc < n) {
            Chunk<T> cq, cqd, cqdd;
            regstate_fetch(ctx, kc, cq, cqd, cqdd);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                regstate_forward_link(sc, 4 * kc + j, cq.v[j], cqd.v[j], cqdd.v[j], x, rs[4 * kc + j]);
        }
    }
    // ---- forward: links RL..n-1 with shared-memory state
    for (int kc = RL / 4; kc < ctx.nchunks; ++kc) {
        Chunk<T> cq, cqd, cqdd;
        regstate_fetch(ctx, kc, cq, cqd, cqdd);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            LinkState<T> ls;
            regstate_forward_link(sc, 4 * kc + j, cq.v[j], cqd.v[j], cqdd.v[j], x, ls);
            put_state<T>(st, 4 * kc + j - RL, tid, BLOCK, ls);
        }
    }

    // ---- backward: links n-1..RL from shared memory
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    LinkXf<T> Xn;
    T cn = T(1), sn = T(0);
    for (int kc = ctx.nchunks - 1; kc >= RL / 4; --kc) {
        Chunk<T> ct;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            LinkState<T> ls;
            get_state<T>(st, 4 * kc + j - RL, tid, BLOCK, ls);
            ct.v[j] = regstate_backward_link(sc, 4 * kc + j, n, ls, F, Xn, cn, sn);
        }
        st_chunk<T, true>(ctx.taur, 4 * kc, n, ct);
    }
    // ---- backward: links RL-1..0 from registers (unrolled)
#pragma unroll
    for (int kc = RL / 4 - 1; kc >= 0; --kc) {
        if (4 * kc < n) {
            Chunk<T> ct;
#pragma unroll
            for (int j = 3; j >= 0; --j)
                ct.v[j] = regstate_backward_link(sc, 4 * kc + j, n, rs[4 * kc + j], F, Xn, cn, sn);
            st_chunk<T, true>(ctx.taur, 4 * kc, n, ct);
        }
    }
}

}  // namespace rdyn
