// rnea_hybrid.cuh -- one thread per instance, per-link backward-sweep state
// kept for the first K links only.
//
// The shared-memory-state kernel (rnea_serial_kernel<kStore>) holds 8 scalars
// per link per thread, which at n = 32 in FP32 leaves room for about five warps
// per SM; the stateless kernel (kRecompute) fills the SM but pays for inverting
// the forward step and re-forming every bias wrench in the backward sweep. Here
// links 0..K-1 keep (F_hat_i, cos q_i, sin q_i) in shared memory and links
// K..n-1 are recomputed: the backward sweep inverts the forward step from the
// tip down to link K, then reads the stored state below. K (a multiple of 4)
// trades instructions for resident warps; K = n is the stored kernel, K = 0
// the stateless one. Same arithmetic as rnea_serial_kernel (Sec. II-A, Eqs.
// id-forward and id-backward, in joint frames).
#pragma once
#include "rnea_serial.cuh"

namespace rdyn {

// Shared memory: n * 24 constants, the cp.async ring (VEC), then K * 8
// scalars of state per thread. K % 4 == 0.
template <typename T, int BLOCK, bool VEC, bool FAST>
__global__ void __launch_bounds__(BLOCK)
rnea_hybrid_kernel(const T *__restrict__ consts, int n, int K, int B, const T *__restrict__ q,
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

    const int nchunks = (n + 3) / 4;
    const int kchunks = K / 4 < nchunks ? K / 4 : nchunks;  // chunks with stored state

    // ---- forward sweep: base -> tip; state of the first K links to shared memory
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
        } else if (i0 + 4 < n) {
            nq = ld_chunk<T, VEC>(qr, i0 + 4, n);
            nqd = ld_chunk<T, VEC>(qdr, i0 + 4, n);
            nqdd = ld_chunk<T, VEC>(qddr, i0 + 4, n);
        }
        const bool keep = kc < kchunks;
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
                if (keep) {
                    LinkState<T> ls;
                    ls.Fh = bias_wrench(L.m, mk3(L.c[0], L.c[1], L.c[2]), L.I, x);
                    ls.c = c;
                    ls.s = s;
                    put_state<T>(st, i, tid, BLOCK, ls);
                }
            }
        }
        if constexpr (!VEC) {
            cq = nq;
            cqd = nqd;
            cqdd = nqdd;
        }
    }

    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    Rot<T> Rn;  // rotation and offset of link i+1 (recomputed region)
    V3<T> bn = mk3(T(0), T(0), T(0));

    // ---- backward sweep, links n-1 .. K: re-derive the motion, re-form F_hat
    const int last0 = ((n - 1) / 4) * 4;
    const int nrc = nchunks - kchunks;  // recomputed chunks, walked tip -> base
    if (nrc > 0) {
        if constexpr (VEC) {
#pragma unroll
            for (int k = 0; k < kStages - 1; ++k) {
                if (k < nrc) stage_chunk<T, BLOCK>(ring, k, tid, qr, qdr, qddr, last0 - 4 * k);
                __pipeline_commit();
            }
        } else {
            cq = ld_chunk<T, VEC>(qr, last0, n);
            cqd = ld_chunk<T, VEC>(qdr, last0, n);
            cqdd = ld_chunk<T, VEC>(qddr, last0, n);
        }
    }
    for (int kb = 0; kb < nrc; ++kb) {
        const int i0 = last0 - 4 * kb;
        Chunk<T> nq = cq, nqd = cqd, nqdd = cqdd;
        if constexpr (VEC) {
            const int ahead = kb + kStages - 1;
            if (ahead < nrc)
                stage_chunk<T, BLOCK>(ring, ahead % kStages, tid, qr, qdr, qddr, last0 - 4 * ahead);
            __pipeline_commit();
            __pipeline_wait_prior(kStages - 1);
            read_chunk<T, BLOCK>(ring, kb % kStages, tid, cq, cqd, cqdd);
        } else if (kb + 1 < nrc) {
            nq = ld_chunk<T, VEC>(qr, i0 - 4, n);
            nqd = ld_chunk<T, VEC>(qdr, i0 - 4, n);
            nqdd = ld_chunk<T, VEC>(qddr, i0 - 4, n);
        }
        Chunk<T> ct;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            ct.v[j] = T(0);
            if (VEC || i < n) {
                LinkC<T> L;
                load_link(sc + i * kLinkConsts, L);
                T s, c;
                joint_trig<T, FAST>(cq.v[j], &s, &c);
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
                ct.v[j] = F.n.z;
            }
        }
        st_chunk<T, VEC>(taur, i0, n, ct);
        if constexpr (!VEC) {
            cq = nq;
            cqd = nqd;
            cqdd = nqdd;
        }
    }

    // ---- backward sweep, links K-1 .. 0: stored state
    LinkXf<T> Xn;  // A, b of link i+1 with (cn, sn), once inside the stored region
    T cn = T(1), sn = T(0);
    for (int kc = kchunks - 1; kc >= 0; --kc) {
        const int i0 = 4 * kc;
        Chunk<T> ct;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            ct.v[j] = T(0);
            if (VEC || i < n) {
                LinkState<T> ls;
                get_state<T>(st, i, tid, BLOCK, ls);
                if (i == n - 1) {
                    F.f = add3(F.f, ls.Fh.f);
                    F.n = add3(F.n, ls.Fh.n);
                } else if (i + 1 == 4 * kchunks) {
                    F = carry_wrench_R(Rn, bn, F, ls.Fh);  // link i+1 was recomputed
                } else {
                    F = carry_wrench(Xn.A, mk3(Xn.b[0], Xn.b[1], Xn.b[2]), cn, sn, F, ls.Fh);
                }
                load_xf(sc + i * kLinkConsts, Xn);
                cn = ls.c;
                sn = ls.s;
                ct.v[j] = F.n.z;
            }
        }
        st_chunk<T, VEC>(taur, i0, n, ct);
    }
}

template <typename T>
__host__ __device__ constexpr size_t hybrid_smem_bytes(int n, int K, int block, bool vec)
{
    return (size_t)n * kLinkConsts * sizeof(T) +
           (vec ? (size_t)stage_bytes_per_thread<T>() * block : 0) +
           (size_t)K * state_bytes_per_link<T>(kStore) * block;
}

}  // namespace rdyn
