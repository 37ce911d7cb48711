// rnea_dht.cuh -- the common-normal-frame RNEA of rnea_dhp.cuh with the
// backward-sweep state of the first links held in tensor memory (TMEM).
//
// rnea_dhp_kernel keeps F_hat, cos and sin of the first K links in shared
// memory; at n = 32 that caps it at 7 blocks of 32 threads per SM, and a batch
// of 65536 runs in two waves. Each SM also has 256 KB of TMEM (128 lanes x 512
// columns of 32 bits), which no other part of this kernel uses. Here a block of
// 128 threads allocates 128 columns: warp w reaches lanes 32 (w % 4) .. +31, so
// every thread owns 128 columns of its lane, room for the 8-scalar state of 16
// links. Four such blocks fill an SM's TMEM, and with the rest of the state in
// shared memory (about 416 bytes per thread) 512 threads per SM stay resident:
// the whole batch in one wave.
//
// Layout per thread: links 0..TL-1 in TMEM (columns 8 i .. 8 i + 7:
// F_hat.f, F_hat.n, cos, sin), links TL..K-1 full state in shared memory, links
// K..n-1 cos/sin only (their motion is re-derived, as in rnea_dhp.cuh). TMEM is
// written with tcgen05.st (one .x8 per link) and read with tcgen05.ld (.x32 per
// chunk of four links) followed by tcgen05.wait::ld.
//
// Every thread of a block runs to the end (threads past their share evaluate
// the share's last row and store nothing), because the tcgen05 instructions are
// warp-wide and the block's TMEM is released after a block barrier. The grid is
// four blocks per SM, each with an equal share of the batch. The dynamic shared
// memory of a block is padded so that at most four blocks share an SM, which
// keeps their allocations within the 512 columns.
#pragma once
#include <cstdint>

#include "rnea_dhp.cuh"

namespace rdyn {

constexpr int kDhtThreads = 128;
constexpr int kDhtCols = 128;        // TMEM columns per block
constexpr int kDhtMaxTmemLinks = 16; // kDhtCols / 8

__device__ __forceinline__ uint32_t dht_smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// TMEM is not memory the compiler sees, so the data movements below carry no
// "memory" clobber (one would force every parameter-space constant to be read
// again after each of them); volatile keeps them in program order.
__device__ __forceinline__ void dht_st8(uint32_t addr, const float v[8])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(addr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])));
}

// 32 consecutive columns of the thread's lane. The registers are valid only
// after tcgen05.wait::ld, which takes them as in-out operands so that no use
// is scheduled between the load and the wait.
__device__ __forceinline__ void dht_ld32_wait(uint32_t addr, uint32_t r[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31]));
}

__device__ __forceinline__ void dht_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;"); }

template <int STAGES>
__host__ __device__ constexpr size_t dht_ring_bytes_per_thread()
{
    return (size_t)STAGES * 3 * 4 * sizeof(float);
}

__host__ __device__ constexpr size_t dht_smem_per_thread(int n, int K, int TL, int stages)
{
    return (size_t)stages * 3 * 4 * sizeof(float) + (size_t)(K - TL) * 8 * sizeof(float) +
           (size_t)(n - K) * 2 * sizeof(float);
}

// FP32 only. Shared memory: the staging ring (STAGES slots), then links TL..K-1
// x 8 scalars, then links K..n-1 x 2 scalars, each interleaved over the block.
template <int NMAX, int TRIG, int STAGES>
__global__ void __launch_bounds__(kDhtThreads, 4)
rnea_dht_kernel(const __grid_constant__ DhParamConsts<float, NMAX> pc, int n, int K, int TL, int B,
                int per_block, int per_round, const float *__restrict__ q,
                const float *__restrict__ qd, const float *__restrict__ qdd,
                float *__restrict__ tau, BaseParams<float> base)
{
    using T = float;
    constexpr int BLOCK = kDhtThreads;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t tmem_base_s;
    unsigned char *ring = smem;
    unsigned char *stf = ring + dht_ring_bytes_per_thread<STAGES>() * BLOCK;  // links TL..K-1
    unsigned char *stc = stf + (size_t)(K - TL) * 8 * sizeof(T) * BLOCK;      // links K..n-1
    const T *sc = pc.c;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         dht_smem_u32(&tmem_base_s)),
                     "n"(kDhtCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s + ((uint32_t)(32 * (warp & 3)) << 16);

    // Block g takes instances [g per_block, (g + 1) per_block) in rounds of
    // per_round threads, so every SM gets the same share of the batch.
    const long long first = (long long)blockIdx.x * per_block;
    const long long end = first + per_block < (long long)B ? first + per_block : (long long)B;
    for (long long r0 = first; r0 < end; r0 += per_round) {
    const long long bi = r0 + tid;
    const bool active = tid < per_round && bi < end;
    const size_t row = (size_t)(active ? bi : end - 1) * (size_t)n;
    const T *qr = q + row, *qdr = qd + row, *qddr = qdd + row;
    T *taur = tau + row;

    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);

    // ---- forward sweep: base -> tip
    const int nchunks = n / 4, kchunks = K / 4, tchunks = TL / 4;
    Chunk<T> cq, cqd, cqdd;
#pragma unroll
    for (int k = 0; k < STAGES - 1; ++k) {
        if (k < nchunks) stage_chunk<T, BLOCK>(ring, k, tid, qr, qdr, qddr, 4 * k);
        __pipeline_commit();
    }
    for (int kc = 0; kc < nchunks; ++kc) {
        const int i0 = 4 * kc;
        const int ahead = kc + STAGES - 1;
        if (ahead < nchunks) stage_chunk<T, BLOCK>(ring, ahead % STAGES, tid, qr, qdr, qddr, 4 * ahead);
        __pipeline_commit();
        __pipeline_wait_prior(STAGES - 1);
        read_chunk<T, BLOCK>(ring, kc % STAGES, tid, cq, cqd, cqdd);
        if (kc < kchunks) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = i0 + j;
                DhLink<T> L;
                load_dh(sc + i * kDhConsts, L);
                T s, c;
                dh_trig<T, TRIG>(cq.v[j] + L.th0, &s, &c);
                x = dh_forward(dh_rot(L.ca, L.sa, c, s), L.b, cqd.v[j], cqdd.v[j], x);
                LinkState<T> ls;
                ls.Fh = bias_wrench(L.m, L.c, L.I, x);
                ls.c = c;
                ls.s = s;
                if (kc < tchunks) {
                    const float v[8] = {ls.Fh.f.x, ls.Fh.f.y, ls.Fh.f.z, ls.Fh.n.x,
                                        ls.Fh.n.y, ls.Fh.n.z, c,         s};
                    dht_st8(tmem + 8 * i, v);
                } else {
                    put_state<T>(stf, i - TL, tid, BLOCK, ls);
                }
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
    dht_wait_st();

    // ---- backward sweep: tip -> base
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    DhRot<T> Rn = dh_rot(T(1), T(0), T(1), T(0));  // rotation of link i+1
    V3<T> bn = mk3(T(0), T(0), T(0));
    const int last0 = n - 4;
    const int nrc = nchunks - kchunks;
    // links K..n-1: motion re-derived; the ring still holds the last STAGES
    // forward chunks, read in place; older ones are staged STAGES - 1 ahead
    for (int kb = 0; kb < nrc; ++kb) {
        const int i0 = last0 - 4 * kb;
        const int ahead = kb + STAGES - 1;
        if (ahead >= STAGES && ahead < nrc) {
            const int c = nchunks - 1 - ahead;
            stage_chunk2<T, BLOCK>(ring, c % STAGES, tid, qdr, qddr, 4 * c);
        }
        __pipeline_commit();
        __pipeline_wait_prior(STAGES - 1);
        Chunk<T> cqd2, cqdd2;
        read_chunk2<T, BLOCK>(ring, (nchunks - 1 - kb) % STAGES, tid, cqd2, cqdd2);
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
            if (i > K) x = dh_recover(R, L.b, cqd2.v[j], cqdd2.v[j], x);
            Rn = R;
            bn = L.b;
            ct.v[j] = F.n.z;
        }
        if (active) st_chunk<T, true>(taur, i0, n, ct);
    }
    // links TL..K-1: full state in shared memory; then 0..TL-1: full state in TMEM
    for (int kb = nrc; kb < nchunks; ++kb) {
        const int i0 = last0 - 4 * kb;
        const bool in_tmem = i0 < TL;
        uint32_t tr[32];
        if (in_tmem) dht_ld32_wait(tmem + 8 * i0, tr);
        Chunk<T> ct;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            LinkState<T> ls;
            if (in_tmem) {
                const uint32_t *r = tr + 8 * j;
                ls.Fh.f = mk3(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]));
                ls.Fh.n = mk3(__uint_as_float(r[3]), __uint_as_float(r[4]), __uint_as_float(r[5]));
                ls.c = __uint_as_float(r[6]);
                ls.s = __uint_as_float(r[7]);
            } else {
                get_state<T>(stf, i - TL, tid, BLOCK, ls);
            }
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
            ct.v[j] = F.n.z;
        }
        if (active) st_chunk<T, true>(taur, i0, n, ct);
    }
    }  // rounds

    // release the block's TMEM once every warp is done with it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_s),
                     "n"(kDhtCols)
                     : "memory");
}

}  // namespace rdyn
