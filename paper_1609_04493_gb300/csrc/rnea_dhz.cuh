// rnea_dhz.cuh -- inverse dynamics straight from and to host memory
// (rnea_batch_host on mapped pinned arrays, FP32).
//
// The host arrays cross the host link once either way, whatever moves them;
// here the kernel moves them itself instead of the copy engines. Each block
// owns BLOCK consecutive rows, which are one contiguous slab of every [B, n]
// array:
//   1. it loads the q, qd and qdd slabs from host memory with 16-byte loads
//      (a warp reads 512 contiguous bytes per instruction) into shared memory,
//      rows padded to n + 1 floats so that the per-row reads below are free of
//      bank conflicts;
//   2. each thread runs the recursion of Sec. II-A on its row in the
//      common-normal frames of spatial_dh.cuh: forward sweep, then the backward
//      sweep re-deriving the motion (the forward operands form a group,
//      Sec. III-B); cos and sin of each joint wait in the slots of q and of tau;
//   3. the block writes its tau slab back to host memory with 16-byte stores.
// Each block walks the slabs with a grid stride, so after the first round the
// blocks of an SM are out of phase and one block's stores overlap another's
// loads.
// For n % 4 == 0, n <= NMAX and 16-byte aligned arrays.
#pragma once
#include "rnea_dhp.cuh"

namespace rdyn {

template <int NMAX, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
rnea_dhz_kernel(const __grid_constant__ DhParamConsts<float, NMAX> pc, int n, int B,
                const float *q, const float *qd, const float *qdd, float *tau,
                BaseParams<float> base)
{
    extern __shared__ float zs[];
    const int ld = n + 1;
    float *sq = zs, *sqd = sq + BLOCK * ld, *sqdd = sqd + BLOCK * ld, *stau = sqdd + BLOCK * ld;
    const int tid = threadIdx.x;
    const int slabs = (B + BLOCK - 1) / BLOCK;
    for (int slab = blockIdx.x; slab < slabs; slab += gridDim.x) {
        const long long b0 = (long long)slab * BLOCK;
        const int rows = (int)(B - b0 < BLOCK ? B - b0 : BLOCK);
        // 16-byte pieces per slab (n % 4 == 0 keeps each piece in one row)
        const int quads = rows * n / 4;
        const size_t off = (size_t)b0 * (size_t)n;

        // ---- 1. slabs in
        {
            const float4 *gq = reinterpret_cast<const float4 *>(q + off);
            const float4 *gqd = reinterpret_cast<const float4 *>(qd + off);
            const float4 *gqdd = reinterpret_cast<const float4 *>(qdd + off);
#pragma unroll 2
            for (int k = tid; k < quads; k += BLOCK) {
                const float4 a = gq[k], b = gqd[k], c = gqdd[k];
                const int e = 4 * k, r = e / n, col = e - r * n;
                float *dq = sq + r * ld + col, *dqd = sqd + r * ld + col;
                float *dqdd = sqdd + r * ld + col;
                dq[0] = a.x; dq[1] = a.y; dq[2] = a.z; dq[3] = a.w;
                dqd[0] = b.x; dqd[1] = b.y; dqd[2] = b.z; dqd[3] = b.w;
                dqdd[0] = c.x; dqdd[1] = c.y; dqdd[2] = c.z; dqdd[3] = c.w;
            }
        }
        __syncthreads();

        // ---- 2. one row per thread
        if (tid < rows) {
            float *rq = sq + tid * ld, *rqd = sqd + tid * ld, *rqdd = sqdd + tid * ld;
            float *rtau = stau + tid * ld;
            const float *sc = pc.c;
            Motion<float> x;
            x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
            x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
            x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
            x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);
            for (int i = 0; i < n; ++i) {
                DhXf<float> X;
                load_dh_xf(sc + i * kDhConsts, X);
                float s, c;
                sincos_poly(rq[i] + X.th0, &s, &c);
                rq[i] = c;
                rtau[i] = s;
                x = dh_forward(dh_rot(X.ca, X.sa, c, s), X.b, rqd[i], rqdd[i], x);
            }
            Wrench<float> F;
            F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
            F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
            DhRot<float> Rn = dh_rot(1.0f, 0.0f, 1.0f, 0.0f);
            V3<float> bn = mk3(0.0f, 0.0f, 0.0f);
            for (int i = n - 1; i >= 0; --i) {
                DhLink<float> L;
                load_dh(sc + i * kDhConsts, L);
                const DhRot<float> R = dh_rot(L.ca, L.sa, rq[i], rtau[i]);
                const Wrench<float> Fh = bias_wrench(L.m, L.c, L.I, x);
                if (i == n - 1) {
                    F.f = add3(F.f, Fh.f);
                    F.n = add3(F.n, Fh.n);
                } else {
                    F = dh_carry(Rn, bn, F, Fh);
                }
                rtau[i] = F.n.z;
                if (i > 0) x = dh_recover(R, L.b, rqd[i], rqdd[i], x);
                Rn = R;
                bn = L.b;
            }
        }
        __syncthreads();

        // ---- 3. tau slab out
        float4 *gt = reinterpret_cast<float4 *>(tau + off);
#pragma unroll 2
        for (int k = tid; k < quads; k += BLOCK) {
            const int e = 4 * k, r = e / n, col = e - r * n;
            const float *src = stau + r * ld + col;
            gt[k] = make_float4(src[0], src[1], src[2], src[3]);
        }
    }
}

}  // namespace rdyn
