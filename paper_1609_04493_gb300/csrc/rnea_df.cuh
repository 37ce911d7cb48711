// rnea_df.cuh -- inverse dynamics of FP64 data in double-float arithmetic
// (RD_VARIANT_SERIAL_DF).
//
// The recursion of Sec. II-A in the common-normal frames of spatial_dh.cuh,
// one thread per instance, with every value a double-float pair (df.cuh,
// about 48 significand bits) instead of an FP64 number. GB300 executes 64
// FP32 fused multiply-adds per FP64 one, so the FP64 kernels are FP64-pipe
// bound; this one issues almost everything to the FP32 pipe. FP64 instructions
// remain only where the data is converted (q, qd, qdd in; tau out) and in the
// angle reduction of df_trig.cuh.
//
// * Constants: the 16 common-normal constants per link split into pairs on the
//   host, and theta0 in FP64 (for the angle reduction), as a __grid_constant__
//   kernel parameter (uniform data path).
// * State: cos and sin of each joint angle (two pairs, 16 bytes) per link in
//   shared memory, interleaved over the block's threads; the backward sweep
//   re-derives the motion by inverting the forward step (the forward operands
//   form a group, Sec. III-B) and recomputes F_hat.
// * Both sweeps iterate one link at a time: the double-float body is about ten
//   times the FP32 one, and unrolled it would not fit the instruction cache.
// For chains of at most NMAX links; rows of any length and alignment.
#pragma once
#include "df_trig.cuh"
#include "rnea_serial.cuh"
#include "spatial_dh.cuh"

namespace rdyn {

template <int NMAX>
struct DfParamConsts {
    DF c[NMAX * kDhConsts];  // common-normal constants of spatial_dh.cuh
    double th0[NMAX];        // joint offsets theta0_i
};

template <int NMAX, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
rnea_df_kernel(const __grid_constant__ DfParamConsts<NMAX> pc, int n, int B,
               const double *__restrict__ q, const double *__restrict__ qd,
               const double *__restrict__ qdd, double *__restrict__ tau, BaseParams<DF> base)
{
    extern __shared__ float4 df_cs[];  // [link][thread]: cos (hi, lo), sin (hi, lo)
    const int tid = threadIdx.x;
    const int b = blockIdx.x * BLOCK + tid;
    if (b >= B) return;
    const size_t row = (size_t)b * (size_t)n;
    const double *qr = q + row, *qdr = qd + row, *qddr = qdd + row;
    double *taur = tau + row;

    Motion<DF> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);

    // ---- forward sweep: base -> tip
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        const DF *p = pc.c + i * kDhConsts;
        DF s, c;
        df_sincos(__ldg(qr + i) + pc.th0[i], &s, &c);
        df_cs[i * BLOCK + tid] = make_float4(c.hi, c.lo, s.hi, s.lo);
        x = dh_forward(dh_rot(p[0], p[1], c, s), mk3(p[2], p[3], p[4]),
                       df_from_double(__ldg(qdr + i)), df_from_double(__ldg(qddr + i)), x);
    }

    // ---- backward sweep: tip -> base
    Wrench<DF> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    DhRot<DF> Rn = dh_rot(DF(1.0f), DF(0.0f), DF(1.0f), DF(0.0f));  // link i+1
    V3<DF> bn = mk3(DF(0.0f), DF(0.0f), DF(0.0f));
#pragma unroll 1
    for (int i = n - 1; i >= 0; --i) {
        const DF *p = pc.c + i * kDhConsts;
        const float4 v = df_cs[i * BLOCK + tid];
        const DhRot<DF> R = dh_rot(p[0], p[1], DF(v.x, v.y), DF(v.z, v.w));
        const V3<DF> bi = mk3(p[2], p[3], p[4]);
        const Wrench<DF> Fh = bias_wrench(p[6], mk3(p[7], p[8], p[9]), p + 10, x);
        if (i == n - 1) {
            F.f = add3(F.f, Fh.f);
            F.n = add3(F.n, Fh.n);
        } else {
            F = dh_carry(Rn, bn, F, Fh);
        }
        taur[i] = df_to_double(F.n.z);
        if (i > 0)
            x = dh_recover(R, bi, df_from_double(__ldg(qdr + i)), df_from_double(__ldg(qddr + i)),
                           x);
        Rn = R;
        bn = bi;
    }
}

}  // namespace rdyn
