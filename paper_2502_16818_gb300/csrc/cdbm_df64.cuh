// Double-float ("df64") arithmetic on the FP32 pipe for the CDBM_FP32_DF64 state.
//
// A value is an unevaluated sum hi + lo of two floats, about 48 significant bits.
// The operations are built from the classical error-free transformations: TwoSum
// (Knuth) for the exact rounding error of a sum, Fast-TwoSum (Dekker) when the
// larger operand is known, and the FMA-based TwoProduct for the exact error of a
// product.
//
// Error model.  Every quantity of the stage equilibrium is at most of the size of
// the reference equilibrium F (the moments of f, their products with O(1) block
// coefficients), and what must be accurate is the *absolute* error, against the
// single-precision deviation g = f - F the result is rounded to.  So the sums use
// the cheap ("sloppy") double-float addition, whose error is a few 2^-48 of its
// operands rather than of its result, and products are left unnormalised (the low
// part may reach a few ulp of the high part); both keep the absolute error of every
// quantity at a few 2^-47 of F, i.e. below 1/100 ulp of any deviation larger than
// about 2^-17 F.  Cancellation against F is harmless under this model: it only
// makes the final rounding to float relative to the smaller deviation.
//
// On GB300 the FP64 pipe runs 1/64 of the FP32 rate, so moving the equilibrium of
// the single-precision state from double to double-float trades each FP64
// instruction for 4-15 FP32 instructions that the four FP32 issue slots per SM
// absorb.
#pragma once

#include "cdbm_device.cuh"

namespace cdbm {

using df = DFPair;

__host__ __device__ inline df df_from(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ df df_of(float v) { return {v, 0.0f}; }

__device__ __forceinline__ float df_to_float(df x) { return __fadd_rn(x.hi, x.lo); }

// s + e = a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0).
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// x + y with an error of a few 2^-48 (|x| + |y|): exact sum of the high parts, the
// low parts added in float, renormalised once.
__device__ __forceinline__ df df_add(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(x.lo, y.lo), s.lo));
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// x * y, unnormalised: the exact error of hi * hi plus the cross terms (x.lo * y.lo
// is below the df rounding and dropped).
__device__ __forceinline__ df df_mul(df x, df y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return {p, e};
}

__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

// 1 / x: hardware float estimate (about 2^-23 relative) refined by one Newton step
// in df64, r + r (1 - x r), which squares the relative error.
__device__ __forceinline__ df df_rcp(df x)
{
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(x.hi));
    const df r = df_of(r0);
    const df e = df_sub(df_of(1.0f), df_mul(x, r));
    return df_add(r, df_mul(r, e));
}

// true iff v > 0 and finite (bit tests).
__device__ __forceinline__ bool positive_finite_f(float v)
{
    const int b = __float_as_int(v);
    return b > 0 && b < 0x7f800000;
}

__device__ __forceinline__ void rebuild_axis_f(float *o, float s0, float dq, float sx, float sy)
{
    const float A = s0 + dq, B = s0 - dq;
    o[0] = A + sx;
    o[2] = A - sx;
    o[1] = B + sy;
    o[3] = B - sy;
}

__device__ __forceinline__ void rebuild_diag_f(float *o, float s0, float q, float sx, float sy)
{
    const float P = s0 + q, Q = s0 - q, U = sx + sy, V = sx - sy;
    o[0] = P + U;
    o[2] = P - U;
    o[1] = Q - V;
    o[3] = Q + V;
}

// Scaled equilibrium deviation of one cell of the single-precision state, in df64:
// heq_i = gamma h (f_eq,i(m(F + g)) - F_i) rounded to float, from the stored
// deviations g (the same steps as primitives() and equilibrium<true>()).
__device__ __forceinline__ void df_equilibrium(const DFBlocks &B, const DFModel &d, const DFShift &R,
                                               const float fs[kNV], float heq[kNV], unsigned *flag)
{
    df s0[4], sx[4], sy[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const float *q = fs + 4 * g;
        if ((g & 1) == 0) {
            s0[g] = df_add(two_sum(q[0], q[2]), two_sum(q[1], q[3]));
            sx[g] = two_sum(q[0], -q[2]);
            sy[g] = two_sum(q[1], -q[3]);
        } else {
            const df e = two_sum(q[0], q[3]), w = two_sum(q[1], q[2]);
            sx[g] = df_sub(e, w);
            sy[g] = df_sub(two_sum(q[0], q[1]), two_sum(q[2], q[3]));
            s0[g] = df_add(e, w);
        }
    }
    const df rho = df_add(df_add(df_add(s0[0], s0[1]), df_add(s0[2], s0[3])), R.rhoF);
    df jx = df_mul(d.c[0], sx[0]), jy = df_mul(d.c[0], sy[0]), E = df_add(df_mul(d.w[0], s0[0]), R.EF);
#pragma unroll
    for (int g = 1; g < 4; ++g) {
        jx = df_fma(d.c[g], sx[g], jx);
        jy = df_fma(d.c[g], sy[g], jy);
        E = df_fma(d.w[g], s0[g], E);
    }
    const df r = df_rcp(rho);
    const df ux = df_mul(jx, r), uy = df_mul(jy, r);
    const df jyuy = df_mul(jy, uy);
    const df ru2 = df_fma(jx, ux, jyuy);
    const df P = df_mul(df_sub(E, ru2), d.invK);
    const df T = df_mul(P, r);
    if (!(positive_finite_f(rho.hi) && positive_finite_f(P.hi))) atomicOr(flag, kFlagNonPhys);

    const df ux2 = df_mul(ux, ux), uy2 = df_mul(uy, uy), u2 = df_add(ux2, uy2), du2 = df_sub(ux2, uy2);
    const df m1416 = df_fma(T, df_fma(d.Kp6, ru2, df_mul(d.twoKp2, P)), df_mul(ru2, u2));
    const df W4 = df_fma(d.Kp4, T, u2);
    const df d57 = df_sub(df_mul(jx, ux), jyuy);
    const df m6 = df_mul(jx, uy);
    float c0[4], cx[4], cy[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const df *S = B.S + 4 * g;
        const df s = df_fma(S[3], m1416, df_fma(S[2], ru2, df_fma(S[1], E, df_mul(S[0], rho))));
        c0[g] = df_to_float(df_sub(s, R.sF[g]));
        // V0 + V1 u_x^2 + V2 u_y^2 + V3 T and its mirror, through the shared part
        // V0 + V3 T + (V1 + V2)/2 u^2 and the odd part (V1 - V2)/2 (u_x^2 - u_y^2)
        const df cm = df_fma(B.Vs[g], u2, df_fma(B.V3[g], T, B.V0[g]));
        const df cd = df_mul(B.Vd[g], du2);
        cx[g] = df_to_float(df_mul(jx, df_add(cm, cd)));
        cy[g] = df_to_float(df_mul(jy, df_sub(cm, cd)));
    }
    const float dqa = df_to_float(df_mul(d57, df_fma(B.B1[1], W4, B.B1[0])));
    const float dqc = df_to_float(df_mul(d57, df_fma(B.B1[3], W4, B.B1[2])));
    const float qb = df_to_float(df_mul(m6, df_fma(B.B2[1], W4, B.B2[0])));
    const float qd = df_to_float(df_mul(m6, df_fma(B.B2[3], W4, B.B2[2])));
    rebuild_axis_f(heq + 0, c0[0], dqa, cx[0], cy[0]);
    rebuild_diag_f(heq + 4, c0[1], qb, cx[1], cy[1]);
    rebuild_axis_f(heq + 8, c0[2], dqc, cx[2], cy[2]);
    rebuild_diag_f(heq + 12, c0[3], qd, cx[3], cy[3]);
}

}  // namespace cdbm
