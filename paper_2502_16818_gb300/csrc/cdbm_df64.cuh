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
// single-precision deviation g = f - F the result is rounded to.  So the sums add
// the high parts exactly and the low parts in float and leave the pair unnormalised
// (df_add_q), with an error of a few 2^-48 of the operands rather than of the result,
// and products are left unnormalised too (the low part may reach a few ulp of the
// high part); both keep the absolute error of every quantity at a few 2^-47 of F,
// i.e. below 1/100 ulp of any deviation larger than about 2^-17 F.  Only the density
// is renormalised, because its reciprocal starts from the high part.  Cancellation
// against F is harmless under this model: it only makes the final rounding to float
// relative to the smaller deviation.
//
// On GB300 the FP64 pipe runs 1/64 of the FP32 rate, so moving the equilibrium of
// the single-precision state from double to double-float trades each FP64
// instruction for 4-15 FP32 instructions that the four FP32 issue slots per SM
// absorb.
//
// Lanes.  Every function is written once over a lane type L: float computes one
// cell, float2 two cells with the packed FP32x2 instructions of sm_100 and later
// (one instruction issue for two IEEE operations).  The packed operations round
// each half exactly as the scalar ones do, so the two-cell form gives, cell by
// cell, the same bits as the one-cell form.
#pragma once

#include "cdbm_device.cuh"

namespace cdbm {

// ---- lane operations: float or float2, each IEEE round-to-nearest ----
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add_rn(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub_rn(float2 a, float2 b) { return __fadd2_rn(a, neg(b)); }
__device__ __forceinline__ float2 mul_rn(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma_rn(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <typename L>
using dfl = DFv<L>;
using df = DFPair;

__host__ __device__ inline df df_from(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

template <typename L>
__device__ __forceinline__ dfl<L> df_of(L v)
{
    if constexpr (std::is_same<L, float>::value) return {v, 0.0f}; else return {v, make_float2(0.0f, 0.0f)};
}

template <typename L>
__device__ __forceinline__ L df_to_float(dfl<L> x) { return add_rn(x.hi, x.lo); }

// s + e = a + b exactly.
template <typename L>
__device__ __forceinline__ dfl<L> two_sum(L a, L b)
{
    const L s = add_rn(a, b);
    const L bb = sub_rn(s, a);
    const L e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0).
template <typename L>
__device__ __forceinline__ dfl<L> fast_two_sum(L a, L b)
{
    const L s = add_rn(a, b);
    const L e = sub_rn(b, sub_rn(s, a));
    return {s, e};
}

// x + y with an error of a few 2^-48 (|x| + |y|): exact sum of the high parts, the
// low parts added in float, renormalised once.
template <typename L>
__device__ __forceinline__ dfl<L> df_add(dfl<L> x, dfl<L> y)
{
    const dfl<L> s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, add_rn(add_rn(x.lo, y.lo), s.lo));
}

template <typename L>
__device__ __forceinline__ dfl<L> df_neg(dfl<L> x) { return {neg(x.hi), neg(x.lo)}; }
template <typename L>
__device__ __forceinline__ dfl<L> df_sub(dfl<L> x, dfl<L> y) { return df_add(x, df_neg(y)); }

// x + y without the final renormalisation of df_add: the exact sum of the high parts
// and, in float, the low parts plus its rounding error.  The pair is left
// unnormalised: its low part may exceed half an ulp of the high part (by the low
// parts of the operands and, after cancellation, by more).  Under the absolute error
// model that costs nothing where the result feeds further sums, products or the final
// rounding to float: each of those forms the high parts exactly and carries the low
// parts as float terms whose rounding is 2^-24 of their own size, i.e. a few 2^-48 of
// the operands.  Only the reciprocal, which starts from the high part, takes a
// normalised operand (df_norm).
template <typename L>
__device__ __forceinline__ dfl<L> df_add_q(dfl<L> x, dfl<L> y)
{
    const dfl<L> s = two_sum(x.hi, y.hi);
    return {s.hi, add_rn(add_rn(x.lo, y.lo), s.lo)};
}
template <typename L>
__device__ __forceinline__ dfl<L> df_sub_q(dfl<L> x, dfl<L> y) { return df_add_q(x, df_neg(y)); }

// The pair renormalised (|lo| <= half an ulp of hi).
template <typename L>
__device__ __forceinline__ dfl<L> df_norm(dfl<L> x) { return fast_two_sum(x.hi, x.lo); }

// x * y, unnormalised: the exact error of hi * hi plus the cross terms (x.lo * y.lo
// is below the df rounding and dropped).
template <typename L>
__device__ __forceinline__ dfl<L> df_mul(dfl<L> x, dfl<L> y)
{
    const L p = mul_rn(x.hi, y.hi);
    L e = fma_rn(x.hi, y.hi, neg(p));
    e = fma_rn(x.hi, y.lo, e);
    e = fma_rn(x.lo, y.hi, e);
    return {p, e};
}

template <typename L>
__device__ __forceinline__ dfl<L> df_fma(dfl<L> a, dfl<L> b, dfl<L> c) { return df_add(df_mul(a, b), c); }
template <typename L>
__device__ __forceinline__ dfl<L> df_fma_q(dfl<L> a, dfl<L> b, dfl<L> c) { return df_add_q(df_mul(a, b), c); }

// x * r for a plain float r: the exact error of hi * r plus lo * r.
template <typename L>
__device__ __forceinline__ dfl<L> df_mul1(dfl<L> x, L r)
{
    const L p = mul_rn(x.hi, r);
    return {p, fma_rn(x.lo, r, fma_rn(x.hi, r, neg(p)))};
}

__device__ __forceinline__ float rcp_estimate(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float2 rcp_estimate(float2 x) { return make_float2(rcp_estimate(x.x), rcp_estimate(x.y)); }

// 1 / x for a normalised x: hardware float estimate r (about 2^-23 relative)
// refined by one Newton step in df64, r + r (1 - x r), which squares the relative
// error.  The result is left unnormalised.
template <typename L>
__device__ __forceinline__ dfl<L> df_rcp(dfl<L> x)
{
    const L r = rcp_estimate(x.hi);
    L one;
    if constexpr (std::is_same<L, float>::value) one = 1.0f; else one = make_float2(1.0f, 1.0f);
    const dfl<L> e = df_sub_q(df_of(one), df_mul1(x, r));
    return df_add_q(df_of(r), df_mul1(e, r));
}

// true iff v > 0 and finite (bit tests), in every lane.
__device__ __forceinline__ bool positive_finite_f(float v)
{
    const int b = __float_as_int(v);
    return b > 0 && b < 0x7f800000;
}
__device__ __forceinline__ bool positive_finite_f(float2 v) { return positive_finite_f(v.x) && positive_finite_f(v.y); }

template <typename L>
__device__ __forceinline__ void rebuild_axis_f(L *o, L s0, L dq, L sx, L sy)
{
    const L A = add_rn(s0, dq), B = sub_rn(s0, dq);
    o[0] = add_rn(A, sx);
    o[2] = sub_rn(A, sx);
    o[1] = add_rn(B, sy);
    o[3] = sub_rn(B, sy);
}

template <typename L>
__device__ __forceinline__ void rebuild_diag_f(L *o, L s0, L q, L sx, L sy)
{
    const L P = add_rn(s0, q), Q = sub_rn(s0, q), U = add_rn(sx, sy), V = sub_rn(sx, sy);
    o[0] = add_rn(P, U);
    o[2] = sub_rn(P, U);
    o[1] = sub_rn(Q, V);
    o[3] = add_rn(Q, V);
}

// The df64 equilibrium in three parts, so that a cell can also be split over four
// threads, one per velocity group (the cluster kernel for small FP64-free grids):
// the group components (s0, sx, sy) of one group's four stored deviations; the
// scalars every group needs (moments, primitives, raw-moment factors); and one
// group's four equilibrium values.  df_equilibrium() is the three in sequence.

// Group components of group g from its four stored deviations q (the operations of
// conserved() on df64 values).
template <typename L>
__device__ __forceinline__ void df_group_components(int g, const L q[4], dfl<L> &s0, dfl<L> &sx, dfl<L> &sy)
{
    if ((g & 1) == 0) {
        s0 = df_add_q(two_sum(q[0], q[2]), two_sum(q[1], q[3]));
        sx = two_sum(q[0], neg(q[2]));
        sy = two_sum(q[1], neg(q[3]));
    } else {
        const dfl<L> e = two_sum(q[0], q[3]), w = two_sum(q[1], q[2]);
        sx = df_sub_q(e, w);
        sy = df_sub_q(two_sum(q[0], q[1]), two_sum(q[2], q[3]));
        s0 = df_add_q(e, w);
    }
}

template <typename L>
struct DFScalars {
    dfl<L> rho, E, jx, jy, r, ux, uy, jyuy, ru2, P, T, u2, du2, m1416, W4, d57, m6;
};

// Conserved moments from the group components of all four groups.  Every sum over
// the groups is taken pairwise, (a + b) + (c + d): two independent chains instead of
// one of three dependent double-float additions.
template <typename L>
__device__ __forceinline__ void df_sums(const DFModelT<L> &d, const DFShiftT<L> &R, const dfl<L> s0[4],
                                        const dfl<L> sx[4], const dfl<L> sy[4], DFScalars<L> &c)
{
    c.rho = df_norm(df_add_q(df_add_q(df_add_q(s0[0], s0[1]), df_add_q(s0[2], s0[3])), R.rhoF));
    c.jx = df_add_q(df_fma_q(d.c[1], sx[1], df_mul(d.c[0], sx[0])), df_fma_q(d.c[3], sx[3], df_mul(d.c[2], sx[2])));
    c.jy = df_add_q(df_fma_q(d.c[1], sy[1], df_mul(d.c[0], sy[0])), df_fma_q(d.c[3], sy[3], df_mul(d.c[2], sy[2])));
    c.E = df_add_q(df_add_q(df_fma_q(d.w[1], s0[1], df_mul(d.w[0], s0[0])),
                            df_fma_q(d.w[3], s0[3], df_mul(d.w[2], s0[2]))),
                   R.EF);
}

// Primitives and raw-moment factors from rho, j and E (the steps of primitives() and
// the shared part of equilibrium<true>()).  With j_x u_x and j_y u_y formed once,
// rho u^2 and m5 - m7 are their sum and difference, and u^2 = rho u^2 / rho,
// u_x^2 - u_y^2 = (m5 - m7) / rho.  Only rho, the operand of the reciprocal, is
// renormalised (in df_sums).
template <typename DM, typename L>
__device__ __forceinline__ void df_chain(const DM &d, DFScalars<L> &c, unsigned *flag)
{
    c.r = df_rcp(c.rho);
    c.ux = df_mul(c.jx, c.r);
    c.uy = df_mul(c.jy, c.r);
    const dfl<L> jxux = df_mul(c.jx, c.ux);
    c.jyuy = df_mul(c.jy, c.uy);
    c.ru2 = df_add_q(jxux, c.jyuy);
    c.d57 = df_sub_q(jxux, c.jyuy);
    c.P = df_mul(df_sub_q(c.E, c.ru2), d.invK);
    c.T = df_mul(c.P, c.r);
    if (flag && !(positive_finite_f(c.rho.hi) && positive_finite_f(c.P.hi))) atomicOr(flag, kFlagNonPhys);
    c.u2 = df_mul(c.ru2, c.r);
    c.du2 = df_mul(c.d57, c.r);
    c.m1416 = df_fma_q(c.T, df_fma_q(d.Kp6, c.ru2, df_mul(d.twoKp2, c.P)), df_mul(c.ru2, c.u2));
    c.W4 = df_fma_q(d.Kp4, c.T, c.u2);
    c.m6 = df_mul(c.jx, c.uy);
}

template <typename L>
__device__ __forceinline__ DFScalars<L> df_scalars(const DFModelT<L> &d, const DFShiftT<L> &R, const dfl<L> s0[4],
                                                   const dfl<L> sx[4], const dfl<L> sy[4], unsigned *flag)
{
    DFScalars<L> c;
    df_sums(d, R, s0, sx, sy, c);
    df_chain(d, c, flag);
    return c;
}

// The four scaled equilibrium deviations of group g.
template <typename L>
__device__ __forceinline__ void df_group_equilibrium(int g, const DFBlocksT<L> &B, const DFShiftT<L> &R,
                                                     const DFScalars<L> &c, L heq[4])
{
    const dfl<L> *S = B.S + 4 * g;
    const dfl<L> s = df_fma_q(S[3], c.m1416, df_fma_q(S[2], c.ru2, df_fma_q(S[1], c.E, df_mul(S[0], c.rho))));
    const L c0 = df_to_float(df_sub_q(s, R.sF[g]));
    // V0 + V1 u_x^2 + V2 u_y^2 + V3 T and its mirror, through the shared part
    // V0 + V3 T + (V1 + V2)/2 u^2 and the odd part (V1 - V2)/2 (u_x^2 - u_y^2)
    const dfl<L> cm = df_fma_q(B.Vs[g], c.u2, df_fma_q(B.V3[g], c.T, B.V0[g]));
    const dfl<L> cd = df_mul(B.Vd[g], c.du2);
    const L cx = df_to_float(df_mul(c.jx, df_add_q(cm, cd)));
    const L cy = df_to_float(df_mul(c.jy, df_sub_q(cm, cd)));
    if ((g & 1) == 0) {                 // g = 0: a, g = 2: c
        const L dq = df_to_float(df_mul(c.d57, df_fma_q(B.B1[g + 1], c.W4, B.B1[g])));
        rebuild_axis_f(heq, c0, dq, cx, cy);
    } else {                            // g = 1: b, g = 3: d
        const L q = df_to_float(df_mul(c.m6, df_fma_q(B.B2[g], c.W4, B.B2[g - 1])));
        rebuild_diag_f(heq, c0, q, cx, cy);
    }
}

// ---- the same on a y-symmetric 1-D state (see conserved_sym): j_y = u_y = 0 ----

// Group components without the y-odd one.
template <typename L>
__device__ __forceinline__ void df_group_components_sym(int g, const L q[4], dfl<L> &s0, dfl<L> &sx)
{
    if ((g & 1) == 0) {
        s0 = df_add_q(two_sum(q[0], q[2]), two_sum(q[1], q[3]));
        sx = two_sum(q[0], neg(q[2]));
    } else {
        const dfl<L> e = two_sum(q[0], q[3]), w = two_sum(q[1], q[2]);
        sx = df_sub_q(e, w);
        s0 = df_add_q(e, w);
    }
}

// df_scalars with j_y = u_y = 0: rho u^2 = m5 - m7 = j_x u_x and u_x^2 - u_y^2 = u^2;
// the fields of j_y, u_y, j_y u_y and m6 are left unset.
template <typename L>
__device__ __forceinline__ DFScalars<L> df_scalars_sym(const DFModelT<L> &d, const DFShiftT<L> &R,
                                                       const dfl<L> s0[4], const dfl<L> sx[4], unsigned *flag)
{
    DFScalars<L> c;
    c.rho = df_norm(df_add_q(df_add_q(df_add_q(s0[0], s0[1]), df_add_q(s0[2], s0[3])), R.rhoF));
    c.jx = df_add_q(df_fma_q(d.c[1], sx[1], df_mul(d.c[0], sx[0])), df_fma_q(d.c[3], sx[3], df_mul(d.c[2], sx[2])));
    c.E = df_add_q(df_add_q(df_fma_q(d.w[1], s0[1], df_mul(d.w[0], s0[0])),
                            df_fma_q(d.w[3], s0[3], df_mul(d.w[2], s0[2]))),
                   R.EF);
    c.r = df_rcp(c.rho);
    c.ux = df_mul(c.jx, c.r);
    c.ru2 = df_mul(c.jx, c.ux);
    c.d57 = c.ru2;
    c.P = df_mul(df_sub_q(c.E, c.ru2), d.invK);
    c.T = df_mul(c.P, c.r);
    if (flag && !(positive_finite_f(c.rho.hi) && positive_finite_f(c.P.hi))) atomicOr(flag, kFlagNonPhys);
    c.u2 = df_mul(c.ru2, c.r);
    c.du2 = c.u2;
    c.m1416 = df_fma_q(c.T, df_fma_q(d.Kp6, c.ru2, df_mul(d.twoKp2, c.P)), df_mul(c.ru2, c.u2));
    c.W4 = df_fma_q(d.Kp4, c.T, c.u2);
    return c;
}

// df_group_equilibrium on a symmetric state: no y-odd part, no diagonal quadrupole;
// heq receives all four members.
template <typename L>
__device__ __forceinline__ void df_group_equilibrium_sym(int g, const DFBlocksT<L> &B, const DFShiftT<L> &R,
                                                         const DFScalars<L> &c, L heq[4])
{
    const dfl<L> *S = B.S + 4 * g;
    const dfl<L> s = df_fma_q(S[3], c.m1416, df_fma_q(S[2], c.ru2, df_fma_q(S[1], c.E, df_mul(S[0], c.rho))));
    const L c0 = df_to_float(df_sub_q(s, R.sF[g]));
    const dfl<L> cm = df_fma_q(B.Vs[g], c.u2, df_fma_q(B.V3[g], c.T, B.V0[g]));
    const dfl<L> cd = df_mul(B.Vd[g], c.du2);
    const L cx = df_to_float(df_mul(c.jx, df_add_q(cm, cd)));
    if ((g & 1) == 0) {
        const L dq = df_to_float(df_mul(c.d57, df_fma_q(B.B1[g + 1], c.W4, B.B1[g])));
        const L A = add_rn(c0, dq), Bv = sub_rn(c0, dq);
        heq[0] = add_rn(A, cx);
        heq[2] = sub_rn(A, cx);
        heq[1] = Bv;
        heq[3] = Bv;
    } else {
        heq[0] = add_rn(c0, cx);
        heq[3] = heq[0];
        heq[1] = sub_rn(c0, cx);
        heq[2] = heq[1];
    }
}

// df_equilibrium on a symmetric state (all 16 values; fs holds all 16, the mirror
// images equal).
template <typename L>
__device__ __forceinline__ void df_equilibrium_sym(const DFBlocksT<L> &B, const DFModelT<L> &d,
                                                   const DFShiftT<L> &R, const L fs[kNV], L heq[kNV],
                                                   unsigned *flag)
{
    dfl<L> s0[4], sx[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) df_group_components_sym(g, fs + 4 * g, s0[g], sx[g]);
    const DFScalars<L> c = df_scalars_sym(d, R, s0, sx, flag);
#pragma unroll
    for (int g = 0; g < 4; ++g) df_group_equilibrium_sym(g, B, R, c, heq + 4 * g);
}

// Scaled equilibrium deviation of one cell (or, with L = float2, of two cells) of
// the single-precision state, in df64: heq_i = gamma h (f_eq,i(m(F + g)) - F_i)
// rounded to float, from the stored deviations g (the same steps as primitives()
// and equilibrium<true>()).
template <typename L>
__device__ __forceinline__ void df_equilibrium(const DFBlocksT<L> &B, const DFModelT<L> &d, const DFShiftT<L> &R,
                                               const L fs[kNV], L heq[kNV], unsigned *flag)
{
    dfl<L> s0[4], sx[4], sy[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) df_group_components(g, fs + 4 * g, s0[g], sx[g], sy[g]);
    const DFScalars<L> c = df_scalars(d, R, s0, sx, sy, flag);
#pragma unroll
    for (int g = 0; g < 4; ++g) df_group_equilibrium(g, B, R, c, heq + 4 * g);
}

}  // namespace cdbm
