// Single-precision equilibrium of the deviation state (CDBM_FP32_DEV).
//
// The state stores g = f - F, F the equilibrium of the reference state (rho0, u = 0,
// T0).  The equilibrium deviation of a cell, gamma h (f_eq(m(F + g)) - F), is the
// factored product of Eqs. (6)-(7) applied to the *differences* of the moments from
// their reference values: the conserved sums of g are the deviations of rho and E
// directly, j and the u-terms vanish at the reference, and the remaining difference,
// that of m14 + m16 = T (K+6) rho u^2 + 2 (K+2) P T + rho u^2 u^2, is expanded as
//   2 (K+2) (P T - P0 T0) + rho u^2 ((K+6) T + u^2),  P T - P0 T0 = dT P + T0 dP,
// with dP = (dE - rho u^2) / K and dT = (dP - T0 drho) / rho.  No quantity of the size
// of F enters a subtraction, so single precision keeps the relative accuracy of the
// deviations themselves: the absolute error of heq is a few 2^-24 of the deviation,
// not of F.  The block coefficients, model constants and reference moments are the
// high parts of the df64 constants (the values rounded to float).
//
// One cell at a time, in scalar float.  The two-column kernel calls it once per
// column: written on the packed float2 lanes of the df64 code, the compiler fuses
// packed multiplies into the following packed additions, which would round
// differently from the one-column kernels, and the stage is not bound by this
// arithmetic.
#pragma once

#include "cdbm_df64.cuh"

namespace cdbm {

// 1 / x: the hardware estimate refined by one Newton step, r + r (1 - x r).
__device__ __forceinline__ float rcp_refined(float x)
{
    const float r = rcp_estimate(x);
    return fma_rn(r, fma_rn(-x, r, 1.0f), r);
}

// S . x for one group's row of the scalar block (four double-float coefficients,
// four float moments), compensated (the dot product of Ogita, Rump and Oishi): each
// product hi * x is split exactly into p + e by an FMA, the p are added with TwoSum,
// and the rounding errors, the e and the coefficients' low parts lo * x are
// accumulated in a second float.  The result is about as accurate as if computed
// in double and rounded, where the plain float sum loses the digits that cancel
// between the four terms (on a strong shock the temperature error of the run fell
// from 5.7e-4 to 6.1e-5).
__device__ __forceinline__ float block_dot(const DFPair *S, float x0, float x1, float x2, float x3)
{
    const float x[4] = {x0, x1, x2, x3};
    float p = mul_rn(S[0].hi, x[0]);
    float e = fma_rn(S[0].lo, x[0], fma_rn(S[0].hi, x[0], neg(p)));
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const float q = mul_rn(S[k].hi, x[k]);
        const float eq = fma_rn(S[k].lo, x[k], fma_rn(S[k].hi, x[k], neg(q)));
        const df t = two_sum(p, q);
        p = t.hi;
        e = add_rn(e, add_rn(t.lo, eq));
    }
    return add_rn(p, e);
}

// heq_i = gamma h (f_eq,i(m(F + g)) - F_i) of one cell from its stored
// deviations fs, in single precision.
//
// Conservation.  The collision invariants hold through identities among the block
// coefficients (the group rest values s_g sum to gamma h rho, and so on); rounded to
// float the coefficients miss them by about 2^-24, which leaves a small bias of
// the same sign in every cell and step (on the Sod tube a mass drift growing to
// 1.5e-5 over 10^4 steps).  So the equilibrium's mass, momentum and energy, taken
// from the group values before they are rebuilt into the 16 velocities (4 s_g,
// k_g (cx, cy)_g with k_g = 2 c_g on the axis groups and 4 c_g on the diagonal ones,
// 4 w_g s_g), are compared with gamma h times the cell's, and the residuals are
// added back along the invariants: s_g += alpha + beta w_g, (cx, cy)_g += c_g gamma.
// What remains is the rounding of these few operations, of either sign.
__device__ __forceinline__ void f32_equilibrium(const DFBlocks &B, const DFModel &d, const DFShift &R,
                                                const DevProj &J, const float fs[kNV], float heq[kNV], unsigned *flag)
{
    // group components (the operations of conserved())
    float s0[4], sx[4], sy[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const float *q = fs + 4 * g;
        if ((g & 1) == 0) {
            s0[g] = add_rn(add_rn(q[0], q[2]), add_rn(q[1], q[3]));
            sx[g] = sub_rn(q[0], q[2]);
            sy[g] = sub_rn(q[1], q[3]);
        } else {
            const float e = add_rn(q[0], q[3]), w = add_rn(q[1], q[2]);
            sx[g] = sub_rn(e, w);
            sy[g] = sub_rn(add_rn(q[0], q[1]), add_rn(q[2], q[3]));
            s0[g] = add_rn(e, w);
        }
    }
    // deviations of rho and E, and j (F carries no momentum); pairwise over the groups
    const float drho = add_rn(add_rn(s0[0], s0[1]), add_rn(s0[2], s0[3]));
    const float jx = add_rn(fma_rn(d.c[1].hi, sx[1], mul_rn(d.c[0].hi, sx[0])),
                        fma_rn(d.c[3].hi, sx[3], mul_rn(d.c[2].hi, sx[2])));
    const float jy = add_rn(fma_rn(d.c[1].hi, sy[1], mul_rn(d.c[0].hi, sy[0])),
                        fma_rn(d.c[3].hi, sy[3], mul_rn(d.c[2].hi, sy[2])));
    const float dE = add_rn(fma_rn(d.w[1].hi, s0[1], mul_rn(d.w[0].hi, s0[0])),
                        fma_rn(d.w[3].hi, s0[3], mul_rn(d.w[2].hi, s0[2])));
    // reference state: rho0 = sum F, P0 = E0 / K, T0 = P0 / rho0
    const float rho0 = R.rhoF.hi;
    const float P0 = mul_rn(R.EF.hi, d.invK.hi);
    const float T0 = mul_rn(P0, rcp_refined(rho0));
    // primitives
    const float rho = add_rn(rho0, drho);
    const float r = rcp_refined(rho);
    const float ux = mul_rn(jx, r), uy = mul_rn(jy, r);
    const float jxux = mul_rn(jx, ux), jyuy = mul_rn(jy, uy);
    const float ru2 = add_rn(jxux, jyuy), d57 = sub_rn(jxux, jyuy);      // rho u^2, m5 - m7
    const float dP = mul_rn(sub_rn(dE, ru2), d.invK.hi);
    const float P = add_rn(P0, dP);
    const float T = mul_rn(P, r);
    if (flag && !(positive_finite_f(rho) && positive_finite_f(P))) atomicOr(flag, kFlagNonPhys);
    const float dT = mul_rn(fma_rn(neg(T0), drho, dP), r);
    const float u2 = mul_rn(ru2, r), du2 = mul_rn(d57, r);              // u^2, u_x^2 - u_y^2
    // deviation of m14 + m16
    const float dm1416 = fma_rn(d.twoKp2.hi, fma_rn(dT, P, mul_rn(T0, dP)), mul_rn(ru2, fma_rn(d.Kp6.hi, T, u2)));
    const float W4 = fma_rn(d.Kp4.hi, T, u2);
    const float m6 = mul_rn(jx, uy);
    // per group: rest value s (the scalar block on the moment deviations), odd
    // components j times V0 + V3 T + (V1 + V2)/2 u^2 +- (V1 - V2)/2 (u_x^2 - u_y^2),
    // and the quadrupole (dq of an axis group, q of a diagonal one)
    float s[4], cx[4], cy[4], qv[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const DFPair *S = B.S + 4 * g;
        s[g] = block_dot(S, drho, dE, ru2, dm1416);
        const float cm = fma_rn(B.Vs[g].hi, u2, fma_rn(B.V3[g].hi, T, B.V0[g].hi));
        const float cd = mul_rn(B.Vd[g].hi, du2);
        cx[g] = mul_rn(jx, add_rn(cm, cd));
        cy[g] = mul_rn(jy, sub_rn(cm, cd));
        qv[g] = (g & 1) == 0 ? mul_rn(d57, fma_rn(B.B1[g + 1].hi, W4, B.B1[g].hi))
                             : mul_rn(m6, fma_rn(B.B2[g].hi, W4, B.B2[g - 1].hi));
    }
    // conservation residuals and their correction along the invariants
    const float two = 2.0f, four = 4.0f;
    const float ms = add_rn(add_rn(s[0], s[1]), add_rn(s[2], s[3]));
    const float es = add_rn(fma_rn(d.w[1].hi, s[1], mul_rn(d.w[0].hi, s[0])),
                        fma_rn(d.w[3].hi, s[3], mul_rn(d.w[2].hi, s[2])));
    // k_g c_g-weighted odd sums: 2 c on the axis groups, 4 c on the diagonal ones
    const float kx = fma_rn(two, add_rn(mul_rn(d.c[0].hi, cx[0]), mul_rn(d.c[2].hi, cx[2])),
                        mul_rn(four, add_rn(mul_rn(d.c[1].hi, cx[1]), mul_rn(d.c[3].hi, cx[3]))));
    const float ky = fma_rn(two, add_rn(mul_rn(d.c[0].hi, cy[0]), mul_rn(d.c[2].hi, cy[2])),
                        mul_rn(four, add_rn(mul_rn(d.c[1].hi, cy[1]), mul_rn(d.c[3].hi, cy[3]))));
    const float rm = fma_rn(neg(four), ms, mul_rn(J.gh, drho));
    const float re = fma_rn(neg(four), es, mul_rn(J.gh, dE));
    const float alpha = fma_rn(J.a01, re, mul_rn(J.a00, rm));
    const float beta = fma_rn(J.a11, re, mul_rn(J.a01, rm));
    const float gx = mul_rn(J.rkc, fma_rn(J.gh, jx, neg(kx)));
    const float gy = mul_rn(J.rkc, fma_rn(J.gh, jy, neg(ky)));
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const float sg = add_rn(s[g], fma_rn(beta, d.w[g].hi, alpha));
        const float cxg = fma_rn(d.c[g].hi, gx, cx[g]);
        const float cyg = fma_rn(d.c[g].hi, gy, cy[g]);
        if ((g & 1) == 0) rebuild_axis_f(heq + 4 * g, sg, qv[g], cxg, cyg);
        else rebuild_diag_f(heq + 4 * g, sg, qv[g], cxg, cyg);
    }
}

}  // namespace cdbm
