// Device building blocks of the CDBM kernels: velocity-set geometry, the
// conserved moments, the factored equilibrium, the minmod limiter and the NND
// transport difference.  Everything here is double precision; integer work
// (limiter decisions, validity tests, neighbour indices) is kept off the FP64
// pipe, which is the scarce unit on GB300.
#pragma once

#include <cstdint>
#include <type_traits>

#include "cdbm_convert.h"
#include "cdbm_internal.h"

namespace cdbm {

// Direction signs of velocity i (Eq. 2 with the fixed member order: axis groups
// (1,0),(0,1),(-1,0),(0,-1); diagonal groups (1,1),(-1,1),(-1,-1),(1,-1)).
__host__ __device__ constexpr int dirx(int i)
{
    return ((i >> 2) & 1) == 0 ? ((i & 3) == 0 ? 1 : ((i & 3) == 2 ? -1 : 0))
                               : (((i & 3) == 0 || (i & 3) == 3) ? 1 : -1);
}
__host__ __device__ constexpr int diry(int i)
{
    return ((i >> 2) & 1) == 0 ? ((i & 3) == 1 ? 1 : ((i & 3) == 3 ? -1 : 0))
                               : (((i & 3) <= 1) ? 1 : -1);
}

// true iff v > 0 and v is finite (sign, zero and exponent tested on the bits of
// the two 32-bit halves, which keeps the test on the integer pipe).
__device__ __forceinline__ bool positive_finite(double v)
{
    const int h = __double2hiint(v);
    const unsigned l = (unsigned)__double2loint(v);
    return h >= 0 && h < 0x7ff00000 && ((unsigned)h | l) != 0u;
}

// minmod of Eq. (16) on the integer pipe: zero when either argument is zero or
// the signs differ, otherwise the argument of smaller magnitude (X on a tie).
// Magnitudes of finite doubles order like their bit patterns without the sign.
// The tests work on the 32-bit halves: written on 64-bit integers they are turned
// back into FP64 compares by the compiler, which costs three FP64 instructions per
// transport difference on a GPU where the FP64 pipe is the bottleneck.
__device__ __forceinline__ double minmod(double X, double Y)
{
    const int hx = __double2hiint(X), lx = __double2loint(X);
    const int hy = __double2hiint(Y), ly = __double2loint(Y);
    const unsigned ahx = (unsigned)hx & 0x7fffffffu, ahy = (unsigned)hy & 0x7fffffffu;
    const bool x_le_y = (ahx < ahy) | ((ahx == ahy) & ((unsigned)lx <= (unsigned)ly));
    const bool keep = ((hx ^ hy) >= 0) & ((ahx | (unsigned)lx) != 0u) & ((ahy | (unsigned)ly) != 0u);
    const int rh = keep ? (x_le_y ? hx : hy) : 0;
    const int rl = keep ? (x_le_y ? lx : ly) : 0;
    return __hiloint2double(rh, rl);
}

// NND transport difference (Eqs. 12-20) in upwind order.  For a velocity
// component v along r, with u2, u1 the values two and one cells upwind, c the
// cell and d1 one cell downwind,
//   (H(j+1/2) - H(j-1/2)) / |v| = (c - u1) + [minmod(d1 - c, c - u1) - minmod(c - u1, u1 - u2)] / 2,
// which is Eqs. (13)-(20) for v > 0 and their mirror image for v < 0
// (f+ = v f, f- = 0, resp. f+ = 0, f- = v f).
__device__ __forceinline__ double nnd(double u2, double u1, double c, double d1)
{
    const double a = c - u1;
    const double b = d1 - c;
    const double e = u1 - u2;
    const double t = minmod(b, a) - minmod(a, e);
    return fma(0.5, t, a);
}

// Single-precision twins of minmod() and nnd() for the single-precision states.
// minmod: min.xorsign.abs gives min(|X|, |Y|) with the sign bit set iff the sign
// bits of X and Y differ; clamping it at zero and giving it X's sign yields the
// smaller magnitude with X's sign when the sign bits agree, else 0 (three
// instructions).  A zero argument gives a zero result either way, and equal
// magnitudes with equal signs are the same value, so this is the Eq. (16) reading
// of the double version; only the sign of an exact zero result may differ.
__device__ __forceinline__ float minmod(float X, float Y)
{
    float r;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(X), "f"(Y));
    return copysignf(fmaxf(r, 0.0f), X);
}

// minmod of the two lanes of packed pairs (no packed form of min.xorsign.abs).
__device__ __forceinline__ float2 minmod(float2 X, float2 Y)
{
    return make_float2(minmod(X.x, Y.x), minmod(X.y, Y.y));
}

__device__ __forceinline__ float nnd(float u2, float u1, float c, float d1)
{
    const float a = c - u1;
    const float b = d1 - c;
    const float e = u1 - u2;
    const float t = minmod(b, a) - minmod(a, e);
    return fmaf(0.5f, t, a);
}

// 1 / a for a > 0: hardware estimate refined by one cubic Newton-Raphson step,
// r (1 + e + e^2) with e = 1 - a r (error ~ e^3, below one ulp).
__device__ __forceinline__ double rcp64(double a)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
    const double e = fma(-a, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

struct Cons {
    double rho, jx, jy, E;   // sum f, sum f v_x, sum f v_y, sum f (v^2 + eta^2)
};

// Conserved moments of f (Eq. 4 rows 1-4 with f in place of f_eq), accumulated
// through the group components s0, sx, sy.
__device__ __forceinline__ Cons conserved(const double f[kNV], const ModelConsts &m)
{
    double s0[4], sx[4], sy[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const double *q = f + 4 * g;
        if ((g & 1) == 0) {          // axis: E N W S
            sx[g] = q[0] - q[2];
            sy[g] = q[1] - q[3];
            s0[g] = (q[0] + q[2]) + (q[1] + q[3]);
        } else {                     // diagonal: NE NW SW SE
            const double e = q[0] + q[3], w = q[1] + q[2];
            sx[g] = e - w;
            sy[g] = (q[0] + q[1]) - (q[2] + q[3]);
            s0[g] = e + w;
        }
    }
    Cons r;
    r.rho = (s0[0] + s0[1]) + (s0[2] + s0[3]);
    r.jx = fma(m.c[3], sx[3], fma(m.c[2], sx[2], fma(m.c[1], sx[1], m.c[0] * sx[0])));
    r.jy = fma(m.c[3], sy[3], fma(m.c[2], sy[2], fma(m.c[1], sy[1], m.c[0] * sy[0])));
    r.E = fma(m.w[3], s0[3], fma(m.w[2], s0[2], fma(m.w[1], s0[1], m.w[0] * s0[0])));
    return r;
}

// Members of an axis group (E N W S) from the group sum s0, the quadrupole dq and the
// odd components j_x px, j_y py (the products fused into the sums).
__device__ __forceinline__ void rebuild_axis(double *o, double s0, double dq, double jx, double px,
                                             double jy, double py)
{
    const double A = s0 + dq, B = s0 - dq;
    o[0] = fma(jx, px, A);
    o[2] = fma(-jx, px, A);
    o[1] = fma(jy, py, B);
    o[3] = fma(-jy, py, B);
}

// Members of a diagonal group (NE NW SW SE), likewise.
__device__ __forceinline__ void rebuild_diag(double *o, double s0, double q, double jx, double px,
                                             double jy, double py)
{
    const double sy = jy * py;
    const double P = s0 + q, Q = s0 - q, U = fma(jx, px, sy), V = fma(jx, px, -sy);
    o[0] = P + U;   // NE
    o[2] = P - U;   // SW
    o[1] = Q - V;   // NW
    o[3] = Q + V;   // SE
}

// One group's members of the scaled equilibrium: s0 from the scalar block, the odd
// polynomials from their common part and half difference (Vc), the quadrupole qv
// (dq of an axis group, q of a diagonal one) given.
__device__ __forceinline__ void equilibrium_group(const EqBlocks &B, int g, double s0, double qv,
                                                  double jx, double jy, double T, double u2,
                                                  double dlt, double *o)
{
    const double *W = B.Vc + 4 * g;
    const double cm = fma(W[2], u2, fma(W[1], T, W[0]));
    const double px = fma(W[3], dlt, cm), py = fma(-W[3], dlt, cm);
    if ((g & 1) == 0) rebuild_axis(o, s0, qv, jx, px, jy, py);
    else rebuild_diag(o, s0, qv, jx, px, jy, py);
}

// Scaled equilibrium out_i = scale * f_eq,i (Eqs. 4-7) in factored form: the raw
// moments of the Maxwellian (binomial shift of the central moments of Eq. 5 by u)
// times the parity-blocked inverse of M(0), with the moment products folded into
// the block coefficients (see EqBlocks).  Inputs: rho, E = sum f (v^2+eta^2),
// j = rho u, u, rho u^2, j_y u_y, P = rho T and T.
// With kShift, s0_shift[g] is subtracted from the group sums before the rebuild,
// i.e. a reference equilibrium constant per group is taken off the result.
template <bool kShift = false>
__device__ __forceinline__ void equilibrium(const EqBlocks &B, const ModelConsts &m, double rho,
                                            double E, double jx, double jy, double ux, double uy,
                                            double ru2, double jyuy, double P, double T,
                                            double out[kNV], const double *s0_shift = nullptr)
{
    const double ux2 = ux * ux, uy2 = uy * uy, u2 = ux2 + uy2, dlt = ux2 - uy2;
    const double m1416 = fma(T, fma(m.Kp6, ru2, m.twoKp2 * P), ru2 * u2);  // m14 + m16
    const double W4 = fma(m.Kp4, T, u2);
    const double d57 = fma(jx, ux, -jyuy);                                  // m5 - m7
    const double m6 = jx * uy;
    double s0[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const double *S = B.S + 4 * g;
        if (kShift)   // the reference group value enters the innermost product as its addend
            s0[g] = fma(S[3], m1416, fma(S[2], ru2, fma(S[1], E, fma(S[0], rho, -s0_shift[g]))));
        else
            s0[g] = fma(S[3], m1416, fma(S[2], ru2, fma(S[1], E, S[0] * rho)));
    }
    const double dqa = d57 * fma(B.B1[1], W4, B.B1[0]);
    const double dqc = d57 * fma(B.B1[3], W4, B.B1[2]);
    const double qb = m6 * fma(B.B2[1], W4, B.B2[0]);
    const double qd = m6 * fma(B.B2[3], W4, B.B2[2]);
    equilibrium_group(B, 0, s0[0], dqa, jx, jy, T, u2, dlt, out + 0);
    equilibrium_group(B, 1, s0[1], qb, jx, jy, T, u2, dlt, out + 4);
    equilibrium_group(B, 2, s0[2], dqc, jx, jy, T, u2, dlt, out + 8);
    equilibrium_group(B, 3, s0[3], qd, jx, jy, T, u2, dlt, out + 12);
}

template <typename TS>
constexpr bool kSingle = std::is_same<TS, float>::value;

__device__ __forceinline__ double fma_t(double x, double y, double z) { return fma(x, y, z); }

// Storage value to double and double to storage value; the single-precision
// conversions run on the integer pipes (cdbm_convert.h).
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return widen_f32(v); }
template <typename TS>
__device__ __forceinline__ TS narrow(double v)
{
    if constexpr (kSingle<TS>) return narrow_f64(v); else return v;
}
__device__ __forceinline__ float fma_t(float x, float y, float z) { return fmaf(x, y, z); }

// Per-cell macroscopic quantities of a stage: conserved moments (in double), then
// u, P = rho T and T through the refined reciprocal of rho.  With kShift, f holds
// g = f - F and the reference moments rhoF, EF are added.
struct Prim {
    Cons q;
    double r;                    // 1 / rho
    double ux, uy, jyuy, ru2, p, T;
};

template <bool kShift>
__device__ __forceinline__ Prim primitives(const double f[kNV], const ModelConsts &m, double rhoF,
                                           double EF, unsigned *flag)
{
    Prim s;
    s.q = conserved(f, m);
    if (kShift) {
        s.q.rho += rhoF;
        s.q.E += EF;
    }
    const double r = rcp64(s.q.rho);
    s.r = r;
    s.ux = s.q.jx * r;
    s.uy = s.q.jy * r;
    s.jyuy = s.q.jy * s.uy;
    s.ru2 = fma(s.q.jx, s.ux, s.jyuy);
    s.p = (s.q.E - s.ru2) * m.invK;
    s.T = s.p * r;
    if (!(positive_finite(s.q.rho) && positive_finite(s.p))) atomicOr(flag, kFlagNonPhys);
    return s;
}

// ---- y-symmetric states of 1-D grids ----
// On a 1-D grid (ny = 1) a state that is mirror-symmetric in y -- f_S = f_N in the
// axis groups, f_SE = f_NE and f_SW = f_NW in the diagonal ones, in every cell --
// stays so under the step: the mirror images have equal x components, so their
// transport is the same, and with j_y = 0 the equilibrium gives them equal values.
// Every initial state with u_y = 0 is such a state (f_eq of u_y = 0 is symmetric).
// There j_y = u_y = 0 exactly, and the *_sym forms below drop every term that then
// vanishes: they return, value for value, what the general forms return on the
// same state (up to the sign of an exact zero).  Only 10 of the 16 velocities are
// distinct.
constexpr int kNSym = 10;
__host__ __device__ constexpr int sym_vel(int k)      // k-th distinct velocity: E N W | NE NW per group pair
{
    return k < 3 ? k : (k < 5 ? k + 1 : (k < 8 ? k + 3 : k + 4));
}
__host__ __device__ constexpr int mirror_y(int i)     // the velocity whose value i holds on a symmetric state
{
    return (i & 3) == 3 && ((i >> 2) & 1) == 0 ? i - 2              // S -> N
           : ((i >> 2) & 1) == 1 && (i & 3) == 2 ? i - 1           // SW -> NW
           : ((i >> 2) & 1) == 1 && (i & 3) == 3 ? i - 3           // SE -> NE
           : i;
}

__host__ __device__ constexpr int sym_partner(int i)  // the mirror image a distinct velocity stands for, or -1
{
    return ((i >> 2) & 1) == 0 ? ((i & 3) == 1 ? i + 2 : -1)  // N -> S
                               : ((i & 3) == 0 ? i + 3 : ((i & 3) == 1 ? i + 1 : -1));   // NE -> SE, NW -> SW
}

// conserved() on a symmetric state (j_y = 0).
__device__ __forceinline__ Cons conserved_sym(const double f[kNV], const ModelConsts &m)
{
    double s0[4], sx[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const double *q = f + 4 * g;
        if ((g & 1) == 0) {
            sx[g] = q[0] - q[2];
            s0[g] = (q[0] + q[2]) + (q[1] + q[3]);
        } else {
            const double e = q[0] + q[3], w = q[1] + q[2];
            sx[g] = e - w;
            s0[g] = e + w;
        }
    }
    Cons r;
    r.rho = (s0[0] + s0[1]) + (s0[2] + s0[3]);
    r.jx = fma(m.c[3], sx[3], fma(m.c[2], sx[2], fma(m.c[1], sx[1], m.c[0] * sx[0])));
    r.jy = 0.0;
    r.E = fma(m.w[3], s0[3], fma(m.w[2], s0[2], fma(m.w[1], s0[1], m.w[0] * s0[0])));
    return r;
}

// primitives<kShift>() on a symmetric state (u_y = 0, rho u^2 = j_x u_x).
template <bool kShift>
__device__ __forceinline__ Prim primitives_sym(const double f[kNV], const ModelConsts &m, double rhoF, double EF,
                                               unsigned *flag)
{
    Prim s;
    s.q = conserved_sym(f, m);
    if (kShift) {
        s.q.rho += rhoF;
        s.q.E += EF;
    }
    const double r = rcp64(s.q.rho);
    s.r = r;
    s.ux = s.q.jx * r;
    s.uy = 0.0;
    s.jyuy = 0.0;
    s.ru2 = __dmul_rn(s.q.jx, s.ux);     // the general fma(j_x, u_x, +0), never contracted
    s.p = (s.q.E - s.ru2) * m.invK;
    s.T = s.p * r;
    if (!(positive_finite(s.q.rho) && positive_finite(s.p))) atomicOr(flag, kFlagNonPhys);
    return s;
}

// equilibrium<kShift>() on a symmetric state: u_y = j_y = 0, so rho u^2 = m5 - m7 =
// j_x u_x, m6 = m15 = 0 (no diagonal quadrupole), u^2 = u_x^2 - u_y^2 = u_x^2, and
// the y-odd members equal their mirror images.  out receives all 16 values.
template <bool kShift = false>
__device__ __forceinline__ void equilibrium_sym(const EqBlocks &B, const ModelConsts &m, double rho, double E,
                                                double jx, double ux, double ru2, double P, double T,
                                                double out[kNV], const double *s0_shift = nullptr)
{
    const double u2 = ux * ux;
    const double m1416 = fma(T, fma(m.Kp6, ru2, m.twoKp2 * P), ru2 * u2);
    const double W4 = fma(m.Kp4, T, u2);
    const double d57 = ru2;
    double s0[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const double *S = B.S + 4 * g;
        if (kShift)
            s0[g] = fma(S[3], m1416, fma(S[2], ru2, fma(S[1], E, fma(S[0], rho, -s0_shift[g]))));
        else
            s0[g] = fma(S[3], m1416, fma(S[2], ru2, fma(S[1], E, S[0] * rho)));
    }
    const double dq[2] = {d57 * fma(B.B1[1], W4, B.B1[0]), d57 * fma(B.B1[3], W4, B.B1[2])};
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const double *W = B.Vc + 4 * g;
        const double px = fma(W[3], u2, fma(W[2], u2, fma(W[1], T, W[0])));
        double *o = out + 4 * g;
        if ((g & 1) == 0) {
            const double A = s0[g] + dq[g >> 1], Bv = s0[g] - dq[g >> 1];
            o[0] = fma(jx, px, A);
            o[2] = fma(-jx, px, A);
            o[1] = Bv;
            o[3] = Bv;
        } else {
            const double U = __dmul_rn(jx, px);   // the general fma(j_x, px, +-0)
            o[0] = s0[g] + U;
            o[3] = o[0];
            o[1] = s0[g] - U;
            o[2] = o[1];
        }
    }
}

// Neighbour index along an axis of n cells: periodic wrap or zero-gradient clamp.
__device__ __forceinline__ int neighbour(int j, int n, int bc)
{
    if (bc == 0) {
        j %= n;
        return j < 0 ? j + n : j;
    }
    return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

}  // namespace cdbm
