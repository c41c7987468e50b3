// Reverse-mode (adjoint) kernels of the double-precision time step on periodic
// grids: the vector-Jacobian product of one Runge-Kutta stage (BGK collision with
// the Jacobian of the factored equilibrium, NND transport with the limiter's
// subgradient), of the initial equilibrium f = f_eq(rho, u, T), and of the read-out
// (rho, u, T)(f).  The host driver (cdbm_api.cu) runs them backward over segments
// recomputed from checkpoints.
//
// Stage (forward):  out = a_base base + (beta - gamma h) g + heq(g) - sum_r l_r D_r(g),
//   heq = gamma h f_eq(m(g)), m = (rho, j_x, j_y, E) = C g (the conserved rows),
//   D_j = U_j + (N_j - N_{j-s}) / 2,  U_j = g_j - g_{j-s},  N_j = minmod(U_{j+s}, U_j)
//   along each axis with upwind sign s of the velocity.
// Its transpose applied to a cotangent o of out:
//   g_bar = (beta - gamma h) o + C^T (d heq / d m)^T o - sum_r l_r (dD_r / dg)^T o,
//   base_bar = a_base o,   tau_bar = sum o . d out / d tau = -sum o . (heq - gamma h g) / tau.
// minmod is piecewise linear; its derivative is that of the branch the forward pass
// took (1 for the chosen argument, 0 for the other, 0 when the result is 0; X on a tie).
// That is the exact derivative of the discrete step (CDBM_ADJ_LIMITER_EXACT).  Two
// approximate linearisations are available for long horizons on fine grids, where
// the exact one can grow without bound: where the limiter picks the downwind slope
// beside an upwind pick its linearisation is anti-diffusive (for the transport
// symbol, Re D(theta) = -cos(theta) (1 - cos(theta)) if that pattern were uniform),
// and over thousands of steps these picks amplify the adjoint while finite
// differences of the forward run stay finite.
//   CDBM_ADJ_LIMITER_FROZEN_RATIO: the limiter value phi = N_k / U_k in [0, 1] is held
//     fixed, dN_k = phi dU_k (the downwind dependence is dropped);
//   CDBM_ADJ_LIMITER_FROZEN: the limiter output is held fixed, dN_k = 0 (the
//     linearisation is first-order upwind transport).
#include "cdbm_device.cuh"

namespace cdbm {

namespace {

constexpr int kAdjThreads = 128;

// Branch of minmod(X, Y): 1 if X is returned, 2 if Y, 0 if zero (same tests as minmod()).
__device__ __forceinline__ int minmod_branch(double X, double Y)
{
    const int hx = __double2hiint(X), lx = __double2loint(X);
    const int hy = __double2hiint(Y), ly = __double2loint(Y);
    const unsigned ahx = (unsigned)hx & 0x7fffffffu, ahy = (unsigned)hy & 0x7fffffffu;
    const bool x_le_y = (ahx < ahy) | ((ahx == ahy) & ((unsigned)lx <= (unsigned)ly));
    const bool keep = ((hx ^ hy) >= 0) & ((ahx | (unsigned)lx) != 0u) & ((ahy | (unsigned)ly) != 0u);
    return keep ? (x_le_y ? 1 : 2) : 0;
}

// Weights (w_X, w_Y) of the linearised minmod(X, Y) = N for the limiter mode kMode.
template <int kMode>
__device__ __forceinline__ void minmod_weights(double X, double Y, double &wx, double &wy)
{
    const int b = minmod_branch(X, Y);
    if (kMode == CDBM_ADJ_LIMITER_EXACT) {
        wx = b == 1 ? 1.0 : 0.0;
        wy = b == 2 ? 1.0 : 0.0;
    } else if (kMode == CDBM_ADJ_LIMITER_FROZEN_RATIO) {
        wx = 0.0;
        wy = b == 1 ? X * rcp64(fabs(Y)) * (Y < 0.0 ? -1.0 : 1.0) : (b == 2 ? 1.0 : 0.0);
    } else {
        wx = 0.0;
        wy = 0.0;
    }
}

struct MomBar {
    double rho, jx, jy, E;
};

// (d out / d m)^T ob for out = equilibrium(B, m, ...) (scaled as B is), m = (rho, jx,
// jy, E): reverse of the forward sequence in equilibrium() and primitives(), step by
// step.  With r = 1/rho, u = j r, ru2 = j.u, P = (E - ru2)/K, T = P r.
// The forward values r = 1/rho, u, j_y u_y, rho u^2, P and T come from the caller
// (primitives() of the forward stage, the same refined reciprocal).
// With oheq != nullptr it also returns *oheq = sum_i ob_i out_i, the cotangent
// applied to the equilibrium itself: the rebuild is a linear butterfly, so that sum
// is the dot product of the transposed group components (s0b, sxb, syb, qb) with
// the forward components (s0, sx, sy, q), and the 16 outputs are never formed.
__device__ __forceinline__ MomBar equilibrium_vjp(const EqBlocks &B, const ModelConsts &m, double rho, double E,
                                                  double jx, double jy, double r, double ux, double uy, double jyuy,
                                                  double ru2, double P, double T, const double ob[kNV],
                                                  double *oheq = nullptr)
{
    // forward values
    const double ux2 = ux * ux, uy2 = uy * uy, u2 = ux2 + uy2, dlt = ux2 - uy2;
    const double Y = fma(m.Kp6, ru2, m.twoKp2 * P);
    const double W4 = fma(m.Kp4, T, u2);
    const double d57 = fma(jx, ux, -jyuy);
    const double m6 = jx * uy;

    // rebuild (butterflies) transposed: group component cotangents
    double s0b[4], sxb[4], syb[4], qb[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const double *o = ob + 4 * g;
        if ((g & 1) == 0) {             // axis: o0 = A + sx, o2 = A - sx, o1 = B + sy, o3 = B - sy
            const double Ab = o[0] + o[2], Bb = o[1] + o[3];
            sxb[g] = o[0] - o[2];
            syb[g] = o[1] - o[3];
            s0b[g] = Ab + Bb;           // A = s0 + dq, B = s0 - dq
            qb[g] = Ab - Bb;
        } else {                        // diag: o0 = P + U, o2 = P - U, o1 = Q - V, o3 = Q + V
            const double Pb = o[0] + o[2], Ub = o[0] - o[2];
            const double Qb = o[1] + o[3], Vb = o[3] - o[1];
            s0b[g] = Pb + Qb;           // P = s0 + q, Q = s0 - q
            qb[g] = Pb - Qb;
            sxb[g] = Ub + Vb;           // U = sx + sy, V = sx - sy
            syb[g] = Ub - Vb;
        }
    }

    double rhob = 0.0, jxb = 0.0, jyb = 0.0, Eb = 0.0;
    double ru2b = 0.0, m1416b = 0.0, Tb = 0.0, u2vb = 0.0, dltb = 0.0, W4b = 0.0;
    const double m1416 = oheq ? fma(T, Y, ru2 * u2) : 0.0;
    double dot = 0.0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const double *S = B.S + 4 * g;
        const double *W = B.Vc + 4 * g;
        // s0 = S0 rho + S1 E + S2 ru2 + S3 m1416
        rhob = fma(S[0], s0b[g], rhob);
        Eb = fma(S[1], s0b[g], Eb);
        ru2b = fma(S[2], s0b[g], ru2b);
        m1416b = fma(S[3], s0b[g], m1416b);
        // sx = jx px, sy = jy py with px, py = cm +/- W3 dlt and cm = W0 + W1 T + W2 u2
        const double cm = fma(W[2], u2, fma(W[1], T, W[0]));
        const double px = fma(W[3], dlt, cm), py = fma(-W[3], dlt, cm);
        const double pxb = jx * sxb[g], pyb = jy * syb[g];
        if (oheq) {
            const double s0 = fma(S[3], m1416, fma(S[2], ru2, fma(S[1], E, S[0] * rho)));
            dot = fma(s0b[g], s0, dot);
            dot = fma(pxb, px, dot);    // sxb sx = (jx sxb) px
            dot = fma(pyb, py, dot);
        }
        jxb = fma(px, sxb[g], jxb);
        jyb = fma(py, syb[g], jyb);
        const double cb = pxb + pyb;
        dltb = fma(W[3], pxb - pyb, dltb);
        u2vb = fma(W[2], cb, u2vb);
        Tb = fma(W[1], cb, Tb);
    }
    // dq_a = d57 (B1_0 + B1_1 W4), dq_c = d57 (B1_2 + B1_3 W4); q_b, q_d likewise with m6
    const double bA = fma(B.B1[1], W4, B.B1[0]), bC = fma(B.B1[3], W4, B.B1[2]);
    const double bB = fma(B.B2[1], W4, B.B2[0]), bD = fma(B.B2[3], W4, B.B2[2]);
    const double d57b = fma(bA, qb[0], bC * qb[2]);
    const double m6b = fma(bB, qb[1], bD * qb[3]);
    if (oheq) *oheq = fma(d57, d57b, fma(m6, m6b, dot));   // + sum of qb_g q_g
    W4b = d57 * fma(B.B1[1], qb[0], B.B1[3] * qb[2]) + m6 * fma(B.B2[1], qb[1], B.B2[3] * qb[3]);
    // m6 = jx uy;  d57 = jx ux - jyuy
    double uxb = 0.0, uyb = 0.0, jyuyb = 0.0;
    jxb = fma(uy, m6b, jxb);
    uyb = fma(jx, m6b, uyb);
    jxb = fma(ux, d57b, jxb);
    uxb = fma(jx, d57b, uxb);
    jyuyb -= d57b;
    // W4 = Kp4 T + u2
    Tb = fma(m.Kp4, W4b, Tb);
    double u2b = W4b;
    // m1416 = T Y + ru2 u2,  Y = Kp6 ru2 + 2 (K+2) P
    Tb = fma(Y, m1416b, Tb);
    const double Yb = T * m1416b;
    ru2b = fma(u2, m1416b, ru2b);
    ru2b = fma(m.Kp6, Yb, ru2b);
    u2b = fma(ru2, m1416b, u2b);
    double Pb = m.twoKp2 * Yb;
    // u2 = ux2 + uy2, dlt = ux2 - uy2; ux2 = ux^2; uy2 = uy^2
    u2b += u2vb;
    const double ux2b = u2b + dltb, uy2b = u2b - dltb;
    uxb = fma(2.0 * ux, ux2b, uxb);
    uyb = fma(2.0 * uy, uy2b, uyb);
    // T = P r
    Pb = fma(r, Tb, Pb);
    double rb = P * Tb;
    // P = (E - ru2) / K
    Eb = fma(m.invK, Pb, Eb);
    ru2b = fma(-m.invK, Pb, ru2b);
    // ru2 = jx ux + jyuy;  jyuy = jy uy
    jxb = fma(ux, ru2b, jxb);
    uxb = fma(jx, ru2b, uxb);
    jyuyb += ru2b;
    jyb = fma(uy, jyuyb, jyb);
    uyb = fma(jy, jyuyb, uyb);
    // ux = jx r, uy = jy r
    jxb = fma(r, uxb, jxb);
    jyb = fma(r, uyb, jyb);
    rb = fma(jx, uxb, fma(jy, uyb, rb));
    // r = 1 / rho
    rhob = fma(-r * r, rb, rhob);
    return {rhob, jxb, jyb, Eb};
}

// Flux transpose along one axis for one velocity: the contribution to g_bar at
// cell m from the terms -l D_j of the cells j whose stencil contains m, given g at
// m-2s .. m+2s (gm2 .. gp2 in upwind order: gm2 = g_{m-2s}, ..., gp2 = g_{m+2s}) and
// the cotangent o at m-s .. m+2s.
//
// With U_k = g_k - g_{k-s}, N_k = minmod(U_{k+s}, U_k) linearised as
// dN_k = w_X(k) dU_{k+s} + w_Y(k) dU_k, and d_k = o_{k+s} - o_k, the transpose of
// -l D_j = -l (U_j + (N_j - N_{j-s}) / 2) collected at g_m is
//   g_bar_m = (l / 2) [ (2 + w_Y(m) - w_X(m)) d_m + w_X(m-s) d_{m-s} - w_Y(m+s) d_{m+s} ],
// written with the halved coefficients so that one product by l remains.  In the
// frozen mode all weights vanish and it is l d_m.
template <int kMode>
__device__ __forceinline__ double flux_vjp(double l, double gm2, double gm1, double g0, double gp1, double gp2,
                                           double om1, double o0, double op1, double op2)
{
    const double d0 = op1 - o0;
    if (kMode == CDBM_ADJ_LIMITER_FROZEN) return l * d0;
    const double dm1 = o0 - om1, dp1 = op2 - op1;
    // U_k at k = m-s, m, m+s, m+2s
    const double Um1 = gm1 - gm2, U0 = g0 - gm1, Up1 = gp1 - g0, Up2 = gp2 - gp1;
    double acc;
    if (kMode == CDBM_ADJ_LIMITER_EXACT) {
        // branch of N_{m-s}, N_m, N_{m+s}: 1 picks X = U_{k+s}, 2 picks Y = U_k, 0 is zero
        const int bm1 = minmod_branch(U0, Um1), b0 = minmod_branch(Up1, U0), bp1 = minmod_branch(Up2, Up1);
        acc = (b0 == 1 ? 0.5 : (b0 == 2 ? 1.5 : 1.0)) * d0;
        acc = fma(bm1 == 1 ? 0.5 : 0.0, dm1, acc);
        acc = fma(bp1 == 2 ? -0.5 : 0.0, dp1, acc);
    } else {
        double xm1, ym1, x0, y0, xp1, yp1;
        minmod_weights<kMode>(U0, Um1, xm1, ym1);
        minmod_weights<kMode>(Up1, U0, x0, y0);
        minmod_weights<kMode>(Up2, Up1, xp1, yp1);
        acc = fma(0.5, y0 - x0, 1.0) * d0;
        acc = fma(0.5 * xm1, dm1, acc);
        acc = fma(-0.5 * yp1, dp1, acc);
    }
    return l * acc;
}

// out_bar = c_prev * prev + VJP of one stage (see header) at stage input g for
// cotangent ob; tau_acc[block] += sum over the block's cells of the tau term.
template <int kMode>
__global__ void __launch_bounds__(kAdjThreads) adjoint_stage_kernel(const double *__restrict__ g,
                                                                    const double *__restrict__ ob,
                                                                    const double *prev, double c_prev,
                                                                    double *out_bar, const StageArgs a,
                                                                    double gamma_h, double inv_tau,
                                                                    double *tau_acc)
{
    __shared__ double red[kAdjThreads];
    const int nx = a.nx, ny = a.ny;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    double tau_part = 0.0;
    if (x < nx) {
        const size_t P = (size_t)nx * ny;
        const size_t row = (size_t)y * nx;
        const size_t c = row + x;
        double f[kNV], o[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            f[i] = g[i * P + c];
            o[i] = ob[i * P + c];
        }
        unsigned nonphys = 0;                              // the forward stage already reported it
        const Prim pr = primitives<false>(f, a.m, 0.0, 0.0, &nonphys);
        const Cons &q = pr.q;
        // tau term: sum_i o_i (gamma h g_i - heq_i) / tau, with sum_i o_i heq_i from the VJP
        double og = 0.0, oheq = 0.0;
#pragma unroll
        for (int i = 0; i < kNV; ++i) og = fma(o[i], f[i], og);
        const MomBar w = equilibrium_vjp(a.eq, a.m, q.rho, q.E, q.jx, q.jy, pr.r, pr.ux, pr.uy, pr.jyuy, pr.ru2,
                                         pr.p, pr.T, o, &oheq);
        tau_part = fma(gamma_h, og, -oheq) * inv_tau;

        int xs[5];
#pragma unroll
        for (int k = -2; k <= 2; ++k) xs[k + 2] = neighbour(x + k, nx, 0);
        int ys[5];
#pragma unroll
        for (int k = -2; k <= 2; ++k) ys[k + 2] = neighbour(y + k, ny, 0);

        // moment part of the VJP per velocity: rho_bar + v . j_bar + (|v|^2 + eta^2) E_bar,
        // formed per group as t +- c jx_bar +- c jy_bar with t = rho_bar + w_g E_bar
        double mb[kNV];
#pragma unroll
        for (int grp = 0; grp < 4; ++grp) {
            const double t = fma(w.E, a.m.w[grp], w.rho);
            const double ax = w.jx * a.m.c[grp], ay = w.jy * a.m.c[grp];
            double *q = mb + 4 * grp;
            if ((grp & 1) == 0) {                    // (1,0), (0,1), (-1,0), (0,-1)
                q[0] = t + ax;
                q[1] = t + ay;
                q[2] = t - ax;
                q[3] = t - ay;
            } else {                                 // (1,1), (-1,1), (-1,-1), (1,-1)
                const double pp = ax + ay, pm = ax - ay;
                q[0] = t + pp;
                q[1] = t - pm;
                q[2] = t - pp;
                q[3] = t + pm;
            }
        }
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            const int grp = i >> 2;
            const double *gp = g + i * P, *op = ob + i * P;
            if constexpr (kMode == CDBM_ADJ_LIMITER_FROZEN) {
                // l (o_{m+s} - o_m) per direction, with the -l o_m terms in the self factor
                const double self = dirx(i) == 0 ? a.a_self_y[grp] : (diry(i) == 0 ? a.a_self_x[grp]
                                                                                    : a.a_self_xy[grp]);
                double gb = fma(self, o[i], mb[i]);
                if (dirx(i) != 0) gb = fma(a.lx[grp], op[row + xs[2 + dirx(i)]], gb);
                if (diry(i) != 0 && ny > 1) gb = fma(a.ly[grp], op[(size_t)ys[2 + diry(i)] * nx + x], gb);
                if (prev) gb = fma(c_prev, prev[i * P + c], gb);
                out_bar[i * P + c] = gb;
                continue;
            }
            double gb = fma(a.a_self, o[i], mb[i]);
            if (dirx(i) != 0) {
                const int s = dirx(i);
                // upwind order: index of m + k s
                const double gm2 = gp[row + xs[2 - 2 * s]], gm1 = gp[row + xs[2 - s]];
                const double gp1 = gp[row + xs[2 + s]], gp2 = gp[row + xs[2 + 2 * s]];
                const double om1 = op[row + xs[2 - s]], op1 = op[row + xs[2 + s]], op2 = op[row + xs[2 + 2 * s]];
                gb += flux_vjp<kMode>(a.lx[grp], gm2, gm1, f[i], gp1, gp2, om1, o[i], op1, op2);
            }
            if (diry(i) != 0 && ny > 1) {
                const int s = diry(i);
                const double gm2 = gp[(size_t)ys[2 - 2 * s] * nx + x], gm1 = gp[(size_t)ys[2 - s] * nx + x];
                const double gp1 = gp[(size_t)ys[2 + s] * nx + x], gp2 = gp[(size_t)ys[2 + 2 * s] * nx + x];
                const double om1 = op[(size_t)ys[2 - s] * nx + x], op1 = op[(size_t)ys[2 + s] * nx + x];
                const double op2 = op[(size_t)ys[2 + 2 * s] * nx + x];
                gb += flux_vjp<kMode>(a.ly[grp], gm2, gm1, f[i], gp1, gp2, om1, o[i], op1, op2);
            }
            if (prev) gb = fma(c_prev, prev[i * P + c], gb);
            out_bar[i * P + c] = gb;
        }
    }
    // deterministic per-block accumulation of the tau term
    red[threadIdx.x] = tau_part;
    __syncthreads();
    for (int w2 = kAdjThreads / 2; w2 > 0; w2 >>= 1) {
        if (threadIdx.x < w2) red[threadIdx.x] += red[threadIdx.x + w2];
        __syncthreads();
    }
    if (threadIdx.x == 0) tau_acc[blockIdx.y * gridDim.x + blockIdx.x] += red[0];
}

// VJP of f = f_eq(rho, u, T) per cell, evaluated at the initial state f0 (whose
// conserved moments are those of the initial fields).
__global__ void __launch_bounds__(128) init_vjp_kernel(const FieldArgs a, const double *__restrict__ f0,
                                                       const double *__restrict__ fbar, double *rho_bar,
                                                       double *ux_bar, double *uy_bar, double *T_bar)
{
    const size_t P = (size_t)a.nx * a.ny;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < P; c += (size_t)gridDim.x * blockDim.x) {
        double f[kNV], o[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            f[i] = f0[i * P + c];
            o[i] = fbar[i * P + c];
        }
        unsigned nonphys = 0;
        const Prim pr = primitives<false>(f, a.m, 0.0, 0.0, &nonphys);
        const Cons &q = pr.q;
        const MomBar w = equilibrium_vjp(a.eq, a.m, q.rho, q.E, q.jx, q.jy, pr.r, pr.ux, pr.uy, pr.jyuy, pr.ru2,
                                         pr.p, pr.T, o);
        // m = (rho, rho u_x, rho u_y, rho (u^2 + K T)) of the fields
        const double u = q.jx / q.rho, v = q.jy / q.rho;
        const double T = (q.E - fma(q.jx, u, q.jy * v)) / (a.m.K * q.rho);
        if (rho_bar) rho_bar[c] = w.rho + w.jx * u + w.jy * v + w.E * (u * u + v * v + a.m.K * T);
        if (ux_bar) ux_bar[c] = q.rho * (w.jx + 2.0 * u * w.E);
        if (uy_bar) uy_bar[c] = q.rho * (w.jy + 2.0 * v * w.E);
        if (T_bar) T_bar[c] = q.rho * a.m.K * w.E;
    }
}

// f_bar_i = rho_bar + ux_bar (v_ix - u_x)/rho + uy_bar (v_iy - u_y)/rho
//           + T_bar (|v_i|^2 + eta_i^2 - 2 u.v_i + u^2 - K T) / (K rho)
// (the transpose of the Jacobian of the read-out rho, u, T of f).
__global__ void __launch_bounds__(128) macros_vjp_kernel(const FieldArgs a, const double *__restrict__ f,
                                                         const double *rho_bar, const double *ux_bar,
                                                         const double *uy_bar, const double *T_bar,
                                                         double *__restrict__ fbar)
{
    const size_t P = (size_t)a.nx * a.ny;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < P; c += (size_t)gridDim.x * blockDim.x) {
        double fc[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) fc[i] = f[i * P + c];
        const Cons q = conserved(fc, a.m);
        const double r = 1.0 / q.rho;
        const double u = q.jx * r, v = q.jy * r;
        const double u2 = u * u + v * v;
        const double T = (q.E - q.rho * u2) / (a.m.K * q.rho);
        const double rb = rho_bar ? rho_bar[c] : 0.0;
        const double ub = ux_bar ? ux_bar[c] * r : 0.0;
        const double vb = uy_bar ? uy_bar[c] * r : 0.0;
        const double Tb = T_bar ? T_bar[c] * r * a.m.invK : 0.0;
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            const double w = a.vx[i] * a.vx[i] + a.vy[i] * a.vy[i] + a.eta[i] * a.eta[i];
            const double uv = u * a.vx[i] + v * a.vy[i];
            fbar[i * P + c] = rb + ub * (a.vx[i] - u) + vb * (a.vy[i] - v) + Tb * (w - 2.0 * uv + u2 - a.m.K * T);
        }
    }
}

__global__ void sum_kernel(const double *__restrict__ v, int n, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += v[k];
        *out = s;
    }
}

unsigned grid1(size_t n)
{
    size_t b = (n + 127) / 128;
    return (unsigned)(b < 1 ? 1 : (b > 1048576 ? 1048576 : b));
}

}  // namespace

dim3 adjoint_grid(int nx, int ny) { return dim3((nx + kAdjThreads - 1) / kAdjThreads, ny, 1); }

cudaError_t launch_adjoint_stage(const double *g, const double *ob, const double *prev, double c_prev,
                                 double *out_bar, const StageArgs &a, double gamma_h, double inv_tau,
                                 int limiter, double *tau_acc, cudaStream_t s)
{
    const dim3 grid = adjoint_grid(a.nx, a.ny);
    if (limiter == CDBM_ADJ_LIMITER_FROZEN_RATIO)
        adjoint_stage_kernel<CDBM_ADJ_LIMITER_FROZEN_RATIO><<<grid, kAdjThreads, 0, s>>>(
            g, ob, prev, c_prev, out_bar, a, gamma_h, inv_tau, tau_acc);
    else if (limiter == CDBM_ADJ_LIMITER_FROZEN)
        adjoint_stage_kernel<CDBM_ADJ_LIMITER_FROZEN><<<grid, kAdjThreads, 0, s>>>(
            g, ob, prev, c_prev, out_bar, a, gamma_h, inv_tau, tau_acc);
    else
        adjoint_stage_kernel<CDBM_ADJ_LIMITER_EXACT><<<grid, kAdjThreads, 0, s>>>(
            g, ob, prev, c_prev, out_bar, a, gamma_h, inv_tau, tau_acc);
    return cudaGetLastError();
}

cudaError_t launch_init_vjp(const FieldArgs &a, const double *f0, const double *fbar, double *rho_bar,
                            double *ux_bar, double *uy_bar, double *T_bar, cudaStream_t s)
{
    init_vjp_kernel<<<grid1((size_t)a.nx * a.ny), 128, 0, s>>>(a, f0, fbar, rho_bar, ux_bar, uy_bar, T_bar);
    return cudaGetLastError();
}

cudaError_t launch_macros_vjp(const FieldArgs &a, const double *f, const double *rho_bar, const double *ux_bar,
                              const double *uy_bar, const double *T_bar, double *fbar, cudaStream_t s)
{
    macros_vjp_kernel<<<grid1((size_t)a.nx * a.ny), 128, 0, s>>>(a, f, rho_bar, ux_bar, uy_bar, T_bar, fbar);
    return cudaGetLastError();
}

cudaError_t launch_sum(const double *v, int n, double *out, cudaStream_t s)
{
    sum_kernel<<<1, 32, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

}  // namespace cdbm
