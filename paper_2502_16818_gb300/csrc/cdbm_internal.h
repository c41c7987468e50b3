// Internal declarations shared by the CDBM library's translation units (host API
// and kernels).  Not part of the public ABI (include/cdbm.h).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

#include "../../include/cdbm.h"

namespace cdbm {

constexpr int kNV = 16;     // discrete velocities, Eq. (2)

// Parity-blocked inverse of the moment matrix at u = 0, pre-multiplied by the
// factors that rebuild f_i from its group components and by a caller scale
// (gamma * dt / tau inside a Runge-Kutta stage, 1 for plain f_eq).
//
// Per group g the four members split into
//   s0 = sum,  sx (x-odd),  sy (y-odd),  dq (axis: (E+W)-(N+S)) or q (diag: (NE+SW)-(NW+SE)),
// and the 16 raw-moment rows of Eq. (6) at u = 0 decouple into blocks
//   scalar  (s0_a..s0_d) <- (m1, m4, m5+m7, m14+m16)          4x4
//   axis q. (dq_a, dq_c) <- (m5-m7, m14-m16)                    2x2
//   diag q. (q_b, q_d)   <- (m6, m15)                           2x2
//   x-odd   (sx_a..sx_d) <- (m2, m8, m10, m12)                  4x4
//   y-odd   (sy_a..sy_d) <- (m3, m9, m13, m11)  (same matrix)   4x4
// The raw Maxwellian moments are folded into the stored coefficients (host side):
//   s0_g = S[g] . (rho, E, rho u^2, m14+m16)            (m5+m7 = (2E + (K-2) rho u^2) / K)
//   dq   = (m5-m7) (B1[r][0] + B1[r][1] W4),  q = m6 (B2[r][0] + B2[r][1] W4),
//          W4 = u^2 + (K+4) T                       (m14-m16 = (m5-m7) W4, m15 = m6 W4)
//   sx_g = j_x (V[g][0] + V[g][1] u_x^2 + V[g][2] u_y^2 + V[g][3] T)
//   sy_g = j_y (V[g][0] + V[g][2] u_x^2 + V[g][1] u_y^2 + V[g][3] T)
//          (m8 = j_x (u^2 + (K+2)T), m10 = j_x (u_x^2 + 3T), m12 = j_x (u_y^2 + T), and
//           the mirror images for y)
// The kernels evaluate the two odd polynomials from their common part and half
// difference, Vc[g] = (V[g][0], V[g][3], (V[g][1] + V[g][2]) / 2, (V[g][1] - V[g][2]) / 2):
//   V[g][0] + V[g][3] T + Vc[g][2] u^2 +/- Vc[g][3] (u_x^2 - u_y^2),
// and fuse the products with j_x, j_y into the rebuild of the four members.
struct EqBlocks {
    double S[16];   // row-major 4x4
    double B1[4];   // row-major 2x2
    double B2[4];   // row-major 2x2
    double V[16];   // row-major 4x4
    double Vc[16];  // per group: V0, V3, (V1 + V2) / 2, (V1 - V2) / 2
};

struct ModelConsts {
    double c[4];      // group speeds v_a..v_d
    double w[4];      // |v_g|^2 + eta_g^2 (|v|^2 = c^2 on axes, 2c^2 on diagonals)
    double invK;      // 1 / (D + I)
    double K;         // D + I
    double Kp2, Kp4, Kp6, twoKp2;   // K + 2, K + 4, K + 6, 2 (K + 2)
};

// Double-float copies of the stage constants for CDBM_FP32_DF64 (each value as the
// unevaluated sum of two floats; see cdbm_df64.cuh).  L is the lane type of the
// arithmetic: float for one cell, float2 for two cells computed together with the
// packed FP32x2 instructions (the constants then hold each value twice).
template <typename L>
struct DFv {
    L hi, lo;
};
using DFPair = DFv<float>;
template <typename L>
struct DFBlocksT {                // EqBlocks (scaled per stage); the x-odd rows of V as
    DFv<L> S[16], B1[4], B2[4];   // V0, V3, (V1 + V2)/2 and (V1 - V2)/2 per group
    DFv<L> V0[4], V3[4], Vs[4], Vd[4];
};
template <typename L>
struct DFModelT {                 // the ModelConsts the equilibrium uses
    DFv<L> c[4], w[4];
    DFv<L> invK, Kp4, Kp6, twoKp2;
};
template <typename L>
struct DFShiftT {                 // reference state of the deviation storage
    DFv<L> sF[4];                 // gamma h F_g
    DFv<L> rhoF, EF;
};
template <typename L>
struct DFConstsT {
    DFBlocksT<L> b;
    DFModelT<L> m;
    DFShiftT<L> r;
};
using DFBlocks = DFBlocksT<float>;
using DFModel = DFModelT<float>;
using DFShift = DFShiftT<float>;
using DFConsts = DFConstsT<float>;

// Conservation projection of the single-precision deviation equilibrium
// (CDBM_FP32_DEV): the group rest values s_g and odd components (cx, cy)_g are
// corrected by alpha + beta w_g and c_g (gamma_x, gamma_y) so that the equilibrium's
// mass, momentum and energy equal gamma h times the cell's; the corrections solve
// [16, 4 sum w; 4 sum w, 4 sum w^2] (alpha, beta) = residuals and gamma = residual /
// sum_i c_ix^2.
struct DevProj {
    float gh;             // gamma h of the stage
    float a00, a01, a11;  // inverse of the 2 x 2 matrix above
    float rkc;            // 1 / sum_i c_ix^2
};

// One Runge-Kutta stage: out = a_base * base + a_self * g + eq(g) - sum_r l_r D_r(g),
// i.e. alpha f^n + beta g + gamma dt L(g) with a_self = beta - gamma h, the
// equilibrium blocks scaled by gamma h and l = gamma dt c_g / dr.
struct StageArgs {
    EqBlocks eq;
    ModelConsts m;
    double a_base;
    double a_self;
    double lx[4];
    double ly[4];
    float a_base_f, a_self_f;     // the same coefficients rounded for the FP32-bulk state
    float lx_f[4], ly_f[4];
    // FP32-bulk state stores g = f - F, F the equilibrium of a constant reference
    // state (rho0, u = 0, T0): F_i = Fg[group of i].  The stage adds F's conserved
    // moments (rhoF, EF; F carries no momentum) to those of g and subtracts
    // gamma h F from the equilibrium (sF = gamma h Fg); the F terms of the update
    // cancel because alpha + beta = 1 in every stage.
    double sF[4];
    double rhoF, EF;
    // a_self minus the transport coefficients of a velocity's directions, per group:
    // x only (E, W), y only (N, S; a_self when ny = 1), both (diagonals; x only when
    // ny = 1).  The frozen-limiter adjoint stage uses them to fold -l o_m into the
    // self term.
    double a_self_x[4], a_self_y[4], a_self_xy[4];
    DFConsts d;                   // df64 copies (CDBM_FP32_DF64; their high parts for CDBM_FP32_DEV)
    DFConstsT<float2> d2;         // the same, each value twice (two-column kernel)
    DevProj dp;                   // conservation projection (CDBM_FP32_DEV)
    float2 a_base_f2, a_self_f2;  // a_base_f, a_self_f, lx_f, ly_f twice
    float2 lx_f2[4], ly_f2[4];
    int nx, ny;
    int bc_x, bc_y;
};

struct FieldArgs {
    EqBlocks eq;     // unscaled
    ModelConsts m;
    double vx[kNV], vy[kNV], eta[kNV];
    double Fg[4];    // reference equilibrium per group (FP32-bulk state only)
    int nx, ny;
};

// Error bits of the device flag word.
constexpr unsigned kFlagNonPhys = 1u;

// ---- host-side constants (cdbm_api.cu) ----
// Model constants and the parity-blocked inverse of M(0) for a velocity set and I;
// CDBM_ESINGULAR with *which naming the block when a block is singular or its
// condition number exceeds 1e12.
cdbm_status build_blocks(const cdbm_vset &vs, double I, ModelConsts &m, EqBlocks &eq,
                         double *cond_out, const char **which);
EqBlocks scaled(const EqBlocks &e, double s);

// Per-thread message buffer that cdbm_last_error(NULL) returns.
constexpr size_t kThreadErrorBytes = 256;
char *thread_error_buffer();

// ---- launchers (cdbm_kernels.cu); each returns the launch error ----
// `prec` is the precision mode (CDBM_FP64, CDBM_FP32_BULK, CDBM_FP32_DF64 or CDBM_FP32_DEV), which
// sets the storage of the distribution buffers; fields, Delta* and sums are always
// double.
cudaError_t launch_init(const FieldArgs &a, const double *rho, const double *ux,
                        const double *uy, const double *T, void *f, int prec, unsigned *flag,
                        cudaStream_t s);
cudaError_t launch_macros(const FieldArgs &a, const void *f, int prec, double *rho, double *ux,
                          double *uy, double *T, cudaStream_t s);
cudaError_t launch_tne(const FieldArgs &a, const void *f, int prec, double *out, cudaStream_t s);
cudaError_t launch_sums(const FieldArgs &a, const void *f, int prec, double *partials, int nblocks,
                        double *out4, cudaStream_t s);
// Copies a whole distribution field [16][ny][nx] between storage precisions: for the
// FP32-bulk state the stored deviation g becomes f = F + g on the way to double and
// f - F on the way back (FieldArgs::Fg).
cudaError_t launch_convert(const FieldArgs &a, const void *src, int src_prec, void *dst, int dst_prec,
                           cudaStream_t s);
// Sums of rho and T over the grid into out2 (for the reference state), using partials.
cudaError_t launch_field_means(const double *rho, const double *T, size_t n, double *partials,
                               int nblocks, double *out2, cudaStream_t s);

// Stage kernel selection and launch geometry, shared with the graph builder.
struct StageLaunch {
    void *func;
    dim3 grid, block;
    size_t smem = 0;              // dynamic shared memory bytes
};
// allow_march = false keeps 2-D grids on the one-cell-per-thread stage kernel;
// allow_split = false keeps FP64 1-D grids on it too (no four-thread split).
StageLaunch stage_launch_config(const StageArgs &a, bool with_base, int sm_count, int prec,
                                bool allow_march = true, bool allow_split = true);

// FP64 stage kernel for 1-D grids with each cell split over four threads
// (cdbm_small1d.cu): kSplitFlatThreads threads per block, 4 nx threads in all.
constexpr int kSplitFlatThreads = 128;
constexpr int kSplitFlatMaxCells = 8192;    // measured per stage: 8.8 against 10.0 us at 8192 cells,
                                            // 16.3 against 10.7 us at 16384
void *split_flat_func(bool with_base);
cudaError_t launch_stage(const StageLaunch &L, const void *g, const void *base, void *out,
                         const StageArgs &a, unsigned *flag, cudaStream_t s);

// Persistent cluster kernel for small 1-D grids (cdbm_small1d.cu): the whole state in
// the shared memory of one thread-block cluster, nsteps steps in one launch.
struct Small1D {
    bool ok;                      // the grid qualifies and the cluster fits on the device
    void *func;
    int cluster, chunk, threads;  // CTAs, cells per CTA, threads per CTA
    size_t smem;                  // dynamic shared memory per CTA
};
Small1D small1d_config(const StageArgs &a, int prec);
cudaError_t launch_small1d(const Small1D &L, void *f, int nsteps, const StageArgs &a0, const StageArgs &a1,
                           unsigned *flag, cudaStream_t s);

// ---- adjoint kernels (cdbm_adjoint.cu), double precision, periodic axes ----
// out_bar = c_prev * prev + (stage VJP at g applied to ob); tau_acc[block] += tau term;
// limiter: a cdbm_adj_limiter linearisation of minmod.
cudaError_t launch_adjoint_stage(const double *g, const double *ob, const double *prev, double c_prev,
                                 double *out_bar, const StageArgs &a, double gamma_h, double inv_tau,
                                 int limiter, double *tau_acc, cudaStream_t s);
dim3 adjoint_grid(int nx, int ny);
cudaError_t launch_init_vjp(const FieldArgs &a, const double *f0, const double *fbar, double *rho_bar,
                            double *ux_bar, double *uy_bar, double *T_bar, cudaStream_t s);
cudaError_t launch_macros_vjp(const FieldArgs &a, const double *f, const double *rho_bar, const double *ux_bar,
                              const double *uy_bar, const double *T_bar, double *fbar, cudaStream_t s);
cudaError_t launch_sum(const double *v, int n, double *out, cudaStream_t s);

// Single-precision storage (FP32 bulk, with the equilibrium in double or in df64).
inline bool single_storage(int prec) { return prec == CDBM_FP32_BULK || prec == CDBM_FP32_DF64 || prec == CDBM_FP32_DEV; }
// Bytes of one distribution value in storage precision `prec`.
inline size_t storage_bytes(int prec) { return single_storage(prec) ? 4 : 8; }
// Double-float copies of double constants (host side, cdbm_kernels.cu).
DFBlocks df_blocks(const EqBlocks &e);
DFModel df_model(const ModelConsts &m);
DFShift df_shift(const double sF[4], double rhoF, double EF);
// Fills a.d from the double constants of a.
void fill_df_consts(StageArgs &a);
// The conservation projection of a stage whose blocks are scaled by gh = gamma h.
DevProj dev_proj(const ModelConsts &m, double gh);
void fill_dev_proj(StageArgs &a, double gh);
// The same constants with each value twice, for the two-column (packed FP32x2) kernels.
DFBlocksT<float2> df_blocks_twice(const DFBlocks &d);
DFModelT<float2> df_model_twice(const DFModel &d);
DFShiftT<float2> df_shift_twice(const DFShift &d);

}  // namespace cdbm
