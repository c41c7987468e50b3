// Batched ensemble of independent 1-D tubes (Ny = 1, zero-gradient ends), each with
// its own length, cell size, I and initial state, advanced together by one
// persistent kernel.
//
// Layout: the tubes are concatenated along x into one [16][P] field (P = total
// cells); tube t owns cells [offset_t, offset_t + nx_t).  A block owns a fixed list
// of whole tubes (a longest-first partition of their cost) and advances each of
// them through all requested steps before moving on, so a tube's two buffers stay
// in L2 for the whole run and the only synchronisation is the block barrier
// between Runge-Kutta stages: tubes never exchange data, so blocks never wait on
// one another.  The tile shape -- threads per block and blocks per SM, which set
// how the tubes are partitioned -- is picked by cdbm_batch_autotune by timing the
// candidates on the batch itself.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "cdbm_stage.cuh"
#include "cdbm_internal.h"

using namespace cdbm;

namespace {

constexpr int kMaxClasses = 4;        // distinct values of I in one batch

struct TubeInfo {
    long long offset;                 // first cell of the tube in the [16][P] planes
    int nx;
    int cls;                          // index of the tube's I in BatchArgs::cls
    double lx[2][4];                  // per stage: gamma dt c_g / dx_t
    float lx_f[2][4];
    float2 lx_f2[2][4];               // lx_f twice (two-column df64 stage)
    double sF[2][4];                  // per stage: gamma h F_g (FP32-bulk reference)
    double Fg[4];                     // reference equilibrium per group
    double rhoF, EF;                  // its conserved moments
    DFShift dfs[2];                   // per stage: the same in df64 (CDBM_FP32_DF64, CDBM_FP32_DEV)
    DFShiftT<float2> dfs2[2];         // dfs with each value twice
};

struct ClassConsts {
    EqBlocks eq[2];                   // per stage, scaled by gamma h
    EqBlocks unit;                    // unscaled (initialisation, macros)
    ModelConsts m;
    DFBlocks dfeq[2];                 // eq[] and m in df64 (CDBM_FP32_DF64; their high parts for CDBM_FP32_DEV)
    DFModel dfm;
    DFBlocksT<float2> dfeq2[2];       // the same with each value twice
    DFModelT<float2> dfm2;
    DevProj dp[2];                    // per stage: conservation projection (CDBM_FP32_DEV)
};

struct BatchArgs {
    ClassConsts cls[kMaxClasses];
    double a_self[2], a_base[2];
    float a_self_f[2], a_base_f[2];
    float2 a_self_f2[2], a_base_f2[2];
    long long P;                      // total cells: stride between velocity planes
};

template <typename TS>
__device__ __forceinline__ TS pick(double d, float f)
{
    if constexpr (kSingle<TS>) return f; else return d;
}

// The 16 values of cell x of a tube; with kSym only the 10 distinct velocities of a
// y-symmetric state are loaded and the mirror images copied from them.
template <typename TS, bool kSym>
__device__ __forceinline__ void load_state(const TS *g, long long P, int x, TS fs[kNV])
{
#pragma unroll
    for (int i = 0; i < kNV; ++i)
        if (!kSym || mirror_y(i) == i) fs[i] = g[i * P + x];
    if constexpr (kSym) {
#pragma unroll
        for (int i = 0; i < kNV; ++i)
            if (mirror_y(i) != i) fs[i] = fs[mirror_y(i)];
    }
}

// One Runge-Kutta stage (kStage 0 or 1) over the nx cells of one tube by the calling
// block.  g, base and out point at the tube's first cell; planes are P apart.  The
// arithmetic per cell is the flat (Ny = 1) stage of the single-grid kernels, with the
// equilibrium in double, in df64 (kEq = kEqDF) or in single precision on the moment
// deviations (kEqF32).  Plain loads: the buffers are written
// inside this kernel, so the read-only path may not be used.
// With kSym the tube's state is y-symmetric (conserved_sym): only the 10 distinct
// velocities are loaded and computed, each result is stored to its plane and to the
// plane of its mirror image, and the equilibrium drops the terms of j_y = 0.  The
// values are those of the general form.
template <typename TS, int kStage, int kEq, bool kSym = false>
__device__ __forceinline__ void tube_stage(const TS *g, const TS *base, TS *out, long long P,
                                           const TubeInfo &t, const ClassConsts &C, TS a_self, TS a_base,
                                           unsigned *flag)
{
    constexpr bool kBase = kStage == 1;
    const int nx = t.nx;
    const double *lx = t.lx[kStage];
    const float *lx_f = t.lx_f[kStage];
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const int xm2 = x >= 2 ? x - 2 : 0, xm1 = x >= 1 ? x - 1 : 0;
        const int xp1 = x + 1 < nx ? x + 1 : nx - 1, xp2 = x + 2 < nx ? x + 2 : nx - 1;
        TS fs[kNV];
        load_state<TS, kSym>(g, P, x, fs);
        TS heq[kNV];
        if constexpr (kEq == kEqF32) {
            // all 16 values (a symmetric state holds its mirror images in fs)
            f32_equilibrium(C.dfeq[kStage], C.dfm, t.dfs[kStage], C.dp[kStage], fs, heq, flag);
        } else if constexpr (kEq == kEqDF) {
            static_assert(kSingle<TS>, "df64 equilibrium is for the single-precision state");
            if constexpr (kSym) df_equilibrium_sym(C.dfeq[kStage], C.dfm, t.dfs[kStage], fs, heq, flag);
            else df_equilibrium(C.dfeq[kStage], C.dfm, t.dfs[kStage], fs, heq, flag);
        } else {
            double f[kNV];
#pragma unroll
            for (int i = 0; i < kNV; ++i) f[i] = widen(fs[i]);
            double h[kNV];
            if constexpr (kSym) {
                const Prim s = primitives_sym<kSingle<TS>>(f, C.m, t.rhoF, t.EF, flag);
                equilibrium_sym<kSingle<TS>>(C.eq[kStage], C.m, s.q.rho, s.q.E, s.q.jx, s.ux, s.ru2, s.p, s.T, h,
                                             t.sF[kStage]);
            } else {
                const Prim s = primitives<kSingle<TS>>(f, C.m, t.rhoF, t.EF, flag);
                equilibrium<kSingle<TS>>(C.eq[kStage], C.m, s.q.rho, s.q.E, s.q.jx, s.q.jy, s.ux, s.uy, s.ru2,
                                         s.jyuy, s.p, s.T, h, t.sF[kStage]);
            }
#pragma unroll
            for (int i = 0; i < kNV; ++i) heq[i] = narrow<TS>(h[i]);
        }
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            if (kSym && mirror_y(i) != i) continue;
            TS o = fma_t(a_self, fs[i], heq[i]);
            if (kBase) o = fma_t(a_base, base[i * P + x], o);
            if (dirx(i) != 0) {
                const TS *gp = g + i * P;
                const TS u2 = gp[dirx(i) > 0 ? xm2 : xp2];
                const TS u1 = gp[dirx(i) > 0 ? xm1 : xp1];
                const TS d1 = gp[dirx(i) > 0 ? xp1 : xm1];
                o = fma_t(-pick<TS>(lx[i >> 2], lx_f[i >> 2]), nnd(u2, u1, fs[i], d1), o);
            }
            out[i * P + x] = o;
            if (kSym && sym_partner(i) >= 0) out[sym_partner(i) * P + x] = o;
        }
    }
}

// The FP64 stage of one tube with the x differences shared: the block covers a chunk
// of blockDim cells at a time; each thread computes U = f_x - f_{x-s} of its cell once
// per velocity into a row buffer in shared memory, the chunk's edge threads add the
// values beyond it (the tube's zero-gradient ends included, through the clamped
// indices), and each cell reads U of its neighbours there: 4 instead of 6 FP64
// instructions per x term, with the operands and operations of nnd(), so the result
// is the same bit for bit.  All threads run the same chunk loop and reach the block
// barriers.
template <int kStage, int kThreads, bool kSym = false>
__device__ __forceinline__ void tube_stage_shared_x(const double *g, const double *base, double *out, long long P,
                                                    const TubeInfo &t, const ClassConsts &C, double a_self,
                                                    double a_base, unsigned *flag, double (*row_u)[kThreads + 2])
{
    // with kSym the mirror images SW, SE (the x-moving ones) are skipped: 8 x terms
    auto xterm = [](int i) { return dirx(i) != 0 && (!kSym || mirror_y(i) == i); };
    constexpr bool kBase = kStage == 1;
    const int nx = t.nx;
    const double *lx = t.lx[kStage];
    const int tid = threadIdx.x;
    for (int xb = 0; xb < nx; xb += kThreads) {
        const int x = xb + tid;
        const bool active = x < nx;
        const int xc = active ? x : nx - 1;
        const int last = (nx - xb < kThreads ? nx - xb : kThreads) - 1;      // last active thread
        const int xm2 = xc >= 2 ? xc - 2 : 0, xm1 = xc >= 1 ? xc - 1 : 0;
        const int xp1 = xc + 1 < nx ? xc + 1 : nx - 1, xp2 = xc + 2 < nx ? xc + 2 : nx - 1;
        double fs[kNV], o[kNV];
        if (active) {
            load_state<double, kSym>(g, P, x, fs);
            double heq[kNV];
            if constexpr (kSym) {
                const Prim s = primitives_sym<false>(fs, C.m, 0.0, 0.0, flag);
                equilibrium_sym<false>(C.eq[kStage], C.m, s.q.rho, s.q.E, s.q.jx, s.ux, s.ru2, s.p, s.T, heq);
            } else {
                const Prim s = primitives<false>(fs, C.m, 0.0, 0.0, flag);
                equilibrium<false>(C.eq[kStage], C.m, s.q.rho, s.q.E, s.q.jx, s.q.jy, s.ux, s.uy, s.ru2, s.jyuy,
                                   s.p, s.T, heq);
            }
            int k = 0;
#pragma unroll
            for (int i = 0; i < kNV; ++i) {
                if (kSym && mirror_y(i) != i) continue;
                o[i] = fma(a_self, fs[i], heq[i]);
                if (kBase) o[i] = fma(a_base, base[i * P + x], o[i]);
                if (xterm(i)) {
                    row_u[k][tid + 1] = fs[i] - g[i * P + (dirx(i) > 0 ? xm1 : xp1)];   // a of nnd()
                    ++k;
                }
            }
            if (tid == 0) {                           // U left of the chunk
                int k2 = 0;
#pragma unroll
                for (int i = 0; i < kNV; ++i) {
                    if (!xterm(i)) continue;
                    const double *gp = g + i * P;
                    row_u[k2][0] = dirx(i) > 0 ? gp[xm1] - gp[xm2] : gp[xm1] - fs[i];
                    ++k2;
                }
            }
            if (tid == last) {                        // U right of the chunk
                int k2 = 0;
#pragma unroll
                for (int i = 0; i < kNV; ++i) {
                    if (!xterm(i)) continue;
                    const double *gp = g + i * P;
                    row_u[k2][last + 2] = dirx(i) > 0 ? gp[xp1] - fs[i] : gp[xp1] - gp[xp2];
                    ++k2;
                }
            }
        }
        __syncthreads();
        if (active) {
            int k = 0;
#pragma unroll
            for (int i = 0; i < kNV; ++i) {
                if (kSym && mirror_y(i) != i) continue;
                if (xterm(i)) {
                    const int s = dirx(i);
                    const double av = row_u[k][tid + 1];          // c - u1
                    const double bv = row_u[k][tid + 1 + s];      // d1 - c
                    const double ev = row_u[k][tid + 1 - s];      // u1 - u2
                    const double tt = minmod(bv, av) - minmod(av, ev);
                    o[i] = fma(-lx[i >> 2], fma(0.5, tt, av), o[i]);
                    ++k;
                }
                out[i * P + x] = o[i];
                if (kSym && sym_partner(i) >= 0) out[sym_partner(i) * P + x] = o[i];
            }
        }
        __syncthreads();                              // the next chunk rewrites the buffer
    }
}

// The df64 stage of one tube with two cells per thread: each thread takes the
// pairs (x, x + 1) of the tube (x even; x + 1 = x for an odd last cell, computed
// twice and stored once) and applies every operation of tube_stage<float, kStage,
// true> to both with the packed FP32x2 instructions, so each cell gets the bits of
// the one-cell form with about half the instruction issues.
template <int kStage, bool kSym = false>
__device__ __forceinline__ void tube_stage2(const float *g, const float *base, float *out, long long P,
                                            const TubeInfo &t, const ClassConsts &C, float2 a_self,
                                            float2 a_base, unsigned *flag)
{
    constexpr bool kBase = kStage == 1;
    const int nx = t.nx;
    const float2 *lx = t.lx_f2[kStage];
    const float2 half2 = make_float2(0.5f, 0.5f);
    for (int x = 2 * threadIdx.x; x < nx; x += 2 * blockDim.x) {
        const bool two = x + 1 < nx;
        const int xb = two ? x + 1 : x;
        const int m2a = x >= 2 ? x - 2 : 0, m1a = x >= 1 ? x - 1 : 0;
        const int p1a = x + 1 < nx ? x + 1 : nx - 1, p2a = x + 2 < nx ? x + 2 : nx - 1;
        const int m2b = xb >= 2 ? xb - 2 : 0, m1b = xb >= 1 ? xb - 1 : 0;
        const int p1b = xb + 1 < nx ? xb + 1 : nx - 1, p2b = xb + 2 < nx ? xb + 2 : nx - 1;
        float2 fs[kNV], heq[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i)
            if (!kSym || mirror_y(i) == i) fs[i] = make_float2(g[i * P + x], g[i * P + xb]);
        if constexpr (kSym) {
#pragma unroll
            for (int i = 0; i < kNV; ++i)
                if (mirror_y(i) != i) fs[i] = fs[mirror_y(i)];
            df_equilibrium_sym(C.dfeq2[kStage], C.dfm2, t.dfs2[kStage], fs, heq, flag);
        } else {
            df_equilibrium(C.dfeq2[kStage], C.dfm2, t.dfs2[kStage], fs, heq, flag);
        }
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            if (kSym && mirror_y(i) != i) continue;
            float2 o = fma_rn(a_self, fs[i], heq[i]);
            if (kBase) o = fma_rn(a_base, make_float2(base[i * P + x], base[i * P + xb]), o);
            if (dirx(i) != 0) {
                const float *gp = g + i * P;
                const bool pos = dirx(i) > 0;
                const float2 u2 = pos ? make_float2(gp[m2a], gp[m2b]) : make_float2(gp[p2a], gp[p2b]);
                const float2 u1 = pos ? make_float2(gp[m1a], gp[m1b]) : make_float2(gp[p1a], gp[p1b]);
                const float2 d1 = pos ? make_float2(gp[p1a], gp[p1b]) : make_float2(gp[m1a], gp[m1b]);
                const float2 av = sub_rn(fs[i], u1);
                const float2 bv = sub_rn(d1, fs[i]);
                const float2 ev = sub_rn(u1, u2);
                const float2 tt = sub_rn(minmod(bv, av), minmod(av, ev));
                o = fma_rn(neg(lx[i >> 2]), fma_rn(half2, tt, av), o);
            }
            out[i * P + x] = o.x;
            if (two) out[i * P + xb] = o.y;
            if (kSym && sym_partner(i) >= 0) {
                out[sym_partner(i) * P + x] = o.x;
                if (two) out[sym_partner(i) * P + xb] = o.y;
            }
        }
    }
}

// Register budget (resident threads per SM the registers must allow): 384 for the
// double-precision equilibrium (168 registers at 128 threads) and for the two-column
// df64 one, whose two cells of float arithmetic take about as many.  The symmetric
// forms keep less live state: 512 for FP64 and FP32_BULK (126 / 116 registers at
// 128 threads, no spills; 1.97e9 / 3.05e9 against 1.95e9 / 2.90e9 cell-updates/s on
// the 1024-tube ensemble) and 640 for df64 (96 registers; 1.13e10 against 1.07e10;
// 768 spilled 380 bytes).  The one-cell deviation equilibrium fits 64 registers
// without spills, so 1024 (32 warps per SM): 1.50e10 against 1.31e10 at 512 (127
// registers); 1280 spilled and fell back to 1.32e10.
constexpr int batch_thread_budget(int eq, bool sym)
{
    return eq == kEqF32 ? 1024 : (sym ? (eq == kEqDF ? 640 : 512) : 384);
}
constexpr int batch_min_blocks(int threads, int eq, bool sym)
{
    return batch_thread_budget(eq, sym) / threads > 0 ? batch_thread_budget(eq, sym) / threads : 1;
}

template <typename TS, int kThreads, int kEq, bool kSym>
__global__ void __launch_bounds__(kThreads, batch_min_blocks(kThreads, kEq, kSym)) batch_kernel(TS *f, TS *f1, const TubeInfo *tubes,
                                                         const int *work, const int *work_off, int nsteps,
                                                         const BatchArgs a, unsigned *flag)
{
    const TS as0 = pick<TS>(a.a_self[0], a.a_self_f[0]), as1 = pick<TS>(a.a_self[1], a.a_self_f[1]);
    const TS ab0 = pick<TS>(a.a_base[0], a.a_base_f[0]), ab1 = pick<TS>(a.a_base[1], a.a_base_f[1]);
    // x row buffer of the FP64 stage (a placeholder for the single-precision states)
    __shared__ double row_u[kSingle<TS> ? 1 : 12][kSingle<TS> ? 1 : kThreads + 2];
    for (int w = work_off[blockIdx.x]; w < work_off[blockIdx.x + 1]; ++w) {
        const TubeInfo &t = tubes[work[w]];
        const ClassConsts &C = a.cls[t.cls];
        TS *ft = f + t.offset;
        TS *f1t = f1 + t.offset;
        for (int s = 0; s < nsteps; ++s) {
            if constexpr (!kSingle<TS>) {
                tube_stage_shared_x<0, kThreads, kSym>(ft, nullptr, f1t, a.P, t, C, as0, ab0, flag, row_u);
                __syncthreads();
                tube_stage_shared_x<1, kThreads, kSym>(f1t, ft, ft, a.P, t, C, as1, ab1, flag, row_u);
            } else if constexpr (kEq == kEqDF) {
                tube_stage2<0, kSym>(ft, nullptr, f1t, a.P, t, C, a.a_self_f2[0], a.a_base_f2[0], flag);
                __syncthreads();
                tube_stage2<1, kSym>(f1t, ft, ft, a.P, t, C, a.a_self_f2[1], a.a_base_f2[1], flag);
            } else {
                tube_stage<TS, 0, kEq, kSym>(ft, nullptr, f1t, a.P, t, C, as0, ab0, flag);
                __syncthreads();
                tube_stage<TS, 1, kEq, kSym>(f1t, ft, ft, a.P, t, C, as1, ab1, flag);
            }
            __syncthreads();
        }
    }
}

// Tube of a global cell index (offsets ascending, ntubes + 1 entries with the total last).
__device__ __forceinline__ int tube_of(const long long *offs, int ntubes, long long c)
{
    int lo = 0, hi = ntubes;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offs[mid] <= c) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename TS>
__global__ void __launch_bounds__(128) batch_init_kernel(const BatchArgs a, const TubeInfo *tubes,
                                                          const long long *offs, int ntubes,
                                                          const double *rho, const double *ux,
                                                          const double *uy, const double *T, TS *f,
                                                          unsigned *flag)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.P;
         c += (long long)gridDim.x * blockDim.x) {
        const TubeInfo &t = tubes[tube_of(offs, ntubes, c)];
        const ClassConsts &C = a.cls[t.cls];
        const double r = rho[c], u = ux[c], v = uy[c], tt = T[c];
        const double jx = r * u, jy = r * v;
        const double jyuy = jy * v;
        const double ru2 = fma(jx, u, jyuy);
        const double p = r * tt;
        const double E = fma(C.m.K, p, ru2);
        double fe[kNV];
        equilibrium(C.unit, C.m, r, E, jx, jy, u, v, ru2, jyuy, p, tt, fe);
        if (!(positive_finite(r) && positive_finite(tt) && isfinite(u) && isfinite(v)))
            atomicOr(flag, kFlagNonPhys);
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            if constexpr (kSingle<TS>)
                f[i * a.P + c] = (float)(fe[i] - t.Fg[i >> 2]);
            else
                f[i * a.P + c] = fe[i];
        }
    }
}

template <typename TS>
__global__ void __launch_bounds__(128) batch_macros_kernel(const BatchArgs a, const TubeInfo *tubes,
                                                            const long long *offs, int ntubes, const TS *f,
                                                            double *rho, double *ux, double *uy, double *T)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.P;
         c += (long long)gridDim.x * blockDim.x) {
        const TubeInfo &t = tubes[tube_of(offs, ntubes, c)];
        const ModelConsts &m = a.cls[t.cls].m;
        // the operations of the single-grid macros kernel: moments of the stored
        // values (plus the reference equilibrium's for a single-precision state)
        // and one reciprocal of rho
        double fc[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) fc[i] = widen(f[i * a.P + c]);
        Cons q = conserved(fc, m);
        if constexpr (kSingle<TS>) {
            q.rho += t.rhoF;
            q.E += t.EF;
        }
        const double r = rcp64(q.rho);
        const double u = q.jx * r, v = q.jy * r;
        const double ru2 = fma(q.jx, u, q.jy * v);
        if (rho) rho[c] = q.rho;
        if (ux) ux[c] = u;
        if (uy) uy[c] = v;
        if (T) T[c] = (q.E - ru2) * m.invK * r;
    }
}

template <typename TS, int kEq, bool kSym>
void *batch_func_t(int threads)
{
    switch (threads) {
    case 64: return (void *)batch_kernel<TS, 64, kEq, kSym>;
    case 256: return (void *)batch_kernel<TS, 256, kEq, kSym>;
    default: return (void *)batch_kernel<TS, 128, kEq, kSym>;
    }
}

// sym: every tube's state is y-symmetric (u_y = 0 at initialisation)
void *batch_func(int precision, int threads, bool sym)
{
    if (precision == CDBM_FP32_DF64)
        return sym ? batch_func_t<float, kEqDF, true>(threads) : batch_func_t<float, kEqDF, false>(threads);
    if (precision == CDBM_FP32_DEV)
        return sym ? batch_func_t<float, kEqF32, true>(threads) : batch_func_t<float, kEqF32, false>(threads);
    if (precision == CDBM_FP32_BULK)
        return sym ? batch_func_t<float, kEqDouble, true>(threads) : batch_func_t<float, kEqDouble, false>(threads);
    return sym ? batch_func_t<double, kEqDouble, true>(threads) : batch_func_t<double, kEqDouble, false>(threads);
}

}  // namespace

struct cdbm_batch {
    int ntubes, precision;
    long long P;
    double tau, dt;
    cudaStream_t stream;
    cdbm_allocator alloc;
    bool user_alloc;
    int sm_count;
    std::vector<int> nx;
    std::vector<long long> offs;       // ntubes + 1
    std::vector<TubeInfo> info;
    std::vector<double> Ivals;         // distinct I per class
    BatchArgs args;
    void *f, *f1;
    TubeInfo *d_tubes;
    long long *d_offs;
    int *d_work, *d_work_off;          // partition: tube ids per block (CSR)
    unsigned *flag;
    unsigned *flag_host;
    int threads, blocks;               // current tile: threads per block, number of blocks
    bool state_set;
    double t;
    cudaGraphExec_t graph;
    int graph_steps;
    bool sym;                          // every tube started with u_y = 0: y-symmetric states
    bool sym_enabled;                  // use the symmetric kernels when sym (default)
    cdbm_status err;
    char msg[256];
};

namespace {

cdbm_status bset_err(cdbm_batch *b, cdbm_status s, const char *fmt, ...)
{
    if (b->err != CDBM_OK) return b->err;
    b->err = s;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->msg, sizeof(b->msg), fmt, ap);
    va_end(ap);
    return s;
}

cdbm_status bcreate_err(cdbm_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(thread_error_buffer(), kThreadErrorBytes, fmt, ap);
    va_end(ap);
    return s;
}

cdbm_status bcuda(cdbm_batch *b, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return CDBM_OK;
    cudaGetLastError();
    return bset_err(b, CDBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *balloc(cdbm_batch *b, size_t bytes)
{
    if (b->user_alloc) return b->alloc.alloc(bytes, (void *)b->stream, b->alloc.user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, b->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void bfree(cdbm_batch *b, void *p, size_t bytes)
{
    if (!p) return;
    if (b->user_alloc)
        b->alloc.free(p, bytes, (void *)b->stream, b->alloc.user);
    else
        cudaFreeAsync(p, b->stream);
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void drop_batch_graph(cdbm_batch *b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// Longest-first partition of the tubes over nblocks blocks; a tube's cost is the
// number of cell slots its stages occupy, ceil(nx / threads) * threads.
void partition(const cdbm_batch *b, int threads, int nblocks, std::vector<int> &work, std::vector<int> &off)
{
    std::vector<int> order(b->ntubes);
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int t) { return (long long)((b->nx[t] + threads - 1) / threads) * threads; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    std::vector<long long> load(nblocks, 0);
    std::vector<std::vector<int>> lists(nblocks);
    for (int t : order) {
        int best = 0;
        for (int k = 1; k < nblocks; ++k)
            if (load[k] < load[best]) best = k;
        load[best] += cost(t);
        lists[best].push_back(t);
    }
    work.clear();
    off.assign(1, 0);
    for (int k = 0; k < nblocks; ++k) {
        for (int t : lists[k]) work.push_back(t);
        off.push_back((int)work.size());
    }
}

cdbm_status set_tile(cdbm_batch *b, int threads, int blocks_per_sm)
{
    const int nblocks = std::max(1, std::min(b->ntubes, blocks_per_sm * b->sm_count));
    std::vector<int> work, off;
    partition(b, threads, nblocks, work, off);
    bfree(b, b->d_work, 0);
    bfree(b, b->d_work_off, 0);
    b->d_work = (int *)balloc(b, sizeof(int) * work.size());
    b->d_work_off = (int *)balloc(b, sizeof(int) * off.size());
    if (!b->d_work || !b->d_work_off) return bset_err(b, CDBM_ENOMEM, "work list allocation failed");
    if (bcuda(b, cudaMemcpyAsync(b->d_work, work.data(), sizeof(int) * work.size(), cudaMemcpyHostToDevice,
                                 b->stream), "work upload") ||
        bcuda(b, cudaMemcpyAsync(b->d_work_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice,
                                 b->stream), "work upload") ||
        bcuda(b, cudaStreamSynchronize(b->stream), "work upload sync"))
        return b->err;
    b->threads = threads;
    b->blocks = nblocks;
    drop_batch_graph(b);
    return CDBM_OK;
}

cdbm_status launch_run(cdbm_batch *b, int nsteps)
{
    void *f = b->f, *f1 = b->f1;
    const TubeInfo *tubes = b->d_tubes;
    const int *work = b->d_work, *off = b->d_work_off;
    void *args[] = {&f, &f1, (void *)&tubes, (void *)&work, (void *)&off, &nsteps, (void *)&b->args, &b->flag};
    void *fn = batch_func(b->precision, b->threads, b->sym && b->sym_enabled);
    return bcuda(b, cudaLaunchKernel(fn, dim3(b->blocks), dim3(b->threads), args, 0, b->stream), "batch launch");
}

// One persistent launch of nsteps steps, replayed from an explicitly built graph.
cdbm_status run_graph(cdbm_batch *b, int nsteps)
{
    if (!b->graph || b->graph_steps != nsteps) {
        drop_batch_graph(b);
        void *f = b->f, *f1 = b->f1;
        const TubeInfo *tubes = b->d_tubes;
        const int *work = b->d_work, *off = b->d_work_off;
        void *args[] = {&f, &f1, (void *)&tubes, (void *)&work, (void *)&off, &nsteps, (void *)&b->args, &b->flag};
        cudaKernelNodeParams p;
        memset(&p, 0, sizeof(p));
        p.func = batch_func(b->precision, b->threads, b->sym && b->sym_enabled);
        p.gridDim = dim3(b->blocks);
        p.blockDim = dim3(b->threads);
        p.kernelParams = args;
        cudaGraph_t g;
        cudaGraphNode_t node;
        if (bcuda(b, cudaGraphCreate(&g, 0), "graph create")) return b->err;
        cudaError_t e = cudaGraphAddKernelNode(&node, g, nullptr, 0, &p);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return bcuda(b, e, "graph build");
        }
        b->graph_steps = nsteps;
    }
    return bcuda(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
}

unsigned cells_grid(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 127) / 128, 1 << 20)); }

}  // namespace

extern "C" {

cdbm_status cdbm_batch_create(int ntubes, const int *nx, const double *dx, const double *I,
                              const cdbm_vset *vset, double tau, double dt, int precision, void *cuda_stream,
                              const cdbm_allocator *allocator, cdbm_batch **out)
{
    if (!out) return bcreate_err(CDBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (ntubes < 1 || !nx || !dx || !I || !vset) return bcreate_err(CDBM_EINVAL, "batch: bad arguments");
    if (!(std::isfinite(dt) && dt > 0 && std::isfinite(tau) && tau > 0))
        return bcreate_err(CDBM_EINVAL, "dt and tau must be finite and > 0");
    if (dt / tau > 2.0) return bcreate_err(CDBM_EINVAL, "dt/tau = %g exceeds 2", dt / tau);
    if (precision != CDBM_FP64 && precision != CDBM_FP32_BULK && precision != CDBM_FP32_DF64 &&
        precision != CDBM_FP32_DEV)
        return bcreate_err(CDBM_EINVAL, "unsupported precision %d", precision);
    double vmax = 0.0;
    for (int g = 0; g < 4; ++g) {
        if (!std::isfinite(vset->v[g]) || !std::isfinite(vset->eta[g]) || vset->v[g] <= 0 || vset->eta[g] < 0)
            return bcreate_err(CDBM_EINVAL, "velocity set: v must be > 0 and eta >= 0");
        vmax = std::max(vmax, vset->v[g]);
    }
    cdbm_batch *b = new (std::nothrow) cdbm_batch();
    if (!b) return bcreate_err(CDBM_ENOMEM, "host allocation failed");
    b->ntubes = ntubes;
    b->precision = precision;
    b->tau = tau;
    b->dt = dt;
    b->stream = (cudaStream_t)cuda_stream;
    b->user_alloc = allocator && allocator->alloc && allocator->free;
    if (b->user_alloc) b->alloc = *allocator;
    b->err = CDBM_OK;
    b->sym = false;
    b->sym_enabled = true;
    strcpy(b->msg, "no error");
    b->nx.assign(nx, nx + ntubes);
    b->offs.assign(ntubes + 1, 0);
    b->info.resize(ntubes);
    const double h = dt / tau;
    const double alpha[2] = {0.0, 0.5}, beta[2] = {1.0, 0.5}, gamma[2] = {1.0, 0.5};
    for (int s = 0; s < 2; ++s) {
        b->args.a_self[s] = beta[s] - gamma[s] * h;
        b->args.a_base[s] = alpha[s];
        b->args.a_self_f[s] = (float)b->args.a_self[s];
        b->args.a_base_f[s] = (float)b->args.a_base[s];
        b->args.a_self_f2[s] = make_float2(b->args.a_self_f[s], b->args.a_self_f[s]);
        b->args.a_base_f2[s] = make_float2(b->args.a_base_f[s], b->args.a_base_f[s]);
    }
    for (int t = 0; t < ntubes; ++t) {
        if (nx[t] < 1 || !(std::isfinite(dx[t]) && dx[t] > 0) || !(std::isfinite(I[t]) && I[t] >= 0)) {
            delete b;
            return bcreate_err(CDBM_EINVAL, "tube %d: nx, dx or I invalid", t);
        }
        if (nx[t] > 1 && vmax * dt / dx[t] > 1.0) {
            delete b;
            return bcreate_err(CDBM_EINVAL, "tube %d: CFL number %g exceeds 1", t, vmax * dt / dx[t]);
        }
        int cls = -1;
        for (size_t k = 0; k < b->Ivals.size(); ++k)
            if (b->Ivals[k] == I[t]) cls = (int)k;
        if (cls < 0) {
            if ((int)b->Ivals.size() == kMaxClasses) {
                delete b;
                return bcreate_err(CDBM_EINVAL, "batch: more than %d distinct values of I", kMaxClasses);
            }
            cls = (int)b->Ivals.size();
            b->Ivals.push_back(I[t]);
            ClassConsts &C = b->args.cls[cls];
            double cond = 0.0;
            const char *which = "";
            if (build_blocks(*vset, I[t], C.m, C.unit, &cond, &which) != CDBM_OK) {
                delete b;
                return bcreate_err(CDBM_ESINGULAR, "moment matrix block '%s' singular (cond %g)", which, cond);
            }
            for (int s = 0; s < 2; ++s) {
                C.eq[s] = scaled(C.unit, gamma[s] * h);
                C.dfeq[s] = df_blocks(C.eq[s]);
                C.dfeq2[s] = df_blocks_twice(C.dfeq[s]);
            }
            C.dfm = df_model(C.m);
            C.dfm2 = df_model_twice(C.dfm);
            for (int s = 0; s < 2; ++s) C.dp[s] = dev_proj(C.m, gamma[s] * h);
        }
        TubeInfo &ti = b->info[t];
        memset(&ti, 0, sizeof(ti));
        ti.offset = b->offs[t];
        ti.nx = nx[t];
        ti.cls = cls;
        for (int s = 0; s < 2; ++s)
            for (int g = 0; g < 4; ++g) {
                ti.lx[s][g] = gamma[s] * dt * vset->v[g] / dx[t];
                ti.lx_f[s][g] = (float)ti.lx[s][g];
                ti.lx_f2[s][g] = make_float2(ti.lx_f[s][g], ti.lx_f[s][g]);
            }
        b->offs[t + 1] = b->offs[t] + nx[t];
    }
    b->P = b->offs[ntubes];
    b->args.P = b->P;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bcreate_err(CDBM_ECUDA, "no CUDA device");
    }
    const size_t fb = storage_bytes(precision) * kNV * (size_t)b->P;
    b->f = balloc(b, fb);
    b->f1 = balloc(b, fb);
    b->d_tubes = (TubeInfo *)balloc(b, sizeof(TubeInfo) * ntubes);
    b->d_offs = (long long *)balloc(b, sizeof(long long) * (ntubes + 1));
    b->flag = (unsigned *)balloc(b, 256);
    if (!b->f || !b->f1 || !b->d_tubes || !b->d_offs || !b->flag ||
        cudaMallocHost(&b->flag_host, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        cdbm_batch_destroy(b);
        return bcreate_err(CDBM_ENOMEM, "batch device allocation failed");
    }
    if (cudaMemsetAsync(b->flag, 0, sizeof(unsigned), b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->d_offs, b->offs.data(), sizeof(long long) * (ntubes + 1), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->d_tubes, b->info.data(), sizeof(TubeInfo) * ntubes, cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess) {
        cudaGetLastError();
        cdbm_batch_destroy(b);
        return bcreate_err(CDBM_ECUDA, "batch upload failed");
    }
    if (set_tile(b, 128, 3) != CDBM_OK) {
        cdbm_status s = b->err;
        cdbm_batch_destroy(b);
        return bcreate_err(s, "batch work partition failed");
    }
    *out = b;
    return CDBM_OK;
}

cdbm_status cdbm_batch_init(cdbm_batch *b, const double *rho, const double *ux, const double *uy, const double *T)
{
    if (!b) return CDBM_EINVAL;
    if (b->err) return b->err;
    if (!rho || !ux || !uy || !T) return bset_err(b, CDBM_EINVAL, "cdbm_batch_init: NULL field");
    const size_t n = (size_t)b->P;
    const double *src[4] = {rho, ux, uy, T};
    std::vector<double> host[4];
    const double *dev[4];
    // the second buffer (16 planes of the storage type) stages host fields: 4 double planes fit
    double *stage = (double *)b->f1;
    for (int k = 0; k < 4; ++k) {
        host[k].resize(n);
        if (bcuda(b, cudaMemcpy(host[k].data(), src[k], sizeof(double) * n, cudaMemcpyDefault), "batch fields read"))
            return b->err;
        if (is_device_ptr(src[k])) {
            dev[k] = src[k];
        } else {
            if (bcuda(b, cudaMemcpyAsync(stage + k * n, src[k], sizeof(double) * n, cudaMemcpyHostToDevice,
                                         b->stream), "batch fields upload"))
                return b->err;
            dev[k] = stage + k * n;
        }
    }
    // u_y = 0 everywhere: every tube's state is y-symmetric and stays so
    bool sym = true;
    for (size_t c = 0; c < n && sym; ++c) sym = host[2][c] == 0.0;
    if (sym != b->sym) {
        b->sym = sym;
        drop_batch_graph(b);
    }
    // per-tube reference state (FP32-bulk): means of rho and T over the tube
    for (int t = 0; t < b->ntubes; ++t) {
        TubeInfo &ti = b->info[t];
        const ClassConsts &C = b->args.cls[ti.cls];
        double sr = 0.0, sT = 0.0;
        for (long long c = b->offs[t]; c < b->offs[t + 1]; ++c) {
            sr += host[0][c];
            sT += host[3][c];
        }
        const double r0 = sr / ti.nx, T0 = sT / ti.nx, K = C.m.K, P0 = r0 * T0;
        ti.rhoF = ti.EF = 0.0;
        for (int g = 0; g < 4; ++g) {
            const double *S = C.unit.S + 4 * g;
            ti.Fg[g] = single_storage(b->precision)
                           ? S[0] * r0 + S[1] * K * P0 + S[3] * 2.0 * (K + 2.0) * P0 * T0
                           : 0.0;
            ti.rhoF += 4.0 * ti.Fg[g];
            ti.EF += 4.0 * ti.Fg[g] * C.m.w[g];
        }
        const double h = b->dt / b->tau, gamma[2] = {1.0, 0.5};
        for (int s = 0; s < 2; ++s) {
            for (int g = 0; g < 4; ++g) ti.sF[s][g] = gamma[s] * h * ti.Fg[g];
            ti.dfs[s] = df_shift(ti.sF[s], ti.rhoF, ti.EF);
            ti.dfs2[s] = df_shift_twice(ti.dfs[s]);
        }
    }
    const unsigned nb = cells_grid(b->P);
    if (bcuda(b, cudaMemcpyAsync(b->d_tubes, b->info.data(), sizeof(TubeInfo) * b->ntubes, cudaMemcpyHostToDevice,
                                 b->stream), "tube upload"))
        return b->err;
    if (single_storage(b->precision))
        batch_init_kernel<float><<<nb, 128, 0, b->stream>>>(b->args, b->d_tubes, b->d_offs, b->ntubes, dev[0], dev[1],
                                                            dev[2], dev[3], (float *)b->f, b->flag);
    else
        batch_init_kernel<double><<<nb, 128, 0, b->stream>>>(b->args, b->d_tubes, b->d_offs, b->ntubes, dev[0],
                                                             dev[1], dev[2], dev[3], (double *)b->f, b->flag);
    if (bcuda(b, cudaGetLastError(), "batch init launch") || bcuda(b, cudaStreamSynchronize(b->stream), "batch init sync"))
        return b->err;
    b->t = 0.0;
    b->state_set = true;
    return CDBM_OK;
}

cdbm_status cdbm_batch_step(cdbm_batch *b, int nsteps)
{
    if (!b) return CDBM_EINVAL;
    if (b->err) return b->err;
    if (nsteps < 0) return bset_err(b, CDBM_EINVAL, "cdbm_batch_step: nsteps < 0");
    if (!b->state_set) return bset_err(b, CDBM_EINVAL, "cdbm_batch_step: state not initialised");
    if (nsteps == 0) return CDBM_OK;
    if (run_graph(b, nsteps)) return b->err;
    b->t += nsteps * b->dt;
    return CDBM_OK;
}

cdbm_status cdbm_batch_autotune(cdbm_batch *b, int trial_steps, int *threads_out, int *blocks_per_sm_out)
{
    if (!b) return CDBM_EINVAL;
    if (b->err) return b->err;
    if (!b->state_set) return bset_err(b, CDBM_EINVAL, "cdbm_batch_autotune: state not initialised");
    if (trial_steps < 1) trial_steps = 1;
    // The trials advance the state; it is saved and restored around them.
    const size_t fb = storage_bytes(b->precision) * kNV * (size_t)b->P;
    void *save = balloc(b, fb);
    if (!save) return bset_err(b, CDBM_ENOMEM, "autotune backup allocation failed");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cand_threads[3] = {64, 128, 256};
    const int cand_bpsm[5] = {1, 2, 3, 4, 6};
    const int max_threads = 1024;
    float best = 1e30f;
    int bt = b->threads, bb = 3;
    cdbm_status st = CDBM_OK;
    if (bcuda(b, cudaMemcpyAsync(save, b->f, fb, cudaMemcpyDeviceToDevice, b->stream), "autotune backup"))
        st = b->err;
    for (int i = 0; i < 3 && st == CDBM_OK; ++i)
        for (int j = 0; j < 5 && st == CDBM_OK; ++j) {
            if (cand_threads[i] * cand_bpsm[j] > max_threads) continue;
            if ((st = set_tile(b, cand_threads[i], cand_bpsm[j])) != CDBM_OK) break;
            if ((st = launch_run(b, 1)) != CDBM_OK) break;        // warm-up
            cudaEventRecord(e0, b->stream);
            if ((st = launch_run(b, trial_steps)) != CDBM_OK) break;
            cudaEventRecord(e1, b->stream);
            if ((st = bcuda(b, cudaEventSynchronize(e1), "autotune sync")) != CDBM_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bt = cand_threads[i];
                bb = cand_bpsm[j];
            }
            if ((st = bcuda(b, cudaMemcpyAsync(b->f, save, fb, cudaMemcpyDeviceToDevice, b->stream),
                            "autotune restore")) != CDBM_OK)
                break;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bfree(b, save, fb);
    if (st != CDBM_OK) return st;
    if (set_tile(b, bt, bb)) return b->err;
    if (bcuda(b, cudaMemsetAsync(b->flag, 0, sizeof(unsigned), b->stream), "flag reset")) return b->err;
    if (threads_out) *threads_out = bt;
    if (blocks_per_sm_out) *blocks_per_sm_out = bb;
    return CDBM_OK;
}

cdbm_status cdbm_batch_set_tile(cdbm_batch *b, int threads, int blocks_per_sm)
{
    if (!b) return CDBM_EINVAL;
    if (b->err) return b->err;
    if ((threads != 64 && threads != 128 && threads != 256) || blocks_per_sm < 1 || blocks_per_sm > 16)
        return bset_err(b, CDBM_EINVAL, "tile: threads must be 64, 128 or 256 and blocks_per_sm in 1..16");
    return set_tile(b, threads, blocks_per_sm);
}

cdbm_status cdbm_batch_set_symmetric(cdbm_batch *b, int enable)
{
    if (!b) return CDBM_EINVAL;
    if (b->err) return b->err;
    if ((enable != 0) != b->sym_enabled) {
        b->sym_enabled = enable != 0;
        drop_batch_graph(b);
    }
    return CDBM_OK;
}

cdbm_status cdbm_batch_macros(cdbm_batch *b, double *rho, double *ux, double *uy, double *T)
{
    if (!b) return CDBM_EINVAL;
    if (b->err) return b->err;
    if (!b->state_set) return bset_err(b, CDBM_EINVAL, "cdbm_batch_macros: state not initialised");
    const size_t n = (size_t)b->P;
    double *dst[4] = {rho, ux, uy, T};
    double *dev[4];
    bool host[4];
    double *stage = (double *)b->f1;
    for (int k = 0; k < 4; ++k) {
        host[k] = dst[k] && !is_device_ptr(dst[k]);
        dev[k] = host[k] ? stage + k * n : dst[k];
    }
    const unsigned nb = cells_grid(b->P);
    if (single_storage(b->precision))
        batch_macros_kernel<float><<<nb, 128, 0, b->stream>>>(b->args, b->d_tubes, b->d_offs, b->ntubes,
                                                              (const float *)b->f, dev[0], dev[1], dev[2], dev[3]);
    else
        batch_macros_kernel<double><<<nb, 128, 0, b->stream>>>(b->args, b->d_tubes, b->d_offs, b->ntubes,
                                                               (const double *)b->f, dev[0], dev[1], dev[2], dev[3]);
    if (bcuda(b, cudaGetLastError(), "batch macros launch")) return b->err;
    for (int k = 0; k < 4; ++k)
        if (host[k] && bcuda(b, cudaMemcpyAsync(dst[k], dev[k], sizeof(double) * n, cudaMemcpyDeviceToHost,
                                                b->stream), "batch macros download"))
            return b->err;
    return bcuda(b, cudaStreamSynchronize(b->stream), "batch macros sync");
}

cdbm_status cdbm_batch_sync(cdbm_batch *b)
{
    if (!b) return CDBM_EINVAL;
    if (b->err) return b->err;
    if (bcuda(b, cudaMemcpyAsync(b->flag_host, b->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream),
              "flag download") ||
        bcuda(b, cudaStreamSynchronize(b->stream), "cdbm_batch_sync"))
        return b->err;
    if (*b->flag_host & kFlagNonPhys)
        return bset_err(b, CDBM_ENONPHYS, "non-physical state (rho <= 0, T <= 0 or non-finite) at t = %g", b->t);
    return CDBM_OK;
}

cdbm_status cdbm_batch_info(const cdbm_batch *b, long long *total_cells, int *threads, int *blocks)
{
    if (!b) return CDBM_EINVAL;
    if (total_cells) *total_cells = b->P;
    if (threads) *threads = b->threads;
    if (blocks) *blocks = b->blocks;
    return b->err;
}

const char *cdbm_batch_last_error(const cdbm_batch *b) { return b ? b->msg : thread_error_buffer(); }

void cdbm_batch_destroy(cdbm_batch *b)
{
    if (!b) return;
    drop_batch_graph(b);
    const size_t fb = storage_bytes(b->precision) * kNV * (size_t)b->P;
    bfree(b, b->f, fb);
    bfree(b, b->f1, fb);
    bfree(b, b->d_tubes, 0);
    bfree(b, b->d_offs, 0);
    bfree(b, b->flag, 256);
    bfree(b, b->d_work, 0);
    bfree(b, b->d_work_off, 0);
    cudaStreamSynchronize(b->stream);
    if (b->flag_host) cudaFreeHost(b->flag_host);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
