// Per-cell pieces of a Runge-Kutta stage shared by the stage kernels: the stage
// coefficients in the storage precision and the scaled equilibrium of one cell.
#pragma once

#include "cdbm_f32dev.cuh"

namespace cdbm {

// Stage coefficients in the storage precision.
template <typename TS>
__device__ __forceinline__ TS a_self_of(const StageArgs &a)
{
    if constexpr (kSingle<TS>) return a.a_self_f; else return a.a_self;
}
template <typename TS>
__device__ __forceinline__ TS a_base_of(const StageArgs &a)
{
    if constexpr (kSingle<TS>) return a.a_base_f; else return a.a_base;
}
template <typename TS>
__device__ __forceinline__ TS lx_of(const StageArgs &a, int g)
{
    if constexpr (kSingle<TS>) return a.lx_f[g]; else return a.lx[g];
}
template <typename TS>
__device__ __forceinline__ TS ly_of(const StageArgs &a, int g)
{
    if constexpr (kSingle<TS>) return a.ly_f[g]; else return a.ly[g];
}

// How a stage forms the equilibrium: in double (CDBM_FP64, CDBM_FP32_BULK), in df64
// (CDBM_FP32_DF64) or in single precision on the deviations (CDBM_FP32_DEV).
constexpr int kEqDouble = 0, kEqDF = 1, kEqF32 = 2;

// gamma h f_eq of one cell in the storage precision (minus gamma h F for the
// single-precision deviation state): moments, primitives and equilibrium in double,
// all of it in df64 (kEq = kEqDF) or in single precision on the moment deviations
// (kEq = kEqF32).
template <typename TS, int kEq>
__device__ __forceinline__ void stage_equilibrium(const StageArgs &a, const TS fs[kNV], TS heq[kNV],
                                                  unsigned *flag)
{
    if constexpr (kEq == kEqF32) {
        static_assert(kSingle<TS>, "the deviation equilibrium is for the single-precision state");
        f32_equilibrium(a.d.b, a.d.m, a.d.r, a.dp, fs, heq, flag);
    } else if constexpr (kEq == kEqDF) {
        static_assert(kSingle<TS>, "df64 equilibrium is for the single-precision state");
        df_equilibrium(a.d.b, a.d.m, a.d.r, fs, heq, flag);
    } else {
        double f[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) f[i] = widen(fs[i]);
        const Prim s = primitives<kSingle<TS>>(f, a.m, a.rhoF, a.EF, flag);
        double h[kNV];
        equilibrium<kSingle<TS>>(a.eq, a.m, s.q.rho, s.q.E, s.q.jx, s.q.jy, s.ux, s.uy, s.ru2, s.jyuy,
                                 s.p, s.T, h, a.sF);
#pragma unroll
        for (int i = 0; i < kNV; ++i) heq[i] = narrow<TS>(h[i]);
    }
}

}  // namespace cdbm
