// CDBM kernels: initial equilibrium, the fused Runge-Kutta stage, macroscopic
// fields, nonequilibrium moments and conserved sums.  The distribution buffers
// are stored in double (CDBM_FP64) or single (CDBM_FP32_BULK, CDBM_FP32_DF64,
// CDBM_FP32_DEV) precision, selected by the template parameter TS; the conserved
// sums and the equilibrium of a stage are computed in double, in double-float
// arithmetic on the FP32 pipe for CDBM_FP32_DF64, or in single precision on the
// moment deviations for CDBM_FP32_DEV (template parameter kEq).
//
// Layout: f[16][ny][nx] (velocity plane outermost, x fastest).  A block covers a
// run of columns along x, so centre loads and stores of a warp are coalesced rows
// and the stencil neighbours (x +- 1, 2 and the rows y +- 1, 2) are served from
// L1/L2 or shared memory.  stage_kernel gives each thread one cell; the
// row-marching kernels give each thread one column (two for the df64 and deviation states) over a
// run of rows.
#include "cdbm_stage.cuh"

namespace cdbm {

namespace {

constexpr int kStageThreads = 128;
#ifndef CDBM_STAGE_MIN_BLOCKS
#define CDBM_STAGE_MIN_BLOCKS 3   // resident stage blocks per SM the register budget must allow
#endif
// The one-cell df64 stage kernel keeps its arithmetic in float registers and hides
// memory latency better with more warps: 6 blocks of 128 threads per SM (80
// registers) measured fastest (2.25 ms per 4096^2 vortex step, against 2.47 ms at 3
// blocks).  Large 2-D df64 grids use the two-column kernel (kMarch2MinBlocks).
#ifndef CDBM_STAGE_MIN_BLOCKS_DF
#define CDBM_STAGE_MIN_BLOCKS_DF 6
#endif
constexpr int stage_min_blocks(int eq) { return eq != kEqDouble ? CDBM_STAGE_MIN_BLOCKS_DF : CDBM_STAGE_MIN_BLOCKS; }

// ---------------------------------------------------------------- init (K0)

template <typename TS>
__global__ void __launch_bounds__(128) init_kernel(const FieldArgs a, const double *__restrict__ rho,
                                                    const double *__restrict__ ux,
                                                    const double *__restrict__ uy,
                                                    const double *__restrict__ T,
                                                    TS *__restrict__ f, unsigned *flag)
{
    const size_t P = (size_t)a.nx * a.ny;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < P;
         c += (size_t)gridDim.x * blockDim.x) {
        const double r = rho[c], u = ux[c], v = uy[c], t = T[c];
        const double jx = r * u, jy = r * v;
        const double jyuy = jy * v;
        const double ru2 = fma(jx, u, jyuy);
        const double p = r * t;
        const double E = fma(a.m.K, p, ru2);
        double fe[kNV];
        equilibrium(a.eq, a.m, r, E, jx, jy, u, v, ru2, jyuy, p, t, fe);
        if (!(positive_finite(r) && positive_finite(t) && isfinite(u) && isfinite(v)))
            atomicOr(flag, kFlagNonPhys);
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            if constexpr (kSingle<TS>)
                f[i * P + c] = (float)(fe[i] - a.Fg[i >> 2]);
            else
                f[i * P + c] = fe[i];
        }
    }
}

// ------------------------------------------------------------ RK stage (K1/K2)

// out = a_base base + a_self g + gamma h f_eq(g) - sum_r l_r D_r(g) for one cell:
// macros -> equilibrium -> BGK -> NND transport of all 16 velocities -> update.
template <typename TS, bool kBase, bool kFlatY, int kEq>
__global__ void __launch_bounds__(kStageThreads, stage_min_blocks(kEq))
    stage_kernel(const TS *__restrict__ g, const TS *base, TS *out, const StageArgs a, unsigned *flag)
{
    const int nx = a.nx, ny = a.ny;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const size_t P = (size_t)nx * ny;
    const int xm2 = neighbour(x - 2, nx, a.bc_x), xm1 = neighbour(x - 1, nx, a.bc_x);
    const int xp1 = neighbour(x + 1, nx, a.bc_x), xp2 = neighbour(x + 2, nx, a.bc_x);
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        const size_t row = (size_t)y * nx;
        const size_t c = row + x;
        size_t rm2 = 0, rm1 = 0, rp1 = 0, rp2 = 0;
        if (!kFlatY) {
            rm2 = (size_t)neighbour(y - 2, ny, a.bc_y) * nx + x;
            rm1 = (size_t)neighbour(y - 1, ny, a.bc_y) * nx + x;
            rp1 = (size_t)neighbour(y + 1, ny, a.bc_y) * nx + x;
            rp2 = (size_t)neighbour(y + 2, ny, a.bc_y) * nx + x;
        }
        TS fs[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) fs[i] = __ldg(g + i * P + c);
        TS heq[kNV];
        stage_equilibrium<TS, kEq>(a, fs, heq, flag);

#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            const int grp = i >> 2;
            const TS *gp = g + i * P;
            TS o = fma_t(a_self_of<TS>(a), fs[i], heq[i]);
            if (kBase) o = fma_t(a_base_of<TS>(a), base[i * P + c], o);
            if (dirx(i) != 0) {
                const TS u2 = __ldg(gp + row + (dirx(i) > 0 ? xm2 : xp2));
                const TS u1 = __ldg(gp + row + (dirx(i) > 0 ? xm1 : xp1));
                const TS d1 = __ldg(gp + row + (dirx(i) > 0 ? xp1 : xm1));
                o = fma_t(-lx_of<TS>(a, grp), nnd(u2, u1, fs[i], d1), o);
            }
            if (!kFlatY && diry(i) != 0) {
                const TS u2 = __ldg(gp + (diry(i) > 0 ? rm2 : rp2));
                const TS u1 = __ldg(gp + (diry(i) > 0 ? rm1 : rp1));
                const TS d1 = __ldg(gp + (diry(i) > 0 ? rp1 : rm1));
                o = fma_t(-ly_of<TS>(a, grp), nnd(u2, u1, fs[i], d1), o);
            }
            out[i * P + c] = o;
        }
    }
}

// Same stage for 2-D grids with the y-direction differences shared along a run of
// rows.  A block covers kStageThreads columns and a run of R = ceil(ny / gridDim.y)
// rows; each thread marches up its column.  For a velocity with y-sign s the
// upwind-ordered difference U_y = f_y - f_{y-s} and N_y = minmod(U_{y+s}, U_y) give
// the transport difference U_y + (N_y - N_{y-s}) / 2, which is the nnd() expression
// with a = U_y, b = U_{y-s}, e = U_{y+s}.  Each row computes one new U and one new N
// per velocity and carries them to the next row in shared memory, so a y-term costs
// 4 instead of 6 arithmetic instructions, with the same operations as stage_kernel.
constexpr int kNY = 12;                             // velocities with a y-component
constexpr size_t kMarchRowBytes = 2 * 12 * (kStageThreads + 2) * sizeof(double);   // FP64 x row buffers
__host__ __device__ constexpr int yvel(int k)       // k-th velocity with diry != 0
{
    return k < 2 ? 1 + 2 * k : (k < 6 ? k + 2 : (k < 8 ? 9 + 2 * (k - 6) : k + 4));
}

template <typename TS, bool kBase, int kEq>
__global__ void __launch_bounds__(kStageThreads, stage_min_blocks(kEq))
    stage_march_kernel(const TS *__restrict__ g, const TS *base, TS *out, const StageArgs a, unsigned *flag)
{
    // In double precision the x differences are shared as well: each thread computes
    // U_x = f_x - f_{x-s} of its cell once per velocity and reads U_{x+s}, U_{x-s} of
    // its neighbours from a row buffer (double-buffered in dynamic shared memory, so
    // one block barrier per row; the edge threads add the halo values), so an x-term
    // costs 4 FP64 instructions plus a share of the halo instead of 6.  The operands and operations are those of nnd(), so the
    // result is the same bit for bit.  In single precision the FP32 arithmetic is not
    // the scarce unit and the plain three-load form is kept.
    constexpr bool kShareX = !kSingle<TS>;
    constexpr int kNXV = 12;                          // velocities with an x component
    __shared__ TS carry_u[kNY][kStageThreads];
    __shared__ TS carry_n[kNY][kStageThreads];
    extern __shared__ __align__(16) unsigned char march_dyn[];   // [2][kNXV][kStageThreads + 2] TS
    TS(*const row_buf)[kStageThreads + 2] = reinterpret_cast<TS(*)[kStageThreads + 2]>(march_dyn);
    const int nx = a.nx, ny = a.ny;
    const int tid = threadIdx.x;
    const int x = blockIdx.x * blockDim.x + tid;
    const bool active = x < nx;
    if (!kShareX && !active) return;
    const int R = (ny + gridDim.y - 1) / gridDim.y;
    const int y0 = blockIdx.y * R;
    const int y1 = y0 + R < ny ? y0 + R : ny;
    if (y0 >= y1) return;                             // the same for the whole block
    const int last = (nx - (int)(blockIdx.x * blockDim.x) < (int)blockDim.x
                          ? nx - (int)(blockIdx.x * blockDim.x) : (int)blockDim.x) - 1;   // last active thread
    const size_t P = (size_t)nx * ny;
    const int xc = active ? x : nx - 1;               // inactive threads only pass the barriers
    const int xm2 = neighbour(xc - 2, nx, a.bc_x), xm1 = neighbour(xc - 1, nx, a.bc_x);
    const int xp1 = neighbour(xc + 1, nx, a.bc_x), xp2 = neighbour(xc + 2, nx, a.bc_x);

    // prologue: U_{y0} and N_{y0 - 1} for s = +1, N_{y0} for s = -1
    if (active) {
        const size_t r0 = (size_t)y0 * nx + x;
        const size_t rm1 = (size_t)neighbour(y0 - 1, ny, a.bc_y) * nx + x;
        const size_t rm2 = (size_t)neighbour(y0 - 2, ny, a.bc_y) * nx + x;
        const size_t rp1 = (size_t)neighbour(y0 + 1, ny, a.bc_y) * nx + x;
#pragma unroll
        for (int k = 0; k < kNY; ++k) {
            const int i = yvel(k);
            const TS *gp = g + i * P;
            const TS f0 = __ldg(gp + r0), fm1 = __ldg(gp + rm1);
            if (diry(i) > 0) {
                const TS u = f0 - fm1;                    // U_{y0}
                const TS um = fm1 - __ldg(gp + rm2);      // U_{y0-1}
                carry_u[k][tid] = u;
                carry_n[k][tid] = minmod(u, um);          // N_{y0-1}
            } else {
                const TS u = f0 - __ldg(gp + rp1);        // U_{y0}
                const TS um = fm1 - f0;                   // U_{y0-1}
                carry_u[k][tid] = u;
                carry_n[k][tid] = minmod(um, u);          // N_{y0}
            }
        }
    }

    for (int y = y0; y < y1; ++y) {
        const size_t row = (size_t)y * nx;
        const size_t c = row + xc;
        // row y writes buffer y & 1; its readers have passed the next row's barrier
        // before row y + 2 writes the same buffer again
        TS(*const row_u)[kStageThreads + 2] = row_buf + (kShareX ? (y & 1) * kNXV : 0);
        TS fs[kNV], o[kNV];
        if (active) {
#pragma unroll
            for (int i = 0; i < kNV; ++i) fs[i] = __ldg(g + i * P + c);
            TS heq[kNV];
            stage_equilibrium<TS, kEq>(a, fs, heq, flag);
            int k = 0;
#pragma unroll
            for (int i = 0; i < kNV; ++i) {
                o[i] = fma_t(a_self_of<TS>(a), fs[i], heq[i]);
                if (kBase) o[i] = fma_t(a_base_of<TS>(a), base[i * P + c], o[i]);
                if (dirx(i) != 0) {
                    const TS *gp = g + i * P + row;
                    const TS u1 = __ldg(gp + (dirx(i) > 0 ? xm1 : xp1));
                    if constexpr (kShareX) {
                        row_u[k][tid + 1] = fs[i] - u1;            // U at x: the upwind-ordered a of nnd()
                    } else {
                        const TS u2 = __ldg(gp + (dirx(i) > 0 ? xm2 : xp2));
                        const TS d1 = __ldg(gp + (dirx(i) > 0 ? xp1 : xm1));
                        o[i] = fma_t(-lx_of<TS>(a, i >> 2), nnd(u2, u1, fs[i], d1), o[i]);
                    }
                    ++k;
                }
            }
        }
        if constexpr (kShareX) {
            // Halo of the row buffer: U_{x-1} left of the block and U_{x+1} right of it (the
            // e or b of nnd() of the edge cells).  One branch taken by the edge threads only,
            // so the other warps do not issue these instructions.
            if (active && tid == 0) {
                int k = 0;
#pragma unroll
                for (int i = 0; i < kNV; ++i) {
                    if (dirx(i) == 0) continue;
                    const TS *gp = g + i * P + row;
                    row_u[k][0] = dirx(i) > 0 ? __ldg(gp + xm1) - __ldg(gp + xm2) : __ldg(gp + xm1) - fs[i];
                    ++k;
                }
            }
            if (active && tid == last) {
                int k = 0;
#pragma unroll
                for (int i = 0; i < kNV; ++i) {
                    if (dirx(i) == 0) continue;
                    const TS *gp = g + i * P + row;
                    row_u[k][last + 2] = dirx(i) > 0 ? __ldg(gp + xp1) - fs[i] : __ldg(gp + xp1) - __ldg(gp + xp2);
                    ++k;
                }
            }
            __syncthreads();
            if (active) {
                int k = 0;
#pragma unroll
                for (int i = 0; i < kNV; ++i) {
                    if (dirx(i) == 0) continue;
                    const int s = dirx(i);
                    const TS av = row_u[k][tid + 1];              // c - u1
                    const TS bv = row_u[k][tid + 1 + s];          // d1 - c
                    const TS ev = row_u[k][tid + 1 - s];          // u1 - u2
                    const TS t = minmod(bv, av) - minmod(av, ev);
                    o[i] = fma_t(-lx_of<TS>(a, i >> 2), fma_t((TS)0.5, t, av), o[i]);
                    ++k;
                }
            }
        }
        if (active) {
            const size_t rp1 = (size_t)neighbour(y + 1, ny, a.bc_y) * nx + x;
            const size_t rp2 = (size_t)neighbour(y + 2, ny, a.bc_y) * nx + x;
#pragma unroll
            for (int k = 0; k < kNY; ++k) {
                const int i = yvel(k);
                const TS *gp = g + i * P;
                const TS u = carry_u[k][tid];
                const TS n = carry_n[k][tid];
                TS t;
                if (diry(i) > 0) {
                    const TS un = __ldg(gp + rp1) - fs[i];                  // U_{y+1}
                    const TS nn = minmod(un, u);                            // N_y
                    t = nn - n;                                             // N_y - N_{y-1}
                    carry_u[k][tid] = un;
                    carry_n[k][tid] = nn;
                } else {
                    const TS un = __ldg(gp + rp1) - __ldg(gp + rp2);        // U_{y+1}
                    const TS nn = minmod(u, un);                            // N_{y+1}
                    t = n - nn;                                             // N_y - N_{y+1}
                    carry_u[k][tid] = un;
                    carry_n[k][tid] = nn;
                }
                o[i] = fma_t(-ly_of<TS>(a, i >> 2), fma_t((TS)0.5, t, u), o[i]);
            }
#pragma unroll
            for (int i = 0; i < kNV; ++i) out[i * P + c] = o[i];
        }
    }
}

// Row-marching stage of the df64 state with two columns per thread.  Thread t of
// block b owns the columns x0 = 2 (b blockDim + t) and x1 = x0 + 1 (x1 = x0 for an
// odd last column, computed twice and stored once) and applies every operation of
// stage_march_kernel<float, kBase, true> to both cells at once with the packed
// FP32x2 instructions: lane by lane the same IEEE operations, so each cell gets the
// bits of the one-column kernel, with about half the instruction issues for the
// arithmetic, which bounds that kernel.  kVec: nx is even, so the pair (x0, x1) of a
// row is 8-byte aligned and moves as one float2.
// The rows a thread needs next are copied ahead into shared memory with cp.async
// (no registers held while they are in flight): at row y the thread stages row y+1,
// which its y transport reads after the equilibrium and which is the state of the
// next row.  Each thread copies and reads only its own two columns, so the copies
// need the thread's own wait only, no block barrier.
#ifndef CDBM_MARCH2_MIN_BLOCKS
#define CDBM_MARCH2_MIN_BLOCKS 3
#endif
constexpr int kMarch2MinBlocks = CDBM_MARCH2_MIN_BLOCKS;
// Rows staged ahead by cp.async: two buffers of [kNV][kStageThreads] float2.
constexpr size_t kMarch2StageBytes = 2 * kNV * kStageThreads * sizeof(float2);

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void *gmem)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <bool kBase, bool kVec, int kEq>
__global__ void __launch_bounds__(kStageThreads, kMarch2MinBlocks)
    stage_march2_kernel(const float *__restrict__ g, const float *base, float *out, const StageArgs a,
                        unsigned *flag)
{
    __shared__ float2 carry_u[kNY][kStageThreads];
    __shared__ float2 carry_n[kNY][kStageThreads];
    extern __shared__ __align__(16) float2 staged[];  // [2][kNV][kStageThreads]
    const int nx = a.nx, ny = a.ny;
    const int tid = threadIdx.x;
    const int x0 = 2 * (int)(blockIdx.x * blockDim.x + tid);
    if (x0 >= nx) return;                             // no block barriers below
    const bool two = x0 + 1 < nx;
    const int x1 = two ? x0 + 1 : x0;
    const int R = (ny + gridDim.y - 1) / gridDim.y;
    const int y0 = blockIdx.y * R;
    const int y1 = y0 + R < ny ? y0 + R : ny;
    if (y0 >= y1) return;
    const size_t P = (size_t)nx * ny;
    const int m2a = neighbour(x0 - 2, nx, a.bc_x), m1a = neighbour(x0 - 1, nx, a.bc_x);
    const int p1a = neighbour(x0 + 1, nx, a.bc_x), p2a = neighbour(x0 + 2, nx, a.bc_x);
    const int m2b = neighbour(x1 - 2, nx, a.bc_x), m1b = neighbour(x1 - 1, nx, a.bc_x);
    const int p1b = neighbour(x1 + 1, nx, a.bc_x), p2b = neighbour(x1 + 2, nx, a.bc_x);
    const float2 half2 = make_float2(0.5f, 0.5f);
    // the two cells of a row, and an arbitrary pair of columns of a row
    auto ld = [&](const float *p) -> float2 {
        if constexpr (kVec) return __ldg(reinterpret_cast<const float2 *>(p + x0));
        else return make_float2(__ldg(p + x0), __ldg(p + x1));
    };
    auto ld_at = [&](const float *p, int ca, int cb) -> float2 { return make_float2(__ldg(p + ca), __ldg(p + cb)); };
    // The x neighbours of the pair outside it are (x0 - 2, x0 - 1) and (x0 + 2, x0 + 3).
    // With nx even each of those is an aligned pair of one row wherever the boundary
    // maps it onto two neighbouring columns (always for periodic edges), and moves as
    // one 8-byte load; otherwise (a clamped edge) as two 4-byte loads.
    const bool pairL = kVec && m1a == m2a + 1 && (m2a & 1) == 0;
    const bool pairR = kVec && p2b == p2a + 1 && (p2a & 1) == 0;
    auto ld_left = [&](const float *p) -> float2 {
        return pairL ? __ldg(reinterpret_cast<const float2 *>(p + m2a)) : make_float2(__ldg(p + m2a), __ldg(p + m1a));
    };
    auto ld_right = [&](const float *p) -> float2 {
        return pairR ? __ldg(reinterpret_cast<const float2 *>(p + p2a)) : make_float2(__ldg(p + p2a), __ldg(p + p2b));
    };
    auto stage_row = [&](int b, size_t row) {       // the thread's two cells of a row, all planes
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            float2 *dst = staged + (b * kNV + i) * kStageThreads + tid;
            const float *src = g + i * P + row;
            if constexpr (kVec) {
                cp_async8(dst, src + x0);
            } else {
                cp_async4(&dst->x, src + x0);
                cp_async4(&dst->y, src + x1);
            }
        }
        cp_async_commit();
    };
    auto staged_at = [&](int b, int i) -> float2 { return staged[(b * kNV + i) * kStageThreads + tid]; };

    // prologue: U_{y0} and N_{y0 - 1} for s = +1, N_{y0} for s = -1
    {
        const size_t r0 = (size_t)y0 * nx;
        const size_t rm1 = (size_t)neighbour(y0 - 1, ny, a.bc_y) * nx;
        const size_t rm2 = (size_t)neighbour(y0 - 2, ny, a.bc_y) * nx;
        const size_t rp1 = (size_t)neighbour(y0 + 1, ny, a.bc_y) * nx;
#pragma unroll
        for (int k = 0; k < kNY; ++k) {
            const int i = yvel(k);
            const float *gp = g + i * P;
            const float2 f0 = ld(gp + r0), fm1 = ld(gp + rm1);
            if (diry(i) > 0) {
                const float2 u = sub_rn(f0, fm1);
                const float2 um = sub_rn(fm1, ld(gp + rm2));
                carry_u[k][tid] = u;
                carry_n[k][tid] = minmod(u, um);
            } else {
                const float2 u = sub_rn(f0, ld(gp + rp1));
                const float2 um = sub_rn(fm1, f0);
                carry_u[k][tid] = u;
                carry_n[k][tid] = minmod(um, u);
            }
        }
    }

    stage_row(0, (size_t)y0 * nx);
    for (int y = y0, b = 0; y < y1; ++y, b ^= 1) {
        const size_t row = (size_t)y * nx;
        const size_t rp1 = (size_t)neighbour(y + 1, ny, a.bc_y) * nx;
        const size_t rp2 = (size_t)neighbour(y + 2, ny, a.bc_y) * nx;
        // With the deviation equilibrium the kernel is bound by load latency. So
        // row y+2 and, in the second stage, the next base row are prefetched into L2
        // without holding registers. Row y+2 is what the downward velocities read in
        // this row and what the next row stages. On the 4096^2 vortex this took the
        // step from 1.34-1.40 to 1.09-1.17 ms (the range over GPUs). The df64
        // kernel, at its register limit, did not gain.
        if constexpr (kEq == kEqF32) {
#pragma unroll
            for (int i = 0; i < kNV; ++i) prefetch_l2(g + i * P + rp2 + x0);
            if (kBase && y + 1 < y1) {
#pragma unroll
                for (int i = 0; i < kNV; ++i) prefetch_l2(base + i * P + row + nx + x0);
            }
        }
        stage_row(b ^ 1, rp1);                        // row y+1 while this one computes
        cp_async_wait<1>();                           // row y, staged one row earlier
        float2 fs[kNV], o[kNV], heq[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) fs[i] = staged_at(b, i);
        // The deviation equilibrium leaves registers free: its x neighbour pairs are
        // loaded before it, so that their latency overlaps its arithmetic (1.37 ->
        // 1.34 ms per 4096^2 step; the df64 equilibrium has no registers to spare).
        constexpr bool kEarlyX = kVec && kEq == kEqF32;
        float2 nl[kNV], nr[kNV];
        if constexpr (kEarlyX) {
#pragma unroll
            for (int i = 0; i < kNV; ++i) {
                if (dirx(i) != 0) {
                    nl[i] = ld_left(g + i * P + row);
                    nr[i] = ld_right(g + i * P + row);
                }
            }
        }
        if constexpr (kEq == kEqF32) {
            // one column at a time (see cdbm_f32dev.cuh)
            float fa[kNV], fb[kNV], ha[kNV], hb[kNV];
#pragma unroll
            for (int i = 0; i < kNV; ++i) {
                fa[i] = fs[i].x;
                fb[i] = fs[i].y;
            }
            f32_equilibrium(a.d.b, a.d.m, a.d.r, a.dp, fa, ha, flag);
            f32_equilibrium(a.d.b, a.d.m, a.d.r, a.dp, fb, hb, flag);
#pragma unroll
            for (int i = 0; i < kNV; ++i) heq[i] = make_float2(ha[i], hb[i]);
        } else {
            df_equilibrium(a.d2.b, a.d2.m, a.d2.r, fs, heq, flag);
        }
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            o[i] = fma_rn(a.a_self_f2, fs[i], heq[i]);
            if (kBase) o[i] = fma_rn(a.a_base_f2, ld(base + i * P + row), o[i]);
            if (dirx(i) != 0) {
                const float *gp = g + i * P + row;
                const bool pos = dirx(i) > 0;
                float2 u2, u1, d1;
                if constexpr (kVec) {
                    // the pair's own cells stand in for the neighbours inside the pair
                    float2 L, Rr;
                    if constexpr (kEarlyX) {
                        L = nl[i];
                        Rr = nr[i];
                    } else {
                        L = ld_left(gp);
                        Rr = ld_right(gp);
                    }
                    u2 = pos ? L : Rr;
                    u1 = pos ? make_float2(L.y, fs[i].x) : make_float2(fs[i].y, Rr.x);
                    d1 = pos ? make_float2(fs[i].y, Rr.x) : make_float2(L.y, fs[i].x);
                } else {
                    u2 = pos ? ld_at(gp, m2a, m2b) : ld_at(gp, p2a, p2b);
                    u1 = pos ? ld_at(gp, m1a, m1b) : ld_at(gp, p1a, p1b);
                    d1 = pos ? ld_at(gp, p1a, p1b) : ld_at(gp, m1a, m1b);
                }
                const float2 av = sub_rn(fs[i], u1);
                const float2 bv = sub_rn(d1, fs[i]);
                const float2 ev = sub_rn(u1, u2);
                const float2 t = sub_rn(minmod(bv, av), minmod(av, ev));
                o[i] = fma_rn(neg(a.lx_f2[i >> 2]), fma_rn(half2, t, av), o[i]);
            }
        }
        cp_async_wait<0>();                           // row y+1
#pragma unroll
        for (int k = 0; k < kNY; ++k) {
            const int i = yvel(k);
            const float *gp = g + i * P;
            const float2 u = carry_u[k][tid];
            const float2 n = carry_n[k][tid];
            float2 t;
            if (diry(i) > 0) {
                const float2 un = sub_rn(staged_at(b ^ 1, i), fs[i]);       // U_{y+1}
                const float2 nn = minmod(un, u);                            // N_y
                t = sub_rn(nn, n);
                carry_u[k][tid] = un;
                carry_n[k][tid] = nn;
            } else {
                const float2 un = sub_rn(staged_at(b ^ 1, i), ld(gp + rp2)); // U_{y+1}
                const float2 nn = minmod(u, un);                            // N_{y+1}
                t = sub_rn(n, nn);
                carry_u[k][tid] = un;
                carry_n[k][tid] = nn;
            }
            o[i] = fma_rn(neg(a.ly_f2[i >> 2]), fma_rn(half2, t, u), o[i]);
        }
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            float *op = out + i * P + row;
            if constexpr (kVec) {
                *reinterpret_cast<float2 *>(op + x0) = o[i];
            } else {
                op[x0] = o[i].x;
                if (two) op[x1] = o[i].y;
            }
        }
    }
}

// ------------------------------------------------------------ macros (K3)

// Moments of the reference equilibrium F that a single-precision state stores its
// deviation g = f - F from: F_g on the four members of group g, so F carries no
// momentum and no odd moment.  The moments are linear in f, so the kernels take the
// moments of g (each value widened exactly) and add these; zero for FP64.
struct RefMoments {
    double rho, E;     // sum F, sum F (v^2 + eta^2)
    double Rxx, Rwxx;  // sum F v_x^2 (= sum F v_y^2), sum F (v^2 + eta^2) v_x^2 (= ... v_y^2)
};

RefMoments ref_moments(const FieldArgs &a, bool single)
{
    RefMoments r{0.0, 0.0, 0.0, 0.0};
    if (!single) return r;
    for (int g = 0; g < 4; ++g) {
        const double s0 = 4.0 * a.Fg[g];
        const double ex = (g & 1) == 0 ? 2.0 * a.Fg[g] : s0;    // members with v_x != 0
        const double c2 = a.m.c[g] * a.m.c[g];
        r.rho += s0;
        r.E += a.m.w[g] * s0;
        r.Rxx += c2 * ex;
        r.Rwxx += a.m.w[g] * c2 * ex;
    }
    return r;
}

// The value stored for velocity i as a double: f itself, or the deviation g (the
// reference moments are added afterwards).
__device__ __forceinline__ double stored(double v) { return v; }
__device__ __forceinline__ double stored(float v) { return widen_f32(v); }

template <typename TS>
__global__ void __launch_bounds__(128) macros_kernel(const FieldArgs a, const RefMoments F, const TS *__restrict__ f,
                                                      double *rho, double *ux, double *uy, double *T)
{
    const size_t P = (size_t)a.nx * a.ny;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < P;
         c += (size_t)gridDim.x * blockDim.x) {
        double fc[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) fc[i] = stored(f[i * P + c]);
        Cons q = conserved(fc, a.m);
        if constexpr (kSingle<TS>) {
            q.rho += F.rho;
            q.E += F.E;
        }
        const double r = rcp64(q.rho);
        const double u = q.jx * r, v = q.jy * r;
        const double ru2 = fma(q.jx, u, q.jy * v);
        if (rho) rho[c] = q.rho;
        if (ux) ux[c] = u;
        if (uy) uy[c] = v;
        if (T) T[c] = (q.E - ru2) * a.m.invK * r;
    }
}

// ------------------------------------------------------------ TNE (K4)

// Powers of the group speed component c_g (v = (+-c_g, 0), (0, +-c_g) on the axis
// groups, (+-c_g, +-c_g) on the diagonal ones) and of W_g = |v|^2 + eta_g^2.
struct TneConsts {
    double c[4], c2[4], c3[4], W[4], Wc[4], Wc2[4];
};

// Rows 5..16 of M(u) (Eq. 6) applied to f - f_eq: Delta* of Eqs. (8)-(11).  f_eq is
// defined by M(u) f_eq = fbar, the prescribed central moments of Eq. (7), so Delta*
// is the central moments of f about u minus rows 5..16 of fbar, whose only nonzero
// entries are rho T (xx, yy of the second order) and (K + 2) rho T^2 (xx, yy of the
// fourth).  The central moments follow from the raw moments R_k = sum_i f_i row_k(v_i)
// by the binomial expansion of (v - u) with j = rho u; the raw moments of a group
// come from its members' sum, x and y differences, the x and y pair sums (axis
// groups) and the xy parity (diagonal groups).
template <typename TS>
__global__ void __launch_bounds__(128) tne_kernel(const FieldArgs a, const TneConsts t, const RefMoments F,
                                                   const TS *__restrict__ f, double *__restrict__ out)
{
    const size_t P = (size_t)a.nx * a.ny;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < P;
         c += (size_t)gridDim.x * blockDim.x) {
        double fc[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) fc[i] = stored(f[i * P + c]);
        // group components: s0 sum, sx / sy odd in x / y, ex / ey the x / y pairs
        // (axis), sxy odd in x and y (diagonal)
        double s0[4], sx[4], sy[4], ex[2], ey[2], sxy[2];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const double *q = fc + 4 * g;
            if ((g & 1) == 0) {          // E N W S
                ex[g >> 1] = q[0] + q[2];
                ey[g >> 1] = q[1] + q[3];
                sx[g] = q[0] - q[2];
                sy[g] = q[1] - q[3];
                s0[g] = ex[g >> 1] + ey[g >> 1];
            } else {                     // NE NW SW SE
                const double e = q[0] + q[3], w = q[1] + q[2];
                sx[g] = e - w;
                sy[g] = (q[0] + q[1]) - (q[2] + q[3]);
                sxy[g >> 1] = (q[0] + q[2]) - (q[1] + q[3]);
                s0[g] = e + w;
            }
        }
        auto dot = [](const double *k, const double *x) {
            return fma(k[3], x[3], fma(k[2], x[2], fma(k[1], x[1], k[0] * x[0])));
        };
        // raw moments R1..R16 (rows of Eq. 6 at u = 0)
        double rho = (s0[0] + s0[1]) + (s0[2] + s0[3]);
        const double jx = dot(t.c, sx), jy = dot(t.c, sy);
        double E = dot(t.W, s0);
        double Rxx = fma(t.c2[3], s0[3], fma(t.c2[2], ex[1], fma(t.c2[1], s0[1], t.c2[0] * ex[0])));
        double Ryy = fma(t.c2[3], s0[3], fma(t.c2[2], ey[1], fma(t.c2[1], s0[1], t.c2[0] * ey[0])));
        const double Rxy = fma(t.c2[3], sxy[1], t.c2[1] * sxy[0]);
        const double Rwx = dot(t.Wc, sx), Rwy = dot(t.Wc, sy);
        const double Rxxx = dot(t.c3, sx), Ryyy = dot(t.c3, sy);
        const double Rxxy = fma(t.c3[3], sy[3], t.c3[1] * sy[1]);
        const double Rxyy = fma(t.c3[3], sx[3], t.c3[1] * sx[1]);
        double Rwxx = fma(t.Wc2[3], s0[3], fma(t.Wc2[2], ex[1], fma(t.Wc2[1], s0[1], t.Wc2[0] * ex[0])));
        double Rwyy = fma(t.Wc2[3], s0[3], fma(t.Wc2[2], ey[1], fma(t.Wc2[1], s0[1], t.Wc2[0] * ey[0])));
        const double Rwxy = fma(t.Wc2[3], sxy[1], t.Wc2[1] * sxy[0]);
        if constexpr (kSingle<TS>) {    // the reference equilibrium's even moments
            rho += F.rho;
            E += F.E;
            Rxx += F.Rxx;
            Ryy += F.Rxx;
            Rwxx += F.Rwxx;
            Rwyy += F.Rwxx;
        }
        // primitives: u = j / rho, p = rho T = (E - rho u^2) / K
        const double r = rcp64(rho);
        const double ux = jx * r, uy = jy * r;
        const double uxuy = ux * uy, u2 = fma(ux, ux, uy * uy);
        const double p = (E - fma(jx, ux, jy * uy)) * a.m.invK;
        const double q4 = a.m.Kp2 * p * (p * r);                 // (K + 2) rho T^2
        const double ax = fma(uy, Rxy, ux * Rxx);                // sum f (v.u) v_x
        const double ay = fma(uy, Ryy, ux * Rxy);                // sum f (v.u) v_y
        // central moments about u, minus fbar
        const double Cxx = fma(-ux, jx, Rxx), Cxy = fma(-ux, jy, Rxy), Cyy = fma(-uy, jy, Ryy);
        const double d[12] = {
            Cxx - p,
            Cxy,
            Cyy - p,
            fma(2.0 * u2, jx, fma(-2.0, ax, fma(-ux, E, Rwx))),
            fma(2.0 * u2, jy, fma(-2.0, ay, fma(-uy, E, Rwy))),
            fma(2.0 * jx, ux * ux, fma(-3.0 * ux, Rxx, Rxxx)),
            fma(2.0 * jx, uxuy, fma(-2.0 * ux, Rxy, fma(-uy, Rxx, Rxxy))),
            fma(2.0 * jy, uxuy, fma(-2.0 * uy, Rxy, fma(-ux, Ryy, Rxyy))),
            fma(2.0 * jy, uy * uy, fma(-3.0 * uy, Ryy, Ryyy)),
            fma(u2, Cxx, fma(-2.0 * jx * ux, u2, fma(4.0 * ux, ax, fma(-2.0, fma(uy, Rxxy, ux * Rxxx),
                fma(ux * ux, E, fma(-2.0 * ux, Rwx, Rwxx)))))) - q4,
            fma(u2, Cxy, fma(-2.0, fma(jx * uy, u2, fma(-ux, ay, fma(-uy, ax, fma(uy, Rxyy, ux * Rxxy)))),
                fma(uxuy, E, fma(-ux, Rwy, fma(-uy, Rwx, Rwxy))))),
            fma(u2, Cyy, fma(-2.0 * jy * uy, u2, fma(4.0 * uy, ay, fma(-2.0, fma(uy, Ryyy, ux * Rxyy),
                fma(uy * uy, E, fma(-2.0 * uy, Rwy, Rwyy)))))) - q4,
        };
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k * P + c] = d[k];
    }
}

// ------------------------------------------------------------ sums (K5)

constexpr int kSumThreads = 256;

// The conserved totals are sums over the 16 velocity planes, each weighted by a
// constant of its velocity (1, v_x, v_y, |v|^2 + eta^2), so the cells are reduced
// plane by plane (one FP64 addition per value) and the weights are applied to the
// 16 plane totals at the end.  Block b reduces cells [b*chunk, (b+1)*chunk) in a
// fixed order and writes its 16 plane sums; the order depends only on the grid size
// and nblocks.  A single-precision state adds its stored deviations g (widened
// exactly), and the reference equilibrium's share, cells x F_g, is added to the
// plane totals.
template <typename TS>
__global__ void __launch_bounds__(kSumThreads) sums_partial_kernel(const FieldArgs a,
                                                                   const TS *__restrict__ f,
                                                                   double *__restrict__ partials)
{
    __shared__ double sh[kNV][kSumThreads / 32];
    const size_t P = (size_t)a.nx * a.ny;
    const size_t chunk = (P + gridDim.x - 1) / gridDim.x;
    const size_t lo = blockIdx.x * chunk;
    const size_t hi = lo + chunk < P ? lo + chunk : P;
    double s[kNV];
#pragma unroll
    for (int i = 0; i < kNV; ++i) s[i] = 0.0;
    for (size_t c = lo + threadIdx.x; c < hi; c += kSumThreads) {
        // A single-precision value is widened by the conversion instruction (at the
        // FP64 pipe's rate) for half the planes and on the integer pipe for the
        // other half, which keeps both units about equally busy.
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            const TS v = f[i * P + c];
            s[i] += i < kNV / 2 ? (double)v : stored(v);
        }
    }
    // warp tree (fixed lane order), then the warps' sums in warp order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kNV; ++i) {
        double v = s[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNV) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kSumThreads / 32; ++w) v += sh[threadIdx.x][w];
        partials[blockIdx.x * kNV + threadIdx.x] = v;
    }
}

// Plane totals in block order, then rho, j_x, j_y and E from them (velocity order).
__global__ void sums_final_kernel(const FieldArgs a, const double *__restrict__ partials, int nblocks,
                                  bool single, double *out4)
{
    __shared__ double tot[kNV];
    if (threadIdx.x < kNV) {
        const int i = threadIdx.x;
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partials[b * kNV + i];
        if (single) v = fma((double)a.nx * (double)a.ny, a.Fg[i >> 2], v);
        tot[i] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < kNV; ++i) {
            r[0] += tot[i];
            r[1] = fma(a.vx[i], tot[i], r[1]);
            r[2] = fma(a.vy[i], tot[i], r[2]);
            r[3] = fma(fma(a.vx[i], a.vx[i], fma(a.vy[i], a.vy[i], a.eta[i] * a.eta[i])), tot[i], r[3]);
        }
        for (int k = 0; k < 4; ++k) out4[k] = r[k];
    }
}

// ------------------------------------------------------------ conversion

// FP32-bulk deviation g <-> f = F + g for a whole [16][plane] field.
__global__ void __launch_bounds__(256) widen_kernel(const FieldArgs a, const float *__restrict__ in,
                                                     double *__restrict__ out, size_t plane)
{
    const size_t n = kNV * plane;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        out[k] = a.Fg[(int)(k / plane) >> 2] + (double)in[k];
}

__global__ void __launch_bounds__(256) narrow_kernel(const FieldArgs a, const double *__restrict__ in,
                                                      float *__restrict__ out, size_t plane)
{
    const size_t n = kNV * plane;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        out[k] = (float)(in[k] - a.Fg[(int)(k / plane) >> 2]);
}

// Block partial sums of rho and T (fixed order), then one block adds the partials.
__global__ void __launch_bounds__(kSumThreads) means_partial_kernel(const double *__restrict__ rho,
                                                                    const double *__restrict__ T, size_t n,
                                                                    double *__restrict__ partials)
{
    __shared__ double sh[2][kSumThreads];
    const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const size_t lo = blockIdx.x * chunk;
    const size_t hi = lo + chunk < n ? lo + chunk : n;
    double s0 = 0.0, s1 = 0.0;
    for (size_t c = lo + threadIdx.x; c < hi; c += kSumThreads) {
        s0 += rho[c];
        s1 += T[c];
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    __syncthreads();
    for (int w = kSumThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 2) partials[blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void means_final_kernel(const double *__restrict__ partials, int nblocks, double *out2)
{
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[b * 4 + threadIdx.x];
        out2[threadIdx.x] = s;
    }
}

unsigned grid_for(size_t cells, int threads)
{
    size_t b = (cells + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > 1048576 ? 1048576 : b));
}

template <int kEq>
void *stage_march2_func_t(bool with_base, bool vec)
{
    if (with_base)
        return vec ? (void *)stage_march2_kernel<true, true, kEq> : (void *)stage_march2_kernel<true, false, kEq>;
    return vec ? (void *)stage_march2_kernel<false, true, kEq> : (void *)stage_march2_kernel<false, false, kEq>;
}

void *stage_march2_func(bool with_base, bool vec, bool dev)
{
    return dev ? stage_march2_func_t<kEqF32>(with_base, vec) : stage_march2_func_t<kEqDF>(with_base, vec);
}

template <typename TS, int kEq>
void *stage_func(bool march, bool with_base, bool flat)
{
    if constexpr (kEq == kEqDouble) {   // the single-precision equilibria march with stage_march2_kernel
        if (march)
            return with_base ? (void *)stage_march_kernel<TS, true, kEq> : (void *)stage_march_kernel<TS, false, kEq>;
    }
    if (with_base)
        return flat ? (void *)stage_kernel<TS, true, true, kEq> : (void *)stage_kernel<TS, true, false, kEq>;
    return flat ? (void *)stage_kernel<TS, false, true, kEq> : (void *)stage_kernel<TS, false, false, kEq>;
}

}  // namespace

cudaError_t launch_init(const FieldArgs &a, const double *rho, const double *ux, const double *uy,
                        const double *T, void *f, int prec, unsigned *flag, cudaStream_t s)
{
    const unsigned nb = grid_for((size_t)a.nx * a.ny, 128);
    if (single_storage(prec))
        init_kernel<float><<<nb, 128, 0, s>>>(a, rho, ux, uy, T, (float *)f, flag);
    else
        init_kernel<double><<<nb, 128, 0, s>>>(a, rho, ux, uy, T, (double *)f, flag);
    return cudaGetLastError();
}

cudaError_t launch_macros(const FieldArgs &a, const void *f, int prec, double *rho, double *ux,
                          double *uy, double *T, cudaStream_t s)
{
    const unsigned nb = grid_for((size_t)a.nx * a.ny, 128);
    const RefMoments F = ref_moments(a, single_storage(prec));
    if (single_storage(prec))
        macros_kernel<float><<<nb, 128, 0, s>>>(a, F, (const float *)f, rho, ux, uy, T);
    else
        macros_kernel<double><<<nb, 128, 0, s>>>(a, F, (const double *)f, rho, ux, uy, T);
    return cudaGetLastError();
}

cudaError_t launch_tne(const FieldArgs &a, const void *f, int prec, double *out, cudaStream_t s)
{
    TneConsts t;
    for (int g = 0; g < 4; ++g) {
        t.c[g] = a.m.c[g];
        t.c2[g] = a.m.c[g] * a.m.c[g];
        t.c3[g] = t.c2[g] * a.m.c[g];
        t.W[g] = a.m.w[g];
        t.Wc[g] = a.m.w[g] * a.m.c[g];
        t.Wc2[g] = a.m.w[g] * t.c2[g];
    }
    const unsigned nb = grid_for((size_t)a.nx * a.ny, 128);
    const RefMoments F = ref_moments(a, single_storage(prec));
    if (single_storage(prec))
        tne_kernel<float><<<nb, 128, 0, s>>>(a, t, F, (const float *)f, out);
    else
        tne_kernel<double><<<nb, 128, 0, s>>>(a, t, F, (const double *)f, out);
    return cudaGetLastError();
}

cudaError_t launch_sums(const FieldArgs &a, const void *f, int prec, double *partials, int nblocks,
                        double *out4, cudaStream_t s)
{
    if (single_storage(prec))
        sums_partial_kernel<float><<<nblocks, kSumThreads, 0, s>>>(a, (const float *)f, partials);
    else
        sums_partial_kernel<double><<<nblocks, kSumThreads, 0, s>>>(a, (const double *)f, partials);
    sums_final_kernel<<<1, 32, 0, s>>>(a, partials, nblocks, single_storage(prec), out4);
    return cudaGetLastError();
}

cudaError_t launch_convert(const FieldArgs &a, const void *src, int src_prec, void *dst, int dst_prec,
                           cudaStream_t s)
{
    const size_t plane = (size_t)a.nx * a.ny;
    const unsigned nb = grid_for(kNV * plane, 256);
    const bool si = single_storage(src_prec), so = single_storage(dst_prec);
    if (si && !so)
        widen_kernel<<<nb, 256, 0, s>>>(a, (const float *)src, (double *)dst, plane);
    else if (!si && so)
        narrow_kernel<<<nb, 256, 0, s>>>(a, (const double *)src, (float *)dst, plane);
    else
        return cudaMemcpyAsync(dst, src, kNV * plane * storage_bytes(src_prec), cudaMemcpyDefault, s);
    return cudaGetLastError();
}

cudaError_t launch_field_means(const double *rho, const double *T, size_t n, double *partials,
                               int nblocks, double *out2, cudaStream_t s)
{
    means_partial_kernel<<<nblocks, kSumThreads, 0, s>>>(rho, T, n, partials);
    means_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, out2);
    return cudaGetLastError();
}

StageLaunch stage_launch_config(const StageArgs &a, bool with_base, int sm_count, int prec, bool allow_march,
                                bool allow_split)
{
    StageLaunch L;
    const bool flat = (a.ny == 1);
    const size_t cells = (size_t)a.nx * a.ny;
    if (allow_split && flat && prec == CDBM_FP64 && a.nx <= kSplitFlatMaxCells) {
        // short FP64 tubes: four threads per cell shorten the dependent chain of a stage
        L.func = split_flat_func(with_base);
        L.block = dim3(kSplitFlatThreads, 1, 1);
        L.grid = dim3((unsigned)((4 * (size_t)a.nx + kSplitFlatThreads - 1) / kSplitFlatThreads), 1, 1);
        return L;
    }
    // The df64 and single-precision deviation equilibria march two columns per thread
    // (stage_march2_kernel).
    const bool pair = prec == CDBM_FP32_DF64 || prec == CDBM_FP32_DEV;
    const int cols = pair ? 2 * kStageThreads : kStageThreads;
    const unsigned xblocks = (unsigned)((a.nx + cols - 1) / cols);
    // Row-marching kernel when runs of at least 8 rows still give two full waves of
    // blocks; runs grow to 32 rows while at least 8 waves remain.  On smaller grids
    // (a 512^2 sound wave has 4 blocks across) runs of 4 or 2 rows are used if they
    // give two waves: each run repeats a 2-row prologue, but the x and y differences
    // are still computed once per cell.
    const size_t wave = (size_t)sm_count * (pair ? kMarch2MinBlocks : stage_min_blocks(kEqDouble));
    int R = 8;
    while (R < 32 && (size_t)xblocks * ((a.ny + 2 * R - 1) / (2 * R)) >= 8 * wave) R *= 2;
    bool march = allow_march && !flat && a.ny >= 16 && (size_t)xblocks * ((a.ny + 7) / 8) >= 2 * wave;
    for (int r = 4; allow_march && !march && !flat && a.ny >= 16 && r >= 2; r /= 2) {
        if ((size_t)xblocks * ((a.ny + r - 1) / r) >= 2 * wave) {
            march = true;
            R = r;
        }
    }
    if (march) {
        L.func = pair ? stage_march2_func(with_base, (a.nx & 1) == 0, prec == CDBM_FP32_DEV)
                 : prec == CDBM_FP32_BULK ? stage_func<float, kEqDouble>(true, with_base, false)
                                          : stage_func<double, kEqDouble>(true, with_base, false);
        if (prec == CDBM_FP64) {
            // the double-buffered x row buffer of stage_march_kernel<double>
            L.smem = kMarchRowBytes;
            if (cudaFuncSetAttribute(L.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem) !=
                cudaSuccess)
                cudaGetLastError();   // the launch then reports the error
        }
        if (pair) {
            // rows staged by cp.async: dynamic shared memory beside the static carries
            L.smem = kMarch2StageBytes;
            if (cudaFuncSetAttribute(L.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem) !=
                cudaSuccess)
                cudaGetLastError();   // the launch then reports the error
        }
        L.block = dim3(kStageThreads, 1, 1);
        const unsigned yblocks = (unsigned)((a.ny + R - 1) / R);
        L.grid = dim3(xblocks, yblocks < 65535 ? yblocks : 65535, 1);
        return L;
    }
    L.func = prec == CDBM_FP32_DEV    ? stage_func<float, kEqF32>(false, with_base, flat)
             : prec == CDBM_FP32_DF64 ? stage_func<float, kEqDF>(false, with_base, flat)
             : prec == CDBM_FP32_BULK ? stage_func<float, kEqDouble>(false, with_base, flat)
                                      : stage_func<double, kEqDouble>(false, with_base, flat);
    // Small grids: narrower blocks so that more SMs share the cells.
    int threads = kStageThreads;
    while (threads > 32 && cells < (size_t)sm_count * threads * 2) threads >>= 1;
    L.block = dim3(threads, 1, 1);
    L.grid = dim3((a.nx + threads - 1) / threads, a.ny < 65535 ? a.ny : 65535, 1);
    return L;
}

DFBlocks df_blocks(const EqBlocks &e)
{
    DFBlocks d;
    for (int k = 0; k < 16; ++k) d.S[k] = df_from(e.S[k]);
    for (int k = 0; k < 4; ++k) {
        d.B1[k] = df_from(e.B1[k]);
        d.B2[k] = df_from(e.B2[k]);
        const double *V = e.V + 4 * k;
        d.V0[k] = df_from(V[0]);
        d.V3[k] = df_from(V[3]);
        d.Vs[k] = df_from(0.5 * (V[1] + V[2]));
        d.Vd[k] = df_from(0.5 * (V[1] - V[2]));
    }
    return d;
}

DFModel df_model(const ModelConsts &m)
{
    DFModel d;
    for (int k = 0; k < 4; ++k) {
        d.c[k] = df_from(m.c[k]);
        d.w[k] = df_from(m.w[k]);
    }
    d.invK = df_from(m.invK);
    d.Kp4 = df_from(m.Kp4);
    d.Kp6 = df_from(m.Kp6);
    d.twoKp2 = df_from(m.twoKp2);
    return d;
}

DFShift df_shift(const double sF[4], double rhoF, double EF)
{
    DFShift d;
    for (int k = 0; k < 4; ++k) d.sF[k] = df_from(sF[k]);
    d.rhoF = df_from(rhoF);
    d.EF = df_from(EF);
    return d;
}

namespace {

DFv<float2> twice(DFPair p) { return {make_float2(p.hi, p.hi), make_float2(p.lo, p.lo)}; }

template <int N>
void twice_all(const DFPair (&in)[N], DFv<float2> (&out)[N])
{
    for (int k = 0; k < N; ++k) out[k] = twice(in[k]);
}

}  // namespace

DFBlocksT<float2> df_blocks_twice(const DFBlocks &d)
{
    DFBlocksT<float2> t;
    twice_all(d.S, t.S);
    twice_all(d.B1, t.B1);
    twice_all(d.B2, t.B2);
    twice_all(d.V0, t.V0);
    twice_all(d.V3, t.V3);
    twice_all(d.Vs, t.Vs);
    twice_all(d.Vd, t.Vd);
    return t;
}

DFModelT<float2> df_model_twice(const DFModel &d)
{
    DFModelT<float2> t;
    twice_all(d.c, t.c);
    twice_all(d.w, t.w);
    t.invK = twice(d.invK);
    t.Kp4 = twice(d.Kp4);
    t.Kp6 = twice(d.Kp6);
    t.twoKp2 = twice(d.twoKp2);
    return t;
}

DFShiftT<float2> df_shift_twice(const DFShift &d)
{
    DFShiftT<float2> t;
    twice_all(d.sF, t.sF);
    t.rhoF = twice(d.rhoF);
    t.EF = twice(d.EF);
    return t;
}

void fill_df_consts(StageArgs &a)
{
    a.d.b = df_blocks(a.eq);
    a.d.m = df_model(a.m);
    a.d.r = df_shift(a.sF, a.rhoF, a.EF);
    // each value twice for the two-column kernel
    a.d2.b = df_blocks_twice(a.d.b);
    a.d2.m = df_model_twice(a.d.m);
    a.d2.r = df_shift_twice(a.d.r);
    a.a_base_f2 = make_float2(a.a_base_f, a.a_base_f);
    a.a_self_f2 = make_float2(a.a_self_f, a.a_self_f);
    for (int g = 0; g < 4; ++g) {
        a.lx_f2[g] = make_float2(a.lx_f[g], a.lx_f[g]);
        a.ly_f2[g] = make_float2(a.ly_f[g], a.ly_f[g]);
    }
}

DevProj dev_proj(const ModelConsts &m, double gh)
{
    double sw = 0.0, sw2 = 0.0, kc = 0.0;
    for (int g = 0; g < 4; ++g) {
        sw += m.w[g];
        sw2 += m.w[g] * m.w[g];
        kc += ((g & 1) == 0 ? 2.0 : 4.0) * m.c[g] * m.c[g];    // sum_i c_ix^2 over the group
    }
    const double m00 = 16.0, m01 = 4.0 * sw, m11 = 4.0 * sw2, det = m00 * m11 - m01 * m01;
    DevProj d;
    d.gh = (float)gh;
    d.a00 = (float)(m11 / det);
    d.a01 = (float)(-m01 / det);
    d.a11 = (float)(m00 / det);
    d.rkc = (float)(1.0 / kc);
    return d;
}

void fill_dev_proj(StageArgs &a, double gh) { a.dp = dev_proj(a.m, gh); }

cudaError_t launch_stage(const StageLaunch &L, const void *g, const void *base, void *out,
                         const StageArgs &a, unsigned *flag, cudaStream_t s)
{
    void *args[] = {(void *)&g, (void *)&base, (void *)&out, (void *)&a, (void *)&flag};
    return cudaLaunchKernel(L.func, L.grid, L.block, args, L.smem, s);
}

}  // namespace cdbm
