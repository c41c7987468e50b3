// Persistent cluster kernel for small 1-D grids (Ny = 1): a whole run of Eq. (1) in
// one launch.
//
// On a grid of a few hundred or thousand cells a stage launch does a few
// microseconds of work, and a step of two launches is bound by launch latency.
// Here one thread-block cluster of C <= 16 CTAs keeps the whole state in shared
// memory for the whole run: CTA r owns the cells [r chunk, (r + 1) chunk) of both
// stage buffers, reads the stencil halo of its edge cells from the neighbouring
// CTAs' shared memory (distributed shared memory of the cluster), and the stages
// are separated by the cluster barrier, a hardware barrier over the co-scheduled
// CTAs (no software spin-wait).  In single precision the per-cell arithmetic is
// that of the flat stage kernel in the same order, so the result is the same bit for
// bit; the df64 variant splits a cell over two threads (split_stage_df) and the FP64
// variant over four (split_stage).  The FP64 four-thread split also runs as an
// ordinary stage launch for tubes too long for one cluster (stage_split_flat_kernel).
#include <cooperative_groups.h>

#include "cdbm_stage.cuh"

namespace cg = cooperative_groups;

namespace cdbm {

namespace {

constexpr int kMaxCluster = 16;

// Value of velocity i at global cell gx (an index already mapped by neighbour())
// from the stage buffer `buf` ([16][chunk] in every CTA of the cluster).
template <typename TS>
__device__ __forceinline__ TS cluster_value(const cg::cluster_group &cl, const TS *buf, int chunk, int rank,
                                            int i, int gx)
{
    const int r = gx / chunk;
    const TS *p = r == rank ? buf : cl.map_shared_rank(buf, (unsigned)r);
    return p[i * chunk + (gx - r * chunk)];
}

// One stage over this CTA's cells: dst = a_base base + a_self src + gamma h f_eq(src)
// - sum l D(src), the operations of stage_kernel<TS, kBase, true, kEq> per cell.  All
// stencil values (and the base) are gathered into registers before the first store,
// so the loads of the edge cells from the neighbouring CTAs overlap instead of each
// waiting behind a store the compiler cannot prove independent.
template <typename TS, bool kBase, int kEq>
__device__ __forceinline__ void cluster_stage(const cg::cluster_group &cl, const TS *src, const TS *base, TS *dst,
                                              const StageArgs &a, int chunk, int rank, int x0, int len,
                                              unsigned *flag)
{
    constexpr int kNX = 12;                            // velocities with an x component
    const int nx = a.nx;
    for (int lx = threadIdx.x; lx < len; lx += blockDim.x) {
        const int gx = x0 + lx;
        TS fs[kNV], bs[kNV], up2[kNX], up1[kNX], dn1[kNX];
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            fs[i] = src[i * chunk + lx];
            if (kBase) bs[i] = base[i * chunk + lx];
        }
        if (lx >= 2 && lx + 2 < len) {                 // stencil inside this CTA, no wrap
            int k = 0;
#pragma unroll
            for (int i = 0; i < kNV; ++i) {
                if (dirx(i) == 0) continue;
                const TS *p = src + i * chunk + lx;
                up2[k] = p[dirx(i) > 0 ? -2 : 2];
                up1[k] = p[dirx(i) > 0 ? -1 : 1];
                dn1[k] = p[dirx(i) > 0 ? 1 : -1];
                ++k;
            }
        } else {
            const int xm2 = neighbour(gx - 2, nx, a.bc_x), xm1 = neighbour(gx - 1, nx, a.bc_x);
            const int xp1 = neighbour(gx + 1, nx, a.bc_x), xp2 = neighbour(gx + 2, nx, a.bc_x);
            int k = 0;
#pragma unroll
            for (int i = 0; i < kNV; ++i) {
                if (dirx(i) == 0) continue;
                up2[k] = cluster_value(cl, src, chunk, rank, i, dirx(i) > 0 ? xm2 : xp2);
                up1[k] = cluster_value(cl, src, chunk, rank, i, dirx(i) > 0 ? xm1 : xp1);
                dn1[k] = cluster_value(cl, src, chunk, rank, i, dirx(i) > 0 ? xp1 : xm1);
                ++k;
            }
        }
        TS heq[kNV];
        stage_equilibrium<TS, kEq>(a, fs, heq, flag);
        int k = 0;
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            TS o = fma_t(a_self_of<TS>(a), fs[i], heq[i]);
            if (kBase) o = fma_t(a_base_of<TS>(a), bs[i], o);
            if (dirx(i) != 0) {
                o = fma_t(-lx_of<TS>(a, i >> 2), nnd(up2[k], up1[k], fs[i], dn1[k]), o);
                ++k;
            }
            dst[i * chunk + lx] = o;
        }
    }
}

template <typename TS, int kEq>
__global__ void __launch_bounds__(256) small1d_kernel(TS *f, int nsteps, const StageArgs a0, const StageArgs a1,
                                                      unsigned *flag, int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TS *s0 = reinterpret_cast<TS *>(smem_raw);     // state f^n, [16][chunk]
    TS *s1 = s0 + kNV * chunk;                     // stage buffer
    const cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int nx = a0.nx;
    const int x0 = rank * chunk;
    const int len = nx - x0 < chunk ? (nx - x0 > 0 ? nx - x0 : 0) : chunk;
    for (int k = threadIdx.x; k < kNV * len; k += blockDim.x) {
        const int i = k / len, lx = k - i * len;
        s0[i * chunk + lx] = f[(size_t)i * nx + x0 + lx];
    }
    cl.sync();
    for (int s = 0; s < nsteps; ++s) {
        cluster_stage<TS, false, kEq>(cl, s0, nullptr, s1, a0, chunk, rank, x0, len, flag);
        cl.sync();
        cluster_stage<TS, true, kEq>(cl, s1, s0, s0, a1, chunk, rank, x0, len, flag);
        cl.sync();
    }
    for (int k = threadIdx.x; k < kNV * len; k += blockDim.x) {
        const int i = k / len, lx = k - i * len;
        f[(size_t)i * nx + x0 + lx] = s0[i * chunk + lx];
    }
}

// The arithmetic of one cell's group g in the four-thread split (the FP64 cluster
// kernel and the flat split stage kernel): from the group's four values q, its base
// values bs and x stencil values, the four updated values o.  The four threads of a
// cell are lanes 4c .. 4c + 3 of one warp.
__device__ __forceinline__ void split_cell(const StageArgs &a, int g, const double q[4], const double bs[4],
                                           const double up2[4], const double up1[4], const double dn1[4],
                                           bool with_base, bool live, unsigned *flag, double o[4])
{
    const int t = threadIdx.x;
    // group components, as conserved()
    double c0, cx, cy;
    if ((g & 1) == 0) {
        cx = q[0] - q[2];
        cy = q[1] - q[3];
        c0 = (q[0] + q[2]) + (q[1] + q[3]);
    } else {
        const double e = q[0] + q[3], w = q[1] + q[2];
        cx = e - w;
        cy = (q[0] + q[1]) - (q[2] + q[3]);
        c0 = e + w;
    }
    const int lane0 = (t & 31) & ~3;
    double S0[4], SX[4], SY[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        S0[h] = __shfl_sync(0xffffffffu, c0, lane0 + h);
        SX[h] = __shfl_sync(0xffffffffu, cx, lane0 + h);
        SY[h] = __shfl_sync(0xffffffffu, cy, lane0 + h);
    }
    const ModelConsts &m = a.m;
    Prim s;
    s.q.rho = (S0[0] + S0[1]) + (S0[2] + S0[3]);
    s.q.jx = fma(m.c[3], SX[3], fma(m.c[2], SX[2], fma(m.c[1], SX[1], m.c[0] * SX[0])));
    s.q.jy = fma(m.c[3], SY[3], fma(m.c[2], SY[2], fma(m.c[1], SY[1], m.c[0] * SY[0])));
    s.q.E = fma(m.w[3], S0[3], fma(m.w[2], S0[2], fma(m.w[1], S0[1], m.w[0] * S0[0])));
    const double r = rcp64(s.q.rho);
    s.ux = s.q.jx * r;
    s.uy = s.q.jy * r;
    s.jyuy = s.q.jy * s.uy;
    s.ru2 = fma(s.q.jx, s.ux, s.jyuy);
    s.p = (s.q.E - s.ru2) * m.invK;
    s.T = s.p * r;
    if (live && g == 0 && !(positive_finite(s.q.rho) && positive_finite(s.p))) atomicOr(flag, kFlagNonPhys);
    // this group's part of equilibrium()
    const EqBlocks &B = a.eq;
    const double ux2 = s.ux * s.ux, uy2 = s.uy * s.uy, u2 = ux2 + uy2, dlt = ux2 - uy2;
    const double m1416 = fma(s.T, fma(m.Kp6, s.ru2, m.twoKp2 * s.p), s.ru2 * u2);
    const double W4 = fma(m.Kp4, s.T, u2);
    const double d57 = fma(s.q.jx, s.ux, -s.jyuy);
    const double m6 = s.q.jx * s.uy;
    const double *S = B.S + 4 * g;
    const double e0 = fma(S[3], m1416, fma(S[2], s.ru2, fma(S[1], s.q.E, S[0] * s.q.rho)));
    const double qv = (g & 1) == 0 ? d57 * fma(B.B1[g + 1], W4, B.B1[g])       // g = 0: a, g = 2: c
                                   : m6 * fma(B.B2[g], W4, B.B2[g - 1]);       // g = 1: b, g = 3: d
    double heq[4];
    equilibrium_group(B, g, e0, qv, s.q.jx, s.q.jy, s.T, u2, dlt, heq);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = 4 * g + j;
        o[j] = fma(a.a_self, q[j], heq[j]);
        if (with_base) o[j] = fma(a.a_base, bs[j], o[j]);
        if (dirx(i) != 0) o[j] = fma(-a.lx[g], nnd(up2[j], up1[j], q[j], dn1[j]), o[j]);
    }
}

// FP64 variant with the work of a cell split over four threads, one per velocity
// group: thread 4c + g of the CTA handles group g of cell c.  A stage of one cell
// is a chain of dependent FP64 instructions whose latency, not throughput, bounds a
// small grid (one warp per SM); splitting the cell shortens the chain about fourfold.
// The four threads exchange their group components (s0, sx, sy) by warp shuffles and
// each forms the moments, primitive variables and the shared part of the
// equilibrium with the operations of conserved(), primitives() and equilibrium() in
// the same order; each then builds and updates its own group's four velocities.
// The compiler may fuse a multiply and an add differently than in the
// one-thread-per-cell kernels, so the two agree to rounding, not bit for bit.
__device__ __forceinline__ void split_stage(const cg::cluster_group &cl, const double *src, const double *base,
                                            double *dst, const StageArgs &a, bool with_base, int chunk, int rank,
                                            int x0, int len, unsigned *flag)
{
    const int t = threadIdx.x;
    const int g = t & 3;                              // velocity group of this thread
    const int lx0 = t >> 2;
    const bool live = lx0 < len;
    const int lx = live ? lx0 : len - 1;              // idle threads mirror the last cell
    const int gx = x0 + lx;
    const int nx = a.nx;
    double q[4], bs[4], up2[4], up1[4], dn1[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        q[j] = src[(4 * g + j) * chunk + lx];
        bs[j] = with_base ? base[(4 * g + j) * chunk + lx] : 0.0;
    }
    const bool inner = lx >= 2 && lx + 2 < len;
    const int xm2 = neighbour(gx - 2, nx, a.bc_x), xm1 = neighbour(gx - 1, nx, a.bc_x);
    const int xp1 = neighbour(gx + 1, nx, a.bc_x), xp2 = neighbour(gx + 2, nx, a.bc_x);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = 4 * g + j;
        const int sx = dirx(i);
        if (sx == 0) {
            up2[j] = up1[j] = dn1[j] = 0.0;
        } else if (inner) {
            const double *p = src + i * chunk + lx;
            up2[j] = p[sx > 0 ? -2 : 2];
            up1[j] = p[sx > 0 ? -1 : 1];
            dn1[j] = p[sx > 0 ? 1 : -1];
        } else {
            up2[j] = cluster_value(cl, src, chunk, rank, i, sx > 0 ? xm2 : xp2);
            up1[j] = cluster_value(cl, src, chunk, rank, i, sx > 0 ? xm1 : xp1);
            dn1[j] = cluster_value(cl, src, chunk, rank, i, sx > 0 ? xp1 : xm1);
        }
    }
    double o[4];
    split_cell(a, g, q, bs, up2, up1, dn1, with_base, live, flag, o);
    if (live) {
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[(4 * g + j) * chunk + lx] = o[j];
    }
}

// One FP64 stage of a 1-D grid as an ordinary launch with each cell split over four
// threads (split_cell), for tubes too long for the cluster kernel.  With one thread
// per cell a tube of a few thousand cells leaves about a warp per SM, and the chain
// of dependent FP64 instructions of one cell, not the launch, sets the time of a
// stage; four threads per cell shorten that chain.  Threads past the last cell
// mirror it (they take part in the shuffles) and store nothing.
template <bool kBase>
__global__ void __launch_bounds__(kSplitFlatThreads) stage_split_flat_kernel(const double *__restrict__ g,
                                                                             const double *base, double *out,
                                                                             const StageArgs a, unsigned *flag)
{
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int gq = t & 3;                             // velocity group of this thread
    const int x0 = t >> 2;
    const int nx = a.nx;
    const bool live = x0 < nx;
    const int x = live ? x0 : nx - 1;
    const size_t P = (size_t)nx;                      // ny = 1
    double q[4], bs[4], up2[4], up1[4], dn1[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        q[j] = g[(4 * gq + j) * P + x];
        bs[j] = kBase ? base[(4 * gq + j) * P + x] : 0.0;
    }
    const int xm2 = neighbour(x - 2, nx, a.bc_x), xm1 = neighbour(x - 1, nx, a.bc_x);
    const int xp1 = neighbour(x + 1, nx, a.bc_x), xp2 = neighbour(x + 2, nx, a.bc_x);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = 4 * gq + j;
        const int sx = dirx(i);
        const double *p = g + i * P;
        up2[j] = sx == 0 ? 0.0 : p[sx > 0 ? xm2 : xp2];
        up1[j] = sx == 0 ? 0.0 : p[sx > 0 ? xm1 : xp1];
        dn1[j] = sx == 0 ? 0.0 : p[sx > 0 ? xp1 : xm1];
    }
    double o[4];
    split_cell(a, gq, q, bs, up2, up1, dn1, kBase, live, flag, o);
    if (live) {
#pragma unroll
        for (int j = 0; j < 4; ++j) out[(4 * gq + j) * P + x] = o[j];
    }
}

__global__ void __launch_bounds__(256) small1d_split_kernel(double *f, int nsteps, const StageArgs a0,
                                                            const StageArgs a1, unsigned *flag, int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *s0 = reinterpret_cast<double *>(smem_raw);
    double *s1 = s0 + kNV * chunk;
    const cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int nx = a0.nx;
    const int x0 = rank * chunk;
    const int len = nx - x0 < chunk ? (nx - x0 > 0 ? nx - x0 : 0) : chunk;
    for (int k = threadIdx.x; k < kNV * len; k += blockDim.x) {
        const int i = k / len, lx = k - i * len;
        s0[i * chunk + lx] = f[(size_t)i * nx + x0 + lx];
    }
    cl.sync();
    for (int s = 0; s < nsteps; ++s) {
        split_stage(cl, s0, nullptr, s1, a0, false, chunk, rank, x0, len, flag);
        cl.sync();
        split_stage(cl, s1, s0, s0, a1, true, chunk, rank, x0, len, flag);
        cl.sync();
    }
    for (int k = threadIdx.x; k < kNV * len; k += blockDim.x) {
        const int i = k / len, lx = k - i * len;
        f[(size_t)i * nx + x0 + lx] = s0[i * chunk + lx];
    }
}

// df64 variant with a cell split over two threads: thread h of the pair takes the
// velocity groups 2h (axis) and 2h + 1 (diagonal), so both threads run the same
// instruction sequence.  The pair exchanges its group components by warp shuffles,
// both form the moments, primitives and raw-moment factors (df_scalars, the same
// operations), and each builds and updates only its own eight velocities.  Every
// value goes through the operations of the one-thread kernel in the same order, so
// the result is the same bit for bit; the dependent chain of a stage is about a third
// shorter, and that chain sets the time of a stage on these grids.
template <bool kBase>
__device__ __forceinline__ void split_stage_df(const cg::cluster_group &cl, const float *src, const float *base,
                                               float *dst, const StageArgs &a, int chunk, int rank, int x0, int len,
                                               unsigned *flag)
{
    const int t = threadIdx.x;
    const int h = t & 1;                              // groups 2h and 2h + 1 of the cell
    const int lx0 = t >> 1;
    const bool live = lx0 < len;
    const int lx = live ? lx0 : len - 1;              // idle threads mirror the last cell
    const int gx = x0 + lx;
    const int nx = a.nx;
    float q[8], bs[8], up2[8], up1[8], dn1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        q[j] = src[(8 * h + j) * chunk + lx];
        bs[j] = kBase ? base[(8 * h + j) * chunk + lx] : 0.0f;
    }
    const bool inner = lx >= 2 && lx + 2 < len;
    const int xm2 = neighbour(gx - 2, nx, a.bc_x), xm1 = neighbour(gx - 1, nx, a.bc_x);
    const int xp1 = neighbour(gx + 1, nx, a.bc_x), xp2 = neighbour(gx + 2, nx, a.bc_x);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = 8 * h + j;
        const int sx = dirx(j);                       // dirx depends on i mod 8 only
        if (sx == 0) {
            up2[j] = up1[j] = dn1[j] = 0.0f;
        } else if (inner) {
            const float *p = src + i * chunk + lx;
            up2[j] = p[sx > 0 ? -2 : 2];
            up1[j] = p[sx > 0 ? -1 : 1];
            dn1[j] = p[sx > 0 ? 1 : -1];
        } else {
            up2[j] = cluster_value(cl, src, chunk, rank, i, sx > 0 ? xm2 : xp2);
            up1[j] = cluster_value(cl, src, chunk, rank, i, sx > 0 ? xm1 : xp1);
            dn1[j] = cluster_value(cl, src, chunk, rank, i, sx > 0 ? xp1 : xm1);
        }
    }
    const DFConsts &D = a.d;
    df a0, ax, ay, b0, bx, by;                        // own axis group 2h, diagonal group 2h + 1
    df_group_components(0, q, a0, ax, ay);
    df_group_components(1, q + 4, b0, bx, by);
    auto other = [](float v) { return __shfl_xor_sync(0xffffffffu, v, 1); };
    const df pa0 = {other(a0.hi), other(a0.lo)}, pax = {other(ax.hi), other(ax.lo)}, pay = {other(ay.hi), other(ay.lo)};
    const df pb0 = {other(b0.hi), other(b0.lo)}, pbx = {other(bx.hi), other(bx.lo)}, pby = {other(by.hi), other(by.lo)};
    df s0[4], sx4[4], sy4[4];
    s0[0] = h ? pa0 : a0;   sx4[0] = h ? pax : ax;   sy4[0] = h ? pay : ay;
    s0[1] = h ? pb0 : b0;   sx4[1] = h ? pbx : bx;   sy4[1] = h ? pby : by;
    s0[2] = h ? a0 : pa0;   sx4[2] = h ? ax : pax;   sy4[2] = h ? ay : pay;
    s0[3] = h ? b0 : pb0;   sx4[3] = h ? bx : pbx;   sy4[3] = h ? by : pby;
    const DFScalars<float> c = df_scalars(D.m, D.r, s0, sx4, sy4, (live && h == 0) ? flag : nullptr);
    float heq[8];
    df_group_equilibrium(2 * h, D.b, D.r, c, heq);
    df_group_equilibrium(2 * h + 1, D.b, D.r, c, heq + 4);
    float o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        o[j] = fmaf(a.a_self_f, q[j], heq[j]);
        if (kBase) o[j] = fmaf(a.a_base_f, bs[j], o[j]);
        if (dirx(j) != 0) o[j] = fmaf(-a.lx_f[2 * h + (j >> 2)], nnd(up2[j], up1[j], q[j], dn1[j]), o[j]);
    }
    if (live) {
#pragma unroll
        for (int j = 0; j < 8; ++j) dst[(8 * h + j) * chunk + lx] = o[j];
    }
}

__global__ void __launch_bounds__(256) small1d_split_df_kernel(float *f, int nsteps, const StageArgs a0,
                                                               const StageArgs a1, unsigned *flag, int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s0 = reinterpret_cast<float *>(smem_raw);
    float *s1 = s0 + kNV * chunk;
    const cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int nx = a0.nx;
    const int x0 = rank * chunk;
    const int len = nx - x0 < chunk ? (nx - x0 > 0 ? nx - x0 : 0) : chunk;
    for (int k = threadIdx.x; k < kNV * len; k += blockDim.x) {
        const int i = k / len, lx = k - i * len;
        s0[i * chunk + lx] = f[(size_t)i * nx + x0 + lx];
    }
    cl.sync();
    for (int s = 0; s < nsteps; ++s) {
        split_stage_df<false>(cl, s0, nullptr, s1, a0, chunk, rank, x0, len, flag);
        cl.sync();
        split_stage_df<true>(cl, s1, s0, s0, a1, chunk, rank, x0, len, flag);
        cl.sync();
    }
    for (int k = threadIdx.x; k < kNV * len; k += blockDim.x) {
        const int i = k / len, lx = k - i * len;
        f[(size_t)i * nx + x0 + lx] = s0[i * chunk + lx];
    }
}

template <typename TS, int kEq>
void *small1d_func() { return (void *)small1d_kernel<TS, kEq>; }

constexpr int kSplitDfMaxChunk = 128;     // two threads per cell within 256 threads

void *small1d_func_of(int prec, int chunk)
{
    if (prec == CDBM_FP32_DF64)
        return chunk <= kSplitDfMaxChunk ? (void *)small1d_split_df_kernel : small1d_func<float, kEqDF>();
    if (prec == CDBM_FP32_DEV) return small1d_func<float, kEqF32>();
    if (prec == CDBM_FP32_BULK) return small1d_func<float, kEqDouble>();
    return (void *)small1d_split_kernel;
}

}  // namespace

void *split_flat_func(bool with_base)
{
    return with_base ? (void *)stage_split_flat_kernel<true> : (void *)stage_split_flat_kernel<false>;
}

Small1D small1d_config(const StageArgs &a, int prec)
{
    Small1D L{};
    if (a.ny != 1 || a.nx < 1) return L;
    // Used while each CTA holds at most two warps' worth of cells (FP64) or eight
    // (single precision).  Measured per stage on 64-4096-cell tubes: single
    // precision with the df64 equilibrium 2.7-3.2 us against 4.3-5.8 us for one
    // launch per stage; FP64 9.3 us against 10.0 us, because there one warp's chain
    // of dependent FP64 instructions, not the launch, sets the time of a stage.  With
    // 128 FP64 cells per CTA (512 threads) a 2000-cell tube took 15.6 us per stage in
    // the cluster against 10.0 us with one launch per stage on all SMs.
    const int per_cta_max = prec == CDBM_FP64 ? 64 : 256;
    const int C = (a.nx + per_cta_max - 1) / per_cta_max > kMaxCluster ? 0 : kMaxCluster;
    if (C == 0) return L;
    int cluster = a.nx < C ? a.nx : C;
    const int chunk = (a.nx + cluster - 1) / cluster;
    cluster = (a.nx + chunk - 1) / chunk;            // no empty CTAs
    const size_t smem = 2 * kNV * (size_t)chunk * storage_bytes(prec);
    // FP64: four threads per cell (split_stage), df64: two (split_stage_df, up to
    // kSplitDfMaxChunk cells), all cells of the CTA in one pass
    const int per_cell = prec == CDBM_FP64 ? 4 : (prec == CDBM_FP32_DF64 && chunk <= kSplitDfMaxChunk ? 2 : 1);
    int threads = ((per_cell * chunk + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    void *func = small1d_func_of(prec, chunk);
    if (cluster > 8 && cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return L;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, func, &cfg) != cudaSuccess || active < 1) {
        cudaGetLastError();
        return L;
    }
    L.ok = true;
    L.func = func;
    L.cluster = cluster;
    L.chunk = chunk;
    L.threads = threads;
    L.smem = smem;
    return L;
}

cudaError_t launch_small1d(const Small1D &L, void *f, int nsteps, const StageArgs &a0, const StageArgs &a1,
                           unsigned *flag, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)L.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)L.cluster, 1, 1);
    cfg.blockDim = dim3((unsigned)L.threads, 1, 1);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int chunk = L.chunk;
    void *args[] = {&f, &nsteps, (void *)&a0, (void *)&a1, &flag, &chunk};
    return cudaLaunchKernelExC(&cfg, L.func, args);
}

}  // namespace cdbm
