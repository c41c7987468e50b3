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
// CTAs (no software spin-wait).  The per-cell arithmetic is that of the flat stage
// kernel in the same order, so the result is the same bit for bit.
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
// - sum l D(src), the operations of stage_kernel<TS, kBase, true, kDF> per cell.  All
// stencil values (and the base) are gathered into registers before the first store,
// so the loads of the edge cells from the neighbouring CTAs overlap instead of each
// waiting behind a store the compiler cannot prove independent.
template <typename TS, bool kBase, bool kDF>
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
        stage_equilibrium<TS, kDF>(a, fs, heq, flag);
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

template <typename TS, bool kDF>
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
        cluster_stage<TS, false, kDF>(cl, s0, nullptr, s1, a0, chunk, rank, x0, len, flag);
        cl.sync();
        cluster_stage<TS, true, kDF>(cl, s1, s0, s0, a1, chunk, rank, x0, len, flag);
        cl.sync();
    }
    for (int k = threadIdx.x; k < kNV * len; k += blockDim.x) {
        const int i = k / len, lx = k - i * len;
        f[(size_t)i * nx + x0 + lx] = s0[i * chunk + lx];
    }
}

template <typename TS, bool kDF>
void *small1d_func() { return (void *)small1d_kernel<TS, kDF>; }

void *small1d_func_of(int prec)
{
    if (prec == CDBM_FP32_DF64) return small1d_func<float, true>();
    if (prec == CDBM_FP32_BULK) return small1d_func<float, false>();
    return small1d_func<double, false>();
}

}  // namespace

Small1D small1d_config(const StageArgs &a, int prec)
{
    Small1D L{};
    if (a.ny != 1 || a.nx < 1) return L;
    // Used while each CTA holds at most two warps' worth of cells (FP64) or eight
    // (single precision).  Measured per stage on 64-4096-cell tubes: single
    // precision with the df64 equilibrium 2.7-3.2 us against 4.3-5.8 us for one
    // launch per stage; FP64 9.3 us against 10.0 us, because there one warp's chain
    // of dependent FP64 instructions, not the launch, sets the time of a stage.
    const int per_cta_max = prec == CDBM_FP64 ? 64 : 256;
    const int C = (a.nx + per_cta_max - 1) / per_cta_max > kMaxCluster ? 0 : kMaxCluster;
    if (C == 0) return L;
    int cluster = a.nx < C ? a.nx : C;
    const int chunk = (a.nx + cluster - 1) / cluster;
    cluster = (a.nx + chunk - 1) / chunk;            // no empty CTAs
    const size_t smem = 2 * kNV * (size_t)chunk * storage_bytes(prec);
    int threads = ((chunk + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    void *func = small1d_func_of(prec);
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
