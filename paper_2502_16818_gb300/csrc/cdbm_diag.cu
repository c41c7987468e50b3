// Diagnostic entry points: one device building block, or one hardware rate probe,
// run on its own.  The paper has no counterpart; they let the tests bound the
// reciprocal of the stage kernels against IEEE division, and let the benchmark
// measure the FP64 fused multiply-add rate that bounds the FP64 stage kernels on
// the same GPU and in the same process as the kernels it is compared with.
#include <cstdarg>
#include <cstdio>

#include "cdbm_device.cuh"
#include "cdbm_internal.h"

using namespace cdbm;

namespace {

constexpr int kDiagThreads = 256;

__global__ void __launch_bounds__(kDiagThreads) rcp64_kernel(const double *__restrict__ x,
                                                            double *__restrict__ y, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        y[k] = rcp64(x[k]);
}

// kChains independent chains of dependent fused multiply-adds per thread,
// x <- x m + c with 0 < m < 1 (the chains converge to c / (1 - m), so no value
// overflows or becomes subnormal).  m and c are kernel arguments, so the compiler
// cannot fold the chains.
constexpr int kChains = 8;

__global__ void fp64_fma_kernel(double *__restrict__ out, int iters, double m, double c)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * k + 1e-7 * threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

cdbm_status fail(cdbm_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(thread_error_buffer(), kThreadErrorBytes, fmt, ap);
    va_end(ap);
    return s;
}

cdbm_status launch_status(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CDBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return CDBM_OK;
}

}  // namespace

extern "C" cdbm_status cdbm_diag_rcp64(const double *x, double *y, long long n, void *cuda_stream)
{
    if (n < 0) return fail(CDBM_EINVAL, "cdbm_diag_rcp64: n < 0");
    if (n == 0) return CDBM_OK;
    if (!x || !y) return fail(CDBM_EINVAL, "cdbm_diag_rcp64: NULL pointer");
    long long blocks = (n + kDiagThreads - 1) / kDiagThreads;
    if (blocks > 65536) blocks = 65536;
    rcp64_kernel<<<(unsigned)blocks, kDiagThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(x, y, n);
    return launch_status("cdbm_diag_rcp64");
}

extern "C" cdbm_status cdbm_diag_fp64_fma(double *out, int blocks, int threads, int iters, void *cuda_stream,
                                          double *flops)
{
    if (!out) return fail(CDBM_EINVAL, "cdbm_diag_fp64_fma: NULL output");
    if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1)
        return fail(CDBM_EINVAL, "cdbm_diag_fp64_fma: need blocks >= 1, threads a multiple of 32 in "
                                 "[32, 1024], iters >= 1");
    fp64_fma_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(out, iters,
                                                                                    0.9999999, 1e-7);
    if (flops) *flops = 2.0 * kChains * (double)iters * (double)blocks * (double)threads;
    return launch_status("cdbm_diag_fp64_fma");
}
