// cdbm_step_noalloc: the Runge-Kutta time step of cdbm_step for callers that must
// not allocate device memory.
//
// Some host programs own every byte of GPU memory themselves: a coupled simulation
// that hands this library one field buffer out of its own pool and forbids any other
// allocation inside its time loop, a plug-in running under a framework that gives it
// device pointers but no allocator, or a latency-sensitive loop where a cudaMalloc
// would synchronise the device.  They cannot create a context (which allocates the
// second state buffer and its flags).  This entry point takes the caller's state
// buffer and keeps its own scratch -- the stage-1 buffer and the error flag -- in one
// file-scope device array that the library image carries, so the call allocates
// nothing.  The price is a fixed maximum grid of CDBM_NOALLOC_MAX_CELLS cells, and
// every GPU that loads the library holds that array (4 MiB) until the process exits.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "cdbm_device.cuh"
#include "cdbm_internal.h"

using namespace cdbm;

namespace {

constexpr size_t kMaxCells = CDBM_NOALLOC_MAX_CELLS;
constexpr size_t kFlagOffset = (size_t)kNV * kMaxCells;   // in doubles, 256-byte aligned
constexpr int kMaxDevices = 64;

// Stage-1 buffer [16][ny][nx] (at most kMaxCells cells) followed by one 256-byte slot
// whose first word is the error flag.  Shared by every call on a device.
static __device__ __align__(256) double g_scratch[kFlagOffset + 32];

std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices];   // device address of g_scratch per device ordinal

// Device address of g_scratch on the current device.  The host-side name g_scratch
// is only a stand-in for the device array, so the address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
cudaError_t scratch_on_current_device(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

cdbm_status fail(cdbm_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(thread_error_buffer(), kThreadErrorBytes, fmt, ap);
    va_end(ap);
    return s;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

extern "C" cdbm_status cdbm_step_noalloc(const cdbm_grid *grid, const cdbm_vset *vset, double I,
                                         double tau, double dt, double *f, int nsteps,
                                         void *cuda_stream)
{
    if (!grid || !vset || !f) return fail(CDBM_EINVAL, "cdbm_step_noalloc: NULL argument");
    if (nsteps < 0) return fail(CDBM_EINVAL, "cdbm_step_noalloc: nsteps < 0");
    if (grid->nx < 1 || grid->ny < 1)
        return fail(CDBM_EINVAL, "grid %d x %d: both sizes must be >= 1", grid->nx, grid->ny);
    const size_t cells = (size_t)grid->nx * (size_t)grid->ny;
    if (cells > kMaxCells)
        return fail(CDBM_EINVAL,
                    "cdbm_step_noalloc: grid of %zu cells exceeds its fixed scratch of %zu cells",
                    cells, kMaxCells);
    if (!finite_pos(grid->dx) || !finite_pos(grid->dy) || !finite_pos(dt) || !finite_pos(tau))
        return fail(CDBM_EINVAL, "dx, dy, dt and tau must be finite and > 0");
    if (!(std::isfinite(I) && I >= 0.0)) return fail(CDBM_EINVAL, "I must be finite and >= 0");
    if ((grid->bc_x != 0 && grid->bc_x != 1) || (grid->bc_y != 0 && grid->bc_y != 1))
        return fail(CDBM_EINVAL, "unknown boundary kind");
    for (int g = 0; g < 4; ++g)
        if (!std::isfinite(vset->v[g]) || !std::isfinite(vset->eta[g]) || vset->v[g] <= 0.0 ||
            vset->eta[g] < 0.0)
            return fail(CDBM_EINVAL, "velocity set: v must be > 0 and eta >= 0");
    if (dt / tau > 2.0)
        return fail(CDBM_EINVAL, "dt/tau = %g exceeds 2 (RK2 relaxation stability)", dt / tau);
    double cfl = 0.0;
    for (int i = 0; i < kNV; ++i) {
        const double s = vset->v[i >> 2];
        const double cx = grid->nx > 1 ? std::abs(dirx(i)) * s * dt / grid->dx : 0.0;
        const double cy = grid->ny > 1 ? std::abs(diry(i)) * s * dt / grid->dy : 0.0;
        cfl = cx + cy > cfl ? cx + cy : cfl;
    }
    if (cfl > 1.0) return fail(CDBM_EINVAL, "CFL number %g exceeds 1", cfl);

    ModelConsts mc;
    EqBlocks eq;
    double cond = 0.0;
    const char *which = "";
    if (build_blocks(*vset, I, mc, eq, &cond, &which) != CDBM_OK)
        return fail(CDBM_ESINGULAR, "moment matrix block '%s' singular (cond %g)", which, cond);

    double *scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    int dev = 0, sm_count = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CDBM_ECUDA, "cdbm_step_noalloc set-up: %s", cudaGetErrorString(e));
    }
    double *f1 = scratch;
    unsigned *flag = reinterpret_cast<unsigned *>(scratch + kFlagOffset);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    // Two-stage TVD Runge-Kutta, the same stage constants as a context would build:
    // f1 = f + dt L(f); f <- f/2 + (f1 + dt L(f1))/2.
    const double h = dt / tau;
    const double alpha[2] = {0.0, 0.5}, beta[2] = {1.0, 0.5}, gamma[2] = {1.0, 0.5};
    StageArgs a[2]{};   // fields the FP64 stage kernels do not read stay zero
    StageLaunch L[2];
    for (int s = 0; s < 2; ++s) {
        a[s].eq = scaled(eq, gamma[s] * h);
        a[s].m = mc;
        a[s].a_base = alpha[s];
        a[s].a_self = beta[s] - gamma[s] * h;
        for (int g = 0; g < 4; ++g) {
            a[s].lx[g] = gamma[s] * dt * mc.c[g] / grid->dx;
            a[s].ly[g] = gamma[s] * dt * mc.c[g] / grid->dy;
        }
        a[s].a_base_f = (float)a[s].a_base;
        a[s].a_self_f = (float)a[s].a_self;
        for (int g = 0; g < 4; ++g) {
            a[s].lx_f[g] = (float)a[s].lx[g];
            a[s].ly_f[g] = (float)a[s].ly[g];
        }
        a[s].nx = grid->nx;
        a[s].ny = grid->ny;
        a[s].bc_x = grid->bc_x;
        a[s].bc_y = grid->bc_y;
        L[s] = stage_launch_config(a[s], s == 1, sm_count, CDBM_FP64);
    }

    // The flag keeps the previous call's value: clear it first.
    e = cudaMemsetAsync(flag, 0, sizeof(unsigned), stream);
    for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
        e = launch_stage(L[0], f, nullptr, f1, a[0], flag, stream);
        if (e == cudaSuccess) e = launch_stage(L[1], f1, f, f, a[1], flag, stream);
    }
    unsigned flag_host = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&flag_host, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CDBM_ECUDA, "cdbm_step_noalloc: %s", cudaGetErrorString(e));
    }
    if (flag_host & kFlagNonPhys)
        return fail(CDBM_ENONPHYS, "cdbm_step_noalloc: non-physical state (rho <= 0, T <= 0 or non-finite)");
    return CDBM_OK;
}
