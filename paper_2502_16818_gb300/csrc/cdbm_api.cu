// Host side of the CDBM library: the C ABI of include/cdbm.h, validation, the
// parity-blocked inverse moment matrix, buffers and the CUDA graph of time steps.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cdbm.h"
#include "cdbm_device.cuh"
#include "cdbm_internal.h"

using namespace cdbm;

namespace {

thread_local char g_create_error[kThreadErrorBytes] = "no error";

constexpr int kGraphSteps = 32;       // time steps per replayed CUDA graph
constexpr int kSmallSteps = 65536;    // time steps per launch of the small-grid cluster kernel
constexpr double kMaxCond = 1e12;     // condition limit of the moment blocks

struct RkStage {
    double alpha, beta, gamma;        // out = alpha f^n + beta g + gamma dt L(g)
    bool with_base;
};

void rk_stages(int rk, RkStage st[2])
{
    if (rk == CDBM_RK2_MIDPOINT) {
        st[0] = {0.0, 1.0, 0.5, false};
        st[1] = {1.0, 0.0, 1.0, true};
    } else {
        st[0] = {0.0, 1.0, 1.0, false};
        st[1] = {0.5, 0.5, 0.5, true};
    }
}

}  // namespace

struct cdbm_ctx {
    cdbm_grid grid;
    cdbm_vset vset;
    double I, tau, dt;
    int precision;
    int rk;
    cudaStream_t stream;
    cdbm_allocator alloc;
    bool user_alloc;
    int device;
    int sm_count;

    size_t plane;                 // nx * ny
    void *f;                      // state [16][ny][nx] in storage precision
    void *f1;                     // stage buffer [16][ny][nx] in storage precision; also
                                  // double staging (16 planes) for host I/O and conversions
    double *partials;             // conserved-sum partials [nblocks][16] (plane sums), field means [nblocks][4]
    double *sums;                 // 4 doubles
    unsigned *flag;               // device error flags
    unsigned *flag_host;          // pinned mirror
    int sum_blocks;
    bool state_set;
    double t;

    EqBlocks eq_unit;
    ModelConsts mc;
    double Fg[4];                 // FP32-bulk reference equilibrium per group (0 for FP64)
    StageArgs stage[2];
    StageLaunch launch[2];
    RkStage rks[2];
    FieldArgs fields;

    cudaGraphExec_t graph;
    Small1D small;                // persistent cluster path for small 1-D grids
    bool small_enabled;
    bool march_enabled;       // row-marching stage kernels on 2-D grids

    // adjoint record of the last cdbm_adjoint_forward
    int adj_steps, adj_every;     // steps recorded, checkpoint interval (0: none)
    long long step_count;         // steps taken since the state was set
    long long adj_end;            // step_count at the end of the recorded run
    int adj_limiter;              // cdbm_adj_limiter of the adjoint (0: exact)
    std::vector<void *> ckpt;     // states at steps 0, k, 2k, ... of the recorded run

    cdbm_status err;
    char msg[256];
};

namespace {

cdbm_status set_err(cdbm_ctx *c, cdbm_status s, const char *fmt, ...)
{
    if (c->err != CDBM_OK) return c->err;
    c->err = s;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
    va_end(ap);
    return s;
}

cdbm_status create_err(cdbm_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_create_error, sizeof(g_create_error), fmt, ap);
    va_end(ap);
    return s;
}

cdbm_status cuda_check(cdbm_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return CDBM_OK;
    return set_err(c, CDBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *ctx_alloc(cdbm_ctx *c, size_t bytes)
{
    if (c->user_alloc) {
        void *p = c->alloc.alloc(bytes, (void *)c->stream, c->alloc.user);
        if (p && ((uintptr_t)p & 15u)) {         // the kernels move 8- and 16-byte words
            c->alloc.free(p, bytes, (void *)c->stream, c->alloc.user);
            return nullptr;
        }
        return p;
    }
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void ctx_free(cdbm_ctx *c, void *p, size_t bytes)
{
    if (!p) return;
    if (c->user_alloc)
        c->alloc.free(p, bytes, (void *)c->stream, c->alloc.user);
    else
        cudaFreeAsync(p, c->stream);
}

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace cdbm {

// In-place Gauss-Jordan inverse with partial pivoting; cond = ||A||_inf ||A^-1||_inf.
bool invert(int n, const double *A, double *Ainv, double *cond)
{
    double a[4][8];
    double anorm = 0.0;
    for (int i = 0; i < n; ++i) {
        double rs = 0.0;
        for (int j = 0; j < n; ++j) {
            a[i][j] = A[i * n + j];
            a[i][n + j] = (i == j) ? 1.0 : 0.0;
            rs += std::fabs(A[i * n + j]);
        }
        anorm = rs > anorm ? rs : anorm;
    }
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(a[i][k]) > std::fabs(a[p][k])) p = i;
        if (a[p][k] == 0.0 || !std::isfinite(a[p][k])) return false;
        if (p != k)
            for (int j = 0; j < 2 * n; ++j) std::swap(a[k][j], a[p][j]);
        const double piv = a[k][k];
        for (int j = 0; j < 2 * n; ++j) a[k][j] /= piv;
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            const double m = a[i][k];
            if (m == 0.0) continue;
            for (int j = 0; j < 2 * n; ++j) a[i][j] -= m * a[k][j];
        }
    }
    double inorm = 0.0;
    for (int i = 0; i < n; ++i) {
        double rs = 0.0;
        for (int j = 0; j < n; ++j) {
            Ainv[i * n + j] = a[i][n + j];
            rs += std::fabs(a[i][n + j]);
        }
        inorm = rs > inorm ? rs : inorm;
    }
    *cond = anorm * inorm;
    return std::isfinite(*cond);
}

// Model constants and the unscaled parity-blocked inverse of M(0) (Eq. 6 at u = 0),
// with the factors 1/4 (s0, dq, q; diagonal sx, sy) and 1/2 (axis sx, sy) that
// rebuild f_i from group components folded into the rows.
cdbm_status build_blocks(const cdbm_vset &vs, double I, ModelConsts &m, EqBlocks &eq, double *cond_out,
                         const char **which)
{
    const double K = 2.0 + I;
    double vv[4];
    for (int g = 0; g < 4; ++g) {
        const double c = vs.v[g];
        m.c[g] = c;
        vv[g] = (g & 1) ? 2.0 * c * c : c * c;
        m.w[g] = vv[g] + vs.eta[g] * vs.eta[g];
    }
    m.K = K;
    m.invK = 1.0 / K;
    m.Kp2 = K + 2.0;
    m.Kp4 = K + 4.0;
    m.Kp6 = K + 6.0;
    m.twoKp2 = 2.0 * (K + 2.0);

    double AS[16], AB1[4], AB2[4], AV[16];
    for (int g = 0; g < 4; ++g) {
        const double c = m.c[g];
        AS[0 * 4 + g] = 1.0;
        AS[1 * 4 + g] = m.w[g];
        AS[2 * 4 + g] = vv[g];
        AS[3 * 4 + g] = m.w[g] * vv[g];
        AV[0 * 4 + g] = c;
        AV[1 * 4 + g] = m.w[g] * c;
        AV[2 * 4 + g] = c * c * c;
        AV[3 * 4 + g] = (g & 1) ? c * c * c : 0.0;
    }
    const double ca = m.c[0], cc = m.c[2], cb = m.c[1], cd = m.c[3];
    AB1[0] = ca * ca;
    AB1[1] = cc * cc;
    AB1[2] = m.w[0] * ca * ca;
    AB1[3] = m.w[2] * cc * cc;
    AB2[0] = cb * cb;
    AB2[1] = cd * cd;
    AB2[2] = m.w[1] * cb * cb;
    AB2[3] = m.w[3] * cd * cd;

    double cond[4];
    double SI[16], B1I[4], B2I[4], VI[16];
    const char *names[4] = {"scalar", "axis quadrupole", "diagonal quadrupole", "vector"};
    bool ok[4] = {invert(4, AS, SI, &cond[0]), invert(2, AB1, B1I, &cond[1]),
                  invert(2, AB2, B2I, &cond[2]), invert(4, AV, VI, &cond[3])};
    double worst = 0.0;
    for (int b = 0; b < 4; ++b) {
        if (!ok[b] || cond[b] > kMaxCond) {
            *which = names[b];
            *cond_out = ok[b] ? cond[b] : INFINITY;
            return CDBM_ESINGULAR;
        }
        worst = cond[b] > worst ? cond[b] : worst;
    }
    *cond_out = worst;
    // Fold the raw Maxwellian moments into the coefficients (layout in EqBlocks):
    // m5 + m7 = (2/K) E + (1 - 2/K) rho u^2; the odd rows are j times quadratics
    // in (u_x^2, u_y^2, T); m14 - m16 and m15 are (m5 - m7) and m6 times W4.
    for (int g = 0; g < 4; ++g) {
        const double fv = (g & 1) ? 0.25 : 0.5;
        const double *s = SI + 4 * g, *v = VI + 4 * g;
        eq.S[g * 4 + 0] = 0.25 * s[0];
        eq.S[g * 4 + 1] = 0.25 * (s[1] + (2.0 / K) * s[2]);
        eq.S[g * 4 + 2] = 0.25 * (1.0 - 2.0 / K) * s[2];
        eq.S[g * 4 + 3] = 0.25 * s[3];
        eq.V[g * 4 + 0] = fv * v[0];
        eq.V[g * 4 + 1] = fv * (v[1] + v[2]);
        eq.V[g * 4 + 2] = fv * (v[1] + v[3]);
        eq.V[g * 4 + 3] = fv * ((K + 2.0) * v[1] + 3.0 * v[2] + v[3]);
        eq.Vc[g * 4 + 0] = eq.V[g * 4 + 0];
        eq.Vc[g * 4 + 1] = eq.V[g * 4 + 3];
        eq.Vc[g * 4 + 2] = 0.5 * (eq.V[g * 4 + 1] + eq.V[g * 4 + 2]);
        eq.Vc[g * 4 + 3] = 0.5 * (eq.V[g * 4 + 1] - eq.V[g * 4 + 2]);
    }
    for (int k = 0; k < 4; ++k) {
        eq.B1[k] = 0.25 * B1I[k];
        eq.B2[k] = 0.25 * B2I[k];
    }
    return CDBM_OK;
}

char *thread_error_buffer() { return g_create_error; }

EqBlocks scaled(const EqBlocks &e, double s)
{
    EqBlocks o;
    for (int k = 0; k < 16; ++k) {
        o.S[k] = s * e.S[k];
        o.V[k] = s * e.V[k];
        o.Vc[k] = s * e.Vc[k];
    }
    for (int k = 0; k < 4; ++k) {
        o.B1[k] = s * e.B1[k];
        o.B2[k] = s * e.B2[k];
    }
    return o;
}

}  // namespace cdbm

namespace {

// Reference equilibrium F = f_eq(rho0, u = 0, T0) of the FP32-bulk deviation
// storage: with u = 0 every member of group g equals the group sum times 1/4, which
// the unit scalar block gives from (rho, E = K P, rho u^2 = 0, m14+m16 = 2 (K+2) P T).
void set_reference(cdbm_ctx *c, double rho0, double T0)
{
    const double K = c->mc.K, P0 = rho0 * T0;
    for (int g = 0; g < 4; ++g) {
        const double *S = c->eq_unit.S + 4 * g;
        c->Fg[g] = (single_storage(c->precision) && std::isfinite(rho0) && std::isfinite(T0))
                       ? S[0] * rho0 + S[1] * K * P0 + S[3] * 2.0 * (K + 2.0) * P0 * T0
                       : 0.0;
        c->fields.Fg[g] = c->Fg[g];
    }
}

void build_stages(cdbm_ctx *c)
{
    rk_stages(c->rk, c->rks);
    const double h = c->dt / c->tau;
    for (int s = 0; s < 2; ++s) {
        const RkStage &r = c->rks[s];
        StageArgs &a = c->stage[s];
        a.eq = scaled(c->eq_unit, r.gamma * h);
        a.m = c->mc;
        a.a_base = r.alpha;
        a.a_self = r.beta - r.gamma * h;
        for (int g = 0; g < 4; ++g) {
            a.lx[g] = r.gamma * c->dt * c->mc.c[g] / c->grid.dx;
            a.ly[g] = r.gamma * c->dt * c->mc.c[g] / c->grid.dy;
        }
        for (int g = 0; g < 4; ++g) {
            const double ly = c->grid.ny > 1 ? a.ly[g] : 0.0;
            a.a_self_x[g] = a.a_self - a.lx[g];
            a.a_self_y[g] = a.a_self - ly;
            a.a_self_xy[g] = a.a_self - a.lx[g] - ly;
        }
        a.a_base_f = (float)a.a_base;
        a.a_self_f = (float)a.a_self;
        for (int g = 0; g < 4; ++g) {
            a.lx_f[g] = (float)a.lx[g];
            a.ly_f[g] = (float)a.ly[g];
        }
        a.rhoF = 0.0;
        a.EF = 0.0;
        for (int g = 0; g < 4; ++g) {
            a.sF[g] = r.gamma * h * c->Fg[g];
            a.rhoF += 4.0 * c->Fg[g];
            a.EF += 4.0 * c->Fg[g] * c->mc.w[g];
        }
        a.nx = c->grid.nx;
        a.ny = c->grid.ny;
        a.bc_x = c->grid.bc_x;
        a.bc_y = c->grid.bc_y;
        fill_df_consts(a);
        fill_dev_proj(a, r.gamma * h);
        c->launch[s] = stage_launch_config(a, r.with_base, c->sm_count, c->precision, c->march_enabled,
                                           c->small_enabled);
    }
    c->small = small1d_config(c->stage[0], c->precision);
}

cdbm_status enqueue_step(cdbm_ctx *c)
{
    cudaError_t e = launch_stage(c->launch[0], c->f, nullptr, c->f1, c->stage[0], c->flag, c->stream);
    if (e == cudaSuccess)
        e = launch_stage(c->launch[1], c->f1, c->f, c->f, c->stage[1], c->flag, c->stream);
    return cuda_check(c, e, "stage launch");
}

// Explicitly built graph of kGraphSteps steps (two kernel nodes per step); no
// stream capture, so it works on the legacy default stream too.
cdbm_status build_graph(cdbm_ctx *c)
{
    cudaGraph_t g;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return cuda_check(c, cudaGetLastError(), "graph create");
    cudaGraphNode_t prev = nullptr;
    const void *nil = nullptr;
    for (int s = 0; s < kGraphSteps; ++s) {
        for (int k = 0; k < 2; ++k) {
            const void *gin = (k == 0) ? c->f : c->f1;
            const void *base = (k == 0) ? nil : c->f;
            void *out = (k == 0) ? c->f1 : c->f;
            void *args[] = {(void *)&gin, (void *)&base, (void *)&out, (void *)&c->stage[k],
                            (void *)&c->flag};
            cudaKernelNodeParams p;
            memset(&p, 0, sizeof(p));
            p.func = c->launch[k].func;
            p.gridDim = c->launch[k].grid;
            p.blockDim = c->launch[k].block;
            p.sharedMemBytes = (unsigned)c->launch[k].smem;
            p.kernelParams = args;
            cudaGraphNode_t node;
            cudaError_t e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &p);
            if (e != cudaSuccess) {
                cudaGraphDestroy(g);
                return cuda_check(c, e, "graph add node");
            }
            prev = node;
        }
    }
    cudaError_t e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        return cuda_check(c, e, "graph instantiate");
    }
    return CDBM_OK;
}

void drop_graph(cdbm_ctx *c)
{
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

extern "C" {

cdbm_status cdbm_create(const cdbm_grid *grid, const cdbm_vset *vset, double I, double tau, double dt,
                        int precision, void *cuda_stream, const cdbm_allocator *allocator,
                        cdbm_ctx **out)
{
    if (!out) return create_err(CDBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !vset) return create_err(CDBM_EINVAL, "grid or vset is NULL");
    if (grid->nx < 1 || grid->ny < 1)
        return create_err(CDBM_EINVAL, "grid %d x %d: both sizes must be >= 1", grid->nx, grid->ny);
    if (!finite_pos(grid->dx) || !finite_pos(grid->dy) || !finite_pos(dt) || !finite_pos(tau))
        return create_err(CDBM_EINVAL, "dx, dy, dt and tau must be finite and > 0");
    if (!(std::isfinite(I) && I >= 0.0)) return create_err(CDBM_EINVAL, "I must be finite and >= 0");
    if ((grid->bc_x != 0 && grid->bc_x != 1) || (grid->bc_y != 0 && grid->bc_y != 1))
        return create_err(CDBM_EINVAL, "unknown boundary kind");
    if (precision != CDBM_FP64 && precision != CDBM_FP32_BULK && precision != CDBM_FP32_DF64 &&
        precision != CDBM_FP32_DEV)
        return create_err(CDBM_EINVAL, "unsupported precision %d", precision);
    for (int g = 0; g < 4; ++g)
        if (!std::isfinite(vset->v[g]) || !std::isfinite(vset->eta[g]) || vset->v[g] <= 0.0 ||
            vset->eta[g] < 0.0)
            return create_err(CDBM_EINVAL, "velocity set: v must be > 0 and eta >= 0");
    if (dt / tau > 2.0)
        return create_err(CDBM_EINVAL, "dt/tau = %g exceeds 2 (RK2 relaxation stability)", dt / tau);
    double cfl = 0.0;
    for (int i = 0; i < kNV; ++i) {
        const double s = vset->v[i >> 2];
        const double cx = grid->nx > 1 ? std::abs(dirx(i)) * s * dt / grid->dx : 0.0;
        const double cy = grid->ny > 1 ? std::abs(diry(i)) * s * dt / grid->dy : 0.0;
        cfl = cx + cy > cfl ? cx + cy : cfl;
    }
    if (cfl > 1.0) return create_err(CDBM_EINVAL, "CFL number %g exceeds 1", cfl);
    if ((size_t)grid->nx * grid->ny > ((size_t)1 << 40))
        return create_err(CDBM_EINVAL, "grid too large");

    cdbm_ctx *c = new (std::nothrow) cdbm_ctx();
    if (!c) return create_err(CDBM_ENOMEM, "host allocation failed");
    c->grid = *grid;
    c->vset = *vset;
    c->I = I;
    c->tau = tau;
    c->dt = dt;
    c->precision = precision;
    c->rk = CDBM_RK2_TVD;
    c->small_enabled = true;
    c->march_enabled = true;
    c->stream = (cudaStream_t)cuda_stream;
    c->user_alloc = allocator && allocator->alloc && allocator->free;
    if (c->user_alloc) c->alloc = *allocator;
    c->err = CDBM_OK;
    strcpy(c->msg, "no error");
    c->plane = (size_t)grid->nx * grid->ny;

    double cond = 0.0;
    const char *which = "";
    if (build_blocks(*vset, I, c->mc, c->eq_unit, &cond, &which) != CDBM_OK) {
        delete c;
        return create_err(CDBM_ESINGULAR, "moment matrix block '%s' singular (cond %g)", which, cond);
    }
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        delete c;
        return create_err(CDBM_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    c->sum_blocks = 2 * c->sm_count;
    build_stages(c);
    c->fields.eq = c->eq_unit;
    c->fields.m = c->mc;
    for (int i = 0; i < kNV; ++i) {
        const double s = vset->v[i >> 2];
        c->fields.vx[i] = dirx(i) * s;
        c->fields.vy[i] = diry(i) * s;
        c->fields.eta[i] = vset->eta[i >> 2];
    }
    c->fields.nx = grid->nx;
    c->fields.ny = grid->ny;

    const size_t fbytes = storage_bytes(precision) * kNV * c->plane;
    const size_t f1bytes = sizeof(double) * kNV * c->plane;
    c->f = ctx_alloc(c, fbytes);
    c->f1 = ctx_alloc(c, f1bytes);
    c->partials = (double *)ctx_alloc(c, sizeof(double) * kNV * c->sum_blocks + sizeof(double) * 4 + 256);
    if (!c->f || !c->f1 || !c->partials || cudaMallocHost(&c->flag_host, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        ctx_free(c, c->f, fbytes);
        ctx_free(c, c->f1, f1bytes);
        ctx_free(c, c->partials, 0);
        cudaStreamSynchronize(c->stream);
        delete c;
        return create_err(CDBM_ENOMEM, "device allocation of %zu bytes failed", fbytes + f1bytes);
    }
    c->sums = c->partials + kNV * c->sum_blocks;
    c->flag = (unsigned *)(c->sums + 4);
    *c->flag_host = 0;
    if (cudaMemsetAsync(c->flag, 0, sizeof(unsigned), c->stream) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        cdbm_destroy(c);
        return create_err(CDBM_ECUDA, "memset: %s", cudaGetErrorString(e));
    }
    *out = c;
    return CDBM_OK;
}

cdbm_status cdbm_set_rk(cdbm_ctx *c, int rk)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (rk != CDBM_RK2_TVD && rk != CDBM_RK2_MIDPOINT) return CDBM_EINVAL;
    if (rk != c->rk) {
        c->rk = rk;
        drop_graph(c);
        build_stages(c);
    }
    return CDBM_OK;
}

cdbm_status cdbm_init(cdbm_ctx *c, const double *rho, const double *ux, const double *uy,
                      const double *T)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (!rho || !ux || !uy || !T) return set_err(c, CDBM_EINVAL, "cdbm_init: NULL field");
    const double *src[4] = {rho, ux, uy, T};
    const double *dev[4];
    bool any_host = false;
    const size_t bytes = sizeof(double) * c->plane;
    for (int k = 0; k < 4; ++k) {
        if (is_device_pointer(src[k])) {
            dev[k] = src[k];
        } else {
            any_host = true;
            double *dst = (double *)c->f1 + k * c->plane;
            if (cuda_check(c, cudaMemcpyAsync(dst, src[k], bytes, cudaMemcpyHostToDevice, c->stream),
                           "cdbm_init upload"))
                return c->err;
            dev[k] = dst;
        }
    }
    if (single_storage(c->precision)) {
        // reference state for the deviation storage: the means of rho and T
        double sum[2] = {0.0, 0.0};
        if (cuda_check(c, launch_field_means(dev[0], dev[3], c->plane, c->partials, c->sum_blocks, c->sums,
                                             c->stream), "means launch") ||
            cuda_check(c, cudaMemcpyAsync(sum, c->sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                       "means download") ||
            cuda_check(c, cudaStreamSynchronize(c->stream), "means sync"))
            return c->err;
        set_reference(c, sum[0] / (double)c->plane, sum[1] / (double)c->plane);
        drop_graph(c);
        build_stages(c);
    }
    if (cuda_check(c, launch_init(c->fields, dev[0], dev[1], dev[2], dev[3], c->f, c->precision, c->flag,
                                  c->stream),
                   "init launch"))
        return c->err;
    if (any_host && cuda_check(c, cudaStreamSynchronize(c->stream), "cdbm_init sync")) return c->err;
    // the step graph of the stage-launch path, built and uploaded here so that the
    // first long cdbm_step does not pay for it
    if (!c->graph && !(c->small.ok && c->small_enabled)) {
        if (build_graph(c)) return c->err;
        if (cuda_check(c, cudaGraphUpload(c->graph, c->stream), "graph upload")) return c->err;
    }
    c->t = 0.0;
    c->state_set = true;
    c->step_count = 0;
    c->adj_steps = 0;
    return CDBM_OK;
}

cdbm_status cdbm_step(cdbm_ctx *c, int nsteps)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (nsteps < 0) return set_err(c, CDBM_EINVAL, "cdbm_step: nsteps < 0");
    if (!c->state_set) return set_err(c, CDBM_EINVAL, "cdbm_step: state not initialised");
    int left = nsteps;
    if (c->small.ok && c->small_enabled) {
        // whole run in persistent launches of at most kSmallSteps steps
        while (left > 0) {
            const int n = left < kSmallSteps ? left : kSmallSteps;
            if (cuda_check(c, launch_small1d(c->small, c->f, n, c->stage[0], c->stage[1], c->flag, c->stream),
                           "small-grid launch"))
                return c->err;
            left -= n;
        }
    }
    if (left >= kGraphSteps && !c->graph && build_graph(c)) return c->err;
    while (left >= kGraphSteps) {
        if (cuda_check(c, cudaGraphLaunch(c->graph, c->stream), "graph launch")) return c->err;
        left -= kGraphSteps;
    }
    for (; left > 0; --left)
        if (enqueue_step(c)) return c->err;
    c->t += nsteps * c->dt;
    c->step_count += nsteps;
    return CDBM_OK;
}

cdbm_status cdbm_set_small_grid_path(cdbm_ctx *c, int enable)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if ((enable != 0) != c->small_enabled) {
        c->small_enabled = enable != 0;
        drop_graph(c);
        build_stages(c);
    }
    return CDBM_OK;
}

cdbm_status cdbm_set_row_marching(cdbm_ctx *c, int enable)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if ((enable != 0) != c->march_enabled) {
        c->march_enabled = enable != 0;
        drop_graph(c);
        build_stages(c);
    }
    return CDBM_OK;
}

cdbm_status cdbm_macros(cdbm_ctx *c, double *rho, double *ux, double *uy, double *T)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (!c->state_set) return set_err(c, CDBM_EINVAL, "cdbm_macros: state not initialised");
    double *dst[4] = {rho, ux, uy, T};
    double *dev[4];
    bool host[4];
    bool any_host = false;
    for (int k = 0; k < 4; ++k) {
        host[k] = dst[k] && !is_device_pointer(dst[k]);
        any_host |= host[k];
        dev[k] = host[k] ? (double *)c->f1 + k * c->plane : dst[k];
    }
    if (cuda_check(c, launch_macros(c->fields, c->f, c->precision, dev[0], dev[1], dev[2], dev[3], c->stream),
                   "macros launch"))
        return c->err;
    for (int k = 0; k < 4; ++k)
        if (host[k] && cuda_check(c, cudaMemcpyAsync(dst[k], dev[k], sizeof(double) * c->plane,
                                                     cudaMemcpyDeviceToHost, c->stream),
                                  "cdbm_macros download"))
            return c->err;
    if (any_host && cuda_check(c, cudaStreamSynchronize(c->stream), "cdbm_macros sync")) return c->err;
    return CDBM_OK;
}

cdbm_status cdbm_tne(cdbm_ctx *c, double *out)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (!out) return set_err(c, CDBM_EINVAL, "cdbm_tne: NULL output");
    if (!c->state_set) return set_err(c, CDBM_EINVAL, "cdbm_tne: state not initialised");
    const bool host = !is_device_pointer(out);
    double *dev = host ? (double *)c->f1 : out;
    if (cuda_check(c, launch_tne(c->fields, c->f, c->precision, dev, c->stream), "tne launch")) return c->err;
    if (host) {
        if (cuda_check(c, cudaMemcpyAsync(out, dev, sizeof(double) * 12 * c->plane,
                                          cudaMemcpyDeviceToHost, c->stream), "cdbm_tne download") ||
            cuda_check(c, cudaStreamSynchronize(c->stream), "cdbm_tne sync"))
            return c->err;
    }
    return CDBM_OK;
}

cdbm_status cdbm_conserved_sums(cdbm_ctx *c, double out[4])
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (!out) return set_err(c, CDBM_EINVAL, "cdbm_conserved_sums: NULL output");
    if (!c->state_set) return set_err(c, CDBM_EINVAL, "cdbm_conserved_sums: state not initialised");
    if (cuda_check(c, launch_sums(c->fields, c->f, c->precision, c->partials, c->sum_blocks, c->sums, c->stream),
                   "sums launch") ||
        cuda_check(c, cudaMemcpyAsync(out, c->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                   "sums download") ||
        cuda_check(c, cudaStreamSynchronize(c->stream), "sums sync"))
        return c->err;
    return CDBM_OK;
}

cdbm_status cdbm_get_state(cdbm_ctx *c, double *f, double *t)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (f) {
        if (!c->state_set) return set_err(c, CDBM_EINVAL, "cdbm_get_state: state not initialised");
        const bool host = !is_device_pointer(f);
        const size_t n = kNV * c->plane;
        if (c->precision == CDBM_FP64) {
            if (cuda_check(c, cudaMemcpyAsync(f, c->f, sizeof(double) * n, cudaMemcpyDefault, c->stream),
                           "cdbm_get_state copy"))
                return c->err;
        } else {
            double *dst = host ? (double *)c->f1 : f;
            if (cuda_check(c, launch_convert(c->fields, c->f, c->precision, dst, CDBM_FP64, c->stream),
                           "cdbm_get_state convert") ||
                (host && cuda_check(c, cudaMemcpyAsync(f, dst, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                                       c->stream), "cdbm_get_state copy")))
                return c->err;
        }
        if (host && cuda_check(c, cudaStreamSynchronize(c->stream), "cdbm_get_state sync")) return c->err;
    }
    if (t) *t = c->t;
    return CDBM_OK;
}

cdbm_status cdbm_set_state(cdbm_ctx *c, const double *f, double t)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (!f || !std::isfinite(t)) return set_err(c, CDBM_EINVAL, "cdbm_set_state: bad argument");
    const bool host = !is_device_pointer(f);
    const size_t n = kNV * c->plane;
    if (c->precision == CDBM_FP64) {
        if (cuda_check(c, cudaMemcpyAsync(c->f, f, sizeof(double) * n, cudaMemcpyDefault, c->stream),
                       "cdbm_set_state copy"))
            return c->err;
    } else {
        const double *src = f;
        if (host) {
            if (cuda_check(c, cudaMemcpyAsync(c->f1, f, sizeof(double) * n, cudaMemcpyHostToDevice,
                                              c->stream), "cdbm_set_state copy"))
                return c->err;
            src = (const double *)c->f1;
        }
        // reference state from the mean conserved moments of the incoming state
        double sum[4];
        if (cuda_check(c, launch_sums(c->fields, src, CDBM_FP64, c->partials, c->sum_blocks, c->sums,
                                      c->stream), "cdbm_set_state sums") ||
            cuda_check(c, cudaMemcpyAsync(sum, c->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                       "cdbm_set_state sums download") ||
            cuda_check(c, cudaStreamSynchronize(c->stream), "cdbm_set_state sync"))
            return c->err;
        set_reference(c, sum[0] / (double)c->plane, sum[3] / (sum[0] * c->mc.K));
        drop_graph(c);
        build_stages(c);
        if (cuda_check(c, launch_convert(c->fields, src, CDBM_FP64, c->f, c->precision, c->stream),
                       "cdbm_set_state convert"))
            return c->err;
    }
    if (host && cuda_check(c, cudaStreamSynchronize(c->stream), "cdbm_set_state sync")) return c->err;
    c->t = t;
    c->state_set = true;
    c->step_count = 0;
    c->adj_steps = 0;
    return CDBM_OK;
}

cdbm_status cdbm_state_ptr(cdbm_ctx *c, void **f)
{
    if (!c || !f) return CDBM_EINVAL;
    *f = c->f;
    return c->err;
}

cdbm_status cdbm_time(const cdbm_ctx *c, double *t)
{
    if (!c || !t) return CDBM_EINVAL;
    *t = c->t;
    return c->err;
}

namespace {

cdbm_status adjoint_supported(cdbm_ctx *c, const char *who)
{
    if (c->precision != CDBM_FP64) return set_err(c, CDBM_EINVAL, "%s: needs CDBM_FP64", who);
    if (c->rk != CDBM_RK2_TVD) return set_err(c, CDBM_EINVAL, "%s: needs CDBM_RK2_TVD", who);
    if ((c->grid.nx > 1 && c->grid.bc_x != CDBM_BC_PERIODIC) || (c->grid.ny > 1 && c->grid.bc_y != CDBM_BC_PERIODIC))
        return set_err(c, CDBM_EINVAL, "%s: needs periodic boundaries", who);
    return CDBM_OK;
}

void free_ckpt(cdbm_ctx *c)
{
    for (void *p : c->ckpt) ctx_free(c, p, sizeof(double) * kNV * c->plane);
    c->ckpt.clear();
    c->adj_steps = 0;
}

}  // namespace

cdbm_status cdbm_adjoint_forward(cdbm_ctx *c, int nsteps, int every)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (adjoint_supported(c, "cdbm_adjoint_forward")) return c->err;
    if (nsteps < 1 || every < 1) return set_err(c, CDBM_EINVAL, "cdbm_adjoint_forward: nsteps, every >= 1");
    if (!c->state_set) return set_err(c, CDBM_EINVAL, "cdbm_adjoint_forward: state not initialised");
    free_ckpt(c);
    const size_t fb = sizeof(double) * kNV * c->plane;
    const int nck = (nsteps + every - 1) / every;
    for (int k = 0; k < nck; ++k) {
        void *p = ctx_alloc(c, fb);
        if (!p) {
            free_ckpt(c);
            return set_err(c, CDBM_ENOMEM, "checkpoint allocation (%d x %zu bytes) failed", nck, fb);
        }
        c->ckpt.push_back(p);
    }
    for (int k = 0; k < nck; ++k) {
        if (cuda_check(c, cudaMemcpyAsync(c->ckpt[k], c->f, fb, cudaMemcpyDeviceToDevice, c->stream), "checkpoint"))
            return c->err;
        const int n = (k + 1) * every <= nsteps ? every : nsteps - k * every;
        if (cdbm_step(c, n)) return c->err;
    }
    c->adj_steps = nsteps;
    c->adj_every = every;
    c->adj_end = c->step_count;
    return CDBM_OK;
}

cdbm_status cdbm_adjoint_backward(cdbm_ctx *c, const double *fbar, double *grad_rho, double *grad_ux,
                                  double *grad_uy, double *grad_T, double *grad_tau)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (!fbar) return set_err(c, CDBM_EINVAL, "cdbm_adjoint_backward: NULL cotangent");
    if (c->adj_steps < 1 || c->step_count != c->adj_end)
        return set_err(c, CDBM_EINVAL, "cdbm_adjoint_backward: no recorded run ending at the current state");
    const int nsteps = c->adj_steps, every = c->adj_every;
    const size_t n = kNV * c->plane, fb = sizeof(double) * n;
    const dim3 ag = adjoint_grid(c->grid.nx, c->grid.ny);
    const int nacc = (int)(ag.x * ag.y);
    const int seglen = every < nsteps ? every : nsteps;
    // B: cotangent of the current state; B1: of the stage-1 state; G1: stage-1 state;
    // seg: the states of one segment, recomputed from its checkpoint
    std::vector<void *> bufs;
    auto grab = [&](size_t bytes) {
        void *p = ctx_alloc(c, bytes);
        bufs.push_back(p);
        return (double *)p;
    };
    double *B = grab(fb), *B1 = grab(fb), *G1 = grab(fb);
    double *acc = grab(sizeof(double) * (nacc + 1));
    std::vector<double *> seg(seglen);
    for (int j = 1; j < seglen; ++j) seg[j] = grab(fb);
    bool ok = true;
    for (void *p : bufs) ok = ok && p;
    cdbm_status st = CDBM_OK;
    if (!ok) st = set_err(c, CDBM_ENOMEM, "adjoint work buffers (%d states) failed", seglen + 2);
    // Optional: the stage-1 states of a segment, kept from its recomputation so the
    // backward sweep does not recompute them (one stage launch per step less, one
    // more segment of memory).  Without the memory the sweep recomputes them.
    std::vector<double *> seg1;
    if (!st) {
        for (int j = 0; j < seglen; ++j) {
            double *p = (double *)ctx_alloc(c, fb);
            if (!p) break;
            seg1.push_back(p);
        }
        if ((int)seg1.size() < seglen) {
            for (double *p : seg1) ctx_free(c, p, fb);
            seg1.clear();
        }
    }
    const bool keep1 = !seg1.empty();
    const double h = c->dt / c->tau, inv_tau = 1.0 / c->tau;
    if (!st && (cuda_check(c, cudaMemcpyAsync(B, fbar, fb, cudaMemcpyDefault, c->stream), "cotangent copy") ||
                cuda_check(c, cudaMemsetAsync(acc, 0, sizeof(double) * (nacc + 1), c->stream), "acc clear")))
        st = c->err;
    const int nseg = (nsteps + every - 1) / every;
    for (int sgi = nseg - 1; sgi >= 0 && !st; --sgi) {
        const int len = (sgi + 1) * every <= nsteps ? every : nsteps - sgi * every;
        seg[0] = (double *)c->ckpt[sgi];
        for (int j = 0; j < len && !st; ++j) {
            if (!keep1 && j + 1 == len) break;
            double *g1 = keep1 ? seg1[j] : G1;
            cudaError_t e = launch_stage(c->launch[0], seg[j], nullptr, g1, c->stage[0], c->flag, c->stream);
            if (e == cudaSuccess && j + 1 < len)
                e = launch_stage(c->launch[1], g1, seg[j], seg[j + 1], c->stage[1], c->flag, c->stream);
            st = cuda_check(c, e, "adjoint recompute");
        }
        for (int j = len - 1; j >= 0 && !st; --j) {
            const double *g1 = keep1 ? seg1[j] : G1;
            cudaError_t e = keep1 ? cudaSuccess
                                  : launch_stage(c->launch[0], seg[j], nullptr, G1, c->stage[0], c->flag, c->stream);
            if (e == cudaSuccess)   // stage 2: f^{n+1} = f^n/2 + f1/2 + dt/2 L(f1)
                e = launch_adjoint_stage(g1, B, nullptr, 0.0, B1, c->stage[1], 0.5 * h, inv_tau, c->adj_limiter, acc,
                                         c->stream);
            if (e == cudaSuccess)   // stage 1: f1 = f^n + dt L(f^n); plus the f^n/2 of stage 2
                e = launch_adjoint_stage(seg[j], B1, B, 0.5, B, c->stage[0], h, inv_tau, c->adj_limiter, acc, c->stream);
            st = cuda_check(c, e, "adjoint stage");
        }
    }
    if (!st && cuda_check(c, launch_init_vjp(c->fields, (const double *)c->ckpt[0], B, grad_rho, grad_ux, grad_uy,
                                             grad_T, c->stream), "init vjp"))
        st = c->err;
    if (!st && grad_tau) {
        if (cuda_check(c, launch_sum(acc, nacc, acc + nacc, c->stream), "tau sum") ||
            cuda_check(c, cudaMemcpyAsync(grad_tau, acc + nacc, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                       "tau download"))
            st = c->err;
    }
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "adjoint sync");
    for (size_t k = 0; k < bufs.size(); ++k) ctx_free(c, bufs[k], k == 3 ? sizeof(double) * (nacc + 1) : fb);
    for (double *p : seg1) ctx_free(c, p, fb);
    return st;
}

cdbm_status cdbm_adjoint_set_limiter(cdbm_ctx *c, int mode)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (mode != CDBM_ADJ_LIMITER_EXACT && mode != CDBM_ADJ_LIMITER_FROZEN_RATIO && mode != CDBM_ADJ_LIMITER_FROZEN)
        return set_err(c, CDBM_EINVAL, "cdbm_adjoint_set_limiter: unknown mode %d", mode);
    c->adj_limiter = mode;
    return CDBM_OK;
}

cdbm_status cdbm_macros_vjp(cdbm_ctx *c, const double *rho_bar, const double *ux_bar, const double *uy_bar,
                            const double *T_bar, double *fbar)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (!fbar) return set_err(c, CDBM_EINVAL, "cdbm_macros_vjp: NULL output");
    if (c->precision != CDBM_FP64) return set_err(c, CDBM_EINVAL, "cdbm_macros_vjp: needs CDBM_FP64");
    if (!c->state_set) return set_err(c, CDBM_EINVAL, "cdbm_macros_vjp: state not initialised");
    return cuda_check(c, launch_macros_vjp(c->fields, (const double *)c->f, rho_bar, ux_bar, uy_bar, T_bar, fbar,
                                           c->stream), "macros vjp");
}

cdbm_status cdbm_sync(cdbm_ctx *c)
{
    if (!c) return CDBM_EINVAL;
    if (c->err) return c->err;
    if (cuda_check(c, cudaMemcpyAsync(c->flag_host, c->flag, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                      c->stream), "flag download") ||
        cuda_check(c, cudaStreamSynchronize(c->stream), "cdbm_sync"))
        return c->err;
    if (*c->flag_host & kFlagNonPhys)
        return set_err(c, CDBM_ENONPHYS, "non-physical state (rho <= 0, T <= 0 or non-finite) at t = %g",
                       c->t);
    return CDBM_OK;
}

const char *cdbm_last_error(const cdbm_ctx *c)
{
    return c ? c->msg : g_create_error;
}

void cdbm_destroy(cdbm_ctx *c)
{
    if (!c) return;
    drop_graph(c);
    for (void *p : c->ckpt) ctx_free(c, p, sizeof(double) * kNV * c->plane);
    c->ckpt.clear();
    ctx_free(c, c->f, storage_bytes(c->precision) * kNV * c->plane);
    ctx_free(c, c->f1, sizeof(double) * kNV * c->plane);
    ctx_free(c, c->partials, sizeof(double) * kNV * c->sum_blocks + sizeof(double) * 4 + 256);
    cudaStreamSynchronize(c->stream);
    if (c->flag_host) cudaFreeHost(c->flag_host);
    cudaGetLastError();
    delete c;
}

}  // extern "C"
