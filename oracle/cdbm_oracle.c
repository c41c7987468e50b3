/*
 * CDBM oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU implementation of the central-moment-based
 * discrete Boltzmann method (CDBM) of Lin, Su, Fei and Luo, "Central-moment-based
 * discrete Boltzmann modeling of compressible flows" (Sec. 2, Eqs. 1-20).  It exists
 * only so that the test-suite, the package smoke check and the benchmark's CPU
 * baseline can check the CUDA library against an independent statement of the
 * method.  It shares no source, header, table or constant with the CUDA library,
 * and nothing in the product path may load it.
 *
 * Everything follows the paper's own formulation, with no factoring:
 *   - the equilibrium is the direct solution of the 16x16 central-moment system
 *     M(u) f_eq = fbar_eq (Eqs. 6-7) by Gaussian elimination with scaled partial
 *     pivoting and one step of iterative refinement, per cell;
 *   - fbar_eq holds the central moments of the Maxwellian with I extra degrees
 *     of freedom (Eq. 5), written out in closed form below;
 *   - the space derivative is the NND scheme with the minmod limiter exactly as
 *     Eqs. (12)-(20) state it, keeping both the left (f+) and right (f-) parts;
 *   - time integration is the two-stage Runge-Kutta scheme (Sec. 2 names a
 *     second-order Runge-Kutta scheme without printing it; rk = 0 takes the
 *     two-stage TVD form, rk = 1 the midpoint form).
 *
 * Readings of the paper this file takes (where the text is silent or garbled):
 *   - Eq. (2) lists one vector per group; the four members of an axis group are
 *     taken as (1,0),(0,1),(-1,0),(0,-1) and of a diagonal group as
 *     (1,1),(-1,1),(-1,-1),(1,-1), each times the group speed (diagonals are
 *     not normalised, so |v| = sqrt(2) v_b).
 *   - The Psi list of Eq. (4) item "v*.v*" is the tensor v*v* (rows 5-7 of Eq. 6),
 *     which gives the 16 rows of the matrix.
 *   - The temperature follows from rho K T = sum_i f_i ((v_i - u)^2 + eta_i^2),
 *     K = D + I, D = 2 (Eq. 4 energy row with <eta^2> = I T from Eq. 5).
 *   - For I = 0 the eta factor of Eq. (5) is taken in its limit <eta^2> = 0.
 *   - Eq. (12) has its sign garbled: the transport term v df/dr is approximated
 *     by +(H(j+1/2) - H(j-1/2)) / dr, so the right-hand side of Eq. (1) becomes
 *     -(H(j+1/2) - H(j-1/2)) / dr - (f - f_eq) / tau.
 *   - minmod (Eq. 16): the ratio test |X/Y| <= 1 is evaluated as |X| <= |Y|, and
 *     "XY <= 0" as "X = 0, Y = 0 or opposite signs" (no product underflow).
 *   - Boundaries are not stated: per axis either periodic or zero-gradient
 *     (ghost cells copy the edge cell).
 *
 * Layout: a distribution field is f[16][ny][nx], x fastest, velocity index i
 * outermost; a scalar field is [ny][nx].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 16

typedef struct {
    int nx, ny;
    int bc_x, bc_y;   /* 0 = periodic, 1 = zero-gradient */
    int rk;           /* 0 = two-stage TVD Runge-Kutta, 1 = midpoint */
    int threads;      /* OpenMP threads; 0 = runtime default */
    double dx, dy, dt, tau, I;
    double vg[4];     /* (v_a, v_b, v_c, v_d), Eq. (2) */
    double eg[4];     /* (eta_a, eta_b, eta_c, eta_d), Eq. (3) */
} orc_params;

/* ---------------------------------------------------------------- Eqs. (2)-(3) */

void orc_velocity_set(const double vg[4], const double eg[4],
                      double vx[NV], double vy[NV], double eta[NV])
{
    /* Groups a and c point along the axes, groups b and d along the diagonals. */
    static const double axis[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
    static const double diag[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    for (int g = 0; g < 4; ++g) {
        for (int k = 0; k < 4; ++k) {
            int i = 4 * g + k;
            const double *e = (g == 0 || g == 2) ? axis[k] : diag[k];
            vx[i] = vg[g] * e[0];
            vy[i] = vg[g] * e[1];
            eta[i] = eg[g];
        }
    }
}

/* ------------------------------------------------------------------- Eq. (6) */

/* Row k of M holds Psi_k evaluated at the peculiar velocity v_i* = v_i - u. */
void orc_central_matrix(const double vx[NV], const double vy[NV], const double eta[NV],
                        double ux, double uy, double M[NV * NV])
{
    for (int i = 0; i < NV; ++i) {
        double cx = vx[i] - ux;
        double cy = vy[i] - uy;
        double w = cx * cx + cy * cy + eta[i] * eta[i];   /* v*^2 + eta^2 */
        M[0 * NV + i] = 1.0;
        M[1 * NV + i] = cx;
        M[2 * NV + i] = cy;
        M[3 * NV + i] = w;
        M[4 * NV + i] = cx * cx;
        M[5 * NV + i] = cx * cy;
        M[6 * NV + i] = cy * cy;
        M[7 * NV + i] = w * cx;
        M[8 * NV + i] = w * cy;
        M[9 * NV + i] = cx * cx * cx;
        M[10 * NV + i] = cx * cx * cy;
        M[11 * NV + i] = cx * cy * cy;
        M[12 * NV + i] = cy * cy * cy;
        M[13 * NV + i] = w * cx * cx;
        M[14 * NV + i] = w * cx * cy;
        M[15 * NV + i] = w * cy * cy;
    }
}

/* ------------------------------------------------------------------- Eq. (5) */

/*
 * Central moments of the Maxwellian of Eq. (5) for the 16 rows of Eq. (6).
 * With c = v - u the translational part is Gaussian with variance T per axis and
 * eta is Gaussian with variance I T, so <c_x^2> = T, <c_x^4> = 3 T^2,
 * <c_x^2 c_y^2> = T^2, <eta^2> = I T and every odd moment vanishes:
 *   <1> = 1, <c^2 + eta^2> = (D + I) T = K T, <c_x^2> = <c_y^2> = T,
 *   <(c^2 + eta^2) c_x^2> = 3T^2 + T^2 + I T^2 = (K + 2) T^2 (same for y).
 * All are multiplied by rho = n m, m = 1.
 */
void orc_central_moments_eq(double I, double rho, double T, double fbar[NV])
{
    const double K = 2.0 + I;
    for (int k = 0; k < NV; ++k) fbar[k] = 0.0;
    fbar[0] = rho;
    fbar[3] = rho * K * T;
    fbar[4] = rho * T;
    fbar[6] = rho * T;
    fbar[13] = rho * (K + 2.0) * T * T;
    fbar[15] = rho * (K + 2.0) * T * T;
}

/* ------------------------------------------------------------------- Eq. (7) */

/*
 * Solves A x = b (n <= 16) by Gaussian elimination with scaled partial pivoting,
 * followed by one step of iterative refinement with the residual in double.
 * Returns 0 on success, 1 if a pivot vanishes.
 */
int orc_solve(int n, const double *A, const double *b, double *x)
{
    double LU[NV * NV], s[NV], y[NV], r[NV];
    int perm[NV];
    if (n > NV) return 1;
    memcpy(LU, A, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) {
        perm[i] = i;
        s[i] = 0.0;
        for (int j = 0; j < n; ++j)
            if (fabs(A[i * n + j]) > s[i]) s[i] = fabs(A[i * n + j]);
        if (s[i] == 0.0) return 1;
    }
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = -1.0;
        for (int i = k; i < n; ++i) {
            double q = fabs(LU[perm[i] * n + k]) / s[perm[i]];
            if (q > best) { best = q; p = i; }
        }
        int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
        double piv = LU[perm[k] * n + k];
        if (piv == 0.0) return 1;
        for (int i = k + 1; i < n; ++i) {
            double m = LU[perm[i] * n + k] / piv;
            LU[perm[i] * n + k] = m;
            for (int j = k + 1; j < n; ++j) LU[perm[i] * n + j] -= m * LU[perm[k] * n + j];
        }
    }
    /* x = LU^-1 b, then one refinement step x += LU^-1 (b - A x). */
    for (int pass = 0; pass < 2; ++pass) {
        const double *rhs = b;
        if (pass == 1) {
            for (int i = 0; i < n; ++i) {
                double acc = b[i];
                for (int j = 0; j < n; ++j) acc -= A[i * n + j] * x[j];
                r[i] = acc;
            }
            rhs = r;
        }
        for (int i = 0; i < n; ++i) {
            double acc = rhs[perm[i]];
            for (int j = 0; j < i; ++j) acc -= LU[perm[i] * n + j] * y[j];
            y[i] = acc;
        }
        for (int i = n - 1; i >= 0; --i) {
            double acc = y[i];
            for (int j = i + 1; j < n; ++j) acc -= LU[perm[i] * n + j] * y[j];
            y[i] = acc / LU[perm[i] * n + i];
        }
        for (int i = 0; i < n; ++i) x[i] = (pass == 0) ? y[i] : x[i] + y[i];
    }
    return 0;
}

/* f_eq(rho, u, T) = M(u)^-1 fbar_eq(rho, T), Eqs. (5)-(7). Returns 0 on success. */
int orc_feq(const orc_params *p, double rho, double ux, double uy, double T, double feq[NV])
{
    double vx[NV], vy[NV], eta[NV], M[NV * NV], fbar[NV];
    orc_velocity_set(p->vg, p->eg, vx, vy, eta);
    orc_central_matrix(vx, vy, eta, ux, uy, M);
    orc_central_moments_eq(p->I, rho, T, fbar);
    return orc_solve(NV, M, fbar, feq);
}

/* ------------------------------------------------------ macroscopic quantities */

/*
 * rho = sum f_i, rho u = sum f_i v_i, rho K T = sum f_i ((v_i - u)^2 + eta_i^2):
 * the conserved rows of Eq. (4) evaluated with f in place of f_eq (Sec. 2, after
 * Eq. 7).
 */
void orc_cell_macros(const orc_params *p, const double f[NV],
                     double *rho, double *ux, double *uy, double *T)
{
    double vx[NV], vy[NV], eta[NV];
    orc_velocity_set(p->vg, p->eg, vx, vy, eta);
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < NV; ++i) {
        r += f[i];
        jx += f[i] * vx[i];
        jy += f[i] * vy[i];
    }
    double u = jx / r, v = jy / r;
    double e = 0.0;
    for (int i = 0; i < NV; ++i) {
        double cx = vx[i] - u, cy = vy[i] - v;
        e += f[i] * (cx * cx + cy * cy + eta[i] * eta[i]);
    }
    *rho = r;
    *ux = u;
    *uy = v;
    *T = e / (r * (2.0 + p->I));
}

/* ----------------------------------------------------------- Eqs. (12)-(20) */

/* Eq. (16). */
double orc_minmod(double X, double Y)
{
    if (X == 0.0 || Y == 0.0) return 0.0;
    if ((X > 0.0) != (Y > 0.0)) return 0.0;
    return (fabs(X) <= fabs(Y)) ? X : Y;
}

/*
 * Approximation of v df/dr at grid point j from the five values
 * f(j-2) .. f(j+2) along r, Eqs. (12)-(20):
 *   f+(k) = (v + |v|)/2 f(k),  f-(k) = (v - |v|)/2 f(k)               (19)-(20)
 *   Df+(k+1/2) = f+(k+1) - f+(k),  Df-(k+1/2) = f-(k+1) - f-(k)         (17)-(18)
 *   H_L(k+1/2) = f+(k) + minmod(Df+(k+1/2), Df+(k-1/2)) / 2              (14)
 *   H_R(k+1/2) = f-(k+1) - minmod(Df-(k+1/2), Df-(k+3/2)) / 2            (15)
 *   H = H_L + H_R                                                         (13)
 *   v df/dr ~ (H(j+1/2) - H(j-1/2)) / dr                                  (12)
 */
double orc_nnd_derivative(double v, const double fs[5], double dr)
{
    double fp[5], fm[5];
    for (int k = 0; k < 5; ++k) {
        fp[k] = 0.5 * (v + fabs(v)) * fs[k];
        fm[k] = 0.5 * (v - fabs(v)) * fs[k];
    }
    /* index 2 is point j; interface k+1/2 sits between fs[k] and fs[k+1]. */
    double dp[4], dm[4];
    for (int k = 0; k < 4; ++k) {
        dp[k] = fp[k + 1] - fp[k];
        dm[k] = fm[k + 1] - fm[k];
    }
    /* H(j+1/2): left point is fs[2] (interface index 2). */
    double HLp = fp[2] + 0.5 * orc_minmod(dp[2], dp[1]);
    double HRp = fm[3] - 0.5 * orc_minmod(dm[2], dm[3]);
    /* H(j-1/2): left point is fs[1] (interface index 1). */
    double HLm = fp[1] + 0.5 * orc_minmod(dp[1], dp[0]);
    double HRm = fm[2] - 0.5 * orc_minmod(dm[1], dm[2]);
    return ((HLp + HRp) - (HLm + HRm)) / dr;
}

static int ghost_index(int j, int n, int bc)
{
    if (bc == 0) {
        j %= n;
        return j < 0 ? j + n : j;
    }
    return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

/* threads > 0 sets the OpenMP thread count for this call; 0 restores the count the
 * runtime started with (omp_set_num_threads would otherwise stick). */
static void set_threads(const orc_params *p)
{
#ifdef _OPENMP
    static int default_threads = 0;
    if (default_threads == 0) default_threads = omp_get_max_threads();
    omp_set_num_threads(p->threads > 0 ? p->threads : default_threads);
#else
    (void)p;
#endif
}

/*
 * Right-hand side of Eq. (1): L_i = -v_i . grad f_i - (f_i - f_i^eq) / tau,
 * with the transport term from the NND scheme along x and y.
 * Returns the number of cells whose equilibrium solve failed.
 */
static int orc_rhs(const orc_params *p, const double *f, double *L)
{
    const int nx = p->nx, ny = p->ny;
    const size_t plane = (size_t)nx * ny;
    double vx[NV], vy[NV], eta[NV];
    orc_velocity_set(p->vg, p->eg, vx, vy, eta);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long c = 0; c < (long)plane; ++c) {
        int x = (int)(c % nx), y = (int)(c / nx);
        double fc[NV], feq[NV], rho, ux, uy, T;
        for (int i = 0; i < NV; ++i) fc[i] = f[i * plane + c];
        orc_cell_macros(p, fc, &rho, &ux, &uy, &T);
        if (orc_feq(p, rho, ux, uy, T, feq) != 0) bad += 1;
        for (int i = 0; i < NV; ++i) {
            const double *fi = f + i * plane;
            double sx[5], sy[5];
            for (int k = -2; k <= 2; ++k) {
                sx[k + 2] = fi[(size_t)y * nx + ghost_index(x + k, nx, p->bc_x)];
                sy[k + 2] = fi[(size_t)ghost_index(y + k, ny, p->bc_y) * nx + x];
            }
            double adv = orc_nnd_derivative(vx[i], sx, p->dx) + orc_nnd_derivative(vy[i], sy, p->dy);
            L[i * plane + c] = -adv - (fc[i] - feq[i]) / p->tau;
        }
    }
    return bad;
}

/* f <- f_eq(rho, u, T) cell by cell (initial state). Returns failed cells. */
int orc_init(const orc_params *p, const double *rho, const double *ux, const double *uy,
             const double *T, double *f)
{
    const size_t plane = (size_t)p->nx * p->ny;
    int bad = 0;
    set_threads(p);
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long c = 0; c < (long)plane; ++c) {
        double feq[NV];
        if (orc_feq(p, rho[c], ux[c], uy[c], T[c], feq) != 0) bad += 1;
        for (int i = 0; i < NV; ++i) f[i * plane + c] = feq[i];
    }
    return bad;
}

/*
 * Advances f by nsteps time steps of dt. rk = 0:
 *   f1 = f + dt L(f),  f <- f/2 + (f1 + dt L(f1))/2;
 * rk = 1 (midpoint):
 *   fh = f + dt/2 L(f),  f <- f + dt L(fh).
 * Returns 0, -1 on allocation failure, or the count of failed solves.
 */
int orc_step(const orc_params *p, double *f, int nsteps)
{
    const size_t n = (size_t)NV * p->nx * p->ny;
    double *L = (double *)malloc(sizeof(double) * n);
    double *g = (double *)malloc(sizeof(double) * n);
    int bad = 0;
    if (!L || !g) { free(L); free(g); return -1; }
    set_threads(p);
    for (int s = 0; s < nsteps; ++s) {
        bad += orc_rhs(p, f, L);
        if (p->rk == 0) {
            for (size_t k = 0; k < n; ++k) g[k] = f[k] + p->dt * L[k];
            bad += orc_rhs(p, g, L);
            for (size_t k = 0; k < n; ++k) f[k] = 0.5 * f[k] + 0.5 * (g[k] + p->dt * L[k]);
        } else {
            for (size_t k = 0; k < n; ++k) g[k] = f[k] + 0.5 * p->dt * L[k];
            bad += orc_rhs(p, g, L);
            for (size_t k = 0; k < n; ++k) f[k] = f[k] + p->dt * L[k];
        }
    }
    free(L);
    free(g);
    return bad;
}

/* rho, u_x, u_y, T fields of f. */
void orc_macros(const orc_params *p, const double *f, double *rho, double *ux, double *uy, double *T)
{
    const size_t plane = (size_t)p->nx * p->ny;
    set_threads(p);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)plane; ++c) {
        double fc[NV];
        for (int i = 0; i < NV; ++i) fc[i] = f[i * plane + c];
        orc_cell_macros(p, fc, rho + c, ux + c, uy + c, T + c);
    }
}

/*
 * Nonequilibrium central moments, Eqs. (8)-(11): out[k][ny][nx] for k = 0..11 holds
 * sum_i (f_i - f_i^eq) Psi_{k+5}(v_i - u), i.e. rows 5..16 of Eq. (6):
 * Delta2 {xx, xy, yy}, Delta31 {x, y}, Delta3 {xxx, xxy, xyy, yyy},
 * Delta42 {xx, xy, yy}.  Returns failed cells.
 */
int orc_tne(const orc_params *p, const double *f, double *out)
{
    const size_t plane = (size_t)p->nx * p->ny;
    double vx[NV], vy[NV], eta[NV];
    orc_velocity_set(p->vg, p->eg, vx, vy, eta);
    int bad = 0;
    set_threads(p);
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long c = 0; c < (long)plane; ++c) {
        double fc[NV], feq[NV], rho, ux, uy, T, M[NV * NV];
        for (int i = 0; i < NV; ++i) fc[i] = f[i * plane + c];
        orc_cell_macros(p, fc, &rho, &ux, &uy, &T);
        if (orc_feq(p, rho, ux, uy, T, feq) != 0) bad += 1;
        orc_central_matrix(vx, vy, eta, ux, uy, M);
        for (int k = 4; k < NV; ++k) {
            double acc = 0.0;
            for (int i = 0; i < NV; ++i) acc += (fc[i] - feq[i]) * M[k * NV + i];
            out[(k - 4) * plane + c] = acc;
        }
    }
    return bad;
}

/* Domain totals of rho, rho u_x, rho u_y and total energy sum f (v^2 + eta^2). */
void orc_conserved_sums(const orc_params *p, const double *f, double out[4])
{
    const size_t plane = (size_t)p->nx * p->ny;
    double vx[NV], vy[NV], eta[NV];
    orc_velocity_set(p->vg, p->eg, vx, vy, eta);
    for (int k = 0; k < 4; ++k) out[k] = 0.0;
    for (size_t c = 0; c < plane; ++c) {
        for (int i = 0; i < NV; ++i) {
            double fi = f[i * plane + c];
            out[0] += fi;
            out[1] += fi * vx[i];
            out[2] += fi * vy[i];
            out[3] += fi * (vx[i] * vx[i] + vy[i] * vy[i] + eta[i] * eta[i]);
        }
    }
}
