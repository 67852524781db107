/*
 * pic_oracle.c -- plain, slow, FP64 CPU reference of the electrostatic
 * particle-in-cell cycle.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the package's smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  It shares no code,
 * header, table or constant with the CUDA path and must never be used as a
 * fallback for it.
 *
 * What it follows (AlgoPlasma paper):
 *   Sec. 2.2  module roles: B_Scatter deposits charge on the grid, C_Gather
 *             interpolates the grid field to particles, D_Poisson solves the
 *             Poisson equation and evaluates E, A_Pusher advances velocities
 *             with the Boris scheme.
 *   Sec. 3.1  the worked example's cycle (Listing 1): load, update the field
 *             (deposit -> Poisson -> potential -> E), initial half push of the
 *             velocities, then per step: full velocity push (gather + Boris),
 *             position update with periodic boundaries, field update.
 * Where the paper is silent, the readings are: node-centred periodic grid,
 * linear (cloud-in-cell) weights shared by deposit and gather, second-order
 * (2d+1)-point Laplacian, centred-difference E, Jacobi-preconditioned CG,
 * backward half push with step -dt/2, x == L wraps to 0.
 *
 * Units are Debye units with eps0 = 1: the field equation is
 *   -lap(phi) = rho,   E = -grad(phi).
 *
 * Layout: grid arrays are flat with axis 0 fastest,
 *   node(j0, j1, j2) = j0 + n0 * (j1 + n1 * j2);
 * vector fields are stored component-major (E[a * cells + node]).
 * Particle positions x are row-major (np x ndim), velocities (np x nv).
 * Every loop is a plain sequential loop; nothing is blocked or reordered.
 * Threading (optional, orc_set_threads): the particle loops of the deposit,
 * gather, pushers, move and kinetic energy split [0, np) into T contiguous
 * ranges, one per thread, each running the same sequential loop; the deposit
 * gives each thread a private rho and sums the copies in thread order, the
 * kinetic energy adds the per-range sums in range order, so results are
 * deterministic for a given T (T = 1, the default, is the sequential code).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int64_t cells_of(int ndim, const int *n)
{
    int64_t c = 1;
    for (int a = 0; a < ndim; ++a) c *= n[a];
    return c;
}

static int64_t node_index(const int *n, const int *j)
{
    return (int64_t)j[0] + (int64_t)n[0] * ((int64_t)j[1] + (int64_t)n[1] * (int64_t)j[2]);
}

/* ---- optional threading of the particle loops ----------------------------------------- */

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : (n > 1024 ? 1024 : n); }
int orc_get_threads(void) { return g_threads; }

typedef void (*range_fn)(void *ctx, int64_t p0, int64_t p1, int t);

struct range_job {
    range_fn fn;
    void *ctx;
    int64_t p0, p1;
    int t;
};

static void *range_thread(void *arg)
{
    struct range_job *j = (struct range_job *)arg;
    j->fn(j->ctx, j->p0, j->p1, j->t);
    return NULL;
}

/* Threads used for np particles: the setting, but at least 1024 particles each. */
static int threads_for(int64_t np)
{
    int64_t t = g_threads;
    if (t > np / 1024) t = np / 1024;
    return t < 1 ? 1 : (int)t;
}

/* fn over [0, np) in T contiguous ranges [t np / T, (t + 1) np / T), range t on
 * thread t (range 0 on the caller).  A thread that cannot be started runs its
 * range on the caller after the others were started. */
static void run_ranges(int64_t np, int T, range_fn fn, void *ctx)
{
    if (T <= 1) {
        fn(ctx, 0, np, 0);
        return;
    }
    pthread_t th[1024];
    int started[1024];
    struct range_job jobs[1024];
    for (int t = 0; t < T; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].p0 = np * t / T;
        jobs[t].p1 = np * (t + 1) / T;
        jobs[t].t = t;
        started[t] = 0;
    }
    for (int t = 1; t < T; ++t) started[t] = pthread_create(&th[t], NULL, range_thread, &jobs[t]) == 0;
    range_thread(&jobs[0]);
    for (int t = 1; t < T; ++t)
        if (!started[t]) range_thread(&jobs[t]);
    for (int t = 1; t < T; ++t)
        if (started[t]) pthread_join(th[t], NULL);
}

/* Cell and in-cell offset of one position: c = floor(x / dx), f = x / dx - c.
 * A position that rounds onto x / dx == n (x at L) belongs to node 0. */
static void locate_one(int ndim, const int *n, const double *dx, const double *x,
                       int *c, double *f)
{
    for (int a = 0; a < 3; ++a) { c[a] = 0; f[a] = 0.0; }
    for (int a = 0; a < ndim; ++a) {
        double u = x[a] / dx[a];
        double fl = floor(u);
        int ca = (int)fl;
        double fa = u - fl;
        if (ca >= n[a] || ca < 0) { ca = 0; fa = 0.0; }  /* x rounding onto L is x = 0 */
        c[a] = ca;
        f[a] = fa;
    }
}

/* Linear cell index and offsets of every particle. */
void orc_locate(int ndim, const int *n, const double *dx, int64_t np, const double *x,
                int64_t *cell, double *off)
{
    for (int64_t p = 0; p < np; ++p) {
        int c[3];
        double f[3];
        locate_one(ndim, n, dx, x + p * ndim, c, f);
        cell[p] = node_index(n, c);
        for (int a = 0; a < ndim; ++a) off[p * ndim + a] = f[a];
    }
}

/* Cloud-in-cell weight of corner s (bit a of s selects the upper node on
 * axis a): product over axes of (1 - f_a) or f_a. */
static double cic_weight(int ndim, const double *f, int s)
{
    double w = 1.0;
    for (int a = 0; a < ndim; ++a) w *= ((s >> a) & 1) ? f[a] : (1.0 - f[a]);
    return w;
}

static int64_t corner_node(int ndim, const int *n, const int *c, int s)
{
    int j[3] = {0, 0, 0};
    for (int a = 0; a < ndim; ++a) {
        j[a] = c[a] + ((s >> a) & 1);
        if (j[a] == n[a]) j[a] = 0;
    }
    return node_index(n, j);
}

/* B_Scatter (Sec. 2.2; module B01 in Sec. 3.1): electron charge density on
 * the nodes, rho_e[j] = (q w / dV) * sum_p W_j(x_p), with W the CIC weights.
 * rho is overwritten. */
static void deposit_serial(int ndim, const int *n, const double *dx, int64_t np,
                           const double *x, double qw, double *rho)
{
    int64_t cells = cells_of(ndim, n);
    double dV = 1.0;
    for (int a = 0; a < ndim; ++a) dV *= dx[a];
    double scale = qw / dV;
    memset(rho, 0, (size_t)cells * sizeof(double));
    for (int64_t p = 0; p < np; ++p) {
        int c[3];
        double f[3];
        locate_one(ndim, n, dx, x + p * ndim, c, f);
        for (int s = 0; s < (1 << ndim); ++s)
            rho[corner_node(ndim, n, c, s)] += scale * cic_weight(ndim, f, s);
    }
}

/* C_Gather (Sec. 2.2; module C01 in Sec. 3.1): field at each particle,
 * Ep[p][a] = sum_j W_j(x_p) E_a[j], with the same weights as the deposit. */
static void gather_serial(int ndim, const int *n, const double *dx, int64_t np,
                          const double *x, const double *E, double *Ep)
{
    int64_t cells = cells_of(ndim, n);
    for (int64_t p = 0; p < np; ++p) {
        int c[3];
        double f[3];
        locate_one(ndim, n, dx, x + p * ndim, c, f);
        for (int a = 0; a < ndim; ++a) Ep[p * ndim + a] = 0.0;
        for (int s = 0; s < (1 << ndim); ++s) {
            int64_t j = corner_node(ndim, n, c, s);
            double w = cic_weight(ndim, f, s);
            for (int a = 0; a < ndim; ++a) Ep[p * ndim + a] += w * E[a * cells + j];
        }
    }
}

/* out = -lap_h(u), the (2d+1)-point periodic Laplacian with sign flipped so
 * that the operator is positive semi-definite. */
void orc_neg_laplacian(int ndim, const int *n, const double *dx, const double *u, double *out)
{
    int n3[3] = {1, 1, 1};
    for (int a = 0; a < ndim; ++a) n3[a] = n[a];
    for (int j2 = 0; j2 < n3[2]; ++j2)
        for (int j1 = 0; j1 < n3[1]; ++j1)
            for (int j0 = 0; j0 < n3[0]; ++j0) {
                int j[3] = {j0, j1, j2};
                int64_t id = node_index(n3, j);
                double acc = 0.0;
                for (int a = 0; a < ndim; ++a) {
                    int jp[3] = {j0, j1, j2}, jm[3] = {j0, j1, j2};
                    jp[a] = (j[a] + 1) % n3[a];
                    jm[a] = (j[a] - 1 + n3[a]) % n3[a];
                    acc += (2.0 * u[id] - u[node_index(n3, jp)] - u[node_index(n3, jm)]) /
                           (dx[a] * dx[a]);
                }
                out[id] = acc;
            }
}

static double dot(int64_t m, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
}

/* D_Poisson (Sec. 2.2; module D02 in Sec. 3.1): solve -lap_h(phi) = rho on the
 * periodic grid.  The singular periodic problem is made consistent by
 * removing the mean of rho, and phi is returned with zero mean.  Jacobi-
 * preconditioned conjugate gradients from phi = 0, stopping when
 * ||r||_2 <= rtol ||b||_2 or after maxit iterations.  Returns 0 on
 * convergence, 1 otherwise; iterations and final relative residual through
 * the pointers. */
int orc_poisson_pcg(int ndim, const int *n, const double *dx, const double *rho, double *phi,
                    double rtol, int maxit, int *iters, double *relres)
{
    int64_t m = cells_of(ndim, n);
    double *b = malloc((size_t)m * sizeof(double));
    double *r = malloc((size_t)m * sizeof(double));
    double *z = malloc((size_t)m * sizeof(double));
    double *p = malloc((size_t)m * sizeof(double));
    double *q = malloc((size_t)m * sizeof(double));
    double mean = 0.0;
    for (int64_t i = 0; i < m; ++i) mean += rho[i];
    mean /= (double)m;
    for (int64_t i = 0; i < m; ++i) b[i] = rho[i] - mean;

    double diag = 0.0;  /* Jacobi preconditioner: the operator's (constant) diagonal */
    for (int a = 0; a < ndim; ++a) diag += 2.0 / (dx[a] * dx[a]);

    for (int64_t i = 0; i < m; ++i) { phi[i] = 0.0; r[i] = b[i]; }
    double bnorm = sqrt(dot(m, b, b));
    int k = 0, status = 0;
    double rel = 0.0;
    if (bnorm > 0.0) {
        for (int64_t i = 0; i < m; ++i) { z[i] = r[i] / diag; p[i] = z[i]; }
        double rz = dot(m, r, z);
        rel = 1.0;
        status = 1;
        while (k < maxit) {
            orc_neg_laplacian(ndim, n, dx, p, q);
            double alpha = rz / dot(m, p, q);
            for (int64_t i = 0; i < m; ++i) { phi[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
            ++k;
            rel = sqrt(dot(m, r, r)) / bnorm;
            if (rel <= rtol) { status = 0; break; }
            for (int64_t i = 0; i < m; ++i) z[i] = r[i] / diag;
            double rz_new = dot(m, r, z);
            double beta = rz_new / rz;
            rz = rz_new;
            for (int64_t i = 0; i < m; ++i) p[i] = z[i] + beta * p[i];
        }
        double pm = 0.0;
        for (int64_t i = 0; i < m; ++i) pm += phi[i];
        pm /= (double)m;
        for (int64_t i = 0; i < m; ++i) phi[i] -= pm;
    }
    if (iters) *iters = k;
    if (relres) *relres = rel;
    free(b); free(r); free(z); free(p); free(q);
    return status;
}

/* D06 (Sec. 3.1): E = -grad(phi) by periodic centred differences,
 * E_a[j] = -(phi[j + e_a] - phi[j - e_a]) / (2 dx_a). */
void orc_efield(int ndim, const int *n, const double *dx, const double *phi, double *E)
{
    int n3[3] = {1, 1, 1};
    for (int a = 0; a < ndim; ++a) n3[a] = n[a];
    int64_t cells = cells_of(ndim, n);
    for (int j2 = 0; j2 < n3[2]; ++j2)
        for (int j1 = 0; j1 < n3[1]; ++j1)
            for (int j0 = 0; j0 < n3[0]; ++j0) {
                int j[3] = {j0, j1, j2};
                int64_t id = node_index(n3, j);
                for (int a = 0; a < ndim; ++a) {
                    int jp[3] = {j0, j1, j2}, jm[3] = {j0, j1, j2};
                    jp[a] = (j[a] + 1) % n3[a];
                    jm[a] = (j[a] - 1 + n3[a]) % n3[a];
                    E[a * cells + id] = -(phi[node_index(n3, jp)] - phi[node_index(n3, jm)]) /
                                        (2.0 * dx[a]);
                }
            }
}

/* A_Pusher, Boris scheme (Sec. 2.2; module A01 in Sec. 3.1), one velocity
 * advance by the step h for every particle:
 *   v- = v + (q/m) E h/2
 *   t  = (q/m) B h/2,  v' = v- + v- x t,  s = 2 t / (1 + |t|^2),  v+ = v- + v' x s
 *   v  = v+ + (q/m) E h/2
 * E is the gathered grid field (ndim components per particle) plus the
 * uniform external E0; B is the uniform B0.  Velocity components beyond nv
 * enter as zero and are not stored back.  With B = 0 this is the leapfrog
 * kick v += (q/m) E h. */
static void boris_serial(int ndim, int nv, int64_t np, double *v, const double *Ep,
                         const double *E0, const double *B0, double qm, double h)
{
    double t[3], tt = 0.0;
    for (int a = 0; a < 3; ++a) { t[a] = qm * B0[a] * 0.5 * h; tt += t[a] * t[a]; }
    double s[3];
    for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + tt);
    for (int64_t p = 0; p < np; ++p) {
        double E[3], u[3];
        for (int a = 0; a < 3; ++a) {
            E[a] = E0[a] + (a < ndim && Ep ? Ep[p * ndim + a] : 0.0);
            u[a] = a < nv ? v[p * nv + a] : 0.0;
        }
        double vm[3], vp[3], w[3];
        for (int a = 0; a < 3; ++a) vm[a] = u[a] + qm * E[a] * 0.5 * h;
        w[0] = vm[0] + (vm[1] * t[2] - vm[2] * t[1]);
        w[1] = vm[1] + (vm[2] * t[0] - vm[0] * t[2]);
        w[2] = vm[2] + (vm[0] * t[1] - vm[1] * t[0]);
        vp[0] = vm[0] + (w[1] * s[2] - w[2] * s[1]);
        vp[1] = vm[1] + (w[2] * s[0] - w[0] * s[2]);
        vp[2] = vm[2] + (w[0] * s[1] - w[1] * s[0]);
        for (int a = 0; a < nv && a < 3; ++a) v[p * nv + a] = vp[a] + qm * E[a] * 0.5 * h;
    }
}

/* Higuera-Cary advance (A_Pusher, Sec. 2.2, the relativistic pusher the paper
 * cites besides Boris) of the momentum per mass u = gamma v by a step h, with
 * eps = (q/m) h / 2, tau = eps B and 1/c^2 = inv_c2 (0: the non-relativistic limit):
 *   u- = u + eps E
 *   sigma = gamma-^2 - tau^2,  gamma-^2 = 1 + |u-|^2 / c^2
 *   gamma_bar^2 = (sigma + sqrt(sigma^2 + 4 (tau^2 + (u- . tau)^2 / c^2))) / 2
 *   t = tau / gamma_bar,  s = 1 / (1 + t . t)
 *   u+ = s (u- + (u- . t) t + u- x t)
 *   u = u+ + eps E + u+ x t
 * gamma_bar is the Lorentz factor of the mean momentum (u- + u+) / 2, so the
 * rotation is the implicit midpoint one, u+ - u- = (u- + u+) x tau / gamma_bar. */
static void hc_serial(int ndim, int nv, int64_t np, double *u, const double *Ep,
                      const double *E0, const double *B0, double qm, double h, double inv_c2)
{
    const double eps = 0.5 * qm * h;
    double tau[3], tau2 = 0.0;
    for (int a = 0; a < 3; ++a) { tau[a] = eps * B0[a]; tau2 += tau[a] * tau[a]; }
    for (int64_t p = 0; p < np; ++p) {
        double E[3], um[3], up[3], t[3];
        for (int a = 0; a < 3; ++a) {
            E[a] = E0[a] + (a < ndim && Ep ? Ep[p * ndim + a] : 0.0);
            um[a] = (a < nv ? u[p * nv + a] : 0.0) + eps * E[a];
        }
        const double um2 = um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
        const double ustar = um[0] * tau[0] + um[1] * tau[1] + um[2] * tau[2];
        const double sigma = 1.0 + um2 * inv_c2 - tau2;
        const double gbar = sqrt(0.5 * (sigma + sqrt(sigma * sigma +
                                                     4.0 * (tau2 + ustar * ustar * inv_c2))));
        double tt = 0.0;
        for (int a = 0; a < 3; ++a) { t[a] = tau[a] / gbar; tt += t[a] * t[a]; }
        const double s = 1.0 / (1.0 + tt);
        const double ut = um[0] * t[0] + um[1] * t[1] + um[2] * t[2];
        up[0] = s * (um[0] + ut * t[0] + (um[1] * t[2] - um[2] * t[1]));
        up[1] = s * (um[1] + ut * t[1] + (um[2] * t[0] - um[0] * t[2]));
        up[2] = s * (um[2] + ut * t[2] + (um[0] * t[1] - um[1] * t[0]));
        const double un[3] = {up[0] + eps * E[0] + (up[1] * t[2] - up[2] * t[1]),
                              up[1] + eps * E[1] + (up[2] * t[0] - up[0] * t[2]),
                              up[2] + eps * E[2] + (up[0] * t[1] - up[1] * t[0])};
        for (int a = 0; a < nv && a < 3; ++a) u[p * nv + a] = un[a];
    }
}

/* Relativistic kinetic energy m w sum (gamma - 1) c^2 = m w sum |u|^2 / (gamma + 1)
 * (the second form has no cancellation; at inv_c2 = 0 it is (1/2) m w sum |u|^2). */
double orc_kinetic_rel(int nv, int64_t np, const double *u, double mw, double inv_c2)
{
    double s = 0.0;
    for (int64_t p = 0; p < np; ++p) {
        double u2 = 0.0;
        for (int a = 0; a < nv; ++a) u2 += u[p * nv + a] * u[p * nv + a];
        s += u2 / (sqrt(1.0 + u2 * inv_c2) + 1.0);
    }
    return mw * s;
}

/* Position update with periodic boundaries (application code in Sec. 3.1):
 * x_a += v_a dt on the ndim spatial axes, then x_a -= L_a floor(x_a / L_a);
 * a result that rounds to L_a is set to 0. */
static void move_serial(int ndim, const int *n, const double *dx, int nv, int64_t np,
                        double *x, const double *v, double dt)
{
    for (int64_t p = 0; p < np; ++p)
        for (int a = 0; a < ndim; ++a) {
            double L = n[a] * dx[a];
            double xa = x[p * ndim + a] + v[p * nv + a] * dt;
            xa -= L * floor(xa / L);
            if (xa >= L || xa < 0.0) xa = 0.0;
            x[p * ndim + a] = xa;
        }
}

/* ---- public particle loops (sequential, or threaded over particle ranges) -------------- */

struct deposit_ctx {
    int ndim;
    const int *n;
    const double *dx, *x;
    double qw;
    double **buf;
};

static void deposit_range(void *c, int64_t p0, int64_t p1, int t)
{
    struct deposit_ctx *d = (struct deposit_ctx *)c;
    deposit_serial(d->ndim, d->n, d->dx, p1 - p0, d->x + p0 * d->ndim, d->qw, d->buf[t]);
}

/* B_Scatter (Sec. 2.2; module B01 in Sec. 3.1), see deposit_serial.  With T > 1
 * threads each range deposits into its own copy of rho (at most about 1 GB of
 * copies: fewer threads on large grids), summed into rho in thread order. */
void orc_deposit(int ndim, const int *n, const double *dx, int64_t np, const double *x,
                 double qw, double *rho)
{
    int64_t cells = cells_of(ndim, n);
    int T = threads_for(np);
    int64_t cap = ((int64_t)1 << 27) / (cells > 0 ? cells : 1);
    if (T > cap) T = cap < 1 ? 1 : (int)cap;
    if (T <= 1) {
        deposit_serial(ndim, n, dx, np, x, qw, rho);
        return;
    }
    double *bufs[1024];
    bufs[0] = rho;
    for (int t = 1; t < T; ++t) {
        bufs[t] = (double *)malloc((size_t)cells * sizeof(double));
        if (!bufs[t]) {  /* out of memory: the sequential loop */
            for (int k = 1; k < t; ++k) free(bufs[k]);
            deposit_serial(ndim, n, dx, np, x, qw, rho);
            return;
        }
    }
    struct deposit_ctx d = {ndim, n, dx, x, qw, bufs};
    run_ranges(np, T, deposit_range, &d);
    for (int64_t j = 0; j < cells; ++j) {
        double acc = bufs[0][j];
        for (int t = 1; t < T; ++t) acc += bufs[t][j];
        rho[j] = acc;
    }
    for (int t = 1; t < T; ++t) free(bufs[t]);
}

struct gather_ctx {
    int ndim;
    const int *n;
    const double *dx, *x, *E;
    double *Ep;
};

static void gather_range(void *c, int64_t p0, int64_t p1, int t)
{
    struct gather_ctx *g = (struct gather_ctx *)c;
    (void)t;
    gather_serial(g->ndim, g->n, g->dx, p1 - p0, g->x + p0 * g->ndim, g->E, g->Ep + p0 * g->ndim);
}

/* C_Gather (Sec. 2.2; module C01 in Sec. 3.1), see gather_serial. */
void orc_gather(int ndim, const int *n, const double *dx, int64_t np, const double *x,
                const double *E, double *Ep)
{
    struct gather_ctx g = {ndim, n, dx, x, E, Ep};
    run_ranges(np, threads_for(np), gather_range, &g);
}

struct push_ctx {
    int ndim, nv;
    double *v;
    const double *Ep, *E0, *B0;
    double qm, h, inv_c2;
    int hc;
};

static void push_range(void *c, int64_t p0, int64_t p1, int t)
{
    struct push_ctx *q = (struct push_ctx *)c;
    (void)t;
    const double *Ep = q->Ep ? q->Ep + p0 * q->ndim : NULL;
    if (q->hc)
        hc_serial(q->ndim, q->nv, p1 - p0, q->v + p0 * q->nv, Ep, q->E0, q->B0, q->qm, q->h,
                  q->inv_c2);
    else
        boris_serial(q->ndim, q->nv, p1 - p0, q->v + p0 * q->nv, Ep, q->E0, q->B0, q->qm, q->h);
}

/* A_Pusher (Sec. 2.2): Boris, see boris_serial. */
void orc_boris(int ndim, int nv, int64_t np, double *v, const double *Ep, const double *E0,
               const double *B0, double qm, double h)
{
    struct push_ctx q = {ndim, nv, v, Ep, E0, B0, qm, h, 0.0, 0};
    run_ranges(np, threads_for(np), push_range, &q);
}

/* A_Pusher (Sec. 2.2): Higuera-Cary, see hc_serial. */
void orc_hc(int ndim, int nv, int64_t np, double *u, const double *Ep, const double *E0,
            const double *B0, double qm, double h, double inv_c2)
{
    struct push_ctx q = {ndim, nv, u, Ep, E0, B0, qm, h, inv_c2, 1};
    run_ranges(np, threads_for(np), push_range, &q);
}

struct move_ctx {
    int ndim, nv;
    const int *n;
    const double *dx;
    double *x;
    const double *v;
    double dt;
};

static void move_range(void *c, int64_t p0, int64_t p1, int t)
{
    struct move_ctx *m = (struct move_ctx *)c;
    (void)t;
    move_serial(m->ndim, m->n, m->dx, m->nv, p1 - p0, m->x + p0 * m->ndim, m->v + p0 * m->nv,
                m->dt);
}

/* Position update with periodic boundaries, see move_serial. */
void orc_move(int ndim, const int *n, const double *dx, int nv, int64_t np, double *x,
              const double *v, double dt)
{
    struct move_ctx m = {ndim, nv, n, dx, x, v, dt};
    run_ranges(np, threads_for(np), move_range, &m);
}

/* Brick-major sort key of a cell: the grid is tiled by bricks of
 * b0 x b1 x b2 cells (the last brick on an axis may be partial); the key is
 *   brick_id * (b0 b1 b2) + local_id,
 *   brick_id = B0 + nb0 * (B1 + nb1 * B2),  B_a = c_a / b_a, nb_a = ceil(n_a / b_a),
 *   local_id = l0 + b0 * (l1 + b1 * l2),    l_a = c_a mod b_a.
 * The ordering of particles by this key is the per-cell sort. */
void orc_sort_key(int ndim, const int *n, const int *brick, int64_t np, const int64_t *cell,
                  int64_t *key)
{
    int n3[3] = {1, 1, 1}, b3[3] = {1, 1, 1};
    for (int a = 0; a < ndim; ++a) { n3[a] = n[a]; b3[a] = brick[a]; }
    int64_t nb[3];
    for (int a = 0; a < 3; ++a) nb[a] = (n3[a] + b3[a] - 1) / b3[a];
    int64_t bcells = (int64_t)b3[0] * b3[1] * b3[2];
    for (int64_t p = 0; p < np; ++p) {
        int64_t c = cell[p];
        int64_t ca[3];
        ca[0] = c % n3[0];
        ca[1] = (c / n3[0]) % n3[1];
        ca[2] = c / ((int64_t)n3[0] * n3[1]);
        int64_t bid = ca[0] / b3[0] + nb[0] * (ca[1] / b3[1] + nb[1] * (ca[2] / b3[2]));
        int64_t lid = ca[0] % b3[0] + b3[0] * (ca[1] % b3[1] + (int64_t)b3[1] * (ca[2] % b3[2]));
        key[p] = bid * bcells + lid;
    }
}

/* Stable counting sort: perm[r] = index of the particle of rank r when
 * particles are ordered by key, ties kept in input order.  Keys lie in
 * [0, nkeys).  Returns 0, or 1 if a key is out of range. */
int orc_counting_sort(int64_t np, const int64_t *key, int64_t nkeys, int64_t *perm)
{
    int64_t *start = calloc((size_t)nkeys + 1, sizeof(int64_t));
    for (int64_t p = 0; p < np; ++p) {
        if (key[p] < 0 || key[p] >= nkeys) { free(start); return 1; }
        start[key[p] + 1] += 1;
    }
    for (int64_t k = 0; k < nkeys; ++k) start[k + 1] += start[k];
    for (int64_t p = 0; p < np; ++p) perm[start[key[p]]++] = p;
    free(start);
    return 0;
}

/* Diagnostics (Sec. 3.2, the energy balance): kinetic energy
 * (1/2) m w sum_p |v_p|^2 over nv components. */
static double sum_squares(int64_t m, const double *v)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += v[i] * v[i];
    return s;
}

struct ke_ctx {
    int nv;
    const double *v;
    double part[1024];
};

static void ke_range(void *c, int64_t p0, int64_t p1, int t)
{
    struct ke_ctx *k = (struct ke_ctx *)c;
    k->part[t] = sum_squares((p1 - p0) * k->nv, k->v + p0 * k->nv);
}

/* Kinetic energy (1/2) m w sum_p |v_p|^2 (threaded: per-range sums added in range
 * order). */
double orc_kinetic(int nv, int64_t np, const double *v, double mw)
{
    const int T = threads_for(np);
    if (T <= 1) return 0.5 * mw * sum_squares(np * nv, v);
    struct ke_ctx k;
    k.nv = nv;
    k.v = v;
    run_ranges(np, T, ke_range, &k);
    double s = 0.0;
    for (int t = 0; t < T; ++t) s += k.part[t];
    return 0.5 * mw * s;
}

/* Field energy (1/2) dV sum_j |E_j|^2. */
double orc_field_energy(int ndim, const int *n, const double *dx, const double *E)
{
    int64_t cells = cells_of(ndim, n);
    double dV = 1.0;
    for (int a = 0; a < ndim; ++a) dV *= dx[a];
    double s = 0.0;
    for (int64_t i = 0; i < cells * ndim; ++i) s += E[i] * E[i];
    return 0.5 * dV * s;
}

/* Total momentum m w sum_p v_p, per component (nv of them). */
void orc_momentum(int nv, int64_t np, const double *v, double mw, double *out)
{
    for (int a = 0; a < nv; ++a) out[a] = 0.0;
    for (int64_t p = 0; p < np; ++p)
        for (int a = 0; a < nv; ++a) out[a] += v[p * nv + a];
    for (int a = 0; a < nv; ++a) out[a] *= mw;
}

/* ---- null-collision Monte Carlo (G_collision, Sec. 2.2, after Vahedi and Surendra) --------- */

/* Counter-based uniform numbers: the output function of SplitMix64 (Steele, Lea and
 * Flood 2014) applied to seed + (counter + 1) * 0x9E3779B97F4A7C15, counter =
 * step * 2^34 + id * 4 + k; the draw is the top 24 bits. */
uint32_t orc_rng24(uint64_t seed, uint64_t step, uint64_t id, int k)
{
    const uint64_t ctr = (step << 34) | (id << 2) | (uint64_t)k;
    uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)(z >> 40);
}

/* out[i] = draw k of particle id0 + i at step (for statistical checks). */
void orc_rng24_fill(uint64_t seed, uint64_t step, uint64_t id0, int64_t n, int k, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_rng24(seed, step, id0 + (uint64_t)i, k);
}

/* The candidate threshold of the null-collision method: a particle is a candidate
 * when its first draw r0 < round(P 2^24), P = 1 - exp(-nu' dt), nu' = n_g (sig_el +
 * sig_exc) vmax the bounding total collision frequency. */
uint32_t orc_mcc_threshold(double ng, double sig_el, double sig_exc, double vmax, double dt)
{
    const double nu_max = ng * (sig_el + sig_exc) * vmax;
    const double P = 1.0 - exp(-nu_max * dt);
    return (uint32_t)floor(P * 16777216.0 + 0.5);
}

/* One null-collision step of the electrons (3 velocity components, ids `id`) against
 * a uniform neutral background of density ng with constant cross sections: elastic
 * sig_el (isotropic, recoil loss 2 m/M per unit of 1 - cos chi) and excitation
 * sig_exc above the threshold energy eps_exc (the electron loses eps_exc, then
 * scatters isotropically).  For a candidate (draw 0 below the threshold) draw 1,
 * u1 = r1 / 2^24, selects elastic if u1 < nu_el / nu', excitation if
 * u1 < (nu_el + nu_exc) / nu', else a null collision; nu_j = ng sig_j |v|.  Draws 2
 * and 3 give the scattering angles: cos chi = 1 - 2 u2 with u2 = (r2 + 1/2) / 2^24,
 * phi = 2 pi u3 with u3 = r3 / 2^24; the new direction is
 * vhat cos chi + sin chi (e1 cos phi + e2 sin phi) with (e1, e2) the orthonormal
 * basis perpendicular to vhat of Duff et al. (2017).  counts: elastic, excitation,
 * candidates whose frequency exceeded nu'. */
void orc_mcc(int64_t np, double *v, const uint32_t *id, uint64_t step, uint64_t seed,
             double ng, double sig_el, double sig_exc, double eps_exc, double mass_ratio,
             double vmax, double m, double dt, int64_t *counts)
{
    const uint32_t thr = orc_mcc_threshold(ng, sig_el, sig_exc, vmax, dt);
    const double nu_max = ng * (sig_el + sig_exc) * vmax;
    const double inv24 = 1.0 / 16777216.0;
    for (int64_t p = 0; p < np; ++p) {
        if (orc_rng24(seed, step, id[p], 0) >= thr) continue;
        double *vp = v + 3 * p;
        const double v2 = vp[0] * vp[0] + vp[1] * vp[1] + vp[2] * vp[2];
        const double speed = sqrt(v2);
        const double energy = 0.5 * m * v2;
        const double nu_el = ng * sig_el * speed;
        const double nu_exc = energy >= eps_exc ? ng * sig_exc * speed : 0.0;
        if (nu_el + nu_exc > nu_max) counts[2] += 1;
        const double u1 = (double)orc_rng24(seed, step, id[p], 1) * inv24;
        double snew;
        if (u1 < nu_el / nu_max) {
            const double u2 = ((double)orc_rng24(seed, step, id[p], 2) + 0.5) * inv24;
            const double cchi = 1.0 - 2.0 * u2;
            snew = speed * sqrt(1.0 - 2.0 * mass_ratio * (1.0 - cchi));
            counts[0] += 1;
        } else if (u1 < (nu_el + nu_exc) / nu_max) {
            const double s2 = v2 - 2.0 * eps_exc / m;
            snew = sqrt(s2 > 0.0 ? s2 : 0.0);
            counts[1] += 1;
        } else {
            continue;  /* null collision */
        }
        const double u2 = ((double)orc_rng24(seed, step, id[p], 2) + 0.5) * inv24;
        const double u3 = (double)orc_rng24(seed, step, id[p], 3) * inv24;
        const double cchi = 1.0 - 2.0 * u2;
        const double schi = sqrt(1.0 - cchi * cchi > 0.0 ? 1.0 - cchi * cchi : 0.0);
        const double phi = 6.283185307179586476925 * u3;  /* 2 pi u3 */
        double n[3] = {1.0, 0.0, 0.0};
        if (speed > 0.0) {
            n[0] = vp[0] / speed;
            n[1] = vp[1] / speed;
            n[2] = vp[2] / speed;
        }
        const double sgn = n[2] >= 0.0 ? 1.0 : -1.0;
        const double a = -1.0 / (sgn + n[2]);
        const double b = n[0] * n[1] * a;
        const double e1[3] = {1.0 + sgn * n[0] * n[0] * a, sgn * b, -sgn * n[0]};
        const double e2[3] = {b, sgn + n[1] * n[1] * a, -n[1]};
        const double cp = cos(phi), sp = sin(phi);
        for (int k = 0; k < 3; ++k)
            vp[k] = snew * (n[k] * cchi + schi * (e1[k] * cp + e2[k] * sp));
    }
}

/* ---- electromagnetic step (E_Maxwell, Sec. 2.2): periodic 2D3V Yee grid ------------------ */
/* Arrays hold three components, component-major ([3][n0 n1]); element (i, j) of a
 * component sits at ((i + sx) dx, (j + sy) dy) with the Yee offsets
 *   Ex (1/2, 0), Ey (0, 1/2), Ez (0, 0);  Bx (0, 1/2), By (1/2, 0), Bz (1/2, 1/2);
 * J is staggered like E, rho lives on the nodes.  Units: eps0 = 1, mu0 = 1 / c^2. */
static const double EM_SX[6] = {0.5, 0.0, 0.0, 0.0, 0.5, 0.5};
static const double EM_SY[6] = {0.0, 0.5, 0.0, 0.5, 0.0, 0.5};

static int64_t at2(const int *n, int i, int j)
{
    i %= n[0];
    if (i < 0) i += n[0];
    j %= n[1];
    if (j < 0) j += n[1];
    return (int64_t)i + (int64_t)n[0] * j;
}

/* Faraday: B -= h curl E (h = dt / 2 for each half of the split B update). */
void orc_yee_b(const int *n, const double *dx, const double *E, double *B, double h)
{
    const int64_t cells = (int64_t)n[0] * n[1];
    const double *Ex = E, *Ey = E + cells, *Ez = E + 2 * cells;
    double *Bx = B, *By = B + cells, *Bz = B + 2 * cells;
    for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
            const int64_t c = at2(n, i, j);
            Bx[c] -= h * (Ez[at2(n, i, j + 1)] - Ez[c]) / dx[1];
            By[c] += h * (Ez[at2(n, i + 1, j)] - Ez[c]) / dx[0];
            Bz[c] -= h * ((Ey[at2(n, i + 1, j)] - Ey[c]) / dx[0] -
                          (Ex[at2(n, i, j + 1)] - Ex[c]) / dx[1]);
        }
}

/* Ampere: E += dt (c^2 curl B - J). */
void orc_yee_e(const int *n, const double *dx, const double *B, const double *J, double c2,
               double dt, double *E)
{
    const int64_t cells = (int64_t)n[0] * n[1];
    const double *Bx = B, *By = B + cells, *Bz = B + 2 * cells;
    double *Ex = E, *Ey = E + cells, *Ez = E + 2 * cells;
    for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
            const int64_t c = at2(n, i, j);
            const double cx = (Bz[c] - Bz[at2(n, i, j - 1)]) / dx[1];
            const double cy = -(Bz[c] - Bz[at2(n, i - 1, j)]) / dx[0];
            const double cz = (By[c] - By[at2(n, i - 1, j)]) / dx[0] -
                              (Bx[c] - Bx[at2(n, i, j - 1)]) / dx[1];
            Ex[c] += dt * (c2 * cx - J[c]);
            Ey[c] += dt * (c2 * cy - J[cells + c]);
            Ez[c] += dt * (c2 * cz - J[2 * cells + c]);
        }
}

/* Discrete divergence of E at the nodes, (Ex(i+1/2) - Ex(i-1/2)) / dx + (Ey(j+1/2) - Ey(j-1/2)) / dy. */
void orc_yee_div_e(const int *n, const double *dx, const double *E, double *div)
{
    const int64_t cells = (int64_t)n[0] * n[1];
    for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
            const int64_t c = at2(n, i, j);
            div[c] = (E[c] - E[at2(n, i - 1, j)]) / dx[0] +
                     (E[cells + c] - E[cells + at2(n, i, j - 1)]) / dx[1];
        }
}

/* Divergence of B at the cell centres (i+1/2, j+1/2) (its z part vanishes in 2D). */
void orc_yee_div_b(const int *n, const double *dx, const double *B, double *div)
{
    const int64_t cells = (int64_t)n[0] * n[1];
    for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
            const int64_t c = at2(n, i, j);
            div[c] = (B[at2(n, i + 1, j)] - B[c]) / dx[0] +
                     (B[cells + at2(n, i, j + 1)] - B[cells + c]) / dx[1];
        }
}

/* E and B at the particles (np x 6: Ex Ey Ez Bx By Bz), CIC on each component's
 * own staggered lattice. */
void orc_em_gather(const int *n, const double *dx, int64_t np, const double *x, const double *E,
                   const double *B, double *out)
{
    const int64_t cells = (int64_t)n[0] * n[1];
    for (int64_t p = 0; p < np; ++p)
        for (int k = 0; k < 6; ++k) {
            const double *F = (k < 3 ? E : B) + (int64_t)(k % 3) * cells;
            const double u = x[2 * p] / dx[0] - EM_SX[k], w = x[2 * p + 1] / dx[1] - EM_SY[k];
            const double iu = floor(u), iw = floor(w);
            const double fu = u - iu, fw = w - iw;
            const int i0 = (int)iu, j0 = (int)iw;
            out[6 * p + k] = (1.0 - fw) * ((1.0 - fu) * F[at2(n, i0, j0)] + fu * F[at2(n, i0 + 1, j0)]) +
                             fw * ((1.0 - fu) * F[at2(n, i0, j0 + 1)] + fu * F[at2(n, i0 + 1, j0 + 1)]);
        }
}

/* Boris with per-particle fields EB (np x 6), velocities np x 3. */
void orc_boris_eb(int64_t np, double *v, const double *EB, double qm, double h)
{
    for (int64_t p = 0; p < np; ++p) {
        const double *e = EB + 6 * p, *b = EB + 6 * p + 3;
        double t[3], s[3], tt = 0.0, vm[3], w[3];
        for (int a = 0; a < 3; ++a) { t[a] = 0.5 * qm * h * b[a]; tt += t[a] * t[a]; }
        for (int a = 0; a < 3; ++a) { s[a] = 2.0 * t[a] / (1.0 + tt); vm[a] = v[3 * p + a] + 0.5 * qm * h * e[a]; }
        w[0] = vm[0] + (vm[1] * t[2] - vm[2] * t[1]);
        w[1] = vm[1] + (vm[2] * t[0] - vm[0] * t[2]);
        w[2] = vm[2] + (vm[0] * t[1] - vm[1] * t[0]);
        const double vp[3] = {vm[0] + (w[1] * s[2] - w[2] * s[1]), vm[1] + (w[2] * s[0] - w[0] * s[2]),
                              vm[2] + (w[0] * s[1] - w[1] * s[0])};
        for (int a = 0; a < 3; ++a) v[3 * p + a] = vp[a] + 0.5 * qm * h * e[a];
    }
}

static double cic1(double d)
{
    const double a = fabs(d);
    return a < 1.0 ? 1.0 - a : 0.0;
}

/* Charge-conserving current of particles moving from x0 to x1 in one step
 * (Esirkepov 2001, 2D3V, CIC shapes); every displacement under one cell per axis
 * (x1 may have wrapped: the displacement is taken modulo the box).  With S0, S1 the
 * node shapes before and after and DS = S1 - S0:
 *   Wx = DSx (S0y + DSy / 2),  Wy = DSy (S0x + DSx / 2),
 *   Wz = S0x S0y + DSx S0y / 2 + S0x DSy / 2 + DSx DSy / 3,
 *   Jx(i+1/2, j) = -(qw / (dy dt)) sum_{i' <= i} Wx(i', j),
 *   Jy(i, j+1/2) = -(qw / (dx dt)) sum_{j' <= j} Wy(i, j'),
 *   Jz(i, j) = qw vz Wz(i, j) / (dx dy),
 * added into J ([3][cells], staggered like E), so that rho1 - rho0 + dt div J = 0. */
void orc_esirkepov(const int *n, const double *dx, int64_t np, const double *x0,
                   const double *x1, const double *vz, double qw, double dt, double *J)
{
    const int64_t cells = (int64_t)n[0] * n[1];
    const double L[2] = {n[0] * dx[0], n[1] * dx[1]};
    for (int64_t p = 0; p < np; ++p) {
        double u0[2], u1[2];
        int base[2];
        double S0[2][4], DS[2][4];
        for (int a = 0; a < 2; ++a) {
            double d = x1[2 * p + a] - x0[2 * p + a];
            d -= L[a] * floor(d / L[a] + 0.5);  /* the displacement modulo the box */
            u0[a] = x0[2 * p + a] / dx[a];
            u1[a] = u0[a] + d / dx[a];
            base[a] = (int)floor(u0[a]) - 1;
            for (int k = 0; k < 4; ++k) {
                S0[a][k] = cic1(u0[a] - (base[a] + k));
                DS[a][k] = cic1(u1[a] - (base[a] + k)) - S0[a][k];
            }
        }
        const double fx = -qw / (dx[1] * dt), fy = -qw / (dx[0] * dt);
        const double fz = qw * vz[p] / (dx[0] * dx[1]);
        for (int b = 0; b < 4; ++b) {
            double run = 0.0;
            for (int a = 0; a < 4; ++a) {
                run += DS[0][a] * (S0[1][b] + 0.5 * DS[1][b]);
                J[at2(n, base[0] + a, base[1] + b)] += fx * run;
            }
        }
        for (int a = 0; a < 4; ++a) {
            double run = 0.0;
            for (int b = 0; b < 4; ++b) {
                run += DS[1][b] * (S0[0][a] + 0.5 * DS[0][a]);
                J[cells + at2(n, base[0] + a, base[1] + b)] += fy * run;
            }
        }
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a) {
                const double wz = S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b] +
                                  0.5 * S0[0][a] * DS[1][b] + DS[0][a] * DS[1][b] / 3.0;
                J[2 * cells + at2(n, base[0] + a, base[1] + b)] += fz * wz;
            }
    }
}

/* ---- electromagnetic step in 3D (E_Maxwell, Sec. 2.2: FDTD on the Yee lattice) --------------
 * Periodic grid of n0 x n1 x n2 nodes, component-major [3][cells] arrays, element
 * (i, j, k) of a component at ((i + sx) dx, (j + sy) dy, (k + sz) dz) with the Yee
 * offsets
 *   Ex (1/2, 0, 0), Ey (0, 1/2, 0), Ez (0, 0, 1/2);
 *   Bx (0, 1/2, 1/2), By (1/2, 0, 1/2), Bz (1/2, 1/2, 0);
 * J staggered like E.  A field that does not depend on z is the 2D3V lattice above
 * (there Ez and Bz sit at the 2D positions (0, 0) and (1/2, 1/2)). */
static const double EM3_S[6][3] = {{0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
                                   {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};

static int64_t at3(const int *n, int i, int j, int k)
{
    i %= n[0];
    if (i < 0) i += n[0];
    j %= n[1];
    if (j < 0) j += n[1];
    k %= n[2];
    if (k < 0) k += n[2];
    return (int64_t)i + (int64_t)n[0] * ((int64_t)j + (int64_t)n[1] * k);
}

/* Faraday: B -= h curl E, each component of curl E by centred differences of E at
 * the B component's own position. */
void orc_yee3_b(const int *n, const double *dx, const double *E, double *B, double h)
{
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    const double *Ex = E, *Ey = E + cells, *Ez = E + 2 * cells;
    double *Bx = B, *By = B + cells, *Bz = B + 2 * cells;
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                const int64_t c = at3(n, i, j, k);
                const double curl_x = (Ez[at3(n, i, j + 1, k)] - Ez[c]) / dx[1] -
                                      (Ey[at3(n, i, j, k + 1)] - Ey[c]) / dx[2];
                const double curl_y = (Ex[at3(n, i, j, k + 1)] - Ex[c]) / dx[2] -
                                      (Ez[at3(n, i + 1, j, k)] - Ez[c]) / dx[0];
                const double curl_z = (Ey[at3(n, i + 1, j, k)] - Ey[c]) / dx[0] -
                                      (Ex[at3(n, i, j + 1, k)] - Ex[c]) / dx[1];
                Bx[c] -= h * curl_x;
                By[c] -= h * curl_y;
                Bz[c] -= h * curl_z;
            }
}

/* Ampere: E += dt (c^2 curl B - J), curl B by centred differences at the E positions. */
void orc_yee3_e(const int *n, const double *dx, const double *B, const double *J, double c2,
                double dt, double *E)
{
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    const double *Bx = B, *By = B + cells, *Bz = B + 2 * cells;
    double *Ex = E, *Ey = E + cells, *Ez = E + 2 * cells;
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                const int64_t c = at3(n, i, j, k);
                const double cx = (Bz[c] - Bz[at3(n, i, j - 1, k)]) / dx[1] -
                                  (By[c] - By[at3(n, i, j, k - 1)]) / dx[2];
                const double cy = (Bx[c] - Bx[at3(n, i, j, k - 1)]) / dx[2] -
                                  (Bz[c] - Bz[at3(n, i - 1, j, k)]) / dx[0];
                const double cz = (By[c] - By[at3(n, i - 1, j, k)]) / dx[0] -
                                  (Bx[c] - Bx[at3(n, i, j - 1, k)]) / dx[1];
                Ex[c] += dt * (c2 * cx - J[c]);
                Ey[c] += dt * (c2 * cy - J[cells + c]);
                Ez[c] += dt * (c2 * cz - J[2 * cells + c]);
            }
}

/* div E at the nodes and div B at the cell centres (i+1/2, j+1/2, k+1/2). */
void orc_yee3_div_e(const int *n, const double *dx, const double *E, double *div)
{
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                const int64_t c = at3(n, i, j, k);
                div[c] = (E[c] - E[at3(n, i - 1, j, k)]) / dx[0] +
                         (E[cells + c] - E[cells + at3(n, i, j - 1, k)]) / dx[1] +
                         (E[2 * cells + c] - E[2 * cells + at3(n, i, j, k - 1)]) / dx[2];
            }
}

void orc_yee3_div_b(const int *n, const double *dx, const double *B, double *div)
{
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                const int64_t c = at3(n, i, j, k);
                div[c] = (B[at3(n, i + 1, j, k)] - B[c]) / dx[0] +
                         (B[cells + at3(n, i, j + 1, k)] - B[cells + c]) / dx[1] +
                         (B[2 * cells + at3(n, i, j, k + 1)] - B[2 * cells + c]) / dx[2];
            }
}

/* E and B at the particles (np x 6: Ex Ey Ez Bx By Bz), trilinear CIC on each
 * component's own staggered lattice; x is np x 3. */
void orc_em3_gather(const int *n, const double *dx, int64_t np, const double *x, const double *E,
                    const double *B, double *out)
{
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    for (int64_t p = 0; p < np; ++p)
        for (int q = 0; q < 6; ++q) {
            const double *F = (q < 3 ? E : B) + (int64_t)(q % 3) * cells;
            int i0[3];
            double f[3];
            for (int a = 0; a < 3; ++a) {
                const double u = x[3 * p + a] / dx[a] - EM3_S[q][a];
                const double iu = floor(u);
                i0[a] = (int)iu;
                f[a] = u - iu;
            }
            double s = 0.0;
            for (int corner = 0; corner < 8; ++corner) {
                const int b0 = corner & 1, b1 = (corner >> 1) & 1, b2 = corner >> 2;
                const double w = (b0 ? f[0] : 1.0 - f[0]) * (b1 ? f[1] : 1.0 - f[1]) *
                                 (b2 ? f[2] : 1.0 - f[2]);
                s += w * F[at3(n, i0[0] + b0, i0[1] + b1, i0[2] + b2)];
            }
            out[6 * p + q] = s;
        }
}

/* Charge-conserving current of particles moving from x0 to x1 in one step (Esirkepov
 * 2001, 3D, CIC shapes); every displacement under one cell per axis, taken modulo the
 * box.  With S0, S1 the node shapes before and after per axis and DS = S1 - S0,
 *   Wx = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3), and cyclically,
 *   Jx(i+1/2, j, k) = -(qw / (dy dz dt)) sum_{i' <= i} Wx(i', j, k), and cyclically,
 * added into J ([3][cells], staggered like E), so that rho1 - rho0 + dt div J = 0. */
void orc_esirkepov3(const int *n, const double *dx, int64_t np, const double *x0,
                    const double *x1, double qw, double dt, double *J)
{
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    const double L[3] = {n[0] * dx[0], n[1] * dx[1], n[2] * dx[2]};
    for (int64_t p = 0; p < np; ++p) {
        double S0[3][4], DS[3][4];
        int base[3];
        for (int a = 0; a < 3; ++a) {
            double d = x1[3 * p + a] - x0[3 * p + a];
            d -= L[a] * floor(d / L[a] + 0.5);
            const double u0 = x0[3 * p + a] / dx[a], u1 = u0 + d / dx[a];
            base[a] = (int)floor(u0) - 1;
            for (int k = 0; k < 4; ++k) {
                S0[a][k] = cic1(u0 - (base[a] + k));
                DS[a][k] = cic1(u1 - (base[a] + k)) - S0[a][k];
            }
        }
        /* axis a's current: prefix sums along a of W_a, for each node of the other two */
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            const double fa = -qw / (dx[b] * dx[c] * dt);
            for (int kb = 0; kb < 4; ++kb)
                for (int kc = 0; kc < 4; ++kc) {
                    const double perp = S0[b][kb] * S0[c][kc] + 0.5 * DS[b][kb] * S0[c][kc] +
                                        0.5 * S0[b][kb] * DS[c][kc] +
                                        DS[b][kb] * DS[c][kc] / 3.0;
                    double run = 0.0;
                    for (int ka = 0; ka < 4; ++ka) {
                        run += DS[a][ka] * perp;
                        int idx[3];
                        idx[a] = base[a] + ka;
                        idx[b] = base[b] + kb;
                        idx[c] = base[c] + kc;
                        J[(int64_t)a * cells + at3(n, idx[0], idx[1], idx[2])] += fa * run;
                    }
                }
        }
    }
}

/* ---- convolutional PML (E_Maxwell, Sec. 2.2, the CPML the paper cites: Roden and
 * Gedney 2000) on a 2D Yee grid with a perfectly conducting wall behind it -------------- */
/* Non-periodic grid of n0 x n1 nodes; the Yee offsets as above; the tangential E on the
 * outer nodes is held at zero (Ez on all four sides, Ex on j = 0 and n1 - 1, Ey on
 * i = 0 and n0 - 1) and values outside the grid count as zero.  Inside the layers
 * every derivative d/da of the update becomes (1 / kappa_a) d/da + psi, with
 *   psi <- b psi + c (dF/da),   b = exp(-(sigma / kappa + alpha) h),
 *   c = sigma (b - 1) / (sigma kappa + kappa^2 alpha)   (0 where sigma = 0),
 * h the step of that update.  The profiles (b, c, 1 / kappa) are given per axis at
 * integer positions (index i = position i) and half positions (index i = i + 1/2),
 * separately for the E update (h = dt) and the B half updates (h = dt / 2).  psi
 * arrays (all [cells]): for B: Bx_y, By_x, Bz_x, Bz_y; for E: Ex_y, Ey_x, Ez_x, Ez_y. */
static double pec_get(const double *F, const int *n, int i, int j)
{
    if (i < 0 || j < 0 || i >= n[0] || j >= n[1]) return 0.0;
    return F[(int64_t)i + (int64_t)n[0] * j];
}

void orc_cpml_b(const int *n, const double *dx, const double *E, double *B, double h,
                const double *const *prof, double *const *psi)
{
    /* prof: [0] bx_half, [1] cx_half, [2] ikx_half, [3] by_half, [4] cy_half, [5] iky_half */
    const int64_t cells = (int64_t)n[0] * n[1];
    const double *Ex = E, *Ey = E + cells, *Ez = E + 2 * cells;
    double *Bx = B, *By = B + cells, *Bz = B + 2 * cells;
    for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
            const int64_t c = (int64_t)i + (int64_t)n[0] * j;
            const double dyEz = (pec_get(Ez, n, i, j + 1) - Ez[c]) / dx[1];
            const double dxEz = (pec_get(Ez, n, i + 1, j) - Ez[c]) / dx[0];
            const double dxEy = (pec_get(Ey, n, i + 1, j) - Ey[c]) / dx[0];
            const double dyEx = (pec_get(Ex, n, i, j + 1) - Ex[c]) / dx[1];
            psi[0][c] = prof[3][j] * psi[0][c] + prof[4][j] * dyEz;
            psi[1][c] = prof[0][i] * psi[1][c] + prof[1][i] * dxEz;
            psi[2][c] = prof[0][i] * psi[2][c] + prof[1][i] * dxEy;
            psi[3][c] = prof[3][j] * psi[3][c] + prof[4][j] * dyEx;
            Bx[c] -= h * (prof[5][j] * dyEz + psi[0][c]);
            By[c] += h * (prof[2][i] * dxEz + psi[1][c]);
            Bz[c] -= h * ((prof[2][i] * dxEy + psi[2][c]) - (prof[5][j] * dyEx + psi[3][c]));
        }
}

void orc_cpml_e(const int *n, const double *dx, const double *B, const double *J, double c2,
                double dt, double *E, const double *const *prof, double *const *psi)
{
    /* prof: [0] bx_int, [1] cx_int, [2] ikx_int, [3] by_int, [4] cy_int, [5] iky_int */
    const int64_t cells = (int64_t)n[0] * n[1];
    const double *Bx = B, *By = B + cells, *Bz = B + 2 * cells;
    double *Ex = E, *Ey = E + cells, *Ez = E + 2 * cells;
    for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
            const int64_t c = (int64_t)i + (int64_t)n[0] * j;
            const double dyBz = (Bz[c] - pec_get(Bz, n, i, j - 1)) / dx[1];
            const double dxBz = (Bz[c] - pec_get(Bz, n, i - 1, j)) / dx[0];
            const double dxBy = (By[c] - pec_get(By, n, i - 1, j)) / dx[0];
            const double dyBx = (Bx[c] - pec_get(Bx, n, i, j - 1)) / dx[1];
            psi[0][c] = prof[3][j] * psi[0][c] + prof[4][j] * dyBz;
            psi[1][c] = prof[0][i] * psi[1][c] + prof[1][i] * dxBz;
            psi[2][c] = prof[0][i] * psi[2][c] + prof[1][i] * dxBy;
            psi[3][c] = prof[3][j] * psi[3][c] + prof[4][j] * dyBx;
            Ex[c] += dt * (c2 * (prof[5][j] * dyBz + psi[0][c]) - J[c]);
            Ey[c] += dt * (-c2 * (prof[2][i] * dxBz + psi[1][c]) - J[cells + c]);
            Ez[c] += dt * (c2 * ((prof[2][i] * dxBy + psi[2][c]) - (prof[5][j] * dyBx + psi[3][c])) -
                           J[2 * cells + c]);
        }
    /* the conducting wall: tangential E on the outer nodes */
    for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
            const int64_t c = (int64_t)i + (int64_t)n[0] * j;
            const int xb = i == 0 || i == n[0] - 1, yb = j == 0 || j == n[1] - 1;
            if (xb || yb) Ez[c] = 0.0;
            if (yb || i == n[0] - 1) Ex[c] = 0.0;
            if (xb || j == n[1] - 1) Ey[c] = 0.0;
        }
}

/* ---- particles on the non-periodic grid (the CPML mode) ---------------------------------
 * Particles live in the box [0, (n0 - 1) dx) x [0, (n1 - 1) dy) between the walls.  The
 * gather, the current and the charge use the periodic forms above with every node
 * outside the grid left out (a field value there counts as zero, a contribution to it
 * is dropped).  A particle whose move leaves the box deposits the current of its whole
 * move (what falls outside the grid is dropped) and is then absorbed by the caller. */
void orc_em_gather_np(const int *n, const double *dx, int64_t np, const double *x,
                      const double *E, const double *B, double *out)
{
    const int64_t cells = (int64_t)n[0] * n[1];
    for (int64_t p = 0; p < np; ++p)
        for (int k = 0; k < 6; ++k) {
            const double *F = (k < 3 ? E : B) + (int64_t)(k % 3) * cells;
            const double u = x[2 * p] / dx[0] - EM_SX[k], w = x[2 * p + 1] / dx[1] - EM_SY[k];
            const double iu = floor(u), iw = floor(w);
            const double fu = u - iu, fw = w - iw;
            const int i0 = (int)iu, j0 = (int)iw;
            out[6 * p + k] = (1.0 - fw) * ((1.0 - fu) * pec_get(F, n, i0, j0) +
                                           fu * pec_get(F, n, i0 + 1, j0)) +
                             fw * ((1.0 - fu) * pec_get(F, n, i0, j0 + 1) +
                                   fu * pec_get(F, n, i0 + 1, j0 + 1));
        }
}

static void add_np(double *F, const int *n, int i, int j, double v)
{
    if (i < 0 || j < 0 || i >= n[0] || j >= n[1]) return;
    F[(int64_t)i + (int64_t)n[0] * j] += v;
}

void orc_esirkepov_np(const int *n, const double *dx, int64_t np, const double *x0,
                      const double *x1, const double *vz, double qw, double dt, double *J)
{
    const int64_t cells = (int64_t)n[0] * n[1];
    for (int64_t p = 0; p < np; ++p) {
        double S0[2][4], DS[2][4];
        int base[2];
        for (int a = 0; a < 2; ++a) {
            const double u0 = x0[2 * p + a] / dx[a], u1 = x1[2 * p + a] / dx[a];
            base[a] = (int)floor(u0) - 1;
            for (int k = 0; k < 4; ++k) {
                S0[a][k] = cic1(u0 - (base[a] + k));
                DS[a][k] = cic1(u1 - (base[a] + k)) - S0[a][k];
            }
        }
        const double fx = -qw / (dx[1] * dt), fy = -qw / (dx[0] * dt);
        const double fz = qw * vz[p] / (dx[0] * dx[1]);
        for (int b = 0; b < 4; ++b) {
            double run = 0.0;
            for (int a = 0; a < 4; ++a) {
                run += DS[0][a] * (S0[1][b] + 0.5 * DS[1][b]);
                add_np(J, n, base[0] + a, base[1] + b, fx * run);
            }
        }
        for (int a = 0; a < 4; ++a) {
            double run = 0.0;
            for (int b = 0; b < 4; ++b) {
                run += DS[1][b] * (S0[0][a] + 0.5 * DS[0][a]);
                add_np(J + cells, n, base[0] + a, base[1] + b, fy * run);
            }
        }
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a) {
                const double wz = S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b] +
                                  0.5 * S0[0][a] * DS[1][b] + DS[0][a] * DS[1][b] / 3.0;
                add_np(J + 2 * cells, n, base[0] + a, base[1] + b, fz * wz);
            }
    }
}

/* CIC charge density (qw / (dx dy) per particle) on the nodes of the non-periodic grid. */
void orc_deposit_np(const int *n, const double *dx, int64_t np, const double *x, double qw,
                    double *rho)
{
    const int64_t cells = (int64_t)n[0] * n[1];
    for (int64_t c = 0; c < cells; ++c) rho[c] = 0.0;
    const double s = qw / (dx[0] * dx[1]);
    for (int64_t p = 0; p < np; ++p) {
        const double u = x[2 * p] / dx[0], w = x[2 * p + 1] / dx[1];
        const double iu = floor(u), iw = floor(w);
        const double fu = u - iu, fw = w - iw;
        const int i0 = (int)iu, j0 = (int)iw;
        add_np(rho, n, i0, j0, s * (1.0 - fu) * (1.0 - fw));
        add_np(rho, n, i0 + 1, j0, s * fu * (1.0 - fw));
        add_np(rho, n, i0, j0 + 1, s * (1.0 - fu) * fw);
        add_np(rho, n, i0 + 1, j0 + 1, s * fu * fw);
    }
}
