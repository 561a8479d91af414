/*
 * FP64 CPU oracle for the checkpointed adjoint-state gradient of acoustic
 * seismic inversion (Kukreja et al., "Combining checkpointing and data
 * compression to accelerate adjoint-based optimization problems").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is loaded by tests/, by
 * __graft_entry__.smoke() and by the cpu_baseline / reference leg of
 * bench.py.  The product library never links, loads or calls it, and it
 * shares no code, header or table with the CUDA path.
 *
 * Everything is written for clarity, not speed: plain loops over the total
 * grid, FP64 throughout, zero Dirichlet values outside the grid handled by
 * explicit bounds tests.  OpenMP is used only on the outer loop of
 * point-wise independent updates, so results do not depend on thread count;
 * every reduction (misfit, receiver sums, dot products) is serial.
 *
 * What the paper fixes (Sec. 6, Eq. "eqn:wave" and the misfit after it):
 *   m u_tt - lap(u) = q,  m = 1/c^2,  phi = 1/2 ||d_sim - d_obs||^2,
 *   gradient by the adjoint-state method, OT2 (2nd order in time) kernel,
 *   and an OT4 kernel (4th order in time) taken from the paper's DSL.
 * What the paper leaves to its DSL and this oracle fixes as a reading:
 *   - Laplacian: 2k-th order central differences, k = so/2, with the
 *     closed-form weights c_j = 2(-1)^(j+1) (k!)^2 / (j^2 (k-j)! (k+j)!),
 *     zero values outside the total grid.
 *   - damping layer of nbl cells on every face, rate
 *     eta = sum over axes of eta_max (delta/L)^2 [1/ms], delta = distance of
 *     the grid point from the first interior point along that axis,
 *     L = nbl*h, eta_max = 3 vmax_damp / (2L) * ln(1/R).  It enters the
 *     equation as  m u_tt + m eta u_t - lap(u) = q  (the unit-consistent
 *     form of a damping rate).
 *   - time stepping (n = 0..N-1, u^0 = u^-1 = 0):
 *       a u^{n+1} = 2 u^n - b u^{n-1} + w (lap u^n + q^n),
 *       w = dt^2 c^2,  a = 1 + eta dt/2,  b = 1 - eta dt/2.
 *   - source / receiver: multilinear weights over the 2^d surrounding grid
 *     points, no 1/h^d factor; q^n = Q^T s^n, d^n = P u^n (n = 0..N).
 *   - misfit over n = 1..N (d^0 = 0 identically).
 *   - adjoint (the exact transpose of the recursion above):
 *       lam^N = lam^{N+1} = 0, for j = N..1:
 *       a lam^{j-1} = 2 lam^j - b lam^{j+1} + w (lap lam^j - P^T r^j)
 *     gradient  dphi/dm = sum_{n=0}^{N-1} lam^n (a u^{n+1} - 2u^n + b u^{n-1})/dt^2
 *                       = sum_{n=0}^{N-1} lam^n (lap u^n + q^n) c^2.
 *   - OT4 (time_order 4): the paper names the kernel and cites its DSL for
 *     it without stating it.  Reading: the modified-equation scheme, which
 *     cancels the leading dt^2/12 u_tttt error of the centred second time
 *     difference by using u_tttt = c^2 lap(c^2 lap u) of the undamped,
 *     source-free equation.  The recursion keeps its form with lap replaced by
 *       A u = lap u + dt^2/12 lap(c^2 lap u)
 *     (the inner field c^2 lap u is zero outside the grid, like u); damping
 *     and sources enter as in OT2.  A is symmetric, so the adjoint is the
 *     same recursion with A, and the exact gradient gains the derivative of
 *     the correction with respect to m = 1/c^2:
 *       dphi/dm = sum_{n=0}^{N-1} [ lam^n (A u^n + q^n) c^2
 *                                  + dt^2/12 c^4 (lap u^n)(lap lam^n) ].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dims;          /* 2 or 3 */
    int nz, ny, nx;    /* total grid incl. damping layer; ny == 1 in 2D */
    int nbl;           /* damping layer width [cells] */
    int so;            /* space order (even) */
    int nt;            /* number of time steps N */
    double h;          /* grid spacing [m] */
    double dt;         /* time step [ms] */
    double vmax_damp;  /* velocity that sets the damping strength [km/s] */
    double refl;       /* target reflection coefficient R of the layer */
    int time_order;    /* 2 (OT2; 0 reads as 2) or 4 (OT4) */
} ora_grid;

enum { ORA_OK = 0, ORA_EINVAL = -1, ORA_ENOMEM = -2 };

static long npts_of(const ora_grid* g) { return (long)g->nz * g->ny * g->nx; }

static int grid_ok(const ora_grid* g)
{
    if (!g) return 0;
    if (g->dims != 2 && g->dims != 3) return 0;
    if (g->nz < 2 || g->nx < 2 || g->ny < 1) return 0;
    if (g->dims == 2 && g->ny != 1) return 0;
    if (g->dims == 3 && g->ny < 2) return 0;
    if (g->so < 2 || (g->so & 1) || g->so > 32) return 0;
    if (g->nt < 1 || !(g->h > 0) || !(g->dt > 0) || g->nbl < 0) return 0;
    if (g->time_order != 0 && g->time_order != 2 && g->time_order != 4) return 0;
    return 1;
}

/* Central-difference weights of the 2k-th order second derivative
 * (closed form of the Fornberg weights).  c[0] = -2 sum_j c[j]. */
int ora_fd_weights(int k, double* c)
{
    if (k < 1 || k > 16 || !c) return ORA_EINVAL;
    double kf = 1.0;
    for (int i = 2; i <= k; ++i) kf *= i;
    double s = 0.0;
    for (int j = 1; j <= k; ++j) {
        double a = 1.0, b = 1.0;
        for (int i = 2; i <= k - j; ++i) a *= i;
        for (int i = 2; i <= k + j; ++i) b *= i;
        double cj = 2.0 * kf * kf / ((double)j * j * a * b);
        if (!(j & 1)) cj = -cj;
        c[j] = cj;
        s += cj;
    }
    c[0] = -2.0 * s;
    return ORA_OK;
}

/* lap(u) with zero values outside the grid. */
int ora_laplacian(const ora_grid* g, const double* u, double* out)
{
    if (!grid_ok(g) || !u || !out) return ORA_EINVAL;
    const int k = g->so / 2;
    double c[17];
    ora_fd_weights(k, c);
    const double ih2 = 1.0 / (g->h * g->h);
    const int nz = g->nz, ny = g->ny, nx = g->nx;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long p = ((long)z * ny + y) * nx + x;
                const double uc = u[p];
                double acc = 0.0;
                for (int j = 1; j <= k; ++j) {
                    /* z axis */
                    double zp = (z + j < nz) ? u[p + (long)j * ny * nx] : 0.0;
                    double zm = (z - j >= 0) ? u[p - (long)j * ny * nx] : 0.0;
                    double xp = (x + j < nx) ? u[p + j] : 0.0;
                    double xm = (x - j >= 0) ? u[p - j] : 0.0;
                    double t = (zp + zm - 2.0 * uc) + (xp + xm - 2.0 * uc);
                    if (g->dims == 3) {
                        double yp = (y + j < ny) ? u[p + (long)j * nx] : 0.0;
                        double ym = (y - j >= 0) ? u[p - (long)j * nx] : 0.0;
                        t += yp + ym - 2.0 * uc;
                    }
                    acc += c[j] * t;
                }
                out[p] = acc * ih2;
            }
    return ORA_OK;
}

/* Damping rate eta [1/ms] at every point of the total grid. */
static double eta_axis(const ora_grid* g, int i, int n)
{
    if (g->nbl <= 0) return 0.0;
    const double L = g->nbl * g->h;
    const double emax = 3.0 * g->vmax_damp / (2.0 * L) * log(1.0 / g->refl);
    double delta = 0.0;
    if (i < g->nbl) delta = (double)(g->nbl - i) * g->h;
    else if (i > n - 1 - g->nbl) delta = (double)(i - (n - 1 - g->nbl)) * g->h;
    double r = delta / L;
    return emax * r * r;
}

int ora_damping(const ora_grid* g, double* eta)
{
    if (!grid_ok(g) || !eta) return ORA_EINVAL;
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                double e = eta_axis(g, z, g->nz) + eta_axis(g, x, g->nx);
                if (g->dims == 3) e += eta_axis(g, y, g->ny);
                eta[((long)z * g->ny + y) * g->nx + x] = e;
            }
    return ORA_OK;
}

/* Ricker wavelet s(t_n), t_n = n dt, n = 0..nt-1 (f0 in kHz, t in ms). */
int ora_ricker(int nt, double dt, double f0, double t0, double amp, double* s)
{
    if (nt < 1 || !s || !(f0 > 0)) return ORA_EINVAL;
    const double pi = 3.14159265358979323846;
    for (int n = 0; n < nt; ++n) {
        double t = n * dt - t0;
        double a = pi * pi * f0 * f0 * t * t;
        s[n] = amp * (1.0 - 2.0 * a) * exp(-a);
    }
    return ORA_OK;
}

/* Multilinear interpolation stencil of a position pos = (z, y, x) [m],
 * measured from the first interior point.  Grid coordinate along an axis:
 * gc = nbl + pos/h, base i0 = min(floor(gc), n-2), fraction f = gc - i0.
 * Writes 2^dims (index, weight) pairs; returns their count or ORA_EINVAL. */
int ora_interp(const ora_grid* g, const double* pos, long* idx, double* wt)
{
    if (!grid_ok(g) || !pos || !idx || !wt) return ORA_EINVAL;
    int ax_n[3] = {g->nz, g->ny, g->nx};
    int i0[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        if (a == 1 && g->dims == 2) continue;
        double gc = g->nbl + pos[a] / g->h;
        if (!(gc >= 0.0) || gc > (double)(ax_n[a] - 1)) return ORA_EINVAL;
        int b = (int)floor(gc);
        if (b > ax_n[a] - 2) b = ax_n[a] - 2;
        i0[a] = b;
        f[a] = gc - b;
    }
    int cnt = 0;
    const int ylim = (g->dims == 3) ? 2 : 1;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < ylim; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dz ? f[0] : 1.0 - f[0]) * (dx ? f[2] : 1.0 - f[2]);
                if (g->dims == 3) w *= dy ? f[1] : 1.0 - f[1];
                idx[cnt] = ((long)(i0[0] + dz) * g->ny + (i0[1] + dy)) * g->nx + (i0[2] + dx);
                wt[cnt] = w;
                ++cnt;
            }
    return cnt;
}

/* ---- shared state of one forward/adjoint problem ---- */
typedef struct {
    const ora_grid* g;
    long np;
    double *ww, *aa, *bb, *c2;        /* per-point coefficients */
    double *t1, *t2;                  /* np scratch values each (OT4 operator) */
    int nsrc, nrec, nstc;             /* stencil size 2^dims */
    long *sidx, *ridx;                /* [nsrc][nstc], [nrec][nstc] */
    double *swt, *rwt;
    const double* sser;               /* [nsrc][nt] */
} problem;

static void problem_free(problem* P)
{
    free(P->ww); free(P->aa); free(P->bb); free(P->c2); free(P->t1); free(P->t2);
    free(P->sidx); free(P->ridx); free(P->swt); free(P->rwt);
}

static int problem_init(problem* P, const ora_grid* g, const double* vel, int nsrc,
                        const double* src_pos, const double* src_series, int nrec,
                        const double* rec_pos)
{
    memset(P, 0, sizeof(*P));
    if (!grid_ok(g) || !vel || nsrc < 0 || nrec < 0) return ORA_EINVAL;
    P->g = g;
    P->np = npts_of(g);
    P->nsrc = nsrc;
    P->nrec = nrec;
    P->nstc = (g->dims == 3) ? 8 : 4;
    P->sser = src_series;
    P->ww = malloc(sizeof(double) * P->np);
    P->aa = malloc(sizeof(double) * P->np);
    P->bb = malloc(sizeof(double) * P->np);
    P->c2 = malloc(sizeof(double) * P->np);
    P->t1 = malloc(sizeof(double) * P->np);
    P->t2 = malloc(sizeof(double) * P->np);
    P->sidx = malloc(sizeof(long) * (nsrc + 1) * P->nstc);
    P->swt = malloc(sizeof(double) * (nsrc + 1) * P->nstc);
    P->ridx = malloc(sizeof(long) * (nrec + 1) * P->nstc);
    P->rwt = malloc(sizeof(double) * (nrec + 1) * P->nstc);
    if (!P->ww || !P->aa || !P->bb || !P->c2 || !P->t1 || !P->t2 || !P->sidx || !P->swt || !P->ridx || !P->rwt) {
        problem_free(P);
        return ORA_ENOMEM;
    }
    if (ora_damping(g, P->aa) != ORA_OK) { problem_free(P); return ORA_EINVAL; }
    for (long p = 0; p < P->np; ++p) {
        double c = vel[p];
        if (!(c > 0) || !isfinite(c)) { problem_free(P); return ORA_EINVAL; }
        double eta = P->aa[p];
        P->c2[p] = c * c;
        P->ww[p] = g->dt * g->dt * c * c;
        P->aa[p] = 1.0 + eta * g->dt / 2.0;
        P->bb[p] = 1.0 - eta * g->dt / 2.0;
    }
    for (int s = 0; s < nsrc; ++s)
        if (ora_interp(g, src_pos + 3 * s, P->sidx + s * P->nstc, P->swt + s * P->nstc) != P->nstc) {
            problem_free(P);
            return ORA_EINVAL;
        }
    for (int r = 0; r < nrec; ++r)
        if (ora_interp(g, rec_pos + 3 * r, P->ridx + r * P->nstc, P->rwt + r * P->nstc) != P->nstc) {
            problem_free(P);
            return ORA_EINVAL;
        }
    return ORA_OK;
}

static int is_ot4(const problem* P) { return P->g->time_order == 4; }

/* The spatial operator of the time step, out = A u:  lap u for OT2,
 * lap u + dt^2/12 lap(c^2 lap u) for OT4.  out must not alias u. */
static void spatial_op(const problem* P, const double* u, double* out)
{
    const ora_grid* g = P->g;
    ora_laplacian(g, u, out);
    if (!is_ot4(P)) return;
    for (long p = 0; p < P->np; ++p) P->t1[p] = P->c2[p] * out[p];
    ora_laplacian(g, P->t1, P->t2);
    const double k = g->dt * g->dt / 12.0;
    for (long p = 0; p < P->np; ++p) out[p] += k * P->t2[p];
}

/* One leapfrog update:  out = (2 cur - b prev + w (lap + src)) / a,
 * where lap already holds lap(cur) plus the injected point sources. */
static void leapfrog(const problem* P, const double* cur, const double* prev,
                     const double* lap, double* out)
{
    const long np = P->np;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < np; ++p)
        out[p] = (2.0 * cur[p] - P->bb[p] * prev[p] + P->ww[p] * lap[p]) / P->aa[p];
}

/* lap += Q^T s^n  (forward source term at step n) */
static void add_sources(const problem* P, int n, double* lap)
{
    if (!P->sser) return;
    for (int s = 0; s < P->nsrc; ++s)
        for (int i = 0; i < P->nstc; ++i)
            lap[P->sidx[s * P->nstc + i]] += P->swt[s * P->nstc + i] * P->sser[(long)s * P->g->nt + n];
}

/* One forward step n of the recursion:  out = u^{n+1} from cur = u^n,
 * prev = u^{n-1} and the source term q^n.  lap: np scratch values. */
static void forward_step(const problem* P, int n, const double* cur, const double* prev,
                         double* lap, double* out)
{
    spatial_op(P, cur, lap);
    add_sources(P, n, lap);
    leapfrog(P, cur, prev, lap, out);
}

/* One reverse step j = N..1 of the adjoint recursion (header):
 * l0 = lam^{j-1} from l1 = lam^j, l2 = lam^{j+1} and the residual row r^j.
 * With grad, adds the gradient term of n = j-1, which reads the forward
 * state un = u^{n}:  lam^n (A u^n + q^n) c^2, and for OT4 also
 * dt^2/12 c^4 lap(u^n) lap(lam^n).  lap, tmp: np scratch values each. */
static void adjoint_step(const problem* P, const double* r, int j, const double* l1, const double* l2,
                         double* l0, const double* un, double* grad, double* lap, double* tmp)
{
    const ora_grid* g = P->g;
    const long np = P->np;
    spatial_op(P, l1, lap);
    for (int rr = 0; rr < P->nrec; ++rr)
        for (int i = 0; i < P->nstc; ++i)
            lap[P->ridx[rr * P->nstc + i]] -= P->rwt[rr * P->nstc + i] * r[(long)j * P->nrec + rr];
    leapfrog(P, l1, l2, lap, l0);
    if (!grad) return;
    const int n = j - 1;
    spatial_op(P, un, tmp);
    add_sources(P, n, tmp);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < np; ++p) grad[p] += l0[p] * tmp[p] * P->c2[p];
    if (is_ot4(P)) {
        /* derivative of the OT4 correction: dt^2/12 c^4 lap u^n lap lam^n */
        const double kk = g->dt * g->dt / 12.0;
        ora_laplacian(g, un, tmp);
        ora_laplacian(g, l0, lap);
        for (long p = 0; p < np; ++p)
            grad[p] += kk * P->c2[p] * P->c2[p] * tmp[p] * lap[p];
    }
}

static void sample(const problem* P, const double* u, double* d_row)
{
    for (int r = 0; r < P->nrec; ++r) {
        double acc = 0.0;
        for (int i = 0; i < P->nstc; ++i) acc += P->rwt[r * P->nstc + i] * u[P->ridx[r * P->nstc + i]];
        d_row[r] = acc;
    }
}

/* Forward modelling.  d: [nt+1][nrec], d[0] = P u^0 = 0.
 * u_final (optional): u^N.  ckpt (optional): every `seg` steps the state
 * pair (u^n, u^{n-1}) for n = 0, seg, 2 seg, ... is written to
 * ckpt[2*(n/seg)] and ckpt[2*(n/seg)+1] (each np values). */
static int forward_run(const problem* P, double* d, double* u_final, double* ckpt, int seg)
{
    const ora_grid* g = P->g;
    const long np = P->np;
    double* a = calloc(np, sizeof(double));   /* u^{n-1} */
    double* b = calloc(np, sizeof(double));   /* u^n */
    double* c = calloc(np, sizeof(double));   /* u^{n+1} */
    double* lap = malloc(sizeof(double) * np);
    if (!a || !b || !c || !lap) { free(a); free(b); free(c); free(lap); return ORA_ENOMEM; }
    if (d) sample(P, b, d);
    for (int n = 0; n < g->nt; ++n) {
        if (ckpt && seg > 0 && n % seg == 0) {
            memcpy(ckpt + (long)(2 * (n / seg)) * np, b, sizeof(double) * np);
            memcpy(ckpt + (long)(2 * (n / seg) + 1) * np, a, sizeof(double) * np);
        }
        forward_step(P, n, b, a, lap, c);
        if (d) sample(P, c, d + (long)(n + 1) * P->nrec);
        double* t = a; a = b; b = c; c = t;
    }
    if (u_final) memcpy(u_final, b, sizeof(double) * np);
    free(a); free(b); free(c); free(lap);
    return ORA_OK;
}

int ora_forward(const ora_grid* g, const double* vel, int nsrc, const double* src_pos,
                const double* src_series, int nrec, const double* rec_pos,
                double* d, double* u_final)
{
    problem P;
    int st = problem_init(&P, g, vel, nsrc, src_pos, src_series, nrec, rec_pos);
    if (st != ORA_OK) return st;
    st = forward_run(&P, d, u_final, NULL, 0);
    problem_free(&P);
    return st;
}

/* One source-free time step:  out = u^{n+1} from cur = u^n, prev = u^{n-1}
 * (the OT2 or OT4 recursion of the grid's time order). */
int ora_step(const ora_grid* g, const double* vel, const double* cur, const double* prev, double* out)
{
    if (!cur || !prev || !out) return ORA_EINVAL;
    problem P;
    int st = problem_init(&P, g, vel, 0, NULL, NULL, 0, NULL);
    if (st != ORA_OK) return st;
    double* lap = malloc(sizeof(double) * P.np);
    if (!lap) { problem_free(&P); return ORA_ENOMEM; }
    spatial_op(&P, cur, lap);
    leapfrog(&P, cur, prev, lap, out);
    free(lap);
    problem_free(&P);
    return ORA_OK;
}

/* Adjoint sweep driven by r ([nt+1][nrec], row 0 unused).
 *  grad   (optional, np): dphi/dm = sum_n lam^n (lap u^n + q^n) c^2
 *  srcadj (optional, [nsrc][nt]): -Q lam^n, n = 0..nt-1, which is the
 *         transpose of the source-to-data map applied to r.
 *  lam0   (optional, np): lam^0.
 * The forward states u^n needed by the gradient are regenerated segment by
 * segment from state pairs stored every `seg` steps (seg <= 0: sqrt rule). */
static int adjoint_run(const problem* P, const double* r, double* grad, double* srcadj,
                       double* lam0, int seg)
{
    const ora_grid* g = P->g;
    const long np = P->np;
    const int N = g->nt;
    if (seg <= 0) {
        seg = (int)ceil(sqrt(2.0 * N));
        if (seg < 1) seg = 1;
    }
    if (seg > N) seg = N;
    const int nck = (N + seg - 1) / seg;
    double* ckpt = NULL;
    double* useg = NULL;
    if (grad) {
        ckpt = malloc(sizeof(double) * np * 2 * (long)nck);
        useg = malloc(sizeof(double) * np * (long)(seg + 1));
        if (!ckpt || !useg) { free(ckpt); free(useg); return ORA_ENOMEM; }
        int st = forward_run(P, NULL, NULL, ckpt, seg);
        if (st != ORA_OK) { free(ckpt); free(useg); return st; }
        memset(grad, 0, sizeof(double) * np);
    }
    double* l2 = calloc(np, sizeof(double));  /* lam^{j+1} */
    double* l1 = calloc(np, sizeof(double));  /* lam^j */
    double* l0 = calloc(np, sizeof(double));  /* lam^{j-1} */
    double* lap = malloc(sizeof(double) * np);
    double* tmp = malloc(sizeof(double) * np);
    if (!l2 || !l1 || !l0 || !lap || !tmp) {
        free(l2); free(l1); free(l0); free(lap); free(tmp); free(ckpt); free(useg);
        return ORA_ENOMEM;
    }
    int j = N;
    for (int k = nck - 1; k >= 0; --k) {
        const int s0 = k * seg;
        const int s1 = (s0 + seg < N) ? s0 + seg : N;   /* segment holds u^{s0..s1-1} */
        if (grad) {
            /* regenerate u^{s0-1} .. u^{s1-1} from the stored pair */
            double* prev = useg;                /* slot 0: u^{s0-1} */
            memcpy(useg + np, ckpt + (long)(2 * k) * np, sizeof(double) * np);   /* u^{s0} */
            memcpy(prev, ckpt + (long)(2 * k + 1) * np, sizeof(double) * np);
            for (int n = s0; n < s1 - 1; ++n) {
                double* cur = useg + (long)(n - s0 + 1) * np;
                forward_step(P, n, cur, cur - np, lap, cur + np);
            }
        }
        for (; j > s0; --j) {
            /* lam^{j-1} from lam^j, lam^{j+1} and -P^T r^j; gradient term of n = j-1 */
            const int n = j - 1;
            const double* un = grad ? useg + (long)(n - s0 + 1) * np : NULL;
            adjoint_step(P, r, j, l1, l2, l0, un, grad, lap, tmp);
            if (srcadj)
                for (int s = 0; s < P->nsrc; ++s) {
                    double acc = 0.0;
                    for (int i = 0; i < P->nstc; ++i) acc += P->swt[s * P->nstc + i] * l0[P->sidx[s * P->nstc + i]];
                    srcadj[(long)s * N + n] = -acc;
                }
            double* t = l2; l2 = l1; l1 = l0; l0 = t;
        }
    }
    if (lam0) memcpy(lam0, l1, sizeof(double) * np);
    free(l2); free(l1); free(l0); free(lap); free(tmp); free(ckpt); free(useg);
    return ORA_OK;
}

int ora_adjoint(const ora_grid* g, const double* vel, int nsrc, const double* src_pos,
                const double* src_series, int nrec, const double* rec_pos, const double* r,
                double* grad, double* srcadj, double* lam0, int seg)
{
    problem P;
    int st = problem_init(&P, g, vel, nsrc, src_pos, src_series, nrec, rec_pos);
    if (st != ORA_OK) return st;
    if (!r) { problem_free(&P); return ORA_EINVAL; }
    st = adjoint_run(&P, r, grad, srcadj, lam0, seg);
    problem_free(&P);
    return st;
}

/* Misfit phi = 1/2 sum_{n=1..N} sum_r (d - dobs)^2, its gradient dphi/dm,
 * and (optionally) the simulated data d_sim [nt+1][nrec]. */
int ora_gradient(const ora_grid* g, const double* vel, int nsrc, const double* src_pos,
                 const double* src_series, int nrec, const double* rec_pos,
                 const double* dobs, double* phi, double* grad, double* d_sim, int seg)
{
    problem P;
    int st = problem_init(&P, g, vel, nsrc, src_pos, src_series, nrec, rec_pos);
    if (st != ORA_OK) return st;
    const long nd = (long)(g->nt + 1) * nrec;
    double* d = malloc(sizeof(double) * (nd > 0 ? nd : 1));
    double* r = malloc(sizeof(double) * (nd > 0 ? nd : 1));
    if (!d || !r) { free(d); free(r); problem_free(&P); return ORA_ENOMEM; }
    st = forward_run(&P, d, NULL, NULL, 0);
    if (st == ORA_OK) {
        double acc = 0.0;
        for (long i = 0; i < nd; ++i) {
            r[i] = (i < nrec) ? 0.0 : d[i] - dobs[i];
            acc += r[i] * r[i];
        }
        if (phi) *phi = 0.5 * acc;
        if (d_sim) memcpy(d_sim, d, sizeof(double) * nd);
        if (grad) st = adjoint_run(&P, r, grad, NULL, NULL, seg);
    }
    free(d); free(r);
    problem_free(&P);
    return st;
}

/* ---- step-level interface ----
 * A problem held between calls, so that a caller can drive single forward
 * and reverse steps in the order a checkpointing schedule prescribes
 * (Sec. 3).  The steps are the ones ora_forward / ora_adjoint run, so a
 * schedule that hands every step its exact inputs reproduces their results
 * bit for bit. */
typedef struct {
    ora_grid g;          /* own copy: problem keeps a pointer to it */
    problem P;
    double* series;      /* own copy of the source series, [nsrc][nt] */
    double *lap, *tmp;   /* np scratch values each */
} ora_handle;

void ora_problem_destroy(void* h)
{
    ora_handle* H = (ora_handle*)h;
    if (!H) return;
    problem_free(&H->P);
    free(H->series); free(H->lap); free(H->tmp);
    free(H);
}

/* Same arguments as ora_forward; NULL on invalid input or no memory. */
void* ora_problem_create(const ora_grid* g, const double* vel, int nsrc, const double* src_pos,
                         const double* src_series, int nrec, const double* rec_pos)
{
    if (!grid_ok(g) || nsrc < 0 || nrec < 0) return NULL;
    if ((nsrc > 0 && !src_pos) || (nrec > 0 && !rec_pos)) return NULL;
    ora_handle* H = calloc(1, sizeof(*H));
    if (!H) return NULL;
    H->g = *g;
    if (src_series && nsrc > 0) {
        H->series = malloc(sizeof(double) * (long)nsrc * g->nt);
        if (!H->series) { free(H); return NULL; }
        memcpy(H->series, src_series, sizeof(double) * (long)nsrc * g->nt);
    }
    if (problem_init(&H->P, &H->g, vel, nsrc, src_pos, H->series, nrec, rec_pos) != ORA_OK) {
        free(H->series);
        free(H);
        return NULL;
    }
    H->lap = malloc(sizeof(double) * H->P.np);
    H->tmp = malloc(sizeof(double) * H->P.np);
    if (!H->lap || !H->tmp) { ora_problem_destroy(H); return NULL; }
    return H;
}

/* out = u^{n+1} from cur = u^n and prev = u^{n-1}, with the source term q^n
 * (0 <= n < nt).  out must not alias cur or prev. */
int ora_problem_fwd_step(void* h, int n, const double* cur, const double* prev, double* out)
{
    ora_handle* H = (ora_handle*)h;
    if (!H || !cur || !prev || !out || n < 0 || n >= H->g.nt) return ORA_EINVAL;
    if (out == cur || out == prev) return ORA_EINVAL;
    forward_step(&H->P, n, cur, prev, H->lap, out);
    return ORA_OK;
}

/* Reverse step j (1 <= j <= nt): l0 = lam^{j-1} from l1 = lam^j,
 * l2 = lam^{j+1} and row j of the residual r ([nt+1][nrec]).  With grad
 * (np values, accumulated), adds the gradient term of n = j-1 read from the
 * forward state un = u^{j-1}.  l0 must not alias l1, l2 or un. */
int ora_problem_adj_step(void* h, const double* r, int j, const double* l1, const double* l2,
                         double* l0, const double* un, double* grad)
{
    ora_handle* H = (ora_handle*)h;
    if (!H || !r || !l1 || !l2 || !l0 || j < 1 || j > H->g.nt) return ORA_EINVAL;
    if (grad && !un) return ORA_EINVAL;
    if (l0 == l1 || l0 == l2 || (un && l0 == un)) return ORA_EINVAL;
    adjoint_step(&H->P, r, j, l1, l2, l0, un, grad, H->lap, H->tmp);
    return ORA_OK;
}
