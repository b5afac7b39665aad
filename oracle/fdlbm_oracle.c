/*
 * CPU oracle for the T2S2-FDLBM D2Q9 step (Chen, Chai, Wang, Shi,
 * "A finite-difference lattice Boltzmann model with second-order accuracy of
 * time and space for incompressible flow", arXiv 1911.12913).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct FP64
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Style: whole-field passes in the order of the paper's computational sequence
 * (Sec. 2D, Steps 1-3), one formula per loop, no fusion, no blocking.  Every
 * function names the equation it follows.  Readings of passages that are silent
 * or garbled in the paper:
 *   - the blend weight `beta` multiplies the second-order UPWIND difference,
 *     D_m = (1-beta) D_c + beta D_u (Eq. 2.36 prints the weights the other way
 *     round; the symbol of Eq. 4.8 and the errors of Table 1 fit this reading).
 *     `beta_is_central = 1` selects the literal print (tests only);
 *   - the c < 0 branch of the upwind difference (Eq. 2.38) is the mirror image
 *     of the c >= 0 branch;
 *   - on a stretched tensor-product grid, d/dx = (d zeta/dx) d/d zeta with the
 *     differences of Eqs. 2.37-2.38 taken in the unit-spaced index coordinate;
 *   - the force terms of Eqs. 2.20, 2.32, 2.34 are kept in every transform, and
 *     the moment of the half-step variable is rho u = sum xi fbar + (h/2) rho F
 *     (the analogue of Eq. 3.3 for the variable of Eq. 2.31);
 *   - walls use the non-equilibrium extrapolation of Eq. 3.10 with the density
 *     of the nearest interior node; the intermediate f* at wall nodes is set the
 *     same way; interior nodes whose upwind stencil would leave the domain use
 *     the central difference alone;
 *   - `incomp = 1` swaps Eq. 3.2 for the incompressible equilibrium of He and
 *     Luo, which Sec. 2 says may be used with both schemes but does not print:
 *     f_i^eq = w_i [rho + rho0 (xi.u / cs^2 + ((xi.u)^2 - cs^2 u.u) / (2 cs^4))],
 *     whose first moment is rho0 u.  Accordingly the velocity is read from
 *     rho0 u = sum xi f + shift rho0 F (Eq. 3.3 with rho0 for rho), and the
 *     forcing term of Eq. 3.12 takes the equilibrium at rho0, so that it adds
 *     no mass and the momentum rho0 F per unit time.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Value type of distributions and fields.  The default build uses real_t; the
 * ORACLE_COMPLEX build runs the identical arithmetic on complex numbers, so
 * that a complex-step perturbation (f + i eps v) yields the exact directional
 * derivative Im(step(f + i eps v)) / eps of the step (used by the tests to
 * assemble the step's Jacobian on tiny grids).  Grid metrics, time parameters
 * and wall velocities are real in both builds. */
#ifdef ORACLE_COMPLEX
#include <complex.h>
typedef double complex real_t;
#else
typedef double real_t;
#endif

/* D2Q9 lattice of Sec. 3 with xi = 1: velocity columns and weights, cs^2 = 1/3. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

typedef struct {
    int nx, ny;
    int periodic_x, periodic_y;   /* 1 periodic, 0 walls at both ends */
    const double *mx, *my;        /* d zeta/dx per column, d mu/dy per row (> 0) */
    double tau, dt, A, beta;      /* relaxation time, time step, t* = tn + A dt, upwind weight */
    int beta_is_central;          /* 1: literal Eq. 2.36 (beta weights the central part) */
    int scheme;                   /* 1: T2S2-FDLBM1 (Eq. 2.23), 2: T2S2-FDLBM2 (Eq. 5.23) */
    const real_t *force;          /* [2][ny][nx] body acceleration, or NULL */
    double wall_u[4][2];          /* velocity of the W, E, S, N walls */
    int nthreads;
    int incomp;                   /* 1: incompressible equilibrium of He and Luo */
    double rho0;                  /* its reference density */
} oracle_cfg;

#define IDX(c, x, y) ((size_t)(y) * (size_t)(c)->nx + (size_t)(x))
#define POP(c, i) ((size_t)(i) * (size_t)(c)->nx * (size_t)(c)->ny)

static int nthreads_of(const oracle_cfg *c) { return c->nthreads > 0 ? c->nthreads : 1; }

/* Eq. 3.2: second-order equilibrium. */
void oracle_feq(real_t rho, real_t ux, real_t uy, real_t *feq)
{
    real_t uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        real_t eu = EX[i] * ux + EY[i] * uy;
        /* uu:(xi xi - cs^2 I) = (xi.u)^2 - cs^2 u.u */
        feq[i] = WQ[i] * rho * (1.0 + eu / CS2 + (eu * eu - CS2 * uu) / (2.0 * CS2 * CS2));
    }
}

/* The incompressible equilibrium of He and Luo (cited in Sec. 2, not printed
 * there): Eq. 3.2 with rho0 in place of rho in every velocity term. */
void oracle_feq_incomp(real_t rho, double rho0, real_t ux, real_t uy, real_t *feq)
{
    real_t uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        real_t eu = EX[i] * ux + EY[i] * uy;
        feq[i] = WQ[i] * (rho + rho0 * (eu / CS2 + (eu * eu - CS2 * uu) / (2.0 * CS2 * CS2)));
    }
}

/* The equilibrium of the configured model at (rho, u). */
static void feq_model(const oracle_cfg *c, real_t rho, real_t ux, real_t uy, real_t *feq)
{
    if (c->incomp) oracle_feq_incomp(rho, c->rho0, ux, uy, feq);
    else oracle_feq(rho, ux, uy, feq);
}

/* Eq. 3.12: forcing term F_i = Fbar.(xi_i - u) f_i^eq / RT with RT = cs^2. */
void oracle_force_term(const real_t *feq, real_t ux, real_t uy, real_t Fx, real_t Fy,
                       real_t *F)
{
    for (int i = 0; i < 9; ++i)
        F[i] = ((EX[i] - ux) * Fx + (EY[i] - uy) * Fy) * feq[i] / CS2;
}

static void force_at(const oracle_cfg *c, size_t n, real_t *Fx, real_t *Fy)
{
    size_t N = (size_t)c->nx * c->ny;
    *Fx = c->force ? c->force[n] : 0.0;
    *Fy = c->force ? c->force[N + n] : 0.0;
}

/* Eq. 3.3 applied to a distribution whose first moment lacks `shift * rho * F`:
 * rho = sum f_i, rho u = sum xi_i f_i + shift rho F.  shift = dt/2 for f~,
 * h/2 for fbar (Eq. 2.31), 0 for the physical f. */
static void moments_node(const oracle_cfg *c, const real_t *f, size_t n, double shift,
                         real_t *rho, real_t *ux, real_t *uy)
{
    size_t N = (size_t)c->nx * c->ny;
    real_t r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        real_t v = f[i * N + n];
        r += v;
        jx += EX[i] * v;
        jy += EY[i] * v;
    }
    real_t Fx, Fy;
    force_at(c, n, &Fx, &Fy);
    /* the density that carries the momentum: rho (Eq. 3.3), or rho0 */
    real_t rm = c->incomp ? (real_t)c->rho0 : r;
    jx += shift * rm * Fx;
    jy += shift * rm * Fy;
    *rho = r;
    *ux = jx / rm;
    *uy = jy / rm;
}

/* f^eq of the model and the forcing term of Eq. 3.12 at one node.  The
 * forcing term takes the equilibrium at rho0 under the incompressible model. */
static void node_feq_force(const oracle_cfg *c, size_t n, real_t rho, real_t ux, real_t uy,
                           real_t *fe, real_t *Fi)
{
    real_t Fx, Fy, fF[9];
    feq_model(c, rho, ux, uy, fe);
    force_at(c, n, &Fx, &Fy);
    if (c->incomp) {
        oracle_feq(c->rho0, ux, uy, fF);
        oracle_force_term(fF, ux, uy, Fx, Fy, Fi);
    } else {
        oracle_force_term(fe, ux, uy, Fx, Fy, Fi);
    }
}

/* Eq. 3.3: density and velocity from f~. */
void oracle_moments(const oracle_cfg *c, const real_t *f, real_t *rho, real_t *ux, real_t *uy)
{
    size_t N = (size_t)c->nx * c->ny;
    for (size_t n = 0; n < N; ++n)
        moments_node(c, f, n, 0.5 * c->dt, &rho[n], &ux[n], &uy[n]);
}

/* Initial f~ from the fields (rho, u) and, optionally, the velocity gradient.
 * The physical distribution is f = f^eq (Eq. 3.2), plus the non-equilibrium
 * part of Eq. 3.5 when grad is given (coefficient read as
 * rho0 w_i (2 tau + dt) / (2 cs^2), which already carries the factor
 * 1 + dt/(2 tau) of the change of variables).  The stored variable is then
 * f~ = f - (dt/2) Omega-bar(f) (Eq. 2.19); with a body force Omega-bar holds
 * the forcing term of Eq. 3.12, so f~ = ... - (dt/2) F_i(rho, u), and Eq. 3.3
 * reads back exactly the velocity u that was given.
 * grad = [dudx, dudy, dvdx, dvdy], each [ny][nx]. */
void oracle_init(const oracle_cfg *c, const real_t *rho, const real_t *ux, const real_t *uy,
                 const real_t *grad, double rho0, real_t *f)
{
    size_t N = (size_t)c->nx * c->ny;
    for (size_t n = 0; n < N; ++n) {
        real_t feq[9], Fi[9];
        node_feq_force(c, n, rho[n], ux[n], uy[n], feq, Fi);
        for (int i = 0; i < 9; ++i) {
            real_t v = feq[i] - 0.5 * c->dt * Fi[i];
            if (grad) {
                double xx = EX[i] * EX[i], xy = EX[i] * EY[i], yy = EY[i] * EY[i];
                real_t ddot = xx * grad[n] + xy * (grad[N + n] + grad[2 * N + n]) +
                              yy * grad[3 * N + n];
                v -= rho0 * WQ[i] * (2.0 * c->tau + c->dt) / (2.0 * CS2) * ddot;
            }
            f[i * N + n] = v;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Space discretisation, Eqs. 2.36-2.38, in the index coordinate k (unit step),
 * scaled by the metric.  Returns d f / d chi_alpha for velocity sign `s`.
 * ------------------------------------------------------------------------- */
static int wrap(int k, int n)
{
    while (k < 0) k += n;
    while (k >= n) k -= n;
    return k;
}

static real_t sample(const oracle_cfg *c, const real_t *fld, int x, int y)
{
    if (c->periodic_x) x = wrap(x, c->nx);
    if (c->periodic_y) y = wrap(y, c->ny);
    return fld[IDX(c, x, y)];
}

/* Central difference, Eq. 2.37 (index space). */
static real_t d_central(const oracle_cfg *c, const real_t *f, int x, int y, int ax)
{
    int dx = ax == 0, dy = ax == 1;
    return (sample(c, f, x + dx, y + dy) - sample(c, f, x - dx, y - dy)) / 2.0;
}

/* Second-order upwind difference, Eq. 2.38 (index space), sign s of xi_alpha. */
static real_t d_upwind(const oracle_cfg *c, const real_t *f, int x, int y, int ax, int s)
{
    int dx = ax == 0, dy = ax == 1;
    if (s >= 0)
        return (3.0 * sample(c, f, x, y) - 4.0 * sample(c, f, x - dx, y - dy) +
                sample(c, f, x - 2 * dx, y - 2 * dy)) / 2.0;
    return -(3.0 * sample(c, f, x, y) - 4.0 * sample(c, f, x + dx, y + dy) +
             sample(c, f, x + 2 * dx, y + 2 * dy)) / 2.0;
}

/* Mixed difference, Eq. 2.36, with the metric: d f/d x_alpha at node (x, y). */
static real_t d_mixed(const oracle_cfg *c, const real_t *f, int x, int y, int ax, int s)
{
    double m = ax == 0 ? c->mx[x] : c->my[y];
    int k = ax == 0 ? x : y, n = ax == 0 ? c->nx : c->ny;
    int per = ax == 0 ? c->periodic_x : c->periodic_y;
    real_t dc = d_central(c, f, x, y, ax);
    /* upwind stencil leaves a walled domain: central difference alone */
    int upwind_ok = per || (s >= 0 ? k - 2 >= 0 : k + 2 <= n - 1);
    if (!upwind_ok) return m * dc;
    real_t du = d_upwind(c, f, x, y, ax, s);
    double wu = c->beta_is_central ? 1.0 - c->beta : c->beta;
    return m * ((1.0 - wu) * dc + wu * du);
}

/* Eq. 2.27: L(f_i) = -xi_i . grad f_i, evaluated at one node for population i. */
static real_t advection(const oracle_cfg *c, const real_t *fi, int x, int y, int i)
{
    real_t L = 0.0;
    if (EX[i]) L -= EX[i] * d_mixed(c, fi, x, y, 0, EX[i]);
    if (EY[i]) L -= EY[i] * d_mixed(c, fi, x, y, 1, EY[i]);
    return L;
}

static int is_wall(const oracle_cfg *c, int x, int y)
{
    return (!c->periodic_x && (x == 0 || x == c->nx - 1)) ||
           (!c->periodic_y && (y == 0 || y == c->ny - 1));
}

/* Nearest interior node along the inward normal (diagonal at corners). */
static void wall_partner(const oracle_cfg *c, int x, int y, int *px, int *py, double *uw)
{
    int jx = x, jy = y;
    if (!c->periodic_x) { if (x == 0) jx = 1; else if (x == c->nx - 1) jx = c->nx - 2; }
    if (!c->periodic_y) { if (y == 0) jy = 1; else if (y == c->ny - 1) jy = c->ny - 2; }
    *px = jx;
    *py = jy;
    /* wall velocity: the W/E walls own the corners (a moving lid stops at the side walls) */
    int side = -1;
    if (!c->periodic_x && x == 0) side = 0;
    else if (!c->periodic_x && x == c->nx - 1) side = 1;
    else if (!c->periodic_y && y == 0) side = 2;
    else if (!c->periodic_y && y == c->ny - 1) side = 3;
    uw[0] = side >= 0 ? c->wall_u[side][0] : 0.0;
    uw[1] = side >= 0 ? c->wall_u[side][1] : 0.0;
}

/* Eq. 3.10: non-equilibrium extrapolation onto every wall node of f.
 * `shift` selects the first-moment convention of f (see moments_node).
 * Pinned by the exact wall moments and convergence under refinement; parity
 * with the paper's Poiseuille error magnitudes unpinned. */
static void apply_nee(const oracle_cfg *c, real_t *f, double shift)
{
    size_t N = (size_t)c->nx * c->ny;
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            if (!is_wall(c, x, y)) continue;
            int jx, jy;
            double uw[2];
            wall_partner(c, x, y, &jx, &jy, uw);
            size_t nb = IDX(c, x, y), nj = IDX(c, jx, jy);
            real_t rj, uxj, uyj, feqj[9], feqb[9];
            moments_node(c, f, nj, shift, &rj, &uxj, &uyj);
            feq_model(c, rj, uxj, uyj, feqj);
            feq_model(c, rj, uw[0], uw[1], feqb);
            for (int i = 0; i < 9; ++i)
                f[i * N + nb] = feqb[i] + (f[i * N + nj] - feqj[i]);
        }
}

typedef struct {
    real_t *rho, *ux, *uy, *feq, *F, *fphys, *fbar_plus, *fbar_star, *fstar, *ftil_plus, *L;
} work_t;

static int work_alloc(const oracle_cfg *c, work_t *w)
{
    size_t N = (size_t)c->nx * c->ny;
    memset(w, 0, sizeof(*w));
    w->rho = malloc(N * sizeof(real_t));
    w->ux = malloc(N * sizeof(real_t));
    w->uy = malloc(N * sizeof(real_t));
    real_t **big[] = {&w->feq, &w->F, &w->fphys, &w->fbar_plus, &w->fbar_star,
                      &w->fstar, &w->ftil_plus, &w->L};
    for (int k = 0; k < 8; ++k) *big[k] = malloc(9 * N * sizeof(real_t));
    int ok = w->rho && w->ux && w->uy;
    for (int k = 0; k < 8; ++k) ok = ok && *big[k];
    return ok ? 0 : -1;
}

static void work_free(work_t *w)
{
    free(w->rho); free(w->ux); free(w->uy); free(w->feq); free(w->F); free(w->fphys);
    free(w->fbar_plus); free(w->fbar_star); free(w->fstar); free(w->ftil_plus); free(w->L);
}

/* Node-local pass: rho, u (Eq. 3.3), f^eq (Eq. 3.2 or He-Luo), F (Eq. 3.12) of a
 * distribution g whose first moment lacks `shift rho F`. */
static void macro_pass(const oracle_cfg *c, const real_t *g, double shift, work_t *w)
{
    size_t N = (size_t)c->nx * c->ny;
#pragma omp parallel for num_threads(nthreads_of(c)) schedule(static)
    for (long long n = 0; n < (long long)N; ++n) {
        real_t fe[9], Fi[9];
        moments_node(c, g, (size_t)n, shift, &w->rho[n], &w->ux[n], &w->uy[n]);
        node_feq_force(c, (size_t)n, w->rho[n], w->ux[n], w->uy[n], fe, Fi);
        for (int i = 0; i < 9; ++i) {
            w->feq[i * N + n] = fe[i];
            w->F[i * N + n] = Fi[i];
        }
    }
}

/* Eq. 2.20: post-collision f~+ from f~, f^eq, F. */
static void post_collision_pass(const oracle_cfg *c, const real_t *f, work_t *w)
{
    size_t N = (size_t)c->nx * c->ny;
    double tau = c->tau, dt = c->dt;
#pragma omp parallel for num_threads(nthreads_of(c)) schedule(static)
    for (long long k = 0; k < (long long)(9 * N); ++k)
        w->ftil_plus[k] = ((2 * tau - dt) * f[k] + 2 * dt * w->feq[k] + 2 * tau * dt * w->F[k]) /
                          (2 * tau + dt);
}

/* Inverse of Eq. 2.31 for the step s (Eq. 2.32): physical f from the
 * half-variable fb = f - (s/2) Omega-bar. */
static void physical_pass(const oracle_cfg *c, const real_t *fb, double s, work_t *w)
{
    size_t N = (size_t)c->nx * c->ny;
    double tau = c->tau;
#pragma omp parallel for num_threads(nthreads_of(c)) schedule(static)
    for (long long k = 0; k < (long long)(9 * N); ++k)
        w->fphys[k] = (2 * tau * fb[k] + s * w->feq[k] + s * tau * w->F[k]) / (2 * tau + s);
}

/* out = f + (h/2) Omega-bar(f) = (1 - h/2tau) f + (h/2tau) f^eq + (h/2) F
 * (Eq. 2.34, left-hand definition) for the physical f in w->fphys. */
static void plus_half_pass(const oracle_cfg *c, double h, work_t *w, real_t *out)
{
    size_t N = (size_t)c->nx * c->ny;
    double tau = c->tau;
#pragma omp parallel for num_threads(nthreads_of(c)) schedule(static)
    for (long long k = 0; k < (long long)(9 * N); ++k)
        out[k] = w->fphys[k] - h / (2 * tau) * (w->fphys[k] - w->feq[k]) + 0.5 * h * w->F[k];
}

/* Characteristic estimate, Eqs. 2.33 and 2.35: out = in - h xi_i . grad in
 * at interior nodes (wall nodes are filled later). */
static void characteristic_pass(const oracle_cfg *c, const real_t *in, double h, real_t *out)
{
    size_t N = (size_t)c->nx * c->ny;
    for (int i = 0; i < 9; ++i) {
#pragma omp parallel for num_threads(nthreads_of(c)) schedule(static)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                size_t n = IDX(c, x, y);
                if (is_wall(c, x, y)) { out[i * N + n] = in[i * N + n]; continue; }
                /* -h xi.grad = +h L (Eq. 2.27) */
                out[i * N + n] = in[i * N + n] + h * advection(c, in + i * N, x, y, i);
            }
    }
}

/* Eq. 2.27 with Eq. 2.36 at interior nodes. */
static void advection_pass(const oracle_cfg *c, const real_t *fin, real_t *L)
{
    size_t N = (size_t)c->nx * c->ny;
    for (int i = 0; i < 9; ++i) {
#pragma omp parallel for num_threads(nthreads_of(c)) schedule(static)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                size_t n = IDX(c, x, y);
                L[i * N + n] = is_wall(c, x, y) ? 0.0 : advection(c, fin + i * N, x, y, i);
            }
    }
}

/* One T2S2-FDLBM1 step (Sec. 2D Steps 1-3; A = 0 gives T1S2, Remark I). */
static void step_scheme1(const oracle_cfg *c, real_t *f, work_t *w)
{
    size_t N = (size_t)c->nx * c->ny;
    double dt = c->dt, tau = c->tau, h = c->A * dt;
    /* Step 1a: f~ -> (rho, u, f^eq, F) -> physical f -> fbar^{+,h} (Eqs. 3.3, 2.19, 2.34) */
    macro_pass(c, f, 0.5 * dt, w);
    physical_pass(c, f, dt, w);
    plus_half_pass(c, h, w, w->fbar_plus);
    /* Step 2 (node-local, uses the same f^eq and F): f~+ (Eq. 2.20) */
    post_collision_pass(c, f, w);
    /* Step 1b: fbar(t*) by the characteristic estimate (Eqs. 2.33, 2.35) */
    characteristic_pass(c, w->fbar_plus, h, w->fbar_star);
    /* Step 1c: moments of fbar*, then f* (Eq. 2.52 with the force term of Eq. 2.32) */
    macro_pass(c, w->fbar_star, 0.5 * h, w);
    physical_pass(c, w->fbar_star, h, w);
    memcpy(w->fstar, w->fphys, 9 * N * sizeof(real_t));
    if (!c->periodic_x || !c->periodic_y) apply_nee(c, w->fstar, 0.0);
    /* Step 1d: L(f*) (Eqs. 2.27, 2.36) */
    advection_pass(c, w->fstar, w->L);
    /* Step 3: f~^{n+1} = f~+ + dt L(f*) (Eq. 2.23), then walls (Eq. 3.10) */
    for (size_t k = 0; k < 9 * N; ++k) f[k] = w->ftil_plus[k] + dt * w->L[k];
    if (!c->periodic_x || !c->periodic_y) apply_nee(c, f, 0.5 * dt);
    (void)tau;
}

/* One T2S2-FDLBM2 step (Sec. 2D, second sequence; Eq. 5.23, h = dt).
 * Pinned by the printed FDLBM2 errors of the grid-convergence table of Sec. 3A
 * (small time step), its second-order time convergence and the exact
 * invariants; parity with the printed FDLBM2 errors at large CFL (Table 4)
 * unpinned: no reading of the sequence tried reproduces them. */
static void step_scheme2(const oracle_cfg *c, real_t *f, work_t *w)
{
    size_t N = (size_t)c->nx * c->ny;
    double dt = c->dt;
    /* Step 1: f~ -> f^n (Eq. 2.52 with h = dt) -> L(f^n) */
    macro_pass(c, f, 0.5 * dt, w);
    physical_pass(c, f, dt, w);
    memcpy(w->fstar, w->fphys, 9 * N * sizeof(real_t));
    if (!c->periodic_x || !c->periodic_y) apply_nee(c, w->fstar, 0.0);
    advection_pass(c, w->fstar, w->L);
    /* Step 2: f~ -> f~+ (Eq. 2.20) -> fbar(t_{n+1}) (Eqs. 2.33, 2.35 with h = dt,
     * fbar^{+,h} = f~+) -> f^{n+1} (Eq. 2.52) -> L(f^{n+1}) */
    post_collision_pass(c, f, w);
    characteristic_pass(c, w->ftil_plus, dt, w->fbar_star);
    macro_pass(c, w->fbar_star, 0.5 * dt, w);
    physical_pass(c, w->fbar_star, dt, w);
    if (!c->periodic_x || !c->periodic_y) apply_nee(c, w->fphys, 0.0);
    /* w->fbar_plus is free here: reuse it for L(f^{n+1}) */
    advection_pass(c, w->fphys, w->fbar_plus);
    /* Step 3: Eq. 5.23 */
    for (size_t k = 0; k < 9 * N; ++k)
        f[k] = w->ftil_plus[k] + 0.5 * dt * (w->L[k] + w->fbar_plus[k]);
    if (!c->periodic_x || !c->periodic_y) apply_nee(c, f, 0.5 * dt);
}

/* Advance f~ (layout [9][ny][nx]) by nsteps.  Returns 0, or -1 on allocation failure. */
int oracle_step(const oracle_cfg *c, real_t *f, int nsteps)
{
    work_t w;
    if (work_alloc(c, &w)) { work_free(&w); return -1; }
    for (int s = 0; s < nsteps; ++s) {
        if (c->scheme == 2) step_scheme2(c, f, &w);
        else step_scheme1(c, f, &w);
    }
    work_free(&w);
    return 0;
}

/* T1S2-FDLBM of Guo et al. written directly from Eqs. 2.18-2.20, independent of
 * step_scheme1: f~^{n+1} = f~+ + dt L(f^n), with f^n recovered from f~ by
 * inverting Eq. 2.19. */
int oracle_step_t1s2(const oracle_cfg *c, real_t *f, int nsteps)
{
    size_t N = (size_t)c->nx * c->ny;
    double dt = c->dt, tau = c->tau;
    real_t *fn = malloc(9 * N * sizeof(real_t));
    real_t *fp = malloc(9 * N * sizeof(real_t));
    real_t *rho = malloc(N * sizeof(real_t)), *ux = malloc(N * sizeof(real_t)),
           *uy = malloc(N * sizeof(real_t));
    if (!fn || !fp || !rho || !ux || !uy) {
        free(fn); free(fp); free(rho); free(ux); free(uy);
        return -1;
    }
    for (int s = 0; s < nsteps; ++s) {
        for (size_t n = 0; n < N; ++n) {
            real_t fe[9], Fi[9];
            moments_node(c, f, n, 0.5 * dt, &rho[n], &ux[n], &uy[n]);
            node_feq_force(c, n, rho[n], ux[n], uy[n], fe, Fi);
            for (int i = 0; i < 9; ++i) {
                size_t k = i * N + n;
                /* f~ = f - (dt/2)[-(f - feq)/tau + F]  =>  f = (f~ + dt/(2tau) feq + dt/2 F)/(1 + dt/(2tau)) */
                fn[k] = (f[k] + dt / (2 * tau) * fe[i] + 0.5 * dt * Fi[i]) / (1 + dt / (2 * tau));
                /* f~+ = f + (dt/2) Omega-bar(f) */
                fp[k] = fn[k] - dt / (2 * tau) * (fn[k] - fe[i]) + 0.5 * dt * Fi[i];
            }
        }
        if (!c->periodic_x || !c->periodic_y) apply_nee(c, fn, 0.0);
        for (int i = 0; i < 9; ++i)
            for (int y = 0; y < c->ny; ++y)
                for (int x = 0; x < c->nx; ++x) {
                    size_t k = i * N + IDX(c, x, y);
                    f[k] = fp[k] + (is_wall(c, x, y) ? 0.0 : dt * advection(c, fn + i * N, x, y, i));
                }
        if (!c->periodic_x || !c->periodic_y) apply_nee(c, f, 0.5 * dt);
    }
    free(fn); free(fp); free(rho); free(ux); free(uy);
    return 0;
}

/* Stand-alone difference operators for the tests of Eqs. 2.36-2.38:
 * out[y][x] = d fld / d x_alpha (with metric) at interior nodes, for sign s. */
void oracle_derivative(const oracle_cfg *c, const real_t *fld, int axis, int s, real_t *out)
{
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x)
            out[IDX(c, x, y)] = is_wall(c, x, y) ? 0.0 : d_mixed(c, fld, x, y, axis, s);
}

/* The intermediate quantities of one T2S2 step for inspection by the tests:
 * fbar^{+,h}, fbar*, f*, f~+ and L(f*) (each [9][ny][nx]). */
int oracle_stages(const oracle_cfg *c, const real_t *f, real_t *fbar_plus, real_t *fbar_star,
                  real_t *fstar, real_t *ftil_plus, real_t *L)
{
    size_t N = (size_t)c->nx * c->ny;
    work_t w;
    real_t *tmp = malloc(9 * N * sizeof(real_t));
    if (!tmp || work_alloc(c, &w)) { free(tmp); work_free(&w); return -1; }
    memcpy(tmp, f, 9 * N * sizeof(real_t));
    double h = c->A * c->dt;
    macro_pass(c, tmp, 0.5 * c->dt, &w);
    physical_pass(c, tmp, c->dt, &w);
    plus_half_pass(c, h, &w, w.fbar_plus);
    post_collision_pass(c, tmp, &w);
    characteristic_pass(c, w.fbar_plus, h, w.fbar_star);
    macro_pass(c, w.fbar_star, 0.5 * h, &w);
    physical_pass(c, w.fbar_star, h, &w);
    memcpy(w.fstar, w.fphys, 9 * N * sizeof(real_t));
    if (!c->periodic_x || !c->periodic_y) apply_nee(c, w.fstar, 0.0);
    advection_pass(c, w.fstar, w.L);
    memcpy(fbar_plus, w.fbar_plus, 9 * N * sizeof(real_t));
    memcpy(fbar_star, w.fbar_star, 9 * N * sizeof(real_t));
    memcpy(fstar, w.fstar, 9 * N * sizeof(real_t));
    memcpy(ftil_plus, w.ftil_plus, 9 * N * sizeof(real_t));
    memcpy(L, w.L, 9 * N * sizeof(real_t));
    free(tmp);
    work_free(&w);
    return 0;
}
