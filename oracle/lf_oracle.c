/*
 * lf_oracle.c -- plain FP64 CPU oracle of the hybrid lattice-Boltzmann /
 * finite-difference time step of Gonnella, Lamura & Tiribocchi, "Thermal and
 * hydrodynamic effects in the ordering of lamellar fluids" (arXiv:1102.3094),
 * Sec. 2 ("The model").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU library computes.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * table or header with the CUDA library, and the library never calls it.
 *
 * Everything is FP64, site by site, whole field per pass, in the order the
 * paper states the model.  Compile with -ffp-contract=off so that the
 * arithmetic is exactly what is written.
 *
 * Readings of the paper that this file takes (the paper is silent on them):
 *   - Stencils (Sec. 2, "second-order finite-difference scheme"): 5-point /
 *     7-point Laplacian, central first differences, nabla^4 = nabla^2 nabla^2
 *     (stencil 0).  stencil 1 takes every first and second derivative with
 *     the weights of the velocity set instead (isotropic 9-point / 19-point
 *     operators, see iso_grad / iso_lap below).
 *   - Walls (Sec. 2, boundary paragraph): the first and last layer along the
 *     last axis are fluid sites; the wall sits half a spacing outside them.
 *     Neutral wetting and the two conservation conditions (a.grad phi =
 *     a.grad nabla^2 phi = a.grad nabla^4 phi = 0) are imposed by even mirror
 *     reflection of phi, nabla^2 phi, nabla^4 phi, mu and a about that plane.
 *     Tensors reflect with one sign flip per wall-normal index.  The
 *     advective flux phi*u normal to the wall is odd (no flux through it).
 *   - LB wall rule: halfway bounce-back (exact mass conservation), which
 *     stands in for the density-conservation prescription the paper cites.
 *   - Force: F_beta = -d_alpha P_ab with P the phi-dependent part of the
 *     pressure tensor (lattice ideal pressure n c_s^2 kept by the LB itself).
 *   - Operator order: every right-hand side uses the fields at time t.
 *   - Temperature: T held at T_w on the two wall layers (t_wall_mode 0) or a
 *     halfway Dirichlet ghost 2 T_w - T (t_wall_mode 1); nsub explicit Euler
 *     sub-steps of xi/nsub per step; xi = +inf is an instantaneous quench.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int d;               /* space dimension, 2 or 3 */
    int walls;           /* 1: walls normal to the last axis; 0: fully periodic */
    int t_wall_mode;     /* 0: T = T_w held on the wall layers; 1: halfway ghost */
    int hydro;           /* 1: LB coupled (Eqs. mass, momentum); 0: phi/T only */
    int nsub;            /* temperature sub-steps per step */
    int stencil;         /* 0: compact 5/7-point, central; 1: isotropic 9/19-point */
    int64_t nx, ny, nz;  /* nz = 1 when d = 2 */
    double b, kappa, c, Gamma, Tc, T0, T_w, xi, tau, n0, phi_amp;
    uint64_t seed;
} or_cfg;

/* ------------------------------------------------------------------------ */
/* Velocity sets.  Sec. 2: nine vectors of moduli 0, c, sqrt(2) c on the     */
/* square lattice with weights 4/9, 1/9, 1/36 (Eq. latticeforceterm text).    */
/* In three dimensions the same rule (all e in {-1,0,1}^3 with |e|^2 <= 2)     */
/* gives the 19 vectors of D3Q19, with weights 1/3, 1/18, 1/36.               */
/* The order here is plain enumeration; tests match populations by vector.    */
/* ------------------------------------------------------------------------ */
int or_velocity_set(int d, int* e /* [Q][3] */, double* w /* [Q] */)
{
    int q = 0;
    for (int ez = (d == 3 ? -1 : 0); ez <= (d == 3 ? 1 : 0); ++ez)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex) {
                int m2 = ex * ex + ey * ey + ez * ez;
                if (m2 > 2) continue;
                if (e) { e[3 * q] = ex; e[3 * q + 1] = ey; e[3 * q + 2] = ez; }
                if (w) {
                    if (d == 2) w[q] = (m2 == 0) ? 4.0 / 9.0 : (m2 == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
                    else        w[q] = (m2 == 0) ? 1.0 / 3.0 : (m2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
                }
                ++q;
            }
    return q;
}

static int opposite(const int* e, int Q, int i)
{
    for (int j = 0; j < Q; ++j)
        if (e[3 * j] == -e[3 * i] && e[3 * j + 1] == -e[3 * i + 1] && e[3 * j + 2] == -e[3 * i + 2])
            return j;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Initial order parameter.  phi is i.i.d. uniform in [-amp, amp): the k-th   */
/* output of SplitMix64 seeded with `seed` (Steele, Lea & Flood 2014), top 53 */
/* bits as u in [0,1), phi = amp * (2u - 1).  k is the unpadded site index.   */
/* ------------------------------------------------------------------------ */
static uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void or_splitmix64(uint64_t seed, int64_t count, uint64_t* out)
{
    for (int64_t k = 0; k < count; ++k) out[k] = splitmix64_at(seed, (uint64_t)k);
}

void or_init(const or_cfg* g, double* f, double* phi, double* T)
{
    int e[19 * 3]; double w[19];
    int Q = or_velocity_set(g->d, e, w);
    int64_t N = g->nx * g->ny * g->nz;
    int64_t L = (g->d == 2) ? g->ny : g->nz;
    int64_t layer = (g->d == 2) ? g->nx : g->nx * g->ny;
    for (int64_t s = 0; s < N; ++s) {
        double u = (double)(splitmix64_at(g->seed, (uint64_t)s) >> 11) * (1.0 / 9007199254740992.0);
        phi[s] = g->phi_amp * (2.0 * u - 1.0);
        int64_t h = s / layer;                      /* position along the wall axis */
        if (isinf(g->xi)) T[s] = g->T_w;            /* instantaneous quench */
        else if (g->walls && g->t_wall_mode == 0 && (h == 0 || h == L - 1)) T[s] = g->T_w;
        else T[s] = g->T0;
        for (int i = 0; i < Q; ++i) f[(int64_t)i * N + s] = w[i] * g->n0;
    }
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry: site index, neighbours, reflection across the walls.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int d, wall_axis, walls;
    int64_t n[3], N;
} geom;

static geom make_geom(const or_cfg* g)
{
    geom G;
    G.d = g->d; G.walls = g->walls;
    G.n[0] = g->nx; G.n[1] = g->ny; G.n[2] = (g->d == 3) ? g->nz : 1;
    G.wall_axis = g->d - 1;
    G.N = G.n[0] * G.n[1] * G.n[2];
    return G;
}

static void coords(const geom* G, int64_t s, int64_t c[3])
{
    c[0] = s % G->n[0];
    c[1] = (s / G->n[0]) % G->n[1];
    c[2] = s / (G->n[0] * G->n[1]);
}

static int64_t index_of(const geom* G, const int64_t c[3])
{
    return c[0] + G->n[0] * (c[1] + G->n[1] * c[2]);
}

/* Neighbour of site s at offset `step` (+1/-1) along `axis`.  Periodic axes
 * wrap.  Along the wall axis, stepping out of the lattice lands on the
 * mirror image of s itself (the reflection plane is half a spacing out), and
 * *crossed is set so that the caller can apply the field's parity. */
static int64_t neighbour(const geom* G, int64_t s, int axis, int step, int* crossed)
{
    int64_t c[3];
    coords(G, s, c);
    int64_t v = c[axis] + step;
    *crossed = 0;
    if (G->walls && axis == G->wall_axis) {
        if (v < 0 || v >= G->n[axis]) { *crossed = 1; return s; }
    } else {
        v = (v % G->n[axis] + G->n[axis]) % G->n[axis];
    }
    c[axis] = v;
    return index_of(G, c);
}

/* Field value at the neighbour with parity `odd` (1: flips sign on reflection). */
static double nb_value(const geom* G, const double* a, int64_t s, int axis, int step, int odd)
{
    int crossed;
    int64_t t = neighbour(G, s, axis, step, &crossed);
    return (crossed && odd) ? -a[t] : a[t];
}

/* Second-order operators (Sec. 2, FD paragraph). */
static double laplacian(const geom* G, const double* a, int64_t s)
{
    double acc = 0.0;
    for (int ax = 0; ax < G->d; ++ax)
        acc += nb_value(G, a, s, ax, +1, 0) + nb_value(G, a, s, ax, -1, 0) - 2.0 * a[s];
    return acc;
}

static double central_diff(const geom* G, const double* a, int64_t s, int axis, int odd)
{
    return 0.5 * (nb_value(G, a, s, axis, +1, odd) - nb_value(G, a, s, axis, -1, odd));
}

/* Isotropic operators (stencil 1).  With the lattice weights w_i, e_i of the
 * velocity set (D2Q9 in 2D, D3Q19 in 3D) and c_s^2 = 1/3,
 *   d_a A   = (1/c_s^2) sum_i w_i e_ia A(r + e_i),
 *   lap A   = (2/c_s^2) sum_i w_i [A(r + e_i) - A(r)],
 * which are second-order accurate and isotropic to the next order (Thampi,
 * Ansumali, Adhikari & Succi, J. Comput. Phys. 234 (2013) 1; Kumar,
 * J. Comput. Phys. 201 (2004) 109).  In 2D the Laplacian is
 * [4 (nearest) + (diagonal) - 20 A]/6.  An offset that leaves the lattice
 * through a wall reads the mirror image of the site across the plane half a
 * spacing out (the wall-normal coordinate stays, the others move), with the
 * field's parity, exactly like the compact stencils. */
static int64_t offset_site(const geom* G, int64_t s, const int* e, int* crossed)
{
    int64_t c[3];
    coords(G, s, c);
    *crossed = 0;
    for (int a = 0; a < G->d; ++a) {
        int64_t v = c[a] + e[a];
        if (G->walls && a == G->wall_axis) {
            if (v < 0 || v >= G->n[a]) { *crossed = 1; v = c[a]; }
        } else {
            v = (v % G->n[a] + G->n[a]) % G->n[a];
        }
        c[a] = v;
    }
    return index_of(G, c);
}

static double iso_grad(const geom* G, const double* A, int64_t s, int axis, int odd)
{
    int e[19 * 3]; double w[19];
    int Q = or_velocity_set(G->d, e, w);
    double acc = 0.0;
    for (int i = 0; i < Q; ++i) {
        if (e[3 * i + axis] == 0) continue;
        int crossed;
        int64_t t = offset_site(G, s, &e[3 * i], &crossed);
        double v = (crossed && odd) ? -A[t] : A[t];
        acc += w[i] * e[3 * i + axis] * v;
    }
    return 3.0 * acc;
}

/* Laplacian of an even field; with `dirichlet` set, a ghost across a wall is
 * 2 value_w - A(mirror site) instead (halfway Dirichlet rule of T). */
static double iso_lap(const geom* G, const double* A, int64_t s, int dirichlet, double value_w)
{
    int e[19 * 3]; double w[19];
    int Q = or_velocity_set(G->d, e, w);
    double acc = 0.0;
    for (int i = 0; i < Q; ++i) {   /* the rest vector adds zero */
        int crossed;
        int64_t t = offset_site(G, s, &e[3 * i], &crossed);
        double v = (crossed && dirichlet) ? 2.0 * value_w - A[t] : A[t];
        acc += w[i] * (v - A[s]);
    }
    return 6.0 * acc;
}

/* The operators the configuration selects. */
static double op_lap(const or_cfg* g, const geom* G, const double* A, int64_t s)
{
    return g->stencil ? iso_lap(G, A, s, 0, 0.0) : laplacian(G, A, s);
}

static double op_grad(const or_cfg* g, const geom* G, const double* A, int64_t s, int axis, int odd)
{
    return g->stencil ? iso_grad(G, A, s, axis, odd) : central_diff(G, A, s, axis, odd);
}

/* ------------------------------------------------------------------------ */
/* Local LB pieces.                                                           */
/* ------------------------------------------------------------------------ */

/* Second-order expansion of the Maxwell-Boltzmann distribution (Qian et al.
 * 1992, cited in Sec. 2 after Eq. moment), c = 1, c_s^2 = 1/3. */
void or_feq(int d, double n, const double* u, double* feq)
{
    int e[19 * 3]; double w[19];
    int Q = or_velocity_set(d, e, w);
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double eu = e[3 * i] * u[0] + e[3 * i + 1] * u[1] + e[3 * i + 2] * u[2];
        feq[i] = w[i] * n * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Forcing term, Eq. latticeforceterm (Guo et al. 2002):
 * F_i = (1 - dt/2tau) w_i [ (e_i - u)/c_s^2 + (e_i.u) e_i / c_s^4 ] . F */
void or_guo(int d, double tau, const double* u, const double* F, double* Fi)
{
    int e[19 * 3]; double w[19];
    int Q = or_velocity_set(d, e, w);
    const double cs2 = 1.0 / 3.0;
    for (int i = 0; i < Q; ++i) {
        double eu = e[3 * i] * u[0] + e[3 * i + 1] * u[1] + e[3 * i + 2] * u[2];
        double acc = 0.0;
        for (int a = 0; a < 3; ++a)
            acc += ((e[3 * i + a] - u[a]) / cs2 + eu * e[3 * i + a] / (cs2 * cs2)) * F[a];
        Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * w[i] * acc;
    }
}

/* Moments, Eq. moment: n = sum f_i, n u = sum f_i e_i + F dt / 2. */
static void moments(int Q, const int* e, const double* fi, const double* F, double* n, double* u)
{
    double m = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        m += fi[i];
        for (int a = 0; a < 3; ++a) j[a] += fi[i] * e[3 * i + a];
    }
    *n = m;
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / m;
}

/* Right-hand side of Eq. evoleqn at one site (dt = 1): the post-collision
 * populations f_i - (f_i - f_i^eq)/tau + F_i. */
void or_collide_site(int d, double tau, const double* fi, const double* F, double* fpost)
{
    int e[19 * 3]; double w[19];
    int Q = or_velocity_set(d, e, w);
    double n, u[3], feq[19], Fi[19];
    moments(Q, e, fi, F, &n, u);
    or_feq(d, n, u, feq);
    or_guo(d, tau, u, F, Fi);
    for (int i = 0; i < Q; ++i) fpost[i] = fi[i] - (fi[i] - feq[i]) / tau + Fi[i];
}

/* ------------------------------------------------------------------------ */
/* Thermodynamic fields at time t: a, nabla^2 phi, nabla^4 phi, mu, P, F.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double *a, *psi, *lam, *mu, *dphi[3], *dpsi[3], *P[3][3], *F[3], *n, *u[3];
} work;

static void work_alloc(work* W, int64_t N)
{
    memset(W, 0, sizeof(*W));
    W->a = calloc(N, sizeof(double)); W->psi = calloc(N, sizeof(double));
    W->lam = calloc(N, sizeof(double)); W->mu = calloc(N, sizeof(double));
    W->n = calloc(N, sizeof(double));
    for (int a = 0; a < 3; ++a) {
        W->dphi[a] = calloc(N, sizeof(double)); W->dpsi[a] = calloc(N, sizeof(double));
        W->F[a] = calloc(N, sizeof(double)); W->u[a] = calloc(N, sizeof(double));
        for (int b = 0; b < 3; ++b) W->P[a][b] = calloc(N, sizeof(double));
    }
}

static void work_free(work* W)
{
    free(W->a); free(W->psi); free(W->lam); free(W->mu); free(W->n);
    for (int a = 0; a < 3; ++a) {
        free(W->dphi[a]); free(W->dpsi[a]); free(W->F[a]); free(W->u[a]);
        for (int b = 0; b < 3; ++b) free(W->P[a][b]);
    }
}

static void thermo_fields(const or_cfg* g, const geom* G, const double* phi, const double* T, work* W)
{
    const int64_t N = G->N;
    const int d = G->d, wa = G->wall_axis;

    /* Eq. aterm: a = (T - Tc)/Tc. */
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) W->a[s] = (T[s] - g->Tc) / g->Tc;

    /* nabla^2 phi */
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) W->psi[s] = op_lap(g, G, phi, s);

    /* nabla^4 phi = nabla^2 (nabla^2 phi); gradients of phi and nabla^2 phi */
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        W->lam[s] = op_lap(g, G, W->psi, s);
        for (int ax = 0; ax < 3; ++ax) {
            W->dphi[ax][s] = (ax < d) ? op_grad(g, G, phi, s, ax, 0) : 0.0;
            W->dpsi[ax][s] = (ax < d) ? op_grad(g, G, W->psi, s, ax, 0) : 0.0;
        }
    }

    /* Eq. chem: mu = a phi + b phi^3 - kappa nabla^2 phi + c nabla^4 phi. */
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        double p = phi[s];
        W->mu[s] = W->a[s] * p + g->b * p * p * p - g->kappa * W->psi[s] + g->c * W->lam[s];
    }

    /* Pressure tensor, phi-dependent part (Sec. 2, Gonnella et al. 1997 form):
     * P_ab = { a phi^2/2 + 3b phi^4/4 - kappa [phi nabla^2 phi + |grad phi|^2 / 2]
     *        + c [phi nabla^4 phi + (nabla^2 phi)^2/2 + d_g phi d_g nabla^2 phi] } delta_ab
     *        + kappa d_a phi d_b phi - c [d_a phi d_b nabla^2 phi + d_b phi d_a nabla^2 phi] */
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        double p = phi[s], psi = W->psi[s], lam = W->lam[s];
        double gp2 = 0.0, gpgs = 0.0;
        for (int ax = 0; ax < d; ++ax) {
            gp2 += W->dphi[ax][s] * W->dphi[ax][s];
            gpgs += W->dphi[ax][s] * W->dpsi[ax][s];
        }
        double iso = W->a[s] * p * p / 2.0 + 3.0 * g->b * p * p * p * p / 4.0
                   - g->kappa * (p * psi + 0.5 * gp2)
                   + g->c * (p * lam + 0.5 * psi * psi + gpgs);
        for (int al = 0; al < 3; ++al)
            for (int be = 0; be < 3; ++be) {
                if (al >= d || be >= d) { W->P[al][be][s] = 0.0; continue; }
                W->P[al][be][s] = (al == be ? iso : 0.0)
                    + g->kappa * W->dphi[al][s] * W->dphi[be][s]
                    - g->c * (W->dphi[al][s] * W->dpsi[be][s] + W->dphi[be][s] * W->dpsi[al][s]);
            }
    }

    /* Eq. ff with the lattice ideal pressure: F_b = - d_a P_ab (central). */
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        for (int be = 0; be < 3; ++be) {
            double acc = 0.0;
            if (be < d)
                for (int al = 0; al < d; ++al) {
                    int odd = ((al == wa) ^ (be == wa));   /* reflection sign of P_ab */
                    acc += op_grad(g, G, W->P[al][be], s, al, odd);
                }
            W->F[be][s] = -acc;
        }
    }
}

/* Moments n, u at every site (Eq. moment), with u = 0 when hydro is off. */
static void velocity_fields(const or_cfg* g, const geom* G, const double* f, work* W)
{
    int e[19 * 3]; double w[19];
    int Q = or_velocity_set(G->d, e, w);
    const int64_t N = G->N;
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        double fi[19], F[3] = {W->F[0][s], W->F[1][s], W->F[2][s]}, n, u[3];
        for (int i = 0; i < Q; ++i) fi[i] = f[(int64_t)i * N + s];
        moments(Q, e, fi, F, &n, u);
        W->n[s] = n;
        for (int a = 0; a < 3; ++a) W->u[a][s] = g->hydro ? u[a] : 0.0;
    }
}

/* Auxiliary fields at time t: mu, F, n, u (u = 0 with hydro off). */
void or_aux(const or_cfg* g, const double* f, const double* phi, const double* T,
            double* mu, double* F /* [3][N] */, double* n, double* u /* [3][N] */)
{
    geom G = make_geom(g);
    work W;
    work_alloc(&W, G.N);
    thermo_fields(g, &G, phi, T, &W);
    velocity_fields(g, &G, f, &W);
    memcpy(mu, W.mu, G.N * sizeof(double));
    memcpy(n, W.n, G.N * sizeof(double));
    for (int a = 0; a < 3; ++a) {
        memcpy(F + a * G.N, W.F[a], G.N * sizeof(double));
        memcpy(u + a * G.N, W.u[a], G.N * sizeof(double));
    }
    work_free(&W);
}

/* ------------------------------------------------------------------------ */
/* One full time step t -> t+1.                                               */
/* ------------------------------------------------------------------------ */
void or_step(const or_cfg* g, const double* f, const double* phi, const double* T,
             double* f_new, double* phi_new, double* T_new)
{
    geom G = make_geom(g);
    const int64_t N = G.N;
    const int d = G.d, wa = G.wall_axis;
    int e[19 * 3]; double w[19];
    int Q = or_velocity_set(d, e, w);
    work W;
    work_alloc(&W, N);

    thermo_fields(g, &G, phi, T, &W);
    velocity_fields(g, &G, f, &W);

    /* Eq. evoleqn: BGK collision with Guo forcing, then streaming along e_i.
     * A population that would leave through a wall returns to its own site
     * reversed (halfway bounce-back). */
    if (g->hydro) {
        #pragma omp parallel for schedule(static)
        for (int64_t s = 0; s < N; ++s) {
            double fi[19], fpost[19], F[3] = {W.F[0][s], W.F[1][s], W.F[2][s]};
            for (int i = 0; i < Q; ++i) fi[i] = f[(int64_t)i * N + s];
            or_collide_site(d, g->tau, fi, F, fpost);
            int64_t c[3];
            coords(&G, s, c);
            for (int i = 0; i < Q; ++i) {
                int64_t cd[3];
                int hits_wall = 0;
                for (int a = 0; a < 3; ++a) {
                    int64_t v = c[a] + e[3 * i + a];
                    if (a >= d) { cd[a] = 0; continue; }
                    if (G.walls && a == wa) {
                        if (v < 0 || v >= G.n[a]) hits_wall = 1;
                        cd[a] = v;
                    } else {
                        cd[a] = (v % G.n[a] + G.n[a]) % G.n[a];
                    }
                }
                if (hits_wall) f_new[(int64_t)opposite(e, Q, i) * N + s] = fpost[i];
                else f_new[(int64_t)i * N + index_of(&G, cd)] = fpost[i];
            }
        }
    } else {
        memcpy(f_new, f, (size_t)Q * N * sizeof(double));
    }

    /* Eq. massdiff, explicit Euler: phi <- phi - d_a(phi u_a) + Gamma nabla^2 mu.
     * The flux component normal to the wall is odd under reflection. */
    double* flux[3];
    for (int a = 0; a < 3; ++a) flux[a] = calloc(N, sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s)
        for (int a = 0; a < 3; ++a) flux[a][s] = phi[s] * W.u[a][s];
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        double div = 0.0;
        for (int a = 0; a < d; ++a) div += op_grad(g, &G, flux[a], s, a, a == wa);
        phi_new[s] = phi[s] - div + g->Gamma * op_lap(g, &G, W.mu, s);
    }
    for (int a = 0; a < 3; ++a) free(flux[a]);

    /* Temperature: d_t T = xi nabla^2 T (equivalently d_t a = xi nabla^2 a). */
    memcpy(T_new, T, N * sizeof(double));
    if (!isinf(g->xi) && g->xi != 0.0) {
        double* Tc = malloc(N * sizeof(double));
        const double dxi = g->xi / g->nsub;
        for (int k = 0; k < g->nsub; ++k) {
            memcpy(Tc, T_new, N * sizeof(double));
            #pragma omp parallel for schedule(static)
            for (int64_t s = 0; s < N; ++s) {
                int64_t c[3];
                coords(&G, s, c);
                int on_wall_layer = G.walls && (c[wa] == 0 || c[wa] == G.n[wa] - 1);
                if (G.walls && g->t_wall_mode == 0 && on_wall_layer) { T_new[s] = g->T_w; continue; }
                double lap = 0.0;
                if (g->stencil) {
                    lap = iso_lap(&G, Tc, s, 1, g->T_w);
                } else {
                    for (int ax = 0; ax < d; ++ax)
                        for (int st = -1; st <= 1; st += 2) {
                            int crossed;
                            int64_t t = neighbour(&G, s, ax, st, &crossed);
                            lap += crossed ? (2.0 * g->T_w - Tc[s]) : Tc[t];
                        }
                    lap -= 2.0 * d * Tc[s];
                }
                T_new[s] = Tc[s] + dxi * lap;
            }
        }
        free(Tc);
    }
    work_free(&W);
}

/* n steps in place (ping-pong inside). */
void or_run(const or_cfg* g, int64_t nsteps, double* f, double* phi, double* T)
{
    geom G = make_geom(g);
    int Q = or_velocity_set(g->d, NULL, NULL);
    double* f2 = malloc((size_t)Q * G.N * sizeof(double));
    double* p2 = malloc(G.N * sizeof(double));
    double* t2 = malloc(G.N * sizeof(double));
    for (int64_t k = 0; k < nsteps; ++k) {
        or_step(g, f, phi, T, f2, p2, t2);
        memcpy(f, f2, (size_t)Q * G.N * sizeof(double));
        memcpy(phi, p2, G.N * sizeof(double));
        memcpy(T, t2, G.N * sizeof(double));
    }
    free(f2); free(p2); free(t2);
}

/* Number of OpenMP threads the oracle's parallel loops use. */
#ifdef _OPENMP
#include <omp.h>
int or_threads(void) { return omp_get_max_threads(); }
#else
int or_threads(void) { return 1; }
#endif
