/*
 * oracle.c -- the oracle: a plain, slow, obviously correct FP64 CPU
 * implementation of the fifth-order WENO-JS finite-difference scheme for the
 * compressible Euler equations (Danis et al., "Tensor-Train WENO Scheme for
 * Compressible Flows"), with global Lax-Friedrichs flux splitting and the
 * third-order SSP Runge-Kutta method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path, and nothing in the CUDA path
 * may call it.
 *
 * Passages followed (section / equation of the paper):
 *   Sec. 2.1, Eq. (euler-system), Eq. (physical-fluxes), ideal-gas pressure
 *   Sec. 2.2, Eq. (1d-scalar-h-pde-fd)   semi-discrete conservative form
 *   Sec. 2.2, Eq. (lax-friedrichs)       f(+/-) = (f(u) +/- alpha u)/2
 *   Sec. 2.2, candidate polynomials, smoothness indicators, nonlinear weights
 *   Sec. 2.2, dimension-by-dimension, component-wise application
 *   Sec. 4.1, Eq. (euler-system-for-loop)  the three flux differences
 *   Sec. 4.3, LF-cross: alpha = max(|u| + a)
 *   Sec. 4.4, Eq. (tt-ssprk3) without rounding (Shu-Osher SSP-RK3 form)
 *   Sec. 4.5, three ghost layers per side; periodic and symmetry-plane rules
 *   Sec. 5.5, Eq. (cfl-other)            dt = lambda h / max(alpha)
 *   Sec. 3.1, Eq. (TT_def)               element of a TT tensor
 *
 * Readings where the paper is silent (each one is listed with its reason in
 * the design notes of the repository):
 *   - the f(-) reconstruction is the mirror image of the f(+) one: the same
 *     formula applied to (v[i+3], v[i+2], v[i+1], v[i], v[i-1]);
 *   - epsilon is a parameter (the paper takes dx^2; the workloads take 1e-6);
 *   - alpha is one global scalar max over interior cells of |u| + a, recomputed
 *     from every stage's state (option: per-direction max of |u_d| + a);
 *   - transmissive boundaries copy the nearest interior cell into the ghosts;
 *   - inflow boundaries hold a given conserved state in all three ghost layers
 *     (the full-grid counterpart of the TT inflow rule of Sec. 4.5, which
 *     zeroes the ghost rows and adds a rank-1 TT of the inflow state);
 *   - the grid is cell-centred: x_i = lo + (i + 1/2) h.
 *
 * Scalar models (linear advection u_t + u_x + u_y + u_z = 0 and Burgers
 * u_t + u u_x + u u_y + u u_z = 0, Sec. 5.1-5.2) reuse the same reconstruction
 * and time stepping; they exist to compare with the paper's Tables 1 and 2.
 *
 * Layout of every state array: [field][k][j][i], i (x) fastest, interior
 * cells only, FP64.  Euler field order: rho, rho*u, (rho*v), (rho*w), rho*E.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { M_EULER = 0, M_ADVECT = 1, M_BURGERS = 2 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_INFLOW = 3 };
enum { ALPHA_GLOBAL_NORM = 0, ALPHA_PER_DIR = 1 };

typedef struct {
    int dim;          /* 1, 2 or 3 */
    int model;        /* M_EULER, M_ADVECT, M_BURGERS */
    int n[3];         /* interior points per direction (1 beyond dim) */
    double lo[3];
    double hi[3];
    double gamma;     /* ratio of specific heats */
    double eps;       /* WENO epsilon */
    int bc[3][2];     /* per direction: [low side, high side] */
    int alpha_mode;   /* ALPHA_GLOBAL_NORM or ALPHA_PER_DIR */
    double bc_state[3][2][5];  /* conserved state of an inflow side (BC_INFLOW) */
} ocfg;

#define NG 3          /* ghost layers per side, Sec. 4.5 */

int o_nfields(const ocfg *c) { return c->model == M_EULER ? c->dim + 2 : 1; }

static int64_t o_ncells(const ocfg *c)
{
    int64_t m = 1;
    for (int d = 0; d < c->dim; ++d) m *= c->n[d];
    return m;
}

double o_spacing(const ocfg *c, int d) { return (c->hi[d] - c->lo[d]) / (double)c->n[d]; }

/* ---------------------------------------------------------------- physics */

/* Ideal-gas pressure p = (gamma-1)(rho E - rho |u|^2 / 2), Sec. 2.1. */
double o_pressure(const ocfg *c, const double *q)
{
    double rho = q[0];
    double ke = 0.0;
    for (int e = 0; e < c->dim; ++e) {
        double ue = q[1 + e] / rho;
        ke += ue * ue;
    }
    return (c->gamma - 1.0) * (q[c->dim + 1] - 0.5 * rho * ke);
}

/* Physical flux in direction d, Eq. (physical-fluxes): component 0 is rho u_d,
 * component 1+e is rho u_e u_d + p delta_ed, the last is u_d (rho E + p). */
void o_flux(const ocfg *c, const double *q, int d, double *f)
{
    if (c->model == M_ADVECT) { f[0] = q[0]; return; }
    if (c->model == M_BURGERS) { f[0] = 0.5 * q[0] * q[0]; return; }
    int D = c->dim;
    double rho = q[0];
    double ud = q[1 + d] / rho;
    double p = o_pressure(c, q);
    f[0] = q[1 + d];
    for (int e = 0; e < D; ++e) f[1 + e] = q[1 + e] * ud + (e == d ? p : 0.0);
    f[D + 1] = ud * (q[D + 1] + p);
}

/* Characteristic speed used for alpha: |u| + a (dir < 0) or |u_d| + a, with
 * a = sqrt(gamma p / rho) (Sec. 4.3 and Eq. (cfl-other)).  For the scalar
 * models it is |f'(u)|: 1 for linear advection, |u| for Burgers. */
double o_wavespeed(const ocfg *c, const double *q, int dir)
{
    if (c->model == M_ADVECT) return 1.0;
    if (c->model == M_BURGERS) return fabs(q[0]);
    double rho = q[0];
    double p = o_pressure(c, q);
    double a = sqrt(c->gamma * p / rho);
    if (dir >= 0) return fabs(q[1 + dir] / rho) + a;
    double u2 = 0.0;
    for (int e = 0; e < c->dim; ++e) {
        double ue = q[1 + e] / rho;
        u2 += ue * ue;
    }
    return sqrt(u2) + a;
}

/* ----------------------------------------------------------- WENO5-JS (+) */

/* Smoothness indicators beta_0..2 of the stencil v = (v[i-2], ..., v[i+2]),
 * Sec. 2.2. */
void o_weno5_beta(const double *v, double *beta)
{
    double vm2 = v[0], vm1 = v[1], v0 = v[2], vp1 = v[3], vp2 = v[4];
    double a, b;
    a = v0 - 2.0 * vp1 + vp2;
    b = 3.0 * v0 - 4.0 * vp1 + vp2;
    beta[0] = 13.0 / 12.0 * a * a + 0.25 * b * b;
    a = vm1 - 2.0 * v0 + vp1;
    b = vm1 - vp1;
    beta[1] = 13.0 / 12.0 * a * a + 0.25 * b * b;
    a = vm2 - 2.0 * vm1 + v0;
    b = vm2 - 4.0 * vm1 + 3.0 * v0;
    beta[2] = 13.0 / 12.0 * a * a + 0.25 * b * b;
}

/* Nonlinear weights omega_r = alpha_r / sum alpha_s with
 * alpha_r = d_r / (beta_r + eps)^2, d = (3/10, 3/5, 1/10), Sec. 2.2. */
void o_weno5_weights(const double *v, double eps, double *omega)
{
    static const double dlin[3] = {3.0 / 10.0, 3.0 / 5.0, 1.0 / 10.0};
    double beta[3], al[3], s = 0.0;
    o_weno5_beta(v, beta);
    for (int r = 0; r < 3; ++r) {
        double t = beta[r] + eps;
        al[r] = dlin[r] / (t * t);
        s += al[r];
    }
    for (int r = 0; r < 3; ++r) omega[r] = al[r] / s;
}

/* Candidate reconstructions v^(r)_{i+1/2} on S_r(i), Sec. 2.2. */
void o_weno5_candidates(const double *v, double *p)
{
    double vm2 = v[0], vm1 = v[1], v0 = v[2], vp1 = v[3], vp2 = v[4];
    p[0] = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0;
    p[1] = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0;
    p[2] = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
}

/* WENO5-JS value at x_{i+1/2} reconstructed from v = (v[i-2], ..., v[i+2]):
 * the convex combination sum_r omega_r v^(r)_{i+1/2}, Sec. 2.2. */
double o_weno5(const double *v, double eps)
{
    double p[3], w[3];
    o_weno5_candidates(v, p);
    o_weno5_weights(v, eps, w);
    return w[0] * p[0] + w[1] * p[1] + w[2] * p[2];
}

/* -------------------------------------------------------------- ghosts */

/* Maps a (possibly ghost) index g of a direction with n interior points to
 * the interior index whose value the ghost holds (Sec. 4.5).  *flip is set
 * to 1 when the ghost is a mirror image (symmetry plane), in which case the
 * caller negates the normal momentum. */
static int o_ghost_source(int g, int n, int bclo, int bchi, int *flip)
{
    *flip = 0;
    if (g >= 0 && g < n) return g;
    int bc = g < 0 ? bclo : bchi;
    if (bc == BC_PERIODIC) return g < 0 ? g + n : g - n;   /* U(-2:0)=U(N-2:N), U(N+1:N+3)=U(1:3) */
    if (bc == BC_TRANSMISSIVE) return g < 0 ? 0 : n - 1;
    *flip = 1;                                           /* q(-2+l) = q(3-l), l = 0,1,2 */
    return g < 0 ? -1 - g : 2 * n - 1 - g;
}

/* Builds the ghost-padded copy P of U: (n_d + 2*NG) points per used
 * direction.  Only the ghost slabs that a one-dimensional stencil can reach
 * are filled (edges and corners are never read). */
static double *o_pad(const ocfg *c, const double *U, int64_t pn[3])
{
    int nf = o_nfields(c);
    for (int d = 0; d < 3; ++d) pn[d] = d < c->dim ? c->n[d] + 2 * NG : 1;
    int64_t pcells = pn[0] * pn[1] * pn[2];
    double *P = (double *)calloc((size_t)(nf * pcells), sizeof(double));
    int64_t nx = c->n[0], ny = c->n[1];
    int off[3];
    for (int d = 0; d < 3; ++d) off[d] = d < c->dim ? NG : 0;
    for (int64_t pk = 0; pk < pn[2]; ++pk)
        for (int64_t pj = 0; pj < pn[1]; ++pj)
            for (int64_t pi = 0; pi < pn[0]; ++pi) {
                int g[3] = {(int)pi - off[0], (int)pj - off[1], (int)pk - off[2]};
                int outside = 0, dout = -1;
                for (int d = 0; d < c->dim; ++d)
                    if (g[d] < 0 || g[d] >= c->n[d]) { ++outside; dout = d; }
                if (outside > 1) continue;
                int src[3] = {g[0], g[1], g[2]};
                int flip = 0;
                int64_t t = (pk * pn[1] + pj) * pn[0] + pi;
                if (outside == 1) {
                    /* inflow (Sec. 4.5): the ghost layers hold the given inflow state */
                    int side = g[dout] < 0 ? 0 : 1;
                    if (c->bc[dout][side] == BC_INFLOW) {
                        for (int f = 0; f < nf; ++f) P[(int64_t)f * pcells + t] = c->bc_state[dout][side][f];
                        continue;
                    }
                    src[dout] = o_ghost_source(g[dout], c->n[dout], c->bc[dout][0], c->bc[dout][1], &flip);
                }
                int64_t s = ((int64_t)src[2] * ny + src[1]) * nx + src[0];
                for (int f = 0; f < nf; ++f) {
                    double val = U[(int64_t)f * o_ncells(c) + s];
                    if (flip && c->model == M_EULER && f == 1 + dout) val = -val;
                    P[(int64_t)f * pcells + t] = val;
                }
            }
    return P;
}

/* ------------------------------------------------------------ residual */

/* alpha for the LF splitting of every direction: out[d], d = 0..2. */
void o_alpha(const ocfg *c, const double *U, double *out)
{
    int nf = o_nfields(c);
    int64_t nc = o_ncells(c);
    double q[5];
    for (int d = 0; d < 3; ++d) out[d] = 0.0;
    for (int64_t i = 0; i < nc; ++i) {
        for (int f = 0; f < nf; ++f) q[f] = U[(int64_t)f * nc + i];
        if (c->alpha_mode == ALPHA_PER_DIR && c->model == M_EULER) {
            for (int d = 0; d < c->dim; ++d) {
                double s = o_wavespeed(c, q, d);
                if (s > out[d]) out[d] = s;
            }
        } else {
            double s = o_wavespeed(c, q, -1);
            for (int d = 0; d < 3; ++d)
                if (s > out[d]) out[d] = s;
        }
    }
}

/* Global alpha max(|u| + a) over interior cells, the CFL wavespeed. */
double o_alpha_max(const ocfg *c, const double *U)
{
    int nf = o_nfields(c);
    int64_t nc = o_ncells(c);
    double q[5], m = 0.0;
    for (int64_t i = 0; i < nc; ++i) {
        for (int f = 0; f < nf; ++f) q[f] = U[(int64_t)f * nc + i];
        double s = o_wavespeed(c, q, -1);
        if (s > m) m = s;
    }
    return m;
}

/* Interface flux F^_{m+1/2} of one component from the split fluxes at the six
 * points m-2..m+3 (fp[k], fm[k] hold point m-2+k):
 * WENO(+) of f+ at m-2..m+2 plus the mirrored WENO(-) of f- at m+3..m-1. */
static double o_interface_flux(const double *fp, const double *fm, double eps)
{
    double vp[5] = {fp[0], fp[1], fp[2], fp[3], fp[4]};
    double vm[5] = {fm[5], fm[4], fm[3], fm[2], fm[1]};
    return o_weno5(vp, eps) + o_weno5(vm, eps);
}

/* R -= (F^_{i+1/2} - F^_{i-1/2}) / h_d for the directions in dirmask, with the
 * splitting constants alpha[d] given.  R is accumulated into, not cleared. */
void o_residual_dirs(const ocfg *c, const double *U, const double *alpha, int dirmask, double *R)
{
    int nf = o_nfields(c);
    int64_t pn[3];
    double *P = o_pad(c, U, pn);
    int64_t pcells = pn[0] * pn[1] * pn[2];
    int64_t nc = o_ncells(c);
    int64_t nx = c->n[0], ny = c->n[1];
    int off[3];
    for (int d = 0; d < 3; ++d) off[d] = d < c->dim ? NG : 0;
    int64_t pstride[3] = {1, pn[0], pn[0] * pn[1]};

    for (int d = 0; d < c->dim; ++d) {
        if (!(dirmask & (1 << d))) continue;
        int n = c->n[d];
        double h = o_spacing(c, d);
        double *Fh = (double *)malloc(sizeof(double) * (size_t)(nf * (n + 1)));
        /* loop over all lines along d through interior cells */
        int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
        int n1 = a1 < c->dim ? c->n[a1] : 1, n2 = a2 < c->dim ? c->n[a2] : 1;
        for (int l2 = 0; l2 < n2; ++l2)
            for (int l1 = 0; l1 < n1; ++l1) {
                /* interfaces m+1/2 for m = -1 .. n-1 */
                for (int m = -1; m < n; ++m) {
                    double fp[5][6], fm[5][6];
                    for (int k = 0; k < 6; ++k) {
                        int pt[3];
                        pt[d] = m - 2 + k + off[d];
                        pt[a1] = l1 + off[a1];
                        pt[a2] = l2 + off[a2];
                        int64_t t = pt[0] * pstride[0] + pt[1] * pstride[1] + pt[2] * pstride[2];
                        double q[5], F[5];
                        for (int f = 0; f < nf; ++f) q[f] = P[(int64_t)f * pcells + t];
                        o_flux(c, q, d, F);
                        for (int f = 0; f < nf; ++f) {
                            fp[f][k] = 0.5 * (F[f] + alpha[d] * q[f]);   /* Eq. (lax-friedrichs) */
                            fm[f][k] = 0.5 * (F[f] - alpha[d] * q[f]);
                        }
                    }
                    for (int f = 0; f < nf; ++f)
                        Fh[f * (n + 1) + (m + 1)] = o_interface_flux(fp[f], fm[f], c->eps);
                }
                for (int i = 0; i < n; ++i) {
                    int ix[3];
                    ix[d] = i;
                    ix[a1] = l1;
                    ix[a2] = l2;
                    int64_t s = ((int64_t)ix[2] * ny + ix[1]) * nx + ix[0];
                    for (int f = 0; f < nf; ++f) {
                        double dF = Fh[f * (n + 1) + (i + 1)] - Fh[f * (n + 1) + i];
                        R[(int64_t)f * nc + s] -= dF / h;
                    }
                }
            }
        free(Fh);
    }
    free(P);
}

/* L(U) = -sum_d (F^_{i+1/2} - F^_{i-1/2}) / h_d with alpha from U itself.
 * alpha_out (3 values, may be NULL) receives the alpha used. */
void o_residual(const ocfg *c, const double *U, double *R, double *alpha_out)
{
    double alpha[3];
    o_alpha(c, U, alpha);
    memset(R, 0, sizeof(double) * (size_t)(o_nfields(c) * o_ncells(c)));
    o_residual_dirs(c, U, alpha, 7, R);
    if (alpha_out) memcpy(alpha_out, alpha, sizeof alpha);
}

/* -------------------------------------------------------------- SSP-RK3 */

/* One step of Eq. (tt-ssprk3) without rounding, in its Shu-Osher form:
 *   u1 = u + dt L(u)
 *   u2 = 3/4 u + 1/4 (u1 + dt L(u1))
 *   u' = 1/3 u + 2/3 (u2 + dt L(u2)) */
void o_ssprk3_step(const ocfg *c, double *U, double dt)
{
    int64_t m = (int64_t)o_nfields(c) * o_ncells(c);
    double *R = (double *)malloc(sizeof(double) * (size_t)m);
    double *U1 = (double *)malloc(sizeof(double) * (size_t)m);
    double *U2 = (double *)malloc(sizeof(double) * (size_t)m);
    o_residual(c, U, R, NULL);
    for (int64_t i = 0; i < m; ++i) U1[i] = U[i] + dt * R[i];
    o_residual(c, U1, R, NULL);
    for (int64_t i = 0; i < m; ++i) U2[i] = 3.0 / 4.0 * U[i] + 1.0 / 4.0 * (U1[i] + dt * R[i]);
    o_residual(c, U2, R, NULL);
    for (int64_t i = 0; i < m; ++i) U[i] = 1.0 / 3.0 * U[i] + 2.0 / 3.0 * (U2[i] + dt * R[i]);
    free(R);
    free(U1);
    free(U2);
}

/* Eq. (cfl-other): dt = lambda h / max(alpha), h the smallest spacing. */
double o_cfl_dt(const ocfg *c, const double *U, double cfl)
{
    double h = o_spacing(c, 0);
    for (int d = 1; d < c->dim; ++d)
        if (o_spacing(c, d) < h) h = o_spacing(c, d);
    return cfl * h / o_alpha_max(c, U);
}

/* Advances U from t0 to t_end.  Each step takes dt = cfl h / alpha (cfl > 0)
 * and, when dt_coef > 0, no more than dt_coef * h^dt_pow (the convergence
 * studies' dt = h^(5/3), Sec. 5.1); the last step is shortened to land on
 * t_end.  Returns the number of steps taken; *t_out receives the final time. */
int64_t o_run(const ocfg *c, double *U, double t0, double t_end, double cfl, double dt_coef,
              double dt_pow, int64_t max_steps, double *t_out)
{
    double h = o_spacing(c, 0);
    for (int d = 1; d < c->dim; ++d)
        if (o_spacing(c, d) < h) h = o_spacing(c, d);
    double t = t0;
    int64_t steps = 0;
    while (t < t_end && steps < max_steps) {
        double dt = 1e300;
        if (cfl > 0.0) dt = o_cfl_dt(c, U, cfl);
        if (dt_coef > 0.0) {
            double dtc = dt_coef * pow(h, dt_pow);
            if (dtc < dt) dt = dtc;
        }
        /* last step: shortened to land on t_end, and the time set to t_end exactly */
        double tn = t + dt;
        if (tn >= t_end) {
            dt = t_end - t;
            tn = t_end;
        }
        o_ssprk3_step(c, U, dt);
        t = tn;
        ++steps;
    }
    if (t_out) *t_out = t;
    return steps;
}

/* Sum over interior cells of every field (conservation check). */
void o_sums(const ocfg *c, const double *U, double *sums)
{
    int nf = o_nfields(c);
    int64_t nc = o_ncells(c);
    for (int f = 0; f < nf; ++f) {
        double s = 0.0;
        for (int64_t i = 0; i < nc; ++i) s += U[(int64_t)f * nc + i];
        sums[f] = s;
    }
}

/* ---------------------------------------------- pointwise, from TT cores */

/* Element of a 3D TT tensor, Eq. (TT_def):
 *   X(i,j,k) = sum_a sum_b G1(1,i,a) G2(a,j,b) G3(b,k,1).
 * Core m is stored as float [n_m][r_{m-1}][r_m] (r_0 = r_3 = 1). */
static double o_tt_element(const float *const *core, const int *r, const int *ix)
{
    int r1 = r[0], r2 = r[1];
    const float *g1 = core[0] + (int64_t)ix[0] * r1;
    const float *g2 = core[1] + (int64_t)ix[1] * r1 * r2;
    const float *g3 = core[2] + (int64_t)ix[2] * r2;
    double s = 0.0;
    for (int a = 0; a < r1; ++a)
        for (int b = 0; b < r2; ++b)
            s += (double)g1[a] * (double)g2[a * r2 + b] * (double)g3[b];
    return s;
}

/* The direction-fd residual contribution -(F^_{i+1/2} - F^_{i-1/2}) / h_fd of
 * the 3D Euler equations at sample points of a TT tensor, the quantity that
 * LF-cross (Algorithm 1) and WENO-cross (Algorithm 2) evaluate elementwise.
 *
 * The samples are the fibers of one cross sweep: for every left multi-index
 * (over the modes before `mode`), every index i of `mode` and every right
 * multi-index (over the modes after it).  The 7-point stencil along fd is
 * taken from the cores, with ghost rows given by the boundary rule of fd
 * (Sec. 4.5, the core-level ghost fill).
 *
 *   n[3], r[2]   mode sizes and TT ranks
 *   cores[15]    cores[f*3 + m] = core m of field f (rho, rho u, rho v, rho w, rho E)
 *   h[3]         spacings; alpha the LF constant; bc[3][2] boundary rules
 *   left         int32 [n_left][mode]; right int32 [n_right][2-mode]
 *   out          FP64 [5][n_left][n[mode]][n_right] */
void o_cross_eval(const int *n, const int *r, const float *const *cores, const double *h, double alpha,
                  double gamma, double eps, const int *bc, int mode, int fd, int64_t n_left,
                  const int32_t *left, int64_t n_right, const int32_t *right, double *out)
{
    ocfg c;
    memset(&c, 0, sizeof c);
    c.dim = 3;
    c.model = M_EULER;
    c.gamma = gamma;
    c.eps = eps;
    int nm = n[mode];
    int nl = mode, nr = 2 - mode;
    for (int64_t l = 0; l < n_left; ++l)
        for (int i = 0; i < nm; ++i)
            for (int64_t rr = 0; rr < n_right; ++rr) {
                int ix[3];
                for (int m = 0; m < nl; ++m) ix[m] = left[l * nl + m];
                ix[mode] = i;
                for (int m = 0; m < nr; ++m) ix[mode + 1 + m] = right[rr * nr + m];
                /* the 7 stencil points along fd: s = -3..3 */
                double fp[5][7], fmn[5][7];
                for (int s = -3; s <= 3; ++s) {
                    int pt[3] = {ix[0], ix[1], ix[2]};
                    int flip = 0;
                    pt[fd] = o_ghost_source(ix[fd] + s, n[fd], bc[fd * 2 + 0], bc[fd * 2 + 1], &flip);
                    double q[5], F[5];
                    for (int f = 0; f < 5; ++f) {
                        q[f] = o_tt_element(cores + f * 3, r, pt);
                        if (flip && f == 1 + fd) q[f] = -q[f];
                    }
                    o_flux(&c, q, fd, F);
                    for (int f = 0; f < 5; ++f) {
                        fp[f][s + 3] = 0.5 * (F[f] + alpha * q[f]);
                        fmn[f][s + 3] = 0.5 * (F[f] - alpha * q[f]);
                    }
                }
                for (int f = 0; f < 5; ++f) {
                    /* interface i-1/2 uses points i-3..i+2, interface i+1/2 uses i-2..i+3 */
                    double Flo = o_interface_flux(&fp[f][0], &fmn[f][0], eps);
                    double Fhi = o_interface_flux(&fp[f][1], &fmn[f][1], eps);
                    out[(((int64_t)f * n_left + l) * nm + i) * n_right + rr] = -(Fhi - Flo) / h[fd];
                }
            }
}

/* Full tensor of one field from its TT cores, [k][j][i] with i fastest. */
void o_tt_full(const int *n, const int *r, const float *const *core3, double *X)
{
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                int ix[3] = {i, j, k};
                X[((int64_t)k * n[1] + j) * n[0] + i] = o_tt_element(core3, r, ix);
            }
}
