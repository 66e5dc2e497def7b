/*
 * lattice_oracle.c -- plain FP64 CPU oracle for the staggered-leapfrog evolution
 * of two interacting scalar fields (phi, chi) on a periodic 3D lattice in an
 * expanding FRW universe, after J. Sainio, "CUDAEASY - a GPU Accelerated
 * Cosmological Lattice Program" (arXiv:0911.5692).
 *
 * TEST INFRASTRUCTURE. This is the slow, obviously-correct reference that the
 * CUDA library is checked against. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it. The product library neither links nor
 * calls it, and the two share no source, header, table or helper. Every loop
 * here is a direct transcription of one equation; nothing is fused or blocked.
 * OpenMP only splits the outermost z loop; every sum is taken per z-plane and
 * the planes are added in index order, so results do not depend on the thread
 * count.
 *
 * Equations followed (all in program units, primes are d/dt_pr):
 *   rescaling          Sec. II.B: f = A a^r phi, x_pr = B x, dt_pr = B a^s dt,
 *                      s - 2r + 3 = 0; for a dominant term cpl/beta phi^beta the
 *                      choice A = 1/phi0, B = sqrt(cpl) phi0^(beta/2-1),
 *                      r = 6/(2+beta), s = 3(2-beta)/(2+beta).
 *   potential          Sec. II.B: V_pr = (A^2/B^2) a^(2r-2s) V(f/(A a^r)).
 *   field equation     Sec. II.B, eq. scalar-evo:
 *                      f'' = a^(-2s-2) Lap f + (r(s-r+2) h^2 + r a''/a) f - dV_pr/df,
 *                      h = a'/a. The printed coefficient r(s-r-2) does not follow
 *                      from eq. fe under the rescaling; r(s-r+2) does (it is the
 *                      one that vanishes in the conformal case r=1, s=-1).
 *   scale factor       Sec. II.B, eq. scale:
 *                      a'' = -(s+2) a'^2/a + (8piG/A^2) a^(-2s-2r-1)
 *                            < sum_i |grad f_i|^2 / 3 + a^(2s+2) V_pr >.
 *   leapfrog           Sec. II.B, eq. evo: fields and momenta stored half a step
 *                      apart, kick then drift; a and a' are staggered the same
 *                      way, and a'' at the field time uses the momentum average
 *                      a'_{n+1/2} = (a'_n + a'_{n+1})/2, which makes the a' update
 *                      an exactly solvable quadratic.
 *   gradient average   Sec. II.B, divergence-theorem identity: on a periodic
 *                      lattice <|grad f|^2> = -<f Lap f>; here it is evaluated
 *                      from forward differences, the 7-point stencil's gradient.
 *   Laplacian          Sec. II.C: the 7-point ("naive", LATTICEEASY) stencil, or the
 *                      paper's 27-point stencil (Patra and Karttunen; second-order
 *                      accurate, fourth-order isotropic); with the 27-point stencil
 *                      the gradient average is -<f L f> with the same L, as the
 *                      paper's kernel forms it from the Laplacian.
 *   initial conditions Sec. II.B, last paragraph: homogeneous values plus Gaussian
 *                      vacuum fluctuations (DEFROST style), converted with
 *                      f = A a^r phi, f' = (A/B) a^(r-s) phidot + r (a'/a) f, then
 *                      fields advanced by dt/2.
 *   energy, pressure   Sec. II.B, eq. rho-pres; residual curvature and w of Sec. III.
 *                      Per site (the paper's second kernel, Sec. II.C): the same
 *                      terms at each site, the gradient energy of a site being half
 *                      the weighted squared differences to all its stencil
 *                      neighbours (each neighbour pair shared evenly by its two
 *                      sites), so that the volume means are the averages above.
 *   spectrum           Sec. IV (named as future work): shell-binned |f_k|^2.
 *   L = 1/H form       Sec. II.B mentions that DEFROST evolves L = 1/H first and a
 *                      from L, which removes the gradient terms; the paper prints no
 *                      equation for it. Here (expansion = 2), from the acceleration
 *                      equation a-double-dot/a = -(4piG/3)(rho + 3p), rho + 3p =
 *                      2 sum phidot^2 - 2V, in program time with h = a'/a, l = 1/h:
 *                        l' = (s + 1) + Gamma l^2,  a' = a / l,  a''/a = -s h^2 - Gamma,
 *                        Gamma = (8piG/(3A^2)) a^(-2r) (sum_i <(f_i' - r h f_i)^2> - <V_pr>),
 *                      so the f coefficient of eq. scalar-evo is r(2-r) h^2 - r Gamma.
 *                      Staggering: l at the momentum times (with a'), a at the field
 *                      times; the step is the implicit midpoint rule for l (solved
 *                      by fixed-point iteration) and a_{n+3/2} = a_{n+1/2} exp(dt/l_{n+1}).
 *
 * Counter-based random numbers: Philox-4x32-10 (J. Salmon, M. Moraes, R. Dror,
 * D. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), normals by the
 * Box-Muller transform.
 *
 * parity unpinned: the physical normalisation of the initial fluctuation
 * spectrum against DEFROST (its source and data are not available); the
 * statistics of the generated spectrum are pinned instead.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 3
#define ORC_ENONFINITE 5

typedef struct {
    int32_t n;          /* lattice is n^3 */
    int32_t model;      /* 0: V = lambda/4 phi^4 + g2/2 phi^2 chi^2; 1: V = m^2/2 phi^2 + g2/2 phi^2 chi^2 */
    int32_t expansion;  /* 0: static space, a = 1; 1: FRW, eq. scale; 2: FRW, L = 1/H form */
    int32_t stencil;    /* Laplacian: 7 (or 0) = 7-point, 27 = 27-point (Sec. II.C) */
    double L, dt;       /* box side and time step, program units */
    double lambda, m, g2;
    double phi0[2], dphi0[2]; /* homogeneous values and physical-time derivatives */
    double eight_pi_G;
    double A, B, r, s;  /* all zero: derive from the dominant term */
    double kcut;        /* fluctuation cutoff in units of 2 pi / L; 0 = n/4 */
    double fluct;       /* multiplier on the vacuum fluctuation amplitude */
    uint64_t seed;
} orc_params;

typedef struct {
    orc_params p;
    int n;
    size_t nsites;
    double dx;
    double A, B, r, s, beta, cpl;
    double cdom0, pdom, kappa0, pint;   /* V_pr = cdom0 a^pdom f^beta/beta + kappa0 a^pint f^2 chi^2 / 2 */
    double *f[2], *pi[2];
    double t;      /* program time of the momenta; fields and a live at t + dt/2 */
    double a;      /* a at t + dt/2 */
    double ad;     /* a' at t */
    double S[4];   /* <|grad f0|^2>, <|grad f1|^2>, <f0^beta/beta>, <f0^2 f1^2/2> at field time */
    int64_t step;
    double ell;    /* L = 1/H form: l = a/a' (program time) at t */
} orc_lattice;

static size_t idx(int n, int x, int y, int z) { return ((size_t)z * n + y) * n + x; }
static int wrap(int i, int n) { return (i % n + n) % n; }

/* ---------------------------------------------------------------- rescaling */

int orc_derive(orc_lattice *L)
{
    const orc_params *p = &L->p;
    if (p->model == 0) { L->cpl = p->lambda; L->beta = 4.0; }
    else if (p->model == 1) { L->cpl = p->m * p->m; L->beta = 2.0; }
    else return ORC_EINVAL;
    if (p->phi0[0] == 0.0 || L->cpl <= 0.0) return ORC_EINVAL;
    if (p->A == 0.0 && p->B == 0.0 && p->r == 0.0 && p->s == 0.0) {
        /* Sec. II.B: rescaling for a dominant term cpl/beta phi^beta */
        L->A = 1.0 / p->phi0[0];
        L->B = sqrt(L->cpl) * pow(fabs(p->phi0[0]), -1.0 + L->beta / 2.0);
        L->r = 6.0 / (2.0 + L->beta);
        L->s = 3.0 * (2.0 - L->beta) / (2.0 + L->beta);
    } else {
        L->A = p->A; L->B = p->B; L->r = p->r; L->s = p->s;
    }
    /* Sec. II.B: the first-derivative term vanishes only if s - 2r + 3 = 0 */
    if (fabs(L->s - 2.0 * L->r + 3.0) > 1e-12 || L->A == 0.0 || L->B <= 0.0) return ORC_EINVAL;
    /* V_pr = (A^2/B^2) a^(2r-2s) V(phi = f / (A a^r)) */
    L->cdom0 = L->cpl * pow(L->A, 2.0 - L->beta) / (L->B * L->B);
    L->pdom = 2.0 * L->r - 2.0 * L->s - L->beta * L->r;
    L->kappa0 = p->g2 / (L->A * L->A * L->B * L->B);
    L->pint = -2.0 * L->r - 2.0 * L->s;
    return ORC_OK;
}

/* physical potential V(phi, chi), Sec. III and the configured lambda model */
static double V_phys(const orc_lattice *L, double phi, double chi)
{
    return L->cpl / L->beta * pow(phi, L->beta) + 0.5 * L->p.g2 * phi * phi * chi * chi;
}

static double cdom_at(const orc_lattice *L, double a) { return L->cdom0 * pow(a, L->pdom); }
static double kappa_at(const orc_lattice *L, double a) { return L->kappa0 * pow(a, L->pint); }

/* program-unit potential and its derivatives at one site */
static double Vpr(const orc_lattice *L, double a, double f0, double f1)
{
    return cdom_at(L, a) * pow(f0, L->beta) / L->beta + 0.5 * kappa_at(L, a) * f0 * f0 * f1 * f1;
}
static double dVpr0(const orc_lattice *L, double a, double f0, double f1)
{
    return cdom_at(L, a) * pow(f0, L->beta - 1.0) + kappa_at(L, a) * f0 * f1 * f1;
}
static double dVpr1(const orc_lattice *L, double a, double f0, double f1)
{
    return kappa_at(L, a) * f0 * f0 * f1;
}

/* ---------------------------------------------------------------- creation */

int orc_create(const orc_params *p, orc_lattice **out)
{
    *out = NULL;
    if (p->n < 2 || p->n > 1024 || p->L <= 0.0 || p->dt <= 0.0) return ORC_EINVAL;
    if (p->stencil != 0 && p->stencil != 7 && p->stencil != 27) return ORC_EINVAL;
    if (p->expansion < 0 || p->expansion > 2) return ORC_EINVAL;
    orc_lattice *L = (orc_lattice *)calloc(1, sizeof(orc_lattice));
    if (!L) return ORC_ENOMEM;
    L->p = *p;
    L->n = p->n;
    L->nsites = (size_t)p->n * p->n * p->n;
    L->dx = p->L / p->n;
    int st = orc_derive(L);
    if (st != ORC_OK) { free(L); return st; }
    for (int i = 0; i < 2; i++) {
        L->f[i] = (double *)calloc(L->nsites, sizeof(double));
        L->pi[i] = (double *)calloc(L->nsites, sizeof(double));
        if (!L->f[i] || !L->pi[i]) {
            for (int j = 0; j < 2; j++) { free(L->f[j]); free(L->pi[j]); }
            free(L);
            return ORC_ENOMEM;
        }
    }
    L->a = 1.0;
    *out = L;
    return ORC_OK;
}

void orc_destroy(orc_lattice *L)
{
    if (!L) return;
    for (int i = 0; i < 2; i++) { free(L->f[i]); free(L->pi[i]); }
    free(L);
}

/* derived constants: A, B, r, s, beta, cdom0, pdom, kappa0, pint, dx */
void orc_get_derived(const orc_lattice *L, double out[10])
{
    out[0] = L->A; out[1] = L->B; out[2] = L->r; out[3] = L->s; out[4] = L->beta;
    out[5] = L->cdom0; out[6] = L->pdom; out[7] = L->kappa0; out[8] = L->pint; out[9] = L->dx;
}

double *orc_array(orc_lattice *L, int field, int what) { return what == 0 ? L->f[field] : L->pi[field]; }

/* scalars: t, a, a', step, S[0..3] */
void orc_get_scalars(const orc_lattice *L, double out[8])
{
    out[0] = L->t; out[1] = L->a; out[2] = L->ad; out[3] = (double)L->step;
    for (int i = 0; i < 4; i++) out[4 + i] = L->S[i];
}

/* ---------------------------------------------------------------- operators */

/* 7-point Laplacian with periodic wrap: (sum of the six neighbours - 6 f) / dx^2 */
void orc_laplacian(int n, double dx, const double *f, double *out)
{
    double inv = 1.0 / (dx * dx);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < n; z++)
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                double nb = f[idx(n, wrap(x + 1, n), y, z)] + f[idx(n, wrap(x - 1, n), y, z)]
                          + f[idx(n, x, wrap(y + 1, n), z)] + f[idx(n, x, wrap(y - 1, n), z)]
                          + f[idx(n, x, y, wrap(z + 1, n))] + f[idx(n, x, y, wrap(z - 1, n))];
                out[idx(n, x, y, z)] = (nb - 6.0 * f[idx(n, x, y, z)]) * inv;
            }
}

/* 27-point Laplacian over the 3x3x3 cube, periodic. The weights (in units of
 * 1/dx^2) depend on the neighbour's distance class: face (6 neighbours) 14/30,
 * edge (12) 3/30, corner (8) 1/30, centre -128/30. With symbol
 * L(k) = c0 + 2 c1 sum cos k_i + 4 c2 sum_{i<j} cos k_i cos k_j + 8 c3 prod cos k_i,
 * L(0) = 0, the k^2 coefficient -1 (second-order accuracy) and an isotropic k^4
 * term (fourth-order isotropy: coefficient of sum_{i<j} k_i^2 k_j^2 twice that of
 * sum k_i^4) leave a one-parameter family c1 = 2 c2 + 8 c3, c2 = (1 - 12 c3)/6;
 * c3 = 1/30 is the member the paper takes from Patra and Karttunen (the one
 * DEFROST uses). */
static const double ORC_W27[4] = {-128.0 / 30.0, 14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0};

void orc_laplacian27(int n, double dx, const double *f, double *out)
{
    double inv = 1.0 / (dx * dx);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < n; z++)
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                double acc = 0.0;
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int ddx = -1; ddx <= 1; ddx++) {
                            int cls = abs(dz) + abs(dy) + abs(ddx);
                            acc += ORC_W27[cls] * f[idx(n, wrap(x + ddx, n), wrap(y + dy, n), wrap(z + dz, n))];
                        }
                out[idx(n, x, y, z)] = acc * inv;
            }
}

/* the configured Laplacian */
static int is27(const orc_lattice *L) { return L->p.stencil == 27; }
static void laplacian_of(const orc_lattice *L, const double *f, double *out)
{
    if (is27(L)) orc_laplacian27(L->n, L->dx, f, out);
    else orc_laplacian(L->n, L->dx, f, out);
}

/* volume average of -f L27 f, the gradient average of the 27-point stencil */
double orc_grad2_mean27(int n, double dx, const double *f)
{
    size_t N3 = (size_t)n * n * n;
    double *lf = (double *)malloc(sizeof(double) * N3);
    orc_laplacian27(n, dx, f, lf);
    double tot = 0.0;
    size_t plane = (size_t)n * n;
    for (int z = 0; z < n; z++) {
        double acc = 0.0;
        for (size_t k = 0; k < plane; k++) acc += -f[(size_t)z * plane + k] * lf[(size_t)z * plane + k];
        tot += acc;
    }
    free(lf);
    return tot / (double)N3;
}

/* volume average of |grad f|^2 with forward differences */
double orc_grad2_mean(int n, double dx, const double *f)
{
    double *plane = (double *)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int z = 0; z < n; z++) {
        double acc = 0.0;
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                double c = f[idx(n, x, y, z)];
                double gx = f[idx(n, wrap(x + 1, n), y, z)] - c;
                double gy = f[idx(n, x, wrap(y + 1, n), z)] - c;
                double gz = f[idx(n, x, y, wrap(z + 1, n))] - c;
                acc += gx * gx + gy * gy + gz * gz;
            }
        plane[z] = acc;
    }
    double tot = 0.0;
    for (int z = 0; z < n; z++) tot += plane[z];
    free(plane);
    return tot / (dx * dx) / ((double)n * n * n);
}

/* volume averages S = (<|grad f0|^2>, <|grad f1|^2>, <f0^beta/beta>, <f0^2 f1^2/2>) */
void orc_sums(orc_lattice *L)
{
    int n = L->n;
    L->S[0] = is27(L) ? orc_grad2_mean27(n, L->dx, L->f[0]) : orc_grad2_mean(n, L->dx, L->f[0]);
    L->S[1] = is27(L) ? orc_grad2_mean27(n, L->dx, L->f[1]) : orc_grad2_mean(n, L->dx, L->f[1]);
    double *pd = (double *)calloc((size_t)n, sizeof(double));
    double *pi = (double *)calloc((size_t)n, sizeof(double));
    const double *f0 = L->f[0], *f1 = L->f[1];
    size_t plane = (size_t)n * n;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < n; z++) {
        double ad = 0.0, ai = 0.0;
        for (size_t k = 0; k < plane; k++) {
            size_t i = (size_t)z * plane + k;
            ad += pow(f0[i], L->beta) / L->beta;
            ai += 0.5 * f0[i] * f0[i] * f1[i] * f1[i];
        }
        pd[z] = ad; pi[z] = ai;
    }
    double td = 0.0, ti = 0.0;
    for (int z = 0; z < n; z++) { td += pd[z]; ti += pi[z]; }
    free(pd); free(pi);
    L->S[2] = td / (double)L->nsites;
    L->S[3] = ti / (double)L->nsites;
}

/* ---------------------------------------------------------------- scale factor */

/* Right-hand side of eq. scale without the a'^2 term:
 * c = (8piG/A^2) a^(-2s-2r-1) ( (S0+S1)/3 + a^(2s+2) <V_pr> ). */
static double scale_source(const orc_lattice *L, double a)
{
    double vpr = cdom_at(L, a) * L->S[2] + kappa_at(L, a) * L->S[3];
    return L->p.eight_pi_G / (L->A * L->A) * pow(a, -2.0 * L->s - 2.0 * L->r - 1.0)
         * ((L->S[0] + L->S[1]) / 3.0 + pow(a, 2.0 * L->s + 2.0) * vpr);
}

/* Staggered update of a' across one step: with a and the sums at t_{n+1/2}
 * and a'_n, solve a'_{n+1} = a'_n + dt a''_{n+1/2} where
 * a''_{n+1/2} = q a'_{n+1/2}^2 + c, q = -(s+2)/a and a'_{n+1/2} = (a'_n + a'_{n+1})/2.
 * With y = a'_n + a'_{n+1}: (dt q/4) y^2 - y + (2 a'_n + dt c) = 0; the root that
 * tends to 2a'_n + dt c as dt -> 0 is y = 2 gamma / (1 + sqrt(1 - 4 alpha gamma)). */
int orc_scale_update(const orc_lattice *L, double *ad_next, double *ad_half, double *add)
{
    double a = L->a, dt = L->p.dt;
    double c = scale_source(L, a);
    double q = -(L->s + 2.0) / a;
    double alpha = dt * q / 4.0;
    double gamma = 2.0 * L->ad + dt * c;
    double disc = 1.0 - 4.0 * alpha * gamma;
    if (!(disc >= 0.0)) return ORC_ENONFINITE;
    double y = 2.0 * gamma / (1.0 + sqrt(disc));
    *ad_half = 0.5 * y;
    *ad_next = y - L->ad;
    *add = q * (*ad_half) * (*ad_half) + c;
    return ORC_OK;
}

/* coefficients of the field equation at the field time:
 * cL = a^(-2s-2), cF = r(s-r+2) h^2 + r a''/a, h = a'/a */
static void field_coefficients(const orc_lattice *L, double a, double ad_half, double add,
                               double *cL, double *cF)
{
    *cL = pow(a, -2.0 * L->s - 2.0);
    double h = ad_half / a;
    *cF = L->r * (L->s - L->r + 2.0) * h * h + L->r * add / a;
}

/* ---------------------------------------------------------------- L = 1/H form */

/* l at the momentum time t from a at the field time t + dt/2 and a' at t:
 * l = a_t / a'_t with a_t = a - (dt/2) a' (the state stores no a at t). */
static double ell_of(double a, double ad, double dt) { return (a - 0.5 * dt * ad) / ad; }

typedef struct {
    double cL, cF;      /* coefficients of eq. scalar-evo at the field time */
    double ad_half;     /* a' at the field time: a h */
    double add;         /* a'' at the field time: a (-s h^2 - Gamma) */
    double ad_next;     /* (a_{n+3/2} - a_{n+1/2}) / dt */
    double ell_next;    /* l_{n+1} */
} orc_lform;

/* The implicit step of the L form at the current field time. Ft_i = cL Lap f_i -
 * dV_pr/df_i (the acceleration without the cF f term). Unknowns l_{n+1} and cF,
 * with Lambda = (l_n + l_{n+1})/2, h = 1/Lambda and the momenta at the field time
 * pi_n + (dt/2)(Ft + cF f):
 *   Gamma    = (8piG/(3A^2)) a^(-2r) (sum_i <(pi_i + (dt/2)(Ft_i + cF f_i) - r h f_i)^2> - <V_pr>)
 *   cF       = r(2-r) h^2 - r Gamma
 *   l_{n+1}  = l_n + dt ((s + 1) + Gamma Lambda^2).
 * Fixed-point iteration from cF = 0, l_{n+1} = l_n, each pass taking the volume
 * average afresh, until neither unknown changes by more than 1e-13 relative to
 * the size of its terms (the iteration contracts by about dt h per pass; below
 * that it cycles through a few rounding levels). */
static int lform_solve(const orc_lattice *L, const double *Ft0, const double *Ft1, orc_lform *o)
{
    const double a = L->a, dt = L->p.dt, r = L->r, s = L->s;
    const double g = L->p.eight_pi_G / (3.0 * L->A * L->A) * pow(a, -2.0 * r);
    const double *f0 = L->f[0], *f1 = L->f[1], *p0 = L->pi[0], *p1 = L->pi[1];
    if (!isfinite(L->ell) || L->ell == 0.0) return ORC_EINVAL;
    double W = 0.0;
    for (size_t k = 0; k < L->nsites; k++) W += Vpr(L, a, f0[k], f1[k]);
    W /= (double)L->nsites;
    double ell_next = L->ell, cF = 0.0, Gam = 0.0;
    int converged = 0;
    for (int it = 0; it < 200 && !converged; it++) {
        double Lam = 0.5 * (L->ell + ell_next), h = 1.0 / Lam;
        double P = 0.0;
        for (size_t k = 0; k < L->nsites; k++) {
            double v0 = p0[k] + 0.5 * dt * (Ft0[k] + cF * f0[k]) - r * h * f0[k];
            double v1 = p1[k] + 0.5 * dt * (Ft1[k] + cF * f1[k]) - r * h * f1[k];
            P += v0 * v0 + v1 * v1;
        }
        P /= (double)L->nsites;
        Gam = g * (P - W);
        double cF_new = r * (2.0 - r) * h * h - r * Gam;
        double ell_new = L->ell + dt * ((s + 1.0) + Gam * Lam * Lam);
        if (!isfinite(cF_new) || !isfinite(ell_new)) return ORC_ENONFINITE;
        /* rounding leaves a cycle of a few ulps of the terms of cF and l */
        converged = fabs(ell_new - ell_next) <= 1e-13 * fabs(ell_new)
                 && fabs(cF_new - cF) <= 1e-13 * fabs(r) * (fabs(2.0 - r) * h * h + fabs(Gam));
        cF = cF_new;
        ell_next = ell_new;
    }
    if (!converged) return ORC_ENONFINITE;
    double h = 2.0 / (L->ell + ell_next);
    o->cL = pow(a, -2.0 * s - 2.0);
    o->cF = cF;
    o->ad_half = a * h;
    o->add = a * (-s * h * h - Gam);
    o->ad_next = a * expm1(dt / ell_next) / dt;   /* a_{n+3/2} - a_{n+1/2} = a (exp(dt/l) - 1) */
    o->ell_next = ell_next;
    return ORC_OK;
}

/* ---------------------------------------------------------------- leapfrog */

/* acceleration F_i = cL Lap f_i + cF f_i - dV_pr/df_i at the field time */
static void accelerations(const orc_lattice *L, double cL, double cF, double *F0, double *F1)
{
    laplacian_of(L, L->f[0], F0);
    laplacian_of(L, L->f[1], F1);
    const double *f0 = L->f[0], *f1 = L->f[1];
    double a = L->a;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)L->nsites; i++) {
        double p0 = f0[i], p1 = f1[i];
        F0[i] = cL * F0[i] + cF * p0 - dVpr0(L, a, p0, p1);
        F1[i] = cL * F1[i] + cF * p1 - dVpr1(L, a, p0, p1);
    }
}

/* The coefficients of the next step at the current field time, from eq. scale
 * (expansion 1) or the L form (expansion 2), and the accelerations
 * F_i = cL Lap f_i + cF f_i - dV_pr/df_i they give. */
static int step_setup(const orc_lattice *L, double *F0, double *F1, double *cL, double *cF, double *ad_next,
                      double *ad_half, double *add, double *ell_next)
{
    *cL = 1.0; *cF = 0.0; *ad_next = 0.0; *ad_half = 0.0; *add = 0.0; *ell_next = L->ell;
    if (L->p.expansion == 1) {
        int st = orc_scale_update(L, ad_next, ad_half, add);
        if (st != ORC_OK) return st;
        field_coefficients(L, L->a, *ad_half, *add, cL, cF);
    }
    if (L->p.expansion == 2) {
        *cL = pow(L->a, -2.0 * L->s - 2.0);
        accelerations(L, *cL, 0.0, F0, F1);
        orc_lform o;
        int st = lform_solve(L, F0, F1, &o);
        if (st != ORC_OK) return st;
        *cF = o.cF; *ad_next = o.ad_next; *ad_half = o.ad_half; *add = o.add; *ell_next = o.ell_next;
        for (size_t k = 0; k < L->nsites; k++) {
            F0[k] += o.cF * L->f[0][k];
            F1[k] += o.cF * L->f[1][k];
        }
        return ORC_OK;
    }
    accelerations(L, *cL, *cF, F0, F1);
    return ORC_OK;
}

/* one step of eq. evo for both fields and for a:
 *   pi_{n+1}    = pi_n + dt F(f_{n+1/2})           (kick, both fields from the same f)
 *   f_{n+3/2}   = f_{n+1/2} + dt pi_{n+1}           (drift)
 *   a_{n+3/2}   = a_{n+1/2} + dt a'_{n+1}
 * (in the L form a'_{n+1} is (a_{n+3/2} - a_{n+1/2})/dt with a_{n+3/2} from l_{n+1},
 * and l advances to l_{n+1}); then the sums are recomputed at the new field time. */
static int one_step(orc_lattice *L, double *F0, double *F1)
{
    double cL, cF, ad_next, ad_half, add, ell_next;
    int st = step_setup(L, F0, F1, &cL, &cF, &ad_next, &ad_half, &add, &ell_next);
    if (st != ORC_OK) return st;
    double dt = L->p.dt;
    double *f0 = L->f[0], *f1 = L->f[1], *p0 = L->pi[0], *p1 = L->pi[1];
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)L->nsites; i++) {
        p0[i] += dt * F0[i];
        p1[i] += dt * F1[i];
    }
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)L->nsites; i++) {
        f0[i] += dt * p0[i];
        f1[i] += dt * p1[i];
    }
    if (L->p.expansion) {
        L->a += dt * ad_next;
        L->ad = ad_next;
        L->ell = ell_next;
    }
    L->t += dt;
    L->step += 1;
    orc_sums(L);
    if (!isfinite(L->S[0]) || !isfinite(L->S[1]) || !isfinite(L->S[2]) || !isfinite(L->S[3])
        || !isfinite(L->a))
        return ORC_ENONFINITE;
    return ORC_OK;
}

int orc_step(orc_lattice *L, int64_t nsteps)
{
    double *F0 = (double *)malloc(L->nsites * sizeof(double));
    double *F1 = (double *)malloc(L->nsites * sizeof(double));
    if (!F0 || !F1) { free(F0); free(F1); return ORC_ENOMEM; }
    int st = ORC_OK;
    for (int64_t k = 0; k < nsteps && st == ORC_OK; k++) st = one_step(L, F0, F1);
    free(F0); free(F1);
    return st;
}

/* Set the scalars of a stored state (t, a, a', step) and recompute the sums. */
void orc_set_scalars(orc_lattice *L, double t, double a, double ad, int64_t step)
{
    L->t = t; L->a = a; L->ad = ad; L->step = step;
    L->ell = ell_of(a, ad, L->p.dt);
    orc_sums(L);
}

/* Threads of the OpenMP loops from here on (timing only; every sum is taken in
 * the same order whatever the count). Returns the count in effect. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* The L form's l = 1/h at the momentum time (set_scalars derives it from a and a'). */
double orc_get_ell(const orc_lattice *L) { return L->ell; }
void orc_set_ell(orc_lattice *L, double ell) { L->ell = ell; }

/* ---------------------------------------------------------------- random numbers */

/* Philox-4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
 * multiplies with the Weyl key schedule. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One standard normal per (seed, field, quantity, site): Philox output words
 * 0 and 1 of counter (site, field, quantity, 0) under key (seed lo, seed hi),
 * mapped to (0,1) as (u + 1/2) 2^-32, then Box-Muller's cosine branch. */
double orc_normal(uint64_t seed, uint32_t field, uint32_t quantity, uint32_t site)
{
    uint32_t ctr[4] = {site, field, quantity, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    double u1 = ((double)o[0] + 0.5) * (1.0 / 4294967296.0);
    double u2 = ((double)o[1] + 0.5) * (1.0 / 4294967296.0);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * ORC_PI * u2);
}

/* ---------------------------------------------------------------- FFT */

/* Recursive mixed-radix Cooley-Tukey DFT of length n (any n >= 1):
 * X[k] = sum_j x[j] exp(sign 2 pi i j k / n). Split by the smallest prime factor p,
 * transform the p decimated subsequences, combine with twiddles. */
static void dft1(int n, const double *xr, const double *xi, int stride, double *yr, double *yi, int sign)
{
    if (n == 1) { yr[0] = xr[0]; yi[0] = xi[0]; return; }
    int p = n;
    for (int d = 2; d * d <= n; d++) if (n % d == 0) { p = d; break; }
    int m = n / p;
    if (m == 1) {
        for (int k = 0; k < n; k++) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < n; j++) {
                double ang = sign * 2.0 * ORC_PI * (double)(((long long)j * k) % n) / n;
                double c = cos(ang), s = sin(ang);
                sr += xr[j * stride] * c - xi[j * stride] * s;
                si += xr[j * stride] * s + xi[j * stride] * c;
            }
            yr[k] = sr; yi[k] = si;
        }
        return;
    }
    double *tr = (double *)malloc(sizeof(double) * n), *ti = (double *)malloc(sizeof(double) * n);
    for (int r = 0; r < p; r++) dft1(m, xr + r * stride, xi + r * stride, stride * p, tr + r * m, ti + r * m, sign);
    for (int k = 0; k < n; k++) {
        int kk = k % m;
        double sr = 0.0, si = 0.0;
        for (int r = 0; r < p; r++) {
            double ang = sign * 2.0 * ORC_PI * (double)(((long long)r * k) % n) / n;
            double c = cos(ang), s = sin(ang);
            sr += tr[r * m + kk] * c - ti[r * m + kk] * s;
            si += tr[r * m + kk] * s + ti[r * m + kk] * c;
        }
        yr[k] = sr; yi[k] = si;
    }
    free(tr); free(ti);
}

void orc_fft1(int n, const double *xr, const double *xi, double *yr, double *yi, int sign)
{
    dft1(n, xr, xi, 1, yr, yi, sign);
}

/* 3D DFT in place on (re, im), x fastest; sign -1 forward, +1 inverse (unnormalised) */
void orc_fft3(int n, double *re, double *im, int sign)
{
    for (int axis = 0; axis < 3; axis++) {
#pragma omp parallel
        {
            double *ar = (double *)malloc(sizeof(double) * n), *ai = (double *)malloc(sizeof(double) * n);
            double *br = (double *)malloc(sizeof(double) * n), *bi = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(static)
            for (int line = 0; line < n * n; line++) {
                int u = line % n, v = line / n;
                for (int j = 0; j < n; j++) {
                    size_t i = axis == 0 ? idx(n, j, u, v) : axis == 1 ? idx(n, u, j, v) : idx(n, u, v, j);
                    ar[j] = re[i]; ai[j] = im[i];
                }
                dft1(n, ar, ai, 1, br, bi, sign);
                for (int j = 0; j < n; j++) {
                    size_t i = axis == 0 ? idx(n, j, u, v) : axis == 1 ? idx(n, u, j, v) : idx(n, u, v, j);
                    re[i] = br[j]; im[i] = bi[j];
                }
            }
            free(ar); free(ai); free(br); free(bi);
        }
    }
}

/* ---------------------------------------------------------------- initial conditions */

static double kcut_of(const orc_lattice *L) { return L->p.kcut > 0.0 ? L->p.kcut : L->n / 4.0; }

/* Gaussian fluctuation of one field (q = 0) or momentum (q = 1): filter white noise
 * W(x) by s(k) in Fourier space. With F(k) = sum_x W(x) e^{-ikx} and the inverse
 * (1/n^3) sum_k, white noise of unit variance has <|F_k|^2> = n^3, and a target
 * per-mode variance P(k) / L^3 in the box needs s(k)^2 = P(k) / dx^3.
 * Vacuum: P = 1/(2 omega) for fields, omega/2 for momenta, with
 * omega^2 = k_lat^2 + m_eff^2 and k_lat^2 = sum_d (2/dx sin(pi n_d / n))^2. The
 * program-unit amplitude carries the factor A B (f = A phi, x_pr = B x). Modes
 * with |n| = 0 or |n| > kcut, and modes with omega^2 <= 0, are left empty. */
/* -L(k) of the configured stencil for the integer wave vector (nx, ny, nz): the
 * lattice k^2 that replaces |k|^2 in the dispersion relation */
static double klat2(const orc_lattice *L, int nx, int ny, int nz)
{
    int n = L->n;
    if (!is27(L)) {
        double sx = 2.0 / L->dx * sin(ORC_PI * nx / n), sy = 2.0 / L->dx * sin(ORC_PI * ny / n),
               sz = 2.0 / L->dx * sin(ORC_PI * nz / n);
        return sx * sx + sy * sy + sz * sz;
    }
    double cx = cos(2.0 * ORC_PI * nx / n), cy = cos(2.0 * ORC_PI * ny / n), cz = cos(2.0 * ORC_PI * nz / n);
    double sym = ORC_W27[0] + 2.0 * ORC_W27[1] * (cx + cy + cz) + 4.0 * ORC_W27[2] * (cx * cy + cx * cz + cy * cz)
               + 8.0 * ORC_W27[3] * cx * cy * cz;
    return -sym / (L->dx * L->dx);
}

static void fluctuation(const orc_lattice *L, int field, int q, double meff2, double *out)
{
    int n = L->n;
    size_t N3 = L->nsites;
    double *re = (double *)malloc(sizeof(double) * N3), *im = (double *)calloc(N3, sizeof(double));
    for (size_t i = 0; i < N3; i++) re[i] = orc_normal(L->p.seed, (uint32_t)field, (uint32_t)q, (uint32_t)i);
    orc_fft3(n, re, im, -1);
    double amp = L->p.fluct * L->A * L->B * pow(L->dx, -1.5);
    double kc = kcut_of(L);
    for (int z = 0; z < n; z++)
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                int nx = x < n / 2 ? x : x - n, ny = y < n / 2 ? y : y - n, nz = z < n / 2 ? z : z - n;
                double nmag = sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
                double w2 = klat2(L, nx, ny, nz) + meff2;
                double scale = 0.0;
                if (nmag > 0.0 && nmag <= kc && w2 > 0.0) {
                    double w = sqrt(w2);
                    scale = amp * (q == 0 ? 1.0 / sqrt(2.0 * w) : sqrt(0.5 * w));
                }
                size_t i = idx(n, x, y, z);
                re[i] *= scale; im[i] *= scale;
            }
    orc_fft3(n, re, im, +1);
    for (size_t i = 0; i < N3; i++) out[i] = re[i] / (double)N3;
    free(re); free(im);
}

/* Sec. II.B, initial values: homogeneous phi0, dphi0 from input, H from the
 * homogeneous energy density, conversion to program units, Gaussian vacuum
 * fluctuations, then the fields (and a) advanced by dt/2. */
int orc_init_fields(orc_lattice *L)
{
    const orc_params *p = &L->p;
    L->t = 0.0; L->a = 1.0; L->step = 0;
    double rho0 = 0.5 * (p->dphi0[0] * p->dphi0[0] + p->dphi0[1] * p->dphi0[1]) + V_phys(L, p->phi0[0], p->phi0[1]);
    L->ad = 0.0;
    if (p->expansion) {
        if (!(rho0 > 0.0)) return ORC_EINVAL;
        double H0 = sqrt(p->eight_pi_G * rho0 / 3.0);
        L->ad = H0 / L->B;  /* a' = a^(1-s) H / B at a = 1 */
    }
    double h0 = L->ad;      /* a'/a at a = 1 */
    double fh[2], ph[2];
    for (int i = 0; i < 2; i++) {
        fh[i] = L->A * p->phi0[i];
        ph[i] = L->A / L->B * p->dphi0[i] + L->r * h0 * fh[i];
    }
    double meff2[2];
    meff2[0] = L->cdom0 * (L->beta - 1.0) * pow(fh[0], L->beta - 2.0) + L->kappa0 * fh[1] * fh[1];
    meff2[1] = L->kappa0 * fh[0] * fh[0];
    double *df = (double *)malloc(sizeof(double) * L->nsites), *dp = (double *)malloc(sizeof(double) * L->nsites);
    if (!df || !dp) { free(df); free(dp); return ORC_ENOMEM; }
    for (int i = 0; i < 2; i++) {
        if (p->fluct != 0.0) {
            fluctuation(L, i, 0, meff2[i], df);
            fluctuation(L, i, 1, meff2[i], dp);
        } else {
            memset(df, 0, sizeof(double) * L->nsites);
            memset(dp, 0, sizeof(double) * L->nsites);
        }
        for (size_t k = 0; k < L->nsites; k++) {
            L->f[i][k] = fh[i] + df[k];
            L->pi[i][k] = ph[i] + dp[k] + L->r * h0 * df[k];
        }
    }
    free(df); free(dp);
    /* half-step desynchronisation: fields (and a) advanced by dt/2 */
    double dt = p->dt;
    for (int i = 0; i < 2; i++)
        for (size_t k = 0; k < L->nsites; k++) L->f[i][k] += 0.5 * dt * L->pi[i][k];
    if (p->expansion) L->a += 0.5 * dt * L->ad;
    L->ell = ell_of(L->a, L->ad, dt);
    orc_sums(L);
    return ORC_OK;
}

/* ---------------------------------------------------------------- diagnostics */

/* Energies at the field time t_{n+1/2}: the momenta there are the average of
 * pi_n and pi_{n+1} (a kick of dt/2 that is not committed), and a' there is the
 * time-centred a'_{n+1/2}. Sec. II.B, eq. rho-pres, converted with
 * phidot = (B/A) a^(s-r) (f' - r h f), grad_x phi = B grad f / (A a^r),
 * V = (B^2/A^2) a^(2s-2r) V_pr:
 *   rho = conv [ sum_i (1/2 (f_i' - r h f_i)^2 + 1/2 a^(-2s-2) |grad f_i|^2) + V_pr ]
 *   p   = conv [ sum_i (1/2 (f_i' - r h f_i)^2 - 1/6 a^(-2s-2) |grad f_i|^2) - V_pr ]
 * with conv = (B^2/A^2) a^(2s-2r). H = B a^s h; K/(a^2H^2) = 8piG<rho>/(3H^2) - 1.
 * out: t, a, a', H, rho, p, w, curv, kin0, kin1, grad0, grad1, pot, mean0, mean1, var0, var1 */
/* Gradient energy density of one site: half of sum over the stencil's
 * neighbours b of w_b (f(x+b) - f(x))^2 / dx^2 (7-point: the six face
 * neighbours with weight 1; 27-point: the 26 neighbours with the weights of
 * ORC_W27). Its volume mean is -<f L f>. */
static double site_grad2(const orc_lattice *L, const double *f, int x, int y, int z)
{
    int n = L->n;
    double c = f[idx(n, x, y, z)], acc = 0.0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int ddx = -1; ddx <= 1; ddx++) {
                int cls = abs(dz) + abs(dy) + abs(ddx);
                if (cls == 0 || (!is27(L) && cls != 1)) continue;
                double w = is27(L) ? ORC_W27[cls] : 1.0;
                double d = f[idx(n, wrap(x + ddx, n), wrap(y + dy, n), wrap(z + dz, n))] - c;
                acc += w * d * d;
            }
    return 0.5 * acc / (L->dx * L->dx);
}

/* Energy density and pressure at every site (eq. rho-pres per site, physical
 * units as in orc_energies): rho = conv (sum_i [kin_i + grad_i] + V),
 * p = conv (sum_i [kin_i - grad_i / 3] - V), with kin_i = (pibar_i - r h f_i)^2 / 2
 * (pibar the momentum at the field time), grad_i = a^(-2s-2) site_grad2 / 2 and
 * V = V_pr. */
int orc_energy_field(orc_lattice *L, double *rho_out, double *p_out)
{
    double cL, cF, ad_next, ad_half, add, ell_next;
    double *F0 = (double *)malloc(L->nsites * sizeof(double)), *F1 = (double *)malloc(L->nsites * sizeof(double));
    if (!F0 || !F1) { free(F0); free(F1); return ORC_ENOMEM; }
    int st = step_setup(L, F0, F1, &cL, &cF, &ad_next, &ad_half, &add, &ell_next);
    if (st != ORC_OK) { free(F0); free(F1); return st; }
    int n = L->n;
    double a = L->a, h = L->p.expansion ? ad_half / a : 0.0, dt = L->p.dt;
    double cg = pow(a, -2.0 * L->s - 2.0);
    double conv = L->B * L->B / (L->A * L->A) * pow(a, 2.0 * L->s - 2.0 * L->r);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < n; z++)
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                size_t k = idx(n, x, y, z);
                double kin = 0.0, grad = 0.0;
                for (int i = 0; i < 2; i++) {
                    const double *F = i == 0 ? F0 : F1;
                    double v = L->pi[i][k] + 0.5 * dt * F[k] - L->r * h * L->f[i][k];
                    kin += 0.5 * v * v;
                    grad += 0.5 * cg * site_grad2(L, L->f[i], x, y, z);
                }
                double V = Vpr(L, a, L->f[0][k], L->f[1][k]);
                rho_out[k] = conv * (kin + grad + V);
                p_out[k] = conv * (kin - grad / 3.0 - V);
            }
    free(F0); free(F1);
    return ORC_OK;
}

int orc_energies(orc_lattice *L, double out[17])
{
    double cL, cF, ad_next, ad_half, add, ell_next;
    double *F0 = (double *)malloc(L->nsites * sizeof(double)), *F1 = (double *)malloc(L->nsites * sizeof(double));
    if (!F0 || !F1) { free(F0); free(F1); return ORC_ENOMEM; }
    int st = step_setup(L, F0, F1, &cL, &cF, &ad_next, &ad_half, &add, &ell_next);
    if (st != ORC_OK) { free(F0); free(F1); return st; }
    double a = L->a, h = L->p.expansion ? ad_half / a : 0.0, dt = L->p.dt;
    double kin[2] = {0, 0}, mean[2] = {0, 0}, var[2] = {0, 0}, pot = 0.0;
    for (int i = 0; i < 2; i++) {
        const double *F = i == 0 ? F0 : F1;
        double acc = 0.0, accm = 0.0;
        for (size_t k = 0; k < L->nsites; k++) {
            double pibar = L->pi[i][k] + 0.5 * dt * F[k];
            double v = pibar - L->r * h * L->f[i][k];
            acc += 0.5 * v * v;
            accm += L->f[i][k];
        }
        kin[i] = acc / (double)L->nsites;
        mean[i] = accm / (double)L->nsites;
        double accv = 0.0;
        for (size_t k = 0; k < L->nsites; k++) { double d = L->f[i][k] - mean[i]; accv += d * d; }
        var[i] = accv / (double)L->nsites;
    }
    for (size_t k = 0; k < L->nsites; k++) pot += Vpr(L, a, L->f[0][k], L->f[1][k]);
    pot /= (double)L->nsites;
    free(F0); free(F1);
    double cg = pow(a, -2.0 * L->s - 2.0);
    double grad[2];
    for (int i = 0; i < 2; i++)
        grad[i] = 0.5 * cg * (is27(L) ? orc_grad2_mean27(L->n, L->dx, L->f[i]) : orc_grad2_mean(L->n, L->dx, L->f[i]));
    double conv = L->B * L->B / (L->A * L->A) * pow(a, 2.0 * L->s - 2.0 * L->r);
    double rho = conv * (kin[0] + kin[1] + grad[0] + grad[1] + pot);
    double pres = conv * (kin[0] + kin[1] - (grad[0] + grad[1]) / 3.0 - pot);
    double H = L->B * pow(a, L->s) * h;
    out[0] = L->t + 0.5 * dt;
    out[1] = a;
    out[2] = L->p.expansion ? ad_half : 0.0;
    out[3] = H;
    out[4] = rho;
    out[5] = pres;
    out[6] = pres / rho;
    out[7] = H != 0.0 ? L->p.eight_pi_G * rho / (3.0 * H * H) - 1.0 : NAN;
    out[8] = conv * kin[0]; out[9] = conv * kin[1];
    out[10] = conv * grad[0]; out[11] = conv * grad[1];
    out[12] = conv * pot;
    out[13] = mean[0]; out[14] = mean[1];
    out[15] = var[0]; out[16] = var[1];
    return ORC_OK;
}

/* Shell-binned power spectrum of one field (Sec. IV names it as future work):
 * bin b = round(|n|), n the integer wave vector; p_out[b] is the shell mean of
 * |F_k|^2 / n^3 (F = forward DFT, so unit white noise gives 1), k_out[b] the shell
 * mean of 2 pi |n| / L, count_out[b] the number of modes. */
int orc_spectrum(orc_lattice *L, int field, int nbins, double *k_out, double *p_out, int64_t *count_out)
{
    int n = L->n;
    size_t N3 = L->nsites;
    double *re = (double *)malloc(sizeof(double) * N3), *im = (double *)calloc(N3, sizeof(double));
    if (!re || !im) { free(re); free(im); return ORC_ENOMEM; }
    memcpy(re, L->f[field], sizeof(double) * N3);
    orc_fft3(n, re, im, -1);
    for (int b = 0; b < nbins; b++) { k_out[b] = 0.0; p_out[b] = 0.0; count_out[b] = 0; }
    for (int z = 0; z < n; z++)
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                int nx = x < n / 2 ? x : x - n, ny = y < n / 2 ? y : y - n, nz = z < n / 2 ? z : z - n;
                double nmag = sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
                int b = (int)floor(nmag + 0.5);
                if (b >= nbins) continue;
                size_t i = idx(n, x, y, z);
                p_out[b] += (re[i] * re[i] + im[i] * im[i]) / (double)N3;
                k_out[b] += 2.0 * ORC_PI * nmag / L->p.L;
                count_out[b] += 1;
            }
    for (int b = 0; b < nbins; b++)
        if (count_out[b] > 0) { p_out[b] /= (double)count_out[b]; k_out[b] /= (double)count_out[b]; }
    free(re); free(im);
    return ORC_OK;
}

/* ---------------------------------------------------------------- coupling */

/* Change g^2 (and with it kappa0 = g^2 / (A^2 B^2)) of an existing lattice; the
 * state and the sums (which do not involve g^2) are kept. */
/* Observable 1 of the derivative: the fraction of the energy density in chi,
 * at the momentum time t of the stored state (fields taken back half a step,
 * f_t = f - (dt/2) pi; a_t = a - (dt/2) a'; h = a'/a_t):
 *   K_i = <(pi_i - r h f_t,i)^2> / 2,   G_i = a_t^(-2s-2) <|grad+ f_t,i|^2> / 2,
 *   W = <V_pr(f_t; a_t)>,   J = (K_1 + G_1) / (K_0 + K_1 + G_0 + G_1 + W),
 * the terms of eq. rho-pres, whose physical factor (B/A)^2 a^(2s-2r) cancels in
 * the ratio; the interaction energy counts in the total only. 7-point gradient.
 * Writes J and, when fbar is not NULL, its gradient with respect to the stored
 * f and pi (fbar, pibar, n^3 each), to a and a' (sb[0], sb[1]) and its direct
 * derivative with respect to g^2 (sb[2]: through kappa0 = g^2/(A^2 B^2) in W,
 * at a fixed state). */
int orc_chi_fraction(const orc_lattice *L, double *J_out, double *fbar[2], double *pibar[2], double sb[3])
{
    const int n = L->n;
    const size_t N3 = L->nsites;
    const double dt = L->p.dt, r = L->r, s = L->s;
    if (L->p.expansion == 2 || is27(L)) return ORC_EINVAL;
    const double at = L->a - 0.5 * dt * L->ad;
    const double h = L->p.expansion ? L->ad / at : 0.0;
    const double cg = pow(at, -2.0 * s - 2.0), cd = cdom_at(L, at), kp = kappa_at(L, at);
    double *ft[2], *lap[2];
    for (int i = 0; i < 2; i++) {
        ft[i] = (double *)malloc(N3 * sizeof(double));
        lap[i] = (double *)malloc(N3 * sizeof(double));
    }
    if (!ft[0] || !ft[1] || !lap[0] || !lap[1]) {
        for (int i = 0; i < 2; i++) { free(ft[i]); free(lap[i]); }
        return ORC_ENOMEM;
    }
    for (int i = 0; i < 2; i++)
        for (size_t k = 0; k < N3; k++) ft[i][k] = L->f[i][k] - 0.5 * dt * L->pi[i][k];
    double K[2], G[2], UF[2], Wd = 0.0, Wi = 0.0;
    for (int i = 0; i < 2; i++) {
        double kk = 0.0, uf = 0.0;
        for (size_t k = 0; k < N3; k++) {
            double u = L->pi[i][k] - r * h * ft[i][k];
            kk += 0.5 * u * u;
            uf += u * ft[i][k];
        }
        K[i] = kk / (double)N3;
        UF[i] = uf / (double)N3;
        G[i] = 0.5 * cg * orc_grad2_mean(n, L->dx, ft[i]);
    }
    for (size_t k = 0; k < N3; k++) {
        Wd += pow(ft[0][k], L->beta) / L->beta;
        Wi += 0.5 * ft[0][k] * ft[0][k] * ft[1][k] * ft[1][k];
    }
    Wd /= (double)N3;
    Wi /= (double)N3;
    const double W = cd * Wd + kp * Wi;
    const double D = K[0] + K[1] + G[0] + G[1] + W, J = (K[1] + G[1]) / D;
    *J_out = J;
    if (fbar) {
        /* dJ = (dN - J dD) / D: weight (1 - J)/D on chi's own terms, -J/D on the rest */
        const double w[2] = {-J / D, (1.0 - J) / D}, wW = -J / D;
        for (int i = 0; i < 2; i++) orc_laplacian(n, L->dx, ft[i], lap[i]);
        for (size_t k = 0; k < N3; k++) {
            const double a0 = ft[0][k], a1 = ft[1][k];
            const double dW[2] = {cd * pow(a0, L->beta - 1.0) + kp * a0 * a1 * a1, kp * a0 * a0 * a1};
            for (int i = 0; i < 2; i++) {
                const double u = L->pi[i][k] - r * h * ft[i][k];
                const double gf = (w[i] * (-r * h * u - cg * lap[i][k]) + wW * dW[i]) / (double)N3;
                fbar[i][k] = gf;
                pibar[i][k] = w[i] * u / (double)N3 - 0.5 * dt * gf;
            }
        }
        const double dJ_dh = w[0] * (-r * UF[0]) + w[1] * (-r * UF[1]);
        const double dJ_dat = (w[0] * G[0] + w[1] * G[1]) * (-2.0 * s - 2.0) / at
                            + wW * (L->pdom * cd * Wd + L->pint * kp * Wi) / at;
        const double dh_da = L->p.expansion ? -L->ad / (at * at) : 0.0;
        const double dh_dad = L->p.expansion ? 1.0 / at + 0.5 * dt * L->ad / (at * at) : 0.0;
        sb[0] = L->p.expansion ? dJ_dat + dJ_dh * dh_da : 0.0;
        sb[1] = L->p.expansion ? -0.5 * dt * dJ_dat + dJ_dh * dh_dad : 0.0;
        sb[2] = wW * Wi * pow(at, L->pint) / (L->A * L->A * L->B * L->B);
    }
    for (int i = 0; i < 2; i++) { free(ft[i]); free(lap[i]); }
    return ORC_OK;
}

int orc_set_g2(orc_lattice *L, double g2)
{
    L->p.g2 = g2;
    return orc_derive(L);
}

/* ---------------------------------------------------------------- adjoint */

/*
 * Reverse-mode derivative (vector-Jacobian product) of nsteps leapfrog steps of
 * one_step above, taken exactly through every dependence of the discrete step:
 * the kick's Laplacian, potential and cF f terms, the drift, the a / a' update,
 * and the dependence of a'', cF, cdom, kappa (and so of every later step) on the
 * volume sums S of the fields, i.e. the coupling of the fields to a(t) through
 * eq. scale. kappa0 (hence g^2) is an input too.
 *
 * Forward step k, state (f_k, pi_k, a_k, a'_k), sums S_k = S(f_k):
 *   c = K a^e1 ((S0+S1)/3 + a^e2 (cdom(a) S2 + kappa(a) S3)), K = 8piG/A^2,
 *       e1 = -2s-2r-1, e2 = 2s+2
 *   q = -(s+2)/a, alpha = dt q/4, gamma = 2a'_k + dt c, y = root of
 *       alpha y^2 - y + gamma = 0, a'_half = y/2, a'' = q a'_half^2 + c
 *   cL = a^(-2s-2), cF = r(s-r+2) (a'_half/a)^2 + r a''/a
 *   pi_{k+1} = pi_k + dt (cL Lap f_k + cF f_k - dV_pr/df(f_k; cdom, kappa))
 *   f_{k+1} = f_k + dt pi_{k+1}
 *   a'_{k+1} = y - a'_k, a_{k+1} = a_k + dt a'_{k+1}
 * (expansion off: a, a' fixed, cL = 1, cF = 0.)
 *
 * The reverse sweep walks the steps backwards; within a step it reverses the
 * statements above in the opposite order. The adjoint of the global sums S_k
 * feeds back to every site through dS/df:
 *   dS0/df0 = -2 Lap f0 / N^3, dS1/df1 = -2 Lap f1 / N^3,
 *   dS2/df0 = f0^(beta-1) / N^3, dS3/df0 = f0 f1^2 / N^3, dS3/df1 = f0^2 f1 / N^3
 * (the first two by the summation-by-parts identity of Sec. II.B).
 *
 * In:  fbar[2], pibar[2] (nsites each): the adjoint of the final f and pi;
 *      sbar[0..1]: the adjoint of the final a and a'.
 * Out: fbar, pibar overwritten by the adjoint of the initial f and pi;
 *      sbar[0..1] the adjoint of the initial a and a', sbar[2] dJ/dkappa0 and
 *      sbar[3] dJ/dg^2 = dJ/dkappa0 / (A^2 B^2).
 * The lattice itself ends advanced by nsteps (as after orc_step). All states
 * are kept in memory: this is meant for small lattices.
 */

/* forward scalars of one step from (a, a', S) */
typedef struct {
    double c, q, alpha, gamma, y, ah, add, cL, cF, cd, kp, vpr, e1v, e2v;
} orc_coefs;

static int step_coefs(const orc_lattice *L, double a, double ad, const double S[4], orc_coefs *o)
{
    memset(o, 0, sizeof(*o));
    o->cd = cdom_at(L, a);
    o->kp = kappa_at(L, a);
    o->cL = 1.0;
    o->cF = 0.0;
    if (!L->p.expansion) return ORC_OK;
    double dt = L->p.dt, r = L->r, s = L->s;
    o->vpr = o->cd * S[2] + o->kp * S[3];
    o->e1v = pow(a, -2.0 * s - 2.0 * r - 1.0);
    o->e2v = pow(a, 2.0 * s + 2.0);
    o->c = L->p.eight_pi_G / (L->A * L->A) * o->e1v * ((S[0] + S[1]) / 3.0 + o->e2v * o->vpr);
    o->q = -(s + 2.0) / a;
    o->alpha = dt * o->q / 4.0;
    o->gamma = 2.0 * ad + dt * o->c;
    double disc = 1.0 - 4.0 * o->alpha * o->gamma;
    if (!(disc >= 0.0)) return ORC_ENONFINITE;
    o->y = 2.0 * o->gamma / (1.0 + sqrt(disc));
    o->ah = 0.5 * o->y;
    o->add = o->q * o->ah * o->ah + o->c;
    o->cL = pow(a, -2.0 * s - 2.0);
    double h = o->ah / a;
    o->cF = r * (s - r + 2.0) * h * h + r * o->add / a;
    return ORC_OK;
}

/* Reverse of step_coefs: from the adjoints of cL, cF, cdom, kappa and y, add to
 * the adjoints of a, a', S[0..3] and kappa0. */
static void step_coefs_adjoint(const orc_lattice *L, double a, const double S[4], const orc_coefs *o,
                               double bcL, double bcF, double bcd, double bkp, double by,
                               double *ba, double *bad, double bS[4], double *bk0)
{
    double r = L->r, s = L->s, dt = L->p.dt;
    if (L->p.expansion) {
        double h = o->ah / a;
        /* cF = r (s-r+2) h^2 + r add / a */
        double bh = bcF * 2.0 * r * (s - r + 2.0) * h;
        double badd = bcF * r / a;
        *ba -= bcF * r * o->add / (a * a);
        /* h = ah / a */
        double bah = bh / a;
        *ba -= bh * o->ah / (a * a);
        /* add = q ah^2 + c */
        double bq = badd * o->ah * o->ah;
        bah += badd * 2.0 * o->q * o->ah;
        double bc = badd;
        /* ah = y / 2 */
        by += 0.5 * bah;
        /* alpha y^2 - y + gamma = 0: dy = (y^2 dalpha + dgamma) / (1 - 2 alpha y) */
        double den = 1.0 - 2.0 * o->alpha * o->y;
        double bgamma = by / den, balpha = by * o->y * o->y / den;
        /* alpha = dt q / 4, gamma = 2 a' + dt c */
        bq += balpha * dt / 4.0;
        *bad += 2.0 * bgamma;
        bc += dt * bgamma;
        /* q = -(s+2)/a */
        *ba += bq * (s + 2.0) / (a * a);
        /* cL = a^(-2s-2) */
        *ba += bcL * (-2.0 * s - 2.0) * pow(a, -2.0 * s - 3.0);
        /* c = K e1v (T + e2v vpr), T = (S0+S1)/3 */
        double K = L->p.eight_pi_G / (L->A * L->A);
        double T = (S[0] + S[1]) / 3.0;
        double be1 = bc * K * (T + o->e2v * o->vpr);
        double bT = bc * K * o->e1v;
        double be2 = bc * K * o->e1v * o->vpr;
        double bvpr = bc * K * o->e1v * o->e2v;
        *ba += be1 * (-2.0 * s - 2.0 * r - 1.0) * pow(a, -2.0 * s - 2.0 * r - 2.0);
        *ba += be2 * (2.0 * s + 2.0) * pow(a, 2.0 * s + 1.0);
        bS[0] += bT / 3.0;
        bS[1] += bT / 3.0;
        /* vpr = cdom S2 + kappa S3 */
        bcd += bvpr * S[2];
        bkp += bvpr * S[3];
        bS[2] += bvpr * o->cd;
        bS[3] += bvpr * o->kp;
    }
    /* cdom = cdom0 a^pdom, kappa = kappa0 a^pint */
    *ba += bcd * L->cdom0 * L->pdom * pow(a, L->pdom - 1.0) + bkp * L->kappa0 * L->pint * pow(a, L->pint - 1.0);
    *bk0 += bkp * pow(a, L->pint);
}

/* sum over all sites of an array, plane by plane in z order */
static double volume_sum(int n, const double *v)
{
    size_t plane = (size_t)n * n;
    double tot = 0.0;
    for (int z = 0; z < n; z++) {
        double acc = 0.0;
        for (size_t k = 0; k < plane; k++) acc += v[(size_t)z * plane + k];
        tot += acc;
    }
    return tot;
}

int orc_adjoint(orc_lattice *L, int64_t nsteps, double *fbar[2], double *pibar[2], double sbar[4])
{
    if (L->p.expansion == 2) return ORC_EINVAL;   /* the reverse pass follows eq. scale only */
    const size_t N3 = L->nsites;
    const int n = L->n;
    const double dt = L->p.dt, beta = L->beta;
    if (nsteps < 0) return ORC_EINVAL;
    /* forward: keep f_k (both fields) and (a_k, a'_k, S_k) of every step */
    double *fs = (double *)malloc(sizeof(double) * 2 * N3 * (size_t)(nsteps + 1));
    double *sc = (double *)malloc(sizeof(double) * 6 * (size_t)(nsteps + 1));
    double *w = (double *)malloc(sizeof(double) * 8 * N3);
    if (!fs || !sc || !w) { free(fs); free(sc); free(w); return ORC_ENOMEM; }
    int st = ORC_OK;
    for (int64_t k = 0; k <= nsteps && st == ORC_OK; k++) {
        memcpy(fs + (size_t)k * 2 * N3, L->f[0], sizeof(double) * N3);
        memcpy(fs + (size_t)k * 2 * N3 + N3, L->f[1], sizeof(double) * N3);
        sc[6 * k + 0] = L->a;
        sc[6 * k + 1] = L->ad;
        for (int i = 0; i < 4; i++) sc[6 * k + 2 + i] = L->S[i];
        if (k < nsteps) st = orc_step(L, 1);
    }
    double *pt0 = w, *pt1 = w + N3, *lp0 = w + 2 * N3, *lp1 = w + 3 * N3;
    double *lf0 = w + 4 * N3, *lf1 = w + 5 * N3, *t0 = w + 6 * N3, *t1 = w + 7 * N3;
    double ba = sbar[0], bad = sbar[1], bk0 = 0.0;
    const double inv_n3 = 1.0 / (double)N3;
    for (int64_t k = nsteps - 1; k >= 0 && st == ORC_OK; k--) {
        const double *f0 = fs + (size_t)k * 2 * N3, *f1 = f0 + N3;
        const double a = sc[6 * k + 0], ad = sc[6 * k + 1], *S = sc + 6 * k + 2;
        orc_coefs o;
        st = step_coefs(L, a, ad, S, &o);
        if (st != ORC_OK) break;
        /* drift f_{k+1} = f_k + dt pi_{k+1}: pi_{k+1} sees pibar + dt fbar */
        for (size_t i = 0; i < N3; i++) {
            pt0[i] = pibar[0][i] + dt * fbar[0][i];
            pt1[i] = pibar[1][i] + dt * fbar[1][i];
        }
        /* a_{k+1} = a_k + dt a'_{k+1}, a'_{k+1} = y - a'_k */
        double by = 0.0;
        if (L->p.expansion) {
            by = bad + dt * ba;
            bad = -by;
        }
        /* kick pi_{k+1} = pi_k + dt (cL Lap f + cF f - dV/df): adjoints of the
         * step coefficients are volume sums */
        laplacian_of(L, f0, lf0);
        laplacian_of(L, f1, lf1);
        for (size_t i = 0; i < N3; i++) t0[i] = pt0[i] * lf0[i] + pt1[i] * lf1[i];
        double bcL = dt * volume_sum(n, t0);
        for (size_t i = 0; i < N3; i++) t0[i] = pt0[i] * f0[i] + pt1[i] * f1[i];
        double bcF = dt * volume_sum(n, t0);
        for (size_t i = 0; i < N3; i++) t0[i] = pt0[i] * pow(f0[i], beta - 1.0);
        double bcd = -dt * volume_sum(n, t0);
        for (size_t i = 0; i < N3; i++) t0[i] = pt0[i] * f0[i] * f1[i] * f1[i] + pt1[i] * f0[i] * f0[i] * f1[i];
        double bkp = -dt * volume_sum(n, t0);
        double bS[4] = {0.0, 0.0, 0.0, 0.0};
        step_coefs_adjoint(L, a, S, &o, bcL, bcF, bcd, bkp, by, &ba, &bad, bS, &bk0);
        /* field adjoints: fbar_k = fbar_{k+1} + dt (dF/df)^T pt + sum_j bS_j dS_j/df */
        laplacian_of(L, pt0, lp0);
        laplacian_of(L, pt1, lp1);
        for (size_t i = 0; i < N3; i++) {
            double p0 = f0[i], p1 = f1[i];
            double h00 = o.cd * (beta - 1.0) * pow(p0, beta - 2.0) + o.kp * p1 * p1;
            double h01 = 2.0 * o.kp * p0 * p1;
            double h11 = o.kp * p0 * p0;
            double g0 = o.cL * lp0[i] + o.cF * pt0[i] - h00 * pt0[i] - h01 * pt1[i];
            double g1 = o.cL * lp1[i] + o.cF * pt1[i] - h01 * pt0[i] - h11 * pt1[i];
            double s0 = bS[0] * (-2.0 * lf0[i]) + bS[2] * pow(p0, beta - 1.0) + bS[3] * p0 * p1 * p1;
            double s1 = bS[1] * (-2.0 * lf1[i]) + bS[3] * p0 * p0 * p1;
            fbar[0][i] += dt * g0 + s0 * inv_n3;
            fbar[1][i] += dt * g1 + s1 * inv_n3;
            pibar[0][i] = pt0[i];
            pibar[1][i] = pt1[i];
        }
    }
    sbar[0] = ba;
    sbar[1] = bad;
    sbar[2] = bk0;
    sbar[3] = bk0 / (L->A * L->A * L->B * L->B);
    free(fs); free(sc); free(w);
    return st;
}

/* Coefficients of one step from the scalars it starts from (a, a' and the
 * volume averages S of its fields): out = (cL, cF, cdom, kappa, y) with
 * y = a'_n + a'_{n+1} (0 without expansion). For drivers that assemble the
 * averages themselves (domain-decomposed runs in the tests). */
int orc_step_coefs(const orc_lattice *L, double a, double ad, const double S[4], double out[5])
{
    if (L->p.expansion == 2) return ORC_EINVAL;
    orc_coefs o;
    int st = step_coefs(L, a, ad, S, &o);
    out[0] = o.cL; out[1] = o.cF; out[2] = o.cd; out[3] = o.kp; out[4] = o.y;
    return st;
}
