/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the per-timestep short-range force
 * evaluation of Pal, Agarwala, Raha & Bhattacharya, "Performance metrics in a hybrid
 * MPI-OpenMP based molecular dynamics simulation with short-range interactions"
 * (arXiv:1507.07068).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library product calls this file: it is
 * loaded by the tests, by the package's smoke check and by the benchmark's CPU
 * baseline leg.  It shares no code, header, table builder or constant with the CUDA
 * path; the two meet only in the seeded inputs and the parameter set they both receive.
 *
 * What it computes (all FP64, C99, no FMA contraction: built with -ffp-contract=off):
 *   - the potential functions of the Appendix: f(r) (Eq. A2), F(rho) and M(P) (Eq. A3),
 *     the Pasianot pair term Phi(x) (Eq. A4) and the Cr-C Morse term phi(y) (Eq. A5),
 *     analytic or as cubic Hermite tables, with an optional shifted-force cutoff;
 *   - the total energy of Eq. A1 plus the Morse film-indenter energy, and the forces
 *     F_i = -dE/dx_i, which reproduce Eq. (1) of Sec. 3.1 with the M(P) term added
 *     (the symmetric (F'_i + F'_j) and (M'_i + M'_j) factors) and the Morse force;
 *   - neighbour sets by brute force over all pairs or by a cell list (Sec. 2.6);
 *   - the time loop of Fig. 5 / Table 1: neighbour-list check and rebuild (Task 1),
 *     indenter motion (Task 2), velocity-Verlet half kick and drift (Task 3,
 *     Eqs. A11-A12), densities and forces (Task 4, Eqs. A1-A10, A13) and the closing
 *     half kick (Task 5);
 *   - energy sums with self-compensated (Neumaier) summation (Sec. 2.3).
 *
 * Per-atom loops carry "omp parallel for" (the paper's thread layer, Sec. 3.3.1);
 * every thread writes only its own atom and every global sum runs afterwards in
 * index order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ parameters */

typedef struct {
    /* EAM, Appendix Eqs. A2-A4 */
    double r_e, f_e, beta;      /* f(r) = f_e (r_e / r)^beta                    */
    double F_o, n, rho_e;       /* F(rho) = -F_o [1 - n ln(rho/rho_e)] (rho/rho_e)^n */
    double alpha, P_e;          /* M(P) = alpha u^2 exp(-u^2), u = P/P_e - 1    */
    double a0, a1, a2, a3, d;   /* Phi(x) = (x-d)^2 (a3 x^3 + a2 x^2 + a1 x + a0), x = r/r_e */
    /* Morse, Eq. A5 */
    double D_o, alpha_x, y_eq;
    /* cutoffs and tabulation */
    double rc, rc_m;
    int32_t shifted, tabulated;
    double r_min, h;
} or_params;

typedef struct {
    or_params p;
    double f_rc, df_rc;          /* unshifted f and f' at rc   (shift constants) */
    double m_rc, dm_rc;          /* unshifted phi and phi' at rc_m               */
    int nf, nm;                  /* table intervals on [r_min, rc] and [r_min, rc_m] */
    double hf, hm;               /* their spacings                              */
    double *tf_v, *tf_d;         /* f knots: value, slope                       */
    double *tp_v, *tp_d;         /* Phi knots                                   */
    double *tm_v, *tm_d;         /* Morse knots                                 */
} or_pot;

enum { OR_F = 0, OR_PHI = 1, OR_MORSE = 2, OR_EMBED = 3, OR_MTERM = 4,
       OR_F_RAW = 5, OR_PHI_AN = 6, OR_MORSE_RAW = 7 };

/* f(r) of Eq. A2 and its derivative */
static double f_raw(const or_params *p, double r) { return p->f_e * pow(p->r_e / r, p->beta); }
static double df_raw(const or_params *p, double r) { return -p->beta * f_raw(p, r) / r; }

/* Phi of Eq. A4 in r; derivative by the product rule on (x-d)^2 * poly(x) */
static void phi_an(const or_params *p, double r, double *v, double *dv)
{
    double x = r / p->r_e;
    if (x > p->d) { *v = 0.0; *dv = 0.0; return; }
    double poly = ((p->a3 * x + p->a2) * x + p->a1) * x + p->a0;
    double dpoly = (3.0 * p->a3 * x + 2.0 * p->a2) * x + p->a1;
    double t = x - p->d;
    *v = t * t * poly;
    *dv = (2.0 * t * poly + t * t * dpoly) / p->r_e;
}

/* Morse of Eq. A5 and its derivative in y */
static void morse_raw(const or_params *p, double y, double *v, double *dv)
{
    double q = y / p->y_eq - 1.0;
    double e1 = exp(-p->alpha_x * q);
    double e2 = exp(-0.5 * p->alpha_x * q);
    *v = p->D_o * (e1 - 2.0 * e2);
    *dv = p->D_o * (-p->alpha_x * e1 + p->alpha_x * e2) / p->y_eq;
}

/* analytic f with the cutoff rule: shifted force f(r) - f(rc) - (r - rc) f'(rc), or plain truncation */
static void f_an(const or_pot *P, double r, double *v, double *dv)
{
    const or_params *p = &P->p;
    if (r >= p->rc) { *v = 0.0; *dv = 0.0; return; }
    *v = f_raw(p, r);
    *dv = df_raw(p, r);
    if (p->shifted) { *v -= P->f_rc + (r - p->rc) * P->df_rc; *dv -= P->df_rc; }
}

static void morse_an(const or_pot *P, double y, double *v, double *dv)
{
    const or_params *p = &P->p;
    if (y >= p->rc_m) { *v = 0.0; *dv = 0.0; return; }
    morse_raw(p, y, v, dv);
    if (p->shifted) { *v -= P->m_rc + (y - p->rc_m) * P->dm_rc; *dv -= P->dm_rc; }
}

/* Knot values of the tables are evaluated in extended precision (long double) and rounded
 * once to FP64: a Hermite slope carries the knot-value rounding amplified by 1.5/h, so knots
 * rounded once from a more precise value make the table reproducible to the last bit. */
static long double f_raw_l(const or_params *p, long double r)
{
    return (long double)p->f_e * powl((long double)p->r_e / r, (long double)p->beta);
}

static void phi_l(const or_params *p, long double r, long double *v, long double *dv)
{
    long double x = r / (long double)p->r_e, d = p->d;
    if (x > d) { *v = 0.0L; *dv = 0.0L; return; }
    long double a0 = p->a0, a1 = p->a1, a2 = p->a2, a3 = p->a3;
    long double poly = ((a3 * x + a2) * x + a1) * x + a0;
    long double dpoly = (3.0L * a3 * x + 2.0L * a2) * x + a1;
    long double t = x - d;
    *v = t * t * poly;
    *dv = (2.0L * t * poly + t * t * dpoly) / (long double)p->r_e;
}

static void morse_l(const or_params *p, long double y, long double *v, long double *dv)
{
    long double q = y / (long double)p->y_eq - 1.0L, ax = p->alpha_x;
    long double e1 = expl(-ax * q), e2 = expl(-0.5L * ax * q);
    *v = (long double)p->D_o * (e1 - 2.0L * e2);
    *dv = (long double)p->D_o * (-ax * e1 + ax * e2) / (long double)p->y_eq;
}

/* cubic Hermite interpolation on knots (value, slope) with spacing h from r0.  The basis
 * h00 + h01 = 1 and h01' = -h00' is used to write both value and slope with the knot
 * difference g_{k+1} - g_k, so no two large terms cancel before the division by h. */
static void hermite(const double *kv, const double *kd, int nint, double r0, double h,
                    double r, double *v, double *dv)
{
    double s = (r - r0) / h;
    int k = (int)floor(s);
    if (k < 0) k = 0;                 /* below r_min: the first cubic is extended */
    if (k > nint - 1) k = nint - 1;
    double t = s - (double)k;
    double t2 = t * t, t3 = t2 * t;
    double h01 = -2.0 * t3 + 3.0 * t2;                          /* = 1 - h00 */
    double h10 = t3 - 2.0 * t2 + t, h11 = t3 - t2;
    double g01 = -6.0 * t2 + 6.0 * t;                           /* = -h00'   */
    double g10 = 3.0 * t2 - 4.0 * t + 1.0, g11 = 3.0 * t2 - 2.0 * t;
    double dg = kv[k + 1] - kv[k];
    *v = kv[k] + h01 * dg + h10 * h * kd[k] + h11 * h * kd[k + 1];
    *dv = g01 * dg / h + g10 * kd[k] + g11 * kd[k + 1];
}

static int n_intervals(double a, double b, double h0)
{
    int n = (int)ceil((b - a) / h0 - 1e-9);
    return n < 1 ? 1 : n;
}

void or_pot_free(or_pot *P)
{
    if (!P) return;
    free(P->tf_v); free(P->tf_d); free(P->tp_v); free(P->tp_d); free(P->tm_v); free(P->tm_d);
    free(P);
}

or_pot *or_pot_new(const or_params *p)
{
    or_pot *P = (or_pot *)calloc(1, sizeof(or_pot));
    if (!P) return NULL;
    P->p = *p;
    P->f_rc = f_raw(p, p->rc);
    P->df_rc = df_raw(p, p->rc);
    morse_raw(p, p->rc_m, &P->m_rc, &P->dm_rc);
    if (p->tabulated) {
        P->nf = n_intervals(p->r_min, p->rc, p->h);
        P->nm = n_intervals(p->r_min, p->rc_m, p->h);
        P->hf = (p->rc - p->r_min) / P->nf;
        P->hm = (p->rc_m - p->r_min) / P->nm;
        P->tf_v = malloc(sizeof(double) * (P->nf + 1)); P->tf_d = malloc(sizeof(double) * (P->nf + 1));
        P->tp_v = malloc(sizeof(double) * (P->nf + 1)); P->tp_d = malloc(sizeof(double) * (P->nf + 1));
        P->tm_v = malloc(sizeof(double) * (P->nm + 1)); P->tm_d = malloc(sizeof(double) * (P->nm + 1));
        if (!P->tf_v || !P->tf_d || !P->tp_v || !P->tp_d || !P->tm_v || !P->tm_d) { or_pot_free(P); return NULL; }
        long double frc = f_raw_l(p, p->rc), dfrc = -(long double)p->beta * frc / (long double)p->rc;
        long double mrc, dmrc;
        morse_l(p, p->rc_m, &mrc, &dmrc);
        for (int k = 0; k <= P->nf; ++k) {
            double r = (k == P->nf) ? p->rc : p->r_min + k * P->hf;
            /* knot at r = rc takes the limit from below (value of the r < rc branch) */
            long double rl = r, fv = f_raw_l(p, rl), fd = -(long double)p->beta * fv / rl, pv, pd;
            if (p->shifted) { fv -= frc + (rl - (long double)p->rc) * dfrc; fd -= dfrc; }
            P->tf_v[k] = (double)fv; P->tf_d[k] = (double)fd;
            phi_l(p, rl, &pv, &pd);
            P->tp_v[k] = (double)pv; P->tp_d[k] = (double)pd;
        }
        for (int k = 0; k <= P->nm; ++k) {
            double y = (k == P->nm) ? p->rc_m : p->r_min + k * P->hm;
            long double yl = y, mv, md;
            morse_l(p, yl, &mv, &md);
            if (p->shifted) { mv -= mrc + (yl - (long double)p->rc_m) * dmrc; md -= dmrc; }
            P->tm_v[k] = (double)mv; P->tm_d[k] = (double)md;
        }
    }
    return P;
}

/* density function f used by the method (cutoff rule + tabulation applied) */
static void pot_f(const or_pot *P, double r, double *v, double *dv)
{
    if (r >= P->p.rc) { *v = 0.0; *dv = 0.0; return; }
    if (P->p.tabulated) hermite(P->tf_v, P->tf_d, P->nf, P->p.r_min, P->hf, r, v, dv);
    else f_an(P, r, v, dv);
}

static void pot_phi(const or_pot *P, double r, double *v, double *dv)
{
    if (r >= P->p.rc) { *v = 0.0; *dv = 0.0; return; }
    if (P->p.tabulated) hermite(P->tp_v, P->tp_d, P->nf, P->p.r_min, P->hf, r, v, dv);
    else phi_an(&P->p, r, v, dv);
}

static void pot_morse(const or_pot *P, double y, double *v, double *dv)
{
    if (y >= P->p.rc_m) { *v = 0.0; *dv = 0.0; return; }
    if (P->p.tabulated) hermite(P->tm_v, P->tm_d, P->nm, P->p.r_min, P->hm, y, v, dv);
    else morse_an(P, y, v, dv);
}

/* F(rho) of Eq. A3 ("ln(rho/rho_e)^n" read as n ln(rho/rho_e)); derivative by the
 * product rule.  rho <= 0 (an isolated atom) gives F = F' = 0. */
static void embed(const or_params *p, double rho, double *v, double *dv)
{
    if (!(rho > 0.0)) { *v = 0.0; *dv = 0.0; return; }
    double s = rho / p->rho_e;
    double sn = pow(s, p->n);
    double lg = log(s);
    double g = 1.0 - p->n * lg;            /* 1 - n ln s     */
    double dg = -p->n / rho;               /* d/drho of g    */
    double dsn = p->n * sn / rho;          /* d/drho of s^n  */
    *v = -p->F_o * g * sn;
    *dv = -p->F_o * (dg * sn + g * dsn);
}

/* M(P) of Eq. A3 and its derivative by the chain rule */
static void mterm(const or_params *p, double P, double *v, double *dv)
{
    if (!(P > 0.0)) { *v = 0.0; *dv = 0.0; return; }
    double u = P / p->P_e - 1.0;
    double e = exp(-u * u);
    *v = p->alpha * u * u * e;
    *dv = p->alpha * (2.0 * u * e - 2.0 * u * u * u * e) / p->P_e;
}

int or_eval(const or_pot *P, int which, double x, double *v, double *dv)
{
    switch (which) {
    case OR_F: pot_f(P, x, v, dv); return 0;
    case OR_PHI: pot_phi(P, x, v, dv); return 0;
    case OR_MORSE: pot_morse(P, x, v, dv); return 0;
    case OR_EMBED: embed(&P->p, x, v, dv); return 0;
    case OR_MTERM: mterm(&P->p, x, v, dv); return 0;
    case OR_F_RAW: *v = f_raw(&P->p, x); *dv = df_raw(&P->p, x); return 0;
    case OR_PHI_AN: phi_an(&P->p, x, v, dv); return 0;
    case OR_MORSE_RAW: morse_raw(&P->p, x, v, dv); return 0;
    default: return -1;
    }
}

/* --------------------------------------------------------------- summation */

/* self-compensated (Neumaier) summation, Sec. 2.3 */
double or_neumaier(const double *x, int64_t n)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double t = s + x[i];
        if (fabs(s) >= fabs(x[i])) c += (s - t) + x[i];
        else c += (x[i] - t) + s;
        s = t;
    }
    return s + c;
}

/* ----------------------------------------------------------------- geometry */

typedef struct {
    double lo[3], hi[3], L[3];
    int32_t per[3];
} or_box;

static void box_set(or_box *b, const double *lo, const double *hi, const int32_t *per)
{
    for (int k = 0; k < 3; ++k) { b->lo[k] = lo[k]; b->hi[k] = hi[k]; b->L[k] = hi[k] - lo[k]; b->per[k] = per[k]; }
}

/* minimum image along periodic directions (one correction: positions are wrapped at
 * every list build and move less than the skin in between) */
static double min_image(const or_box *b, int k, double dxk)
{
    if (b->per[k]) {
        double half = 0.5 * b->L[k];
        if (dxk > half) dxk -= b->L[k];
        else if (dxk < -half) dxk += b->L[k];
    }
    return dxk;
}

/* displacement xj - xi and its squared length, summed as ((dx^2 + dy^2) + dz^2) */
static double disp2(const or_box *b, const double *xi, const double *xj, double *d)
{
    d[0] = min_image(b, 0, xj[0] - xi[0]);
    d[1] = min_image(b, 1, xj[1] - xi[1]);
    d[2] = min_image(b, 2, xj[2] - xi[2]);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

/* wrap a coordinate into the periodic box: x - floor((x - lo)/L) * L */
static double wrap_coord(const or_box *b, int k, double x)
{
    if (!b->per[k]) return x;
    double m = floor((x - b->lo[k]) / b->L[k]);
    return x - m * b->L[k];
}

/* cell grid for cut-off `cut`: n_k = max(1, floor(L_k / cut)), w_k = L_k / n_k;
 * a periodic direction needs at least 3 cells. */
int or_grid(const double *lo, const double *hi, const int32_t *per, double cut, int32_t *n, double *w)
{
    for (int k = 0; k < 3; ++k) {
        double L = hi[k] - lo[k];
        if (!(L > 0.0)) return -1;
        int nk = (int)floor(L / cut);
        if (nk < 1) nk = 1;
        if (per[k] && nk < 3) return -2;
        n[k] = nk; w[k] = L / nk;
    }
    return 0;
}

/* cell coordinate of a (wrapped) coordinate: floor((x - lo)/w), clamped to [0, n-1] */
static int cell_coord(double x, double lo, double w, int n)
{
    double t = floor((x - lo) / w);
    if (!(t >= 0.0)) return 0;            /* also catches NaN */
    if (t > (double)(n - 1)) return n - 1;
    return (int)t;
}

/* cell coordinates (ix, iy, iz) of every atom after wrapping; returns 0 */
int or_cell_coords(int32_t n_atoms, const double *x, const double *lo, const double *hi,
                   const int32_t *per, double cut, int32_t *cxyz)
{
    or_box b; int32_t ng[3]; double w[3];
    box_set(&b, lo, hi, per);
    if (or_grid(lo, hi, per, cut, ng, w)) return -1;
    for (int32_t i = 0; i < n_atoms; ++i)
        for (int k = 0; k < 3; ++k)
            cxyz[3 * i + k] = cell_coord(wrap_coord(&b, k, x[3 * i + k]), lo[k], w[k], ng[k]);
    return 0;
}

/* -------------------------------------------------------------- neighbours */

typedef struct {
    int32_t n;          /* atoms */
    int64_t *off;       /* n+1 */
    int32_t *idx;       /* off[n] entries, ascending within each atom */
} or_list;

static void list_free(or_list *l) { free(l->off); free(l->idx); l->off = NULL; l->idx = NULL; }

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* All j != i with |x_j - x_i|^2 < cut^2.  method 0 = brute force over all pairs,
 * method 1 = cell list (27-cell stencil on wrapped copies of the positions). */
static int build_list(int32_t n, const double *x, const or_box *b, double cut, int method, or_list *out)
{
    double cut2 = cut * cut;
    int32_t *cnt = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    out->n = n;
    out->off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!cnt || !out->off) { free(cnt); return -1; }
    int32_t ng[3] = {1, 1, 1}; double w[3] = {0, 0, 0};
    int32_t *cstart = NULL, *catoms = NULL, *ckey = NULL;
    double *xw = NULL;
    if (method == 1) {
        if (or_grid(b->lo, b->hi, b->per, cut, ng, w)) { free(cnt); return -2; }
        int64_t nc = (int64_t)ng[0] * ng[1] * ng[2];
        cstart = (int32_t *)calloc((size_t)nc + 1, sizeof(int32_t));
        catoms = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
        ckey = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
        xw = (double *)malloc(sizeof(double) * 3 * ((size_t)n + 1));
        if (!cstart || !catoms || !ckey || !xw) { free(cnt); free(cstart); free(catoms); free(ckey); free(xw); return -1; }
        for (int32_t i = 0; i < n; ++i) {
            int c[3];
            for (int k = 0; k < 3; ++k) {
                xw[3 * i + k] = wrap_coord(b, k, x[3 * i + k]);
                c[k] = cell_coord(xw[3 * i + k], b->lo[k], w[k], ng[k]);
            }
            ckey[i] = (c[2] * ng[1] + c[1]) * ng[0] + c[0];
            cstart[ckey[i] + 1]++;
        }
        for (int64_t c = 0; c < nc; ++c) cstart[c + 1] += cstart[c];
        int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)nc);
        memcpy(fill, cstart, sizeof(int32_t) * (size_t)nc);
        for (int32_t i = 0; i < n; ++i) catoms[fill[ckey[i]]++] = i;   /* ascending id within a cell */
        free(fill);
    }
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            out->off[0] = 0;
            for (int32_t i = 0; i < n; ++i) out->off[i + 1] = out->off[i] + cnt[i];
            out->idx = (int32_t *)malloc(sizeof(int32_t) * ((size_t)out->off[n] + 1));
            if (!out->idx) { free(cnt); free(cstart); free(catoms); free(ckey); free(xw); return -1; }
        }
        #pragma omp parallel for schedule(dynamic, 256)
        for (int32_t i = 0; i < n; ++i) {
            int32_t m = 0;
            int64_t base = pass ? out->off[i] : 0;
            double d[3];
            if (method == 0) {
                for (int32_t j = 0; j < n; ++j) {
                    if (j == i) continue;
                    if (disp2(b, &x[3 * i], &x[3 * j], d) < cut2) {
                        if (pass) out->idx[base + m] = j;
                        ++m;
                    }
                }
            } else {
                int c[3];
                for (int k = 0; k < 3; ++k) c[k] = cell_coord(xw[3 * i + k], b->lo[k], w[k], ng[k]);
                for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int q[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
                    int ok = 1;
                    for (int k = 0; k < 3; ++k) {
                        if (q[k] < 0 || q[k] >= ng[k]) {
                            if (!b->per[k]) { ok = 0; break; }
                            q[k] = (q[k] + ng[k]) % ng[k];
                        }
                    }
                    if (!ok) continue;
                    int32_t key = (q[2] * ng[1] + q[1]) * ng[0] + q[0];
                    for (int32_t s = cstart[key]; s < cstart[key + 1]; ++s) {
                        int32_t j = catoms[s];
                        if (j == i) continue;
                        if (disp2(b, &xw[3 * i], &xw[3 * j], d) < cut2) {
                            if (pass) out->idx[base + m] = j;
                            ++m;
                        }
                    }
                }
                if (pass) qsort(&out->idx[base], (size_t)m, sizeof(int32_t), cmp_i32);
            }
            if (!pass) cnt[i] = m;
        }
    }
    free(cnt); free(cstart); free(catoms); free(ckey); free(xw);
    return 0;
}

/* Cr-C neighbours: every indenter atom c with |x_c - x_i|^2 < cut^2 (minimum image), by
 * brute force over the indenter for the film atoms that lie within `cut` of the indenter's
 * bounding box.  The box test can only skip an atom when |minimum-image offset| > extent/2
 * + cut, which needs L > extent + 2 cut: exactly when no periodic image of the indenter
 * can reach the atom either. */
static int build_clist(int32_t n, const double *x, int32_t nc, const double *xc, const or_box *b,
                       double cut, or_list *out)
{
    double cut2 = cut * cut;
    out->n = n;
    out->off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *cnt = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!out->off || !cnt) { free(cnt); return -1; }
    double bl[3] = {0, 0, 0}, bh[3] = {0, 0, 0}, bc[3], bw[3];
    for (int32_t c = 0; c < nc; ++c)
        for (int k = 0; k < 3; ++k) {
            double v = xc[3 * c + k];
            if (c == 0 || v < bl[k]) bl[k] = v;
            if (c == 0 || v > bh[k]) bh[k] = v;
        }
    for (int k = 0; k < 3; ++k) { bc[k] = 0.5 * (bl[k] + bh[k]); bw[k] = 0.5 * (bh[k] - bl[k]) + cut; }
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            out->off[0] = 0;
            for (int32_t i = 0; i < n; ++i) out->off[i + 1] = out->off[i] + cnt[i];
            out->idx = (int32_t *)malloc(sizeof(int32_t) * ((size_t)out->off[n] + 1));
            if (!out->idx) { free(cnt); return -1; }
        }
        #pragma omp parallel for schedule(dynamic, 256)
        for (int32_t i = 0; i < n; ++i) {
            int32_t m = 0;
            int near = nc > 0;
            for (int k = 0; k < 3 && near; ++k)
                if (fabs(min_image(b, k, x[3 * i + k] - bc[k])) > bw[k]) near = 0;
            if (near) {
                double d[3];
                for (int32_t c = 0; c < nc; ++c) {
                    if (disp2(b, &x[3 * i], &xc[3 * c], d) < cut2) {
                        if (pass) out->idx[out->off[i] + m] = c;
                        ++m;
                    }
                }
            }
            if (!pass) cnt[i] = m;
        }
    }
    free(cnt);
    return 0;
}

/* exported: neighbour sets for the tests; returns the number of entries, or -1 on error /
 * insufficient capacity (then *need holds the required capacity) */
int64_t or_neighbors(int32_t n, const double *x, const double *lo, const double *hi, const int32_t *per,
                     double cut, int32_t method, int64_t *off, int32_t *idx, int64_t cap, int64_t *need)
{
    or_box b; or_list l = {0};
    box_set(&b, lo, hi, per);
    if (build_list(n, x, &b, cut, method, &l)) { list_free(&l); return -1; }
    int64_t tot = l.off[n];
    if (need) *need = tot;
    if (tot > cap) { list_free(&l); return -1; }
    memcpy(off, l.off, sizeof(int64_t) * ((size_t)n + 1));
    memcpy(idx, l.idx, sizeof(int32_t) * (size_t)tot);
    list_free(&l);
    return tot;
}

int64_t or_cneighbors(int32_t n, const double *x, int32_t nc, const double *xc, const double *lo,
                      const double *hi, const int32_t *per, double cut, int64_t *off, int32_t *idx,
                      int64_t cap, int64_t *need)
{
    or_box b; or_list l = {0};
    box_set(&b, lo, hi, per);
    if (build_clist(n, x, nc, xc, &b, cut, &l)) { list_free(&l); return -1; }
    int64_t tot = l.off[n];
    if (need) *need = tot;
    if (tot > cap) { list_free(&l); return -1; }
    memcpy(off, l.off, sizeof(int64_t) * ((size_t)n + 1));
    memcpy(idx, l.idx, sizeof(int32_t) * (size_t)tot);
    list_free(&l);
    return tot;
}

/* ----------------------------------------------------------- energy, forces */

/* Energy components and load of one force evaluation (Eq. A1 + Morse). */
typedef struct { double embed, pair, mterm, morse, load; } or_epot;

/* Per-atom virial (the potential part of the per-atom stress times volume; stresses are
 * among the quantities Task 4 can give, Sec. 2.1, and their histories are derived along
 * the run, Sec. 3.1).  Every pair term of the energy depends on one distance r; with
 * c = (dE/dr) / r the force on i from j is c (x_j - x_i), and each of the two atoms of a
 * pair takes half of c (x_j - x_i) (x) (x_j - x_i); a Cr-C pair gives its half to the Cr
 * atom.  Summed over the atoms this is dE/d(strain) under a homogeneous deformation.
 * Components xx, yy, zz, xy, xz, yz. */
static void add_virial(double *w, double c, const double *d)
{
    w[0] += c * d[0] * d[0]; w[1] += c * d[1] * d[1]; w[2] += c * d[2] * d[2];
    w[3] += c * d[0] * d[1]; w[4] += c * d[0] * d[2]; w[5] += c * d[1] * d[2];
}

/*
 * Task 4 (Sec. 2.1; Sec. 3.3.1.2 and 3.3.1.3): two passes over neighbour lists whose
 * entries are filtered by r < rc (the inner list of Sec. 2.6).
 *   pass 1: rho_i = sum_j f(r_ij), P_i = sum_j f(r_ij)^2 (Eq. A2); F'(rho_i), M'(P_i)
 *   pass 2: F_i = -sum_j [(F'_i + F'_j) f' + (M'_i + M'_j) 2 f f' + Phi'] (x_i - x_j)/r
 *                 -sum_c phi'(y) (x_i - x_c)/y
 * The per-atom energies are stored and summed afterwards with Neumaier summation.
 */
static int eval_forces(const or_pot *P, int32_t n, const double *x, const or_box *b,
                       const or_list *nl, int32_t nc, const double *xc, const or_list *cl,
                       double *F, double *rho_out, double *P_out, double *eatom_out, or_epot *E,
                       double *W, const uint8_t *given, const double *fm_in, double *fm_out)
{
    const or_params *p = &P->p;
    double rc2 = p->rc * p->rc, rcm2 = p->rc_m * p->rc_m;
    double *Fp = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *Mp = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *e_emb = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *e_m = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *e_pair = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *e_mor = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *ld = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    if (!Fp || !Mp || !e_emb || !e_m || !e_pair || !e_mor || !ld) {
        free(Fp); free(Mp); free(e_emb); free(e_m); free(e_pair); free(e_mor); free(ld); return -1;
    }
    #pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double rho = 0.0, Ps = 0.0, d[3];
        for (int64_t s = nl->off[i]; s < nl->off[i + 1]; ++s) {
            int32_t j = nl->idx[s];
            double r2 = disp2(b, &x[3 * i], &x[3 * j], d);
            if (r2 >= rc2) continue;
            double fv, fd;
            pot_f(P, sqrt(r2), &fv, &fd);
            rho += fv;
            Ps += fv * fv;
        }
        double Fv, Fd, Mv, Md;
        embed(p, rho, &Fv, &Fd);
        mterm(p, Ps, &Mv, &Md);
        Fp[i] = Fd; Mp[i] = Md; e_emb[i] = Fv; e_m[i] = Mv;
        if (fm_out) { fm_out[2 * i] = Fd; fm_out[2 * i + 1] = Md; }
        /* F'(rho_i), M'(P_i) that arrived from elsewhere (the exchange between the two
         * passes, Sec. 3.3.2) replace the local ones */
        if (given && given[i]) { Fp[i] = fm_in[2 * i]; Mp[i] = fm_in[2 * i + 1]; }
        if (rho_out) rho_out[i] = rho;
        if (P_out) P_out[i] = Ps;
    }
    #pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0, ep = 0.0, em = 0.0, lz = 0.0, d[3];
        double w[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int64_t s = nl->off[i]; s < nl->off[i + 1]; ++s) {
            int32_t j = nl->idx[s];
            double r2 = disp2(b, &x[3 * i], &x[3 * j], d);   /* d = x_j - x_i */
            if (r2 >= rc2) continue;
            double r = sqrt(r2);
            double fv, fd, pv, pd;
            pot_f(P, r, &fv, &fd);
            pot_phi(P, r, &pv, &pd);
            double coef = (Fp[i] + Fp[j]) * fd + (Mp[i] + Mp[j]) * 2.0 * fv * fd + pd;
            /* F_i = -coef * (x_i - x_j)/r = +coef * d / r */
            fx += coef * d[0] / r; fy += coef * d[1] / r; fz += coef * d[2] / r;
            ep += 0.5 * pv;
            if (W) add_virial(w, 0.5 * coef / r, d);
        }
        if (cl) {
            for (int64_t s = cl->off[i]; s < cl->off[i + 1]; ++s) {
                int32_t c = cl->idx[s];
                double y2 = disp2(b, &x[3 * i], &xc[3 * c], d);   /* d = x_c - x_i */
                if (y2 >= rcm2) continue;
                double y = sqrt(y2);
                double mv, md;
                pot_morse(P, y, &mv, &md);
                double gx = md * d[0] / y, gy = md * d[1] / y, gz = md * d[2] / y;
                fx += gx; fy += gy; fz += gz;
                em += mv;
                lz -= gz;          /* load = -sum_i F^Morse_{i,z} */
                if (W) add_virial(w, 0.5 * md / y, d);
            }
        }
        F[3 * i] = fx; F[3 * i + 1] = fy; F[3 * i + 2] = fz;
        if (W) for (int k = 0; k < 6; ++k) W[6 * i + k] = w[k];
        e_pair[i] = ep; e_mor[i] = em; ld[i] = lz;
    }
    E->embed = or_neumaier(e_emb, n);
    E->pair = or_neumaier(e_pair, n);
    E->mterm = or_neumaier(e_m, n);
    E->morse = or_neumaier(e_mor, n);
    E->load = or_neumaier(ld, n);
    if (eatom_out)
        for (int32_t i = 0; i < n; ++i) eatom_out[i] = e_emb[i] + e_pair[i] + e_m[i] + e_mor[i];
    free(Fp); free(Mp); free(e_emb); free(e_m); free(e_pair); free(e_mor); free(ld);
    return 0;
}

/* exported stateless evaluation at the given positions, with exact neighbour sets at the
 * cutoffs (method 0 brute force, 1 cell list).  epot[5] = {embed, pair, M, morse, load}. */
int or_forces(const or_pot *P, int32_t n, const double *x, const double *lo, const double *hi,
              const int32_t *per, int32_t nc, const double *xc, int32_t method,
              double *F, double *epot, double *rho, double *Pden, double *eatom)
{
    or_box b; or_list nl = {0}, cl = {0};
    box_set(&b, lo, hi, per);
    int err = build_list(n, x, &b, P->p.rc, method, &nl);
    if (!err && nc > 0) err = build_clist(n, x, nc, xc, &b, P->p.rc_m, &cl);
    or_epot E = {0, 0, 0, 0, 0};
    if (!err) err = eval_forces(P, n, x, &b, &nl, nc, xc, nc > 0 ? &cl : NULL, F, rho, Pden, eatom, &E, NULL,
                             NULL, NULL, NULL);
    list_free(&nl); list_free(&cl);
    if (err) return err;
    epot[0] = E.embed; epot[1] = E.pair; epot[2] = E.mterm; epot[3] = E.morse; epot[4] = E.load;
    return 0;
}

/* as or_forces, with the two passes of Task 4 open to an exchange between them (the
 * paper's F', M' Allgatherv, Sec. 3.3.2): fm_out (2n, may be NULL) receives F'(rho_i),
 * M'(P_i) of every atom from pass 1; for atoms with given[i] != 0, pass 2 uses
 * fm_in[2i], fm_in[2i + 1] instead (values computed where those atoms' whole
 * neighbourhoods are known).  eatom: per-atom energies (embedding + M of the atom's own
 * pass-1 values, half its pair terms, its Morse terms). */
int or_forces_given(const or_pot *P, int32_t n, const double *x, const double *lo, const double *hi,
                    const int32_t *per, int32_t nc, const double *xc, const uint8_t *given,
                    const double *fm_in, double *fm_out, double *F, double *epot, double *eatom)
{
    or_box b; or_list nl = {0}, cl = {0};
    box_set(&b, lo, hi, per);
    int err = build_list(n, x, &b, P->p.rc, 1, &nl);
    if (!err && nc > 0) err = build_clist(n, x, nc, xc, &b, P->p.rc_m, &cl);
    or_epot E = {0, 0, 0, 0, 0};
    if (!err) err = eval_forces(P, n, x, &b, &nl, nc, xc, nc > 0 ? &cl : NULL, F, NULL, NULL, eatom, &E, NULL,
                                given, fm_in, fm_out);
    list_free(&nl); list_free(&cl);
    if (err) return err;
    epot[0] = E.embed; epot[1] = E.pair; epot[2] = E.mterm; epot[3] = E.morse; epot[4] = E.load;
    return 0;
}

/* as or_forces, with the per-atom virial W (6 per atom, see add_virial) */
int or_virial(const or_pot *P, int32_t n, const double *x, const double *lo, const double *hi,
              const int32_t *per, int32_t nc, const double *xc, int32_t method, double *F, double *epot,
              double *W)
{
    or_box b; or_list nl = {0}, cl = {0};
    box_set(&b, lo, hi, per);
    int err = build_list(n, x, &b, P->p.rc, method, &nl);
    if (!err && nc > 0) err = build_clist(n, x, nc, xc, &b, P->p.rc_m, &cl);
    or_epot E = {0, 0, 0, 0, 0};
    if (!err) err = eval_forces(P, n, x, &b, &nl, nc, xc, nc > 0 ? &cl : NULL, F, NULL, NULL, NULL, &E, W,
                             NULL, NULL, NULL);
    list_free(&nl); list_free(&cl);
    if (err) return err;
    epot[0] = E.embed; epot[1] = E.pair; epot[2] = E.mterm; epot[3] = E.morse; epot[4] = E.load;
    return 0;
}

/* ------------------------------------------------------------- time loop */

#define OR_ACC 9.6485332e-3       /* 1 eV/(A u) in A/fs^2 */
#define OR_KB 8.617333262e-5      /* eV/K */

typedef struct {
    const or_pot *P;
    int32_t n, nc;
    double *x, *v, *F, *xb, *xc0, *xc;
    uint8_t *fixed;
    double mass, dt, z_ind, v_ind, z_build, skin;
    int32_t rebuild_every, since_build, method;
    int64_t step, rebuilds;
    or_box b;
    or_list nl, cl;
    or_epot E;
    double ke;
} or_sim;

static void sim_place_indenter(or_sim *S)
{
    for (int32_t c = 0; c < S->nc; ++c) {
        S->xc[3 * c] = S->xc0[3 * c];
        S->xc[3 * c + 1] = S->xc0[3 * c + 1];
        S->xc[3 * c + 2] = S->xc0[3 * c + 2] + S->z_ind;
    }
}

/* Task 1: wrap, then rebuild both Verlet lists at cut-off + skin (Sec. 2.6) */
static int sim_rebuild(or_sim *S)
{
    for (int32_t i = 0; i < S->n; ++i)
        for (int k = 0; k < 3; ++k) S->x[3 * i + k] = wrap_coord(&S->b, k, S->x[3 * i + k]);
    list_free(&S->nl); list_free(&S->cl);
    sim_place_indenter(S);
    int err = build_list(S->n, S->x, &S->b, S->P->p.rc + S->skin, S->method, &S->nl);
    if (!err && S->nc > 0) err = build_clist(S->n, S->x, S->nc, S->xc, &S->b, S->P->p.rc_m + S->skin, &S->cl);
    memcpy(S->xb, S->x, sizeof(double) * 3 * (size_t)S->n);
    S->z_build = S->z_ind;
    S->since_build = 0;
    S->rebuilds++;
    return err;
}

static int sim_forces(or_sim *S)
{
    sim_place_indenter(S);
    return eval_forces(S->P, S->n, S->x, &S->b, &S->nl, S->nc, S->xc, S->nc > 0 ? &S->cl : NULL,
                       S->F, NULL, NULL, NULL, &S->E, NULL, NULL, NULL, NULL);
}

static void sim_kinetic(or_sim *S)
{
    double *ke = (double *)malloc(sizeof(double) * ((size_t)S->n + 1));
    for (int32_t i = 0; i < S->n; ++i) {
        const double *v = &S->v[3 * i];
        ke[i] = 0.5 * S->mass * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / OR_ACC;
    }
    S->ke = or_neumaier(ke, S->n);
    free(ke);
}

/* the Task 1 test: rebuild when max_i |x_i - x_build,i| exceeds skin/2 (Sec. 2.6), when
 * that displacement plus the indenter's own travel exceeds the skin (Cr-C pairs), or
 * every `rebuild_every` steps when that is set */
static int sim_need_rebuild(const or_sim *S)
{
    if (S->rebuild_every > 0) return S->since_build >= S->rebuild_every;
    double m2 = 0.0;
    for (int32_t i = 0; i < S->n; ++i) {
        double dx = S->x[3 * i] - S->xb[3 * i];
        double dy = S->x[3 * i + 1] - S->xb[3 * i + 1];
        double dz = S->x[3 * i + 2] - S->xb[3 * i + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 > m2) m2 = d2;
    }
    double dmax = sqrt(m2);
    if (2.0 * dmax > S->skin) return 1;
    if (S->nc > 0 && dmax + fabs(S->z_ind - S->z_build) > S->skin) return 1;
    return 0;
}

void or_sim_free(or_sim *S)
{
    if (!S) return;
    free(S->x); free(S->v); free(S->F); free(S->xb); free(S->xc0); free(S->xc); free(S->fixed);
    list_free(&S->nl); list_free(&S->cl);
    free(S);
}

or_sim *or_sim_new(const or_pot *P, int32_t n, const double *x, const double *v, const uint8_t *fixed,
                   int32_t nc, const double *xc0, const double *lo, const double *hi, const int32_t *per,
                   double z_ind0, double v_ind, double dt, double mass, double skin,
                   int32_t rebuild_every, int32_t method)
{
    or_sim *S = (or_sim *)calloc(1, sizeof(or_sim));
    if (!S) return NULL;
    S->P = P; S->n = n; S->nc = nc;
    size_t b3 = sizeof(double) * 3 * ((size_t)n + 1), c3 = sizeof(double) * 3 * ((size_t)nc + 1);
    S->x = malloc(b3); S->v = malloc(b3); S->F = malloc(b3); S->xb = malloc(b3);
    S->xc0 = malloc(c3); S->xc = malloc(c3); S->fixed = malloc((size_t)n + 1);
    if (!S->x || !S->v || !S->F || !S->xb || !S->xc0 || !S->xc || !S->fixed) { or_sim_free(S); return NULL; }
    memcpy(S->x, x, sizeof(double) * 3 * (size_t)n);
    memcpy(S->v, v, sizeof(double) * 3 * (size_t)n);
    if (nc) memcpy(S->xc0, xc0, sizeof(double) * 3 * (size_t)nc);
    for (int32_t i = 0; i < n; ++i) S->fixed[i] = fixed ? fixed[i] : 0;
    box_set(&S->b, lo, hi, per);
    S->z_ind = z_ind0; S->v_ind = v_ind; S->dt = dt; S->mass = mass; S->skin = skin;
    S->rebuild_every = rebuild_every; S->method = method;
    int32_t ng[3]; double w[3];
    if (or_grid(lo, hi, per, P->p.rc + skin, ng, w)) { or_sim_free(S); return NULL; }
    /* initial list and forces at t = 0 (the accelerations Task 3 needs at the first step) */
    if (sim_rebuild(S) || sim_forces(S)) { or_sim_free(S); return NULL; }
    S->rebuilds = 0;
    sim_kinetic(S);
    return S;
}

/* advance n time steps in the order of Fig. 5 */
int or_sim_step(or_sim *S, int64_t nsteps)
{
    double c = OR_ACC / S->mass;
    for (int64_t s = 0; s < nsteps; ++s) {
        /* Task 1 */
        if (sim_need_rebuild(S) && sim_rebuild(S)) return -1;
        /* Task 2: the rigid indenter moves by v_ind dt */
        S->z_ind += S->v_ind * S->dt;
        /* Task 3: v(t + dt/2) = v + a dt/2 (Eq. A12); x(t + dt) = x + v(t + dt/2) dt (== Eq. A11) */
        #pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < S->n; ++i) {
            if (S->fixed[i]) continue;
            for (int k = 0; k < 3; ++k) {
                S->v[3 * i + k] += 0.5 * S->dt * c * S->F[3 * i + k];
                S->x[3 * i + k] += S->dt * S->v[3 * i + k];
            }
        }
        /* Task 4: a(t + dt) = T / m (Eq. A13) */
        if (sim_forces(S)) return -1;
        /* Task 5: v(t + dt) = v(t + dt/2) + a(t + dt) dt/2 */
        #pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < S->n; ++i) {
            if (S->fixed[i]) continue;
            for (int k = 0; k < 3; ++k) S->v[3 * i + k] += 0.5 * S->dt * c * S->F[3 * i + k];
        }
        sim_kinetic(S);
        S->step++;
        S->since_build++;
    }
    return 0;
}

/* the per-atom virial (see add_virial) of the current state, from the current lists */
int or_sim_virial(or_sim *S, double *W)
{
    sim_place_indenter(S);
    return eval_forces(S->P, S->n, S->x, &S->b, &S->nl, S->nc, S->xc, S->nc > 0 ? &S->cl : NULL,
                       S->F, NULL, NULL, NULL, &S->E, W, NULL, NULL, NULL);
}

/* the indenter's velocity from the next step on (Task 2; the loading and unloading legs
 * of an indentation run, Sec. 2.5) */
void or_sim_set_v_ind(or_sim *S, double v_ind) { S->v_ind = v_ind; }

/* out[8] = {embed, pair, M, morse, kinetic, potential, total, load}; counters[2] = {step, rebuilds} */
void or_sim_get(const or_sim *S, double *x, double *v, double *F, double *out, double *z_ind, int64_t *counters)
{
    if (x) memcpy(x, S->x, sizeof(double) * 3 * (size_t)S->n);
    if (v) memcpy(v, S->v, sizeof(double) * 3 * (size_t)S->n);
    if (F) memcpy(F, S->F, sizeof(double) * 3 * (size_t)S->n);
    if (out) {
        double pe = S->E.embed + S->E.pair + S->E.mterm + S->E.morse;
        out[0] = S->E.embed; out[1] = S->E.pair; out[2] = S->E.mterm; out[3] = S->E.morse;
        out[4] = S->ke; out[5] = pe; out[6] = pe + S->ke; out[7] = S->E.load;
    }
    if (z_ind) *z_ind = S->z_ind;
    if (counters) { counters[0] = S->step; counters[1] = S->rebuilds; }
}

/* list of the current Verlet list (cut-off + skin) for the parity tests */
int64_t or_sim_list(const or_sim *S, int32_t which, int64_t *off, int32_t *idx, int64_t cap)
{
    const or_list *l = which ? &S->cl : &S->nl;
    if (which && S->nc == 0) { for (int32_t i = 0; i <= S->n; ++i) off[i] = 0; return 0; }
    int64_t tot = l->off[S->n];
    if (tot > cap) return -1;
    memcpy(off, l->off, sizeof(int64_t) * ((size_t)S->n + 1));
    memcpy(idx, l->idx, sizeof(int32_t) * (size_t)tot);
    return tot;
}

int or_set_threads(int32_t t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}
