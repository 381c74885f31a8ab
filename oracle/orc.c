/*
 * orc.c -- plain FP64 CPU oracle of the ternary free-energy entropic lattice
 * Boltzmann update of arXiv:1710.07486.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  Every step is written out in the order of the
 * algorithm, without blocking or fusion.  The plain build is single-threaded;
 * the OpenMP pragmas on the loops over nodes (independent per node, no
 * reductions) only take effect in the separately built timing copy
 * (-fopenmp) that the CPU baseline uses on all host cores.
 *
 * The paper states the continuum model (Eqs. 1-8) and names the discrete
 * schemes (entropic LBM with exact-difference forcing for the density
 * populations f, BGK for the phase-field populations g) but defers the
 * discrete formulas to its supplement, which is not available.  Where that
 * is the case the reading used is stated at the function ("reading: ...").
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_ctx {
    int D, Q, nx, ny, nz;
    long N;
    int bc[3];
    orc_params p;
    double rho_g, rho_l, mu_coex, p_coex;
    double tau, beta;
    int c[27][3];
    double w[27];
    int opp[27];
    int rest;
    long *gamma_fallbacks;  /* counter of exact-stabiliser fallbacks */
    unsigned char *solid;   /* copy of the solid mask, or NULL */
};

/* ------------------------------------------------------------------------- */
/* Thermodynamics: Carnahan-Starling free energy, Eq. 4 (without C).         */
/* ------------------------------------------------------------------------- */

/* Psi~(rho) = rho ( -a rho - 8RT(b rho - 6)/(b rho - 4)^2 + RT ln rho ), Eq. 4
   with C = 0. */
static double cs_psi(double a, double b, double R, double T, double rho)
{
    double br = b * rho;
    return rho * (-a * rho - 8.0 * R * T * (br - 6.0) / ((br - 4.0) * (br - 4.0))
                  + R * T * log(rho));
}

/* d Psi~ / d rho, differentiated by hand from Eq. 4:
   -2 a rho - 8RT (24 - 2 b rho)/(b rho - 4)^3 + RT (ln rho + 1). */
static double cs_dpsi(double a, double b, double R, double T, double rho)
{
    double br = b * rho;
    double d = br - 4.0;
    return -2.0 * a * rho - 8.0 * R * T * (24.0 - 2.0 * br) / (d * d * d)
           + R * T * (log(rho) + 1.0);
}

/* The other two equations of state the text names as alternatives (their
   formulas are in the unavailable supplement; these are the textbook forms,
   with Psi~ obtained, like Eq. 4, by integrating p_eos = rho Psi' - Psi, i.e.
   Psi~/rho = int p_eos / rho^2 drho, integration constant zero):
     van der Waals:  p = rho R T/(1 - b rho) - a rho^2
                     Psi~ = rho R T ln(rho/(1 - b rho)) - a rho^2
     Peng-Robinson:  p = rho R T/(1 - b rho) - a alpha rho^2/(1 + 2 b rho - b^2 rho^2)
                     Psi~ = rho R T ln(rho/(1 - b rho))
                            - a alpha/(2 sqrt2 b) rho ln((1 + (1+sqrt2) b rho)/(1 + (1-sqrt2) b rho))
     alpha(T) = (1 + k (1 - sqrt(T/T_c)))^2, k = 0.37464 + 1.54226 w - 0.26992 w^2,
     T_c = 0.07780 a/(0.45724 b R) (acentric factor w). */
double orc_pr_tc(double a, double b, double R) { return 0.07780 * a / (0.45724 * b * R); }

static double pr_alpha(const orc_eos *e)
{
    double k = 0.37464 + 1.54226 * e->omega - 0.26992 * e->omega * e->omega;
    double q = 1.0 + k * (1.0 - sqrt(e->T / orc_pr_tc(e->a, e->b, e->R)));
    return q * q;
}

double orc_eos_psi(const orc_eos *e, double rho)
{
    double a = e->a, b = e->b, RT = e->R * e->T;
    switch (e->kind) {
    case ORC_EOS_VDW:
        return rho * RT * log(rho / (1.0 - b * rho)) - a * rho * rho;
    case ORC_EOS_PR: {
        double s2 = sqrt(2.0), aa = a * pr_alpha(e);
        return rho * RT * log(rho / (1.0 - b * rho))
               - aa / (2.0 * s2 * b) * rho * log((1.0 + (1.0 + s2) * b * rho) / (1.0 + (1.0 - s2) * b * rho));
    }
    default:
        return cs_psi(a, b, e->R, e->T, rho);
    }
}

/* d Psi~/d rho, by hand from the forms above:
     vdW: RT ln(rho/(1 - b rho)) + RT/(1 - b rho) - 2 a rho
     PR:  RT ln(rho/(1 - b rho)) + RT/(1 - b rho)
          - a alpha/(2 sqrt2 b) ln((1 + (1+sqrt2) b rho)/(1 + (1-sqrt2) b rho))
          - a alpha rho/(1 + 2 b rho - b^2 rho^2) */
double orc_eos_dpsi(const orc_eos *e, double rho)
{
    double a = e->a, b = e->b, RT = e->R * e->T;
    switch (e->kind) {
    case ORC_EOS_VDW:
        return RT * log(rho / (1.0 - b * rho)) + RT / (1.0 - b * rho) - 2.0 * a * rho;
    case ORC_EOS_PR: {
        double s2 = sqrt(2.0), aa = a * pr_alpha(e);
        return RT * log(rho / (1.0 - b * rho)) + RT / (1.0 - b * rho)
               - aa / (2.0 * s2 * b) * log((1.0 + (1.0 + s2) * b * rho) / (1.0 + (1.0 - s2) * b * rho))
               - aa * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
    }
    default:
        return cs_dpsi(a, b, e->R, e->T, rho);
    }
}

/* p_eos = rho dPsi/drho - Psi (text before Eq. 4); C cancels. */
double orc_eos_p(const orc_eos *e, double rho)
{
    return rho * orc_eos_dpsi(e, rho) - orc_eos_psi(e, rho);
}

/* upper end of the density range: the packing limit 4/b (CS) or 1/b */
static double rho_limit(const orc_eos *e) { return (e->kind == ORC_EOS_CS ? 4.0 : 1.0) / e->b; }

double orc_psi_tilde(double a, double b, double R, double T, double rho)
{
    orc_eos e = {ORC_EOS_CS, a, b, R, T, 0.0};
    return orc_eos_psi(&e, rho);
}
double orc_dpsi_tilde(double a, double b, double R, double T, double rho)
{
    orc_eos e = {ORC_EOS_CS, a, b, R, T, 0.0};
    return orc_eos_dpsi(&e, rho);
}
double orc_p_eos(double a, double b, double R, double T, double rho)
{
    orc_eos e = {ORC_EOS_CS, a, b, R, T, 0.0};
    return orc_eos_p(&e, rho);
}

/* Locate the van der Waals loop of p_eos: the local maximum rho_s1 and the
   following local minimum rho_s2.  Returns 0 if found, -1 otherwise. */
static int spinodals(const orc_eos *e, double *s1, double *s2)
{
    const int M = 20000;
    double lo = log(1e-7), hi = log(0.98 * rho_limit(e));
    double prev_p = orc_eos_p(e, exp(lo));
    int state = 0; /* 0 rising, 1 falling */
    int i_max = -1, i_min = -1;
    for (int i = 1; i <= M; i++) {
        double x = lo + (hi - lo) * i / M;
        double pv = orc_eos_p(e, exp(x));
        if (state == 0 && pv < prev_p) { state = 1; i_max = i - 1; }
        else if (state == 1 && pv > prev_p) { i_min = i - 1; break; }
        prev_p = pv;
    }
    if (i_max < 0 || i_min < 0) return -1;
    /* golden-section refinement of the extremum in [i-1, i+1] grid cells */
    for (int which = 0; which < 2; which++) {
        int ic = which == 0 ? i_max : i_min;
        double xa = lo + (hi - lo) * (ic - 1) / M, xb = lo + (hi - lo) * (ic + 1) / M;
        double g = 0.5 * (sqrt(5.0) - 1.0);
        for (int it = 0; it < 200; it++) {
            double x1 = xb - g * (xb - xa), x2 = xa + g * (xb - xa);
            double p1 = orc_eos_p(e, exp(x1)), p2 = orc_eos_p(e, exp(x2));
            int keep_left = which == 0 ? (p1 > p2) : (p1 < p2);
            if (keep_left) xb = x2; else xa = x1;
        }
        if (which == 0) *s1 = exp(0.5 * (xa + xb)); else *s2 = exp(0.5 * (xa + xb));
    }
    return 0;
}

/* root of p_eos(rho) = target on [lo, hi] where p_eos is increasing */
static double p_root(const orc_eos *e, double target, double lo, double hi)
{
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_eos_p(e, mid) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Common-tangent (Maxwell) construction: the coexisting densities have equal
   pressure and equal dPsi/drho.  Choosing C = -mu_coex and
   Psi_0 = Psi_eos(rho_g) = Psi_eos(rho_l) = -p_coex meets the condition stated
   after Eq. 4.  Solved by bisection on the saturation pressure. */
int orc_eos_coexistence(const orc_eos *e, double out[4])
{
    double s1, s2;
    if (!(e->a > 0 && e->b > 0 && e->R > 0 && e->T > 0)) return -1;
    if (e->kind < 0 || e->kind > 2) return -1;
    if (spinodals(e, &s1, &s2)) return -1;
    double rmax = 0.98 * rho_limit(e);
    double p_hi = orc_eos_p(e, s1);
    double p_lo = orc_eos_p(e, s2);
    if (p_lo < 0.0) p_lo = 0.0;
    if (orc_eos_p(e, rmax) <= p_hi) return -1;
    double rg = 0, rl = 0;
    for (int it = 0; it < 400; it++) {
        double ps = 0.5 * (p_lo + p_hi);
        if (ps <= p_lo || ps >= p_hi) break;
        rg = p_root(e, ps, 1e-300, s1);
        rl = p_root(e, ps, s2, rmax);
        double dmu = orc_eos_dpsi(e, rl) - orc_eos_dpsi(e, rg);
        /* dmu > 0: the saturation pressure is too low */
        if (dmu > 0.0) p_lo = ps; else p_hi = ps;
    }
    double ps = 0.5 * (p_lo + p_hi);
    rg = p_root(e, ps, 1e-300, s1);
    rl = p_root(e, ps, s2, rmax);
    out[0] = rg;
    out[1] = rl;
    out[2] = 0.5 * (orc_eos_dpsi(e, rg) + orc_eos_dpsi(e, rl));
    out[3] = 0.5 * (orc_eos_p(e, rg) + orc_eos_p(e, rl));
    return 0;
}

int orc_coexistence(double a, double b, double R, double T, double out[4])
{
    orc_eos e = {ORC_EOS_CS, a, b, R, T, 0.0};
    return orc_eos_coexistence(&e, out);
}

/* Critical point of the CS isotherms.  Along the spinodal dp/drho = 0; with
   dp/drho = rho d2Psi~/drho2 and d2Psi~/drho2 = -2a - 32RTb(b rho - 16)/(b rho
   - 4)^4 + RT/rho this gives T_s(rho) = 2 a rho / (R (1 - 32 b rho (b rho - 16)
   / (b rho - 4)^4)).  T_c is the maximum of T_s, rho_c its argument. */
static double t_spinodal(double a, double b, double R, double rho)
{
    double br = b * rho, d = br - 4.0;
    return 2.0 * a * rho / (R * (1.0 - 32.0 * br * (br - 16.0) / (d * d * d * d)));
}

int orc_critical_point(double a, double b, double R, double out[2])
{
    if (!(a > 0 && b > 0 && R > 0)) return -1;
    double xa = 0.05 / b, xb = 3.5 / b, g = 0.5 * (sqrt(5.0) - 1.0);
    for (int it = 0; it < 300; it++) {
        double x1 = xb - g * (xb - xa), x2 = xa + g * (xb - xa);
        if (t_spinodal(a, b, R, x1) > t_spinodal(a, b, R, x2)) xb = x2; else xa = x1;
    }
    out[1] = 0.5 * (xa + xb);
    out[0] = t_spinodal(a, b, R, out[1]);
    return 0;
}

/* The coexistence ratio rho_l/rho_g falls monotonically with T: bisection. */
int orc_temperature_for_ratio(double a, double b, double R, double ratio, double *T)
{
    double cp[2], co[4];
    if (!(ratio > 1.0) || orc_critical_point(a, b, R, cp)) return -1;
    double lo = 0.3 * cp[0], hi = 0.999 * cp[0];
    if (orc_coexistence(a, b, R, lo, co)) return -1;
    if (co[1] / co[0] < ratio) return -1;
    if (orc_coexistence(a, b, R, hi, co)) return -1;
    if (co[1] / co[0] > ratio) return -1;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_coexistence(a, b, R, mid, co)) return -1;
        if (co[1] / co[0] > ratio) lo = mid; else hi = mid;
    }
    *T = 0.5 * (lo + hi);
    return 0;
}

/* Critical point of any of the three equations of state, found without its
   closed form: T_c is the lowest temperature at which p_eos(rho) no longer
   has a van der Waals loop (bisection on T), rho_c the density of the
   loop's vanishing extrema.  (CS: the maximum of the spinodal curve above.) */
int orc_eos_critical_point(int kind, double a, double b, double R, double omega, double out[2])
{
    if (kind == ORC_EOS_CS) return orc_critical_point(a, b, R, out);
    if (!(a > 0 && b > 0 && R > 0) || kind < 0 || kind > 2) return -1;
    double hi = 2.0 * a / (b * R), lo = hi, s1, s2;
    orc_eos e = {kind, a, b, R, hi, omega};
    if (!spinodals(&e, &s1, &s2)) return -1;
    /* step down until a loop appears: the bracket [lo, hi] of T_c */
    int found = 0;
    for (int it = 0; it < 60 && !found; it++) {
        hi = lo;
        lo *= 0.8;
        e.T = lo;
        found = !spinodals(&e, &s1, &s2);
    }
    if (!found) return -1;
    for (int it = 0; it < 80; it++) {
        e.T = 0.5 * (lo + hi);
        if (spinodals(&e, &s1, &s2)) hi = e.T; else lo = e.T;
    }
    e.T = lo;
    if (spinodals(&e, &s1, &s2)) return -1;
    out[0] = 0.5 * (lo + hi);
    out[1] = 0.5 * (s1 + s2);
    return 0;
}

int orc_eos_temperature_for_ratio(int kind, double a, double b, double R, double omega, double ratio, double *T)
{
    if (kind == ORC_EOS_CS) return orc_temperature_for_ratio(a, b, R, ratio, T);
    double cp[2], co[4];
    if (!(ratio > 1.0) || orc_eos_critical_point(kind, a, b, R, omega, cp)) return -1;
    orc_eos e = {kind, a, b, R, 0.3 * cp[0], omega};
    double lo = 0.3 * cp[0], hi = 0.995 * cp[0];
    if (orc_eos_coexistence(&e, co) || co[1] / co[0] < ratio) return -1;
    e.T = hi;
    if (orc_eos_coexistence(&e, co) || co[1] / co[0] > ratio) return -1;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        e.T = mid;
        if (orc_eos_coexistence(&e, co)) return -1;
        if (co[1] / co[0] > ratio) lo = mid; else hi = mid;
    }
    *T = 0.5 * (lo + hi);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Lattice: D2Q9 and D3Q27, c_s^2 = 1/3.                                      */
/* ------------------------------------------------------------------------- */

/* D2Q9, listed with the x component running fastest. */
static const int C_D2Q9[9][2] = {
    {-1, -1}, {0, -1}, {1, -1},
    {-1, 0},  {0, 0},  {1, 0},
    {-1, 1},  {0, 1},  {1, 1}};
static const double W_D2Q9[9] = {
    1.0 / 36, 1.0 / 9, 1.0 / 36,
    1.0 / 9,  4.0 / 9, 1.0 / 9,
    1.0 / 36, 1.0 / 9, 1.0 / 36};

/* D3Q27 weights by the number of non-zero components: rest 8/27, the six face
   neighbours 2/27, the twelve edge neighbours 1/54, the eight corners 1/216. */
static double w_d3q27(int cx, int cy, int cz)
{
    int k = (cx != 0) + (cy != 0) + (cz != 0);
    if (k == 0) return 8.0 / 27;
    if (k == 1) return 2.0 / 27;
    if (k == 2) return 1.0 / 54;
    return 1.0 / 216;
}

orc_ctx *orc_create(int lattice, int nx, int ny, int nz, const orc_params *p,
                    const int bc[3])
{
    if (lattice != 0 && lattice != 1) return NULL;
    if (nx < 1 || ny < 1 || nz < 1) return NULL;
    if (lattice == 0 && nz != 1) return NULL;
    orc_ctx *o = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (!o) return NULL;
    o->gamma_fallbacks = (long *)calloc(1, sizeof(long));
    if (!o->gamma_fallbacks) { free(o); return NULL; }
    o->D = lattice == 0 ? 2 : 3;
    o->Q = lattice == 0 ? 9 : 27;
    o->nx = nx; o->ny = ny; o->nz = nz;
    o->N = (long)nx * ny * nz;
    for (int a = 0; a < 3; a++) o->bc[a] = bc ? bc[a] : 0;
    if (lattice == 0) o->bc[2] = 0;
    o->p = *p;
    o->p.solid = NULL;
    if (p->solid) {
        o->solid = (unsigned char *)malloc((size_t)o->N);
        if (!o->solid) { free(o->gamma_fallbacks); free(o); return NULL; }
        for (long n = 0; n < o->N; n++) o->solid[n] = p->solid[n] != 0;
    }
    if (lattice == 0) {
        for (int i = 0; i < 9; i++) {
            o->c[i][0] = C_D2Q9[i][0];
            o->c[i][1] = C_D2Q9[i][1];
            o->c[i][2] = 0;
            o->w[i] = W_D2Q9[i];
        }
    } else {
        int i = 0;
        for (int cz = -1; cz <= 1; cz++)
            for (int cy = -1; cy <= 1; cy++)
                for (int cx = -1; cx <= 1; cx++) {
                    o->c[i][0] = cx; o->c[i][1] = cy; o->c[i][2] = cz;
                    o->w[i] = w_d3q27(cx, cy, cz);
                    i++;
                }
    }
    for (int i = 0; i < o->Q; i++) {
        if (o->c[i][0] == 0 && o->c[i][1] == 0 && o->c[i][2] == 0) o->rest = i;
        for (int j = 0; j < o->Q; j++)
            if (o->c[j][0] == -o->c[i][0] && o->c[j][1] == -o->c[i][1] &&
                o->c[j][2] == -o->c[i][2])
                o->opp[i] = j;
    }
    double co[4];
    orc_eos e = {p->eos, p->a, p->b, p->R, p->T, p->omega};
    if (orc_eos_coexistence(&e, co)) { free(o->solid); free(o->gamma_fallbacks); free(o); return NULL; }
    o->rho_g = co[0]; o->rho_l = co[1]; o->mu_coex = co[2]; o->p_coex = co[3];
    /* nu = c_s^2 (tau - 1/2) with c_s^2 = 1/3; KBC uses beta = 1/(2 tau) */
    o->tau = 3.0 * p->nu + 0.5;
    o->beta = 1.0 / (2.0 * o->tau);
    return o;
}

void orc_destroy(orc_ctx *o)
{
    if (o) {
        free(o->gamma_fallbacks);
        free(o->solid);
    }
    free(o);
}

static int is_solid(const orc_ctx *o, long n) { return o->solid && o->solid[n]; }
long orc_gamma_fallbacks(const orc_ctx *o) { return *o->gamma_fallbacks; }
int orc_Q(const orc_ctx *o) { return o->Q; }
long orc_N(const orc_ctx *o) { return o->N; }

void orc_velocities(const orc_ctx *o, int *c, double *w)
{
    for (int i = 0; i < o->Q; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = o->c[i][a];
        w[i] = o->w[i];
    }
}

void orc_derived(const orc_ctx *o, double out[6])
{
    out[0] = o->rho_g; out[1] = o->rho_l; out[2] = o->mu_coex; out[3] = o->p_coex;
    out[4] = o->tau; out[5] = o->beta;
}

/* ------------------------------------------------------------------------- */
/* Free energy and chemical potentials (Eqs. 1-5 and the definitions of      */
/* mu_rho, mu_phi after Eq. 8).                                              */
/* ------------------------------------------------------------------------- */

/* Psi_eos - Psi_0 with C = -mu_coex and Psi_0 = -p_coex (text after Eq. 4) */
static double psi_shifted(const orc_ctx *o, double rho)
{
    const orc_params *p = &o->p;
    orc_eos e = {p->eos, p->a, p->b, p->R, p->T, p->omega};
    return orc_eos_psi(&e, rho) - o->mu_coex * rho + o->p_coex;
}

/* C_l1 and C_l2 from (rho, phi), text before Eq. 5 */
static double conc_l1(const orc_ctx *o, double rho, double phi)
{
    return 0.5 * (1.0 + phi / o->p.chi - (rho - o->rho_l) / (o->rho_g - o->rho_l));
}
static double conc_l2(const orc_ctx *o, double rho, double phi)
{
    return 0.5 * (1.0 - phi / o->p.chi - (rho - o->rho_l) / (o->rho_g - o->rho_l));
}

/* Eq. 2 */
double orc_f_bulk(const orc_ctx *o, double rho, double phi)
{
    double c1 = conc_l1(o, rho, phi), c2 = conc_l2(o, rho, phi);
    return 0.5 * o->p.lambda1 * psi_shifted(o, rho)
           + 0.5 * o->p.lambda2 * c1 * c1 * (1.0 - c1) * (1.0 - c1)
           + 0.5 * o->p.lambda3 * c2 * c2 * (1.0 - c2) * (1.0 - c2);
}

/* Neighbour of node (x,y,z) along c under the axis rules only: periodic
   axes wrap; on a bounce-back axis the ghost node beyond the half-way wall
   mirrors the first fluid node, so -1 -> 0 and n -> n-1 (reading: zero
   normal gradient, neutral wetting).  sgn[a] is -1 for each axis on which the
   neighbour was mirrored (the component of a vector normal to the mirror
   changes sign). */
static long axis_nb(const orc_ctx *o, int x, int y, int z, const int *c, int sgn[3])
{
    int q[3] = {x + c[0], y + c[1], z + c[2]};
    int n[3] = {o->nx, o->ny, o->nz};
    for (int a = 0; a < 3; a++) {
        sgn[a] = 1;
        if (q[a] < 0) {
            if (o->bc[a] == 0) q[a] += n[a]; else { q[a] = 0; sgn[a] = -1; }
        } else if (q[a] >= n[a]) {
            if (o->bc[a] == 0) q[a] -= n[a]; else { q[a] = n[a] - 1; sgn[a] = -1; }
        }
    }
    return (long)q[0] + (long)o->nx * ((long)q[1] + (long)o->ny * q[2]);
}

/* Neighbour for the stencils, with solid nodes (reading, the same neutral
   wetting as at the axis walls): when the neighbour along c is solid, the
   stencil reads a ghost that mirrors a fluid node across the solid surface:
   the components of c are set to zero, fewest first and in axis order
   ({x}, {y}, {z}, {x,y}, {x,z}, {y,z}, {x,y,z}), until the node reached is
   fluid; the vector components along the zeroed axes change sign.  Zeroing
   every component reaches the node itself.  Where solid layers fill the ends
   of an axis this is exactly the axis wall rule above. */
static long stencil_nb_vec(const orc_ctx *o, int x, int y, int z, const int *c, int sgn[3])
{
    static const int subsets[7] = {1, 2, 4, 3, 5, 6, 7};
    long m = axis_nb(o, x, y, z, c, sgn);
    if (!is_solid(o, m)) return m;
    for (int k = 0; k < 7; k++) {
        int S = subsets[k], cc[3], sg[3], skip = 0;
        for (int a = 0; a < 3; a++) {
            if ((S >> a) & 1) {
                if (c[a] == 0) skip = 1;
                cc[a] = 0;
            } else {
                cc[a] = c[a];
            }
        }
        if (skip) continue;
        long q = axis_nb(o, x, y, z, cc, sg);
        if (!is_solid(o, q)) {
            for (int a = 0; a < 3; a++) sgn[a] = ((S >> a) & 1) ? -sg[a] : sg[a];
            return q;
        }
    }
    return m;  /* a solid node with no fluid neighbour: its values are unused */
}

/* Value of a scalar field seen by a stencil at (x,y,z) along c.  Reading
   (wetting; not in the paper, which only says that wetting boundary
   conditions fit the model): the ghost across a wall or a solid surface is
   the mirrored fluid value plus wet for each axis the read was mirrored on,
   i.e. the field is continued linearly with a prescribed change wet per
   lattice spacing into the wall -- a gradient (Cahn-type) wetting condition.
   wet = 0 is the neutral mirror.  It enters where the free energy is
   differentiated: the Laplacians of density and composition in the chemical
   potentials.  The gradients keep the plain mirror: the chemical potentials'
   (no diffusive flux into the wall), and the density gradient of the force's
   ideal-pressure term, which stands for the pressure the populations carry,
   and at a bounce-back wall that pressure has no ghost. */
static double stencil_val(const orc_ctx *o, const double *psi, double wet, int x, int y, int z, const int *c)
{
    int sg[3];
    long m = stencil_nb_vec(o, x, y, z, c, sg);
    if (wet == 0.0) return psi[m];
    int k = (sg[0] < 0) + (sg[1] < 0) + (sg[2] < 0);
    return psi[m] + wet * k;
}

/* Reading (stencils; not in the paper): the lattice-weight isotropic
   Laplacian  lap psi = (2/c_s^2) sum_i w_i (psi(x+c_i) - psi(x)). */
void orc_laplacian_wet(const orc_ctx *o, const double *psi, double wet, double *lap)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                long n = x + (long)o->nx * (y + (long)o->ny * z);
                double s = 0.0;
                for (int i = 0; i < o->Q; i++)
                    s += o->w[i] * (stencil_val(o, psi, wet, x, y, z, o->c[i]) - psi[n]);
                lap[n] = 6.0 * s;
            }
}

void orc_laplacian(const orc_ctx *o, const double *psi, double *lap)
{
    orc_laplacian_wet(o, psi, 0.0, lap);
}

/* Reading (stencils): the isotropic gradient
   grad psi = (1/c_s^2) sum_i w_i c_i psi(x+c_i).  grad is [3][N]. */
static void gradient_wet(const orc_ctx *o, const double *psi, double wet, double *grad)
{
    long N = o->N;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                long n = x + (long)o->nx * (y + (long)o->ny * z);
                double s[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < o->Q; i++) {
                    double v = stencil_val(o, psi, wet, x, y, z, o->c[i]);
                    for (int a = 0; a < 3; a++) s[a] += o->w[i] * o->c[i][a] * v;
                }
                for (int a = 0; a < 3; a++) grad[a * N + n] = 3.0 * s[a];
            }
}

void orc_gradient(const orc_ctx *o, const double *psi, double *grad)
{
    gradient_wet(o, psi, 0.0, grad);
}

/* mu_rho = dF/drho and mu_phi = dF/dphi of Eq. 1 written with Eq. 5:
     mu_rho = (lambda1/2) dPsi_eos/drho
              - [lambda2 w'(C1) + lambda3 w'(C2)] / (2 Delta)
              - [kappa1 + (kappa2+kappa3)/(4 Delta^2)] lap rho
              - (kappa3-kappa2)/(4 chi Delta) lap phi
     mu_phi = [lambda2 w'(C1) - lambda3 w'(C2)] / (2 chi)
              - (kappa2+kappa3)/(4 chi^2) lap phi
              - (kappa3-kappa2)/(4 chi Delta) lap rho
   with Delta = rho_g - rho_l and w'(C) = C (1-C) (1-2C). */
void orc_chem_pot(const orc_ctx *o, const double *rho, const double *phi,
                  double *mu_rho, double *mu_phi)
{
    const orc_params *p = &o->p;
    long N = o->N;
    double *lr = (double *)malloc(sizeof(double) * N);
    double *lp = (double *)malloc(sizeof(double) * N);
    orc_laplacian_wet(o, rho, o->p.wet_rho, lr);
    orc_laplacian_wet(o, phi, o->p.wet_phi, lp);
    double Dl = o->rho_g - o->rho_l, chi = p->chi;
    orc_eos e = {p->eos, p->a, p->b, p->R, p->T, p->omega};
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        double c1 = conc_l1(o, rho[n], phi[n]), c2 = conc_l2(o, rho[n], phi[n]);
        double w1 = c1 * (1.0 - c1) * (1.0 - 2.0 * c1);
        double w2 = c2 * (1.0 - c2) * (1.0 - 2.0 * c2);
        double dpsi = orc_eos_dpsi(&e, rho[n]) - o->mu_coex;
        mu_rho[n] = 0.5 * p->lambda1 * dpsi
                    - (p->lambda2 * w1 + p->lambda3 * w2) / (2.0 * Dl)
                    - (p->kappa1 + (p->kappa2 + p->kappa3) / (4.0 * Dl * Dl)) * lr[n]
                    - (p->kappa3 - p->kappa2) / (4.0 * chi * Dl) * lp[n];
        mu_phi[n] = (p->lambda2 * w1 - p->lambda3 * w2) / (2.0 * chi)
                    - (p->kappa2 + p->kappa3) / (4.0 * chi * chi) * lp[n]
                    - (p->kappa3 - p->kappa2) / (4.0 * chi * Dl) * lr[n];
    }
    free(lr);
    free(lp);
}

/* Force on the density populations.  The paper gives div P = rho grad mu_rho
   + phi grad mu_phi (after Eq. 8) and applies the force of the entropic LBM
   with exact-difference forcing; the equilibrium of f already carries the
   ideal pressure rho c_s^2, so (reading) F = -rho grad mu_rho - phi grad
   mu_phi + F_id with F_id the ideal-pressure term.

   force_form 0 (potential form): F_id = c_s^2 grad rho.

   force_form 1 (lattice-consistent form; reading): at a steady state of the
   lattice update the streamed populations average the applied force over the
   neighbours and carry the exact-difference momentum flux F F/(4 rho), so the
   update balances (I + A)/2 F - div(F F/(4 rho)) = c_s^2 grad rho with
   A[G]_a(x) = sum_i 3 w_i c_ia (c_i . G(x - c_i)).  Taking, with G = grad rho,
     F_id = c_s^2 (3/2 G - 1/2 A[G]) + div(c_s^4 G G / (4 rho))
   makes that balance hold, to the next order, exactly when rho grad mu_rho
   + phi grad mu_phi = 0, i.e. at the thermodynamic equilibrium of Eq. 1. */
void orc_force(const orc_ctx *o, const double *rho, const double *phi,
               const double *mu_rho, const double *mu_phi, double *F)
{
    long N = o->N;
    const double cs2 = 1.0 / 3.0;
    double *gm = (double *)malloc(sizeof(double) * 3 * N);
    double *gp = (double *)malloc(sizeof(double) * 3 * N);
    double *gr = (double *)malloc(sizeof(double) * 3 * N);
    orc_gradient(o, mu_rho, gm);
    orc_gradient(o, mu_phi, gp);
    orc_gradient(o, rho, gr);
    for (int a = 0; a < 3; a++)
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; n++)
            F[a * N + n] = -rho[n] * gm[a * N + n] - phi[n] * gp[a * N + n];
    if (o->p.force_form == 0) {
        for (long n = 0; n < 3 * N; n++) F[n] += cs2 * gr[n];
    } else {
#pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < o->nz; z++)
            for (int y = 0; y < o->ny; y++)
                for (int x = 0; x < o->nx; x++) {
                    long n = x + (long)o->nx * (y + (long)o->ny * z);
                    double AG[3] = {0, 0, 0}, divT[3] = {0, 0, 0};
                    for (int i = 0; i < o->Q; i++) {
                        int sg[3], mc[3] = {-o->c[i][0], -o->c[i][1], -o->c[i][2]};
                        /* A[G] reads G at x - c_i */
                        long m = stencil_nb_vec(o, x, y, z, mc, sg);
                        double cG = 0.0;
                        for (int b = 0; b < 3; b++) cG += o->c[i][b] * sg[b] * gr[b * N + m];
                        for (int a = 0; a < 3; a++) AG[a] += 3.0 * o->w[i] * o->c[i][a] * cG;
                        /* div T reads T = c_s^4 G G/(4 rho) at x + c_i */
                        long p = stencil_nb_vec(o, x, y, z, o->c[i], sg);
                        for (int a = 0; a < 3; a++)
                            for (int b = 0; b < 3; b++) {
                                double T = cs2 * cs2 * (sg[a] * gr[a * N + p]) * (sg[b] * gr[b * N + p])
                                           / (4.0 * rho[p]);
                                divT[a] += 3.0 * o->w[i] * o->c[i][b] * T;
                            }
                    }
                    for (int a = 0; a < 3; a++)
                        F[a * N + n] += cs2 * (1.5 * gr[a * N + n] - 0.5 * AG[a]) + divT[a];
                }
    }
    free(gm);
    free(gp);
    free(gr);
}

/* ------------------------------------------------------------------------- */
/* Collision of f: entropic equilibrium, KBC split, stabiliser, exact-       */
/* difference forcing.  The paper names the entropic LBM with exact-         */
/* difference forcing (paragraph after Eq. 8); the formulas below are those  */
/* of the cited KBC/ELBM method (reading).                                   */
/* ------------------------------------------------------------------------- */

/* Entropic (product-form) equilibrium:
   f_i = rho w_i prod_a (2 - S_a) ((2 u_a + S_a)/(1 - u_a))^{c_ia},
   S_a = sqrt(1 + 3 u_a^2). */
void orc_feq(const orc_ctx *o, double rho, const double u[3], double *feq)
{
    for (int i = 0; i < o->Q; i++) {
        double prod = 1.0;
        for (int a = 0; a < o->D; a++) {
            double S = sqrt(1.0 + 3.0 * u[a] * u[a]);
            double X = (2.0 * u[a] + S) / (1.0 - u[a]);
            double pw = o->c[i][a] == 1 ? X : (o->c[i][a] == -1 ? 1.0 / X : 1.0);
            prod *= (2.0 - S) * pw;
        }
        feq[i] = rho * o->w[i] * prod;
    }
}

/* Dual basis of the one-dimensional moments {1, c, c^2} on c in {-1,0,1}:
   sum_c d_k(c) c^m = delta_km. */
static double dual(int k, int c)
{
    if (k == 0) return c == 0 ? 1.0 : 0.0;
    if (k == 1) return 0.5 * c;
    return c == 0 ? -1.0 : 0.5;
}

/* The population vector whose natural moments M_pqr = sum_i X_i cx^p cy^q cz^r
   are all zero except M(e) = 1: product of the one-dimensional duals. */
static double dual_vec(const orc_ctx *o, int i, const int e[3])
{
    double v = 1.0;
    for (int a = 0; a < o->D; a++) v *= dual(e[a], o->c[i][a]);
    return v;
}

/* Exact stabiliser (reading of "gamma solved per node"): the KBC collision
   f'(gamma) = f - beta (2 Delta s + gamma Delta h) keeps the relaxation of the
   stress part fixed and picks gamma so that the post-collision state has the
   largest entropy along this line, i.e. minimises H(f') = sum_i f'_i ln(f'_i/w_i).
   dH/dgamma = -beta sum_i Delta h_i (ln(f'_i/w_i) + 1); the +1 drops because
   Delta h carries no mass, and ln(feq_i/w_i) is affine in c_i for the entropic
   equilibrium while Delta h carries no mass or momentum, so the condition is
     G = sum_i Delta h_i ln(f'_i / feq_i) = 0.
   Its second-order expansion in f - f^eq is the closed form of the collision.
   Written in t = 1 - beta gamma:  f'_i(t) = A_i + t Delta h_i with
   A_i = feq_i + (1 - 2 beta) Delta s_i, so G(t) is strictly increasing,
   G'(t) = sum_i Delta h_i^2 / f'_i(t), on the interval where every f'_i > 0,
   and runs from -inf to +inf across it: the root is unique.  Found by Newton
   from the closed form, kept inside a bracket by bisection. */
int orc_gamma_exact(const orc_ctx *o, const double *feq, const double *ds, const double *dh,
                    double gamma0, double *gamma)
{
    int Q = o->Q;
    double beta = o->beta;
    double A[27];
    double lo = -HUGE_VAL, hi = HUGE_VAL;
    int npos = 0, nneg = 0;
    *gamma = gamma0;
    /* Delta h carries no mass, so it has entries of both signs unless it is
       rounding noise; then the closed form is kept (not a failure) */
    for (int i = 0; i < Q; i++) {
        npos += dh[i] > 0.0;
        nneg += dh[i] < 0.0;
    }
    if (npos == 0 || nneg == 0) return -2;
    for (int i = 0; i < Q; i++) {
        A[i] = feq[i] + (1.0 - 2.0 * beta) * ds[i];
        if (dh[i] > 0.0) {
            double b = -A[i] / dh[i];
            if (b > lo) lo = b;
        } else if (dh[i] < 0.0) {
            double b = -A[i] / dh[i];
            if (b < hi) hi = b;
        } else if (!(A[i] > 0.0)) {
            return -1;
        }
    }
    if (!(lo < hi) || !isfinite(lo) || !isfinite(hi)) return -1;
    double t = 1.0 - beta * gamma0;
    if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
    double a = lo, b = hi;
    for (int it = 1; it <= ORC_GAMMA_MAX_ITER; it++) {
        double G = 0.0, dG = 0.0, S = 0.0;
        for (int i = 0; i < Q; i++) {
            double x = ((1.0 - 2.0 * beta) * ds[i] + t * dh[i]) / feq[i];
            G += dh[i] * log1p(x);
            /* size of the term before the two parts of x cancel: the scale
               of G's rounding */
            S += fabs(dh[i]) * (fabs((1.0 - 2.0 * beta) * ds[i]) + fabs(t * dh[i])) / feq[i];
            dG += dh[i] * dh[i] / (feq[i] * (1.0 + x));
        }
        /* converged: G vanishes to the rounding of its terms */
        if (fabs(G) <= 1e-13 * S) {
            *gamma = (1.0 - t) / beta;
            return it;
        }
        if (G > 0.0) b = t; else a = t;
        if (!(b - a > 1e-15 * (1.0 + fabs(t)))) {
            *gamma = (1.0 - 0.5 * (a + b)) / beta;
            return it;
        }
        /* Newton step, or bisection when it leaves the bracket.  A step
           below rounding ends the iteration when G is at its rounding floor
           (within 1e3 of the bar), and bisects when it is not: next to a
           pole of ln f'_i the derivative is huge and the step tiny while G
           is large */
        double tn = t - G / dG;
        if (!(tn > a && tn < b)) {
            tn = 0.5 * (a + b);
        } else if (fabs(tn - t) <= 1e-15 * (1.0 + fabs(t))) {
            if (fabs(G) <= 1e-10 * S) {
                *gamma = (1.0 - tn) / beta;
                return it;
            }
            tn = 0.5 * (a + b);
        }
        t = tn;
    }
    return -1;
}

int orc_collide_f(const orc_ctx *o, const double *f, const double F[3],
                  double *fout, double *ds_out, double *gamma)
{
    int Q = o->Q, D = o->D;
    double rho = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; i++) {
        rho += f[i];
        for (int a = 0; a < 3; a++) j[a] += f[i] * o->c[i][a];
    }
    if (!(rho > 0.0)) return -3;
    double u[3], uF[3];
    for (int a = 0; a < 3; a++) {
        u[a] = j[a] / rho;
        uF[a] = u[a] + F[a] / rho;
    }
    for (int a = 0; a < D; a++)
        if (!(fabs(u[a]) < 1.0) || !(fabs(uF[a]) < 1.0)) return -3;
    double feq[27], feqF[27], dl[27], ds[27], dh[27];
    orc_feq(o, rho, u, feq);
    orc_feq(o, rho, uF, feqF);
    for (int i = 0; i < Q; i++) dl[i] = f[i] - feq[i];
    /* second-order moments of Delta = f - f^eq */
    double Pi[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            Pi[a][b] = 0.0;
            for (int i = 0; i < Q; i++) Pi[a][b] += dl[i] * o->c[i][a] * o->c[i][b];
        }
    double tr = 0.0;
    for (int a = 0; a < D; a++) tr += Pi[a][a];
    /* Delta s: the deviatoric part of the stress; every other natural moment
       (density, momentum, the trace of the stress, all higher moments) is 0
       (reading: trace left in h). */
    for (int i = 0; i < Q; i++) {
        double s = 0.0;
        for (int a = 0; a < D; a++) {
            int e[3] = {0, 0, 0};
            e[a] = 2;
            s += (Pi[a][a] - tr / D) * dual_vec(o, i, e);
            for (int b = a + 1; b < D; b++) {
                int e2[3] = {0, 0, 0};
                e2[a] = 1;
                e2[b] = 1;
                s += Pi[a][b] * dual_vec(o, i, e2);
            }
        }
        ds[i] = s;
        dh[i] = dl[i] - ds[i];
    }
    /* entropic scalar products <X|Y> = sum_i X_i Y_i / f^eq_i */
    double sh = 0.0, hh = 0.0;
    for (int i = 0; i < Q; i++) {
        sh += ds[i] * dh[i] / feq[i];
        hh += dh[i] * dh[i] / feq[i];
    }
    double beta = o->beta;
    double g = 2.0;
    if (hh > 1e-30 * rho * rho) {
        g = 1.0 / beta - (2.0 - 1.0 / beta) * sh / hh;
        if (o->p.gamma_mode == ORC_GAMMA_EXACT) {
            double ge;
            int it = orc_gamma_exact(o, feq, ds, dh, g, &ge);
            if (it >= 0) g = ge;
            else if (it == -1) {
#pragma omp atomic
                (*o->gamma_fallbacks)++;
            }
        }
    }
    for (int i = 0; i < Q; i++) {
        fout[i] = f[i] - beta * (2.0 * ds[i] + g * dh[i]) + (feqF[i] - feq[i]);
        if (ds_out) ds_out[i] = ds[i];
    }
    if (gamma) *gamma = g;
    for (int i = 0; i < Q; i++)
        if (!isfinite(fout[i])) return -3;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Phase field: BGK with the standard Cahn-Hilliard equilibrium (paragraph    */
/* after Eq. 8 cites the textbook scheme; reading):                           */
/*   g_i = w_i [Gamma mu_phi / c_s^2 + phi c_i.u / c_s^2                      */
/*              + phi ((c_i.u)^2 / (2 c_s^4) - u.u / (2 c_s^2))],  i != 0      */
/*   g_0 = phi - sum_{i != 0} g_i.                                             */
/* ------------------------------------------------------------------------- */
void orc_geq(const orc_ctx *o, double phi, double mu_phi, const double u[3],
             double *geq)
{
    const double cs2 = 1.0 / 3.0;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double others = 0.0;
    for (int i = 0; i < o->Q; i++) {
        if (i == o->rest) continue;
        double cu = o->c[i][0] * u[0] + o->c[i][1] * u[1] + o->c[i][2] * u[2];
        geq[i] = o->w[i] * (o->p.Gamma * mu_phi / cs2 + phi * cu / cs2
                            + phi * (cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2)));
        others += geq[i];
    }
    geq[o->rest] = phi - others;
}

void orc_collide_g(const orc_ctx *o, const double *g, double phi, double mu_phi,
                   const double u[3], double *gout)
{
    double geq[27];
    orc_geq(o, phi, mu_phi, u, geq);
    for (int i = 0; i < o->Q; i++) gout[i] = g[i] - (g[i] - geq[i]) / o->p.tau_g;
}

/* ------------------------------------------------------------------------- */
/* Streaming (pull) with periodic wrap and half-way bounce-back.             */
/* ------------------------------------------------------------------------- */

/* Source of population i at node (x,y,z): returns the source node index, or
   -1 when x - c_i lies beyond a bounce-back wall or is a solid node. */
static long pull_src(const orc_ctx *o, int x, int y, int z, int i)
{
    int q[3] = {x - o->c[i][0], y - o->c[i][1], z - o->c[i][2]};
    int n[3] = {o->nx, o->ny, o->nz};
    for (int a = 0; a < 3; a++) {
        if (q[a] < 0 || q[a] >= n[a]) {
            if (o->bc[a] != 0) return -1;
            q[a] = (q[a] + n[a]) % n[a];
        }
    }
    long s = (long)q[0] + (long)o->nx * ((long)q[1] + (long)o->ny * q[2]);
    return is_solid(o, s) ? -1 : s;  /* half-way bounce-back at a solid node */
}

void orc_stream(const orc_ctx *o, const double *post, double *pre)
{
    long N = o->N;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                long n = x + (long)o->nx * (y + (long)o->ny * z);
                for (int i = 0; i < o->Q; i++) {
                    long s = pull_src(o, x, y, z, i);
                    if (is_solid(o, n)) pre[i * N + n] = 0.0;
                    else pre[i * N + n] = s >= 0 ? post[i * N + s] : post[o->opp[i] * N + n];
                }
            }
}

void orc_unstream(const orc_ctx *o, const double *pre, double *post)
{
    long N = o->N;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                long n = x + (long)o->nx * (y + (long)o->ny * z);
                if (is_solid(o, n)) {
                    for (int i = 0; i < o->Q; i++) post[i * N + n] = 0.0;
                    continue;
                }
                for (int i = 0; i < o->Q; i++) {
                    long s = pull_src(o, x, y, z, i);
                    if (s >= 0) post[i * N + s] = pre[i * N + n];
                    else post[o->opp[i] * N + n] = pre[i * N + n];
                }
            }
}

/* ------------------------------------------------------------------------- */
/* Whole step                                                                */
/* ------------------------------------------------------------------------- */

typedef struct {
    double *fpre, *gpre, *rho, *phi, *j, *mr, *mp, *F;
} work_t;

static int work_alloc(const orc_ctx *o, work_t *w)
{
    long N = o->N, Q = o->Q;
    w->fpre = (double *)malloc(sizeof(double) * Q * N);
    w->gpre = (double *)malloc(sizeof(double) * Q * N);
    w->rho = (double *)malloc(sizeof(double) * N);
    w->phi = (double *)malloc(sizeof(double) * N);
    w->j = (double *)malloc(sizeof(double) * 3 * N);
    w->mr = (double *)malloc(sizeof(double) * N);
    w->mp = (double *)malloc(sizeof(double) * N);
    w->F = (double *)malloc(sizeof(double) * 3 * N);
    if (!w->fpre || !w->gpre || !w->rho || !w->phi || !w->j || !w->mr || !w->mp || !w->F)
        return -2;
    return 0;
}

static void work_free(work_t *w)
{
    free(w->fpre); free(w->gpre); free(w->rho); free(w->phi);
    free(w->j); free(w->mr); free(w->mp); free(w->F);
}

/* stream, then the moments rho = sum f, j = sum f c, phi = sum g, then the
   chemical potentials and the force */
static void pre_collision(const orc_ctx *o, const double *f, const double *g, work_t *w)
{
    long N = o->N;
    orc_stream(o, f, w->fpre);
    orc_stream(o, g, w->gpre);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        double r = 0.0, p = 0.0, jj[3] = {0, 0, 0};
        for (int i = 0; i < o->Q; i++) {
            r += w->fpre[i * N + n];
            p += w->gpre[i * N + n];
            for (int a = 0; a < 3; a++) jj[a] += w->fpre[i * N + n] * o->c[i][a];
        }
        w->rho[n] = r;
        w->phi[n] = p;
        for (int a = 0; a < 3; a++) w->j[a * N + n] = jj[a];
        if (is_solid(o, n)) {
            /* placeholder moments of a solid node: no stencil of a fluid node
               reads them (ghosts), they only keep the arithmetic finite */
            w->rho[n] = o->rho_l;
            w->phi[n] = 0.0;
            for (int a = 0; a < 3; a++) w->j[a * N + n] = 0.0;
        }
    }
    orc_chem_pot(o, w->rho, w->phi, w->mr, w->mp);
    orc_force(o, w->rho, w->phi, w->mr, w->mp, w->F);
}

int orc_step(const orc_ctx *o, double *f, double *g, int nsteps)
{
    long N = o->N;
    int Q = o->Q, rc = 0;
    work_t w;
    if (nsteps < 0) return -1;
    if (work_alloc(o, &w)) { work_free(&w); return -2; }
    for (int s = 0; s < nsteps && rc == 0; s++) {
        pre_collision(o, f, g, &w);
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; n++) {
            double fl[27], gl[27], fo[27], go[27], F[3], u[3];
            if (is_solid(o, n)) {  /* the state of a solid node is zero */
                for (int i = 0; i < Q; i++) f[i * N + n] = g[i * N + n] = 0.0;
                continue;
            }
            for (int i = 0; i < Q; i++) {
                fl[i] = w.fpre[i * N + n];
                gl[i] = w.gpre[i * N + n];
            }
            for (int a = 0; a < 3; a++) F[a] = w.F[a * N + n];
            int e = orc_collide_f(o, fl, F, fo, NULL, NULL);
            if (e) {
#pragma omp atomic write
                rc = e;
            }
            /* the phase field is advected with u = (j + F/2)/rho (reading) */
            for (int a = 0; a < 3; a++) u[a] = (w.j[a * N + n] + 0.5 * F[a]) / w.rho[n];
            orc_collide_g(o, gl, w.phi[n], w.mp[n], u, go);
            for (int i = 0; i < Q; i++) {
                f[i * N + n] = fo[i];
                g[i * N + n] = go[i];
            }
        }
    }
    work_free(&w);
    return rc;
}

/* Initial state from rho, phi, u (reading): f = f^eq(rho, u - F/(2 rho)),
   g = g^eq(phi, mu_phi, u), placed so that the first step streams them back
   onto the nodes they belong to. */
int orc_init(const orc_ctx *o, const double *rho, const double *phi,
             const double *u, double *f, double *g)
{
    long N = o->N;
    int Q = o->Q, D = o->D, rc = 0;
    double *mr = (double *)malloc(sizeof(double) * N);
    double *mp = (double *)malloc(sizeof(double) * N);
    double *F = (double *)malloc(sizeof(double) * 3 * N);
    double *fpre = (double *)malloc(sizeof(double) * Q * N);
    double *gpre = (double *)malloc(sizeof(double) * Q * N);
    if (!mr || !mp || !F || !fpre || !gpre) rc = -2;
    if (rc == 0) {
        orc_chem_pot(o, rho, phi, mr, mp);
        orc_force(o, rho, phi, mr, mp, F);
        for (long n = 0; n < N && rc == 0; n++) {
            double us[3] = {0, 0, 0}, uu[3] = {0, 0, 0}, fe[27], ge[27];
            if (is_solid(o, n)) continue;  /* zeroed by orc_unstream */
            if (!(rho[n] > 0.0)) { rc = -3; break; }
            for (int a = 0; a < D; a++) {
                uu[a] = u[a * N + n];
                us[a] = uu[a] - F[a * N + n] / (2.0 * rho[n]);
                if (!(fabs(us[a]) < 1.0)) rc = -3;
            }
            orc_feq(o, rho[n], us, fe);
            orc_geq(o, phi[n], mp[n], uu, ge);
            for (int i = 0; i < Q; i++) {
                fpre[i * N + n] = fe[i];
                gpre[i * N + n] = ge[i];
            }
        }
        if (rc == 0) {
            orc_unstream(o, fpre, f);
            orc_unstream(o, gpre, g);
        }
    }
    free(mr); free(mp); free(F); free(fpre); free(gpre);
    return rc;
}

/* Fields of the state: the moments of the streamed populations, the physical
   velocity u = (j + F/2)/rho and the isotropic part of the pressure tensor
   p = rho mu_rho + phi mu_phi - f_B - f_I (f_I of Eq. 5 with the isotropic
   gradients). */
int orc_fields(const orc_ctx *o, const double *f, const double *g, double *rho,
               double *phi, double *u, double *p)
{
    long N = o->N;
    int D = o->D;
    work_t w;
    if (work_alloc(o, &w)) { work_free(&w); return -2; }
    pre_collision(o, f, g, &w);
    for (long n = 0; n < N; n++) {
        rho[n] = w.rho[n];
        phi[n] = w.phi[n];
        for (int a = 0; a < D; a++) u[a * N + n] = (w.j[a * N + n] + 0.5 * w.F[a * N + n]) / w.rho[n];
    }
    if (p) {
        const orc_params *q = &o->p;
        double *gr = (double *)malloc(sizeof(double) * 3 * N);
        double *gp = (double *)malloc(sizeof(double) * 3 * N);
        orc_gradient(o, w.rho, gr);
        orc_gradient(o, w.phi, gp);
        double Dl = o->rho_g - o->rho_l, chi = q->chi;
        double A = 0.5 * q->kappa1 + (q->kappa2 + q->kappa3) / (8.0 * Dl * Dl);
        double B = (q->kappa2 + q->kappa3) / (8.0 * chi * chi);
        double X = (q->kappa3 - q->kappa2) / (4.0 * chi * Dl);
        for (long n = 0; n < N; n++) {
            double rr = 0, pp = 0, rp = 0;
            for (int a = 0; a < 3; a++) {
                rr += gr[a * N + n] * gr[a * N + n];
                pp += gp[a * N + n] * gp[a * N + n];
                rp += gr[a * N + n] * gp[a * N + n];
            }
            double fI = A * rr + B * pp + X * rp;
            p[n] = w.rho[n] * w.mr[n] + w.phi[n] * w.mp[n] - orc_f_bulk(o, w.rho[n], w.phi[n]) - fI;
        }
        free(gr);
        free(gp);
    }
    int rc = 0;
    for (long n = 0; n < N; n++) {
        if (is_solid(o, n)) {  /* the fields of a solid node are zero */
            rho[n] = phi[n] = 0.0;
            for (int a = 0; a < D; a++) u[a * N + n] = 0.0;
            if (p) p[n] = 0.0;
            continue;
        }
        if (!(w.rho[n] > 0.0) || !isfinite(w.phi[n])) rc = -3;
    }
    work_free(&w);
    return rc;
}
