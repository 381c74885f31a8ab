/*
 * orc.h -- plain FP64 CPU oracle of the ternary free-energy entropic lattice
 * Boltzmann update (Woehrwag, Semprebon, Mazloomi M., Karlin, Kusumaatmaja,
 * "Ternary free-energy entropic lattice Boltzmann model with high density
 * ratio", arXiv:1710.07486).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library.  Only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (own to the oracle):
 *   lattice 0 = D2Q9 (nz must be 1), lattice 1 = D3Q27.
 *   velocity i has components c[i] in {-1,0,1}^D, listed explicitly in orc.c.
 *   node index n = x + nx*(y + ny*z);  populations are SoA: f[i*N + n].
 *   bc[a] = 0 periodic along axis a, 1 = half-way bounce-back walls at both
 *   ends of axis a.
 *   Solid nodes (params.solid): half-way bounce-back wherever a pull would
 *   read a solid node; stencil reads of a solid neighbour take a fluid ghost
 *   (see orc.c, ghost_nb); the state and fields of a solid node are zero.
 *   The stored state is the post-collision population set, i.e. what the
 *   next step streams (pulls) from.
 *
 * All functions return 0 on success and a negative code on failure:
 *   -1 bad argument, -2 out of memory, -3 unstable node (rho<=0, |u+F/rho|>=1
 *   or a non-finite value).
 */
#ifndef ORC_H
#define ORC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double a, b, R, T;                 /* Carnahan-Starling constants, Eq. 4  */
    double lambda1, lambda2, lambda3;  /* bulk weights, Eq. 2                 */
    double kappa1, kappa2, kappa3;     /* square-gradient weights, Eq. 3      */
    double chi;                        /* phase-field scale (text after Eq. 4)*/
    double nu;                         /* kinematic viscosity, tau = 3 nu + 1/2 */
    double Gamma, tau_g;               /* mobility M = Gamma (tau_g - 1/2)    */
    int force_form;                    /* 0 potential form, 1 lattice-consistent */
    int eos;                           /* ORC_EOS_CS (Eq. 4), ORC_EOS_VDW, ORC_EOS_PR */
    double omega;                      /* Peng-Robinson acentric factor          */
    int gamma_mode;                    /* ORC_GAMMA_CLOSED or ORC_GAMMA_EXACT    */
    const unsigned char *solid;        /* per-node solid mask [N] (nonzero =
                                          solid), copied at create; NULL: none */
    double wet_rho, wet_phi;           /* wetting gradients at walls and solid
                                          nodes (0: neutral); see orc_laplacian_wet */
} orc_params;

/* Stabiliser of the KBC collision: the closed form (the root of the entropy
   condition to second order in f - f^eq) or the exact per-node root of the
   entropy condition (safeguarded Newton, falling back to the closed form). */
enum { ORC_GAMMA_CLOSED = 0, ORC_GAMMA_EXACT = 1 };
#define ORC_GAMMA_MAX_ITER 20

/* Equations of state: Carnahan-Starling (Eq. 4), and the van der Waals and
   Peng-Robinson forms the text names as alternatives (textbook forms). */
enum { ORC_EOS_CS = 0, ORC_EOS_VDW = 1, ORC_EOS_PR = 2 };
typedef struct {
    int kind;
    double a, b, R, T, omega;
} orc_eos;
double orc_eos_psi(const orc_eos *e, double rho);
double orc_eos_dpsi(const orc_eos *e, double rho);
double orc_eos_p(const orc_eos *e, double rho);
int orc_eos_coexistence(const orc_eos *e, double out[4]);
int orc_eos_critical_point(int kind, double a, double b, double R, double omega, double out[2]);
int orc_eos_temperature_for_ratio(int kind, double a, double b, double R, double omega, double ratio, double *T);
double orc_pr_tc(double a, double b, double R);

typedef struct orc_ctx orc_ctx;

/* --- thermodynamics (Eq. 4, common tangent) ------------------------------ */
double orc_psi_tilde(double a, double b, double R, double T, double rho);
double orc_dpsi_tilde(double a, double b, double R, double T, double rho);
double orc_p_eos(double a, double b, double R, double T, double rho);
/* out = {rho_g, rho_l, mu_coex, p_coex} */
int orc_coexistence(double a, double b, double R, double T, double out[4]);
/* critical temperature of the CS EOS found numerically: out = {T_c, rho_c} */
int orc_critical_point(double a, double b, double R, double out[2]);
/* temperature whose coexistence densities have rho_l/rho_g = ratio */
int orc_temperature_for_ratio(double a, double b, double R, double ratio, double *T);

/* --- context ---------------------------------------------------------------- */
orc_ctx *orc_create(int lattice, int nx, int ny, int nz, const orc_params *p,
                    const int bc[3]);
void orc_destroy(orc_ctx *o);
int orc_Q(const orc_ctx *o);
long orc_N(const orc_ctx *o);
/* c[27*3] (int) and w[27] of the oracle's velocity set */
void orc_velocities(const orc_ctx *o, int *c, double *w);
/* out = {rho_g, rho_l, mu_coex, p_coex, tau, beta} */
void orc_derived(const orc_ctx *o, double out[6]);

/* --- single-node pieces ------------------------------------------------------ */
/* bulk free-energy density f_B(rho,phi) of Eq. 2, with Psi_0 and C from the
   common tangent */
double orc_f_bulk(const orc_ctx *o, double rho, double phi);
/* entropic equilibrium f^eq(rho,u) */
void orc_feq(const orc_ctx *o, double rho, const double u[3], double *feq);
/* KBC collision + exact-difference forcing of one node.  f[Q] pre-collision,
   F[3] force.  fout[Q] post-collision.  ds_out[Q] (nullable) receives Delta s.
   Returns gamma in *gamma. */
int orc_collide_f(const orc_ctx *o, const double *f, const double F[3],
                  double *fout, double *ds_out, double *gamma);
/* Exact stabiliser: the root gamma of the entropy condition
     sum_i dh_i ln(f'_i(gamma) / feq_i) = 0,  f'(gamma) = f - beta (2 ds + gamma dh)
   for one node, given f^eq, Delta s and Delta h = f - f^eq - Delta s.  Starts
   from gamma0.  Returns the number of Newton/bisection iterations (>= 0) with
   *gamma the root; -1 when there is no admissible gamma (some f'_i <= 0 for
   every gamma) or the iteration did not converge in ORC_GAMMA_MAX_ITER steps
   (a fallback); -2 when Delta h has entries of one sign only, which a
   massless Delta h can only have as rounding noise (not a fallback).  In
   both negative cases *gamma = gamma0. */
int orc_gamma_exact(const orc_ctx *o, const double *feq, const double *ds, const double *dh,
                    double gamma0, double *gamma);
/* Number of nodes whose exact stabiliser fell back to the closed form since
   the context was created (ORC_GAMMA_EXACT only). */
long orc_gamma_fallbacks(const orc_ctx *o);
void orc_geq(const orc_ctx *o, double phi, double mu_phi, const double u[3],
             double *geq);
void orc_collide_g(const orc_ctx *o, const double *g, double phi, double mu_phi,
                   const double u[3], double *gout);

/* --- whole-lattice pieces ----------------------------------------------------- */
/* pull-stream a post-collision state into pre-collision populations */
void orc_stream(const orc_ctx *o, const double *post, double *pre);
/* inverse of orc_stream: the post-collision state that streams into pre */
void orc_unstream(const orc_ctx *o, const double *pre, double *post);
/* chemical potentials (rho,phi fields -> mu_rho, mu_phi) */
void orc_chem_pot(const orc_ctx *o, const double *rho, const double *phi,
                  double *mu_rho, double *mu_phi);
/* F[3*N] (SoA, component-major) from rho, phi, mu_rho, mu_phi */
void orc_force(const orc_ctx *o, const double *rho, const double *phi,
               const double *mu_rho, const double *mu_phi, double *F);
/* isotropic gradient [3*N] and Laplacian [N] of a scalar field */
void orc_gradient(const orc_ctx *o, const double *psi, double *grad);
void orc_laplacian(const orc_ctx *o, const double *psi, double *lap);
/* The Laplacian of a density-like field with a wetting gradient: a ghost
   read across a wall or a solid surface takes the mirrored fluid value plus
   wet times the number of axes mirrored (the chemical potentials' Laplacians
   of density and composition use it with wet_rho and wet_phi). */
void orc_laplacian_wet(const orc_ctx *o, const double *psi, double wet, double *lap);

/* rho[N], phi[N], u[D*N] (SoA) -> post-collision state f[Q*N], g[Q*N] */
int orc_init(const orc_ctx *o, const double *rho, const double *phi,
             const double *u, double *f, double *g);
/* advance the state by nsteps */
int orc_step(const orc_ctx *o, double *f, double *g, int nsteps);
/* macroscopic fields of the state: rho, phi, u_phys[D*N], p (nullable) */
int orc_fields(const orc_ctx *o, const double *f, const double *g, double *rho,
               double *phi, double *u, double *p);

#ifdef __cplusplus
}
#endif
#endif
