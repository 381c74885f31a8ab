/*
 * ternelbm.h -- C ABI of libternelbm, a CUDA (sm_103a) implementation of the
 * per-timestep lattice update of the ternary free-energy entropic lattice
 * Boltzmann method of Woehrwag, Semprebon, Mazloomi M., Karlin and
 * Kusumaatmaja, "Ternary free-energy entropic lattice Boltzmann model with
 * high density ratio" (arXiv:1710.07486).
 *
 * The model (paper, Eqs. 1-8): one gas and two liquids described by the
 * density rho and the phase field phi; bulk free energy of Eq. 2 with the
 * Carnahan-Starling free energy of Eq. 4; square-gradient energy of Eqs. 3
 * and 5; chemical potentials mu_rho = dF/drho, mu_phi = dF/dphi and pressure
 * tensor with div P = rho grad mu_rho + phi grad mu_phi (text after Eq. 8).
 * The density/momentum populations f use the entropic (KBC) collision with
 * exact-difference forcing, the phase-field populations g a BGK collision
 * (text after Eq. 8).  Lattices D2Q9 and D3Q27 (c_s^2 = 1/3), periodic or
 * half-way bounce-back boundaries per axis.
 *
 * Conventions
 *   - Node index n = x + nx*(y + ny*z), x fastest.  nz = 1 for D2Q9.
 *   - Velocity i has c_i = (i%3 - 1, (i/3)%3 - 1, i/9 - 1) (the z component
 *     only for D3Q27); the opposite of i is Q-1-i.
 *   - Field arrays are FP64: rho[N], phi[N], u[D*N] component-major
 *     (u[a*N + n]), p[N].  Population arrays are FP64 [Q][N].
 *   - Host pointers are caller-owned and only read/written during the call;
 *     nothing is retained.  "_device" entry points take caller-owned device
 *     pointers on the context's device.
 *   - The context owns all device memory it allocates (populations, double
 *     buffered; scratch for fields and state conversion; an error word).
 *   - All work is enqueued on the context's stream (default: a stream the
 *     library creates; see tel_set_stream).  tel_step is asynchronous; host
 *     entry points that return data synchronise the stream.
 *
 * Errors: every int-returning call returns TEL_OK (0) or a negative code;
 * tel_last_error() gives a message for the last failing call on a context.
 * A numerically unstable node (rho <= 0, a velocity component with
 * |u| >= 1 or |u + F/rho| >= 1 where the entropic equilibrium is undefined,
 * or a non-finite value) sets a device flag; it is reported as TEL_EUNSTABLE
 * by the next synchronising call (tel_sync, tel_fields, tel_get_state).
 */
#ifndef TERNELBM_H
#define TERNELBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TEL_OK 0
#define TEL_EINVAL (-1)    /* bad lattice, size, pointer or parameter */
#define TEL_ENOMEM (-2)    /* device allocation failed */
#define TEL_ECUDA (-3)     /* CUDA runtime error (launch, copy, device) */
#define TEL_EUNSTABLE (-4) /* the device flagged an unstable node */
#define TEL_ESTATE (-5)    /* call out of order (e.g. step before init) */

typedef enum { TEL_D2Q9 = 0, TEL_D3Q27 = 1 } tel_lattice;

/* TEL_FP64: populations stored and updated in FP64.
 * TEL_FP32_SHIFTED: populations stored in FP32 as f_i - w_i rho_ref (and
 * g_i - w_i * 0); arithmetic in FP32.  Where a cancellation happens the
 * value of the FP64 expression rounded to FP32 is obtained in double-float
 * FP32 arithmetic (error-free transformations, one final rounding): the
 * entropic stabiliser beta gamma = 1 - (2 beta - 1) q from the ratio q of its
 * scalar products, and, on the gas side (rho < sqrt(rho_g rho_l)), the sum of
 * the cancellation-free pieces of the equation-of-state chemical potential's
 * difference to its value at rho_g (Eq. 4; the van der Waals and
 * Peng-Robinson gas sides are FP64 throughout). */
typedef enum { TEL_FP64 = 0, TEL_FP32_SHIFTED = 1 } tel_precision;

typedef enum { TEL_PERIODIC = 0, TEL_BOUNCEBACK = 1 } tel_bc;

/* Discretisation of the ideal-pressure part of the force
 * F = -rho grad mu_rho - phi grad mu_phi + F_id:
 *   TEL_FORCE_POTENTIAL: F_id = c_s^2 grad rho (isotropic gradient);
 *   TEL_FORCE_LATTICE:   F_id = c_s^2 (3/2 G - 1/2 A[G]) + div(c_s^4 G G/(4 rho)),
 *     G = grad rho, A[G]_a(x) = sum_i 3 w_i c_ia c_i.G(x - c_i): the form for
 *     which a steady state of the update is the thermodynamic equilibrium to
 *     the next order (see the oracle and design notes). */
typedef enum { TEL_FORCE_POTENTIAL = 0, TEL_FORCE_LATTICE = 1 } tel_force_form;

typedef struct {
    double a, b, R, T;                /* Carnahan-Starling EOS, Eq. 4 (absolute T) */
    double lambda1, lambda2, lambda3; /* Eq. 2 */
    double kappa1, kappa2, kappa3;    /* Eq. 3 */
    double chi;                       /* phase-field scale: minima at (rho_l, +-chi) */
    double nu;                        /* kinematic viscosity; tau = 3 nu + 1/2, beta = 1/(2 tau) */
    double Gamma, tau_g;              /* mobility M = Gamma (tau_g - 1/2) */
    double rho_ref;                   /* FP32 shift density; <= 0 selects rho_g */
    int precision;                    /* tel_precision */
    int force_form;                   /* tel_force_form */
    int bc[3];                        /* tel_bc per axis (bc[2] ignored for D2Q9) */
    int eos;                          /* tel_eos: TEL_EOS_CS (Eq. 4, default 0), TEL_EOS_VDW, TEL_EOS_PR */
    double omega;                     /* Peng-Robinson acentric factor (TEL_EOS_PR only) */
    int gamma_mode;                   /* tel_gamma_mode: TEL_GAMMA_CLOSED (default 0), TEL_GAMMA_EXACT,
                                         TEL_GAMMA_CLOSED_F64SUM */
    const unsigned char *solid;       /* optional host solid mask [nz][ny][nx] (nonzero = solid),
                                         copied by tel_create; NULL = no solid nodes (see below) */
    double wet_rho, wet_phi;          /* wetting gradients at walls and solid nodes (see below);
                                         0, 0 = neutral wetting */
    int moments;                      /* tel_moments: TEL_MOMENTS_CARRIED (default 0) or
                                         TEL_MOMENTS_PULLED (see below) */
} tel_params;

/* Solid nodes (tel_params.solid; not in the paper, which names wetting
 * boundaries only as an outlook): half-way bounce-back wherever a pull would
 * read a solid node, f_i(x) = f*_{Q-1-i}(x); a stencil that would read a
 * solid neighbour along c reads a fluid ghost instead -- the components of c
 * set to zero, fewest first and in axis order x, y, z, until the node reached
 * is fluid; the vector components along zeroed axes change sign -- the same
 * neutral-wetting rule as the walls at the ends of a bounce-back axis, which
 * solid layers there reproduce exactly.  The state (populations) and the
 * fields of a solid node are zero; tel_init ignores its input fields there.
 * A lattice with solid nodes takes the kernel's walled path (64-bit indices,
 * per-pull tests).  Not available for batches or tel_fields_noalloc. */

/* Wetting (tel_params.wet_rho, wet_phi; not in the paper, which says only
 * that wetting boundary conditions fit the model): a gradient (Cahn-type)
 * condition.  In the Laplacians of density and composition in the chemical
 * potentials (Eq. 5), a ghost read across a bounce-back wall or a solid
 * surface is the mirrored fluid value plus wet_rho (wet_phi) for each axis
 * the read was mirrored on: the field continues linearly with that change
 * per lattice spacing into the wall.  wet_rho > 0 draws density to the wall
 * (the liquid wets it), wet_phi > 0 favours liquid 1 (phi > 0) there.  The
 * gradients keep the plain mirror: the chemical potentials' (no diffusive
 * flux into the wall) and the density gradient of the force's ideal-pressure
 * term, which stands for the pressure the bounced-back populations carry.
 * Both 0 gives the neutral rule above; both must be finite; they act only
 * where walls or solid nodes exist. */

/* Stabiliser gamma of the KBC collision f' = f - beta (2 Delta s + gamma
 * Delta h) (the entropic scheme named after Eq. 8):
 *   TEL_GAMMA_CLOSED: gamma = 1/beta - (2 - 1/beta) <Delta s|Delta h>/<Delta h|Delta h>,
 *     <X|Y> = sum_i X_i Y_i / feq_i, the root of the entropy condition below
 *     expanded to second order in f - f^eq;
 *   TEL_GAMMA_EXACT: per node, the root of the entropy condition
 *     sum_i Delta h_i ln(f'_i / feq_i) = 0 (the gamma that maximises the
 *     entropy of f' on the collision line), by Newton from the closed form
 *     kept in a bracket by bisection (at most 20 evaluations; FP64, or FP32
 *     in the FP32 mode, where a few unbracketed Newton steps come first).
 *     Where no gamma keeps every f'_i positive, or the iteration does not
 *     converge, the node keeps the closed form and a device counter is
 *     incremented (tel_gamma_fallbacks).  Where Delta h has entries of one
 *     sign only -- a massless Delta h does so only as rounding noise -- the
 *     closed form is kept without counting.
 *   TEL_GAMMA_CLOSED_F64SUM: the closed form with its two scalar products
 *     accumulated in FP64 (a precision variant of TEL_FP32_SHIFTED; with
 *     TEL_FP64 storage it is TEL_GAMMA_CLOSED).
 * gamma = 2 (BGK) wherever <Delta h|Delta h> <= 1e-30 rho^2.  Batches
 * (tel_batch_*) use the closed form. */
typedef enum { TEL_GAMMA_CLOSED = 0, TEL_GAMMA_EXACT = 1, TEL_GAMMA_CLOSED_F64SUM = 2 } tel_gamma_mode;

/* Equations of state.  TEL_EOS_CS is Eq. 4 (Carnahan-Starling).  The text
 * names van der Waals and Peng-Robinson as alternatives (their formulas are
 * in the unavailable supplement); these are the textbook forms, with the free
 * energy obtained like Eq. 4 by integrating p_eos = rho Psi' - Psi:
 *   TEL_EOS_VDW: p = rho R T/(1 - b rho) - a rho^2
 *   TEL_EOS_PR:  p = rho R T/(1 - b rho) - a alpha(T) rho^2/(1 + 2 b rho - b^2 rho^2),
 *                alpha = (1 + k (1 - sqrt(T/T_c)))^2,
 *                k = 0.37464 + 1.54226 omega - 0.26992 omega^2,
 *                T_c = 0.07780 a/(0.45724 b R).
 * The common tangent (C, Psi_0) is constructed the same way for all three. */
typedef enum { TEL_EOS_CS = 0, TEL_EOS_VDW = 1, TEL_EOS_PR = 2 } tel_eos;

/* How a step obtains the moments rho, phi (Eqs. 6-8: the zeroth moments of
 * the pulled f and g) that its stencils read on the tile + ring 2.  The
 * update computed is the same either way; the two differ only in the
 * rounding of those stencil inputs.
 *   TEL_MOMENTS_CARRIED: where it applies -- D3Q27, TEL_FP32_SHIFTED, every
 *     axis periodic, no solid node, nx % 32 == 0, ny % 4 == 0 -- each step
 *     also adds every post-collision population into the moments of the node
 *     that the next step's pull brings it to (FP32 atomic additions into a
 *     device array, so their summation order, and the last bit of those
 *     moments, varies from run to run), and the next step reads them instead
 *     of pulling the 54 populations of every ring node again.  The node's
 *     own collision still takes its mass from its pulled populations, so
 *     mass stays conserved to rounding.  tel_create then allocates three
 *     moment arrays (24 bytes per node); after tel_init, tel_init_device or
 *     tel_set_state the next tel_step first sums them from the state (one
 *     extra launch).  tel_step keeps a rotation over those arrays on the
 *     host, so a graph captured from tel_step calls repeats correctly only
 *     for a multiple of 6 steps.  Elsewhere this mode pulls (as below).
 *   TEL_MOMENTS_PULLED: every step pulls the populations of the tile and its
 *     ring to form their moments (deterministic). */
typedef enum { TEL_MOMENTS_CARRIED = 0, TEL_MOMENTS_PULLED = 1 } tel_moments;

typedef struct tel_ctx tel_ctx;

/* Create a lattice of nx*ny*nz nodes on the current CUDA device.
 * Validates the parameters (tau > 1/2, tau_g > 1/2, chi > 0, kappa >= 0,
 * lambda >= 0, T below the critical temperature, every extent >= 4, nz == 1
 * for D2Q9), solves the common-tangent construction for rho_g, rho_l
 * (text after Eq. 4), allocates the double-buffered populations (and, where
 * TEL_MOMENTS_CARRIED applies, three moment arrays of 2 N floats) and returns
 * the context in *out.  Errors: TEL_EINVAL, TEL_ENOMEM, TEL_ECUDA. */
int tel_create(int lattice, int nx, int ny, int nz, const tel_params *params,
               tel_ctx **out);

/* Release all device memory and the library-created stream. NULL is a no-op. */
void tel_destroy(tel_ctx *ctx);

/* Message for the last failing call on ctx; when ctx is NULL, the message of
 * the last failing context-free call (tel_create, tel_batch_create,
 * tel_fields_noalloc) made by the calling thread (each thread keeps its own).  Valid until the next
 * failing call of the same kind (same context, or same thread). */
const char *tel_last_error(const tel_ctx *ctx);

/* Run subsequent work on a caller stream (a cudaStream_t, e.g. PyTorch's
 * current stream); NULL returns to the library's own stream.  The caller
 * keeps ownership of its stream. */
int tel_set_stream(tel_ctx *ctx, void *cuda_stream);

/* Initial state from host fields rho[N], phi[N], u[D*N] (u is the physical
 * velocity): f = f^eq(rho, u - F/(2 rho)), g = g^eq(phi, mu_phi, u), placed
 * so that the first step streams them onto their nodes (reading of the
 * initialisation; the paper defers it to its supplement).  Synchronises. */
int tel_init(tel_ctx *ctx, const double *rho, const double *phi, const double *u);

/* As tel_init with device pointers (FP64, same layouts); asynchronous. */
int tel_init_device(tel_ctx *ctx, const double *rho, const double *phi, const double *u);

/* Advance nsteps time steps: per node pull-stream f and g, moments,
 * chemical potentials (Eqs. 1-5) on the isotropic stencils, force,
 * KBC collision with per-node stabiliser and exact-difference forcing for f,
 * BGK for g.  One fused kernel launch per step (plus, with carried moments,
 * one launch that sums them after a new state; see tel_moments).
 * Asynchronous.  TEL_ESTATE before initialisation. */
int tel_step(tel_ctx *ctx, int nsteps);

/* Wait for the context's stream and report the device's instability flag
 * (TEL_EUNSTABLE), then clear it. */
int tel_sync(tel_ctx *ctx);

/* Number of nodes (summed over steps) whose exact stabiliser fell back to the
 * closed form since tel_create (TEL_GAMMA_EXACT only).  Synchronises. */
int tel_gamma_fallbacks(tel_ctx *ctx, unsigned long long *count);

/* Macroscopic fields of the current state, on the host: rho, phi, physical
 * velocity u = (j + F/2)/rho [D*N], and (if p != NULL) the isotropic part of
 * the pressure tensor p = rho mu_rho + phi mu_phi - f_B - f_I.  Any of rho,
 * phi, u may be NULL to skip it.  Synchronises; reports TEL_EUNSTABLE. */
int tel_fields(tel_ctx *ctx, double *rho, double *phi, double *u, double *p);

/* As tel_fields into caller device buffers (any may be NULL); asynchronous. */
int tel_fields_device(tel_ctx *ctx, double *rho, double *phi, double *u, double *p);

/* Copy the state (post-collision populations, the arrays the next step
 * streams from) to / from host FP64 arrays f[Q*N], g[Q*N].  In the FP32
 * mode the shift is removed / applied.  tel_get_state synchronises. */
int tel_get_state(tel_ctx *ctx, double *f, double *g);
int tel_set_state(tel_ctx *ctx, const double *f, const double *g);

/* Sizes and derived constants: out[0..9] = {D, Q, nx, ny, nz, N, rho_g,
 * rho_l, mu_coex, p_coex}. */
int tel_info(const tel_ctx *ctx, double out[10]);

/* Context-free thermodynamics of the CS free energy (Eq. 4): coexistence
 * out[4] = {rho_g, rho_l, mu_coex, p_coex} at temperature T, and the
 * temperature at which rho_l/rho_g equals ratio.  TEL_EINVAL when there is
 * no liquid-gas coexistence. */
int tel_coexistence(double a, double b, double R, double T, double out[4]);
int tel_temperature_for_ratio(double a, double b, double R, double ratio, double *T);
/* The same two for any tel_eos (omega: Peng-Robinson acentric factor). */
int tel_coexistence_eos(int eos, double a, double b, double R, double T, double omega, double out[4]);
int tel_temperature_for_ratio_eos(int eos, double a, double b, double R, double omega, double ratio, double *T);

/* Batched D2Q9 lattices (many uneven, independent cases advanced in one
 * persistent launch).  ncases independent D2Q9 lattices of nx[c] x ny[c]
 * nodes with their own parameters (one precision for all) live in one set of
 * device buffers; each tel_batch_step step is ONE launch of a persistent
 * kernel that walks a work list of (case, tile, chunk) items, largest cases
 * first, so that small lattices no longer leave the GPU idle.  Pairs of steps
 * are replayed from a captured CUDA graph.  Each case evolves as a
 * tel_create lattice with the same parameters would, up to rounding (same
 * per-node source, compiled separately).  tel_batch_tune times every (tile width 32/64, chunk
 * 8/16/32/64) configuration on steps_per_config real steps (plus one warm-up
 * step each: they advance the state) and keeps the fastest; out = {tile width,
 * chunk, steps advanced}.  tel_batch_init (fields as for tel_init) must come
 * before the first step; called later it restarts case c from the given
 * fields; tel_batch_fields returns host fields of case c and reports
 * TEL_EUNSTABLE if any case flagged a node.  tel_batch_info out = {ncases,
 * total nodes, tile width, chunk, work items, persistent CTAs}. */
typedef struct tel_batch tel_batch;
int tel_batch_create(int ncases, const int *nx, const int *ny, const tel_params *params, tel_batch **out);
void tel_batch_destroy(tel_batch *b);
const char *tel_batch_last_error(const tel_batch *b);
/* As tel_set_stream: later batch work is issued on cuda_stream (NULL: the
 * batch's own stream).  The stream must not be the legacy default stream
 * (step pairs are captured into a graph on it). */
int tel_batch_set_stream(tel_batch *b, void *cuda_stream);
int tel_batch_init(tel_batch *b, int c, const double *rho, const double *phi, const double *u);
/* As tel_batch_init from device FP64 arrays (rho[N], phi[N], u[2N]) on the
 * batch's stream; asynchronous (no host copy, no synchronisation; a flagged
 * node shows in tel_batch_sync / tel_batch_errors). */
int tel_batch_init_device(tel_batch *b, int c, const double *rho, const double *phi, const double *u);
int tel_batch_step(tel_batch *b, int nsteps);
int tel_batch_sync(tel_batch *b);
int tel_batch_fields(tel_batch *b, int c, double *rho, double *phi, double *u, double *p);
/* As tel_fields_device for case c: device FP64 arrays (rho[N], phi[N],
 * u[2N], p[N], each may be NULL), asynchronous on the batch's stream; no
 * error-word check (see tel_batch_errors). */
int tel_batch_fields_device(tel_batch *b, int c, double *rho, double *phi, double *u, double *p);
/* Synchronises, copies every case's error word to flags[ncases] (0 = no
 * flagged node; else the TEL error bits) and clears them. */
int tel_batch_errors(tel_batch *b, unsigned *flags);
int tel_batch_tune(tel_batch *b, int steps_per_config, int out[3]);
int tel_batch_info(const tel_batch *b, double out[6]);

/* Allocation-free field extraction (the paper has no counterpart; this is a
 * service of the library).  For callers that cannot let a library allocate
 * device memory -- applications that give the whole device to their own
 * memory pool at start-up or must keep their device footprint fixed, and code
 * paths without access to cudaMalloc.  The caller holds the state in its own
 * device buffers, in the layout tel_get_state describes ([Q][N]; FP64, or
 * FP32 storing f_i - w_i rho_ref and g_i when params->precision is
 * TEL_FP32_SHIFTED, with rho_ref = params->rho_ref, or rho_g when that is
 * <= 0), and receives rho, phi, u, p (any may be NULL) in host buffers, as
 * tel_fields returns them.  No device or pinned memory is allocated: the
 * library stages the fields through a fixed device array of at most
 * TEL_NOALLOC_MAX_NODES nodes (about 12.6 MB).  Larger lattices are rejected
 * with TEL_EINVAL.
 * When the array's device memory is taken: under CUDA's lazy module loading
 * (the default) the array is loaded on a device by the FIRST call on that
 * device, and stays until the process exits.  So make one call on each device
 * at start-up, before handing the device's memory to your own pool (else that
 * first call can fail with TEL_ECUDA, out of memory), and before any stream
 * capture.  With eager loading (CUDA_MODULE_LOADING=EAGER) every GPU holds it
 * from the moment the library is loaded.
 * Calls share the array: calls that overlap on the GPU race with each other.
 * The work runs on cuda_stream (NULL: the legacy default stream) and the call
 * synchronises it.  Errors as for tel_fields; the message is available from
 * tel_last_error(NULL) on the calling thread. */
#define TEL_NOALLOC_MAX_NODES 262144
int tel_fields_noalloc(int lattice, int nx, int ny, int nz, const tel_params *params,
                       const void *f_state, const void *g_state, double *rho, double *phi,
                       double *u, double *p, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TERNELBM_H */
