// tel_api.cu -- host side of libternelbm: the C ABI declared in
// include/ternelbm.h.  Validates parameters, solves the common-tangent
// construction of the Carnahan-Starling free energy (text after Eq. 4 of
// arXiv:1710.07486), owns the device state and launches the fused kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "ternelbm.h"
#include "tel_kernels.cuh"

struct tel_ctx {
    int lattice, D, Q, nx, ny, nz;
    long long N;
    tel_params p;
    tel::DevParams dp;
    void *f[2], *g[2];
    int cur;
    unsigned *d_err;
    unsigned *h_err;  // pinned
    unsigned long long *d_gfall;  // exact-stabiliser fallbacks
    unsigned char *d_solid;       // device copy of the solid mask, or NULL
    double *scratch;  // FP64 fields / state staging, lazily allocated
    size_t scratch_elems;
    // carried moments (tel_moments): three arrays of 2N floats; mom[mom_r]
    // holds the moments of the current state when mom_valid
    float *mom[3];
    int mom_r, mom_valid;
    cudaStream_t own_stream, stream;
    int initialized;
    char msg[512];
};

// Message of the last failing context-free call (tel_create, the
// thermodynamics helpers, tel_batch_create, tel_fields_noalloc) on the calling
// thread: thread-local, so concurrent failures on different threads do not
// overwrite each other's text.
static thread_local char g_create_msg[512] = "";

static int fail(tel_ctx *c, int code, const char *fmt, ...)
{
    char *dst = c ? c->msg : g_create_msg;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_OR_FAIL(ctx, expr)                                                              \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), TEL_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));          \
    } while (0)

// ---------------------------------------------------------------------------
// Carnahan-Starling thermodynamics (Eq. 4).  With eta = b rho / 4 the
// pressure p = rho dPsi/drho - Psi is rho R T (1 + eta + eta^2 - eta^3)/(1 -
// eta)^3 - a rho^2; the chemical potential m = dPsi~/drho is the derivative
// of Eq. 4 with C = 0.  Coexistence: equal p and equal m.  Solved here by
// bisection on the chemical potential (gas and liquid branches bracketed by
// the spinodals, where dp/drho = 0), then Newton polishing of the 2x2 system.
// ---------------------------------------------------------------------------
namespace {
// The equation of state's pressure p, dPsi~/drho (m) and d2Psi~/drho2 (dm,
// with dp/drho = rho dm).  CS is Eq. 4; VDW and PR are the textbook forms
// (see tel_eos).
struct CS {
    int kind;
    double a, b, R, T, omega;
    double aal, A, c1, c2;  // PR: a alpha(T), a alpha/(2 sqrt2 b), (1 +- sqrt2) b
    CS(double a_, double b_, double R_, double T_, int kind_ = TEL_EOS_CS, double omega_ = 0.0)
        : kind(kind_), a(a_), b(b_), R(R_), T(T_), omega(omega_)
    {
        const double s2 = std::sqrt(2.0);
        double alpha = 1.0;
        if (kind == TEL_EOS_PR) {
            const double k = 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
            const double q = 1.0 + k * (1.0 - std::sqrt(T / (0.07780 * a / (0.45724 * b * R))));
            alpha = q * q;
        }
        aal = a * alpha;
        A = aal / (2.0 * s2 * b);
        c1 = (1.0 + s2) * b;
        c2 = (1.0 - s2) * b;
    }
    double limit() const { return (kind == TEL_EOS_CS ? 4.0 : 1.0) / b; }
    double p(double r) const
    {
        if (kind == TEL_EOS_VDW) return r * R * T / (1.0 - b * r) - a * r * r;
        if (kind == TEL_EOS_PR) return r * R * T / (1.0 - b * r) - aal * r * r / (1.0 + 2.0 * b * r - b * b * r * r);
        const double e = 0.25 * b * r;
        return r * R * T * (1 + e + e * e - e * e * e) / ((1 - e) * (1 - e) * (1 - e)) - a * r * r;
    }
    double m(double r) const  // dPsi~/drho
    {
        if (kind != TEL_EOS_CS) {
            double v = R * T * (std::log(r / (1.0 - b * r)) + 1.0 / (1.0 - b * r));
            if (kind == TEL_EOS_VDW) return v - 2.0 * a * r;
            return v - A * std::log((1.0 + c1 * r) / (1.0 + c2 * r)) - aal * r / (1.0 + 2.0 * b * r - b * b * r * r);
        }
        const double d = b * r - 4.0;
        return -2.0 * a * r - 8.0 * R * T * (24.0 - 2.0 * b * r) / (d * d * d) + R * T * (std::log(r) + 1.0);
    }
    double dm(double r) const  // d2Psi~/drho2
    {
        if (kind != TEL_EOS_CS) {
            const double q = 1.0 - b * r;
            double v = R * T * (1.0 / r + b / q + b / (q * q));
            if (kind == TEL_EOS_VDW) return v - 2.0 * a;
            const double D = 1.0 + 2.0 * b * r - b * b * r * r;
            return v - 2.0 * aal / D + aal * r * (2.0 * b - 2.0 * b * b * r) / (D * D);
        }
        const double d = b * r - 4.0;
        return -2.0 * a - 32.0 * R * T * b * (b * r - 16.0) / (d * d * d * d) + R * T / r;
    }
};

// spinodals: the two roots of dm = 0 below the density limit; false above T_c
bool spinodals(const CS &s, double &s1, double &s2)
{
    const double hi = 0.999 * s.limit();
    const int M = 4000;
    double prev = s.dm(1e-6 / s.b), x_prev = 1e-6 / s.b;
    int found = 0;
    double roots[2];
    for (int k = 1; k <= M && found < 2; ++k) {
        const double x = 1e-6 / s.b * std::pow(hi / (1e-6 / s.b), (double)k / M);
        const double v = s.dm(x);
        if ((prev > 0) != (v > 0)) {
            double lo_ = x_prev, hi_ = x;
            for (int it = 0; it < 200; ++it) {
                const double mid = 0.5 * (lo_ + hi_);
                if ((s.dm(mid) > 0) == (s.dm(lo_) > 0)) lo_ = mid; else hi_ = mid;
            }
            roots[found++] = 0.5 * (lo_ + hi_);
        }
        prev = v;
        x_prev = x;
    }
    if (found < 2) return false;
    s1 = roots[0];
    s2 = roots[1];
    return true;
}

// root of m(r) = target on a branch where m is increasing
double m_root(const CS &s, double target, double lo, double hi)
{
    for (int it = 0; it < 300; ++it) {
        const double mid = lo + 0.5 * (hi - lo);
        if (mid <= lo || mid >= hi) break;
        if (s.m(mid) < target) lo = mid; else hi = mid;
    }
    return lo + 0.5 * (hi - lo);
}

bool coexist(const CS &s, double out[4])
{
    double s1, s2;
    if (!(s.a > 0 && s.b > 0 && s.R > 0 && s.T > 0)) return false;
    if (!spinodals(s, s1, s2)) return false;
    const double rmax = 0.999 * s.limit();
    // chemical potentials spanned by both branches
    double mlo = s.m(s2), mhi = s.m(s1);
    if (!(mhi > mlo)) return false;
    double rg = 0, rl = 0;
    for (int it = 0; it < 300; ++it) {
        const double mu = 0.5 * (mlo + mhi);
        if (mu <= mlo || mu >= mhi) break;
        rg = m_root(s, mu, 1e-300, s1);
        rl = m_root(s, mu, s2, rmax);
        // too high a chemical potential leaves the liquid at the higher pressure
        if (s.p(rl) > s.p(rg)) mhi = mu; else mlo = mu;
    }
    const double mu = 0.5 * (mlo + mhi);
    rg = m_root(s, mu, 1e-300, s1);
    rl = m_root(s, mu, s2, rmax);
    // Newton polish on (m(rl) - m(rg), p(rl) - p(rg)) = 0
    for (int it = 0; it < 4; ++it) {
        const double F1 = s.m(rl) - s.m(rg), F2 = s.p(rl) - s.p(rg);
        const double a11 = -s.dm(rg), a12 = s.dm(rl), a21 = -rg * s.dm(rg), a22 = rl * s.dm(rl);
        const double det = a11 * a22 - a12 * a21;
        if (!(std::fabs(det) > 0)) break;
        const double drg = (F1 * a22 - F2 * a12) / det, drl = (a11 * F2 - a21 * F1) / det;
        const double nrg = rg - drg, nrl = rl - drl;
        if (!(nrg > 0 && nrg < s1 && nrl > s2 && nrl < rmax)) break;
        rg = nrg;
        rl = nrl;
    }
    out[0] = rg;
    out[1] = rl;
    out[2] = 0.5 * (s.m(rg) + s.m(rl));
    out[3] = 0.5 * (s.p(rg) + s.p(rl));
    return std::isfinite(out[0]) && std::isfinite(out[1]);
}
}  // namespace

extern "C" int tel_coexistence_eos(int eos, double a, double b, double R, double T, double omega, double out[4])
{
    if (!out || eos < TEL_EOS_CS || eos > TEL_EOS_PR) return TEL_EINVAL;
    if (!(a > 0 && b > 0 && R > 0 && T > 0)) return TEL_EINVAL;
    CS s(a, b, R, T, eos, omega);
    return coexist(s, out) ? TEL_OK : TEL_EINVAL;
}

extern "C" int tel_coexistence(double a, double b, double R, double T, double out[4])
{
    return tel_coexistence_eos(TEL_EOS_CS, a, b, R, T, 0.0, out);
}

extern "C" int tel_temperature_for_ratio_eos(int eos, double a, double b, double R, double omega, double ratio,
                                             double *T)
{
    if (!T || !(ratio > 1.0) || !(a > 0 && b > 0 && R > 0) || eos < TEL_EOS_CS || eos > TEL_EOS_PR)
        return TEL_EINVAL;
    // bracket: a low temperature with a larger ratio, and one near T_c
    double lo = 0.02 * a / (b * R), hi = lo, out[4];
    {
        CS s(a, b, R, lo, eos, omega);
        if (!coexist(s, out) || out[1] / out[0] < ratio) return TEL_EINVAL;
    }
    // walk up until coexistence disappears or the ratio falls below target
    for (double t = lo; t < 1.0 * a / (b * R); t *= 1.01) {
        CS s(a, b, R, t, eos, omega);
        if (!coexist(s, out) || out[1] / out[0] < ratio) { hi = t; break; }
        lo = t;
    }
    if (!(hi > lo)) return TEL_EINVAL;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        CS s(a, b, R, mid, eos, omega);
        if (coexist(s, out) && out[1] / out[0] > ratio) lo = mid; else hi = mid;
    }
    *T = 0.5 * (lo + hi);
    return TEL_OK;
}

extern "C" int tel_temperature_for_ratio(double a, double b, double R, double ratio, double *T)
{
    return tel_temperature_for_ratio_eos(TEL_EOS_CS, a, b, R, 0.0, ratio, T);
}

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
template <typename T>
static void fill_coef(const tel::DevParams &d, tel::Coef<T> &k)
{
    k.b = (T)d.b; k.a2 = (T)(-2.0 * d.a); k.RT8 = (T)(8.0 * d.RT); k.RT = (T)d.RT;
    k.mu_coex = (T)d.mu_coex; k.lam1h = (T)d.lam1h;
    k.rho_l = (T)d.rho_l; k.inv_Dl = (T)d.inv_Dl; k.inv_chi = (T)d.inv_chi;
    k.lam2 = (T)d.lam2; k.lam3 = (T)d.lam3; k.inv_2Dl = (T)d.inv_2Dl; k.inv_2chi = (T)d.inv_2chi;
    k.Kr = (T)d.Kr; k.Kp = (T)d.Kp; k.Kx = (T)d.Kx;
    k.rho_switch = (T)d.rho_switch; k.rho_ref = (T)d.rho_ref;
    k.beta = (T)d.beta; k.Gamma3 = (T)(3.0 * d.Gamma); k.inv_tau_g = (T)d.inv_tau_g;
    k.aal = (T)d.aal; k.prA = (T)d.prA; k.c1 = (T)d.c1; k.c2 = (T)d.c2;
    k.wr = (T)d.wet_rho; k.wp = (T)d.wet_phi;
}

static int validate(int lattice, int nx, int ny, int nz, const tel_params *p)
{
    if (lattice != TEL_D2Q9 && lattice != TEL_D3Q27) return fail(nullptr, TEL_EINVAL, "lattice must be 0 (D2Q9) or 1 (D3Q27)");
    if (nx < 4 || ny < 4 || (lattice == TEL_D3Q27 && nz < 4))
        return fail(nullptr, TEL_EINVAL, "every lattice extent must be >= 4 (got %d x %d x %d)", nx, ny, nz);
    if (lattice == TEL_D2Q9 && nz != 1) return fail(nullptr, TEL_EINVAL, "nz must be 1 for D2Q9");
    if (!p) return fail(nullptr, TEL_EINVAL, "params is NULL");
    if (!(p->nu > 0) || !std::isfinite(p->nu)) return fail(nullptr, TEL_EINVAL, "nu must be > 0 (tau > 1/2)");
    if (!(p->tau_g > 0.5) || !std::isfinite(p->tau_g)) return fail(nullptr, TEL_EINVAL, "tau_g must be > 1/2");
    if (!(p->chi > 0)) return fail(nullptr, TEL_EINVAL, "chi must be > 0");
    if (!(p->Gamma >= 0)) return fail(nullptr, TEL_EINVAL, "Gamma must be >= 0");
    if (!(p->kappa1 >= 0 && p->kappa2 >= 0 && p->kappa3 >= 0)) return fail(nullptr, TEL_EINVAL, "kappa must be >= 0");
    if (!(p->lambda1 >= 0 && p->lambda2 >= 0 && p->lambda3 >= 0)) return fail(nullptr, TEL_EINVAL, "lambda must be >= 0");
    if (p->precision != TEL_FP64 && p->precision != TEL_FP32_SHIFTED) return fail(nullptr, TEL_EINVAL, "bad precision");
    if (p->eos != TEL_EOS_CS && p->eos != TEL_EOS_VDW && p->eos != TEL_EOS_PR) return fail(nullptr, TEL_EINVAL, "bad eos");
    if (p->force_form != TEL_FORCE_POTENTIAL && p->force_form != TEL_FORCE_LATTICE) return fail(nullptr, TEL_EINVAL, "bad force_form");
    if (p->gamma_mode != TEL_GAMMA_CLOSED && p->gamma_mode != TEL_GAMMA_EXACT && p->gamma_mode != TEL_GAMMA_CLOSED_F64SUM)
        return fail(nullptr, TEL_EINVAL, "bad gamma_mode");
    if (p->moments != TEL_MOMENTS_CARRIED && p->moments != TEL_MOMENTS_PULLED)
        return fail(nullptr, TEL_EINVAL, "bad moments mode");
    if (!std::isfinite(p->wet_rho) || !std::isfinite(p->wet_phi))
        return fail(nullptr, TEL_EINVAL, "wetting gradients must be finite");
    for (int a = 0; a < 3; ++a)
        if (p->bc[a] != TEL_PERIODIC && p->bc[a] != TEL_BOUNCEBACK) return fail(nullptr, TEL_EINVAL, "bad bc[%d]", a);
    if (((long long)nx * ny * nz) >= (1LL << 31)) return fail(nullptr, TEL_EINVAL, "lattice too large (N must be < 2^31)");
    return TEL_OK;
}

// Device-side parameter block of a validated lattice and its coexistence
// point co = {rho_g, rho_l, mu_coex, p_coex}.
namespace tel {
// Resident CTAs per SM of the D2Q9 single-lattice step kernel (tel_d2q9.cu).
cudaError_t d2q9_step_ctas_per_sm(int precision, bool fast, bool vec, int *out);
}  // namespace tel

static void fill_devparams(int lattice, int nx, int ny, int nz, const tel_params &p, const double co[4],
                           tel::DevParams &d)
{
    d.nx = nx; d.ny = ny; d.nz = lattice == TEL_D2Q9 ? 1 : nz;
    for (int a = 0; a < 3; ++a) d.bc[a] = p.bc[a];
    d.N = (long long)nx * ny * d.nz;
    {
        // planes per CTA along the marching axis: long enough to amortise the
        // five warm-up planes of the pipeline, short enough to give about four
        // CTAs per SM (152 SMs): 8..32 planes
        const long long tiles = lattice == TEL_D2Q9 ? (nx + 63) / 64 : (long long)((nx + 31) / 32) * ((ny + 7) / 8);
        const long long planes = lattice == TEL_D2Q9 ? ny : nz;
        const long long want = (4 * 152 + tiles - 1) / tiles;
        long long ch = (planes + want - 1) / want;
        ch = ch < 8 ? 8 : (ch > 32 ? 32 : ch);
        d.chunk = (int)ch;
    }
    if (const char *ev = std::getenv("TEL_CHUNK")) {  // tuning override: planes per CTA
        const int v = std::atoi(ev);
        if (v >= 1) d.chunk = v;
    }
    d.force_form = p.force_form;
    d.eos = p.eos;
    d.a = p.a; d.b = p.b; d.RT = p.R * p.T;
    {
        const CS s(p.a, p.b, p.R, p.T, p.eos, p.omega);
        d.aal = s.aal; d.prA = s.A; d.c1 = s.c1; d.c2 = s.c2;
    }
    d.rho_g = co[0]; d.rho_l = co[1]; d.mu_coex = co[2]; d.p_coex = co[3];
    const double Dl = co[0] - co[1];
    d.lam1h = 0.5 * p.lambda1; d.lam2 = p.lambda2; d.lam3 = p.lambda3;
    d.inv_Dl = 1.0 / Dl;
    d.inv_chi = 1.0 / p.chi;
    d.inv_2Dl = 1.0 / (2.0 * Dl);
    d.inv_2chi = 1.0 / (2.0 * p.chi);
    d.Kr = p.kappa1 + (p.kappa2 + p.kappa3) / (4.0 * Dl * Dl);
    d.Kp = (p.kappa2 + p.kappa3) / (4.0 * p.chi * p.chi);
    d.Kx = (p.kappa3 - p.kappa2) / (4.0 * p.chi * Dl);
    d.AI = 0.5 * p.kappa1 + (p.kappa2 + p.kappa3) / (8.0 * Dl * Dl);
    d.BI = (p.kappa2 + p.kappa3) / (8.0 * p.chi * p.chi);
    d.XI = (p.kappa3 - p.kappa2) / (4.0 * p.chi * Dl);
    d.rho_switch = std::sqrt(co[0] * co[1]);
    d.inv_rho_g = 1.0 / co[0];
    d.inv_rho_g_f = (float)d.inv_rho_g;
    {
        d.gRT = d.lam1h * d.RT;
        d.rg_hi = (float)co[0];
        d.rg_lo = (float)(co[0] - (double)d.rg_hi);
        d.b_f = (float)p.b;
        const double q = 1.0 / (p.b * co[0] - 4.0);
        d.q_g = (float)q;
        d.q_g2 = (float)(q * q);
        d.q_g_x2 = (float)(2.0 * q);
        d.gRT8b_f = (float)(d.lam1h * 8.0 * d.RT * p.b);
        d.ga2_f = (float)(d.lam1h * 2.0 * p.a);
        d.gRT_hi = (float)d.gRT;
        d.gRT_lo = (float)(d.gRT - (double)d.gRT_hi);
    }
    const double tau = 3.0 * p.nu + 0.5;
    d.beta = 1.0 / (2.0 * tau);
    d.inv_beta = 2.0 * tau;
    d.c_gb = 2.0 * d.beta - 1.0;
    d.c_gb_hi = (float)d.c_gb;
    d.c_gb_lo = (float)(d.c_gb - (double)d.c_gb_hi);
    d.Gamma = p.Gamma;
    d.inv_tau_g = 1.0 / p.tau_g;
    d.rho_ref = p.precision == TEL_FP32_SHIFTED ? (p.rho_ref > 0 ? p.rho_ref : co[0]) : 0.0;
    d.gamma_mode = p.gamma_mode;
    d.wet_rho = p.wet_rho;
    d.wet_phi = p.wet_phi;
    d.solid = nullptr;  // the device copy is set by tel_create
    fill_coef(d, d.cf);
    fill_coef(d, d.cd);
}

extern "C" int tel_create(int lattice, int nx, int ny, int nz, const tel_params *params, tel_ctx **out)
{
    if (!out) return fail(nullptr, TEL_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(lattice, nx, ny, nz, params);
    if (rc) return rc;
    double co[4];
    if (tel_coexistence_eos(params->eos, params->a, params->b, params->R, params->T, params->omega, co) != TEL_OK)
        return fail(nullptr, TEL_EINVAL, "no liquid-gas coexistence at T=%g (T must be below the critical temperature)",
                    params->T);
    tel_ctx *c = new (std::nothrow) tel_ctx();
    if (!c) return fail(nullptr, TEL_ENOMEM, "host allocation failed");
    std::memset(c, 0, sizeof(*c));
    c->lattice = lattice;
    c->D = lattice == TEL_D2Q9 ? 2 : 3;
    c->Q = lattice == TEL_D2Q9 ? 9 : 27;
    c->nx = nx; c->ny = ny; c->nz = lattice == TEL_D2Q9 ? 1 : nz;
    c->N = (long long)nx * ny * c->nz;
    c->p = *params;
    if (lattice == TEL_D2Q9) c->p.bc[2] = TEL_PERIODIC;

    tel::DevParams &d = c->dp;
    const tel_params &p = c->p;
    fill_devparams(lattice, nx, ny, nz, p, co, d);
    c->p.rho_ref = d.rho_ref;
    if (lattice == TEL_D2Q9 && !std::getenv("TEL_CHUNK")) {
        // rows per CTA: the fewest (at least 2, at most 16) with which one
        // wave of the step kernel's resident CTAs covers the lattice.  Rows
        // of 64 march along y, so a small lattice has few CTAs unless their
        // columns are short: 512^2 FP32 measured 9827 MLUPS with 8 rows
        // (a third of the resident slots), 11605 with 4 and 12750 with 3;
        // 2048^2 18520 with 32, 19385 with 16 and 18725 with 8.
        const bool fast = !p.bc[0] && !p.bc[1] && !params->solid && 9LL * c->N < (1LL << 31);
        const bool vec = fast && p.precision == TEL_FP32_SHIFTED && nx % 4 == 0;
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            tel::d2q9_step_ctas_per_sm(p.precision, fast, vec, &per_sm) == cudaSuccess && sms > 0 && per_sm > 0) {
            const long long slots = (long long)sms * per_sm, tiles = (nx + 63) / 64;
            long long ch = ((long long)ny * tiles + slots - 1) / slots;
            d.chunk = (int)(ch < 2 ? 2 : (ch > 16 ? 16 : ch));
        } else {
            cudaGetLastError();  // keep the default chunk
        }
    }

    const size_t es = p.precision == TEL_FP64 ? sizeof(double) : sizeof(float);
    const size_t bytes = es * (size_t)c->Q * (size_t)c->N;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&c->f[k], bytes);
        if (e == cudaSuccess) e = cudaMalloc(&c->g[k], bytes);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_gfall, sizeof(unsigned long long));
    if (e == cudaSuccess && params->solid) {
        e = cudaMalloc(&c->d_solid, (size_t)c->N);
        unsigned char *h = e == cudaSuccess ? new (std::nothrow) unsigned char[(size_t)c->N] : nullptr;
        if (e == cudaSuccess && !h) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) {
            for (long long n = 0; n < c->N; ++n) h[n] = params->solid[n] ? 1 : 0;
            e = cudaMemcpy(c->d_solid, h, (size_t)c->N, cudaMemcpyHostToDevice);
        }
        delete[] h;
    }
    // carried moments: D3Q27 FP32, periodic, no solid node, full tiles of
    // rows of 32, 32-bit population indices (the step kernel's fast path)
    const bool carried = p.moments == TEL_MOMENTS_CARRIED && lattice == TEL_D3Q27 && p.precision == TEL_FP32_SHIFTED &&
                         !p.bc[0] && !p.bc[1] && !p.bc[2] && !params->solid && nx % 32 == 0 &&
                         ny % tel::d3q27_carried_tile_y() == 0 && 27LL * c->N < (1LL << 31);
    for (int k = 0; k < 3 && carried && e == cudaSuccess; ++k) e = cudaMalloc(&c->mom[k], 2 * sizeof(float) * (size_t)c->N);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->own_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_gfall, 0, sizeof(unsigned long long), c->own_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->own_stream);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        tel_destroy(c);
        return fail(nullptr, oom ? TEL_ENOMEM : TEL_ECUDA, "device setup failed: %s", cudaGetErrorString(e));
    }
    c->stream = c->own_stream;
    d.err = c->d_err;
    d.gfall = c->d_gfall;
    d.solid = c->d_solid;
    c->p.solid = nullptr;  // the host mask is not retained
    *out = c;
    return TEL_OK;
}

extern "C" void tel_destroy(tel_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int k = 0; k < 2; ++k) {
        if (c->f[k]) cudaFree(c->f[k]);
        if (c->g[k]) cudaFree(c->g[k]);
    }
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_gfall) cudaFree(c->d_gfall);
    if (c->d_solid) cudaFree(c->d_solid);
    for (int k = 0; k < 3; ++k)
        if (c->mom[k]) cudaFree(c->mom[k]);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->scratch) cudaFree(c->scratch);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

extern "C" const char *tel_last_error(const tel_ctx *c) { return c ? c->msg : g_create_msg; }

extern "C" int tel_set_stream(tel_ctx *c, void *s)
{
    if (!c) return TEL_EINVAL;
    c->stream = s ? (cudaStream_t)s : c->own_stream;
    return TEL_OK;
}

extern "C" int tel_info(const tel_ctx *c, double out[10])
{
    if (!c || !out) return TEL_EINVAL;
    out[0] = c->D; out[1] = c->Q; out[2] = c->nx; out[3] = c->ny; out[4] = c->nz;
    out[5] = (double)c->N; out[6] = c->dp.rho_g; out[7] = c->dp.rho_l; out[8] = c->dp.mu_coex; out[9] = c->dp.p_coex;
    return TEL_OK;
}

static cudaError_t launch(tel_ctx *c, int mode, const tel::LaunchArgs &A)
{
    if (c->lattice == TEL_D2Q9) return tel::launch_d2q9(c->p.precision, mode, c->dp, A, c->stream);
    return tel::launch_d3q27(c->p.precision, mode, c->dp, A, c->stream);
}

static int ensure_scratch(tel_ctx *c, size_t elems)
{
    if (c->scratch_elems >= elems) return TEL_OK;
    if (c->scratch) {
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_elems = 0;
    }
    cudaError_t e = cudaMalloc(&c->scratch, elems * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, TEL_ENOMEM, "scratch allocation of %zu doubles failed: %s", elems, cudaGetErrorString(e));
    }
    c->scratch_elems = elems;
    return TEL_OK;
}

static int check_flag(tel_ctx *c)
{
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    const unsigned f = *c->h_err;
    if (f) {
        CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
        return fail(c, TEL_EUNSTABLE, "unstable node(s) flagged on the device:%s%s%s",
                    (f & tel::ERR_RHO) ? " non-positive density;" : "",
                    (f & tel::ERR_VEL) ? " |u| or |u+F/rho| >= 1;" : "",
                    (f & tel::ERR_NAN) ? " non-finite value;" : "");
    }
    return TEL_OK;
}

extern "C" int tel_init_device(tel_ctx *c, const double *rho, const double *phi, const double *u)
{
    if (!c) return TEL_EINVAL;
    if (!rho || !phi || !u) return fail(c, TEL_EINVAL, "tel_init: rho, phi and u are required");
    tel::LaunchArgs A{};
    A.in_rho = rho; A.in_phi = phi; A.in_u = u;
    A.fdst = c->f[c->cur]; A.gdst = c->g[c->cur];
    c->mom_valid = 0;
    CUDA_OR_FAIL(c, launch(c, tel::MODE_INIT, A));
    c->initialized = 1;
    return TEL_OK;
}

extern "C" int tel_init(tel_ctx *c, const double *rho, const double *phi, const double *u)
{
    if (!c) return TEL_EINVAL;
    if (!rho || !phi || !u) return fail(c, TEL_EINVAL, "tel_init: rho, phi and u are required");
    const size_t N = (size_t)c->N;
    int rc = ensure_scratch(c, (size_t)(2 + c->D) * N);
    if (rc) return rc;
    double *d = c->scratch;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(d, rho, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(d + N, phi, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(d + 2 * N, u, (size_t)c->D * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    rc = tel_init_device(c, d, d + N, d + 2 * N);
    if (rc) return rc;
    return check_flag(c);
}

extern "C" int tel_step(tel_ctx *c, int nsteps)
{
    if (!c) return TEL_EINVAL;
    if (nsteps < 0) return fail(c, TEL_EINVAL, "nsteps must be >= 0");
    if (!c->initialized) return fail(c, TEL_ESTATE, "tel_step before tel_init/tel_set_state");
    const bool carried = c->mom[0] != nullptr;
    if (carried && !c->mom_valid && nsteps > 0) {
        // moments of the new state into mom[r]; mom[r + 1] (the first step's
        // accumulator) cleared
        c->mom_r = 0;
        CUDA_OR_FAIL(c, tel::launch_d3q27_moments(c->dp, (const float *)c->f[c->cur], (const float *)c->g[c->cur],
                                                  c->mom[0], c->mom[1], c->stream));
        c->mom_valid = 1;
    }
    for (int s = 0; s < nsteps; ++s) {
        tel::LaunchArgs A{};
        A.fsrc = c->f[c->cur]; A.gsrc = c->g[c->cur];
        A.fdst = c->f[1 - c->cur]; A.gdst = c->g[1 - c->cur];
        if (carried) {
            A.m_read = c->mom[c->mom_r];
            A.m_acc = c->mom[(c->mom_r + 1) % 3];
            A.m_zero = c->mom[(c->mom_r + 2) % 3];
        }
        const int mode = c->p.gamma_mode == TEL_GAMMA_EXACT ? tel::MODE_STEP_EXACT
                         : (c->p.gamma_mode == TEL_GAMMA_CLOSED_F64SUM ? tel::MODE_STEP_G64 : tel::MODE_STEP);
        const cudaError_t e = launch(c, mode, A);
        if (e != cudaSuccess) {
            c->mom_valid = 0;
            return fail(c, TEL_ECUDA, "step launch: %s", cudaGetErrorString(e));
        }
        c->cur = 1 - c->cur;
        if (carried) c->mom_r = (c->mom_r + 1) % 3;
    }
    return TEL_OK;
}

extern "C" int tel_sync(tel_ctx *c)
{
    if (!c) return TEL_EINVAL;
    return check_flag(c);
}

extern "C" int tel_gamma_fallbacks(tel_ctx *c, unsigned long long *count)
{
    if (!c || !count) return c ? fail(c, TEL_EINVAL, "tel_gamma_fallbacks: NULL count") : TEL_EINVAL;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(count, c->d_gfall, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return TEL_OK;
}

extern "C" int tel_fields_device(tel_ctx *c, double *rho, double *phi, double *u, double *p)
{
    if (!c) return TEL_EINVAL;
    if (!c->initialized) return fail(c, TEL_ESTATE, "tel_fields before tel_init/tel_set_state");
    tel::LaunchArgs A{};
    A.fsrc = c->f[c->cur]; A.gsrc = c->g[c->cur];
    A.out_rho = rho; A.out_phi = phi; A.out_u = u; A.out_p = p;
    CUDA_OR_FAIL(c, launch(c, tel::MODE_FIELDS, A));
    return TEL_OK;
}

extern "C" int tel_fields(tel_ctx *c, double *rho, double *phi, double *u, double *p)
{
    if (!c) return TEL_EINVAL;
    if (!c->initialized) return fail(c, TEL_ESTATE, "tel_fields before tel_init/tel_set_state");
    const size_t N = (size_t)c->N;
    int rc = ensure_scratch(c, (size_t)(3 + c->D) * N);
    if (rc) return rc;
    double *d = c->scratch;
    rc = tel_fields_device(c, rho ? d : nullptr, phi ? d + N : nullptr, u ? d + 2 * N : nullptr,
                           p ? d + (2 + c->D) * N : nullptr);
    if (rc) return rc;
    if (rho) CUDA_OR_FAIL(c, cudaMemcpyAsync(rho, d, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (phi) CUDA_OR_FAIL(c, cudaMemcpyAsync(phi, d + N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (u) CUDA_OR_FAIL(c, cudaMemcpyAsync(u, d + 2 * N, (size_t)c->D * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (p) CUDA_OR_FAIL(c, cudaMemcpyAsync(p, d + (2 + c->D) * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return check_flag(c);
}

extern "C" int tel_get_state(tel_ctx *c, double *f, double *g)
{
    if (!c || !f || !g) return c ? fail(c, TEL_EINVAL, "tel_get_state: NULL array") : TEL_EINVAL;
    if (!c->initialized) return fail(c, TEL_ESTATE, "tel_get_state before tel_init/tel_set_state");
    const size_t QN = (size_t)c->Q * (size_t)c->N;
    if (c->p.precision == TEL_FP64) {
        CUDA_OR_FAIL(c, cudaMemcpyAsync(f, c->f[c->cur], QN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(g, c->g[c->cur], QN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    } else {
        int rc = ensure_scratch(c, QN);
        if (rc) return rc;
        CUDA_OR_FAIL(c, tel::launch_state_to_f64(c->lattice, (const float *)c->f[c->cur], c->scratch, c->N, c->dp.rho_ref, c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(f, c->scratch, QN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
        CUDA_OR_FAIL(c, tel::launch_state_to_f64(c->lattice, (const float *)c->g[c->cur], c->scratch, c->N, 0.0, c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(g, c->scratch, QN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    return check_flag(c);
}

extern "C" int tel_set_state(tel_ctx *c, const double *f, const double *g)
{
    if (!c || !f || !g) return c ? fail(c, TEL_EINVAL, "tel_set_state: NULL array") : TEL_EINVAL;
    const size_t QN = (size_t)c->Q * (size_t)c->N;
    if (c->p.precision == TEL_FP64) {
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->f[c->cur], f, QN * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->g[c->cur], g, QN * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    } else {
        int rc = ensure_scratch(c, QN);
        if (rc) return rc;
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->scratch, f, QN * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CUDA_OR_FAIL(c, tel::launch_state_from_f64(c->lattice, c->scratch, (float *)c->f[c->cur], c->N, c->dp.rho_ref, c->stream));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->scratch, g, QN * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CUDA_OR_FAIL(c, tel::launch_state_from_f64(c->lattice, c->scratch, (float *)c->g[c->cur], c->N, 0.0, c->stream));
    }
    c->mom_valid = 0;
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    c->initialized = 1;
    return TEL_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free field extraction.
//
// Some callers cannot let a library allocate device memory: applications
// that hand the whole device to their own memory pool up front, or that must
// keep their device footprint fixed after start-up, and code paths where
// cudaMalloc is not available to them.  tel_fields_noalloc serves them: the
// state lives in the caller's own device buffers, the results go to the
// caller's host buffers, and the only device memory used besides those is a
// fixed array of this file.
//
// tel_noalloc_scratch holds (3 + D) field arrays of up to
// TEL_NOALLOC_MAX_NODES nodes followed by the error word.  This translation
// unit has no kernels, so its module holds only this array; under CUDA's lazy
// module loading the module, and with it the array's device memory, is
// loaded on a device by the first call there (the first address lookup) and
// then kept until the process exits.  In host code the array's name is only a
// host-side stand-in: its device address is looked up with
// cudaGetSymbolAddress on every call, with the caller's device current, and
// passed to the kernel (so no address is kept across a device reset, which
// reloads the module, possibly elsewhere).  All calls share the array: the
// error word is cleared on every call, and calls that overlap on the GPU race
// with each other.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double tel_noalloc_scratch[6 * TEL_NOALLOC_MAX_NODES + 32];

namespace {
// failure of tel_fields_noalloc: the message goes to the calling thread's
// context-free error text (tel_last_error(NULL))
int noalloc_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::snprintf(g_create_msg, sizeof(g_create_msg), "%s", buf);
    return code;
}
}  // namespace

extern "C" int tel_fields_noalloc(int lattice, int nx, int ny, int nz, const tel_params *params,
                                  const void *f_state, const void *g_state, double *rho, double *phi,
                                  double *u, double *p, void *cuda_stream)
{
    int rc = validate(lattice, nx, ny, nz, params);
    if (rc) return noalloc_fail(rc, "%s", g_create_msg);
    const int D = lattice == TEL_D2Q9 ? 2 : 3;
    const long long N = (long long)nx * ny * (lattice == TEL_D2Q9 ? 1 : nz);
    if (N > TEL_NOALLOC_MAX_NODES)
        return noalloc_fail(TEL_EINVAL, "tel_fields_noalloc: %lld nodes exceed the fixed scratch of %d nodes",
                            N, TEL_NOALLOC_MAX_NODES);
    if (!f_state || !g_state) return noalloc_fail(TEL_EINVAL, "tel_fields_noalloc: NULL state buffer");
    if (params->solid) return noalloc_fail(TEL_EINVAL, "tel_fields_noalloc: solid masks need a context (tel_create)");
    double co[4];
    if (tel_coexistence_eos(params->eos, params->a, params->b, params->R, params->T, params->omega, co) != TEL_OK)
        return noalloc_fail(TEL_EINVAL, "no liquid-gas coexistence at T=%g", params->T);
    tel_params pp = *params;
    if (lattice == TEL_D2Q9) pp.bc[2] = TEL_PERIODIC;

    // device address of the fixed array on the current device (the first
    // lookup on a device loads the array there)
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, tel_noalloc_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(TEL_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    }
    double *scratch = static_cast<double *>(ptr);
    tel::DevParams d{};
    fill_devparams(lattice, nx, ny, nz, pp, co, d);
    unsigned *err = reinterpret_cast<unsigned *>(scratch + 6 * (size_t)TEL_NOALLOC_MAX_NODES);
    d.err = err;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t n = (size_t)N;
    double *o_rho = scratch, *o_phi = scratch + n, *o_u = scratch + 2 * n, *o_p = scratch + (2 + D) * n;
    tel::LaunchArgs A{};
    A.fsrc = f_state; A.gsrc = g_state;
    A.out_rho = rho ? o_rho : nullptr; A.out_phi = phi ? o_phi : nullptr;
    A.out_u = u ? o_u : nullptr; A.out_p = p ? o_p : nullptr;
#define NOALLOC_CUDA(expr)                                                                       \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) return noalloc_fail(TEL_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)
    NOALLOC_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    NOALLOC_CUDA(lattice == TEL_D2Q9 ? tel::launch_d2q9(pp.precision, tel::MODE_FIELDS, d, A, s)
                                     : tel::launch_d3q27(pp.precision, tel::MODE_FIELDS, d, A, s));
    if (rho) NOALLOC_CUDA(cudaMemcpyAsync(rho, o_rho, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (phi) NOALLOC_CUDA(cudaMemcpyAsync(phi, o_phi, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (u) NOALLOC_CUDA(cudaMemcpyAsync(u, o_u, (size_t)D * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (p) NOALLOC_CUDA(cudaMemcpyAsync(p, o_p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    unsigned flag = 0;
    NOALLOC_CUDA(cudaMemcpyAsync(&flag, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    NOALLOC_CUDA(cudaStreamSynchronize(s));
#undef NOALLOC_CUDA
    if (flag) return noalloc_fail(TEL_EUNSTABLE, "unstable node(s) flagged on the device (bits 0x%x)", flag);
    return TEL_OK;
}

// ---------------------------------------------------------------------------
// Batched D2Q9 lattices: many independent cases advanced by one persistent
// kernel launch per step (see batch_kernel), with an autotuned tile width and
// chunk length, and CUDA-graph replay of pairs of steps.
// ---------------------------------------------------------------------------
struct tel_batch {
    int ncases, precision;
    bool fast;
    bool vec;                    // vector phase A: FP32, fast, every nx % 4 == 0
    int *nx, *ny;
    long long *off;              // element offset of each case's arrays in one buffer
    long long total;             // total nodes
    tel::DevParams *hP;          // host copies (chunk set by the tuner)
    tel::DevParams *dP;          // device parameter blocks
    tel::LaunchArgs *dA[2];      // device launch arguments: src = buffer k, dst = buffer 1-k
    void *f[2], *g[2];
    unsigned *d_err;             // one error word per case
    int4 *d_items;
    int nitems, grid, tx, chunk;
    int cur;
    double *scratch;             // fields staging (largest case)
    size_t scratch_elems;
    cudaStream_t stream, own_stream;
    cudaGraphExec_t graph[2];    // two steps starting from buffer 0 / 1
    int initialized;
    char msg[512];
};

static int bfail(tel_batch *b, int code, const char *fmt, ...)
{
    char *dst = b ? b->msg : g_create_msg;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define BCUDA(b, expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) return bfail((b), TEL_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

static void batch_free_graphs(tel_batch *b)
{
    for (int k = 0; k < 2; ++k)
        if (b->graph[k]) { cudaGraphExecDestroy(b->graph[k]); b->graph[k] = nullptr; }
}

// Work list for tile width tx and chunk length ch: every (case, tile, chunk),
// largest cases first so that the tail of the persistent loop is short.
static int batch_build(tel_batch *b, int tx, int ch)
{
    int n = 0;
    for (int c = 0; c < b->ncases; ++c) n += ((b->nx[c] + tx - 1) / tx) * ((b->ny[c] + ch - 1) / ch);
    int4 *h = new (std::nothrow) int4[n];
    int *order = new (std::nothrow) int[b->ncases];
    if (!h || !order) { delete[] h; delete[] order; return bfail(b, TEL_ENOMEM, "host allocation failed"); }
    for (int c = 0; c < b->ncases; ++c) order[c] = c;
    for (int i = 1; i < b->ncases; ++i)  // insertion sort by node count, descending
        for (int j = i; j > 0 && (long long)b->nx[order[j]] * b->ny[order[j]] >
                                     (long long)b->nx[order[j - 1]] * b->ny[order[j - 1]]; --j) {
            const int t = order[j]; order[j] = order[j - 1]; order[j - 1] = t;
        }
    int k = 0;
    for (int oi = 0; oi < b->ncases; ++oi) {
        const int c = order[oi];
        const int tiles = (b->nx[c] + tx - 1) / tx, chunks = (b->ny[c] + ch - 1) / ch;
        for (int bm = 0; bm < chunks; ++bm)
            for (int bx = 0; bx < tiles; ++bx) h[k++] = make_int4(c, bx, bm, 0);
    }
    delete[] order;
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(int4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_items, h, sizeof(int4) * (size_t)n, cudaMemcpyHostToDevice);
    delete[] h;
    if (e != cudaSuccess) return bfail(b, TEL_ECUDA, "work list upload: %s", cudaGetErrorString(e));
    for (int c = 0; c < b->ncases; ++c) b->hP[c].chunk = ch;
    BCUDA(b, cudaMemcpy(b->dP, b->hP, sizeof(tel::DevParams) * (size_t)b->ncases, cudaMemcpyHostToDevice));
    int nb = tel::batch_blocks_per_sm(b->precision, tx, b->fast, b->vec);
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b->grid = nb * nsm < n ? nb * nsm : n;
    b->nitems = n;
    b->tx = tx;
    b->chunk = ch;
    batch_free_graphs(b);
    return TEL_OK;
}

extern "C" int tel_batch_create(int ncases, const int *nx, const int *ny, const tel_params *params, tel_batch **out)
{
    if (!out) return bfail(nullptr, TEL_EINVAL, "out is NULL");
    *out = nullptr;
    if (ncases < 1 || !nx || !ny || !params) return bfail(nullptr, TEL_EINVAL, "bad batch arguments");
    const int prec = params[0].precision;
    bool walls = false;
    long long total = 0;
    for (int c = 0; c < ncases; ++c) {
        int rc = validate(TEL_D2Q9, nx[c], ny[c], 1, &params[c]);
        if (rc) return bfail(nullptr, rc, "case %d: %s", c, g_create_msg);
        if (params[c].precision != prec) return bfail(nullptr, TEL_EINVAL, "all cases must share one precision");
        if (params[c].gamma_mode != TEL_GAMMA_CLOSED)
            return bfail(nullptr, TEL_EINVAL, "case %d: batches use the closed-form stabiliser (gamma_mode 0)", c);
        if (params[c].solid)
            return bfail(nullptr, TEL_EINVAL, "case %d: batches take no solid mask (walls only)", c);
        walls = walls || params[c].bc[0] || params[c].bc[1];
        total += (long long)nx[c] * ny[c];
    }
    tel_batch *b = new (std::nothrow) tel_batch();
    if (!b) return bfail(nullptr, TEL_ENOMEM, "host allocation failed");
    std::memset(b, 0, sizeof(*b));
    b->ncases = ncases;
    b->precision = prec;
    b->total = total;
    b->fast = !walls && 9LL * total < (1LL << 31);
    // vector phase A: every case's row a whole number of aligned four-node
    // vectors, so that each case's arrays (offsets sums of nx * ny) stay
    // 16-byte aligned
    b->vec = b->fast && prec == TEL_FP32_SHIFTED;
    for (int c = 0; c < ncases; ++c) b->vec = b->vec && nx[c] % 4 == 0;
    b->nx = new (std::nothrow) int[ncases];
    b->ny = new (std::nothrow) int[ncases];
    b->off = new (std::nothrow) long long[ncases];
    b->hP = new (std::nothrow) tel::DevParams[ncases];
    if (!b->nx || !b->ny || !b->off || !b->hP) { tel_batch_destroy(b); return bfail(nullptr, TEL_ENOMEM, "host allocation failed"); }
    const size_t es = prec == TEL_FP64 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&b->f[k], es * 9 * (size_t)total);
        if (e == cudaSuccess) e = cudaMalloc(&b->g[k], es * 9 * (size_t)total);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(unsigned) * (size_t)ncases);
    if (e == cudaSuccess) e = cudaMalloc(&b->dP, sizeof(tel::DevParams) * (size_t)ncases);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&b->dA[k], sizeof(tel::LaunchArgs) * (size_t)ncases);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
    b->stream = b->own_stream;
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(unsigned) * (size_t)ncases);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        tel_batch_destroy(b);
        return bfail(nullptr, oom ? TEL_ENOMEM : TEL_ECUDA, "batch device setup: %s", cudaGetErrorString(e));
    }
    long long o = 0;
    tel::LaunchArgs *hA[2];
    hA[0] = new (std::nothrow) tel::LaunchArgs[ncases];
    hA[1] = new (std::nothrow) tel::LaunchArgs[ncases];
    if (!hA[0] || !hA[1]) { delete[] hA[0]; delete[] hA[1]; tel_batch_destroy(b); return bfail(nullptr, TEL_ENOMEM, "host allocation failed"); }
    for (int c = 0; c < ncases; ++c) {
        b->nx[c] = nx[c];
        b->ny[c] = ny[c];
        b->off[c] = o;
        double co[4];
        if (tel_coexistence_eos(params[c].eos, params[c].a, params[c].b, params[c].R, params[c].T, params[c].omega,
                                co) != TEL_OK) {
            delete[] hA[0]; delete[] hA[1]; tel_batch_destroy(b);
            return bfail(nullptr, TEL_EINVAL, "case %d: no liquid-gas coexistence at T=%g", c, params[c].T);
        }
        tel_params pp = params[c];
        pp.bc[2] = TEL_PERIODIC;
        fill_devparams(TEL_D2Q9, nx[c], ny[c], 1, pp, co, b->hP[c]);
        b->hP[c].err = b->d_err + c;
        const size_t base = es * 9 * (size_t)o;
        for (int k = 0; k < 2; ++k) {
            tel::LaunchArgs A{};
            A.fsrc = (char *)b->f[k] + base; A.gsrc = (char *)b->g[k] + base;
            A.fdst = (char *)b->f[1 - k] + base; A.gdst = (char *)b->g[1 - k] + base;
            hA[k][c] = A;
        }
        o += (long long)nx[c] * ny[c];
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = cudaMemcpy(b->dA[k], hA[k], sizeof(tel::LaunchArgs) * (size_t)ncases, cudaMemcpyHostToDevice);
    delete[] hA[0];
    delete[] hA[1];
    if (e != cudaSuccess) { tel_batch_destroy(b); return bfail(nullptr, TEL_ECUDA, "batch upload: %s", cudaGetErrorString(e)); }
    int rc = batch_build(b, 64, 16);
    if (rc) { std::snprintf(g_create_msg, sizeof(g_create_msg), "%s", b->msg); tel_batch_destroy(b); return rc; }
    *out = b;
    return TEL_OK;
}

extern "C" void tel_batch_destroy(tel_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free_graphs(b);
    for (int k = 0; k < 2; ++k) {
        if (b->f[k]) cudaFree(b->f[k]);
        if (b->g[k]) cudaFree(b->g[k]);
        if (b->dA[k]) cudaFree(b->dA[k]);
    }
    if (b->d_err) cudaFree(b->d_err);
    if (b->dP) cudaFree(b->dP);
    if (b->d_items) cudaFree(b->d_items);
    if (b->scratch) cudaFree(b->scratch);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete[] b->nx; delete[] b->ny; delete[] b->off; delete[] b->hP;
    delete b;
}

extern "C" const char *tel_batch_last_error(const tel_batch *b) { return b ? b->msg : g_create_msg; }

extern "C" int tel_batch_set_stream(tel_batch *b, void *s)
{
    if (!b) return TEL_EINVAL;
    b->stream = s ? (cudaStream_t)s : b->own_stream;
    return TEL_OK;
}

static tel::LaunchArgs batch_case_args(const tel_batch *b, int c, int k)
{
    const size_t es = b->precision == TEL_FP64 ? sizeof(double) : sizeof(float);
    const size_t base = es * 9 * (size_t)b->off[c];
    tel::LaunchArgs A{};
    A.fsrc = (char *)b->f[k] + base; A.gsrc = (char *)b->g[k] + base;
    A.fdst = (char *)b->f[1 - k] + base; A.gdst = (char *)b->g[1 - k] + base;
    return A;
}

static int batch_scratch(tel_batch *b, size_t elems)
{
    if (b->scratch_elems >= elems) return TEL_OK;
    if (b->scratch) { BCUDA(b, cudaStreamSynchronize(b->stream)); cudaFree(b->scratch); b->scratch = nullptr; }
    cudaError_t e = cudaMalloc(&b->scratch, elems * sizeof(double));
    if (e != cudaSuccess) { cudaGetLastError(); return bfail(b, TEL_ENOMEM, "scratch: %s", cudaGetErrorString(e)); }
    b->scratch_elems = elems;
    return TEL_OK;
}

extern "C" int tel_batch_init_device(tel_batch *b, int c, const double *rho, const double *phi, const double *u)
{
    if (!b) return TEL_EINVAL;
    if (c < 0 || c >= b->ncases || !rho || !phi || !u)
        return bfail(b, TEL_EINVAL, "tel_batch_init_device: bad case or NULL field");
    tel::LaunchArgs A = batch_case_args(b, c, 1 - b->cur);  // writes the buffer the next step reads
    A.in_rho = rho; A.in_phi = phi; A.in_u = u;
    A.fsrc = A.gsrc = nullptr;
    BCUDA(b, tel::launch_d2q9(b->precision, tel::MODE_INIT, b->hP[c], A, b->stream));
    b->initialized = 1;
    return TEL_OK;
}

extern "C" int tel_batch_init(tel_batch *b, int c, const double *rho, const double *phi, const double *u)
{
    if (!b) return TEL_EINVAL;
    if (c < 0 || c >= b->ncases || !rho || !phi || !u) return bfail(b, TEL_EINVAL, "tel_batch_init: bad case or NULL field");
    const size_t N = (size_t)b->nx[c] * b->ny[c];
    int rc = batch_scratch(b, 4 * N);
    if (rc) return rc;
    double *d = b->scratch;
    BCUDA(b, cudaMemcpyAsync(d, rho, N * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BCUDA(b, cudaMemcpyAsync(d + N, phi, N * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BCUDA(b, cudaMemcpyAsync(d + 2 * N, u, 2 * N * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    tel::LaunchArgs A = batch_case_args(b, c, 1 - b->cur);  // writes the buffer the next step reads
    A.in_rho = d; A.in_phi = d + N; A.in_u = d + 2 * N;
    A.fsrc = A.gsrc = nullptr;
    BCUDA(b, tel::launch_d2q9(b->precision, tel::MODE_INIT, b->hP[c], A, b->stream));
    b->initialized = 1;
    return tel_batch_sync(b);
}

static int batch_launch(tel_batch *b, int k)
{
    BCUDA(b, tel::launch_d2q9_batch(b->precision, b->tx, b->fast, b->vec, b->dP, b->dA[k], b->d_items, b->nitems, b->grid,
                                    b->stream));
    return TEL_OK;
}

extern "C" int tel_batch_step(tel_batch *b, int nsteps)
{
    if (!b) return TEL_EINVAL;
    if (nsteps < 0) return bfail(b, TEL_EINVAL, "nsteps must be >= 0");
    if (!b->initialized) return bfail(b, TEL_ESTATE, "tel_batch_step before tel_batch_init");
    int s = 0;
    if (nsteps >= 2) {
        // two steps (cur -> 1-cur -> cur) as one captured graph, replayed
        const int k = b->cur;
        if (!b->graph[k]) {
            int rc = batch_launch(b, k);  // first launch outside capture (kernel attributes)
            if (rc) return rc;
            rc = batch_launch(b, 1 - k);
            if (rc) return rc;
            s = 2;
            cudaGraph_t gr;
            BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            int r1 = batch_launch(b, k), r2 = r1 ? r1 : batch_launch(b, 1 - k);
            cudaError_t ec = cudaStreamEndCapture(b->stream, &gr);
            if (r1 || r2) return r1 ? r1 : r2;
            if (ec != cudaSuccess) return bfail(b, TEL_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
            cudaError_t ei = cudaGraphInstantiate(&b->graph[k], gr, 0);
            cudaGraphDestroy(gr);
            if (ei != cudaSuccess) return bfail(b, TEL_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        }
        for (; s + 2 <= nsteps; s += 2) BCUDA(b, cudaGraphLaunch(b->graph[k], b->stream));
    }
    for (; s < nsteps; ++s) {
        int rc = batch_launch(b, b->cur);
        if (rc) return rc;
        b->cur = 1 - b->cur;
    }
    return TEL_OK;
}

extern "C" int tel_batch_sync(tel_batch *b)
{
    if (!b) return TEL_EINVAL;
    BCUDA(b, cudaStreamSynchronize(b->stream));
    unsigned *h = new (std::nothrow) unsigned[b->ncases];
    if (!h) return bfail(b, TEL_ENOMEM, "host allocation failed");
    cudaError_t e = cudaMemcpy(h, b->d_err, sizeof(unsigned) * (size_t)b->ncases, cudaMemcpyDeviceToHost);
    int bad = -1;
    for (int c = 0; c < b->ncases && e == cudaSuccess; ++c)
        if (h[c]) { bad = c; break; }
    delete[] h;
    if (e != cudaSuccess) return bfail(b, TEL_ECUDA, "error words: %s", cudaGetErrorString(e));
    if (bad >= 0) {
        cudaMemset(b->d_err, 0, sizeof(unsigned) * (size_t)b->ncases);
        return bfail(b, TEL_EUNSTABLE, "case %d flagged an unstable node", bad);
    }
    return TEL_OK;
}

extern "C" int tel_batch_fields(tel_batch *b, int c, double *rho, double *phi, double *u, double *p)
{
    if (!b) return TEL_EINVAL;
    if (c < 0 || c >= b->ncases) return bfail(b, TEL_EINVAL, "tel_batch_fields: bad case");
    if (!b->initialized) return bfail(b, TEL_ESTATE, "tel_batch_fields before tel_batch_init");
    const size_t N = (size_t)b->nx[c] * b->ny[c];
    int rc = batch_scratch(b, 5 * N);
    if (rc) return rc;
    double *d = b->scratch;
    tel::LaunchArgs A = batch_case_args(b, c, b->cur);
    A.fdst = A.gdst = nullptr;
    A.out_rho = rho ? d : nullptr; A.out_phi = phi ? d + N : nullptr;
    A.out_u = u ? d + 2 * N : nullptr; A.out_p = p ? d + 4 * N : nullptr;
    BCUDA(b, tel::launch_d2q9(b->precision, tel::MODE_FIELDS, b->hP[c], A, b->stream));
    if (rho) BCUDA(b, cudaMemcpyAsync(rho, d, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (phi) BCUDA(b, cudaMemcpyAsync(phi, d + N, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (u) BCUDA(b, cudaMemcpyAsync(u, d + 2 * N, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (p) BCUDA(b, cudaMemcpyAsync(p, d + 4 * N, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    return tel_batch_sync(b);
}

extern "C" int tel_batch_fields_device(tel_batch *b, int c, double *rho, double *phi, double *u, double *p)
{
    if (!b) return TEL_EINVAL;
    if (c < 0 || c >= b->ncases) return bfail(b, TEL_EINVAL, "tel_batch_fields_device: bad case");
    if (!b->initialized) return bfail(b, TEL_ESTATE, "tel_batch_fields_device before tel_batch_init");
    tel::LaunchArgs A = batch_case_args(b, c, b->cur);
    A.fdst = A.gdst = nullptr;
    A.out_rho = rho; A.out_phi = phi; A.out_u = u; A.out_p = p;
    BCUDA(b, tel::launch_d2q9(b->precision, tel::MODE_FIELDS, b->hP[c], A, b->stream));
    return TEL_OK;
}

extern "C" int tel_batch_errors(tel_batch *b, unsigned *flags)
{
    if (!b || !flags) return TEL_EINVAL;
    BCUDA(b, cudaStreamSynchronize(b->stream));
    BCUDA(b, cudaMemcpy(flags, b->d_err, sizeof(unsigned) * (size_t)b->ncases, cudaMemcpyDeviceToHost));
    BCUDA(b, cudaMemset(b->d_err, 0, sizeof(unsigned) * (size_t)b->ncases));
    return TEL_OK;
}

extern "C" int tel_batch_tune(tel_batch *b, int steps_per_config, int out[3])
{
    if (!b) return TEL_EINVAL;
    if (steps_per_config < 1) return bfail(b, TEL_EINVAL, "steps_per_config must be >= 1");
    if (!b->initialized) return bfail(b, TEL_ESTATE, "tel_batch_tune before tel_batch_init");
    static const int txs[2] = {32, 64}, chs[4] = {8, 16, 32, 64};
    cudaEvent_t e0, e1;
    BCUDA(b, cudaEventCreate(&e0));
    BCUDA(b, cudaEventCreate(&e1));
    float best = 1e30f;
    int btx = 64, bch = 16, done = 0;
    for (int a = 0; a < 2; ++a)
        for (int q = 0; q < 4; ++q) {
            int rc = batch_build(b, txs[a], chs[q]);
            if (rc) return rc;
            rc = batch_launch(b, b->cur);  // warm-up (also a real step)
            if (rc) return rc;
            b->cur = 1 - b->cur;
            ++done;
            BCUDA(b, cudaEventRecord(e0, b->stream));
            for (int s = 0; s < steps_per_config; ++s) {
                rc = batch_launch(b, b->cur);
                if (rc) return rc;
                b->cur = 1 - b->cur;
                ++done;
            }
            BCUDA(b, cudaEventRecord(e1, b->stream));
            BCUDA(b, cudaEventSynchronize(e1));
            float ms = 0;
            BCUDA(b, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; btx = txs[a]; bch = chs[q]; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc = batch_build(b, btx, bch);
    if (rc) return rc;
    if (out) { out[0] = btx; out[1] = bch; out[2] = done; }
    return TEL_OK;
}

extern "C" int tel_batch_info(const tel_batch *b, double out[6])
{
    if (!b || !out) return TEL_EINVAL;
    out[0] = b->ncases; out[1] = (double)b->total; out[2] = b->tx; out[3] = b->chunk; out[4] = b->nitems; out[5] = b->grid;
    return TEL_OK;
}
