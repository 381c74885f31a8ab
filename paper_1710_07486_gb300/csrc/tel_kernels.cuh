// tel_kernels.cuh -- the fused per-timestep kernel of the ternary free-energy
// entropic lattice Boltzmann update (arXiv:1710.07486), D2Q9 and D3Q27,
// FP64 or FP32-shifted storage.
//
// One launch advances every node by one time step.  A CTA owns a tile of
// TX x TY nodes in the plane normal to the last axis (the "marching" axis: y
// for D2Q9, z for D3Q27) and marches along that axis through a chunk of
// planes.  Per plane it runs three phases, each in shared memory:
//   A  moments rho, phi of plane m+2 on the tile plus a ring of 2 nodes,
//      from populations pulled out of the source buffers;
//   B  chemical potentials mu_rho, mu_phi (Eqs. 1-5) of plane m+1 on the tile
//      plus a ring of 1 (isotropic Laplacians of the plane-m..m+2 moments),
//      and, for the lattice-consistent force, grad rho there;
//   C  for each node of plane m: the force, the KBC collision with per-node
//      stabiliser and exact-difference forcing of f, the BGK collision of g,
//      and the store of the post-collision populations to the destination
//      buffers (pull streaming: the next step reads them at x + c_i).
// So every population is read from HBM once (the ring pulls of phase A and
// the second pull of phase C are served by L1/L2) and written once.
//
// The same template also initialises the state from fields (MODE_INIT) and
// extracts the fields of the state (MODE_FIELDS).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tel {

// MODE_STEP_EXACT: the step with the exact per-node stabiliser (root of the
// entropy condition) instead of its closed form.  MODE_STEP_G64: the closed
// form with its two scalar products accumulated in FP64 (FP32 storage).
enum Mode { MODE_STEP = 0, MODE_INIT = 1, MODE_FIELDS = 2, MODE_STEP_EXACT = 3, MODE_STEP_G64 = 4 };

// Equations of state (values of tel_eos): Carnahan-Starling (Eq. 4), and the
// textbook van der Waals and Peng-Robinson forms named as alternatives.
enum Eos : int { EOS_CS = 0, EOS_VDW = 1, EOS_PR = 2 };

// Error bits raised by the device (see TEL_EUNSTABLE).
enum : unsigned { ERR_RHO = 1u, ERR_VEL = 2u, ERR_NAN = 4u };

// Raise error bits in the device error word.  The word is read first and the
// atomic skipped when the bits are already set: when a whole lattice goes
// bad every node would otherwise queue an atomic on the same address.
__device__ __forceinline__ void raise_err(unsigned *err, unsigned bits)
{
    if ((*reinterpret_cast<volatile unsigned *>(err) & bits) != bits) atomicOr(err, bits);
}

// Model coefficients in the compute precision (float copies for the FP32
// path so that no double-to-float conversion runs on the slow FP64 pipe).
template <typename T>
struct Coef {
    T b, a2, RT8, RT, mu_coex, lam1h;  // a2 = -2a, RT8 = 8RT
    T rho_l, inv_Dl, inv_chi, lam2, lam3, inv_2Dl, inv_2chi;
    T Kr, Kp, Kx;
    T rho_switch, rho_ref;
    T beta, Gamma3, inv_tau_g;         // Gamma3 = 3 Gamma
    T aal, prA, c1, c2;                // PR: a alpha(T), a alpha/(2 sqrt2 b), (1 +- sqrt2) b
    T wr, wp;                          // wetting gradients of rho and phi at walls and solid nodes
};

struct DevParams {
    int nx, ny, nz;          // lattice extents (nz = 1 for D2Q9)
    int bc[3];               // 0 periodic, 1 bounce-back walls at both ends
    long long N;             // nodes
    int chunk;               // planes per CTA along the marching axis
    int force_form;          // 0 potential, 1 lattice-consistent
    int eos;                 // Eos
    // equation-of-state free energy (Eq. 4 or an alternative), shifted by the
    // common tangent
    double a, b, RT, mu_coex, p_coex;
    double aal, prA, c1, c2;          // Peng-Robinson constants at T (see Coef)
    double lam1h, lam2, lam3;         // lambda1/2, lambda2, lambda3
    double rho_g, rho_l;
    double inv_Dl;                    // 1/(rho_g - rho_l)
    double inv_chi;                   // 1/chi
    double inv_2Dl, inv_2chi;         // 1/(2 Delta), 1/(2 chi)
    double Kr, Kp, Kx;                // Laplacian weights of mu (Eq. 5)
    double AI, BI, XI;                // f_I = AI |grad rho|^2 + BI |grad phi|^2 + XI grad rho.grad phi
    double rho_switch;                // FP32 mode: gas side is rho < rho_switch
    double inv_rho_g;                 // 1/rho_g
    double gRT;                       // lambda1/2 times RT (gas-side chemical potential)
    // FP32 constants of the gas-side chemical potential (mu_eos_gas)
    float inv_rho_g_f;                // 1/rho_g
    float rg_hi, rg_lo;               // rho_g = rg_hi + rg_lo, two floats
    float b_f;                        // b
    float q_g, q_g2, q_g_x2;          // q = 1/(b rho_g - 4), q^2, 2q
    float gRT8b_f, ga2_f;             // lambda1/2 times 8 RT b and 2a
    float gRT_hi, gRT_lo;             // lambda1/2 times RT as two floats (hi + lo)
    // collision
    double beta, inv_beta;            // beta = 1/(2 tau)
    double c_gb;                      // 2 beta - 1: beta gamma = 1 - (2 beta - 1) <ds|dh>/<dh|dh>
    float c_gb_hi, c_gb_lo;           // 2 beta - 1 as two floats (hi + lo)
    double Gamma, inv_tau_g;
    double rho_ref;                   // FP32 shift (0 in FP64)
    int gamma_mode;                   // 0 closed-form stabiliser, 1 exact root
    double wet_rho, wet_phi;          // wetting gradients (0: neutral walls)
    const unsigned char *solid;       // per-node solid mask (device), or NULL
    unsigned *err;                    // device error word
    unsigned long long *gfall;        // count of exact-stabiliser fallbacks
    Coef<float> cf;
    Coef<double> cd;
};

template <typename T> __device__ __forceinline__ const Coef<T> &coef(const DevParams &P);
template <> __device__ __forceinline__ const Coef<float> &coef<float>(const DevParams &P) { return P.cf; }
template <> __device__ __forceinline__ const Coef<double> &coef<double>(const DevParams &P) { return P.cd; }

struct LaunchArgs {
    const void *fsrc, *gsrc;                  // populations (step, fields)
    void *fdst, *gdst;                        // populations (step, init)
    const double *in_rho, *in_phi, *in_u;     // init
    double *out_rho, *out_phi, *out_u, *out_p;// fields (nullable)
    // carried moments (step, D3Q27 FP32 periodic): m_read holds the moments
    // of this step's pull (rho - rho_ref for nodes 0..N-1, then phi), m_acc
    // (zero on entry) receives the next step's, m_zero is cleared for the
    // step after that
    const float *m_read;
    float *m_acc, *m_zero;
};

// ---------------------------------------------------------------------------
// Lattice: c_i = (i%3 - 1, (i/3)%3 - 1, i/9 - 1); D2Q9 uses the first two.
// The in-plane components are (X, Y) and the marching component is M:
//   D2Q9: X = c_x, Y = 0, M = c_y;  D3Q27: X = c_x, Y = c_y, M = c_z.
// ---------------------------------------------------------------------------
template <int D> struct Lat {
    static constexpr int Q = D == 2 ? 9 : 27;
    static constexpr int REST = D == 2 ? 4 : 13;
    __host__ __device__ static constexpr int cx(int i) { return i % 3 - 1; }
    __host__ __device__ static constexpr int cy(int i) { return (i / 3) % 3 - 1; }
    __host__ __device__ static constexpr int cz(int i) { return D == 2 ? 0 : i / 9 - 1; }
    __host__ __device__ static constexpr int c(int i, int a) { return a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i)); }
    __host__ __device__ static constexpr int pX(int i) { return cx(i); }
    __host__ __device__ static constexpr int pY(int i) { return D == 2 ? 0 : cy(i); }
    __host__ __device__ static constexpr int pM(int i) { return D == 2 ? cy(i) : cz(i); }
    __host__ __device__ static constexpr int nnz(int i) { return (cx(i) != 0) + (cy(i) != 0) + (cz(i) != 0); }
    // weights: D2Q9 {4/9, 1/9, 1/36}, D3Q27 {8/27, 2/27, 1/54, 1/216}
    __host__ __device__ static constexpr double w(int i)
    {
        return D == 2 ? (nnz(i) == 0 ? 4.0 / 9 : (nnz(i) == 1 ? 1.0 / 9 : 1.0 / 36))
                      : (nnz(i) == 0 ? 8.0 / 27 : (nnz(i) == 1 ? 2.0 / 27 : (nnz(i) == 2 ? 1.0 / 54 : 1.0 / 216)));
    }
};

// Ghost/ring coordinate map: periodic axes wrap; on a bounce-back axis the
// ghost beyond the half-way wall mirrors the fluid node (-1 -> 0, n -> n-1).
__device__ __forceinline__ int map_coord(int q, int n, int wall)
{
    if (q >= 0 && q < n) return q;
    if (!wall) {
        q %= n;
        return q < 0 ? q + n : q;
    }
    int p = 2 * n;
    q %= p;
    if (q < 0) q += p;
    return q < n ? q : p - 1 - q;
}

template <typename T> __device__ __forceinline__ T sqrt_(T x);
template <> __device__ __forceinline__ double sqrt_<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float sqrt_<float>(float x) { return sqrtf(x); }
// Pairs and quads of the compute type.  In FP32, pair arithmetic uses the
// packed FP32x2 instructions of sm_100+ (__ffma2_rn, __fadd2_rn).
template <typename T> struct Vec;
template <> struct Vec<float> {
    typedef float2 v2;
    typedef float4 v4;
    __device__ static __forceinline__ v2 pair(float a, float b) { return make_float2(a, b); }
    __device__ static __forceinline__ v2 fma(v2 a, v2 b, v2 c) { return __ffma2_rn(a, b, c); }
    __device__ static __forceinline__ v2 add(v2 a, v2 b) { return __fadd2_rn(a, b); }
    __device__ static __forceinline__ v2 sub(v2 a, v2 b);
    __device__ static __forceinline__ v4 quad(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
struct __align__(16) dquad { double x, y, z, w; };
template <> struct Vec<double> {
    typedef double2 v2;
    typedef dquad v4;
    __device__ static __forceinline__ v2 pair(double a, double b) { return make_double2(a, b); }
    __device__ static __forceinline__ v2 fma(v2 a, v2 b, v2 c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
    __device__ static __forceinline__ v2 add(v2 a, v2 b) { return make_double2(a.x + b.x, a.y + b.y); }
    __device__ static __forceinline__ v2 sub(v2 a, v2 b) { return make_double2(a.x - b.x, a.y - b.y); }
    __device__ static __forceinline__ v4 quad(double a, double b, double c, double d) { v4 q; q.x = a; q.y = b; q.z = c; q.w = d; return q; }
};

// Packed FP32x2 arithmetic (sm_100+): one instruction for two lanes.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
        "sub.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 Vec<float>::sub(float2 a, float2 b) { return sub2(a, b); }

// Asynchronous 4-byte copies global -> shared (sm_80+): the thread goes on
// while they are in flight and waits for its own before reading them.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename T> __device__ __forceinline__ T log_(T x);
template <> __device__ __forceinline__ double log_<double>(double x) { return log(x); }
template <> __device__ __forceinline__ float log_<float>(float x) { return logf(x); }

// Local (gradient-free) parts of the chemical potentials at (rho, phi):
//   mu_rho = lambda1/2 (dPsi~/drho - mu_coex) - (lambda2 w'(C1) + lambda3 w'(C2))/(2 Delta)
//   mu_phi = (lambda2 w'(C1) - lambda3 w'(C2))/(2 chi),  w'(C) = C (1-C)(1-2C)
// with dPsi~/drho = -2 a rho - 8RT (24 - 2 b rho)/(b rho - 4)^3 + RT (ln rho + 1).
// mu_eos is the first (equation-of-state) term, mu_wells the rest.
template <typename T>
__device__ __forceinline__ T mu_eos(const DevParams &P, T rho)
{
    const Coef<T> &K = coef<T>(P);
    if (P.eos != EOS_CS) {
        // dPsi~/drho = RT (ln(rho/(1 - b rho)) + 1/(1 - b rho)) - 2 a rho            (vdW)
        //            ... - a alpha/(2 sqrt2 b) ln((1 + c1 rho)/(1 + c2 rho))
        //                - a alpha rho/(1 + 2 b rho - b^2 rho^2)                     (PR)
        const T q = (T)1 - K.b * rho;
        T dpsi = K.RT * (log_<T>(rho / q) + (T)1 / q);
        if (P.eos == EOS_VDW)
            dpsi += K.a2 * rho;
        else
            dpsi -= K.prA * log_<T>(((T)1 + K.c1 * rho) / ((T)1 + K.c2 * rho))
                    + K.aal * rho / ((T)1 + (T)2 * K.b * rho - K.b * K.b * rho * rho);
        return K.lam1h * (dpsi - K.mu_coex);
    }
    const T br = K.b * rho;
    const T d = br - (T)4;
    const T dpsi = K.a2 * rho - K.RT8 * ((T)24 - (T)2 * br) / (d * d * d) + K.RT * (log_<T>(rho) + (T)1)
                   - K.mu_coex;
    return K.lam1h * dpsi;
}

template <typename T>
__device__ __forceinline__ void mu_wells(const DevParams &P, T rho, T phi, T &mr, T &mp)
{
    const Coef<T> &K = coef<T>(P);
    const T s = (rho - K.rho_l) * K.inv_Dl;
    const T pc = phi * K.inv_chi;
    const T c1 = (T)0.5 * ((T)1 + pc - s);
    const T c2 = (T)0.5 * ((T)1 - pc - s);
    const T w1 = c1 * ((T)1 - c1) * ((T)1 - (T)2 * c1);
    const T w2 = c2 * ((T)1 - c2) * ((T)1 - (T)2 * c2);
    mr = -(K.lam2 * w1 + K.lam3 * w2) * K.inv_2Dl;
    mp = (K.lam2 * w1 - K.lam3 * w2) * K.inv_2chi;
}

// FP32-storage mode, gas side (rho < rho_switch): the equation-of-state part
// of mu_rho from its difference to the gas coexistence point, where
// mu_coex = dPsi~/drho(rho_g):
//   dPsi~(rho) - dPsi~(rho_g) = RT ln(rho/rho_g) - 8RT (h(rho) - h(rho_g)) - 2a D,
//   D = rho - rho_g,  h(rho) = (24 - 2 b rho)/(b rho - 4)^3 = 16 r^3 - 2 r^2,
//   r = 1/(b rho - 4).
// Every piece is proportional to D and is evaluated without cancellation:
//  - D from rho_g split into two floats (near rho_g the first subtraction is
//    exact by Sterbenz's lemma);
//  - ln(rho/rho_g) = log1p(D/rho_g);
//  - with q = 1/(b rho_g - 4), r - q = -b D r q and
//    h(rho) - h(rho_g) = (r - q) [16 (r^2 + r q + q^2) - 2 (r + q)] = -b D B,
//    B = 2 r q [8 (r^2 + r q + q^2) - (r + q)], a sum of terms of one sign
//    (r, q < 0 for b rho < 4).
// So the result is (lambda1/2) [RT ln(rho/rho_g) + D (8RT b B - 2a)].  Its
// two products are added in double-float arithmetic: each product's rounding
// error recovered by an FMA, the sum's by Knuth's TwoSum, and everything
// rounded once to FP32 at the end -- the value of an FP64 sum rounded to FP32,
// to within one FP32 ulp, at the issue cost of a dozen FP32 operations (the
// FP64 pipe of this GPU runs at 1/64 of the FP32 rate).  The _rn intrinsics
// keep the compiler from contracting the products into the sums.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// 1/x from the approximate reciprocal and one Newton-Raphson step, r (2 - x r):
// within about one ulp.
__device__ __forceinline__ float rcp_nr(float x)
{
    const float r = rcp_approx(x);
    return fmaf(r, fmaf(-x, r, 1.f), r);
}
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <typename T> __device__ __forceinline__ T inv_(T x);
template <> __device__ __forceinline__ double inv_<double>(double x) { return 1.0 / x; }
template <> __device__ __forceinline__ float inv_<float>(float x) { return rcp_nr(x); }

__device__ __forceinline__ float mu_eos_gas(const DevParams &P, float rho)
{
    const float D = (rho - P.rg_hi) - P.rg_lo;
    const float L = log1pf(D * P.inv_rho_g_f);
    const float r = rcp_nr(fmaf(P.b_f, rho, -4.f));
    const float rq = r + P.q_g;
    const float B = (P.q_g_x2 * r) * fmaf(8.f, fmaf(r, rq, P.q_g2), -rq);
    const float c = fmaf(P.gRT8b_f, B, -P.ga2_f);
    const float p1 = __fmul_rn(P.gRT_hi, L);
    const float p2 = __fmul_rn(D, c);
    float e = fmaf(P.gRT_hi, L, -p1);
    e = fmaf(P.gRT_lo, L, e);
    e = __fadd_rn(e, fmaf(D, c, -p2));
    const float sum = __fadd_rn(p1, p2);
    const float bp = __fsub_rn(sum, p1);
    e = __fadd_rn(e, __fadd_rn(__fsub_rn(p1, __fsub_rn(sum, bp)), __fsub_rn(p2, bp)));
    return __fadd_rn(sum, e);
}

// Bulk free energy f_B of Eq. 2 (Psi_eos - Psi_0 with the common tangent).
__device__ __forceinline__ double f_bulk(const DevParams &P, double rho, double phi)
{
    double psi;
    if (P.eos == EOS_CS) {
        const double br = P.b * rho, d = br - 4.0;
        psi = rho * (-P.a * rho - 8.0 * P.RT * (br - 6.0) / (d * d) + P.RT * log(rho));
    } else {
        psi = rho * P.RT * log(rho / (1.0 - P.b * rho));
        if (P.eos == EOS_VDW)
            psi -= P.a * rho * rho;
        else
            psi -= P.prA * rho * log((1.0 + P.c1 * rho) / (1.0 + P.c2 * rho));
    }
    psi += -P.mu_coex * rho + P.p_coex;
    const double s = (rho - P.rho_l) * P.inv_Dl, pc = phi * P.inv_chi;
    const double c1 = 0.5 * (1.0 + pc - s), c2 = 0.5 * (1.0 - pc - s);
    return P.lam1h * psi + 0.5 * P.lam2 * c1 * c1 * (1 - c1) * (1 - c1)
           + 0.5 * P.lam3 * c2 * c2 * (1 - c2) * (1 - c2);
}

// One-dimensional factors of the entropic equilibrium, including the
// one-dimensional weight: e[c+1] for c = -1, 0, 1 with
//   e[1] = 2/3 (2 - S),  e[2] = 1/6 (2 - S)(S + 2u)/(1 - u),
//   e[0] = 1/6 (2 - S)(S - 2u)/(1 + u),  S = sqrt(1 + 3u^2),
// so that f^eq_i = rho prod_a e_a[c_ia + 1].
template <typename T>
__device__ __forceinline__ void eq_factors(T u, T e[3])
{
    const T S = sqrt_<T>((T)1 + (T)3 * u * u);
    const T t = (T)2 - S;
    e[1] = (T)(2.0 / 3.0) * t;
    e[2] = (T)(1.0 / 6.0) * t * (S + (T)2 * u) / ((T)1 - u);
    e[0] = (T)(1.0 / 6.0) * t * (S - (T)2 * u) / ((T)1 + u);
}

// FP32 form of eq_factors for the FP32-storage step: S from the approximate
// square root; 1/(1 - u) = (1 + u)/(1 - u^2) and 1/(1 + u) = (1 - u)/(1 - u^2)
// from one refined reciprocal.
__device__ __forceinline__ void eq_factors_f(float u, float e[3])
{
    const float S = sqrt_approx(fmaf(3.f * u, u, 1.f));
    const float t = 2.f - S;
    const float r = rcp_nr(fmaf(-u, u, 1.f)) * ((1.f / 6.f) * t);
    e[1] = (2.f / 3.f) * t;
    e[2] = (S + 2.f * u) * (1.f + u) * r;
    e[0] = (S - 2.f * u) * (1.f - u) * r;
}

// ---------------------------------------------------------------------------
// Exact stabiliser.  The KBC collision f' = f - beta (2 Delta s + gamma
// Delta h) fixes the relaxation of the stress part; gamma is the value that
// maximises the entropy of f' on this line, i.e. the root of
//   G = sum_i Delta h_i ln(f'_i / feq_i) = 0
// (the +1 of dH/dgamma and ln(feq_i/w_i), affine in c_i, drop because Delta h
// carries no mass or momentum).  In t = 1 - beta gamma,
// f'_i = feq_i + (1 - 2 beta) Delta s_i + t Delta h_i, G is strictly
// increasing on the interval where every f'_i > 0 and spans (-inf, inf)
// there, so the root is unique.  Newton from the closed form's t, kept in a
// bracket by bisection (also when a step next to a pole of ln f'_i stalls);
// at most GAMMA_MAX_ITER evaluations.  parts(i, feq, ds, dh) supplies the
// node's values of velocity i.  Returns 1 with t the root; 0 when Delta h has
// entries of one sign only, which a massless Delta h has only as rounding
// noise (the caller keeps the closed form); -1 when no t keeps every f'_i
// positive or the iteration does not converge (the caller keeps the closed
// form and counts a fallback).
// ---------------------------------------------------------------------------
constexpr int GAMMA_MAX_ITER = 20;
template <typename T> __device__ __forceinline__ T log1p_(T x);
template <> __device__ __forceinline__ double log1p_<double>(double x) { return log1p(x); }
template <> __device__ __forceinline__ float log1p_<float>(float x) { return log1pf(x); }

// FP32 ln(1 + x) for the exact stabiliser's fast path: the Taylor series to
// x^5 where |x| < 2^-6 (remainder below 2e-10 of x), log1pf elsewhere.
__device__ __forceinline__ float log1p_fast(float x)
{
    if (fabsf(x) < 0.015625f)
        return x * fmaf(-x, fmaf(-x, fmaf(-x, fmaf(-x, 0.2f, 0.25f), 1.f / 3.f), 0.5f), 1.f);
    return log1pf(x);
}

template <typename T, int Q, typename Parts>
__device__ __forceinline__ int gamma_root_bracketed(const Parts &parts, T beta, T &t, T tolG, T tolT);

// FP32: plain Newton from the closed form first (no bracket, approximate
// reciprocals, the short series for ln(1 + x)); near equilibrium it meets
// the bar in one or two evaluations.  If an iterate leaves the interval where
// every f'_i > 0, or does not settle in 4 evaluations, the bracketed solver
// below starts afresh.  FP64 takes the bracketed solver directly.
template <typename T, int Q, typename Parts>
__device__ __forceinline__ int gamma_root(const Parts &parts, T beta, T &t, T tolG, T tolT)
{
    if constexpr (sizeof(T) == sizeof(float)) {
        const float c = 1.f - 2.f * beta;
        float tt = t;
#pragma unroll 1
        for (int it = 0; it < 4; ++it) {
            float G = 0.f, dG = 0.f, S = 0.f;
            bool inside = true, pos = false, neg = false;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float fe, ds, dh;
                parts(i, fe, ds, dh);
                const float r = rcp_nr(fe);
                const float x = (c * ds + tt * dh) * r;
                inside = inside && x > -1.f;
                pos = pos || dh > 0.f;
                neg = neg || dh < 0.f;
                G = fmaf(dh, log1p_fast(x), G);
                S = fmaf(fabsf(dh), (fabsf(c * ds) + fabsf(tt * dh)) * r, S);
                dG = fmaf(dh * dh, r * rcp_nr(1.f + x), dG);
            }
            if (!pos || !neg) return 0;
            if (!inside) break;
            if (fabsf(G) <= tolG * S) { t = tt; return 1; }
            const float tn = tt - G / dG;
            if (fabsf(tn - tt) <= tolT * (1.f + fabsf(tt))) {
                if (fabsf(G) <= 1e3f * tolG * S) { t = tn; return 1; }
                break;
            }
            tt = tn;
        }
    }
    return gamma_root_bracketed<T, Q>(parts, beta, t, tolG, tolT);
}

template <typename T, int Q, typename Parts>
__device__ __forceinline__ int gamma_root_bracketed(const Parts &parts, T beta, T &t, T tolG, T tolT)
{
    const T c = (T)1 - (T)2 * beta;
    T lo = -(T)INFINITY, hi = (T)INFINITY;
    bool ok = true, pos = false, neg = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T fe, ds, dh;
        parts(i, fe, ds, dh);
        const T A = fe + c * ds;
        pos = pos || dh > (T)0;
        neg = neg || dh < (T)0;
        if (dh > (T)0) lo = fmax(lo, -A / dh);
        else if (dh < (T)0) hi = fmin(hi, -A / dh);
        else if (!(A > (T)0)) ok = false;
    }
    if (!pos || !neg) return 0;
    if (!ok || !(lo < hi) || !isfinite(lo) || !isfinite(hi)) return -1;
    T tt = (t > lo && t < hi) ? t : (T)0.5 * (lo + hi);
    T a = lo, b = hi;
    for (int it = 0; it < GAMMA_MAX_ITER; ++it) {
        T G = 0, dG = 0, S = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T fe, ds, dh;
            parts(i, fe, ds, dh);
            const T x = (c * ds + tt * dh) / fe;
            G += dh * log1p_<T>(x);
            // size of the term before the two parts of x cancel: the scale
            // of G's rounding
            S += fabs(dh) * (fabs(c * ds) + fabs(tt * dh)) / fe;
            dG += dh * dh / (fe * ((T)1 + x));
        }
        if (fabs(G) <= tolG * S) { t = tt; return 1; }
        if (G > (T)0) b = tt; else a = tt;
        if (!(b - a > tolT * ((T)1 + fabs(tt)))) { t = (T)0.5 * (a + b); return 1; }
        // Newton step, or bisection when it leaves the bracket; a step below
        // rounding ends the iteration when G is at its rounding floor
        // (within 1e3 of the bar) and bisects when it is not (next to a pole
        // of ln f'_i the derivative is huge and the step tiny while G is large)
        T tn = tt - G / dG;
        if (!(tn > a && tn < b)) {
            tn = (T)0.5 * (a + b);
        } else if (fabs(tn - tt) <= tolT * ((T)1 + fabs(tt))) {
            if (fabs(G) <= (T)1e3 * tolG * S) { t = tn; return 1; }
            tn = (T)0.5 * (a + b);
        }
        tt = tn;
    }
    return -1;
}

template <typename ST> struct StoreTraits;
template <> struct StoreTraits<double> { typedef double CT; static constexpr bool shifted = false; };
template <> struct StoreTraits<float> { typedef float CT; static constexpr bool shifted = true; };

// ---------------------------------------------------------------------------
// The fused kernel.
// ---------------------------------------------------------------------------
// FAST: no bounce-back axis and Q N < 2^31, so pulls need no wall test and
// their indices fit 32 bits.
// VEC: phase A reads the populations as aligned four-node vectors along x
// (D3Q27, FP32 storage, periodic, nx a multiple of 4, 32 x 8 tiles).
// MOM (carried moments; D3Q27 FP32 periodic step, rows of 32, nx % 32 == 0
// and ny % TY == 0): the
// step scatters each post-collision population to the node that the next
// step's pull brings it to, so that the next step's phase A reads rho and phi
// (Eqs. 6-8, the zeroth moments of the pulled f and g) instead of pulling the
// 54 populations of every node of the tile + ring 2 again.
template <int D, int TX, int TY, typename ST, int MODE, bool FAST, bool VEC = false, bool MOM = false>
struct Fused {
    typedef Lat<D> L;
    typedef typename StoreTraits<ST>::CT CT;
    typedef Vec<CT> V;
    typedef typename V::v2 V2;
    typedef typename V::v4 V4;
    static constexpr int Q = L::Q;
    static constexpr int NT = TX * TY;
    static constexpr bool STEPPING = MODE == MODE_STEP || MODE == MODE_STEP_EXACT || MODE == MODE_STEP_G64;
    static constexpr bool EXACT = MODE == MODE_STEP_EXACT;
    static constexpr int R2X = TX + 4, R2Y = (D == 3 ? TY + 4 : 1), NA = R2X * R2Y;
    static constexpr int R1X = TX + 2, R1Y = (D == 3 ? TY + 2 : 1), NB = R1X * R1Y;
    static constexpr int OY2 = (D == 3 ? 2 : 0), OY1 = (D == 3 ? 1 : 0);
    // vector phase A: 8 warps, each with 3 rows of 10 chunks of 4 nodes
    // (x0 - 4 .. x0 + TX + 3) in lanes 0-29; warps 0-3 sum f, warps 4-7 g,
    // over the TY + 4 rows of tile + ring 2
    static constexpr int NAV = 256;
    // D2Q9: one row of NV2 four-node vectors (x0 - 4 .. x0 + TX + 3) per
    // population set; with one warp, f in lanes 0 .. NV2-1 and g in lanes
    // NV2 .. 2 NV2-1; with two warps, f in warp 0 and g in warp 1, lanes
    // 0 .. NV2-1.  The warps' other lanes take chemical-potential items in
    // the same round.
    static constexpr int NV2 = TX / 4 + 2;
    static constexpr int AV2 = (NT == 32) ? 2 * NV2 : NV2;  // vector lanes per warp
    static constexpr int NB0 = (NT / 32) * (32 - AV2);      // chemical-potential items in round 0
    static_assert(!VEC || (STEPPING && FAST && StoreTraits<ST>::shifted &&
                           ((D == 3 && TX == 32 && TY == 8) ||
                            (D == 2 && TY == 1 && (TX == 32 || TX == 64)))),
                  "vector phase A: FP32 periodic step, D3Q27 32 x 8 or D2Q9 rows of 32 or 64");
    static_assert(!MOM || (D == 3 && TX == 32 && !VEC && STEPPING && FAST && StoreTraits<ST>::shifted),
                  "carried moments: the D3Q27 FP32 periodic step with rows of 32 (one warp per row)");

    // shared memory layout (in CT units)
    // ring buffers over planes: RS slots of rho, phi (tile + ring 2), MS of
    // mu and grad rho (tile + ring 1)
    // (rho, phi) and (mu_rho, mu_phi) are stored as pairs, (grad rho,
    // c_s^4/(4 rho)) as quads, so that a stencil neighbour is one load.
    // SPLIT (D3Q27): phases A and B in separate passes, pipeline depth 2,
    // RS = 4, MS = 3; otherwise one merged A/B pass, depth 3, RS = 6, MS = 4.
    static constexpr bool SPLIT = (D == 3);
    static constexpr int RS = SPLIT ? 4 : 6, MS = SPLIT ? 3 : 4;
    static constexpr int OFF_RP = 0;                         // pairs [RS][NA]
    static constexpr int OFF_MU = OFF_RP + 2 * RS * NA;      // pairs [MS][NB]
    static constexpr int OFF_G = OFF_MU + 2 * MS * NB;       // quads [MS][NB]
    static constexpr int OFF_F = OFF_G + 4 * MS * NB;        // per-thread population stash
    // FP64 storage: [Q][NT] pulled populations.  FP32 storage: [REST][NT]
    // pairs of pulled populations (the rest population stays in a register).
    static constexpr int STASH = StoreTraits<ST>::shifted ? 2 * L::REST * NT : Q * NT;
    static constexpr int SMEM_ELEMS = OFF_F + (STEPPING ? STASH : 0);
    // walled path: solid flags of the moment ring, RS slots of NA bytes after
    // the CT data (none on the fast path, which has no solid nodes)
    static constexpr size_t SOL_OFF = sizeof(CT) * SMEM_ELEMS;
    static constexpr size_t SOL_BYTES = FAST ? 0 : (((size_t)RS * NA + 15) / 16) * 16;
    static constexpr size_t SMEM_BYTES = SOL_OFF + SOL_BYTES;

    __device__ static __forceinline__ int idx2(int ox, int oy) { return (ox + 2) + R2X * (oy + OY2); }
    __device__ static __forceinline__ int idx1(int ox, int oy) { return (ox + 1) + R1X * (oy + OY1); }
    __device__ static __forceinline__ int slotR(int m) { int s = m % RS; return s < 0 ? s + RS : s; }
    __device__ static __forceinline__ int slotM(int m) { int s = m % MS; return s < 0 ? s + MS : s; }

    // Solid nodes (walled path only).  Phase A records, per moment slot, a
    // flag for every node of the tile + ring 2.  A stencil centred at ring
    // position (ox, oy) of plane m that reads along (cX, cY, cM) gets the
    // neighbour, or, when that is solid, a fluid ghost mirroring it across
    // the solid surface: the components of c are set to zero, fewest first
    // and in axis order x, y, z, until the node reached is fluid (the
    // reading of the axis walls' neutral wetting, which it reproduces where
    // solid layers fill the ends of an axis).  flip gets bit a for each
    // physical axis a that was zeroed: the vector component that changes sign.
    __device__ static __forceinline__ unsigned char *sol_ring()
    {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        return smem_raw + SOL_OFF;
    }
    __device__ static __forceinline__ bool ring_solid(const unsigned char *sol, int ox, int oy, int m)
    {
        return sol[slotR(m) * NA + idx2(ox, oy)] != 0;
    }
    __device__ static __forceinline__ void resolve(const unsigned char *sol, int ox, int oy, int m, int &cX, int &cY,
                                                   int &cM, unsigned &flip)
    {
        flip = 0u;
        if (!ring_solid(sol, ox + cX, oy + cY, m + cM)) return;
        // physical axes: D3Q27 (x, y, z) = (X, Y, M); D2Q9 (x, y) = (X, M)
        const int c0 = cX, c1 = D == 3 ? cY : cM, c2 = D == 3 ? cM : 0;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const unsigned S = k < 3 ? (1u << k) : (k == 3 ? 3u : (k == 4 ? 5u : (k == 5 ? 6u : 7u)));
            if (((S & 1u) && !c0) || ((S & 2u) && !c1) || ((S & 4u) && !c2)) continue;
            const int t0 = (S & 1u) ? 0 : c0, t1 = (S & 2u) ? 0 : c1, t2 = (S & 4u) ? 0 : c2;
            const int tX = t0, tY = D == 3 ? t1 : 0, tM = D == 3 ? t2 : t1;
            if (!ring_solid(sol, ox + tX, oy + tY, m + tM)) {
                cX = tX; cY = tY; cM = tM;
                flip = S;
                return;
            }
        }
        flip = (c0 ? 1u : 0u) | (c1 ? 2u : 0u) | (c2 ? 4u : 0u);  // the centre itself
        cX = cY = cM = 0;
    }

    // Bounce-back walls seen by a stencil centred at the lattice position
    // (gx, gy, gm) (gy unused in D2Q9; positions outside the lattice are
    // ghost slots whose values are not used): walls_crossed counts the axes
    // along which the read c leaves the lattice through a wall, wall_zero
    // sets those components of c to zero (the read goes to the mirrored
    // node, the centre's own coordinate on that axis), walls_adjacent counts
    // the wall sides next to the position.
    __device__ static __forceinline__ int walls_crossed(const DevParams &P, int gx, int gy, int gm, int cX, int cY,
                                                        int cM)
    {
        const int PX = P.nx, PY = (D == 3 ? P.ny : 1), PM = (D == 3 ? P.nz : P.ny);
        const int bX = P.bc[0], bY = (D == 3 ? P.bc[1] : 0), bM = (D == 3 ? P.bc[2] : P.bc[1]);
        int k = 0;
        if (bX && (gx + cX < 0 || gx + cX >= PX)) ++k;
        if (D == 3 && bY && (gy + cY < 0 || gy + cY >= PY)) ++k;
        if (bM && (gm + cM < 0 || gm + cM >= PM)) ++k;
        return k;
    }
    __device__ static __forceinline__ void wall_zero(const DevParams &P, int gx, int gy, int gm, int &cX, int &cY,
                                                     int &cM)
    {
        const int PX = P.nx, PY = (D == 3 ? P.ny : 1), PM = (D == 3 ? P.nz : P.ny);
        const int bX = P.bc[0], bY = (D == 3 ? P.bc[1] : 0), bM = (D == 3 ? P.bc[2] : P.bc[1]);
        if (bX && (gx + cX < 0 || gx + cX >= PX)) cX = 0;
        if (D == 3 && bY && (gy + cY < 0 || gy + cY >= PY)) cY = 0;
        if (bM && (gm + cM < 0 || gm + cM >= PM)) cM = 0;
    }
    __device__ static __forceinline__ int walls_adjacent(const DevParams &P, int gx, int gy, int gm)
    {
        const int PX = P.nx, PY = (D == 3 ? P.ny : 1), PM = (D == 3 ? P.nz : P.ny);
        const int bX = P.bc[0], bY = (D == 3 ? P.bc[1] : 0), bM = (D == 3 ? P.bc[2] : P.bc[1]);
        int k = 0;
        if (bX) k += (gx == 0) + (gx == PX - 1);
        if (D == 3 && bY) k += (gy == 0) + (gy == PY - 1);
        if (bM) k += (gm == 0) + (gm == PM - 1);
        return k;
    }

    // Sources of the populations pulled into node (x, y, m): per axis the
    // source coordinate x - c for c = -1, 0, 1 (periodic wrap) as an offset,
    // and a bit per (axis, c) when that source lies beyond a bounce-back wall
    // (the node then takes its own reversed population, half-way bounce-back).
    struct Nbr {
        int n;                // node index (N < 2^31 is enforced at creation)
        int off[3][3];        // [axis X, Y, M][c + 1]
        unsigned out;         // bit 3*axis + (c + 1)
        unsigned sol;         // bit i: the source x - c_i is a solid node (walled path only)
    };

    __device__ static __forceinline__ void make_nbr(const DevParams &P, int PX, int PY, int PM, int x, int y,
                                                    int m, Nbr &b)
    {
        const int bx = P.bc[0], by = (D == 3 ? P.bc[1] : 0), bm = (D == 3 ? P.bc[2] : P.bc[1]);
        b.n = x + PX * (y + PY * m);
        b.out = 0u;
        const int q[3] = {x, y, m}, ext[3] = {PX, PY, PM}, wall[3] = {bx, by, bm};
        const int stride[3] = {1, PX, PX * PY};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int c = -1; c <= 1; ++c) {
                int sc = q[a] - c;
                if (a == 1 && D == 2) sc = 0;
                bool o = false;
                if (FAST) {
                    if (sc < 0) sc += ext[a];
                    else if (sc >= ext[a]) sc -= ext[a];
                } else {
                    if (sc < 0) { if (wall[a]) o = true; else sc += ext[a]; }
                    else if (sc >= ext[a]) { if (wall[a]) o = true; else sc -= ext[a]; }
                }
                b.off[a][c + 1] = sc * stride[a];
                if (o) b.out |= 1u << (3 * a + c + 1);
            }
        }
        b.sol = 0u;
        if constexpr (!FAST) {
            // half-way bounce-back wherever the source of a pull is solid
            if (P.solid) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int cX = L::pX(i) + 1, cY = L::pY(i) + 1, cM = L::pM(i) + 1;
                    const unsigned mask = (1u << cX) | (D == 3 ? (1u << (3 + cY)) : 0u) | (1u << (6 + cM));
                    if (!(b.out & mask) && P.solid[b.off[0][cX] + b.off[1][cY] + b.off[2][cM]]) b.sol |= 1u << i;
                }
            }
        }
    }

    // population i pulled into the node described by b
    __device__ static __forceinline__ CT pull(const ST *base, const Nbr &b, long long N, int i)
    {
        if (FAST) {
            const int cX = L::pX(i) + 1, cY = L::pY(i) + 1, cM = L::pM(i) + 1;
            const unsigned k = (unsigned)i * (unsigned)N + (unsigned)(b.off[0][cX] + b.off[1][cY] + b.off[2][cM]);
            return (CT)__ldg(base + k);
        }
        return (CT)__ldg(base + src_index(b, N, i));
    }

    // address of population i pulled into the node described by b
    __device__ static __forceinline__ const ST *pull_ptr(const ST *base, const Nbr &b, long long N, int i)
    {
        if (FAST) {
            const int cX = L::pX(i) + 1, cY = L::pY(i) + 1, cM = L::pM(i) + 1;
            return base + ((unsigned)i * (unsigned)N + (unsigned)(b.off[0][cX] + b.off[1][cY] + b.off[2][cM]));
        }
        return base + src_index(b, N, i);
    }

    // global index of population i pulled into the node described by b
    __device__ static __forceinline__ long long src_index(const Nbr &b, long long N, int i)
    {
        const int cX = L::pX(i) + 1, cY = L::pY(i) + 1, cM = L::pM(i) + 1;
        const unsigned mask = (1u << cX) | (D == 3 ? (1u << (3 + cY)) : 0u) | (1u << (6 + cM));
        if ((b.out & mask) || ((b.sol >> i) & 1u)) return (long long)(Q - 1 - i) * N + b.n;
        return (long long)i * N + (b.off[0][cX] + b.off[1][cY] + b.off[2][cM]);
    }

    __device__ static void run(const DevParams &P, const LaunchArgs &A)
    {
        run_tile(P, A, blockIdx.x, D == 3 ? blockIdx.y : 0, D == 3 ? blockIdx.z : blockIdx.y);
    }

    // One CTA's work: the tile (bx, by) of the plane normal to the marching
    // axis, through chunk bm of planes.
    __device__ static void run_tile(const DevParams &P, const LaunchArgs &A, int bx, int by, int bm)
    {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        CT *sm = reinterpret_cast<CT *>(smem_raw);
        V2 *rp_s = reinterpret_cast<V2 *>(sm + OFF_RP);
        V2 *mu_s = reinterpret_cast<V2 *>(sm + OFF_MU);
        V4 *g_s = reinterpret_cast<V4 *>(sm + OFF_G);

        const int PX = P.nx, PY = (D == 3 ? P.ny : 1), PM = (D == 3 ? P.nz : P.ny);
        const int bX = P.bc[0], bY = (D == 3 ? P.bc[1] : 0), bM = (D == 3 ? P.bc[2] : P.bc[1]);
        const int tid = threadIdx.x;
        const int x0 = bx * TX;
        const int y0 = (D == 3 ? by * TY : 0);
        const int m0 = bm * P.chunk;
        const int m1 = min(m0 + P.chunk, PM);
        const CT shift = coef<CT>(P).rho_ref;
        const ST *fs = reinterpret_cast<const ST *>(A.fsrc);
        const ST *gs = reinterpret_cast<const ST *>(A.gsrc);

        // Software pipeline over planes.  SPLIT: iteration it computes the
        // moments of mA (phase A), then, after a barrier, the chemical
        // potentials of mB = mA - 1 (phase B), then, after a barrier, the
        // collision of mC = mA - 2 (phase C).  The next iteration's phase A
        // may overlap this phase C: with RS = 4 the moment slot it writes is
        // not one that phase C reads (one more barrier when phase C reads the
        // neighbouring planes' moments, for grad rho and grad phi); phase B
        // only starts once every thread has passed the next barrier, so MS = 3.
        // Merged (D2Q9): phases A (plane mA) and B (mB = mA - 2) share one
        // load-balanced pass, then, after the barrier, phase C collides
        // mC = mA - 3; with RS = 6 and MS = 4 the next A/B pass never writes a
        // slot that phase C is still reading.
        const int tid_x = tid % TX, tid_y = tid / TX;
        // phase C reads the neighbouring planes' moments (or, with solid
        // nodes, their flags): then one more barrier per iteration
        const bool need_grp = (MODE == MODE_FIELDS) || P.force_form == 0 || (!FAST && P.solid != nullptr);
        const int iters = (m1 - m0) + (SPLIT ? 4 : 5);
        // marching direction: with TEL_ALT_MARCH, odd chunks march downwards,
        // so that two neighbouring chunks read their shared halo planes at
        // about the same time
#ifdef TEL_ALT_MARCH
        const int dir = (bm & 1) ? -1 : 1;
#else
        const int dir = 1;
#endif
        for (int it = 0; it < iters; ++it) {
            const int mA = dir > 0 ? m0 - 2 + it : m1 + 1 - it;
            const int mB = mA - dir * (SPLIT ? 1 : 2);
            const int mC = mA - dir * (SPLIT ? 2 : 3);
            const bool doA = dir > 0 ? mA <= m1 + 1 : mA >= m0 - 2;
            const bool doB = mB >= m0 - 1 && mB <= m1;
            const int nA = doA ? (VEC ? NAV : NA) : 0;
            const int mm = map_coord(mA, PM, bM);
            auto item_a = [&](int w) {
                if constexpr (MOM) {
                    phase_a_mom(P, A.m_read, rp_s + slotR(mA) * NA, w, x0, y0, mm, shift);
                    return;
                }
                if constexpr (VEC && D == 3) {
                    phase_a_vec(P, fs, gs, rp_s + slotR(mA) * NA, w, x0, y0, mm, shift);
                    return;
                }
                // ---------------- phase A: moments of plane mA on tile + ring 2
                const int r = w;
                const int ox = r % R2X - 2, oy = (D == 3 ? r / R2X - 2 : 0);
                const int xx = map_coord(x0 + ox, PX, bX);
                const int yy = (D == 3 ? map_coord(y0 + oy, PY, bY) : 0);
                CT rho, phi;
                bool solid = false;
                if constexpr (!FAST) {
                    if (P.solid) {
                        const long long n = (long long)xx + (long long)PX * ((long long)yy + (long long)PY * mm);
                        solid = P.solid[n] != 0;
                        sol_ring()[slotR(mA) * NA + r] = solid ? 1 : 0;
                    }
                }
                if (solid) {
                    // placeholder moments of a solid node: no fluid stencil reads them
                    rho = coef<CT>(P).rho_l;
                    phi = 0;
                } else if (MODE == MODE_INIT) {
                    const long long n = (long long)xx + (long long)PX * ((long long)yy + (long long)PY * mm);
                    rho = (CT)A.in_rho[n];
                    phi = (CT)A.in_phi[n];
                } else {
                    Nbr nb;
                    make_nbr(P, PX, PY, PM, xx, yy, mm, nb);
                    CT sr = 0, sp = 0;
#pragma unroll
                    for (int i = 0; i < Q; ++i) sr += pull(fs, nb, P.N, i);
#pragma unroll
                    for (int i = 0; i < Q; ++i) sp += pull(gs, nb, P.N, i);
                    rho = StoreTraits<ST>::shifted ? shift + sr : sr;
                    phi = sp;
                }
                rp_s[slotR(mA) * NA + r] = V::pair(rho, phi);
            };
            auto item_b = [&](int s) {
                // ---------------- phase B: chemical potentials of plane mB on tile + ring 1
                const int sB = slotM(mB);
                const int ox = s % R1X - 1, oy = (D == 3 ? s / R1X - 1 : 0);
                const int c0 = idx2(ox, oy);
                const V2 cp = rp_s[slotR(mB) * NA + c0];
                const CT r0 = cp.x, p0 = cp.y;
                const V2 ncp = V::pair(-r0, -p0);
                V2 lap = V::pair((CT)0, (CT)0);
                CT gx = 0, gy = 0, gz = 0;
                // wetting: sum of w_i times the axes mirrored by read i (the
                // ghost of rho, phi in the Laplacians is the mirrored value
                // plus wet_rho, wet_phi per mirrored axis)
                CT wet_w = 0;
                bool masked = false;
                if constexpr (!FAST) masked = P.solid != nullptr;
                if (masked) {
                    // solid nodes: each neighbour through its ghost; a solid
                    // centre is never read by a fluid stencil
                    const unsigned char *sol = sol_ring();
                    if (ring_solid(sol, ox, oy, mB)) {
                        mu_s[sB * NB + s] = V::pair((CT)0, (CT)0);
                        if (P.force_form == 1) g_s[sB * NB + s] = V::quad((CT)0, (CT)0, (CT)0, (CT)0);
                        return;
                    }
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        if (i == L::REST) continue;
                        int cX = L::pX(i), cY = L::pY(i), cM = L::pM(i);
                        unsigned fl;
                        resolve(sol, ox, oy, mB, cX, cY, cM, fl);
                        const V2 v = rp_s[slotR(mB + cM) * NA + idx2(ox + cX, oy + cY)];
                        const CT wi = (CT)L::w(i);
                        wet_w += wi * (CT)(__popc(fl) + walls_crossed(P, x0 + ox, y0 + oy, mB, cX, cY, cM));
                        lap = V::fma(V::pair(wi, wi), V::add(v, ncp), lap);
                        if (L::cx(i)) gx += wi * (CT)L::cx(i) * v.x;
                        if (L::cy(i)) gy += wi * (CT)L::cy(i) * v.x;
                        if (D == 3 && L::cz(i)) gz += wi * (CT)L::cz(i) * v.x;
                    }
                } else {
                    // over opposite neighbours (i, Q-1-i): the Laplacian takes
                    // both differences to the centre, the gradient the
                    // difference of the two
#pragma unroll
                    for (int i = 0; i < L::REST; ++i) {
                        const int io = Q - 1 - i;
                        const V2 va = rp_s[slotR(mB + L::pM(i)) * NA + idx2(ox + L::pX(i), oy + L::pY(i))];
                        const V2 vb = rp_s[slotR(mB + L::pM(io)) * NA + idx2(ox + L::pX(io), oy + L::pY(io))];
                        const CT wi = (CT)L::w(i);
                        lap = V::fma(V::pair(wi, wi), V::add(V::add(va, ncp), V::add(vb, ncp)), lap);
                        const CT d = va.x - vb.x;
                        if (L::cx(i)) gx += wi * (CT)L::cx(i) * d;
                        if (L::cy(i)) gy += wi * (CT)L::cy(i) * d;
                        if (D == 3 && L::cz(i)) gz += wi * (CT)L::cz(i) * d;
                    }
                    // at the walls the ghost slots hold the mirrored values;
                    // the reads across one wall side carry weight 1/6 in all
                    if constexpr (!FAST) wet_w = (CT)walls_adjacent(P, x0 + ox, y0 + oy, mB) * (CT)(1.0 / 6.0);
                }
                const CT lr = (CT)6 * (coef<CT>(P).wr * wet_w + lap.x);
                const CT lp = (CT)6 * (coef<CT>(P).wp * wet_w + lap.y);
                CT mr, mp;
                mu_wells<CT>(P, r0, p0, mr, mp);
                if (StoreTraits<ST>::shifted && r0 < coef<CT>(P).rho_switch)  // FP64 gas side
                    mr = (P.eos == EOS_CS ? (CT)mu_eos_gas(P, (float)r0) : (CT)mu_eos<double>(P, (double)r0)) + mr;
                else
                    mr = mu_eos<CT>(P, r0) + mr;
                mu_s[sB * NB + s] = V::pair(mr - coef<CT>(P).Kr * lr - coef<CT>(P).Kx * lp,
                                            mp - coef<CT>(P).Kp * lp - coef<CT>(P).Kx * lr);
                if (P.force_form == 1)  // grad rho and c_s^4/(4 rho) (lattice-consistent force)
                    g_s[sB * NB + s] = V::quad((CT)3 * gx, (CT)3 * gy, (CT)3 * gz, (CT)(1.0 / 36.0) * inv_<CT>(r0));
            };
            if constexpr (SPLIT) {
                for (int w = tid; w < nA; w += NT) item_a(w);
                __syncthreads();
                if (doB)
                    for (int s = tid; s < NB; s += NT) item_b(s);
            } else if constexpr (VEC) {
                // D2Q9 vector phase A: round 0 runs the row's vectors in the
                // first AV2 lanes of each warp and chemical-potential items in
                // the others; the vectors' end elements are exchanged after
                // the branches, with every lane of the warp present
                const int lane = tid & 31, q = tid >> 5;
                const bool a_lane = doA && lane < AV2;
                const bool is_g = (NT == 32) ? lane >= NV2 : q == 1;
                const int c = (NT == 32 && lane >= NV2) ? lane - NV2 : lane;
                float2 h[3][2];
                if (a_lane) {
                    row_vec_sums(P, fs, gs, c, is_g, x0, mm, h);
                } else {
                    const int b = q * (32 - AV2) + (lane - AV2);
                    if (doB && lane >= AV2 && b < NB) item_b(b);
#pragma unroll
                    for (int a = 0; a < 3; ++a) h[a][0] = h[a][1] = bc2(0.f);
                }
                const float hl = __shfl_up_sync(0xffffffffu, h[2][1].y, 1);
                const float hr = __shfl_down_sync(0xffffffffu, h[0][0].x, 1);
                if (a_lane) row_vec_store(rp_s + slotR(mA) * NA, c, is_g, h, hl, hr, shift);
                if (doB)
                    for (int b = NB0 + tid; b < NB; b += NT) item_b(b);
            } else {
                const int nW = nA + (doB ? NB : 0);
                for (int w = tid; w < nW; w += NT) {
                    if (w < nA) item_a(w);
                    else item_b(w - nA);
                }
            }
            __syncthreads();
            // ---------------- phase C: collide plane mC
            if (mC >= m0 && mC < m1) {
                const int x = x0 + tid_x, y = y0 + tid_y;
                if (x < PX && (D == 2 || y < PY))
                    node(P, A, fs, gs, rp_s, mu_s, g_s, sm + OFF_F, x, y, mC, tid_x, tid_y);
            }
            if constexpr (SPLIT) {
                if (need_grp) __syncthreads();
            }
        }
    }

    // Phase A with carried moments: item w is node (w % R2X - 2, w / R2X - 2)
    // of the tile + ring 2 (periodic wrap), whose rho - rho_ref and phi the
    // previous step (or the moments kernel after a new state) has summed.
    __device__ static __forceinline__ void phase_a_mom(const DevParams &P, const float *mr, V2 *rp_plane, int w,
                                                       int x0, int y0, int m, CT shift)
    {
        const int ox = w % R2X - 2, oy = w / R2X - 2;
        int xx = x0 + ox, yy = y0 + oy;
        if (xx < 0) xx += P.nx; else if (xx >= P.nx) xx -= P.nx;
        if (yy < 0) yy += P.ny; else if (yy >= P.ny) yy -= P.ny;
        const unsigned n = (unsigned)xx + (unsigned)P.nx * ((unsigned)yy + (unsigned)P.ny * (unsigned)m);
        rp_plane[w] = V::pair(shift + __ldg(mr + n), __ldg(mr + (unsigned)P.N + n));
    }

    // Carried moments: the post-collision populations c = (c_x, cy, cz),
    // c_x = -1, 0, 1, of the warp's row (lane = x - x0) reach the nodes
    // x + c of row y + cy of plane z + cz in the next step's pull.  The three
    // that reach node x are summed across lanes first (one atomic add per
    // node of the row), the two that leave the warp's 32 nodes (x0 - 1 from
    // lane 0, x0 + 32 from lane 31) are added by one more instruction.  Every
    // lane of the warp is present (full tiles).
    __device__ static __forceinline__ void scatter_row(float *M, const Nbr &nb, int cy, int cz, float vm, float v0,
                                                       float vp)
    {
        const int lane = threadIdx.x & 31;
        const float up = __shfl_up_sync(0xffffffffu, vp, 1);    // c_x = +1 of node x - 1
        const float dn = __shfl_down_sync(0xffffffffu, vm, 1);  // c_x = -1 of node x + 1
        const float sum = v0 + (lane > 0 ? up : 0.f) + (lane < 31 ? dn : 0.f);
        const unsigned row = (unsigned)(nb.off[1][1 - cy] + nb.off[2][1 - cz]);
        atomicAdd(M + row + (unsigned)nb.off[0][1], sum);
        if (lane == 0 || lane == 31)
            atomicAdd(M + row + (unsigned)(lane == 0 ? nb.off[0][2] : nb.off[0][0]), lane == 0 ? vm : vp);
    }

    // Phase A on four-node vectors along x.  Item w (all 32 lanes of warp
    // w / 32 present) sums f (warps 0-3) or g (warps 4-7) over row
    // oy = 3 (w / 32 % 4) + (w % 32) / 10 - 2 for the chunk
    // x0 - 4 + 4c .. x0 - 1 + 4c, c = (w % 32) % 10; lanes 30, 31 idle.
    // Population i pulled into node x is f_i(x - c_ix) of row y - c_iy and
    // plane m - c_iz: with the populations of one sign of c_ix summed per
    // vector, the shifted element comes from the same vector or, at its end,
    // from the neighbouring lane's.  Only the nodes of tile + ring 2 are
    // stored (the outermost node of chunks 0 and 9 takes a neighbour row's
    // value and is not needed).
    __device__ static void phase_a_vec(const DevParams &P, const ST *fs, const ST *gs, V2 *rp_plane, int w,
                                       int x0, int y0, int m, CT shift)
    {
        const int lane = w & 31, rr = lane / 10, c = lane - 10 * rr;
        const bool is_g = (w >> 5) >= 4;
        const int oy = 3 * ((w >> 5) & 3) + rr - 2;
        const bool act = lane < 30;
        const int PX = P.nx, PY = P.ny, PM = P.nz;
        // periodic wrap; with nx % 4 == 0 a chunk never straddles the seam
        int X = (x0 - 4 + 4 * c) % PX;
        if (X < 0) X += PX;
        const int y = y0 + oy;
        int ro[3], po[3];
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
            int yy = (y - d) % PY, mm = m - d;  // m is already in [0, PM)
            if (yy < 0) yy += PY;
            if (mm < 0) mm += PM; else if (mm >= PM) mm -= PM;
            ro[d + 1] = yy * PX;
            po[d + 1] = mm * PX * PY;
        }
        const ST *src = is_g ? gs : fs;
        float2 h[3][2];  // [c_x + 1][low, high half of the vector]
#pragma unroll
        for (int a = 0; a < 3; ++a) h[a][0] = h[a][1] = bc2(0.f);
        if (act) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const unsigned k = (unsigned)i * (unsigned)P.N + (unsigned)(ro[L::cy(i) + 1] + po[L::cz(i) + 1] + X);
                const float4 v = __ldg(reinterpret_cast<const float4 *>(src + k));
                const int a = L::cx(i) + 1;
                h[a][0] = add2(h[a][0], make_float2(v.x, v.y));
                h[a][1] = add2(h[a][1], make_float2(v.z, v.w));
            }
        }
        // c_x = +1 pulls from x - 1, c_x = -1 from x + 1
        const float hl = __shfl_up_sync(0xffffffffu, h[2][1].y, 1);
        const float hr = __shfl_down_sync(0xffffffffu, h[0][0].x, 1);
        const float sum[4] = {h[1][0].x + hl + h[0][0].y, h[1][0].y + h[2][0].x + h[0][1].x,
                              h[1][1].x + h[2][0].y + h[0][1].y, h[1][1].y + h[2][1].x + hr};
        if (act) {
            float *dst = reinterpret_cast<float *>(rp_plane) + (is_g ? 1 : 0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int ox = 4 * c - 4 + e;
                if (ox >= -2 && ox < TX + 2) dst[2 * idx2(ox, oy)] = is_g ? sum[e] : shift + sum[e];
            }
        }
    }

    // D2Q9 phase A on four-node vectors along x (rows of the marching axis
    // y): lane item c sums f or g over x0 - 4 + 4c .. x0 - 1 + 4c of row m,
    // keeping the populations of each sign of c_ix apart (h[c_x + 1]), which
    // row_vec_store shifts by one node with the neighbouring lanes' end
    // elements.  Population i pulled into node x of row m is f_i(x - c_ix)
    // of row m - c_iy.  nx % 4 == 0, so no vector straddles the periodic seam.
    __device__ static void row_vec_sums(const DevParams &P, const ST *fs, const ST *gs, int c, bool is_g, int x0,
                                        int m, float2 (&h)[3][2])
    {
        const int PX = P.nx, PM = P.ny;
        int X = (x0 - 4 + 4 * c) % PX;
        if (X < 0) X += PX;
        int po[3];
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
            int mm = m - d;  // m is already in [0, PM)
            if (mm < 0) mm += PM; else if (mm >= PM) mm -= PM;
            po[d + 1] = mm * PX;
        }
        const ST *src = is_g ? gs : fs;
#pragma unroll
        for (int a = 0; a < 3; ++a) h[a][0] = h[a][1] = bc2(0.f);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const unsigned k = (unsigned)i * (unsigned)P.N + (unsigned)(po[L::cy(i) + 1] + X);
            const float4 v = __ldg(reinterpret_cast<const float4 *>(src + k));
            const int a = L::cx(i) + 1;
            h[a][0] = add2(h[a][0], make_float2(v.x, v.y));
            h[a][1] = add2(h[a][1], make_float2(v.z, v.w));
        }
    }
    // The four nodes' sums (c_x = +1 pulls from x - 1, c_x = -1 from x + 1;
    // hl, hr: the previous lane's last and the next lane's first element),
    // stored for the nodes of tile + ring 2.  The outermost node of the first
    // and the last vector takes another item's value and is not stored.
    __device__ static void row_vec_store(V2 *rp_plane, int c, bool is_g, const float2 (&h)[3][2], float hl, float hr,
                                         CT shift)
    {
        const float sum[4] = {h[1][0].x + hl + h[0][0].y, h[1][0].y + h[2][0].x + h[0][1].x,
                              h[1][1].x + h[2][0].y + h[0][1].y, h[1][1].y + h[2][1].x + hr};
        float *dst = reinterpret_cast<float *>(rp_plane) + (is_g ? 1 : 0);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int ox = 4 * c - 4 + e;
            if (ox >= -2 && ox < TX + 2) dst[2 * idx2(ox, 0)] = is_g ? sum[e] : shift + sum[e];
        }
    }

    __device__ static void node(const DevParams &P, const LaunchArgs &A, const ST *fs, const ST *gs,
                                const V2 *rp_s, const V2 *mu_s, const V4 *g_s, CT *stash, int x, int y, int m,
                                int tx, int ty)
    {
        CT *fq = stash + (tx + TX * ty);  // this thread's column of the population stash
        const int PX = P.nx, PY = (D == 3 ? P.ny : 1), PM = (D == 3 ? P.nz : P.ny);
        const long long n = (long long)x + (long long)PX * ((long long)y + (long long)PY * m);
        const int ox = tx, oy = (D == 3 ? ty : 0);
        const V2 rp0 = rp_s[slotR(m) * NA + idx2(ox, oy)];
        const CT rho = rp0.x, phi = rp0.y;
        const Coef<CT> &K = coef<CT>(P);
        const CT shift = K.rho_ref;
        bool masked = false;
        if constexpr (!FAST) masked = P.solid != nullptr;
        if (masked && ring_solid(sol_ring(), ox, oy, m)) {
            // a solid node: zero state (own slots) and zero fields
            if constexpr (MODE == MODE_FIELDS) {
                if (A.out_rho) A.out_rho[n] = 0.0;
                if (A.out_phi) A.out_phi[n] = 0.0;
                if (A.out_u)
                    for (int a = 0; a < D; ++a) A.out_u[(long long)a * P.N + n] = 0.0;
                if (A.out_p) A.out_p[n] = 0.0;
            } else {
                ST *fd = reinterpret_cast<ST *>(A.fdst);
                ST *gd = reinterpret_cast<ST *>(A.gdst);
                for (int i = 0; i < Q; ++i) {
                    fd[(long long)i * P.N + n] = (ST)0;
                    gd[(long long)i * P.N + n] = (ST)0;
                }
            }
            return;
        }

        // FP32 storage, step mode: start the copies of the node's f pulls into
        // its column of the stash now, so that they are in flight during the
        // stencils below (pairs (f_k, f_{Q-1-k}); the rest population into a
        // register).
        Nbr nbc;
        CT f_rest = 0;
        if constexpr (StoreTraits<ST>::shifted && STEPPING) {
            make_nbr(P, PX, PY, PM, x, y, m, nbc);
            CT *col = stash + 2 * (tx + TX * ty);
#pragma unroll
            for (int k = 0; k < L::REST; ++k) {
                cp_async4(col + 2 * k * NT, pull_ptr(fs, nbc, P.N, k));
                cp_async4(col + 2 * k * NT + 1, pull_ptr(fs, nbc, P.N, Q - 1 - k));
            }
            cp_async_commit();
            f_rest = pull(fs, nbc, P.N, L::REST);
        }

        // gradients at the node: grad (mu_rho, mu_phi) from the ring-1 pairs,
        // grad (rho, phi) from the ring-2 pairs (the latter only for the
        // potential-form force and the field output), as packed pairs
        V2 gmu[3], grp[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) { gmu[a] = V::pair((CT)0, (CT)0); grp[a] = V::pair((CT)0, (CT)0); }
        const bool need_grp = (MODE == MODE_FIELDS) || P.force_form == 0;
        if (masked) {
            // solid nodes: each neighbour through its ghost (scalar fields)
            const unsigned char *sol = sol_ring();
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (i == L::REST) continue;
                int cX = L::pX(i), cY = L::pY(i), cM = L::pM(i);
                unsigned fl;
                resolve(sol, ox, oy, m, cX, cY, cM, fl);
                const V2 vr = rp_s[slotR(m + cM) * NA + idx2(ox + cX, oy + cY)];
                // the chemical potentials' ghost across a wall is the mirrored
                // node's value
                wall_zero(P, x, y, m, cX, cY, cM);
                const V2 vm = mu_s[slotM(m + cM) * NB + idx1(ox + cX, oy + cY)];
                const CT wi = (CT)L::w(i);
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const int ca = L::c(i, a);
                    if (ca) {
                        gmu[a] = V::fma(V::pair(wi * (CT)ca, wi * (CT)ca), vm, gmu[a]);
                        if (need_grp) grp[a] = V::fma(V::pair(wi * (CT)ca, wi * (CT)ca), vr, grp[a]);
                    }
                }
            }
        } else {
            // over opposite neighbours (i, Q-1-i): w_i c_i (v(x + c_i) - v(x - c_i))
#pragma unroll
            for (int i = 0; i < L::REST; ++i) {
                const int io = Q - 1 - i;
                int aX = L::pX(i), aY = L::pY(i), aM = L::pM(i);
                int bX_ = L::pX(io), bY_ = L::pY(io), bM_ = L::pM(io);
                if constexpr (!FAST) {
                    // walls: the chemical potentials' ghost is the mirrored
                    // node's value
                    wall_zero(P, x, y, m, aX, aY, aM);
                    wall_zero(P, x, y, m, bX_, bY_, bM_);
                }
                const V2 vm = V::sub(mu_s[slotM(m + aM) * NB + idx1(ox + aX, oy + aY)],
                                     mu_s[slotM(m + bM_) * NB + idx1(ox + bX_, oy + bY_)]);
                const CT wi = (CT)L::w(i);
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const int ca = L::c(i, a);
                    if (ca) gmu[a] = V::fma(V::pair(wi * (CT)ca, wi * (CT)ca), vm, gmu[a]);
                }
                if (need_grp) {
                    const V2 vr = V::sub(rp_s[slotR(m + L::pM(i)) * NA + idx2(ox + L::pX(i), oy + L::pY(i))],
                                         rp_s[slotR(m + L::pM(io)) * NA + idx2(ox + L::pX(io), oy + L::pY(io))]);
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        const int ca = L::c(i, a);
                        if (ca) grp[a] = V::fma(V::pair(wi * (CT)ca, wi * (CT)ca), vr, grp[a]);
                    }
                }
            }
        }
        CT gm[3], gp[3], gr[3], gf[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gm[a] = gmu[a].x; gp[a] = gmu[a].y; gr[a] = grp[a].x; gf[a] = grp[a].y;
        }
        CT F[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            gm[a] *= (CT)3; gp[a] *= (CT)3; gr[a] *= (CT)3; gf[a] *= (CT)3;
            F[a] = -rho * gm[a] - phi * gp[a];
        }
        const CT cs2 = (CT)(1.0 / 3.0);
        if (P.force_form == 0) {
#pragma unroll
            for (int a = 0; a < D; ++a) F[a] += cs2 * gr[a];
        } else {
            // A[G]_a = sum_i 3 w_i c_ia c_i.G(x - c_i) = sum_j 3 w_j c_ja c_j.G(x + c_j)
            // (j the opposite of i), and div T with T = c_s^4 G G/(4 rho):
            // sum_b c_jb T_ab(x + c_j) = s_j G_a (c_j.G) with s = c_s^4/(4 rho).
            // Both read the same 26 neighbours (G and s stored per ring-1 node).
            CT AG[3] = {0, 0, 0}, dT[3] = {0, 0, 0};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (L::nnz(i) == 0) continue;
                const CT wi3 = (CT)(3.0 * L::w(i));
                int cX = L::pX(i), cY = L::pY(i), cM = L::pM(i);
                unsigned fl = 0u;
                if (masked) resolve(sol_ring(), ox, oy, m, cX, cY, cM, fl);
                const int sp_ = slotM(m + cM);
                const int kp = idx1(ox + cX, oy + cY);
                const V4 gq = g_s[sp_ * NB + kp];
                // G at a ghost: the components along mirrored axes change sign
                const CT Gp[3] = {(fl & 1u) ? -gq.x : gq.x, (fl & 2u) ? -gq.y : gq.y, (fl & 4u) ? -gq.z : gq.z};
                const CT sj = gq.w;
                CT cG = 0;
#pragma unroll
                for (int b = 0; b < D; ++b)
                    if (L::c(i, b)) cG += (CT)L::c(i, b) * Gp[b];
                const CT t = wi3 * cG;
#pragma unroll
                for (int a = 0; a < D; ++a)
                    if (L::c(i, a)) AG[a] += (CT)L::c(i, a) * t;
                const CT q = t * sj;
#pragma unroll
                for (int a = 0; a < D; ++a) dT[a] += q * Gp[a];
            }
            const V4 g0 = g_s[slotM(m) * NB + idx1(ox, oy)];
            const CT G0[3] = {g0.x, g0.y, g0.z};
#pragma unroll
            for (int a = 0; a < D; ++a)
                F[a] += cs2 * ((CT)1.5 * G0[a] - (CT)0.5 * AG[a]) + dT[a];
        }
        const V2 mu0 = mu_s[slotM(m) * NB + idx1(ox, oy)];
        const CT mu_phi = mu0.y;

        if (MODE == MODE_INIT) {
            init_node(P, A, n, x, y, m, rho, phi, mu_phi, F);
            return;
        }
        if constexpr (StoreTraits<ST>::shifted && STEPPING) {
            if constexpr (MOM) {
                // the buffer that the step after the next one accumulates into
                A.m_zero[n] = 0.f;
                A.m_zero[P.N + n] = 0.f;
            }
            collide_pairs(P, A, gs, nbc, f_rest, reinterpret_cast<float2 *>(stash) + (tx + TX * ty), n, rho, phi,
                          mu_phi, F);
            return;
        }

        // ---- pull f: momentum and second moments.  The pulled populations
        // are kept in this thread's column of shared memory (fq[i * NT]) for
        // the two later passes instead of 27 registers.
        Nbr nb;
        make_nbr(P, PX, PY, PM, x, y, m, nb);
        CT j[3] = {0, 0, 0};
        CT Pi[6] = {0, 0, 0, 0, 0, 0};  // xx yy zz xy xz yz
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const CT fi = pull(fs, nb, P.N, i);
            if (STEPPING) fq[i * NT] = fi;
            if (L::cx(i)) { j[0] += (CT)L::cx(i) * fi; Pi[0] += fi; }
            if (L::cy(i)) { j[1] += (CT)L::cy(i) * fi; Pi[1] += fi; }
            if (D == 3 && L::cz(i)) { j[2] += (CT)L::cz(i) * fi; Pi[2] += fi; }
            if (L::cx(i) * L::cy(i)) Pi[3] += (CT)(L::cx(i) * L::cy(i)) * fi;
            if (D == 3 && L::cx(i) * L::cz(i)) Pi[4] += (CT)(L::cx(i) * L::cz(i)) * fi;
            if (D == 3 && L::cy(i) * L::cz(i)) Pi[5] += (CT)(L::cy(i) * L::cz(i)) * fi;
        }
        if (StoreTraits<ST>::shifted) {
            // the shift w_i rho_ref adds rho_ref c_s^2 to each diagonal second moment
            Pi[0] += shift * cs2; Pi[1] += shift * cs2; if (D == 3) Pi[2] += shift * cs2;
        }
        CT u[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = j[a] / rho;

        unsigned bad = 0;
        if (!(rho > (CT)0)) bad |= ERR_RHO;

        if (MODE == MODE_FIELDS) {
            fields_node(P, A, n, rho, phi, j, F, gr, gf, mu0.x, mu_phi);
            if (bad) raise_err(P.err, bad);
            return;
        }

        if constexpr (!StoreTraits<ST>::shifted) {
            // ---- FP64 storage, step mode.  Phase field first (its pulls reuse
            // the offsets just computed): BGK towards g^eq(phi, mu_phi, u_phys)
            CT up[3] = {0, 0, 0};
            CT uu = 0;
#pragma unroll
            for (int a = 0; a < D; ++a) { up[a] = (j[a] + (CT)0.5 * F[a]) / rho; uu += up[a] * up[a]; }
            const CT Gm3 = K.Gamma3 * mu_phi;
            // sum of g^eq over the moving velocities, by lattice isotropy
            // (sum_{i != 0} w_i = 1 - w_0, sum w_i (c_i.u)^2 = u.u/3)
            const CT w0 = (CT)L::w(L::REST);
            const CT others = ((CT)1 - w0) * Gm3 + (CT)1.5 * w0 * phi * uu;
            const CT itg = K.inv_tau_g;
            ST *gd = reinterpret_cast<ST *>(A.gdst);
            // opposite velocities (i, Q-1-i) share w_i and the even part of g^eq;
            // c.u changes sign: g^eq = even +- odd
#pragma unroll
            for (int i = 0; i < L::REST; ++i) {
                const int io = Q - 1 - i;
                CT cu = 0;
#pragma unroll
                for (int a = 0; a < D; ++a)
                    if (L::c(i, a)) cu += (CT)L::c(i, a) * up[a];
                const CT wi = (CT)L::w(i);
                const CT even = wi * (Gm3 + phi * ((CT)4.5 * cu * cu - (CT)1.5 * uu));
                const CT odd = wi * (CT)3 * phi * cu;
                const CT gi = pull(gs, nb, P.N, i), gio = pull(gs, nb, P.N, io);
                gd[(long long)i * P.N + n] = gi - (gi - (even + odd)) * itg;
                gd[(long long)io * P.N + n] = gio - (gio - (even - odd)) * itg;
            }
            {
                const CT gi = pull(gs, nb, P.N, L::REST);
                gd[(long long)L::REST * P.N + n] = gi - (gi - (phi - others)) * itg;
            }

            CT uF[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) {
                uF[a] = u[a] + F[a] / rho;
                if (!(fabs(u[a]) < (CT)1) || !(fabs(uF[a]) < (CT)1)) bad |= ERR_VEL;
            }
            // equilibrium factors at u and at u + F/rho
            CT e[3][3], eF[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a < D) { eq_factors<CT>(u[a], e[a]); eq_factors<CT>(uF[a], eF[a]); }
                else { e[a][0] = 0; e[a][1] = 1; e[a][2] = 0; eF[a][0] = 0; eF[a][1] = 1; eF[a][2] = 0; }
            }
            // second moments of f^eq from the factor moments M0 = sum e, M1 = sum c e, M2 = sum c^2 e
            CT M0[3], M1[3], M2[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                M0[a] = e[a][0] + e[a][1] + e[a][2];
                M1[a] = e[a][2] - e[a][0];
                M2[a] = e[a][2] + e[a][0];
            }
            CT dPi[6];
            dPi[0] = Pi[0] - rho * M2[0] * M0[1] * M0[2];
            dPi[1] = Pi[1] - rho * M0[0] * M2[1] * M0[2];
            dPi[2] = (D == 3) ? Pi[2] - rho * M0[0] * M0[1] * M2[2] : (CT)0;
            dPi[3] = Pi[3] - rho * M1[0] * M1[1] * M0[2];
            dPi[4] = (D == 3) ? Pi[4] - rho * M1[0] * M0[1] * M1[2] : (CT)0;
            dPi[5] = (D == 3) ? Pi[5] - rho * M0[0] * M1[1] * M1[2] : (CT)0;
            const CT tr = dPi[0] + dPi[1] + dPi[2];
            const CT dev[3] = {dPi[0] - tr / (CT)D, dPi[1] - tr / (CT)D, dPi[2] - tr / (CT)D};

            // entropic scalar products <ds|dh>, <dh|dh> (weights 1/f^eq)
            CT sh = 0, hh = 0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const CT fi = fq[i * NT];
                const CT feq = rho * e[0][L::cx(i) + 1] * e[1][L::cy(i) + 1] * e[2][L::cz(i) + 1];
                const CT ds = ds_of(i, dev, dPi);
                const CT dh = fi - feq - ds;
                const CT r = (CT)1 / feq;
                // <ds|dh> has terms only where ds != 0 (one or two non-zero components of c_i)
                if (L::nnz(i) == 1 || L::nnz(i) == 2) sh += ds * dh * r;
                hh += dh * dh * r;
            }
            // stabiliser gamma = 1/beta - (2 - 1/beta) <ds|dh>/<dh|dh>, applied
            // as beta gamma = 1 - (2 beta - 1) <ds|dh>/<dh|dh> (gamma = 2, i.e.
            // beta gamma = 2 beta, when <dh|dh> vanishes)
            CT gb = hh > (CT)1e-30 * rho * rho ? (CT)1 - (CT)P.c_gb * (sh / hh) : (CT)2 * K.beta;
            if constexpr (EXACT) {
                // exact root of the entropy condition, from the closed form
                if (hh > (CT)1e-30 * rho * rho) {
                    auto parts = [&](int i, CT &fe, CT &dsv, CT &dh) {
                        fe = rho * e[0][L::cx(i) + 1] * e[1][L::cy(i) + 1] * e[2][L::cz(i) + 1];
                        dsv = ds_of(i, dev, dPi);
                        dh = fq[i * NT] - fe - dsv;
                    };
                    CT t = (CT)1 - gb;
                    const int rc = gamma_root<CT, Q>(parts, K.beta, t, (CT)1e-13, (CT)1e-15);
                    if (rc > 0) gb = (CT)1 - t;
                    else if (rc < 0) atomicAdd(P.gfall, 1ull);
                }
            }
            const CT bet = K.beta;
            if (!isfinite(gb)) bad |= ERR_NAN;
            ST *fd = reinterpret_cast<ST *>(A.fdst);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const CT fi = fq[i * NT];
                const CT feq = rho * e[0][L::cx(i) + 1] * e[1][L::cy(i) + 1] * e[2][L::cz(i) + 1];
                const CT feqF = rho * eF[0][L::cx(i) + 1] * eF[1][L::cy(i) + 1] * eF[2][L::cz(i) + 1];
                const CT ds = ds_of(i, dev, dPi);
                const CT dh = fi - feq - ds;
                fd[(long long)i * P.N + n] = fi - ((CT)2 * bet * ds + gb * dh) + (feqF - feq);
            }
            if (bad) raise_err(P.err, bad);
        }
    }

    // FP32 storage, step mode: the collision of one node over the pairs of
    // opposite velocities (k, Q-1-k), k < REST, in packed FP32x2 arithmetic.
    // The two members of a pair share w_i and Delta s_i; their equilibria are
    // the same products of the one-dimensional factors with c reversed, their
    // g equilibria differ in the sign of c.u, and they enter the odd moments
    // through their difference and the even moments through their sum.
    // The f pulls arrive in this thread's column of the stash (copies started
    // by node()) and stay there for the gamma and output passes; the g pulls
    // are all issued before the f moments are formed.
    __device__ static void collide_pairs(const DevParams &P, const LaunchArgs &A, const ST *gs, const Nbr &nb,
                                         float f0, float2 *stash2, long long n, float rho, float phi, float mu_phi,
                                         const float F[3])
    {
        constexpr int NP = L::REST;
        const Coef<float> &K = P.cf;
        const float shift = K.rho_ref;
        float2 gp[NP];  // (g_{Q-1-k}, g_k)
#pragma unroll
        for (int k = 0; k < NP; ++k) gp[k] = make_float2(pull(gs, nb, P.N, Q - 1 - k), pull(gs, nb, P.N, k));
        cp_async_wait_all();
        auto didx = [&](int i) -> long long {
            if (FAST) return (long long)((unsigned)i * (unsigned)P.N + (unsigned)n);
            return (long long)i * P.N + n;
        };

        // ---- pull f: mass, momentum and second moments
        float fsum = 0.f;
        float j[3] = {0.f, 0.f, 0.f};
        float Pi[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // xx yy zz xy xz yz
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 fp = stash2[k * NT];
            const float fa = fp.x, fb = fp.y;
            const float sp = fa + fb, dp = fa - fb;
            fsum += sp;
            if (L::cx(k)) { j[0] += (float)L::cx(k) * dp; Pi[0] += sp; }
            if (L::cy(k)) { j[1] += (float)L::cy(k) * dp; Pi[1] += sp; }
            if (D == 3 && L::cz(k)) { j[2] += (float)L::cz(k) * dp; Pi[2] += sp; }
            if (L::cx(k) * L::cy(k)) Pi[3] += (float)(L::cx(k) * L::cy(k)) * sp;
            if (D == 3 && L::cx(k) * L::cz(k)) Pi[4] += (float)(L::cx(k) * L::cz(k)) * sp;
            if (D == 3 && L::cy(k) * L::cz(k)) Pi[5] += (float)(L::cy(k) * L::cz(k)) * sp;
        }
        fsum += f0;  // rho - rho_ref as pulled
        const float cs2 = 1.f / 3.f;
        // the shift w_i rho_ref adds rho_ref c_s^2 to each diagonal second moment
        Pi[0] = fmaf(shift, cs2, Pi[0]);
        Pi[1] = fmaf(shift, cs2, Pi[1]);
        if (D == 3) Pi[2] = fmaf(shift, cs2, Pi[2]);

        unsigned bad = 0;
        if (!(rho > 0.f)) bad |= ERR_RHO;
        const float ir = rcp_nr(rho);
        float u[3] = {0.f, 0.f, 0.f}, up[3] = {0.f, 0.f, 0.f}, uF[3] = {0.f, 0.f, 0.f};
        float uu = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            u[a] = j[a] * ir;
            up[a] = fmaf(0.5f, F[a], j[a]) * ir;  // velocity with half the force (Eq. for the g equilibrium)
            uF[a] = fmaf(F[a], ir, u[a]);         // u + F/rho (exact-difference forcing)
            uu = fmaf(up[a], up[a], uu);
            if (!(fabsf(u[a]) < 1.f) || !(fabsf(uF[a]) < 1.f)) bad |= ERR_VEL;
        }

        // ---- g: BGK towards g^eq_i = w_i [Gm3 - 1.5 phi u.u + cu (3 phi + 4.5 phi cu)],
        // cu = c_i.u; the pair's second member has -cu.  The rest population
        // closes the node's phase-field sum.
        {
            const float2 G0 = bc2(fmaf(-1.5f * phi, uu, K.Gamma3 * mu_phi));
            const float2 P3 = bc2(3.f * phi), P45 = bc2(4.5f * phi), IT = bc2(K.inv_tau_g);
            float2 U2[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) U2[a] = make_float2(up[a], -up[a]);
            float2 goth = bc2(0.f);
            float *gd = reinterpret_cast<float *>(A.gdst);
            float sG[3], sN[3];  // carried moments: row groups of k and of Q-1-k
            // pair (kp, k), kp = Q-1-k: the member kp has a positive last
            // non-zero component of c, so c.u is U2 of that axis plus or minus
            // the others
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const int kp = Q - 1 - k;
                float2 cu = bc2(0.f);
                bool first = true;
#pragma unroll
                for (int a = D - 1; a >= 0; --a) {
                    const int ca = L::c(kp, a);
                    if (!ca) continue;
                    cu = first ? U2[a] : (ca > 0 ? add2(cu, U2[a]) : sub2(cu, U2[a]));
                    first = false;
                }
                const float2 geq = mul2(bc2((float)L::w(k)), fma2(cu, fma2(P45, cu, P3), G0));
                const float2 g2 = gp[k];
                const float2 go = fma2(IT, sub2(geq, g2), g2);
                goth = add2(goth, go);
                gd[didx(kp)] = go.x;
                gd[didx(k)] = go.y;
                if constexpr (MOM) {
                    // k = c_x + 1 + 3 (cy + 1) + 9 (cz + 1): the pairs k of one
                    // row group complete it and the opposite group
                    const int jx = k % 3;
                    sG[jx] = go.y;
                    sN[2 - jx] = go.x;
                    if (jx == 2) {
                        scatter_row(A.m_acc + P.N, nb, L::cy(k), L::cz(k), sG[0], sG[1], sG[2]);
                        scatter_row(A.m_acc + P.N, nb, L::cy(kp), L::cz(kp), sN[0], sN[1], sN[2]);
                    }
                }
            }
            const float grest = phi - (goth.x + goth.y);
            gd[didx(L::REST)] = grest;
            if constexpr (MOM) scatter_row(A.m_acc + P.N, nb, 0, 0, sG[0], grest, sN[2]);
        }

        // ---- equilibrium factors at u; second moments of f^eq
        float e[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a < D) eq_factors_f(u[a], e[a]);
            else { e[a][0] = 0.f; e[a][1] = 1.f; e[a][2] = 0.f; }
        }
        float M0[3], M1[3], M2[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            M0[a] = e[a][0] + e[a][1] + e[a][2];
            M1[a] = e[a][2] - e[a][0];
            M2[a] = e[a][2] + e[a][0];
        }
        float dPi[6];
        dPi[0] = Pi[0] - rho * M2[0] * M0[1] * M0[2];
        dPi[1] = Pi[1] - rho * M0[0] * M2[1] * M0[2];
        dPi[2] = (D == 3) ? Pi[2] - rho * M0[0] * M0[1] * M2[2] : 0.f;
        dPi[3] = Pi[3] - rho * M1[0] * M1[1] * M0[2];
        dPi[4] = (D == 3) ? Pi[4] - rho * M1[0] * M0[1] * M1[2] : 0.f;
        dPi[5] = (D == 3) ? Pi[5] - rho * M0[0] * M1[1] * M1[2] : 0.f;
        const float tr = (dPi[0] + dPi[1] + dPi[2]) * (1.f / (float)D);
        // Delta s: 1/2 of the deviatoric normal stress on the velocities along
        // one axis, +-1/4 of the shear stress on the velocities in one plane
        float2 DS1[3], DS2[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            DS1[a] = bc2(0.5f * (dPi[a] - tr));
            DS2[a] = bc2(0.25f * dPi[3 + a]);
        }
        // pair factors: X[c] = rho (e_x[c], e_x[-c]), Y[c], Z[c] likewise
        float2 X[3], Y[3], Z[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X[c] = make_float2(rho * e[0][c], rho * e[0][2 - c]);
            Y[c] = make_float2(e[1][c], e[1][2 - c]);
            Z[c] = make_float2(e[2][c], e[2][2 - c]);
        }
        auto feq2 = [&](int k, const float2 *Xa, const float2 *Ya, const float2 *Za) -> float2 {
            const float2 v = mul2(Xa[L::cx(k) + 1], Ya[L::cy(k) + 1]);
            return D == 3 ? mul2(v, Za[L::cz(k) + 1]) : v;
        };
        // Delta h = Delta - Delta s of pair k, Delta = f - f^eq
        auto dh2 = [&](int k, float2 dl) -> float2 {
            if (L::nnz(k) == 1) return sub2(dl, DS1[L::cx(k) ? 0 : (L::cy(k) ? 1 : 2)]);
            if (L::nnz(k) == 2) {
                const int pl = L::cz(k) == 0 ? 0 : (L::cy(k) == 0 ? 1 : 2);
                const int sg = L::cz(k) == 0 ? L::cx(k) * L::cy(k) : (L::cy(k) == 0 ? L::cx(k) * L::cz(k)
                                                                                  : L::cy(k) * L::cz(k));
                return sg > 0 ? sub2(dl, DS2[pl]) : add2(dl, DS2[pl]);
            }
            return dl;
        };

        // ---- entropic scalar products <ds|dh> and <dh|dh> (weights 1/f^eq).
        // Delta = f - f^eq replaces f in the stash: the output pass needs no
        // f^eq(u) then.
        float2 hh2 = bc2(0.f), shp = bc2(0.f), shn = bc2(0.f);  // <ds|dh>: terms of Delta s sign +, -
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 f2 = stash2[k * NT];
            const float2 fe = feq2(k, X, Y, Z);
            const float2 dl = sub2(f2, sub2(fe, bc2((float)L::w(k) * shift)));
            stash2[k * NT] = dl;
            const float2 dh = dh2(k, dl);
            const float2 t = mul2(dh, make_float2(rcp_approx(fe.x), rcp_approx(fe.y)));  // weight 1/f^eq
            hh2 = fma2(dh, t, hh2);
            if (L::nnz(k) == 1) {
                shp = fma2(DS1[L::cx(k) ? 0 : (L::cy(k) ? 1 : 2)], t, shp);
            } else if (L::nnz(k) == 2) {
                const int pl = L::cz(k) == 0 ? 0 : (L::cy(k) == 0 ? 1 : 2);
                const int sg = L::cz(k) == 0 ? L::cx(k) * L::cy(k) : (L::cy(k) == 0 ? L::cx(k) * L::cz(k)
                                                                                  : L::cy(k) * L::cz(k));
                if (sg > 0) shp = fma2(DS2[pl], t, shp);
                else shn = fma2(DS2[pl], t, shn);
            }
        }
        const float fe0 = rho * e[0][1] * e[1][1] * e[2][1];
        const float dl0 = f0 - (fe0 - (float)L::w(L::REST) * shift);
        const float hh = fmaf(dl0 * dl0, rcp_approx(fe0), hh2.x + hh2.y);
        const float sh = (shp.x + shp.y) - (shn.x + shn.y);

        // ---- stabiliser: beta gamma = 1 - (2 beta - 1) <ds|dh>/<dh|dh> from the
        // FP32 ratio q, with 2 beta - 1 as two floats and one rounding (the
        // value of the FP64 expression rounded to FP32); gamma = 2, beta gamma
        // = 2 beta, when <dh|dh> vanishes
        const bool has_q = hh > 1e-30f * rho * rho;
        const float q = has_q ? sh * rcp_nr(hh) : 0.f;
        float gb = 2.f * K.beta;
        if constexpr (MODE == MODE_STEP_G64) {
            double gbd = 2.0 * P.beta;
            // variant: both scalar products accumulated in FP64 from the
            // FP32 Delta s, Delta h and the FP32 weights 1/f^eq
            double hhd = 0.0, shd = 0.0;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float2 dh = dh2(k, stash2[k * NT]);
                const float2 fe = feq2(k, X, Y, Z);
                const double tx = (double)dh.x * (double)rcp_approx(fe.x);
                const double ty = (double)dh.y * (double)rcp_approx(fe.y);
                hhd = fma((double)dh.x, tx, fma((double)dh.y, ty, hhd));
                float dsk = 0.f;
                if (L::nnz(k) == 1) {
                    dsk = DS1[L::cx(k) ? 0 : (L::cy(k) ? 1 : 2)].x;
                } else if (L::nnz(k) == 2) {
                    const int pl = L::cz(k) == 0 ? 0 : (L::cy(k) == 0 ? 1 : 2);
                    const int sg = L::cz(k) == 0 ? L::cx(k) * L::cy(k)
                                                 : (L::cy(k) == 0 ? L::cx(k) * L::cz(k) : L::cy(k) * L::cz(k));
                    dsk = sg > 0 ? DS2[pl].x : -DS2[pl].x;
                }
                if (L::nnz(k) == 1 || L::nnz(k) == 2) shd = fma((double)dsk, tx + ty, shd);
            }
            hhd = fma((double)dl0 * (double)dl0, (double)rcp_approx(fe0), hhd);
            if (hhd > 1e-30 * (double)rho * (double)rho) gbd = fma(-P.c_gb, shd / hhd, 1.0);
            gb = (float)gbd;
        } else {
            if (has_q) gb = fmaf(-P.c_gb_hi, q, fmaf(-P.c_gb_lo, q, 1.f));
        }
        if constexpr (EXACT) {
            // exact root of the entropy condition, from the closed form, in
            // FP32 on the stashed Delta of each pair
            if (has_q) {
                auto ds_pair = [&](int k) -> float {
                    if (L::nnz(k) == 1) return DS1[L::cx(k) ? 0 : (L::cy(k) ? 1 : 2)].x;
                    if (L::nnz(k) == 2) {
                        const int pl = L::cz(k) == 0 ? 0 : (L::cy(k) == 0 ? 1 : 2);
                        const int sg = L::cz(k) == 0 ? L::cx(k) * L::cy(k)
                                                     : (L::cy(k) == 0 ? L::cx(k) * L::cz(k) : L::cy(k) * L::cz(k));
                        return sg > 0 ? DS2[pl].x : -DS2[pl].x;
                    }
                    return 0.f;
                };
                auto parts = [&](int i, float &fe, float &dsv, float &dh) {
                    if (i == L::REST) { fe = fe0; dsv = 0.f; dh = dl0; return; }
                    const int k = i < L::REST ? i : Q - 1 - i;
                    const float2 fe2 = feq2(k, X, Y, Z);
                    const float2 dl2 = stash2[k * NT];
                    dsv = ds_pair(k);
                    fe = i < L::REST ? fe2.x : fe2.y;
                    dh = (i < L::REST ? dl2.x : dl2.y) - dsv;
                };
                // t = 1 - beta gamma = (2 beta - 1) q, the closed form
                float t = fmaf(P.c_gb_hi, q, P.c_gb_lo * q);
                const int rc = gamma_root<float, Q>(parts, K.beta, t, 1e-5f, 1e-7f);
                if (rc > 0) gb = 1.f - t;
                else if (rc < 0) atomicAdd(P.gfall, 1ull);
            }
        }
        if (!isfinite(gb)) bad |= ERR_NAN;

        // ---- output: f - beta (2 Delta s + gamma Delta h) + f^eq(u + F/rho) - f^eq(u)
        //   = (1 - beta gamma) Delta + f^eq(u + F/rho) + (beta gamma - 2 beta) Delta s,
        // stored shifted by -w_i rho_ref.  The rest population closes the
        // node's mass to the pulled mass.
        float eF[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a < D) eq_factors_f(uF[a], eF[a]);
            else { eF[a][0] = 0.f; eF[a][1] = 1.f; eF[a][2] = 0.f; }
        }
        float2 XF[3], YF[3], ZF[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            XF[c] = make_float2(rho * eF[0][c], rho * eF[0][2 - c]);
            YF[c] = make_float2(eF[1][c], eF[1][2 - c]);
            ZF[c] = make_float2(eF[2][c], eF[2][2 - c]);
        }
        const float2 OMG = bc2(1.f - gb), PG = bc2(gb - 2.f * K.beta), NG = bc2(2.f * K.beta - gb);
        float *fd = reinterpret_cast<float *>(A.fdst);
        float2 oth = bc2(0.f);
        float sG[3], sN[3];  // carried moments: row groups of k and of Q-1-k
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float2 out = fma2(OMG, stash2[k * NT], sub2(feq2(k, XF, YF, ZF), bc2((float)L::w(k) * shift)));
            if (L::nnz(k) == 1) {
                out = fma2(PG, DS1[L::cx(k) ? 0 : (L::cy(k) ? 1 : 2)], out);
            } else if (L::nnz(k) == 2) {
                const int pl = L::cz(k) == 0 ? 0 : (L::cy(k) == 0 ? 1 : 2);
                const int sg = L::cz(k) == 0 ? L::cx(k) * L::cy(k) : (L::cy(k) == 0 ? L::cx(k) * L::cz(k)
                                                                                  : L::cy(k) * L::cz(k));
                out = fma2(sg > 0 ? PG : NG, DS2[pl], out);
            }
            oth = add2(oth, out);
            fd[didx(k)] = out.x;
            fd[didx(Q - 1 - k)] = out.y;
            if constexpr (MOM) {
                const int jx = k % 3;
                sG[jx] = out.x;
                sN[2 - jx] = out.y;
                if (jx == 2) {
                    scatter_row(A.m_acc, nb, L::cy(k), L::cz(k), sG[0], sG[1], sG[2]);
                    scatter_row(A.m_acc, nb, L::cy(Q - 1 - k), L::cz(Q - 1 - k), sN[0], sN[1], sN[2]);
                }
            }
        }
        const float frest = fsum - (oth.x + oth.y);
        fd[didx(L::REST)] = frest;
        if constexpr (MOM) scatter_row(A.m_acc, nb, 0, 0, sG[0], frest, sN[2]);

        if (bad) raise_err(P.err, bad);
    }

    // Delta s_i: the population vector whose natural moments vanish except
    // the deviatoric second moments of Delta (dual basis of {1, c, c^2} per
    // axis; trace left in the higher-order part).
    __device__ static __forceinline__ CT ds_of(int i, const CT dev[3], const CT dPi[6])
    {
        const int k = L::nnz(i);
        if (k == 1) {
            if (L::cx(i)) return (CT)0.5 * dev[0];
            if (L::cy(i)) return (CT)0.5 * dev[1];
            return (CT)0.5 * dev[2];
        }
        if (k == 2) {
            if (L::cz(i) == 0) return (CT)(0.25 * L::cx(i) * L::cy(i)) * dPi[3];
            if (L::cy(i) == 0) return (CT)(0.25 * L::cx(i) * L::cz(i)) * dPi[4];
            return (CT)(0.25 * L::cy(i) * L::cz(i)) * dPi[5];
        }
        return (CT)0;
    }

    // g^eq_i, i != rest: w_i [3 Gamma mu_phi + 3 phi c.u + phi (9/2 (c.u)^2 - 3/2 u.u)]
    __device__ static __forceinline__ CT geq_of(int i, CT Gm3, CT phi, const CT up[3], CT uu)
    {
        CT cu = 0;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (L::c(i, a)) cu += (CT)L::c(i, a) * up[a];
        return (CT)L::w(i) * (Gm3 + (CT)3 * phi * cu + phi * ((CT)4.5 * cu * cu - (CT)1.5 * uu));
    }

    __device__ static void init_node(const DevParams &P, const LaunchArgs &A, long long n, int x, int y, int m,
                                     CT rho, CT phi, CT mu_phi, const CT F[3])
    {
        const int PX = P.nx, PY = (D == 3 ? P.ny : 1), PM = (D == 3 ? P.nz : P.ny);
        const CT shift = coef<CT>(P).rho_ref;
        CT u[3] = {0, 0, 0}, us[3] = {0, 0, 0}, uu = 0;
        unsigned bad = 0;
        if (!(rho > (CT)0)) bad |= ERR_RHO;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            u[a] = (CT)A.in_u[(long long)a * P.N + n];
            us[a] = u[a] - F[a] / ((CT)2 * rho);
            uu += u[a] * u[a];
            if (!(fabs(us[a]) < (CT)1)) bad |= ERR_VEL;
        }
        CT e[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a < D) eq_factors<CT>(us[a], e[a]);
            else { e[a][0] = 0; e[a][1] = 1; e[a][2] = 0; }
        }
        const CT Gm3 = coef<CT>(P).Gamma3 * mu_phi;
        CT others = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (i != L::REST) others += geq_of(i, Gm3, phi, u, uu);
        ST *fd = reinterpret_cast<ST *>(A.fdst);
        ST *gd = reinterpret_cast<ST *>(A.gdst);
        const int bx = P.bc[0], by = (D == 3 ? P.bc[1] : 0), bm = (D == 3 ? P.bc[2] : P.bc[1]);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            CT feq = rho * e[0][L::cx(i) + 1] * e[1][L::cy(i) + 1] * e[2][L::cz(i) + 1];
            if (StoreTraits<ST>::shifted) feq -= (CT)L::w(i) * shift;
            const CT ge = (i == L::REST) ? phi - others : geq_of(i, Gm3, phi, u, uu);
            // place the value where the first pull of node n in direction i reads it
            int sx = x - L::pX(i), sy = y - L::pY(i), sm = m - L::pM(i);
            bool bb = false;
            if (sx < 0) { if (bx) bb = true; else sx += PX; } else if (sx >= PX) { if (bx) bb = true; else sx -= PX; }
            if (D == 3) { if (sy < 0) { if (by) bb = true; else sy += PY; } else if (sy >= PY) { if (by) bb = true; else sy -= PY; } }
            if (sm < 0) { if (bm) bb = true; else sm += PM; } else if (sm >= PM) { if (bm) bb = true; else sm -= PM; }
            if constexpr (!FAST) {
                // a solid source: the node's own reversed slot (bounce-back)
                if (!bb && P.solid &&
                    P.solid[(long long)sx + (long long)PX * ((long long)sy + (long long)PY * sm)])
                    bb = true;
            }
            const long long k = bb ? (long long)(Q - 1 - i) * P.N + n
                                   : (long long)i * P.N + (long long)sx + (long long)PX * ((long long)sy + (long long)PY * sm);
            fd[k] = (ST)feq;
            gd[k] = (ST)ge;
        }
        if (bad) raise_err(P.err, bad);
    }

    __device__ static void fields_node(const DevParams &P, const LaunchArgs &A, long long n, CT rho, CT phi,
                                       const CT j[3], const CT F[3], const CT gr[3], const CT gf[3], CT mu_rho,
                                       CT mu_phi)
    {
        if (A.out_rho) A.out_rho[n] = (double)rho;
        if (A.out_phi) A.out_phi[n] = (double)phi;
        if (A.out_u) {
#pragma unroll
            for (int a = 0; a < D; ++a) A.out_u[(long long)a * P.N + n] = (double)((j[a] + (CT)0.5 * F[a]) / rho);
        }
        if (A.out_p) {
            double rr = 0, pp = 0, rp = 0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                rr += (double)gr[a] * (double)gr[a];
                pp += (double)gf[a] * (double)gf[a];
                rp += (double)gr[a] * (double)gf[a];
            }
            const double fI = P.AI * rr + P.BI * pp + P.XI * rp;
            A.out_p[n] = (double)rho * (double)mu_rho + (double)phi * (double)mu_phi
                         - f_bulk(P, (double)rho, (double)phi) - fI;
        }
    }
};

// Minimum resident CTAs per SM requested from the register allocator.
// D3Q27 FP32: 16 warps per SM (2 CTAs of 32 x 8, 4 of 32 x 4; up to 128
// registers).  Measured on the carried-moment step at 256^3: 32 x 4 tiles at
// 4 CTAs per SM 8300 MLUPS, at 5 (96 registers) 8267, 32 x 8 at 2 7735 and
// at 3 (80 registers, spills) 7360, 32 x 16 at 1 6706, 32 x 2 at 8 7140.
#ifndef TEL_D3_FP32_WARPS_PER_SM
#define TEL_D3_FP32_WARPS_PER_SM 16
#endif
// D2Q9 single lattices: measured with 4 (2 CTAs of rows of 64 requested,
// 98 registers) and 24 warps per SM (80 registers): 7961 / 14620 MLUPS and
// 7594 / 14762 MLUPS on 512^2 / 2048^2 FP32, so 4 stays.
#ifndef TEL_D2Q9_WARPS_PER_SM
#define TEL_D2Q9_WARPS_PER_SM 4
#endif
// With the vector phase A the row's loads are in flight together and the
// kernel asks for more registers (130 unbounded), so the request is set
// separately: 18 warps per SM (96 registers, no spills) measured 10250 /
// 18366 MLUPS on 512^2 / 2048^2 FP32, against 10595 / 15150 with 4 and
// 9819 / 18096 with 24.
#ifndef TEL_D2Q9_VEC_WARPS_PER_SM
#define TEL_D2Q9_VEC_WARPS_PER_SM 18
#endif
// FP64: one CTA; FP32: TEL_D3_FP32_WARPS_PER_SM or TEL_D2Q9_(VEC_)WARPS_PER_SM
// warps per SM requested
template <int D, int NTH, typename ST, bool VEC> struct KernelMinBlocks {
    static constexpr int value = 1;
};
template <int NTH, bool VEC> struct KernelMinBlocks<3, NTH, float, VEC> {
    static constexpr int value = TEL_D3_FP32_WARPS_PER_SM * 32 / NTH;
};
template <int NTH, bool VEC> struct KernelMinBlocks<2, NTH, float, VEC> {
    static constexpr int value = (VEC ? TEL_D2Q9_VEC_WARPS_PER_SM : TEL_D2Q9_WARPS_PER_SM) * 32 / NTH;
};

template <int D, int TX, int TY, typename ST, int MODE, bool FAST, bool VEC = false, bool MOM = false>
__global__ void __launch_bounds__(TX * TY, (KernelMinBlocks<D, TX * TY, ST, VEC>::value))
    fused_kernel(const DevParams P, const LaunchArgs A)
{
    Fused<D, TX, TY, ST, MODE, FAST, VEC, MOM>::run(P, A);
}

// Batched persistent D2Q9 step: each CTA walks a work list of (case, tile,
// chunk) items over many independent lattices; each case's parameter block
// and buffers are copied into shared memory before its item runs.
// Resident CTAs per SM requested for the batched kernel.  FP32: 24 warps
// per SM (24 CTAs of width 32, 12 of width 64), which caps the registers at
// 80-85 per thread without spills (measured with width 32 on the 256-case
// workload: 15640 MLUPS, against 14168 with 2 CTAs requested (115 registers,
// 17 CTAs resident) and 13553 with 32 (64 registers, small spills)).  With
// the vector phase A (80 registers, 16-24 bytes of spills): 18000 MLUPS at
// 24 warps, 17690 at 20 and 17400 at 16.  FP64: 2, its collision needs its
// registers.
#ifndef TEL_BATCH_WARPS_PER_SM
#define TEL_BATCH_WARPS_PER_SM 24
#endif
template <int TX, typename ST> struct BatchMinBlocks { static constexpr int value = 2; };
template <int TX> struct BatchMinBlocks<TX, float> { static constexpr int value = TEL_BATCH_WARPS_PER_SM * 32 / TX; };

template <int TX, typename ST, bool FAST, bool VEC = false>
__global__ void __launch_bounds__(TX, (BatchMinBlocks<TX, ST>::value))
    batch_kernel(const DevParams *Ps, const LaunchArgs *As, const int4 *items, int nitems)
{
    __shared__ DevParams Psh;
    __shared__ LaunchArgs Ash;
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const int4 it = items[w];  // (case, tile along x, chunk along y, -)
        __syncthreads();           // the previous item is done with shared memory
        {
            const int *src = reinterpret_cast<const int *>(Ps + it.x);
            int *dst = reinterpret_cast<int *>(&Psh);
            for (int k = threadIdx.x; k < (int)(sizeof(DevParams) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
            const int *sa = reinterpret_cast<const int *>(As + it.x);
            int *da = reinterpret_cast<int *>(&Ash);
            for (int k = threadIdx.x; k < (int)(sizeof(LaunchArgs) / sizeof(int)); k += blockDim.x) da[k] = sa[k];
        }
        __syncthreads();
        Fused<2, TX, 1, ST, MODE_STEP, FAST, VEC>::run_tile(Psh, Ash, it.y, 0, it.z);
    }
}

// Batched launcher (tel_d2q9.cu): tx in {32, 64}; grid = persistent CTAs;
// vec: vector phase A (FP32, fast, every case with nx % 4 == 0).
cudaError_t launch_d2q9_batch(int precision, int tx, bool fast, bool vec, const DevParams *Ps,
                              const LaunchArgs *As, const int4 *items, int nitems, int grid, cudaStream_t s);
// Resident CTAs per SM of the batched kernel with shape tx.
int batch_blocks_per_sm(int precision, int tx, bool fast, bool vec);

// Tile shapes and launcher (defined per lattice in tel_d2q9.cu / tel_d3q27.cu).
cudaError_t launch_d2q9(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s);
cudaError_t launch_d3q27(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s);
// Tile of the D3Q27 step with carried moments (TX = 32 x TY nodes of the
// xy plane): a lattice takes that path only if nx % 32 == 0 and ny % TY == 0.
int d3q27_carried_tile_y();

// Carried moments of a new state (D3Q27 FP32, periodic): m_out gets the
// sums of the populations each node pulls in the next step (rho - rho_ref,
// then phi), m_zero (2N floats) is cleared.
cudaError_t launch_d3q27_moments(const DevParams &P, const float *f, const float *g, float *m_out, float *m_zero,
                                 cudaStream_t s);

// Shift conversion of whole population arrays (FP32 mode state get/set).
cudaError_t launch_state_to_f64(int lattice, const float *src, double *dst, long long N, double shift,
                                cudaStream_t s);
cudaError_t launch_state_from_f64(int lattice, const double *src, float *dst, long long N, double shift,
                                  cudaStream_t s);

}  // namespace tel
