// D3Q27 instantiation of the fused kernel: 32 x 8 tiles in the xy plane
// marching along z (32 x 4 for the step with carried moments); also the
// moments of a new state and the FP32-shift conversions of whole state arrays.
#include "tel_launch.cuh"

#ifndef TEL_D3_TX
#define TEL_D3_TX 32
#endif
#ifndef TEL_D3_TY
#define TEL_D3_TY 8
#endif
// carried moments: rows of 32 (one warp per row), 4 rows, 4 CTAs per SM
#ifndef TEL_D3_MOM_TY
#define TEL_D3_MOM_TY 4
#endif

namespace tel {
// The FP32 step with carried moments (A.m_read set): periodic fast path,
// full tiles only (every lane of a warp takes part in the row scatter).
static cudaError_t launch_carried(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    constexpr int TY = TEL_D3_MOM_TY;
    const bool fast = !P.bc[0] && !P.bc[1] && !P.bc[2] && P.solid == nullptr && 27LL * P.N < (1LL << 31);
    if (precision != 1 || !fast || P.nx % 32 != 0 || P.ny % TY != 0 || !A.m_acc || !A.m_zero)
        return cudaErrorInvalidValue;
    if (mode == MODE_STEP_EXACT) return launch_one<3, 32, TY, float, MODE_STEP_EXACT, true, false, true>(P, A, s);
    if (mode == MODE_STEP_G64) return launch_one<3, 32, TY, float, MODE_STEP_G64, true, false, true>(P, A, s);
    if (mode == MODE_STEP) return launch_one<3, 32, TY, float, MODE_STEP, true, false, true>(P, A, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_d3q27(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    if (A.m_read) return launch_carried(precision, mode, P, A, s);
    return launch_lattice<3, TEL_D3_TX, TEL_D3_TY>(precision, mode, P, A, s);
}
int d3q27_carried_tile_y() { return TEL_D3_MOM_TY; }

// Carried moments of a state: node n pulls f_i from n - c_i (periodic), so
// its rho - rho_ref and phi for the next step are the sums of the stored
// (shifted) f and of g over those sources; the buffer that the first step
// accumulates into is cleared.
__global__ void moments_kernel(const float *f, const float *g, float *m_out, float *m_zero, int nx, int ny, int nz)
{
    typedef Lat<3> L;
    const int N = nx * ny * nz;  // Q N < 2^31 on the periodic fast path
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
        float sf = 0.f, sg = 0.f;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            int sx = x - L::cx(i), sy = y - L::cy(i), sz = z - L::cz(i);
            if (sx < 0) sx += nx; else if (sx >= nx) sx -= nx;
            if (sy < 0) sy += ny; else if (sy >= ny) sy -= ny;
            if (sz < 0) sz += nz; else if (sz >= nz) sz -= nz;
            const int k = i * N + sx + nx * (sy + ny * sz);
            sf += __ldg(f + k);
            sg += __ldg(g + k);
        }
        m_out[n] = sf;
        m_out[N + n] = sg;
        m_zero[n] = 0.f;
        m_zero[N + n] = 0.f;
    }
}

cudaError_t launch_d3q27_moments(const DevParams &P, const float *f, const float *g, float *m_out, float *m_zero,
                                 cudaStream_t s)
{
    if ((long long)Lat<3>::Q * P.N >= (1LL << 31)) return cudaErrorInvalidValue;
    moments_kernel<<<152 * 8, 256, 0, s>>>(f, g, m_out, m_zero, P.nx, P.ny, P.nz);
    return cudaGetLastError();
}

// f_i = fbar_i + w_i shift (shift = 0 for g)
template <int D>
__global__ void to_f64_kernel(const float *src, double *dst, long long N, double shift)
{
    const long long total = (long long)Lat<D>::Q * N;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / N);
        double w = 0;
#pragma unroll
        for (int q = 0; q < Lat<D>::Q; ++q)
            if (q == i) w = Lat<D>::w(q);
        dst[k] = (double)src[k] + w * shift;
    }
}

template <int D>
__global__ void from_f64_kernel(const double *src, float *dst, long long N, double shift)
{
    const long long total = (long long)Lat<D>::Q * N;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / N);
        double w = 0;
#pragma unroll
        for (int q = 0; q < Lat<D>::Q; ++q)
            if (q == i) w = Lat<D>::w(q);
        dst[k] = (float)(src[k] - w * shift);
    }
}

cudaError_t launch_state_to_f64(int lattice, const float *src, double *dst, long long N, double shift,
                                cudaStream_t s)
{
    const int blocks = 152 * 8;
    if (lattice == 0) to_f64_kernel<2><<<blocks, 256, 0, s>>>(src, dst, N, shift);
    else to_f64_kernel<3><<<blocks, 256, 0, s>>>(src, dst, N, shift);
    return cudaGetLastError();
}

cudaError_t launch_state_from_f64(int lattice, const double *src, float *dst, long long N, double shift,
                                  cudaStream_t s)
{
    const int blocks = 152 * 8;
    if (lattice == 0) from_f64_kernel<2><<<blocks, 256, 0, s>>>(src, dst, N, shift);
    else from_f64_kernel<3><<<blocks, 256, 0, s>>>(src, dst, N, shift);
    return cudaGetLastError();
}
}  // namespace tel
