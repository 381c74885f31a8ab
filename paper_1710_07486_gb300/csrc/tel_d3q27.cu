// D3Q27 instantiation of the fused kernel: 32 x 8 tiles in the xy plane
// marching along z; also the FP32-shift conversions of whole state arrays.
#include "tel_launch.cuh"

#ifndef TEL_D3_TX
#define TEL_D3_TX 32
#endif
#ifndef TEL_D3_TY
#define TEL_D3_TY 8
#endif

namespace tel {
cudaError_t launch_d3q27(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    return launch_lattice<3, TEL_D3_TX, TEL_D3_TY>(precision, mode, P, A, s);
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
