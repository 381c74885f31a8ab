// tel_launch.cuh -- host launcher shared by the per-lattice translation units.
#pragma once

#include "tel_kernels.cuh"

namespace tel {

template <int D, int TX, int TY, typename ST, int MODE>
static cudaError_t launch_one(const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    typedef Fused<D, TX, TY, ST, MODE> K;
    static bool configured = false;  // per-instantiation: opt in to > 48 KB of shared memory
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(fused_kernel<D, TX, TY, ST, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int PX = P.nx, PY = (D == 3 ? P.ny : 1), PM = (D == 3 ? P.nz : P.ny);
    dim3 grid((PX + TX - 1) / TX, 1, 1);
    const int nch = (PM + P.chunk - 1) / P.chunk;
    if (D == 3) {
        grid.y = (PY + TY - 1) / TY;
        grid.z = nch;
    } else {
        grid.y = nch;
    }
    fused_kernel<D, TX, TY, ST, MODE><<<grid, K::NT, K::SMEM_BYTES, s>>>(P, A);
    return cudaGetLastError();
}

template <int D, int TX, int TY>
static cudaError_t launch_lattice(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    if (precision == 0) {
        if (mode == MODE_STEP) return launch_one<D, TX, TY, double, MODE_STEP>(P, A, s);
        if (mode == MODE_INIT) return launch_one<D, TX, TY, double, MODE_INIT>(P, A, s);
        return launch_one<D, TX, TY, double, MODE_FIELDS>(P, A, s);
    }
    if (mode == MODE_STEP) return launch_one<D, TX, TY, float, MODE_STEP>(P, A, s);
    if (mode == MODE_INIT) return launch_one<D, TX, TY, float, MODE_INIT>(P, A, s);
    return launch_one<D, TX, TY, float, MODE_FIELDS>(P, A, s);
}

}  // namespace tel
