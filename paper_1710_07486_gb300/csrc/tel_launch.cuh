// tel_launch.cuh -- host launcher shared by the per-lattice translation units.
#pragma once

#include "tel_kernels.cuh"
#include "tel_once.cuh"

namespace tel {

template <int D, int TX, int TY, typename ST, int MODE, bool FAST, bool VEC = false, bool MOM = false>
static cudaError_t launch_one(const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    typedef Fused<D, TX, TY, ST, MODE, FAST, VEC, MOM> K;
    static DeviceOnce once;  // per instantiation and device: opt in to > 48 KB of shared memory
    cudaError_t e = once.run([] {
        return cudaFuncSetAttribute(fused_kernel<D, TX, TY, ST, MODE, FAST, VEC, MOM>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM_BYTES);
    });
    if (e != cudaSuccess) return e;
    const int PX = P.nx, PY = (D == 3 ? P.ny : 1), PM = (D == 3 ? P.nz : P.ny);
    dim3 grid((PX + TX - 1) / TX, 1, 1);
    const int nch = (PM + P.chunk - 1) / P.chunk;
    if (D == 3) {
        grid.y = (PY + TY - 1) / TY;
        grid.z = nch;
    } else {
        grid.y = nch;
    }
    fused_kernel<D, TX, TY, ST, MODE, FAST, VEC, MOM><<<grid, K::NT, K::SMEM_BYTES, s>>>(P, A);
    return cudaGetLastError();
}

template <int D, int TX, int TY, bool FAST>
static cudaError_t launch_prec(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    if (precision == 0) {
        // FP64 storage sums everything in FP64 already
        if (mode == MODE_STEP || mode == MODE_STEP_G64) return launch_one<D, TX, TY, double, MODE_STEP, FAST>(P, A, s);
        if (mode == MODE_STEP_EXACT) return launch_one<D, TX, TY, double, MODE_STEP_EXACT, FAST>(P, A, s);
        if (mode == MODE_INIT) return launch_one<D, TX, TY, double, MODE_INIT, FAST>(P, A, s);
        return launch_one<D, TX, TY, double, MODE_FIELDS, FAST>(P, A, s);
    }
    if (mode == MODE_STEP || mode == MODE_STEP_EXACT || mode == MODE_STEP_G64) {
        // aligned four-node vectors in phase A (D3Q27 32 x 8 or D2Q9 rows of
        // 32 or 64, periodic, nx % 4 == 0)
        if constexpr (((D == 3 && TX == 32 && TY == 8) || (D == 2 && TY == 1 && (TX == 32 || TX == 64))) && FAST)
            if (P.nx % 4 == 0) {
                if (mode == MODE_STEP_EXACT) return launch_one<D, TX, TY, float, MODE_STEP_EXACT, FAST, true>(P, A, s);
                if (mode == MODE_STEP_G64) return launch_one<D, TX, TY, float, MODE_STEP_G64, FAST, true>(P, A, s);
                return launch_one<D, TX, TY, float, MODE_STEP, FAST, true>(P, A, s);
            }
        if (mode == MODE_STEP_EXACT) return launch_one<D, TX, TY, float, MODE_STEP_EXACT, FAST>(P, A, s);
        if (mode == MODE_STEP_G64) return launch_one<D, TX, TY, float, MODE_STEP_G64, FAST>(P, A, s);
        return launch_one<D, TX, TY, float, MODE_STEP, FAST>(P, A, s);
    }
    if (mode == MODE_INIT) return launch_one<D, TX, TY, float, MODE_INIT, FAST>(P, A, s);
    return launch_one<D, TX, TY, float, MODE_FIELDS, FAST>(P, A, s);
}

template <int D, int TX, int TY>
static cudaError_t launch_lattice(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    // fast pulls: no bounce-back axis, no solid node and 32-bit population indices
    const bool walls = P.bc[0] || P.bc[1] || (D == 3 && P.bc[2]) || P.solid != nullptr;
    const bool fast = !walls && (long long)Lat<D>::Q * P.N < (1LL << 31);
    if (fast) return launch_prec<D, TX, TY, true>(precision, mode, P, A, s);
    return launch_prec<D, TX, TY, false>(precision, mode, P, A, s);
}

}  // namespace tel
