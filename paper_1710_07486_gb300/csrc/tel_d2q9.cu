// D2Q9 instantiation of the fused kernel: rows of 64 nodes along x marching
// along y.
#include "tel_launch.cuh"

namespace tel {
cudaError_t launch_d2q9(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    return launch_lattice<2, 64, 1>(precision, mode, P, A, s);
}

// Resident CTAs per SM of the single-lattice step kernel that launch_d2q9
// picks for this storage and path (MODE_STEP).
template <typename ST, bool FAST, bool VEC>
static cudaError_t step_occupancy(int *out)
{
    typedef Fused<2, 64, 1, ST, MODE_STEP, FAST, VEC> K;
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<2, 64, 1, ST, MODE_STEP, FAST, VEC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fused_kernel<2, 64, 1, ST, MODE_STEP, FAST, VEC>,
                                                         K::NT, K::SMEM_BYTES);
}

cudaError_t d2q9_step_ctas_per_sm(int precision, bool fast, bool vec, int *out)
{
    if (precision == 0) return fast ? step_occupancy<double, true, false>(out) : step_occupancy<double, false, false>(out);
    if (!fast) return step_occupancy<float, false, false>(out);
    return vec ? step_occupancy<float, true, true>(out) : step_occupancy<float, true, false>(out);
}
}  // namespace tel

namespace tel {
template <int TX, typename ST, bool FAST, bool VEC>
static cudaError_t launch_batch_one(const DevParams *Ps, const LaunchArgs *As, const int4 *items, int nitems,
                                    int grid, cudaStream_t s)
{
    typedef Fused<2, TX, 1, ST, MODE_STEP, FAST, VEC> K;
    static DeviceOnce once;
    cudaError_t e = once.run([] {
        return cudaFuncSetAttribute(batch_kernel<TX, ST, FAST, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)K::SMEM_BYTES);
    });
    if (e != cudaSuccess) return e;
    batch_kernel<TX, ST, FAST, VEC><<<grid, TX, K::SMEM_BYTES, s>>>(Ps, As, items, nitems);
    return cudaGetLastError();
}

template <int TX, typename ST, bool FAST, bool VEC>
static int blocks_one()
{
    typedef Fused<2, TX, 1, ST, MODE_STEP, FAST, VEC> K;
    cudaFuncSetAttribute(batch_kernel<TX, ST, FAST, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)K::SMEM_BYTES);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<TX, ST, FAST, VEC>, TX, K::SMEM_BYTES) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_d2q9_batch(int precision, int tx, bool fast, bool vec, const DevParams *Ps,
                              const LaunchArgs *As, const int4 *items, int nitems, int grid, cudaStream_t s)
{
#define TEL_BATCH_CASE(TXV, STT, FV, VV) \
    if (tx == TXV && fast == FV && vec == VV) return launch_batch_one<TXV, STT, FV, VV>(Ps, As, items, nitems, grid, s);
    if (precision == 0) {
        TEL_BATCH_CASE(32, double, true, false) TEL_BATCH_CASE(32, double, false, false)
        TEL_BATCH_CASE(64, double, true, false) TEL_BATCH_CASE(64, double, false, false)
    } else {
        TEL_BATCH_CASE(32, float, true, true) TEL_BATCH_CASE(32, float, true, false)
        TEL_BATCH_CASE(32, float, false, false)
        TEL_BATCH_CASE(64, float, true, true) TEL_BATCH_CASE(64, float, true, false)
        TEL_BATCH_CASE(64, float, false, false)
    }
#undef TEL_BATCH_CASE
    return cudaErrorInvalidValue;
}

int batch_blocks_per_sm(int precision, int tx, bool fast, bool vec)
{
    if (precision == 0) {
        if (tx == 32) return fast ? blocks_one<32, double, true, false>() : blocks_one<32, double, false, false>();
        return fast ? blocks_one<64, double, true, false>() : blocks_one<64, double, false, false>();
    }
    if (tx == 32) {
        if (fast) return vec ? blocks_one<32, float, true, true>() : blocks_one<32, float, true, false>();
        return blocks_one<32, float, false, false>();
    }
    if (fast) return vec ? blocks_one<64, float, true, true>() : blocks_one<64, float, true, false>();
    return blocks_one<64, float, false, false>();
}
}  // namespace tel
