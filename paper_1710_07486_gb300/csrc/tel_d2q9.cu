// D2Q9 instantiation of the fused kernel: rows of 64 nodes along x marching
// along y.
#include "tel_launch.cuh"

namespace tel {
cudaError_t launch_d2q9(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    return launch_lattice<2, 64, 1>(precision, mode, P, A, s);
}
}  // namespace tel

namespace tel {
template <int TX, typename ST, bool FAST>
static cudaError_t launch_batch_one(const DevParams *Ps, const LaunchArgs *As, const int4 *items, int nitems,
                                    int grid, cudaStream_t s)
{
    typedef Fused<2, TX, 1, ST, MODE_STEP, FAST> K;
    static DeviceOnce once;
    cudaError_t e = once.run([] {
        return cudaFuncSetAttribute(batch_kernel<TX, ST, FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)K::SMEM_BYTES);
    });
    if (e != cudaSuccess) return e;
    batch_kernel<TX, ST, FAST><<<grid, TX, K::SMEM_BYTES, s>>>(Ps, As, items, nitems);
    return cudaGetLastError();
}

template <int TX, typename ST, bool FAST>
static int blocks_one()
{
    typedef Fused<2, TX, 1, ST, MODE_STEP, FAST> K;
    cudaFuncSetAttribute(batch_kernel<TX, ST, FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM_BYTES);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<TX, ST, FAST>, TX, K::SMEM_BYTES) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_d2q9_batch(int precision, int tx, bool fast, const DevParams *Ps, const LaunchArgs *As,
                              const int4 *items, int nitems, int grid, cudaStream_t s)
{
#define TEL_BATCH_CASE(TXV, STT, FV) \
    if (tx == TXV && fast == FV) return launch_batch_one<TXV, STT, FV>(Ps, As, items, nitems, grid, s);
    if (precision == 0) {
        TEL_BATCH_CASE(32, double, true) TEL_BATCH_CASE(32, double, false)
        TEL_BATCH_CASE(64, double, true) TEL_BATCH_CASE(64, double, false)
    } else {
        TEL_BATCH_CASE(32, float, true) TEL_BATCH_CASE(32, float, false)
        TEL_BATCH_CASE(64, float, true) TEL_BATCH_CASE(64, float, false)
    }
#undef TEL_BATCH_CASE
    return cudaErrorInvalidValue;
}

int batch_blocks_per_sm(int precision, int tx, bool fast)
{
    if (precision == 0) {
        if (tx == 32) return fast ? blocks_one<32, double, true>() : blocks_one<32, double, false>();
        return fast ? blocks_one<64, double, true>() : blocks_one<64, double, false>();
    }
    if (tx == 32) return fast ? blocks_one<32, float, true>() : blocks_one<32, float, false>();
    return fast ? blocks_one<64, float, true>() : blocks_one<64, float, false>();
}
}  // namespace tel
