// D2Q9 instantiation of the fused kernel: rows of 64 nodes along x marching
// along y.
#include "tel_launch.cuh"

namespace tel {
cudaError_t launch_d2q9(int precision, int mode, const DevParams &P, const LaunchArgs &A, cudaStream_t s)
{
    return launch_lattice<2, 64, 1>(precision, mode, P, A, s);
}
}  // namespace tel
