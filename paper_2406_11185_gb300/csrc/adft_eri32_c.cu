// Class-pair ERI kernels (FP32 band), bra classes [0, 1, 2, 3, 4, 5, 6]: explicit
// instantiations of the launchers of adft_eri.cuh, compiled in parallel with the
// other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<float, 0, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 1, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 1, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 2, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 2, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 2, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 3, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 3, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 3, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 3, 3>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 4, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 4, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 4, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 4, 3>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 4, 4>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 5, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 5, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 5, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 5, 3>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 5, 4>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 5, 5>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 6, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 6, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 6, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 6, 3>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 6, 4>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 6, 5>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<float, 6, 6>(const JKLaunch&, int, cudaStream_t);

}  // namespace adft
