// Class-pair ERI kernels (double-float evaluation of the FP64 band), bra classes [7, 8]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel with
// the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<df, 7, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 7, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 7, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 7, 3>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 7, 4>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 7, 5>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 7, 6>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 7, 7>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 8, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 8, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 8, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 8, 3>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 8, 4>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 8, 5>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 8, 6>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 8, 7>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 8, 8>(const JKLaunch&, int, cudaStream_t);

}  // namespace adft
