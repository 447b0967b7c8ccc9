// Class-pair ERI kernels (double-float evaluation of the FP64 band), bra classes [9]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel with
// the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<df, 9, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 9, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 9, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 9, 3>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 9, 4>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 9, 5>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 9, 6>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 9, 7>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 9, 8>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 9, 9>(const JKLaunch&, int, cudaStream_t);

}  // namespace adft
