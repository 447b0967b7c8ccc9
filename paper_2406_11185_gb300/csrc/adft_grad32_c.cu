// Nuclear-gradient kernels (FP32 band), class pairs with bra class in [0, 1, 2, 6, 7, 8, 9]:
// explicit instantiations of the gradient launchers of adft_gradk.cuh,
// compiled in parallel with the other groups.
#include "adft_eri.cuh"
#include "adft_gradk.cuh"

namespace adft {

template cudaError_t launch_grad_one<float, 0, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 1, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 1, 1>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 2, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 2, 1>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 2, 2>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 6, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 6, 1>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 6, 2>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 6, 3>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 6, 4>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 6, 5>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 6, 6>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 7, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 7, 1>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 7, 2>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 7, 3>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 7, 4>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 7, 5>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 7, 6>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 7, 7>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 8, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 8, 1>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 8, 2>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 8, 3>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 8, 4>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 8, 5>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 8, 6>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 8, 7>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 8, 8>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 1>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 2>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 3>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 4>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 5>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 6>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 7>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 8>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 9, 9>(const GradLaunch&, int, cudaStream_t);

}  // namespace adft
