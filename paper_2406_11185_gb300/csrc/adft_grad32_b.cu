// Nuclear-gradient kernels (FP32 band), class pairs with bra class in [3, 4]:
// explicit instantiations of the gradient launchers of adft_gradk.cuh,
// compiled in parallel with the other groups.
#include "adft_eri.cuh"
#include "adft_gradk.cuh"

namespace adft {

template cudaError_t launch_grad_one<float, 3, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 3, 1>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 3, 2>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 3, 3>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 4, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 4, 1>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 4, 2>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 4, 3>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<float, 4, 4>(const GradLaunch&, int, cudaStream_t);

}  // namespace adft
