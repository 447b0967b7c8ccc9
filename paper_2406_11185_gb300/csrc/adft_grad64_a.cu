// Nuclear-gradient kernels (FP64 band), class pairs with bra class in [5]:
// explicit instantiations of the gradient launchers of adft_gradk.cuh,
// compiled in parallel with the other groups.
#include "adft_eri.cuh"
#include "adft_gradk.cuh"

namespace adft {

template cudaError_t launch_grad_one<double, 5, 0>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<double, 5, 1>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<double, 5, 2>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<double, 5, 3>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<double, 5, 4>(const GradLaunch&, int, cudaStream_t);
template cudaError_t launch_grad_one<double, 5, 5>(const GradLaunch&, int, cudaStream_t);

}  // namespace adft
