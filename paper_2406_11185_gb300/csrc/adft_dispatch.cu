// Dispatch tables of the class-pair ERI launchers (instantiated in
// adft_eri64_*.cu and adft_eri32_*.cu).
#define ADFT_ERI_DECLARE_ONLY
#include "adft_eri.cuh"

namespace adft {

template <typename T, int... I>
static cudaError_t dispatch(int X, int Y, const JKLaunch& a, int grid, int variant, cudaStream_t s,
                            KernelInfo* info, std::integer_sequence<int, I...>) {
  using Fn = cudaError_t (*)(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
  // entries with Y > X are never called (guarded below); they point at a valid launcher
  static constexpr Fn table[] = {&launch_one<T, I / NCLS, (I % NCLS <= I / NCLS ? I % NCLS : 0)>...};
  if (X < 0 || Y < 0 || X >= NCLS || Y > X) return cudaErrorInvalidValue;
  return table[X * NCLS + Y](a, grid, variant, s, info);
}

cudaError_t launch_jk_fp64(int X, int Y, const JKLaunch& a, int grid, int variant, cudaStream_t s,
                           KernelInfo* info) {
  return dispatch<double>(X, Y, a, grid, variant, s, info, std::make_integer_sequence<int, NCLS * NCLS>{});
}

cudaError_t launch_jk_fp32(int X, int Y, const JKLaunch& a, int grid, int variant, cudaStream_t s,
                           KernelInfo* info) {
  return dispatch<float>(X, Y, a, grid, variant, s, info, std::make_integer_sequence<int, NCLS * NCLS>{});
}

}  // namespace adft
