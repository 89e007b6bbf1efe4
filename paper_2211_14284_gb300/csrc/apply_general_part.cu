// One object of general-apply instantiations: space RM_GENERAL_K, degrees
// RM_GENERAL_PLO .. RM_GENERAL_PLO + 3 (the build compiles this file once per
// pair, in parallel).
#include "apply_general.cuh"

#if !defined(RM_GENERAL_K) || !defined(RM_GENERAL_PLO)
#error "RM_GENERAL_K and RM_GENERAL_PLO select the instantiations of this object"
#endif

namespace rmd {

template <int K, int PLO>
cudaError_t launch_general_part(int p, const ApplyDev &A, const double *x, double *y, cudaStream_t s) {
  return launch_range<K, PLO>(p, A, x, y, s, std::make_integer_sequence<int, 4>{});
}
template cudaError_t launch_general_part<RM_GENERAL_K, RM_GENERAL_PLO>(int, const ApplyDev &, const double *,
                                                                       double *, cudaStream_t);

}  // namespace rmd
