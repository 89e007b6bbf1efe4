// One object of Cartesian-apply instantiations: space RM_CART_K, degrees
// 1 .. kCartMaxP, FP64 and double-float (the build compiles this file once
// per space, in parallel).
#include "apply_cart.cuh"

#if !defined(RM_CART_K)
#error "RM_CART_K selects the space of this object"
#endif

namespace rmd {

template <int K>
cudaError_t launch_cart_part(const ApplyDev &A, const double *x, double *y, cudaStream_t s) {
  return launch_cart_range<K>(A, x, y, s, std::make_integer_sequence<int, kCartMaxP>{});
}
template cudaError_t launch_cart_part<RM_CART_K>(const ApplyDev &, const double *, double *, cudaStream_t);
template <int K>
cudaError_t launch_cart_assemble_part(const ApplyDev &A, double *y, cudaStream_t s) {
  return launch_assemble_range<K>(A, y, s, std::make_integer_sequence<int, kCartMaxP>{});
}
template cudaError_t launch_cart_assemble_part<RM_CART_K>(const ApplyDev &, double *, cudaStream_t);

}  // namespace rmd
