// Operator apply on general (trilinear) cells: the pullback metric at the
// quadrature points (setup) and the dispatch to the compile-time (k, p)
// instantiations of the apply kernel (apply_general.cuh).
#include "apply_cart.cuh"
#include "apply_general.cuh"

namespace rmd {
namespace {

__device__ __forceinline__ void jac(const double *X8, double x0, double x1, double x2, double J[9]) {
  const double N0[2] = {0.5 * (1.0 - x0), 0.5 * (1.0 + x0)};
  const double N1[2] = {0.5 * (1.0 - x1), 0.5 * (1.0 + x1)};
  const double N2[2] = {0.5 * (1.0 - x2), 0.5 * (1.0 + x2)};
  const double dN[2] = {-0.5, 0.5};
#pragma unroll
  for (int i = 0; i < 9; ++i) J[i] = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int c1 = c & 1, c2 = (c >> 1) & 1, c3 = c >> 2;
    const double g0 = dN[c1] * N1[c2] * N2[c3];
    const double g1 = N0[c1] * dN[c2] * N2[c3];
    const double g2 = N0[c1] * N1[c2] * dN[c3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double v = X8[3 * c + a];
      J[3 * a + 0] = fma(v, g0, J[3 * a + 0]);
      J[3 * a + 1] = fma(v, g1, J[3 * a + 1]);
      J[3 * a + 2] = fma(v, g2, J[3 * a + 2]);
    }
  }
}

// Pullback weight of kk-forms (Sec. 3.1) times cw = coefficient x quadrature
// weight: kk = 0: det J; kk = 3: 1/det J; kk = 1: det J J^-1 J^-T =
// adj(J) adj(J)^T / det J; kk = 2: J^T J / det J.  Symmetric entries are
// returned as (00, 11, 22, 01, 02, 12).
__device__ __forceinline__ int point_weight(int kk, double cw, const double J[9], double W[6]) {
  const double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                     J[2] * (J[3] * J[7] - J[4] * J[6]);
  if (kk == 0) { W[0] = cw * det; return 1; }
  const double s = cw / det;
  if (kk == 3) { W[0] = s; return 1; }
  double A[9];
  if (kk == 1) {  // rows of the adjugate
    A[0] = J[4] * J[8] - J[5] * J[7];
    A[1] = J[2] * J[7] - J[1] * J[8];
    A[2] = J[1] * J[5] - J[2] * J[4];
    A[3] = J[5] * J[6] - J[3] * J[8];
    A[4] = J[0] * J[8] - J[2] * J[6];
    A[5] = J[2] * J[3] - J[0] * J[5];
    A[6] = J[3] * J[7] - J[4] * J[6];
    A[7] = J[1] * J[6] - J[0] * J[7];
    A[8] = J[0] * J[4] - J[1] * J[3];
  } else {        // columns of J as rows
    A[0] = J[0]; A[1] = J[3]; A[2] = J[6];
    A[3] = J[1]; A[4] = J[4]; A[5] = J[7];
    A[6] = J[2]; A[7] = J[5]; A[8] = J[8];
  }
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int e = 0; e < 6; ++e)
    W[e] = s * (A[3 * ia[e]] * A[3 * ib[e]] + A[3 * ia[e] + 1] * A[3 * ib[e] + 1] +
                A[3 * ia[e] + 2] * A[3 * ib[e] + 2]);
  return 6;
}

// Setup: the weights of both stages at every quadrature point of every cell,
// G[cell][entry][point], entries = stage A (V^k, beta) then stage B
// (V^{k+1}, alpha), stored in the apply's number type R.
template <typename R>
__global__ void metric_kernel(ApplyDev P, R *__restrict__ G) {
  const int p = P.p, q = P.q, q3 = q * q * q;
  const int c = blockIdx.x;
  const int e[3] = {c % P.n[0], (c / P.n[0]) % P.n[1], c / (P.n[0] * P.n[1])};
  __shared__ double X8[24];
  if (threadIdx.x < 24) {
    const int corner = threadIdx.x / 3, comp = threadIdx.x % 3;
    const int c1 = corner & 1, c2 = (corner >> 1) & 1, c3 = corner >> 2;
    const long long v = (e[0] + c1) + (long long)(P.n[0] + 1) * ((e[1] + c2) + (long long)(P.n[1] + 1) * (e[2] + c3));
    X8[threadIdx.x] = P.X[3 * v + comp];
  }
  __syncthreads();
  const double *xq = P.tabs + q * (p + 1) + q * p + p * (p + 1);
  const double *wq = xq + q;
  R *Gc = G + (size_t)c * P.nAB * q3;
  for (int pt = threadIdx.x; pt < q3; pt += blockDim.x) {
    const int a1 = pt % q, a2 = (pt / q) % q, a3 = pt / (q * q);
    double J[9], W[6];
    jac(X8, xq[a1], xq[a2], xq[a3], J);
    const double w = wq[a1] * wq[a2] * wq[a3];
    const int na = point_weight(P.k, P.beta[c] * w, J, W);
    for (int j = 0; j < na; ++j) Gc[(size_t)j * q3 + pt] = rfrom<R>(W[j]);
    const int nb = point_weight(P.k + 1, P.alpha[c] * w, J, W);
    for (int j = 0; j < nb; ++j) Gc[(size_t)(na + j) * q3 + pt] = rfrom<R>(W[j]);
  }
}

}  // namespace

cudaError_t launch_metric(const ApplyDev &A, void *G, cudaStream_t s) {
  const int ncell = A.n[0] * A.n[1] * A.n[2];
  if (A.arith) metric_kernel<DF><<<ncell, 256, 0, s>>>(A, static_cast<DF *>(G));
  else metric_kernel<double><<<ncell, 256, 0, s>>>(A, static_cast<double *>(G));
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_apply_cart(const ApplyDev &A, const double *x, double *y, cudaStream_t s) {
  cudaError_t err = cudaErrorInvalidValue;
  if (A.k == 0) err = launch_cart_part<0>(A, x, y, s);
  else if (A.k == 1) err = launch_cart_part<1>(A, x, y, s);
  else if (A.k == 2) err = launch_cart_part<2>(A, x, y, s);
  if (err == cudaSuccess) add_launches(2);
  return err;
}

cudaError_t launch_apply_general(const ApplyDev &A, const double *x, double *y, cudaStream_t s) {
  static_assert(kMaxGeneralP == 8, "the build instantiates p = 1..4 and 5..8");
  const bool lo = A.p <= 4;
  cudaError_t err = cudaErrorInvalidValue;
  if (A.k == 0) err = lo ? launch_general_part<0, 1>(A.p, A, x, y, s) : launch_general_part<0, 5>(A.p, A, x, y, s);
  else if (A.k == 1) err = lo ? launch_general_part<1, 1>(A.p, A, x, y, s) : launch_general_part<1, 5>(A.p, A, x, y, s);
  else if (A.k == 2) err = lo ? launch_general_part<2, 1>(A.p, A, x, y, s) : launch_general_part<2, 5>(A.p, A, x, y, s);
  if (err != cudaSuccess) return err;
  // the cells' products to y: fixed-order sums, Dirichlet entries 0
  if (A.k == 0) err = launch_cart_assemble_part<0>(A, y, s);
  else if (A.k == 1) err = launch_cart_assemble_part<1>(A, y, s);
  else err = launch_cart_assemble_part<2>(A, y, s);
  if (err == cudaSuccess) add_launches(2);
  return err;
}

}  // namespace rmd
