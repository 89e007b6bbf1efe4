// Mixed formulation of the Hodge Laplacians (Sec. 5.3): find (sigma, u) in
// V^{k-1} x V^k, Gamma_D empty, with
//     -(tau, sigma) + (d tau, u) = 0,   (v, d sigma) + (d v, d u) = F(v),
// solved by MINRES preconditioned with blockdiag(R_{k-1}^-1, R_k^-1), each
// Riesz map (alpha = beta = 1) inverted approximately by Chebyshev
// iterations preconditioned by its SC relaxation plus the p = 1 coarse
// correction (SC-PAFW on V^0, SC-PH on V^1, V^2; point-Jacobi on the L2
// block of k = 3).  The operators are the library's own handles: the Riesz
// maps (rm_setup with the relaxation), the masses and the derivative term
// (operator-only handles, alpha or beta 0), the discrete derivative d^{k-1}
// in FDM coefficients (a CSR product) and, for k = 3, the V^3 mass (CSR).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/rm.h"
#include "device.cuh"
#include "host_setup.h"

using namespace rm;
using namespace rmd;

namespace {
thread_local std::string g_hodge_error;

struct HodgeCudaError : std::runtime_error {
  explicit HodgeCudaError(const std::string &s) : std::runtime_error(s) {}
};
#define HK(x)                                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) throw HodgeCudaError(std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define HR(h, x)                                                                                \
  do {                                                                                          \
    int rc_ = (x);                                                                              \
    if (rc_ != RM_OK) throw std::runtime_error(std::string(#x) + ": " + rm_last_error(h));      \
  } while (0)

// y = a x1 + b x2 + c x3 (x2, x3 may be null)
__global__ void lincomb_kernel(long long n, double *y, double a, const double *x1, double b,
                               const double *x2, double c, const double *x3) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = a * x1[i];
    if (x2) v = fma(b, x2[i], v);
    if (x3) v = fma(c, x3[i], v);
    y[i] = v;
  }
}
// y = x / d
__global__ void divide_kernel(long long n, double *__restrict__ y, const double *__restrict__ x,
                              const double *__restrict__ d) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] / d[i];
}

// Eigenvalues of a symmetric tridiagonal matrix (diagonal a, off-diagonal b)
// by bisection on the Sturm sequence counts.
std::vector<double> tridiag_eigenvalues(const std::vector<double> &a, const std::vector<double> &b) {
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++c;
    }
    return c;
  };
  std::vector<double> ev(m);
  for (int j = 0; j < m; ++j) {
    double l = lo, h = hi;
    for (int it = 0; it < 200 && h - l > 1e-14 * std::max(std::fabs(l), std::fabs(h)); ++it) {
      const double mid = 0.5 * (l + h);
      if (count_below(mid) > j) h = mid;
      else l = mid;
    }
    ev[j] = 0.5 * (l + h);
  }
  return ev;
}
}  // namespace

struct rm_hodge {
  std::string err;
  int k = 0, p = 0;
  cudaStream_t stream = nullptr;
  rm_options opt{};
  int cheb_its = 4;
  rm_handle *R0 = nullptr, *Rk = nullptr;              // Riesz maps with their relaxations
  rm_handle *M0 = nullptr, *Mk = nullptr, *Kk = nullptr;  // operator-only handles
  long long n0 = 0, nk = 0;
  DevCsr D, DT, M3;                                     // d^{k-1} and its transpose; V^3 mass (k = 3)
  double *m3diag = nullptr;
  double int0[2] = {0, 0}, intk[2] = {0, 0};            // Chebyshev intervals
  std::vector<void *> allocs;
  double *partial = nullptr, *scal = nullptr;
  // work vectors (sized n0 + nk): MINRES and the Chebyshev / apply temporaries
  double *mv[10] = {};
  double *ct[8] = {};
  double setup_s = 0.0;

  template <typename T>
  T *dalloc(size_t count) {
    void *ptr = nullptr;
    if (count == 0) count = 1;
    HK(cudaMalloc(&ptr, count * sizeof(T)));
    allocs.push_back(ptr);
    return (T *)ptr;
  }
  ~rm_hodge() {
    for (rm_handle *h : {R0, Rk, M0, Mk, Kk})
      if (h) rm_destroy(h);
    for (void *a : allocs) cudaFree(a);
  }
};

namespace {

int hfail(rm_hodge *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  g_hodge_error = msg;
  return code;
}

DevCsr upload_full(rm_hodge *h, const Csr &A) {
  DevCsr M;
  M.nrows = A.nrows;
  std::vector<int> rid(A.nrows), ptr(A.nrows + 1);
  for (int i = 0; i < A.nrows; ++i) rid[i] = i;
  for (int i = 0; i <= A.nrows; ++i) ptr[i] = (int)A.ptr[i];
  M.tpr = spmv_tpr(A.nrows ? (double)A.nnz() / A.nrows : 1.0);
  M.rid = h->dalloc<int>(rid.size());
  M.ptr = h->dalloc<int>(ptr.size());
  M.col = h->dalloc<int>(A.col.size());
  double *val = h->dalloc<double>(A.val.size());
  HK(cudaMemcpy(M.rid, rid.data(), rid.size() * sizeof(int), cudaMemcpyHostToDevice));
  HK(cudaMemcpy(M.ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!A.col.empty()) {
    HK(cudaMemcpy(M.col, A.col.data(), A.col.size() * sizeof(int), cudaMemcpyHostToDevice));
    HK(cudaMemcpy(val, A.val.data(), A.val.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  M.val = val;
  M.vt = 0;
  return M;
}

void lincomb(rm_hodge *h, long long n, double *y, double a, const double *x1, double b = 0.0,
             const double *x2 = nullptr, double c = 0.0, const double *x3 = nullptr) {
  const long long g = std::min<long long>((n + 255) / 256, 1184);
  lincomb_kernel<<<(int)std::max<long long>(g, 1), 256, 0, h->stream>>>(n, y, a, x1, b, x2, c, x3);
  add_launches(1);
  HK(cudaGetLastError());
}

double dot(rm_hodge *h, long long n, const double *a, const double *b) {
  HK(launch_dot(n, a, b, h->partial, h->scal, 0, h->stream));
  double v = 0.0;
  HK(cudaMemcpyAsync(&v, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HK(cudaStreamSynchronize(h->stream));
  return v;
}

// Riesz operator and inner preconditioner of block b (0: V^{k-1}, 1: V^k)
void riesz_apply(rm_hodge *h, int b, const double *x, double *y) {
  if (b == 1 && h->k == 3) {
    HK(launch_spmv(h->M3, x, y, nullptr, 0, 1.0, h->stream));
    return;
  }
  rm_handle *R = b == 0 ? h->R0 : h->Rk;
  HR(R, rm_apply(R, x, y));
}
void riesz_prec(rm_hodge *h, int b, const double *r, double *z) {
  if (b == 1 && h->k == 3) {
    const long long n = h->nk;
    divide_kernel<<<(int)std::min<long long>((n + 255) / 256, 1184), 256, 0, h->stream>>>(n, z, r, h->m3diag);
    add_launches(1);
    HK(cudaGetLastError());
    return;
  }
  rm_handle *R = b == 0 ? h->R0 : h->Rk;
  HR(R, rm_precondition(R, r, z));
}

// [0.9 theta_min, 1.1 theta_max] of the preconditioned Riesz map of block b
// from the CG tridiagonal of `steps` PCG iterations on a seeded right-hand
// side (the interval of the Chebyshev iteration)
void ritz_interval(rm_hodge *h, int b, double out[2], int steps = 20) {
  const long long n = b == 0 ? h->n0 : h->nk;
  double *x = h->ct[0], *r = h->ct[1], *z = h->ct[2], *pv = h->ct[3], *q = h->ct[4];
  std::vector<double> rhs(n);
  unsigned long long s = 0x9E3779B97F4A7C15ULL ^ (unsigned long long)(b + 1);
  for (long long i = 0; i < n; ++i) {  // splitmix64 uniforms in [-1, 1)
    s += 0x9E3779B97F4A7C15ULL;
    unsigned long long t = s;
    t = (t ^ (t >> 30)) * 0xBF58476D1CE4E5B9ULL;
    t = (t ^ (t >> 27)) * 0x94D049BB133111EBULL;
    t ^= t >> 31;
    rhs[i] = (double)(t >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
  HK(cudaMemcpyAsync(r, rhs.data(), n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  HK(cudaMemsetAsync(x, 0, n * sizeof(double), h->stream));
  riesz_prec(h, b, r, z);
  lincomb(h, n, pv, 1.0, z);
  double rz = dot(h, n, r, z);
  const double rz0 = rz;
  std::vector<double> al, be;
  for (int it = 0; it < steps; ++it) {
    riesz_apply(h, b, pv, q);
    const double a = rz / dot(h, n, pv, q);
    lincomb(h, n, r, 1.0, r, -a, q);
    riesz_prec(h, b, r, z);
    const double rzn = dot(h, n, r, z);
    al.push_back(a);
    be.push_back(rzn / rz);
    rz = rzn;
    lincomb(h, n, pv, 1.0, z, be.back(), pv);
    if (!(rz > 1e-28 * rz0)) break;
  }
  const int m = (int)al.size();
  std::vector<double> diag(m), off(std::max(m - 1, 0));
  for (int j = 0; j < m; ++j) {
    diag[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < m) off[j] = std::sqrt(be[j]) / al[j];
  }
  const std::vector<double> ev = tridiag_eigenvalues(diag, off);
  out[0] = 0.9 * ev.front();
  out[1] = 1.1 * ev.back();
}

// z = the Chebyshev approximation of R_b^-1 r (cheb_its steps from zero)
void chebyshev(rm_hodge *h, int b, const double *r, double *x) {
  const long long n = b == 0 ? h->n0 : h->nk;
  const double *iv = b == 0 ? h->int0 : h->intk;
  double *res = h->ct[5], *d = h->ct[6], *zc = h->ct[7];
  const double theta = 0.5 * (iv[1] + iv[0]), delta = 0.5 * (iv[1] - iv[0]);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  lincomb(h, n, res, 1.0, r);
  riesz_prec(h, b, res, zc);
  lincomb(h, n, d, 1.0 / theta, zc);
  HK(cudaMemsetAsync(x, 0, n * sizeof(double), h->stream));
  for (int it = 0; it < h->cheb_its; ++it) {
    lincomb(h, n, x, 1.0, x, 1.0, d);
    if (it == h->cheb_its - 1) break;
    riesz_apply(h, b, d, zc);
    lincomb(h, n, res, 1.0, res, -1.0, zc);
    riesz_prec(h, b, res, zc);
    const double rn = 1.0 / (2.0 * sigma - rho);
    lincomb(h, n, d, rn * rho, d, 2.0 * rn / delta, zc);
    rho = rn;
  }
}

// y = K x, x = (sigma, u)
void hodge_apply(rm_hodge *h, const double *x, double *y) {
  const long long n0 = h->n0, nk = h->nk;
  const double *sg = x, *u = x + n0;
  double *ys = y, *yu = y + n0;
  double *w = h->ct[0], *t = h->ct[1], *t0 = h->ct[2];
  // y_sigma = D^T (M_k u) - M_{k-1} sigma
  if (h->k == 3) HK(launch_spmv(h->M3, u, w, nullptr, 0, 1.0, h->stream));
  else HR(h->Mk, rm_apply(h->Mk, u, w));
  HK(launch_spmv(h->DT, w, ys, nullptr, 0, 1.0, h->stream));
  HR(h->M0, rm_apply(h->M0, sg, t0));
  lincomb(h, n0, ys, 1.0, ys, -1.0, t0);
  // y_u = M_k (D sigma) + K_k u
  HK(launch_spmv(h->D, sg, t, nullptr, 0, 1.0, h->stream));
  if (h->k == 3) {
    HK(launch_spmv(h->M3, t, yu, nullptr, 0, 1.0, h->stream));
  } else {
    HR(h->Mk, rm_apply(h->Mk, t, yu));
    HR(h->Kk, rm_apply(h->Kk, u, w));
    lincomb(h, nk, yu, 1.0, yu, 1.0, w);
  }
}

void hodge_precondition(rm_hodge *h, const double *r, double *z) {
  chebyshev(h, 0, r, z);
  chebyshev(h, 1, r + h->n0, z + h->n0);
}

}  // namespace

extern "C" {

int rm_hodge_setup(rm_hodge **out, int k, const rm_mesh *mesh, int p, const rm_options *opt, int cheb_its,
                   void *stream) {
  if (!out || !mesh) return hfail(nullptr, RM_ERR_ARG, "rm_hodge_setup: NULL argument");
  *out = nullptr;
  if (k < 1 || k > 3) return hfail(nullptr, RM_ERR_ARG, "rm_hodge_setup: k must be 1, 2 or 3");
  if (cheb_its < 1 || cheb_its > 64) return hfail(nullptr, RM_ERR_ARG, "rm_hodge_setup: cheb_its in 1..64");
  std::unique_ptr<rm_hodge> h(new rm_hodge());
  const auto t0 = std::chrono::steady_clock::now();
  try {
    h->k = k;
    h->p = p;
    h->stream = (cudaStream_t)stream;
    h->opt = opt ? *opt : rm_default_options();
    h->cheb_its = cheb_its;
    const int ncell = mesh->nx * mesh->ny * mesh->nz;
    if (mesh->nx < 2 || mesh->ny < 2 || mesh->nz < 2) throw std::invalid_argument("at least 2 cells per direction");
    std::vector<double> one(ncell, 1.0), zero(ncell, 0.0);
    // the Riesz maps (alpha = beta = 1, Gamma_D empty) with their relaxations
    rm_options ro = h->opt;
    ro.boundary = RM_BC_NONE;
    ro.static_condensation = 1;
    ro.relaxation = 1;
    ro.composition = RM_ADDITIVE;
    auto riesz = [&](int kk) {
      rm_options o = ro;
      o.decomposition = kk == 0 ? RM_PAFW : RM_PH;
      rm_handle *r = nullptr;
      if (rm_setup(&r, kk, mesh, p, one.data(), one.data(), &o, stream) != RM_OK)
        throw std::runtime_error(std::string("Riesz map of V^") + std::to_string(kk) + ": " + rm_last_error(nullptr));
      return r;
    };
    auto oper = [&](int kk, const double *al, const double *be) {
      rm_options o = ro;
      o.relaxation = 0;
      rm_handle *r = nullptr;
      if (rm_setup(&r, kk, mesh, p, al, be, &o, stream) != RM_OK)
        throw std::runtime_error(std::string("operator of V^") + std::to_string(kk) + ": " + rm_last_error(nullptr));
      return r;
    };
    h->R0 = riesz(k - 1);
    h->M0 = oper(k - 1, zero.data(), one.data());
    long long nfree = 0;
    rm_ndofs(h->R0, &h->n0, &nfree);
    int n[3] = {mesh->nx, mesh->ny, mesh->nz};
    Layout La(k - 1, n, p, true), Lb(k, n, p, true);
    if (k < 3) {
      h->Rk = riesz(k);
      h->Mk = oper(k, zero.data(), one.data());
      h->Kk = oper(k, one.data(), zero.data());
      rm_ndofs(h->Rk, &h->nk, &nfree);
    } else {
      Geometry geo;
      for (int d = 0; d < 3; ++d) geo.n[d] = n[d];
      const size_t nv = (size_t)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
      geo.X.resize(3 * nv);
      if (mesh->vertices) {
        std::memcpy(geo.X.data(), mesh->vertices, 3 * nv * sizeof(double));
      } else {
        for (int a3 = 0; a3 <= n[2]; ++a3)
          for (int a2 = 0; a2 <= n[1]; ++a2)
            for (int a1 = 0; a1 <= n[0]; ++a1) {
              const size_t v = a1 + (size_t)(n[0] + 1) * (a2 + (size_t)(n[1] + 1) * a3);
              geo.X[3 * v + 0] = (double)a1 / n[0];
              geo.X[3 * v + 1] = (double)a2 / n[1];
              geo.X[3 * v + 2] = (double)a3 / n[2];
            }
      }
      Csr M3 = mass_v3(Lb, geo, one.data());
      h->nk = Lb.size;
      h->M3 = upload_full(h.get(), M3);
      std::vector<double> dg(Lb.size, 0.0);
      for (int i = 0; i < M3.nrows; ++i)
        for (int64_t e = M3.ptr[i]; e < M3.ptr[i + 1]; ++e)
          if (M3.col[e] == i) dg[i] = M3.val[e];
      h->m3diag = h->dalloc<double>(dg.size());
      HK(cudaMemcpy(h->m3diag, dg.data(), dg.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (h->n0 != La.size || h->nk != Lb.size) throw std::runtime_error("lattice sizes disagree");
    std::vector<int> rows(Lb.size), cols(La.size);
    for (long long i = 0; i < Lb.size; ++i) rows[i] = (int)i;
    for (long long i = 0; i < La.size; ++i) cols[i] = (int)i;
    Csr D = discrete_derivative(La, Lb, rows, cols);
    h->D = upload_full(h.get(), D);
    h->DT = upload_full(h.get(), transpose(D));
    h->partial = h->dalloc<double>(kPartialDoubles);
    HK(cudaMemset(h->partial, 0, kPartialDoubles * sizeof(double)));
    h->scal = h->dalloc<double>(S_COUNT);
    const long long nt = h->n0 + h->nk;
    for (auto &v : h->mv) v = h->dalloc<double>(nt);
    for (auto &v : h->ct) v = h->dalloc<double>(std::max(h->n0, h->nk));
    ritz_interval(h.get(), 0, h->int0);
    ritz_interval(h.get(), 1, h->intk);
    HK(cudaStreamSynchronize(h->stream));
  } catch (const HodgeCudaError &e) {
    return hfail(nullptr, RM_ERR_CUDA, std::string("rm_hodge_setup: ") + e.what());
  } catch (const std::invalid_argument &e) {
    return hfail(nullptr, RM_ERR_ARG, std::string("rm_hodge_setup: ") + e.what());
  } catch (const std::exception &e) {
    std::string w = e.what();
    return hfail(nullptr, w.find("breakdown") != std::string::npos ? RM_ERR_BREAKDOWN : RM_ERR_ARG,
                 std::string("rm_hodge_setup: ") + w);
  }
  h->setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = h.release();
  return RM_OK;
}

int rm_hodge_ndofs(const rm_hodge *h, long long *n_sigma, long long *n_u) {
  if (!h) return hfail(nullptr, RM_ERR_ARG, "rm_hodge_ndofs: NULL handle");
  if (n_sigma) *n_sigma = h->n0;
  if (n_u) *n_u = h->nk;
  return RM_OK;
}

int rm_hodge_intervals(const rm_hodge *h, double interval0[2], double interval1[2]) {
  if (!h) return hfail(nullptr, RM_ERR_ARG, "rm_hodge_intervals: NULL handle");
  if (interval0) std::memcpy(interval0, h->int0, 2 * sizeof(double));
  if (interval1) std::memcpy(interval1, h->intk, 2 * sizeof(double));
  return RM_OK;
}

int rm_hodge_apply(rm_hodge *h, const double *x, double *y) {
  if (!h || !x || !y || x == y) return hfail(h, RM_ERR_ARG, "rm_hodge_apply: bad argument");
  try {
    hodge_apply(h, x, y);
  } catch (const std::exception &e) {
    return hfail(h, RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}

int rm_hodge_precondition(rm_hodge *h, const double *r, double *z) {
  if (!h || !r || !z || r == z) return hfail(h, RM_ERR_ARG, "rm_hodge_precondition: bad argument");
  try {
    hodge_precondition(h, r, z);
  } catch (const std::exception &e) {
    return hfail(h, RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}

// Preconditioned MINRES (Paige-Saunders, Lanczos form) from x = 0, stopping
// when the natural norm sqrt(r^T P r) has fallen by 1/rtol (Sec. 5.3).
int rm_hodge_solve(rm_hodge *h, const double *b, double *x, rm_info *info) {
  if (!h || !b || !x) return hfail(h, RM_ERR_ARG, "rm_hodge_solve: NULL argument");
  const long long n = h->n0 + h->nk;
  int status = RM_ERR_NOT_CONVERGED, it = 0;
  double rel = 1.0;
  float ms = 0.f;
  try {
    cudaEvent_t e0, e1;
    HK(cudaEventCreate(&e0));
    HK(cudaEventCreate(&e1));
    HK(cudaEventRecord(e0, h->stream));
    double *v_old = h->mv[0], *v = h->mv[1], *z = h->mv[2], *zn = h->mv[3], *Az = h->mv[4];
    double *w_old = h->mv[5], *w = h->mv[6], *wn = h->mv[7], *vn = h->mv[8];
    HK(cudaMemsetAsync(x, 0, n * sizeof(double), h->stream));
    HK(cudaMemsetAsync(v_old, 0, n * sizeof(double), h->stream));
    HK(cudaMemsetAsync(w_old, 0, n * sizeof(double), h->stream));
    HK(cudaMemsetAsync(w, 0, n * sizeof(double), h->stream));
    lincomb(h, n, v, 1.0, b);
    hodge_precondition(h, v, z);
    double gamma = std::sqrt(std::max(dot(h, n, v, z), 0.0)), gamma_old = 1.0;
    const double eta0 = gamma;
    double eta = gamma, s_old = 0.0, s = 0.0, c_old = 1.0, c = 1.0;
    if (!(eta0 > 0.0)) {
      status = std::isfinite(eta0) ? RM_OK : RM_ERR_NAN;
      rel = 0.0;
    }
    while (status == RM_ERR_NOT_CONVERGED && it < h->opt.max_it) {
      lincomb(h, n, z, 1.0 / gamma, z);
      hodge_apply(h, z, Az);
      const double delta = dot(h, n, z, Az);
      lincomb(h, n, vn, 1.0, Az, -delta / gamma, v, -gamma / gamma_old, v_old);
      hodge_precondition(h, vn, zn);
      const double gn2 = dot(h, n, vn, zn);
      if (!std::isfinite(gn2) || !std::isfinite(delta)) { status = RM_ERR_NAN; break; }
      if (gn2 < 0.0) { status = RM_ERR_BREAKDOWN; break; }  // the preconditioner is not SPD
      const double gn = std::sqrt(gn2);
      const double a0 = c * delta - c_old * s * gamma;
      const double a1 = std::sqrt(a0 * a0 + gn * gn);
      const double a2 = s * delta + c_old * c * gamma;
      const double a3 = s_old * gamma;
      const double cn = a0 / a1, sn = gn / a1;
      lincomb(h, n, wn, 1.0 / a1, z, -a3 / a1, w_old, -a2 / a1, w);
      lincomb(h, n, x, 1.0, x, cn * eta, wn);
      eta = -sn * eta;
      ++it;
      rel = std::fabs(eta) / eta0;
      if (rel <= h->opt.rtol) status = RM_OK;
      std::swap(v_old, v);
      std::swap(v, vn);  // v_old = v, v = vn
      std::swap(z, zn);
      std::swap(w_old, w);
      std::swap(w, wn);  // w_old = w, w = wn
      gamma_old = gamma;
      gamma = gn;
      c_old = c;
      c = cn;
      s_old = s;
      s = sn;
    }
    HK(cudaEventRecord(e1, h->stream));
    HK(cudaEventSynchronize(e1));
    HK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  } catch (const std::exception &e) {
    if (info) info->status = RM_ERR_CUDA;
    return hfail(h, RM_ERR_CUDA, e.what());
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iterations = it;
    info->status = status;
    info->rel_res_l2 = -1.0;
    info->rel_res_natural = rel;
    info->iterations_natural = status == RM_OK ? it : -1;
    info->setup_s = h->setup_s;
    info->solve_ms = ms;
    info->fallback_at = -1;
    info->judge_eta = -1.0;
  }
  if (status != RM_OK) hfail(h, status, "rm_hodge_solve: not converged");
  return status;
}

void rm_hodge_destroy(rm_hodge *h) { delete h; }

const char *rm_hodge_last_error(const rm_hodge *h) { return h ? h->err.c_str() : g_hodge_error.c_str(); }

}  // extern "C"
