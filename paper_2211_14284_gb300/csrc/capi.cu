// C ABI (include/rm.h): setup on the host in FP64, upload, and the
// device-resident apply / precondition / PCG loop on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/rm.h"
#include "device.cuh"
#include "host_basis.h"
#include "host_setup.h"
#include "learned.cuh"

using namespace rm;
using namespace rmd;

namespace {
thread_local std::string g_last_error;

struct CudaError : std::runtime_error {
  explicit CudaError(const std::string &s) : std::runtime_error(s) {}
};
#define CK(x)                                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess)                                                                      \
      throw CudaError(std::string(#x) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};
}  // namespace

namespace {
// Scratch of rm_precondition_noalloc: the coarse right-hand side and
// correction, 2 x RM_NOALLOC_MAX_COARSE doubles = 128 KiB, a file-scope
// device array present on every GPU that loads the library until exit.
static __device__ __align__(256) double g_noalloc_scratch[2 * RM_NOALLOC_MAX_COARSE];

std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[64] = {};  // device address of the array, per device ordinal

// In host code the array's name is only a host-side stand-in; its device
// address is looked up with the device current.  rm_setup (which may
// allocate, and runs before any handle exists) calls this every time, so a
// handle created after a cudaDeviceReset re-reads the address of the new
// context; rm_precondition_noalloc itself only reads the cached pointer.
void refresh_noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (dev < 0 || dev >= 64) throw std::runtime_error("device ordinal out of range");
  void *ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) throw CudaError(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  g_noalloc_ptr[dev] = (double *)ptr;
}
double *noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (dev < 0 || dev >= 64 || !g_noalloc_ptr[dev])
    throw std::runtime_error("no handle was set up on this device");
  return g_noalloc_ptr[dev];
}
}  // namespace

struct rm_handle {
  std::string err;
  cudaStream_t stream = nullptr;
  rm_options opt{};
  int k = 0, p = 0, n[3] = {0, 0, 0};
  Layout L;
  long long size = 0, nfree = 0;
  bool sc = false, ph = false;
  int vt = 0;  // 0 double, 1 float preconditioner data
  std::vector<void *> allocs;
  ApplyDev ad{};
  uint8_t *mask = nullptr;
  DevCsr Binv, E, Et, R0, R0T, Dt, DtT;
  void *A0inv = nullptr;
  int nc = 0;
  // coarse multigrid (RM_COARSE_GMG): per level A, P (l+1 -> l), P^T, Jacobi
  // weights and vectors B (right-hand side), X (iterate), T, R (work)
  int mg_levels = 0, mg_ncoarsest = 0;
  std::vector<DevCsr> mgA, mgP, mgPT;
  std::vector<double *> mgW, mgB, mgX, mgT, mgR;
  std::vector<int> mgN;
  double *mgAinv = nullptr;
  std::vector<DevPatch> mgStar;  // k = 1, 2: vertex-star smoother per level
  double mgOmega = 0.125;
  // k = 1, 2 Hiptmair-Jacobi smoother: per level G, G^T, the potential's
  // Jacobi weights and a potential-space vector
  bool mgHip = false;
  std::vector<DevCsr> mgG, mgGT;
  std::vector<double *> mgWB, mgU;
  std::vector<int> mgNB;
  // RM_HYBRID: residual and second relaxation vectors
  double *hy_t = nullptr, *hy_w = nullptr;
  bool op_only = false;  // relaxation = 0: the operator alone
  std::vector<DevPatch> fam;   // families acting on the main space
  std::vector<DevPatch> pfam;  // potential-space families (Hiptmair)
  long long size0 = 0;         // potential (H(grad)) lattice size
  double *w = nullptr, *rt = nullptr, *u0 = nullptr, *v0 = nullptr, *cc = nullptr, *ce = nullptr;
  double *r = nullptr, *z = nullptr, *pv = nullptr, *qv = nullptr, *scal = nullptr, *partial = nullptr;
  double *hscal = nullptr;  // pinned
  // residual histories of the last solve: hrr[k] = (r_k, r_k), hrz[k] = (r_k, B r_k)
  // (device, max_it + 1 each), and how many entries the solve wrote
  double *hrr = nullptr, *hrz = nullptr;
  int nhrr = 0, nhrz = 0;
  double setup_s = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> evpool;  // profile = 1: start/stop pairs
  // independent branches of the relaxation (patch families, the Hiptmair
  // potential branch, the coarse correction) run on their own streams
  static constexpr int kBranches = 5;
  cudaStream_t br[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {};
  long long stat_patches = 0, stat_slots = 0, stat_nnz = 0;
  // learned coarse corrector (k = 0): coarse operator, grid maps, centred
  // log alpha at the grid vertices, network and its batch-1 buffers
  DevCsr A0;
  int cdims[3] = {0, 0, 0};
  long long cnvox = 0;
  int *c_free2lat = nullptr, *c_lat2free = nullptr;
  float *c_logal = nullptr, *cx = nullptr, *cy = nullptr;
  double *cl = nullptr, *cq = nullptr, *lscal = nullptr, *lpart = nullptr;
  rmn::Net *net = nullptr;
  int corr_mode = RM_CORRECTOR_PLAIN, judge_every = 8;
  double judge_max = 0.9;
  // per solve: calls, judged calls, fallback call, last eta
  int lc_calls = 0, lc_judged = 0, lc_fallback = -1;
  double lc_eta = -1.0;
  // recording of r_0 = R_0 r for training (device, rec_cap x nc)
  double *rec = nullptr;
  int rec_cap = 0, rec_n = 0;
  // z = B r on the solver's own r, z captured once as a CUDA graph (the
  // branch streams' fork and join become graph edges) for the corrector
  // mode it was captured in; replayed every CG iteration
  cudaGraphExec_t pgraph = nullptr;
  int pgraph_mode = -1;
  long long pgraph_launches = 0;
  cudaStream_t cap = nullptr;  // capture stream (the caller's may be the legacy one)

  template <typename T>
  T *dalloc(size_t count) {
    void *ptr = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
    if (e != cudaSuccess) throw CudaError(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back(ptr);
    return (T *)ptr;
  }
  template <typename T>
  T *upload(const std::vector<T> &v) {
    T *d = dalloc<T>(v.size());
    if (!v.empty()) CK(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
  }
  void *upload_vals(const std::vector<double> &v) {
    if (vt == 0) return upload(v);
    std::vector<float> f(v.begin(), v.end());
    return upload(f);
  }
  ~rm_handle() {
    if (pgraph) cudaGraphExecDestroy(pgraph);
    if (net) rmn::destroy(net);
    for (void *a : allocs) cudaFree(a);
    if (hscal) cudaFreeHost(hscal);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (cudaEvent_t e : evpool) cudaEventDestroy(e);
    for (int i = 0; i < kBranches; ++i) {
      if (br[i]) cudaStreamDestroy(br[i]);
      if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace {

// Upload a free-indexed (or arbitrary) CSR with explicit row/col maps.
// rows: the rows to keep (in A's numbering), empty ones included, so that a
// "y = u + a A x" product writes every row of the set; NULL keeps the
// non-empty rows.
DevCsr upload_csr(rm_handle *h, const Csr &A, const std::vector<int> *rowmap,
                  const std::vector<int> *colmap, const std::vector<int> *rows = nullptr,
                  bool force_double = false) {
  std::vector<int> rid, ptr{0}, col;
  std::vector<double> val;
  std::vector<int> all;
  if (!rows) {
    for (int i = 0; i < A.nrows; ++i)
      if (A.ptr[i + 1] != A.ptr[i]) all.push_back(i);
    rows = &all;
  }
  for (int i : *rows) {
    rid.push_back(rowmap ? (*rowmap)[i] : i);
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      col.push_back(colmap ? (*colmap)[A.col[e]] : A.col[e]);
      val.push_back(A.val[e]);
    }
    if (val.size() > (size_t)2147483647) throw std::runtime_error("CSR too large");
    ptr.push_back((int)col.size());
  }
  DevCsr D;
  D.nrows = (int)rid.size();
  double avg = D.nrows ? (double)col.size() / D.nrows : 1.0;
  D.tpr = spmv_tpr(avg);
  D.rid = h->upload(rid);
  D.ptr = h->upload(ptr);
  D.col = h->upload(col);
  int saved = h->vt;
  if (force_double) h->vt = 0;
  D.val = h->upload_vals(val);
  D.vt = h->vt;
  h->vt = saved;
  return D;
}

DevPatch upload_family(rm_handle *h, const PatchFamily &F) {
  DevPatch D;
  D.nslots = F.nslots;
  D.npatch = F.npatch;
  D.nnz = F.nnz();
  D.nflev = (int)F.flev.size() - 1;
  D.nblev = (int)F.blev.size() - 1;
  D.slotmap = h->upload(F.slotmap);
  D.rowptr = h->upload(F.rowptr);
  D.col = h->upload(F.col);
  D.tptr = h->upload(F.tptr);
  D.trow = h->upload(F.trow);
  D.tpos = h->upload(F.tpos);
  D.flev = h->upload(F.flev);
  D.frows = h->upload(F.frows);
  D.blev = h->upload(F.blev);
  D.brows = h->upload(F.brows);
  D.vt = h->vt;
  if (F.inverse) {
    D.inverse = 1;
    D.ivals = F.ivals();
    D.pos_slot = h->upload(F.pos_slot);
    D.pos_blk = h->upload(F.pos_blk);
    D.bptr = h->upload(F.bptr);
    D.boff = h->upload(F.boff);
    D.val = h->upload_vals(F.device_values());
    D.vstride = D.nnz;
  } else {
    // factor values per patch padded to 16 bytes (the warp kernel's bulk
    // copies); the template as 16-bit arrays when its sizes allow
    const int per16 = h->vt == 0 ? 2 : 4;
    D.vstride = (D.nnz + per16 - 1) / per16 * per16;
    const std::vector<double> v = F.device_values();
    std::vector<double> vp((size_t)F.npatch * D.vstride, 0.0);
    for (int pi = 0; pi < F.npatch; ++pi)
      std::copy(v.begin() + (size_t)pi * D.nnz, v.begin() + (size_t)(pi + 1) * D.nnz,
                vp.begin() + (size_t)pi * D.vstride);
    D.val = h->upload_vals(vp);
    if (F.nslots + 1 < 65536 && D.nnz < 65536) {
      const std::vector<int> *parts[9] = {&F.rowptr, &F.col, &F.flev, &F.frows, &F.blev,
                                          &F.brows, &F.tptr, &F.trow, &F.tpos};
      std::vector<unsigned short> blob;
      for (int a = 0; a < 9; ++a) {
        D.toff[a] = (int)blob.size();
        for (int v16 : *parts[a]) blob.push_back((unsigned short)v16);
      }
      while ((blob.size() * sizeof(unsigned short)) % 16) blob.push_back(0);
      D.tmpl = h->upload(blob);
      D.tmpl_bytes = (int)(blob.size() * sizeof(unsigned short));
      D.wpb = patch_warps_per_block(D);
    }
  }
  if (h->opt.deterministic) {
    // the family's scatter as a gather: per lattice entry, its (patch, slot)
    // values in increasing patch-major order
    std::vector<std::pair<int, long long>> ent;
    for (int pi = 0; pi < F.npatch; ++pi)
      for (int sl = 0; sl < F.nslots; ++sl) {
        const int g = F.slotmap[(size_t)pi * F.nslots + sl];
        if (g >= 0) ent.emplace_back(g, (long long)pi * F.nslots + sl);
      }
    std::sort(ent.begin(), ent.end());
    if ((size_t)F.npatch * F.nslots > (size_t)INT32_MAX)
      throw std::runtime_error("deterministic relaxation: patch family too large");
    std::vector<int> grow, gptr{0}, gidx;
    for (size_t e = 0; e < ent.size(); ++e) {
      if (e == 0 || ent[e].first != ent[e - 1].first) {
        if (e > 0) gptr.push_back((int)gidx.size());
        grow.push_back(ent[e].first);
      }
      gidx.push_back((int)ent[e].second);
    }
    if (!ent.empty()) gptr.push_back((int)gidx.size());
    D.ng = (int)grow.size();
    D.grow = h->upload(grow);
    D.gptr = h->upload(gptr);
    D.gidx = h->upload(gidx);
    D.zp = h->dalloc<double>((size_t)F.npatch * F.nslots);
  }
  h->stat_patches += F.npatch;
  h->stat_slots += (long long)F.npatch * F.nslots;
  h->stat_nnz += (long long)F.npatch * (F.inverse ? F.ivals() : F.nnz());
  if ((size_t)F.nslots * sizeof(double) > 200 * 1024) throw std::runtime_error("patch too large for shared memory");
  return D;
}

void build_apply(rm_handle *h, const Geometry &geo, const std::vector<double> &alpha,
                 const std::vector<double> &beta) {
  const int k = h->k, p = h->p;
  const int q = quad_points(p);
  Basis1D B(p);
  std::vector<double> xq, wq;
  gll_rule(q, xq, wq);
  std::vector<double> tabs(q * (p + 1) + q * p + p * (p + 1) + 2 * q);
  B.tab_s(xq.data(), q, tabs.data());
  B.tab_r(xq.data(), q, tabs.data() + q * (p + 1));
  std::copy(B.D.begin(), B.D.end(), tabs.begin() + q * (p + 1) + q * p);
  std::copy(xq.begin(), xq.end(), tabs.begin() + q * (p + 1) + q * p + p * (p + 1));
  std::copy(wq.begin(), wq.end(), tabs.begin() + q * (p + 1) + q * p + p * (p + 1) + q);
  // reflection split of both tabulations (appended after wq)
  std::vector<double> eod;
  std::vector<int> eoh;
  if (!eo_tables(tabs.data(), q, p + 1, eod, eoh) ||
      !eo_tables(tabs.data() + q * (p + 1), q, p, eod, eoh))
    throw std::runtime_error("1D tabulations lack the reflection symmetry of the GLL points");
  tabs.insert(tabs.end(), eod.begin(), eod.end());
  ApplyDev &A = h->ad;
  Layout L1(k + 1, h->n, p);
  A.k = k;
  A.p = p;
  A.q = q;
  for (int d = 0; d < 3; ++d) A.n[d] = h->n[d];
  A.nc0 = h->L.ncomp;
  A.nc1 = L1.ncomp;
  for (int m = 0; m < 3; ++m)
    for (int d = 0; d < 3; ++d) {
      A.N[m][d] = (int)h->L.N[m][d];
      A.ld0[m][d] = h->L.ld[m][d];
      A.ld1[m][d] = L1.ld[m][d];
      A.t0[m][d] = h->L.t[m][d];
      A.t1[m][d] = L1.t[m][d];
    }
  for (int m = 0; m < 3; ++m) A.off[m] = h->L.off[m];
  for (int m = 0; m < 4; ++m) {
    A.loff0[m] = h->L.loff[m];
    A.loff1[m] = L1.loff[m];
  }
  A.nloc0 = h->L.nloc;
  A.nloc1 = L1.nloc;
  A.X = h->upload(geo.X);
  A.alpha = h->upload(alpha);
  A.beta = h->upload(beta);
  A.tabs = h->upload(tabs);
  const size_t q3 = (size_t)q * q * q;
  const int ncell = h->n[0] * h->n[1] * h->n[2];
  // Cartesian fast path when every cell is an axis-aligned box
  {
    std::vector<double> hc(3 * (size_t)ncell);
    bool cart = true;
    for (int c = 0; c < ncell && cart; ++c) {
      double X8[24];
      geo.cell_vertices(c % h->n[0], (c / h->n[0]) % h->n[1], c / (h->n[0] * h->n[1]), X8);
      double hh[3];
      for (int d = 0; d < 3; ++d) hh[d] = X8[3 * (1 << d) + d] - X8[d];
      const double tol = 1e-12 * std::max(hh[0], std::max(hh[1], hh[2]));
      for (int d = 0; d < 3; ++d)
        if (!(hh[d] > 0)) cart = false;
      for (int corner = 0; corner < 8 && cart; ++corner)
        for (int d = 0; d < 3; ++d)
          if (std::fabs(X8[3 * corner + d] - (X8[d] + ((corner >> d) & 1) * hh[d])) > tol) cart = false;
      for (int d = 0; d < 3; ++d) hc[3 * (size_t)c + d] = hh[d];
    }
    A.cartesian = cart ? 1 : 0;
    if (cart) {
      A.bh_a = B.Bhat[0];
      A.bh_b = B.Bhat[p];
      const size_t smem = cart_local_smem_doubles(h->k, p, A.nloc0, A.nloc1);
      if (smem * sizeof(double) > 227 * 1024)
        throw std::runtime_error("degree too high for the Cartesian apply kernel's shared memory");
      A.Y = h->dalloc<double>((size_t)ncell * A.nloc0);  // unassembled cell products
      // per cell: beta x the box metric of each V^k component, alpha x that of
      // each V^{k+1} component (J = diag(h/2); the pullbacks of Sec. 3.1)
      std::vector<double> cc((size_t)ncell * 8, 0.0);
      auto box_metric = [](int kk, int m, const double *hh) {
        const double det = 0.125 * hh[0] * hh[1] * hh[2];
        if (kk == 0) return det;
        if (kk == 3) return 1.0 / det;
        if (kk == 1) return det * 4.0 / (hh[m] * hh[m]);
        return 0.25 * hh[m] * hh[m] / det;
      };
      const int nc0 = k == 0 ? 1 : 3, nc1 = k == 2 ? 1 : 3;
      for (int c = 0; c < ncell; ++c) {
        const double *hh = &hc[3 * (size_t)c];
        for (int m = 0; m < nc0; ++m) cc[(size_t)c * 8 + m] = beta[c] * box_metric(k, m, hh);
        for (int t = 0; t < nc1; ++t) cc[(size_t)c * 8 + 3 + t] = alpha[c] * box_metric(k + 1, t, hh);
      }
      A.ccoef = h->upload(cc);
      A.G = nullptr;
      return;
    }
  }
  if (p > kMaxGeneralP ||
      (size_t)general_smem_doubles(k, p) * sizeof(double) > 227 * 1024)
    throw std::runtime_error("degree too high for the general apply kernel's shared memory (p <= 8)");
  if (!eo_rule_holds(p, eoh, eod))
    throw std::runtime_error("1D tabulations do not follow the parity pattern the general apply is built for");
  // pullback weights at every quadrature point, computed once on the device
  A.nA = k == 0 ? 1 : 6;
  A.nAB = A.nA + (k == 2 ? 1 : 6);
  double *G = h->dalloc<double>((size_t)ncell * A.nAB * q3);
  A.G = G;
  A.Y = h->dalloc<double>((size_t)ncell * A.nloc0);  // unassembled cell products
  CK(launch_metric(A, G, h->stream));
  CK(cudaStreamSynchronize(h->stream));
}

int fail(rm_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  g_last_error = msg;
  return code;
}

// One symmetric V(2,2) cycle on level l: X[l] = V_l B[l] (damped Jacobi,
// Galerkin coarse levels, dense solve on the coarsest).
void vcycle(rm_handle *h, int l) {
  cudaStream_t s = h->stream;
  if (l == h->mg_levels) {
    CK(launch_gemv(h->mg_ncoarsest, h->mgAinv, 0, h->mgB[l], h->mgX[l], s));
    return;
  }
  const DevCsr &A = h->mgA[l];
  const int nl = h->mgN[l];
  double *b = h->mgB[l], *x = h->mgX[l], *t = h->mgT[l], *w = h->mgW[l], *r = h->mgR[l];
  if (h->mgHip) {
    // Hiptmair-Jacobi (Sec. 5.1): damped Jacobi on A, then on the potential
    // operator through G: x += G W_B G^T (b - A x); the post-smoother runs
    // the two in reverse order, so the cycle stays symmetric
    const DevCsr &G = h->mgG[l], &GT = h->mgGT[l];
    double *u = h->mgU[l];
    const double *wb = h->mgWB[l];
    const int nb = h->mgNB[l];
    auto pot = [&](double *xx) {
      CK(launch_spmv(A, xx, r, b, 2, -1.0, s));       // r = b - A x
      CK(launch_spmv(GT, r, u, nullptr, 0, 1.0, s));  // u = G^T r
      CK(launch_diag_scale(nb, wb, u, u, s));         // u = W_B u
      CK(launch_spmv(G, u, xx, nullptr, 1, 1.0, s));  // x += G u
    };
    CK(launch_diag_scale(nl, w, b, t, s));  // space sweep from 0
    pot(t);
    CK(launch_jacobi(A, b, t, w, x, s));    // x = t + W (b - A t)
    pot(x);
    CK(launch_spmv(A, x, r, b, 2, -1.0, s));
    CK(launch_spmv(h->mgPT[l], r, h->mgB[l + 1], nullptr, 0, 1.0, s));
    vcycle(h, l + 1);
    CK(launch_spmv(h->mgP[l], h->mgX[l + 1], x, nullptr, 1, 1.0, s));
    pot(x);
    CK(launch_jacobi(A, b, x, w, t, s));
    pot(t);
    CK(launch_jacobi(A, b, t, w, x, s));
    return;
  }
  if (!h->mgStar.empty()) {
    // additive vertex-star smoother: x += omega sum_v R_v^T A_v^-1 R_v (b - A x)
    const DevPatch &F = h->mgStar[l];
    auto sweep = [&](bool first) {
      const double *rhs = b;
      if (!first) {
        CK(launch_spmv(A, x, r, b, 2, -1.0, s));
        rhs = r;
      }
      CK(cudaMemsetAsync(t, 0, nl * sizeof(double), s));
      CK(launch_patches(F, rhs, t, s));
      CK(launch_axpy(nl, h->mgOmega, t, x, first ? 0 : 1, s));
    };
    sweep(true);
    sweep(false);
    CK(launch_spmv(A, x, r, b, 2, -1.0, s));
    CK(launch_spmv(h->mgPT[l], r, h->mgB[l + 1], nullptr, 0, 1.0, s));
    vcycle(h, l + 1);
    CK(launch_spmv(h->mgP[l], h->mgX[l + 1], x, nullptr, 1, 1.0, s));
    sweep(false);
    sweep(false);
    return;
  }
  CK(launch_diag_scale(nl, w, b, t, s));                        // sweep 1 from 0
  CK(launch_jacobi(A, b, t, w, x, s));                          // sweep 2
  CK(launch_spmv(A, x, r, b, 2, -1.0, s));                      // r = b - A x
  CK(launch_spmv(h->mgPT[l], r, h->mgB[l + 1], nullptr, 0, 1.0, s));
  vcycle(h, l + 1);
  CK(launch_spmv(h->mgP[l], h->mgX[l + 1], x, nullptr, 1, 1.0, s));
  CK(launch_jacobi(A, b, x, w, t, s));
  CK(launch_jacobi(A, b, t, w, x, s));
}

// Coarse-grid data of the learned corrector (H(grad)): A_0, the maps between
// coarse free DOFs and the (n+1)^3 vertex grid, and log alpha at the
// vertices (mean over the adjacent cells) minus its mean over the grid.
void corrector_data(rm_handle *h, const CoarseData &cd, const std::vector<double> &alpha) {
  std::vector<int> rows(cd.nc);
  for (int i = 0; i < cd.nc; ++i) rows[i] = i;
  h->A0 = upload_csr(h, cd.A0, nullptr, nullptr, &rows, true);
  for (int d = 0; d < 3; ++d) h->cdims[d] = h->n[d] + 1;
  h->cnvox = (long long)h->cdims[0] * h->cdims[1] * h->cdims[2];
  std::vector<int> l2f(h->cnvox, -1);
  for (int f = 0; f < cd.nc; ++f) l2f[cd.free2lat[f]] = f;
  h->c_free2lat = h->upload(cd.free2lat);
  h->c_lat2free = h->upload(l2f);
  std::vector<double> s(h->cnvox, 0.0), cnt(h->cnvox, 0.0);
  for (int e3 = 0; e3 < h->n[2]; ++e3)
    for (int e2 = 0; e2 < h->n[1]; ++e2)
      for (int e1 = 0; e1 < h->n[0]; ++e1) {
        const double la = std::log(alpha[e1 + (size_t)h->n[0] * (e2 + (size_t)h->n[1] * e3)]);
        for (int c = 0; c < 8; ++c) {
          const long long v = (e1 + (c & 1)) +
                              h->cdims[0] * ((e2 + ((c >> 1) & 1)) + (long long)h->cdims[1] * (e3 + (c >> 2)));
          s[v] += la;
          cnt[v] += 1.0;
        }
      }
  double mean = 0.0;
  for (long long v = 0; v < h->cnvox; ++v) mean += (s[v] /= cnt[v]);
  mean /= (double)h->cnvox;
  std::vector<float> la(h->cnvox);
  for (long long v = 0; v < h->cnvox; ++v) la[v] = (float)(s[v] - mean);
  h->c_logal = h->upload(la);
  h->cx = h->dalloc<float>(2 * h->cnvox);
  h->cy = h->dalloc<float>(h->cnvox);
  h->cl = h->dalloc<double>(h->nc);
  h->cq = h->dalloc<double>(h->nc);
  h->lscal = h->dalloc<double>(8);
  h->lpart = h->dalloc<double>(kPartialDoubles);
  CK(cudaMemset(h->lpart, 0, kPartialDoubles * sizeof(double)));
}

// ce = A_0^-1 cc (dense inverse) or its V(2,2) approximation
void plain_coarse(rm_handle *h) {
  if (h->mg_levels > 0 || h->mgAinv) vcycle(h, 0);
  else CK(launch_gemv(h->nc, h->A0inv, 0, h->cc, h->ce, h->stream));
}

// ce = t N(cc) with the A_0-energy optimal step t; on judged calls the plain
// correction decides whether to keep the network (see rm_corrector_use)
void learned_coarse(rm_handle *h) {
  cudaStream_t s = h->stream;
  const int nc = h->nc;
  CK(launch_dot(nc, h->cc, h->cc, h->lpart, h->lscal, 0, s));
  rmn::corr_pack(nc, h->cnvox, h->cc, h->c_lat2free, h->c_logal, h->lscal, h->cx, s);
  rmn::forward(h->net, 1, h->cx, h->cy);
  rmn::corr_gather(nc, h->cy, h->c_free2lat, h->cl, s);
  CK(launch_spmv(h->A0, h->cl, h->cq, nullptr, 0, 1.0, s));
  CK(launch_dot(nc, h->cl, h->cc, h->lpart, h->lscal, 1, s));
  CK(launch_dot(nc, h->cl, h->cq, h->lpart, h->lscal, 2, s));
  const int call = h->lc_calls++;
  if (h->judge_every > 0 && call % h->judge_every == 0) {
    plain_coarse(h);
    CK(launch_dot(nc, h->cc, h->ce, h->lpart, h->lscal, 3, s));
    double hs[4];
    CK(cudaMemcpyAsync(hs, h->lscal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double a = hs[1], b = hs[2], e = hs[3];
    double eta = 1.0;
    if (b > 0.0 && e > 0.0) eta = std::sqrt(std::min(1.0, std::max(0.0, 1.0 - a * a / (b * e))));
    h->lc_judged++;
    h->lc_eta = eta;
    if (!(eta <= h->judge_max)) {
      h->lc_fallback = call;  // ce already holds the plain correction
      return;
    }
  }
  rmn::corr_scale(nc, h->cl, h->lscal, h->ce, s);
}

// z = B r.  The additive terms of the interface relaxation (each patch
// family, the Hiptmair potential branch) only add into z with atomic adds,
// so they run concurrently on the handle's branch streams between a fork
// after the condensation and a join before the interior expansion; the
// coarse solve runs beside them and its prolongation is added last (it
// enters the interior rows too, which the expansion overwrites).
void apply(rm_handle *h, const double *x, double *y);

// z += C r, the coarse correction R_0^T A_0^-1 R_0 r (or its cycle / learned
// form), on the handle's stream (the hybrid composition)
void coarse_add(rm_handle *h, const double *r, double *z) {
  if (h->nc == 0 || h->corr_mode == RM_CORRECTOR_OFF) return;
  cudaStream_t s = h->stream;
  CK(launch_spmv(h->R0, r, h->cc, nullptr, 0, 1.0, s));
  if (h->rec && h->rec_n < h->rec_cap) {
    CK(cudaMemcpyAsync(h->rec + (size_t)h->rec_n * h->nc, h->cc, h->nc * sizeof(double),
                       cudaMemcpyDeviceToDevice, s));
    h->rec_n++;
  }
  if (h->corr_mode == RM_CORRECTOR_LEARNED && h->net && h->lc_fallback < 0) learned_coarse(h);
  else plain_coarse(h);
  CK(launch_spmv(h->R0T, h->ce, z, nullptr, 1, 1.0, s));
}

void relax(rm_handle *h, const double *r, double *z, bool with_coarse);

// z = B r.  RM_ADDITIVE: B = S + C; RM_HYBRID: the V(1,1) cycle
// z = w S r, z += C (r - A z), z += w S (r - A z) (Sec. 5).
void precondition(rm_handle *h, const double *r, double *z) {
  if (h->opt.composition != RM_HYBRID) {
    relax(h, r, z, true);
    return;
  }
  cudaStream_t s = h->stream;
  const int n = (int)h->size;
  const double om = h->opt.hybrid_omega;
  relax(h, r, z, false);
  CK(launch_axpy(n, om, z, z, 0, s));              // z = w S r
  apply(h, z, h->hy_t);
  CK(launch_sub(n, h->mask, r, h->hy_t, h->hy_t, s));  // t = r - A z
  coarse_add(h, h->hy_t, z);
  apply(h, z, h->hy_t);
  CK(launch_sub(n, h->mask, r, h->hy_t, h->hy_t, s));
  relax(h, h->hy_t, h->hy_w, false);
  CK(launch_axpy(n, om, h->hy_w, z, 1, s));        // z += w S t
}

// z = S r (+ C r with with_coarse): the additive relaxation
void relax(rm_handle *h, const double *r, double *z, bool with_coarse) {
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(z, 0, h->size * sizeof(double), s));
  const double *rr = r;
  if (h->sc) {
    CK(launch_spmv(h->Binv, r, h->w, nullptr, 0, 1.0, s));       // w_I = P_II^-1 r_I
    CK(launch_spmv(h->E, r, h->rt, r, 2, -1.0, s));              // rt_G = r_G - P_GI P_II^-1 r_I
    rr = h->rt;
  }
  // the learned coarse term talks to the host (judge), and the deterministic
  // relaxation orders every addition into z: keep everything on s
  const bool det = h->opt.deterministic != 0;
  const bool fork = h->corr_mode != RM_CORRECTOR_LEARNED && !det;
  int nb = 0;
  auto branch = [&]() -> cudaStream_t {
    if (!fork) return s;
    cudaStream_t b = h->br[nb % rm_handle::kBranches];
    if (nb < rm_handle::kBranches) CK(cudaStreamWaitEvent(b, h->fork, 0));
    ++nb;
    return b;
  };
  if (fork) CK(cudaEventRecord(h->fork, s));
  for (auto &F : h->fam) {
    cudaStream_t b = branch();
    CK(launch_patches(F, rr, z, b));                               // z_G += sum_v S_v^-1 rt
    CK(launch_patch_gather(F, z, b));                              // (deterministic form)
  }
  if (h->ph) {
    cudaStream_t b = branch();
    CK(launch_spmv(h->DtT, rr, h->u0, nullptr, 0, 1.0, b));        // u0 = D~^T rt
    CK(cudaMemsetAsync(h->v0, 0, h->size0 * sizeof(double), b));
    for (auto &F : h->pfam) {
      CK(launch_patches(F, h->u0, h->v0, b));
      CK(launch_patch_gather(F, h->v0, b));
    }
    CK(launch_spmv(h->Dt, h->v0, z, nullptr, det ? 1 : 3, 1.0, b)); // z_G += D~ v0
  }
  const bool record = with_coarse && h->rec && h->rec_n < h->rec_cap;
  if (with_coarse && h->nc > 0 && (h->corr_mode != RM_CORRECTOR_OFF || record)) {
    cudaStream_t b = branch();
    std::swap(h->stream, b);  // the coarse helpers launch on h->stream
    try {
      CK(launch_spmv(h->R0, r, h->cc, nullptr, 0, 1.0, h->stream));
      if (record) {
        CK(cudaMemcpyAsync(h->rec + (size_t)h->rec_n * h->nc, h->cc, h->nc * sizeof(double),
                           cudaMemcpyDeviceToDevice, h->stream));
        h->rec_n++;
      }
      if (h->corr_mode != RM_CORRECTOR_OFF) {
        if (h->corr_mode == RM_CORRECTOR_LEARNED && h->net && h->lc_fallback < 0) learned_coarse(h);
        else plain_coarse(h);                                      // cc -> ce
      }
    } catch (...) {
      std::swap(h->stream, b);
      throw;
    }
    std::swap(h->stream, b);
  }
  if (fork)
    for (int i = 0; i < std::min(nb, (int)rm_handle::kBranches); ++i) {
      CK(cudaEventRecord(h->join[i], h->br[i]));
      CK(cudaStreamWaitEvent(s, h->join[i], 0));
    }
  if (h->sc) CK(launch_spmv(h->Et, z, z, h->w, 2, -1.0, s));       // z_I = w_I - E^T z_G
  // the coarse term enters every row, after the interior expansion
  if (with_coarse && h->nc > 0 && h->corr_mode != RM_CORRECTOR_OFF)
    CK(launch_spmv(h->R0T, h->ce, z, nullptr, 1, 1.0, s));       // z += R_0^T ce
}

void apply(rm_handle *h, const double *x, double *y) {
  // both applies write every entry of y (cell products, then a fixed-order assembly)
  CK(launch_apply(h->ad, x, y, h->stream));
}

}  // namespace

extern "C" {

rm_options rm_default_options(void) {
  rm_options o;
  o.precision = RM_FP64;
  o.decomposition = RM_PAFW;
  o.static_condensation = 0;
  o.factor = RM_CHOL;
  o.coarse = RM_COARSE_P1;
  o.flexible = 0;
  o.rtol = 1e-8;
  o.max_it = 500;
  o.check_every = 1;
  o.profile = 0;
  o.norm = RM_NORM_L2;
  o.arith = RM_ARITH_FP64;
  o.boundary = RM_BC_DIRICHLET;
  o.coarse_smoother = RM_SMOOTH_STAR;
  o.composition = RM_ADDITIVE;
  o.hybrid_omega = 0.125;
  o.relaxation = 1;
  o.deterministic = 0;
  return o;
}

int rm_setup(rm_handle **out, int space, const rm_mesh *mesh, int p, const double *alpha,
             const double *beta, const rm_options *opt, void *stream) {
  if (!out) return fail(nullptr, RM_ERR_ARG, "rm_setup: out is NULL");
  *out = nullptr;
  if (!mesh) return fail(nullptr, RM_ERR_ARG, "rm_setup: mesh is NULL");
  if (space < 0 || space > 2) return fail(nullptr, RM_ERR_ARG, "rm_setup: space must be 0, 1 or 2");
  if (p < 1 || p > 15) return fail(nullptr, RM_ERR_ARG, "rm_setup: p must be in 1..15");
  if (mesh->nx < 2 || mesh->ny < 2 || mesh->nz < 2)
    return fail(nullptr, RM_ERR_ARG, "rm_setup: at least 2 cells per direction");
  std::unique_ptr<rm_handle> h(new rm_handle());
  const auto t_setup = std::chrono::steady_clock::now();
  try {
    h->opt = opt ? *opt : rm_default_options();
    h->stream = (cudaStream_t)stream;
    h->k = space;
    h->p = p;
    h->n[0] = mesh->nx;
    h->n[1] = mesh->ny;
    h->n[2] = mesh->nz;
    const rm_options &o = h->opt;
    if (o.precision != RM_FP64 && o.precision != RM_FP32) throw std::invalid_argument("precision");
    if (o.decomposition == RM_PH && (space == RM_HGRAD || !o.static_condensation))
      throw std::invalid_argument("RM_PH needs RM_HCURL or RM_HDIV and static_condensation = 1");
    if (o.rtol <= 0 || o.max_it < 1 || o.check_every < 1) throw std::invalid_argument("rtol/max_it/check_every");
    if (o.norm != RM_NORM_L2 && o.norm != RM_NORM_NATURAL) throw std::invalid_argument("norm");
    if (o.coarse_smoother != RM_SMOOTH_STAR && o.coarse_smoother != RM_SMOOTH_HIPTMAIR)
      throw std::invalid_argument("coarse_smoother");
    if (o.composition != RM_ADDITIVE && o.composition != RM_HYBRID) throw std::invalid_argument("composition");
    if (o.deterministic != 0 && o.deterministic != 1) throw std::invalid_argument("deterministic");
    if (o.composition == RM_HYBRID && !(o.hybrid_omega > 0.0 && o.hybrid_omega <= 1.0))
      throw std::invalid_argument("hybrid_omega must be in (0, 1]");
    if (o.arith != RM_ARITH_FP64 && o.arith != RM_ARITH_DF64) throw std::invalid_argument("arith");
    if (o.boundary != RM_BC_DIRICHLET && o.boundary != RM_BC_NONE) throw std::invalid_argument("boundary");
    h->ad.arith = o.arith == RM_ARITH_DF64 ? 1 : 0;
    h->ad.natural = o.boundary == RM_BC_NONE ? 1 : 0;
    h->vt = o.precision == RM_FP32 ? 1 : 0;
    h->sc = o.static_condensation != 0;
    h->ph = o.decomposition == RM_PH;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    h->L = Layout(space, h->n, p, o.boundary == RM_BC_NONE);
    h->size = h->L.size;
    const int ncell = h->n[0] * h->n[1] * h->n[2];
    Geometry geo;
    for (int d = 0; d < 3; ++d) geo.n[d] = h->n[d];
    const size_t nv = (size_t)(h->n[0] + 1) * (h->n[1] + 1) * (h->n[2] + 1);
    geo.X.resize(3 * nv);
    if (mesh->vertices) {
      std::memcpy(geo.X.data(), mesh->vertices, 3 * nv * sizeof(double));
    } else {
      for (int a3 = 0; a3 <= h->n[2]; ++a3)
        for (int a2 = 0; a2 <= h->n[1]; ++a2)
          for (int a1 = 0; a1 <= h->n[0]; ++a1) {
            size_t v = a1 + (size_t)(h->n[0] + 1) * (a2 + (size_t)(h->n[1] + 1) * a3);
            geo.X[3 * v + 0] = (double)a1 / h->n[0];
            geo.X[3 * v + 1] = (double)a2 / h->n[1];
            geo.X[3 * v + 2] = (double)a3 / h->n[2];
          }
    }
    std::vector<double> al(ncell, 1.0), be(ncell, 1.0);
    if (alpha) std::memcpy(al.data(), alpha, ncell * sizeof(double));
    if (beta) std::memcpy(be.data(), beta, ncell * sizeof(double));
    const bool relax_on = o.relaxation != 0;
    for (int c = 0; c < ncell; ++c)
      if (relax_on ? (!(al[c] > 0) || !(be[c] >= 0)) : (!(al[c] >= 0) || !(be[c] >= 0)))
        throw std::invalid_argument(relax_on ? "alpha must be > 0 and beta >= 0" : "alpha and beta must be >= 0");
    build_apply(h.get(), geo, al, be);
    FreeMap fm(h->L);
    h->nfree = (long long)fm.free2lat.size();
    {
      std::vector<uint8_t> mask(h->size, 1);
      for (int l : fm.free2lat) mask[l] = 0;
      h->mask = h->upload(mask);
    }
    h->op_only = !relax_on;
    if (h->op_only) {
      CK(cudaDeviceSynchronize());
      h->setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_setup).count();
      *out = h.release();
      return RM_OK;
    }
    // relaxation
    Csr P = assemble_aux(h->L, geo, be.data(), al.data(), fm);
    if (!h->sc) {
      if (o.decomposition != RM_PAFW) throw std::invalid_argument("non-condensed relaxation is PAFW only");
      PatchFamily F = build_patches(h->L, fm, P, 0, false, o.factor == RM_ICC ? 1 : 0);
      h->fam.push_back(upload_family(h.get(), F));
    } else {
      Condensed C = condense(h->L, fm, P);
      P = Csr();
      // the interior solve and the harmonic extension stay FP64 in every
      // precision: an FP32 interior expansion leaves rounding noise in the
      // cell-interior DOFs, whose stiffness (up to alpha p^4 / h^2) makes A z
      // dominated by that noise at high degree and coefficient contrast
      // (H(div), 16^3, p = 10, alpha in [1e-2, 1e2]: FCG diverged); the
      // extension of an FP32 interface correction is energy-minimising, so
      // the FP32 patch solves do not have that problem
      h->Binv = upload_csr(h.get(), C.Binv, &fm.free2lat, &fm.free2lat, &C.I, true);
      h->E = upload_csr(h.get(), C.E, &fm.free2lat, &fm.free2lat, &C.G, true);
      h->Et = upload_csr(h.get(), C.Et, &fm.free2lat, &fm.free2lat, &C.I, true);
      if (!h->ph) {
        PatchFamily F = build_patches(h->L, fm, C.S, 0, true, o.factor == RM_ICC ? 1 : 0);
        h->fam.push_back(upload_family(h.get(), F));
      } else {
        // stars of the k-entities on S, exact Cholesky (Eq. sc-asm-hiptmair):
        // edges for H(curl); faces for H(div), whose blocks of S are diagonal
        // in the FDM basis (the relaxation is point-Jacobi on S, Sec. 4.5)
        for (int m = 0; m < 3; ++m) {
          const int span = space == RM_HCURL ? (1 << m) : (7 & ~(1 << m));
          PatchFamily F = build_patches(h->L, fm, C.S, span, true, 0);
          h->fam.push_back(upload_family(h.get(), F));
        }
        // potential space V^{k-1}, B = (d phi, beta d psi) (Sec. 4.3) as its
        // auxiliary operator with derivative coefficient beta and mass
        // coefficient 0 (H(curl)) or eps beta (H(div): the curl-curl patch
        // matrices are singular, Remark after Eq. ph); stars of the
        // (k-1)-entities: vertices (H(curl)) or edges (H(div))
        Layout L0(space - 1, h->n, p, h->L.natural);
        FreeMap fm0(L0);
        std::vector<double> pmass(ncell, 0.0);
        if (space == RM_HDIV)
          for (int c = 0; c < ncell; ++c) pmass[c] = kHdivPotentialEps * be[c];
        Csr B = assemble_aux(L0, geo, pmass.data(), be.data(), fm0);
        Condensed C0 = condense(L0, fm0, B);
        if (space == RM_HCURL) {
          h->pfam.push_back(upload_family(h.get(), build_patches(L0, fm0, C0.S, 0, true, o.factor == RM_ICC ? 1 : 0)));
        } else {
          for (int m = 0; m < 3; ++m)
            h->pfam.push_back(
                upload_family(h.get(), build_patches(L0, fm0, C0.S, 1 << m, true, o.factor == RM_ICC ? 1 : 0)));
        }
        h->size0 = L0.size;
        std::vector<int> G1, G0;
        for (int f : C.G) G1.push_back(fm.free2lat[f]);
        for (int f : C0.G) G0.push_back(fm0.free2lat[f]);
        Csr D = discrete_derivative(L0, h->L, G1, G0);
        h->Dt = upload_csr(h.get(), D, nullptr, nullptr, &G1);
        h->DtT = upload_csr(h.get(), transpose(D), nullptr, nullptr, &G0);
        h->u0 = h->dalloc<double>(h->size0);
        h->v0 = h->dalloc<double>(h->size0);
      }
      h->w = h->dalloc<double>(h->size);
      h->rt = h->dalloc<double>(h->size);
    }
    if (o.coarse == RM_COARSE_P1) {
      CoarseData cd = build_coarse(h->L, geo, al.data(), be.data());
      h->nc = cd.nc;
      std::vector<int> crow(cd.nc);
      for (int i = 0; i < cd.nc; ++i) crow[i] = i;
      h->R0 = upload_csr(h.get(), cd.R0, nullptr, nullptr, &crow, true);  // coarse in FP64
      h->R0T = upload_csr(h.get(), cd.R0T, nullptr, nullptr, nullptr, true);
      h->A0inv = h->upload(cd.A0inv);
      h->cc = h->dalloc<double>(h->nc);
      h->ce = h->dalloc<double>(h->nc);
      if (space == RM_HGRAD) corrector_data(h.get(), cd, al);
    } else if (o.coarse == RM_COARSE_GMG) {
      CoarseGMG mg;
      CoarseData cd = build_coarse_gmg(h->L, geo, al.data(), be.data(), mg,
                                       o.coarse_smoother == RM_SMOOTH_HIPTMAIR);
      h->mgHip = mg.hiptmair;
      h->nc = cd.nc;
      std::vector<int> crow(cd.nc);
      for (int i = 0; i < cd.nc; ++i) crow[i] = i;
      h->R0 = upload_csr(h.get(), cd.R0, nullptr, nullptr, &crow, true);  // coarse in FP64
      h->R0T = upload_csr(h.get(), cd.R0T, nullptr, nullptr, nullptr, true);
      h->mg_levels = mg.levels;
      h->mg_ncoarsest = mg.ncoarsest;
      for (int l = 0; l <= mg.levels; ++l) {
        const int nl = mg.A[l].nrows;
        std::vector<int> rows(nl);
        for (int i = 0; i < nl; ++i) rows[i] = i;
        h->mgN.push_back(nl);
        h->mgB.push_back(h->dalloc<double>(nl));
        h->mgX.push_back(h->dalloc<double>(nl));
        if (l == mg.levels) break;
        h->mgA.push_back(upload_csr(h.get(), mg.A[l], nullptr, nullptr, &rows, true));
        std::vector<int> prow(mg.P[l].nrows), trow(mg.PT[l].nrows);
        for (size_t i = 0; i < prow.size(); ++i) prow[i] = (int)i;
        for (size_t i = 0; i < trow.size(); ++i) trow[i] = (int)i;
        h->mgP.push_back(upload_csr(h.get(), mg.P[l], nullptr, nullptr, &prow, true));
        h->mgPT.push_back(upload_csr(h.get(), mg.PT[l], nullptr, nullptr, &trow, true));
        h->mgW.push_back(h->upload(mg.dinv[l]));
        if (mg.hiptmair) {
          const int nb = mg.G[l].ncols;
          std::vector<int> grow(nl), trow(nb);
          for (int i = 0; i < nl; ++i) grow[i] = i;
          for (int i = 0; i < nb; ++i) trow[i] = i;
          h->mgG.push_back(upload_csr(h.get(), mg.G[l], nullptr, nullptr, &grow, true));
          h->mgGT.push_back(upload_csr(h.get(), mg.GT[l], nullptr, nullptr, &trow, true));
          h->mgWB.push_back(h->upload(mg.dinvB[l]));
          h->mgU.push_back(h->dalloc<double>(nb));
          h->mgNB.push_back(nb);
        }
        if (!mg.star.empty()) {
          const int saved = h->vt;
          h->vt = 0;  // the coarse cycle stays in FP64
          h->mgStar.push_back(upload_family(h.get(), mg.star[l]));
          h->vt = saved;
          h->mgOmega = mg.star_omega;
        }
        h->mgT.push_back(h->dalloc<double>(nl));
        h->mgR.push_back(h->dalloc<double>(nl));
      }
      h->mgAinv = h->upload(mg.Ainv);
      h->cc = h->mgB[0];
      h->ce = h->mgX[0];
      if (space == RM_HGRAD) corrector_data(h.get(), cd, al);
    }
    if (o.composition == RM_HYBRID) {
      h->hy_t = h->dalloc<double>(h->size);
      h->hy_w = h->dalloc<double>(h->size);
    }
    h->r = h->dalloc<double>(h->size);
    h->z = h->dalloc<double>(h->size);
    h->pv = h->dalloc<double>(h->size);
    h->qv = h->dalloc<double>(h->size);
    h->scal = h->dalloc<double>(S_COUNT);
    h->partial = h->dalloc<double>(kPartialDoubles);
    CK(cudaMemset(h->partial, 0, kPartialDoubles * sizeof(double)));
    CK(cudaMallocHost((void **)&h->hscal, S_COUNT * sizeof(double)));
    h->hrr = h->dalloc<double>((size_t)o.max_it + 1);
    h->hrz = h->dalloc<double>((size_t)o.max_it + 1);
    CK(cudaEventCreate(&h->ev0));
    CK(cudaEventCreate(&h->ev1));
    CK(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
    for (int i = 0; i < rm_handle::kBranches; ++i) {
      CK(cudaStreamCreateWithFlags(&h->br[i], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&h->join[i], cudaEventDisableTiming));
    }
    CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    CK(cudaDeviceSynchronize());
    refresh_noalloc_scratch(dev);
  } catch (const CudaError &e) {
    return fail(nullptr, RM_ERR_CUDA, std::string("rm_setup: ") + e.what());
  } catch (const std::bad_alloc &) {
    return fail(nullptr, RM_ERR_OOM, "rm_setup: host allocation failed");
  } catch (const std::invalid_argument &e) {
    return fail(nullptr, RM_ERR_ARG, std::string("rm_setup: invalid option: ") + e.what());
  } catch (const std::exception &e) {
    std::string w = e.what();
    int code = w.find("breakdown") != std::string::npos ? RM_ERR_BREAKDOWN : RM_ERR_ARG;
    return fail(nullptr, code, std::string("rm_setup: ") + w);
  }
  h->setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_setup).count();
  *out = h.release();
  return RM_OK;
}

int rm_ndofs(const rm_handle *h, long long *lattice, long long *free_dofs) {
  if (!h) return fail(nullptr, RM_ERR_ARG, "rm_ndofs: NULL handle");
  if (lattice) *lattice = h->size;
  if (free_dofs) *free_dofs = h->nfree;
  return RM_OK;
}

int rm_stats(const rm_handle *h, long long *patches, long long *slots, long long *factor_nnz) {
  if (!h) return fail(nullptr, RM_ERR_ARG, "rm_stats: NULL handle");
  if (patches) *patches = h->stat_patches;
  if (slots) *slots = h->stat_slots;
  if (factor_nnz) *factor_nnz = h->stat_nnz;
  return RM_OK;
}

int rm_layout(const rm_handle *h, int comp, int dims[3], long long *offset) {
  if (!h || !dims) return fail(nullptr, RM_ERR_ARG, "rm_layout: NULL argument");
  if (comp < 0 || comp >= h->L.ncomp)
    return fail(nullptr, RM_ERR_ARG, "rm_layout: component out of range");
  for (int d = 0; d < 3; ++d) dims[d] = (int)h->L.N[comp][d];
  if (offset) *offset = h->L.off[comp];
  return RM_OK;
}

int rm_history(const rm_handle *h, int which, double *out, int cap, int *len) {
  if (!h || (!out && cap > 0) || cap < 0) return fail(nullptr, RM_ERR_ARG, "rm_history: bad argument");
  if (which != RM_NORM_L2 && which != RM_NORM_NATURAL) return fail(nullptr, RM_ERR_ARG, "rm_history: which");
  const double *src = which == RM_NORM_L2 ? h->hrr : h->hrz;
  const int nrec = which == RM_NORM_L2 ? h->nhrr : h->nhrz;
  const int m = std::min(cap, nrec);
  if (len) *len = m;
  if (m == 0) return RM_OK;
  std::vector<double> v(nrec);
  // the first entry normalises: ||b|| for the l2 history (recorded as b's
  // masked norm in the scalars), (r_0, B r_0) for the natural one
  cudaError_t e = cudaMemcpy(v.data(), src, nrec * sizeof(double), cudaMemcpyDeviceToHost);
  double bb = 0.0;
  if (e == cudaSuccess && which == RM_NORM_L2)
    e = cudaMemcpy(&bb, h->scal + S_BB, sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(nullptr, RM_ERR_CUDA, std::string("rm_history: ") + cudaGetErrorString(e));
  const double d = which == RM_NORM_L2 ? bb : v[0];
  for (int k = 0; k < m; ++k) out[k] = d > 0.0 ? std::sqrt(std::max(0.0, v[k]) / d) : 0.0;
  return RM_OK;
}

int rm_apply(rm_handle *h, const double *x, double *y) {
  if (!h || !x || !y) return fail(h, RM_ERR_ARG, "rm_apply: NULL argument");
  try {
    apply(h, x, y);
  } catch (const std::exception &e) {
    return fail(h, RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}

int rm_precondition(rm_handle *h, const double *r, double *z) {
  if (!h || !r || !z) return fail(h, RM_ERR_ARG, "rm_precondition: NULL argument");
  if (h->op_only) return fail(h, RM_ERR_ARG, "rm_precondition: handle built with relaxation = 0");
  if (r == z) return fail(h, RM_ERR_ARG, "rm_precondition: r and z must not alias");
  try {
    precondition(h, r, z);
  } catch (const std::exception &e) {
    return fail(h, RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}

int rm_solve(rm_handle *h, const double *b, double *x, rm_info *info) {
  if (!h || !b || !x) return fail(h, RM_ERR_ARG, "rm_solve: NULL argument");
  if (h->op_only) return fail(h, RM_ERR_ARG, "rm_solve: handle built with relaxation = 0");
  const long long n = h->size;
  cudaStream_t s = h->stream;
  int status = RM_OK, it = 0;
  double rel = 0.0;
  float ms = 0.f;
  const bool prof = h->opt.profile != 0;
  std::vector<int> kinds;  // 0 apply, 1 precondition, per recorded pair
  auto timed = [&](int kind, const std::function<void()> &f) {
    if (!prof) { f(); return; }
    size_t i = 2 * kinds.size();
    while (h->evpool.size() < i + 2) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      h->evpool.push_back(e);
    }
    CK(cudaEventRecord(h->evpool[i], s));
    f();
    CK(cudaEventRecord(h->evpool[i + 1], s));
    kinds.push_back(kind);
  };
  double tk[2] = {0.0, 0.0};
  const long long launches0 = launch_count();
  h->lc_calls = 0;
  h->lc_judged = 0;
  h->lc_fallback = -1;
  h->lc_eta = -1.0;
  // the learned coarse term makes the preconditioner nonlinear: flexible CG
  const int flexible = h->opt.flexible || (h->corr_mode == RM_CORRECTOR_LEARNED && h->net);
  int nk[2] = {0, 0};
  try {
    CK(cudaEventRecord(h->ev0, s));
    // x Dirichlet entries -> 0; r = b - A x
    CK(launch_mask_copy(n, h->mask, x, x, s));
    timed(0, [&] { apply(h, x, h->qv); });
    CK(launch_sub(n, h->mask, b, h->qv, h->r, s));
    CK(launch_mask_copy(n, h->mask, b, h->z, s));
    CK(launch_dot(n, h->z, h->z, h->partial, h->scal, S_BB, s));
    CK(launch_dot(n, h->r, h->r, h->partial, h->scal, S_RR, s, h->hrr));
    h->nhrr = 1;
    h->nhrz = 0;
    timed(1, [&] { precondition(h, h->r, h->z); });
    // replay the preconditioner as a graph unless it talks to the host (the
    // learned corrector's judge) or records coarse residuals
    const bool replay = h->corr_mode != RM_CORRECTOR_LEARNED && !(h->rec && h->rec_n < h->rec_cap);
    if (replay && (!h->pgraph || h->pgraph_mode != h->corr_mode)) {
      if (h->pgraph) CK(cudaGraphExecDestroy(h->pgraph));
      h->pgraph = nullptr;
      const long long l0 = launch_count();
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed));
      h->stream = h->cap;  // precondition() launches on h->stream
      try {
        precondition(h, h->r, h->z);
      } catch (...) {
        h->stream = s;
        cudaStreamEndCapture(h->cap, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      h->stream = s;
      CK(cudaStreamEndCapture(h->cap, &g));
      h->pgraph_launches = launch_count() - l0;
      add_launches(-h->pgraph_launches);  // captured, not launched
      cudaGraphExec_t ge = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      CK(ei);
      h->pgraph = ge;
      h->pgraph_mode = h->corr_mode;
    }
    auto prec = [&] {
      if (replay) {
        CK(cudaGraphLaunch(h->pgraph, s));
        add_launches(h->pgraph_launches);
      } else {
        precondition(h, h->r, h->z);
      }
    };
    CK(launch_dot(n, h->r, h->z, h->partial, h->scal, S_RZ, s, h->hrz));
    h->nhrz = 1;
    CK(cudaMemcpyAsync(h->pv, h->z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->hscal, h->scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double bb = h->hscal[S_BB];
    const double tol2 = h->opt.rtol * h->opt.rtol * bb;
    // natural norm (Sec. 5.1): (r_k, B r_k) <= rtol^2 (r_0, B r_0)
    const bool natural = h->opt.norm == RM_NORM_NATURAL;
    const double rz0 = h->hscal[S_RZ];
    const double tol2n = h->opt.rtol * h->opt.rtol * rz0;
    double rr = h->hscal[S_RR];
    if (bb == 0.0) {
      rel = 0.0;
    } else if (!std::isfinite(rr) || !std::isfinite(rz0)) {
      status = RM_ERR_NAN;
      rel = std::sqrt(rr / bb);
    } else if (rr == 0.0 || (!natural && rr <= tol2)) {
      rel = std::sqrt(rr / bb);
    } else if (natural && !(rz0 > 0.0)) {
      status = RM_ERR_BREAKDOWN;  // (r_0, B r_0) <= 0: B is not positive definite
      rel = std::sqrt(rr / bb);
    } else {
      status = RM_ERR_NOT_CONVERGED;
      while (it < h->opt.max_it) {
        timed(0, [&] { apply(h, h->pv, h->qv); });
        CK(launch_alpha(n, h->pv, h->qv, h->partial, h->scal, s));
        CK(launch_update_xr(n, x, h->r, h->pv, h->qv, h->partial, h->scal, s, h->hrr + it + 1));
        ++it;
        h->nhrr = it + 1;
        const bool check = it % h->opt.check_every == 0 || it == h->opt.max_it;
        if (!natural && check) {
          CK(cudaMemcpyAsync(h->hscal, h->scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
          CK(cudaStreamSynchronize(s));
          rr = h->hscal[S_RR];
          if (!std::isfinite(rr)) { status = RM_ERR_NAN; break; }
          if (!(h->hscal[S_PQ] > 0.0)) { status = RM_ERR_BREAKDOWN; break; }
          if (rr <= tol2) { status = RM_OK; break; }
        }
        timed(1, prec);
        CK(launch_dot2(n, h->r, h->z, h->qv, h->partial, h->scal, flexible, s, h->hrz + it));
        h->nhrz = it + 1;
        if (natural && check) {
          CK(cudaMemcpyAsync(h->hscal, h->scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
          CK(cudaStreamSynchronize(s));
          rr = h->hscal[S_RR];
          const double rz = h->hscal[S_RZ];
          if (!std::isfinite(rr) || !std::isfinite(rz)) { status = RM_ERR_NAN; break; }
          if (!(h->hscal[S_PQ] > 0.0)) { status = RM_ERR_BREAKDOWN; break; }
          if (rz <= tol2n) { status = RM_OK; break; }
        }
        CK(launch_update_p(n, h->pv, h->z, h->scal, s));
      }
      if (natural) rr = h->hscal[S_RR];
      rel = std::sqrt(rr / bb);
    }
    CK(cudaEventRecord(h->ev1, s));
    CK(cudaEventSynchronize(h->ev1));
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    {
      cudaError_t te = cudaSuccess;
      if (patch_timeouts(&te)) status = RM_ERR_TIMEOUT;  // a patch kernel's bounded wait gave up
      CK(te);
      if (h->net && rmn::conv_timeouts(&te)) status = RM_ERR_TIMEOUT;  // a tensor-core conv's wait
      CK(te);
    }
    for (size_t j = 0; j < kinds.size(); ++j) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, h->evpool[2 * j], h->evpool[2 * j + 1]));
      tk[kinds[j]] += t;
      nk[kinds[j]]++;
    }
  } catch (const std::exception &e) {
    if (info) info->status = RM_ERR_CUDA;
    return fail(h, RM_ERR_CUDA, e.what());
  }
  // the natural-norm history: its final ratio and the paper's count
  double rel_nat = -1.0;
  int it_nat = -1;
  if (h->nhrz > 0) {
    std::vector<double> hz(h->nhrz);
    if (cudaMemcpy(hz.data(), h->hrz, h->nhrz * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess &&
        hz[0] > 0.0) {
      for (int k = 0; k < h->nhrz; ++k) {
        const double ratio = std::sqrt(std::max(0.0, hz[k]) / hz[0]);
        rel_nat = ratio;
        if (it_nat < 0 && ratio <= h->opt.rtol) it_nat = k;
      }
    }
  }
  if (info) {
    info->iterations = it;
    info->status = status;
    info->rel_res_l2 = rel;
    info->rel_res_natural = rel_nat;
    info->iterations_natural = it_nat;
    info->history_len = h->nhrr;
    info->setup_s = h->setup_s;
    info->solve_ms = ms;
    info->apply_ms = tk[0];
    info->apply_calls = nk[0];
    info->precond_ms = tk[1];
    info->precond_calls = nk[1];
    info->kernel_launches = launch_count() - launches0;
    const bool learned = h->corr_mode == RM_CORRECTOR_LEARNED && h->net;
    info->learned_calls =
        learned ? (h->lc_fallback < 0 ? h->lc_calls : h->lc_fallback) : 0;
    info->judge_calls = h->lc_judged;
    info->fallback_at = h->lc_fallback;
    info->judge_eta = h->lc_eta;
  }
  if (status != RM_OK) {
    const char *why = status == RM_ERR_NOT_CONVERGED ? "max_it reached"
                      : status == RM_ERR_NAN         ? "NaN/Inf residual"
                      : status == RM_ERR_TIMEOUT     ? "a device wait timed out in the relaxation"
                                                     : "CG breakdown (p^T A p <= 0 or r^T B r <= 0)";
    fail(h, status, std::string("rm_solve: ") + why);
  }
  return status;
}

void rm_destroy(rm_handle *h) { delete h; }

const char *rm_last_error(const rm_handle *h) {
  if (h) return h->err.c_str();
  return g_last_error.c_str();
}

// ---------------------------------------------------------------------------
// learned coarse corrector

// iterations of each one-level solve that supplies training pairs
static const int kOffSolveIterations = 64;

rm_train_options rm_default_train_options(void) {
  rm_train_options o;
  o.pairs = 2000;
  o.epochs = 20;
  o.batch = 16;
  o.lr = 1e-3f;
  o.levels = 3;
  o.width = 16;
  o.seed = 20221125ULL;
  o.val_fraction = 0.1;
  o.target_cycles = 12;
  o.off_fraction = 0.0;
  o.rounds = 0;
  o.round_pairs = 500;
  o.round_epochs = 5;
  return o;
}

int rm_corrector_train(rm_handle *h, const rm_train_options *opt, int nrhs, const double *rhs,
                       rm_train_info *info) {
  if (!h || !rhs || nrhs < 1) return fail(h, RM_ERR_ARG, "rm_corrector_train: bad argument");
  if (h->k != RM_HGRAD || !h->c_logal)
    return fail(h, RM_ERR_ARG,
                "rm_corrector_train: needs an H(grad) handle with RM_COARSE_P1 or RM_COARSE_GMG");
  const rm_train_options o = opt ? *opt : rm_default_train_options();
  if (o.pairs < 2 || o.epochs < 1 || o.batch < 1 || o.batch > 256 || !(o.lr > 0.f) ||
      o.levels < 0 || o.levels > 4 || o.width < 1 || o.width > 128 || !(o.val_fraction >= 0.0) ||
      o.val_fraction > 0.5 || o.target_cycles < 1 || !(o.off_fraction >= 0.0) ||
      o.off_fraction > 1.0 || o.rounds < 0 || o.rounds > 16 || o.round_pairs < 1 || o.round_epochs < 1)
    return fail(h, RM_ERR_ARG, "rm_corrector_train: option out of range");
  for (int d = 0; d < 3; ++d)
    if (h->n[d] % (1 << o.levels) != 0)
      return fail(h, RM_ERR_ARG, "rm_corrector_train: the mesh size must be divisible by 2^levels");
  using clock = std::chrono::steady_clock;
  cudaStream_t s = h->stream;
  const int nc = h->nc;
  const long long nv = h->cnvox;
  const int saved_mode = h->corr_mode;
  try {
    const auto t0 = clock::now();
    // 1. r_0 = R_0 r at every preconditioner call of plain solves
    const int total_pairs = o.pairs + o.rounds * o.round_pairs;
    DevBuf recb, xb;
    CK(cudaMalloc(&recb.p, (size_t)total_pairs * nc * sizeof(double)));
    CK(cudaMalloc(&xb.p, h->size * sizeof(double)));
    double *rec = (double *)recb.p, *x = (double *)xb.p;
    h->rec = rec;
    h->rec_n = 0;
    int solves = 0;
    // the first off_fraction of the pairs from one-level solves (no coarse
    // term: residuals rich in the coarse-scale error the corrector must
    // remove), the rest from plain two-level solves
    const int n_off = (int)(o.off_fraction * o.pairs);
    const int max_it = h->opt.max_it;
    for (int i = 0; i < nrhs && h->rec_n < o.pairs; ++i) {
      const bool off = h->rec_n < n_off;
      h->corr_mode = off ? RM_CORRECTOR_OFF : RM_CORRECTOR_PLAIN;
      h->rec_cap = off ? n_off : o.pairs;
      h->opt.max_it = off ? std::min(max_it, kOffSolveIterations) : max_it;
      CK(cudaMemsetAsync(x, 0, h->size * sizeof(double), s));
      rm_info inf;
      const int st = rm_solve(h, rhs + (size_t)i * h->size, x, &inf);
      h->opt.max_it = max_it;
      ++solves;
      if (st != RM_OK && st != RM_ERR_NOT_CONVERGED) throw std::runtime_error(h->err);
    }
    h->rec = nullptr;
    h->rec_cap = 0;
    h->corr_mode = saved_mode;
    const int np = h->rec_n;
    if (np < o.pairs)
      return fail(h, RM_ERR_ARG,
                  "rm_corrector_train: " + std::to_string(nrhs) + " right-hand sides gave only " +
                      std::to_string(np) + " pairs; pass more");
    // 2. targets c* = A_0^-1 r_0; inputs and targets scaled to sqrt(nc) / norm
    DevBuf Rb, Tb, cb, db;
    CK(cudaMalloc(&Rb.p, (size_t)total_pairs * nc * sizeof(float)));
    CK(cudaMalloc(&Tb.p, (size_t)total_pairs * nc * sizeof(float)));
    CK(cudaMalloc(&cb.p, (size_t)nc * sizeof(double)));
    CK(cudaMalloc(&db.p, (size_t)3 * total_pairs * sizeof(double)));
    float *R = (float *)Rb.p, *T = (float *)Tb.p;
    double *cs = (double *)cb.p, *dd = (double *)db.p;
    // targets c* = A_0^-1 r_0 of the recorded pairs j0 .. j1-1, their norms,
    // and the network's scaled inputs and targets
    auto make_targets = [&](int j0, int j1) {
    for (int j = j0; j < j1; ++j) {
      const double *r0 = rec + (size_t)j * nc;
      if (h->mgAinv) {
        CK(cudaMemsetAsync(cs, 0, nc * sizeof(double), s));
        for (int c = 0; c < o.target_cycles; ++c) {
          CK(launch_spmv(h->A0, cs, h->mgB[0], r0, 2, -1.0, s));  // B = r0 - A0 c
          vcycle(h, 0);
          CK(launch_axpy(nc, 1.0, h->mgX[0], cs, 1, s));
        }
      } else {
        CK(launch_gemv(nc, h->A0inv, 0, r0, cs, s));
      }
      CK(launch_dot(nc, r0, r0, h->lpart, dd, 3 * j, s));
      CK(launch_dot(nc, cs, cs, h->lpart, dd, 3 * j + 1, s));
      CK(launch_dot(nc, r0, cs, h->lpart, dd, 3 * j + 2, s));
      rmn::corr_normalise(nc, r0, dd + 3 * j, R + (size_t)j * nc, s);
      rmn::corr_normalise(nc, cs, dd + 3 * j + 1, T + (size_t)j * nc, s);
    }
    };
    make_targets(0, np);
    std::vector<double> hd(3 * (size_t)total_pairs);
    CK(cudaMemcpyAsync(hd.data(), dd, 3 * (size_t)np * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double gen_s = std::chrono::duration<double>(clock::now() - t0).count();
    // 3. split (seeded permutation), network, training
    uint64_t st = o.seed ^ 0x5DEECE66DULL;
    auto next = [&st]() {
      uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
      return z ^ (z >> 31);
    };
    std::vector<int> perm(np);
    for (int j = 0; j < np; ++j) perm[j] = j;
    for (int j = np - 1; j > 0; --j) std::swap(perm[j], perm[next() % (uint64_t)(j + 1)]);
    const int nval = std::min(np - 1, (int)(o.val_fraction * np));
    int ntrain = np - nval;
    if (h->net) {
      rmn::destroy(h->net);
      h->net = nullptr;
    }
    rmn::NetSpec spec{{h->cdims[0], h->cdims[1], h->cdims[2]}, o.levels, o.width, 2, o.batch};
    h->net = rmn::create(spec, o.seed, s);
    DevBuf Xb, Ttb, Yb, dYb, mb, ib, lb;
    const int B = o.batch;
    CK(cudaMalloc(&Xb.p, (size_t)B * nv * 2 * sizeof(float)));
    CK(cudaMalloc(&Ttb.p, (size_t)B * nv * sizeof(float)));
    CK(cudaMalloc(&Yb.p, (size_t)B * nv * sizeof(float)));
    CK(cudaMalloc(&dYb.p, (size_t)B * nv * sizeof(float)));
    CK(cudaMalloc(&mb.p, (size_t)nv));
    CK(cudaMalloc(&ib.p, (size_t)total_pairs * sizeof(int)));
    CK(cudaMalloc(&lb.p, 2 * sizeof(double)));
    float *X = (float *)Xb.p, *Tt = (float *)Ttb.p, *Y = (float *)Yb.p, *dY = (float *)dYb.p;
    uint8_t *mask = (uint8_t *)mb.p;
    int *idx = (int *)ib.p;
    double *loss = (double *)lb.p;
    {
      std::vector<int> l2f(nv);
      CK(cudaMemcpy(l2f.data(), h->c_lat2free, nv * sizeof(int), cudaMemcpyDeviceToHost));
      std::vector<uint8_t> m(nv);
      for (long long v = 0; v < nv; ++v) m[v] = l2f[v] >= 0;
      CK(cudaMemcpy(mask, m.data(), nv, cudaMemcpyHostToDevice));
    }
    const auto t1 = clock::now();
    double train_loss = 0.0;
    // epochs over the training pairs perm[0 .. ntrain); lr halved at 1/2
    // and 3/4 of the epochs of this call
    auto train = [&](int epochs, float lr0) {
      for (int e = 0; e < epochs; ++e) {
        for (int j = ntrain - 1; j > 0; --j) std::swap(perm[j], perm[next() % (uint64_t)(j + 1)]);
        CK(cudaMemcpyAsync(idx, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        float lr = lr0;
        if (2 * e >= epochs) lr *= 0.5f;
        if (4 * e >= 3 * epochs) lr *= 0.5f;
        CK(cudaMemsetAsync(loss, 0, sizeof(double), s));
        int nb = 0;
        for (int off = 0; off < ntrain; off += B) {
          const int bs = std::min(B, ntrain - off);
          rmn::corr_batch(bs, nc, nv, idx + off, R, T, h->c_lat2free, h->c_logal, X, Tt, s);
          rmn::forward(h->net, bs, X, Y);
          rmn::mse(bs, (int)nv, Y, Tt, mask, 1.f / ((float)bs * nc), dY, loss, s);
          rmn::backward(h->net, dY, nullptr);
          rmn::adam(h->net, lr, 0.9f, 0.999f, 1e-8f);
          ++nb;
        }
        double hl = 0.0;
        CK(cudaMemcpyAsync(&hl, loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        train_loss = hl / nb;
      }
    };
    train(o.epochs, o.lr);
    // on-policy rounds: residuals of solves that use the current network
    // (they drift away from those of plain solves), appended to the
    // training pairs; the held-out pairs stay the first recording's
    for (int rd = 0; rd < o.rounds; ++rd) {
      const int j0 = h->rec_n;
      h->rec = rec;
      h->rec_cap = j0 + o.round_pairs;
      h->corr_mode = RM_CORRECTOR_LEARNED;
      const int saved_je = h->judge_every;
      h->judge_every = 0;
      for (int i = 0; h->rec_n < h->rec_cap; ++i) {
        CK(cudaMemsetAsync(x, 0, h->size * sizeof(double), s));
        rm_info inf;
        const int st = rm_solve(h, rhs + (size_t)(i % nrhs) * h->size, x, &inf);
        ++solves;
        if (st != RM_OK && st != RM_ERR_NOT_CONVERGED) {
          h->judge_every = saved_je;
          throw std::runtime_error(h->err);
        }
        if (i > 4 * nrhs) break;  // solves that record nothing (converged at once)
      }
      h->judge_every = saved_je;
      h->rec = nullptr;
      h->rec_cap = 0;
      h->corr_mode = saved_mode;
      const int j1 = h->rec_n;
      if (j1 == j0) break;
      make_targets(j0, j1);
      CK(cudaMemcpyAsync(hd.data() + 3 * (size_t)j0, dd + 3 * (size_t)j0, 3 * (size_t)(j1 - j0) * sizeof(double),
                         cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      // new pairs join the training part of perm, before the held-out ones
      std::vector<int> np2(perm.begin(), perm.begin() + ntrain);
      for (int j = j0; j < j1; ++j) np2.push_back(j);
      np2.insert(np2.end(), perm.begin() + ntrain, perm.end());
      perm.swap(np2);
      ntrain += j1 - j0;
      train(o.round_epochs, 0.5f * o.lr);
    }
    const int np_all = (int)perm.size();
    const double train_s = std::chrono::duration<double>(clock::now() - t1).count();
    // 4. held-out pairs: loss and eta of the optimally scaled correction
    double val_loss = 0.0, val_eta = 0.0;
    if (nval > 0) {
      DevBuf vb;
      CK(cudaMalloc(&vb.p, 2 * (size_t)nval * sizeof(double)));
      double *vd = (double *)vb.p;
      CK(cudaMemsetAsync(loss, 0, sizeof(double), s));
      int nb = 0;
      for (int off = ntrain; off < np_all; off += B) {
        const int bs = std::min(B, np_all - off);
        rmn::corr_batch(bs, nc, nv, idx + off, R, T, h->c_lat2free, h->c_logal, X, Tt, s);
        rmn::forward(h->net, bs, X, Y);
        rmn::mse(bs, (int)nv, Y, Tt, mask, 1.f / ((float)bs * nc), dY, loss, s);
        for (int b = 0; b < bs; ++b) {
          const int j = perm[off + b], v = off + b - ntrain;
          rmn::corr_gather(nc, Y + (size_t)b * nv, h->c_free2lat, h->cl, s);
          CK(launch_spmv(h->A0, h->cl, h->cq, nullptr, 0, 1.0, s));
          CK(launch_dot(nc, h->cl, rec + (size_t)j * nc, h->lpart, vd, 2 * v, s));
          CK(launch_dot(nc, h->cl, h->cq, h->lpart, vd, 2 * v + 1, s));
        }
        ++nb;
      }
      std::vector<double> hv(2 * (size_t)nval);
      double hl = 0.0;
      CK(cudaMemcpyAsync(hv.data(), vd, hv.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&hl, loss, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      val_loss = hl / nb;
      for (int v = 0; v < nval; ++v) {
        const double a = hv[2 * v], b = hv[2 * v + 1], ee = hd[3 * (size_t)perm[ntrain + v] + 2];
        double eta = 1.0;
        if (b > 0.0 && ee > 0.0) eta = std::sqrt(std::min(1.0, std::max(0.0, 1.0 - a * a / (b * ee))));
        val_eta += eta / nval;
      }
    }
    if (info) {
      info->pairs = np_all;
      info->solves = solves;
      info->params = rmn::num_params(h->net);
      info->gen_s = gen_s;
      info->train_s = train_s;
      info->train_loss = train_loss;
      info->val_loss = val_loss;
      info->val_eta = val_eta;
    }
  } catch (const std::exception &e) {
    h->rec = nullptr;
    h->rec_cap = 0;
    h->corr_mode = saved_mode;
    return fail(h, RM_ERR_CUDA, std::string("rm_corrector_train: ") + e.what());
  }
  return RM_OK;
}

int rm_corrector_save(const rm_handle *h, const char *path) {
  if (!h || !path || !h->net) return fail(nullptr, RM_ERR_ARG, "rm_corrector_save: no network");
  try {
    const rmn::NetSpec &sp = rmn::spec(h->net);
    const long long np = rmn::num_params(h->net);
    std::vector<float> w(np);
    rmn::get_params(h->net, w.data());
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(nullptr, RM_ERR_ARG, std::string("rm_corrector_save: cannot open ") + path);
    int32_t hdr[6] = {sp.dims[0], sp.dims[1], sp.dims[2], sp.levels, sp.width, sp.in_ch};
    int64_t n64 = np;
    bool ok = std::fwrite("RMCORR01", 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              std::fwrite(&n64, sizeof(n64), 1, f) == 1 &&
              std::fwrite(w.data(), sizeof(float), np, f) == (size_t)np;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(nullptr, RM_ERR_ARG, "rm_corrector_save: write failed");
  } catch (const std::exception &e) {
    return fail(nullptr, RM_ERR_CUDA, std::string("rm_corrector_save: ") + e.what());
  }
  return RM_OK;
}

int rm_corrector_load(rm_handle *h, const char *path) {
  if (!h || !path) return fail(h, RM_ERR_ARG, "rm_corrector_load: NULL argument");
  if (h->k != RM_HGRAD || !h->c_logal)
    return fail(h, RM_ERR_ARG,
                "rm_corrector_load: needs an H(grad) handle with RM_COARSE_P1 or RM_COARSE_GMG");
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(h, RM_ERR_ARG, std::string("rm_corrector_load: cannot open ") + path);
  char magic[8];
  int32_t hdr[6];
  int64_t n64 = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "RMCORR01", 8) == 0 &&
            std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(&n64, sizeof(n64), 1, f) == 1;
  if (!ok || hdr[0] != h->cdims[0] || hdr[1] != h->cdims[1] || hdr[2] != h->cdims[2] ||
      hdr[5] != 2 || n64 <= 0) {
    std::fclose(f);
    return fail(h, RM_ERR_ARG,
                "rm_corrector_load: not a corrector file for this coarse grid (magic, dims or channels)");
  }
  try {
    rmn::NetSpec spec{{hdr[0], hdr[1], hdr[2]}, hdr[3], hdr[4], hdr[5], 1};
    rmn::Net *net = rmn::create(spec, 0, h->stream);
    if (rmn::num_params(net) != n64) {
      rmn::destroy(net);
      std::fclose(f);
      return fail(h, RM_ERR_ARG, "rm_corrector_load: parameter count does not match the layers");
    }
    std::vector<float> w(n64);
    const bool rd = std::fread(w.data(), sizeof(float), n64, f) == (size_t)n64;
    std::fclose(f);
    f = nullptr;
    if (!rd) {
      rmn::destroy(net);
      return fail(h, RM_ERR_ARG, "rm_corrector_load: truncated file");
    }
    rmn::set_params(net, w.data());
    if (h->net) rmn::destroy(h->net);
    h->net = net;
  } catch (const std::exception &e) {
    if (f) std::fclose(f);
    return fail(h, RM_ERR_CUDA, std::string("rm_corrector_load: ") + e.what());
  }
  return RM_OK;
}

int rm_corrector_use(rm_handle *h, int mode, int judge_every, double judge_max) {
  if (!h) return fail(nullptr, RM_ERR_ARG, "rm_corrector_use: NULL handle");
  if (mode < RM_CORRECTOR_PLAIN || mode > RM_CORRECTOR_OFF || judge_every < 0 || !(judge_max >= 0.0))
    return fail(h, RM_ERR_ARG, "rm_corrector_use: bad mode, judge_every or judge_max");
  if (mode == RM_CORRECTOR_LEARNED && !h->net)
    return fail(h, RM_ERR_ARG, "rm_corrector_use: no network; train or load one first");
  h->corr_mode = mode;
  h->judge_every = judge_every;
  h->judge_max = judge_max;
  // a new mode starts without a fallback (rm_solve also resets these)
  h->lc_calls = 0;
  h->lc_judged = 0;
  h->lc_fallback = -1;
  h->lc_eta = -1.0;
  return RM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free preconditioner entry point.
//
// Its scratch (the restricted residual and the coarse solution of the p = 1
// correction) lives in the file-scope device array g_noalloc_scratch instead
// of in buffers owned by the handle.  Every GPU that loads the library holds
// the array (2 x RM_NOALLOC_MAX_COARSE doubles = 128 KiB) until the process
// exits.  Its device address was looked up by rm_setup, so a call only reads
// the cached pointer.  All calls share the array and it keeps the last call's
// contents; both halves are fully overwritten before they are read, so
// nothing needs clearing.  Calls whose work overlaps on the GPU (on different
// streams) race on the array.
// ---------------------------------------------------------------------------

extern "C" int rm_debug_patch_timeout(int on) {
  const cudaError_t e = patch_inject_timeout(on);
  if (e != cudaSuccess) return fail(nullptr, RM_ERR_CUDA, std::string("rm_debug_patch_timeout: ") + cudaGetErrorString(e));
  return RM_OK;
}

extern "C" int rm_precondition_noalloc(rm_handle *h, const double *r, double *z) {
  if (!h || !r || !z) return fail(h, RM_ERR_ARG, "rm_precondition_noalloc: NULL argument");
  if (r == z) return fail(h, RM_ERR_ARG, "rm_precondition_noalloc: r and z must not alias");
  if (h->sc)
    return fail(h, RM_ERR_ARG,
                "rm_precondition_noalloc: statically condensed relaxations need "
                "lattice-sized scratch; use rm_precondition");
  if (h->opt.deterministic)
    return fail(h, RM_ERR_ARG,
                "rm_precondition_noalloc: the deterministic relaxation gathers from per-patch "
                "scratch; use rm_precondition");
  if (h->mgAinv)
    return fail(h, RM_ERR_ARG,
                "rm_precondition_noalloc: the coarse multigrid cycle needs per-level vectors; "
                "use rm_precondition");
  if (h->corr_mode == RM_CORRECTOR_LEARNED)
    return fail(h, RM_ERR_ARG,
                "rm_precondition_noalloc: the learned coarse term needs the network's buffers; "
                "use rm_precondition");
  if (h->nc > RM_NOALLOC_MAX_COARSE)
    return fail(h, RM_ERR_ARG,
                "rm_precondition_noalloc: coarse space has " + std::to_string(h->nc) +
                    " DOFs, more than RM_NOALLOC_MAX_COARSE = " +
                    std::to_string(RM_NOALLOC_MAX_COARSE));
  try {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    double *scratch = noalloc_scratch(dev);
    double *cc = scratch, *ce = scratch + RM_NOALLOC_MAX_COARSE;
    cudaStream_t s = h->stream;
    CK(cudaMemsetAsync(z, 0, h->size * sizeof(double), s));
    for (auto &F : h->fam) CK(launch_patches(F, r, z, s));
    if (h->nc > 0 && h->corr_mode != RM_CORRECTOR_OFF) {
      CK(launch_spmv(h->R0, r, cc, nullptr, 0, 1.0, s));
      CK(launch_gemv(h->nc, h->A0inv, 0, cc, ce, s));
      CK(launch_spmv(h->R0T, ce, z, nullptr, 1, 1.0, s));
    }
  } catch (const std::exception &e) {
    return fail(h, RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}
