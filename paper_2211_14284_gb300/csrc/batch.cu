// Batched solver: many independent Riesz-map problems (uneven mesh size and
// degree, Cartesian meshes) solved together.  Every problem is set up on the
// host as rm_setup would; the device objects are then concatenated into one
// block-diagonal system: vectors back to back, SpMV matrices with offset
// rows/columns, patch families of identical templates (same space, p and
// family) merged into one launch, every problem's apply by the per-handle
// Cartesian kernel pair on its slice of the vectors.  CG runs in lock step
// with per-problem scalars and convergence masks entirely on the device; one
// iteration is captured in a CUDA graph and replayed `check_every` times
// between host reads of the convergence flags.  The assembly grid per
// (space, degree) is picked at setup by timing the candidates (autotuner).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/rm.h"
#include "device.cuh"
#include "host_basis.h"
#include "host_setup.h"

using namespace rm;
using namespace rmd;

namespace {

thread_local std::string g_batch_error;

struct BatchError : std::runtime_error {
  explicit BatchError(const std::string &s) : std::runtime_error(s) {}
};
#define BK(x)                                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) throw BatchError(std::string(#x) + ": " + cudaGetErrorString(e_));   \
  } while (0)

// Host-side setup products of one problem.
struct HostProb {
  int k = 0, p = 0, n[3] = {0, 0, 0};
  Layout L, L0;
  FreeMap fm, fm0;
  std::vector<double> al, be, hcell, D1;
  bool sc = false, ph = false;
  Condensed C;
  std::vector<PatchFamily> fam;   // main-space families
  std::vector<PatchFamily> pfam;  // potential-space families
  Csr D;                          // discrete gradient (lattice ids), PH only
  std::vector<int> G1, G0;        // interface lattice ids (main, potential)
  CoarseData cd;
  double bh_a = 0, bh_b = 0;
};

HostProb build_prob(int k, const rm_mesh &mesh, int p, const double *alpha, const double *beta,
                    const rm_options &o) {
  HostProb H;
  H.k = k;
  H.p = p;
  H.n[0] = mesh.nx;
  H.n[1] = mesh.ny;
  H.n[2] = mesh.nz;
  H.L = Layout(k, H.n, p);
  H.fm = FreeMap(H.L);
  const int ncell = H.n[0] * H.n[1] * H.n[2];
  Geometry geo;
  for (int d = 0; d < 3; ++d) geo.n[d] = H.n[d];
  const size_t nv = (size_t)(H.n[0] + 1) * (H.n[1] + 1) * (H.n[2] + 1);
  geo.X.resize(3 * nv);
  if (mesh.vertices) {
    std::memcpy(geo.X.data(), mesh.vertices, 3 * nv * sizeof(double));
  } else {
    for (int a3 = 0; a3 <= H.n[2]; ++a3)
      for (int a2 = 0; a2 <= H.n[1]; ++a2)
        for (int a1 = 0; a1 <= H.n[0]; ++a1) {
          size_t v = a1 + (size_t)(H.n[0] + 1) * (a2 + (size_t)(H.n[1] + 1) * a3);
          geo.X[3 * v + 0] = (double)a1 / H.n[0];
          geo.X[3 * v + 1] = (double)a2 / H.n[1];
          geo.X[3 * v + 2] = (double)a3 / H.n[2];
        }
  }
  H.al.assign(ncell, 1.0);
  H.be.assign(ncell, 1.0);
  if (alpha) std::memcpy(H.al.data(), alpha, ncell * sizeof(double));
  if (beta) std::memcpy(H.be.data(), beta, ncell * sizeof(double));
  for (int c = 0; c < ncell; ++c)
    if (!(H.al[c] > 0) || !(H.be[c] >= 0)) throw std::invalid_argument("alpha must be > 0 and beta >= 0");
  // Cartesian cells only (the batched apply is the Kronecker kernel)
  H.hcell.resize(3 * (size_t)ncell);
  for (int c = 0; c < ncell; ++c) {
    double X8[24];
    geo.cell_vertices(c % H.n[0], (c / H.n[0]) % H.n[1], c / (H.n[0] * H.n[1]), X8);
    double hh[3];
    for (int d = 0; d < 3; ++d) hh[d] = X8[3 * (1 << d) + d] - X8[d];
    const double tol = 1e-12 * std::max(hh[0], std::max(hh[1], hh[2]));
    for (int corner = 0; corner < 8; ++corner)
      for (int d = 0; d < 3; ++d)
        if (!(hh[d] > 0) || std::fabs(X8[3 * corner + d] - (X8[d] + ((corner >> d) & 1) * hh[d])) > tol)
          throw std::invalid_argument("the batched solver needs axis-aligned (Cartesian) cells");
    for (int d = 0; d < 3; ++d) H.hcell[3 * (size_t)c + d] = hh[d];
  }
  Basis1D B(p);
  H.D1 = B.D;
  H.bh_a = B.Bhat[0];
  H.bh_b = B.Bhat[p];
  H.sc = o.static_condensation != 0;
  H.ph = o.decomposition == RM_PH;
  const int fac = o.factor == RM_ICC ? 1 : 0;
  Csr P = assemble_aux(H.L, geo, H.be.data(), H.al.data(), H.fm);
  if (!H.sc) {
    H.fam.push_back(build_patches(H.L, H.fm, P, 0, false, fac));
  } else {
    H.C = condense(H.L, H.fm, P);
    P = Csr();
    if (!H.ph) {
      H.fam.push_back(build_patches(H.L, H.fm, H.C.S, 0, true, fac));
    } else {
      for (int m = 0; m < 3; ++m) H.fam.push_back(build_patches(H.L, H.fm, H.C.S, 1 << m, true, 0));
      H.L0 = Layout(0, H.n, p);
      H.fm0 = FreeMap(H.L0);
      std::vector<double> zero(ncell, 0.0);
      Csr Bm = assemble_aux(H.L0, geo, zero.data(), H.be.data(), H.fm0);
      Condensed C0 = condense(H.L0, H.fm0, Bm);
      H.pfam.push_back(build_patches(H.L0, H.fm0, C0.S, 0, true, fac));
      for (int f : H.C.G) H.G1.push_back(H.fm.free2lat[f]);
      for (int f : C0.G) H.G0.push_back(H.fm0.free2lat[f]);
      H.D = discrete_gradient(H.L0, H.L, H.G1, H.G0);
    }
    H.C.S = Csr();
  }
  if (o.coarse == RM_COARSE_P1) H.cd = build_coarse(H.L, geo, H.al.data(), H.be.data());
  else if (o.coarse != RM_COARSE_NONE)
    throw std::invalid_argument("the batched solver supports RM_COARSE_P1 or RM_COARSE_NONE");
  return H;
}

// Concatenation of CSR pieces with offset row / column ids.
struct CsrCat {
  std::vector<int> rid, ptr{0}, col, rprob;
  std::vector<double> val;
  int prob = 0;  // the problem whose rows append() adds
  // rows: row indices of A to append (empty rows kept); rmap/cmap: index maps
  // (nullptr = identity) applied before adding the offsets.
  void append(const Csr &A, const std::vector<int> *rows, const std::vector<int> *rmap,
              const std::vector<int> *cmap, long long roff, long long coff) {
    std::vector<int> all;
    if (!rows) {
      for (int i = 0; i < A.nrows; ++i)
        if (A.ptr[i + 1] != A.ptr[i]) all.push_back(i);
      rows = &all;
    }
    for (int i : *rows) {
      rid.push_back((int)((rmap ? (*rmap)[i] : i) + roff));
      rprob.push_back(prob);
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
        col.push_back((int)((cmap ? (*cmap)[A.col[e]] : A.col[e]) + coff));
        val.push_back(A.val[e]);
      }
      if (col.size() > (size_t)2147483647) throw std::runtime_error("batched CSR too large");
      ptr.push_back((int)col.size());
    }
  }
};

// Patch families with identical templates, concatenated.
struct FamCat {
  PatchFamily tmpl;
  std::vector<int> slotmap, pprob;
  std::vector<double> val;
  int npatch = 0;
};

bool same_template(const PatchFamily &a, const PatchFamily &b) {
  return a.nslots == b.nslots && a.inverse == b.inverse && a.rowptr == b.rowptr && a.col == b.col &&
         a.bptr == b.bptr && a.pos_slot == b.pos_slot;
}

}  // namespace

// problems of one (space, degree): the autotuner picks their assembly grid
struct ApplyGroup {
  int k = 0, p = 0;
  std::vector<int> probs;
};

struct rm_batch {
  std::string err;
  cudaStream_t stream = nullptr;
  // independent relaxation branches (merged patch families, the Hiptmair
  // potential branch, the coarse solve) fork onto these streams; inside the
  // captured iteration they become parallel graph branches
  static constexpr int kBranches = 8;
  cudaStream_t br[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {};
  rm_options opt{};
  int nprob = 0;
  int vt = 0;
  bool sc = false, ph = false;
  double setup_s = 0.0;  // wall time of rm_batch_setup
  std::vector<long long> off, off0, coff, size;
  long long N = 0, N0 = 0, NC = 0;
  std::vector<void *> allocs;
  std::vector<ApplyGroup> groups;
  std::vector<ApplyDev> capply;  // per problem: the Cartesian apply (cell products + assembly)
  uint8_t *mask = nullptr;
  DevCsr Binv, E, Et, Dt, DtT, R0, R0T;
  std::vector<DevPatch> fam, pfam;
  double *A0inv = nullptr;
  long long *aoff = nullptr;
  int *cstart = nullptr, *csz = nullptr, *rowprob = nullptr;
  double *x = nullptr, *b = nullptr, *r = nullptr, *z = nullptr, *pv = nullptr, *qv = nullptr;
  double *w = nullptr, *rt = nullptr, *u0 = nullptr, *v0 = nullptr, *cc = nullptr, *ce = nullptr;
  int4 *chunk = nullptr;
  int *cptr = nullptr;
  int nchunk = 0;
  double *partial = nullptr, *scal = nullptr;
  int *done = nullptr, *iters = nullptr;
  int *hdone = nullptr;  // pinned
  double *hscal = nullptr;
  cudaGraphExec_t graph = nullptr;
  long long graph_launches = 0;

  template <typename T>
  T *dalloc(size_t count) {
    void *ptr = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
    if (e != cudaSuccess) throw BatchError(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back(ptr);
    return (T *)ptr;
  }
  template <typename T>
  T *upload(const std::vector<T> &v) {
    T *d = dalloc<T>(v.size());
    if (!v.empty()) BK(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
  }
  void *upload_vals(const std::vector<double> &v, bool force_double = false) {
    if (vt == 0 || force_double) return upload(v);
    std::vector<float> f(v.begin(), v.end());
    return upload(f);
  }
  DevCsr upload_cat(const CsrCat &c, bool force_double = false) {
    DevCsr D;
    D.nrows = (int)c.rid.size();
    double avg = D.nrows ? (double)c.col.size() / D.nrows : 1.0;
    D.tpr = spmv_tpr(avg);
    D.rid = upload(c.rid);
    D.ptr = upload(c.ptr);
    D.col = upload(c.col);
    D.val = upload_vals(c.val, force_double);
    D.vt = force_double ? 0 : vt;
    D.rprob = upload(c.rprob);
    return D;
  }
  DevPatch upload_fam(const FamCat &f) {
    const PatchFamily &F = f.tmpl;
    DevPatch D;
    D.nslots = F.nslots;
    D.npatch = f.npatch;
    D.nnz = F.nnz();
    D.nflev = std::max(0, (int)F.flev.size() - 1);
    D.nblev = std::max(0, (int)F.blev.size() - 1);
    D.slotmap = upload(f.slotmap);
    D.rowptr = upload(F.rowptr);
    D.col = upload(F.col);
    D.tptr = upload(F.tptr);
    D.trow = upload(F.trow);
    D.tpos = upload(F.tpos);
    D.flev = upload(F.flev);
    D.frows = upload(F.frows);
    D.blev = upload(F.blev);
    D.brows = upload(F.brows);
    D.vt = vt;
    D.val = upload_vals(f.val);
    D.pprob = upload(f.pprob);
    if (F.inverse) {
      D.inverse = 1;
      D.ivals = F.ivals();
      D.pos_slot = upload(F.pos_slot);
      D.pos_blk = upload(F.pos_blk);
      D.bptr = upload(F.bptr);
      D.boff = upload(F.boff);
    }
    return D;
  }
  ~rm_batch() {
    if (graph) cudaGraphExecDestroy(graph);
    for (void *a : allocs) cudaFree(a);
    if (hdone) cudaFreeHost(hdone);
    if (hscal) cudaFreeHost(hscal);
    if (stream) cudaStreamDestroy(stream);
    for (int i = 0; i < kBranches; ++i) {
      if (br[i]) cudaStreamDestroy(br[i]);
      if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
  }
};

namespace {

int bfail(rm_batch *b, int code, const std::string &msg) {
  if (b) b->err = msg;
  g_batch_error = msg;
  return code;
}

// y = A x for every problem: the per-handle Cartesian kernel pair on each
// problem's slice of the concatenated vectors (every entry written; a
// converged problem's cells are skipped and its entries set to 0)
void batch_apply(rm_batch *B, const double *x, double *y) {
  for (const ApplyDev &A : B->capply) BK(launch_apply_cart(A, x, y, B->stream));
}

// z = B r for every problem: the condensation on the batch stream, then the
// additive interface terms (merged patch families, the Hiptmair potential
// branch) and the coarse solve concurrently on the branch streams (atomic
// adds into z), joined before the interior expansion; the coarse
// prolongation is added last.
void batch_precondition(rm_batch *B, const double *r, double *z) {
  cudaStream_t s = B->stream;
  BK(cudaMemsetAsync(z, 0, B->N * sizeof(double), s));
  const double *rr = r;
  if (B->sc) {
    BK(launch_spmv(B->Binv, r, B->w, nullptr, 0, 1.0, s));
    BK(launch_spmv(B->E, r, B->rt, r, 2, -1.0, s));
    rr = B->rt;
  }
  BK(cudaEventRecord(B->fork, s));
  int nb = 0;
  auto branch = [&]() {
    cudaStream_t b = B->br[nb % rm_batch::kBranches];
    if (nb < rm_batch::kBranches) BK(cudaStreamWaitEvent(b, B->fork, 0));
    ++nb;
    return b;
  };
  for (auto &F : B->fam) BK(launch_patches(F, rr, z, branch()));
  if (B->ph) {
    cudaStream_t b = branch();
    BK(launch_spmv(B->DtT, rr, B->u0, nullptr, 0, 1.0, b));
    BK(cudaMemsetAsync(B->v0, 0, B->N0 * sizeof(double), b));
    for (auto &F : B->pfam) BK(launch_patches(F, B->u0, B->v0, b));
    BK(launch_spmv(B->Dt, B->v0, z, nullptr, 3, 1.0, b));
  }
  if (B->NC > 0) {
    cudaStream_t b = branch();
    BK(launch_spmv(B->R0, r, B->cc, nullptr, 0, 1.0, b));
    BK(launch_gemv_batch((int)B->NC, B->rowprob, B->aoff, B->cstart, B->csz, B->A0inv, B->cc, B->ce, b));
  }
  for (int i = 0; i < std::min(nb, (int)rm_batch::kBranches); ++i) {
    BK(cudaEventRecord(B->join[i], B->br[i]));
    BK(cudaStreamWaitEvent(s, B->join[i], 0));
  }
  if (B->sc) BK(launch_spmv(B->Et, z, z, B->w, 2, -1.0, s));
  if (B->NC > 0) BK(launch_spmv(B->R0T, B->ce, z, nullptr, 1, 1.0, s));
}

// One lock-step iteration (captured in the graph).
void batch_iteration(rm_batch *B, double tol2) {
  cudaStream_t s = B->stream;
  batch_apply(B, B->pv, B->qv);
  BK(launch_seg_dot(B->chunk, B->nchunk, B->cptr, B->nprob, B->pv, B->qv, B->partial, B->scal, B->done,
                    B->iters, S_PQ, 1, tol2, s));
  BK(launch_seg_update_xr(B->chunk, B->nchunk, B->cptr, B->nprob, B->x, B->r, B->pv, B->qv, B->partial,
                          B->scal, B->done, B->iters, tol2, s));
  batch_precondition(B, B->r, B->z);
  BK(launch_seg_dot2(B->chunk, B->nchunk, B->cptr, B->nprob, B->r, B->z, B->qv, B->partial, B->scal,
                     B->done, B->iters, B->opt.flexible, s));
  BK(launch_seg_update_p(B->chunk, B->nchunk, B->pv, B->z, B->scal, s));
}

}  // namespace

extern "C" {

int rm_batch_setup(rm_batch **out, int nprob, const int *space, const rm_mesh *meshes, const int *p,
                   const double *const *alpha, const double *const *beta, const rm_options *opt,
                   void *stream) {
  (void)stream;
  if (!out || nprob < 1 || !space || !meshes || !p)
    return bfail(nullptr, RM_ERR_ARG, "rm_batch_setup: invalid argument");
  if (nprob > 4096) return bfail(nullptr, RM_ERR_ARG, "rm_batch_setup: at most 4096 problems");
  *out = nullptr;
  std::unique_ptr<rm_batch> B(new rm_batch());
  const auto t_setup = std::chrono::steady_clock::now();
  try {
    B->opt = opt ? *opt : rm_default_options();
    const rm_options &o = B->opt;
    if (o.precision != RM_FP64 && o.precision != RM_FP32) throw std::invalid_argument("precision");
    if (o.norm != RM_NORM_L2) throw std::invalid_argument("norm: the batched lock step stops on the l2 residual");
    if (o.arith != RM_ARITH_FP64 && o.arith != RM_ARITH_DF64) throw std::invalid_argument("arith");
    if (o.boundary != RM_BC_DIRICHLET) throw std::invalid_argument("boundary: only RM_BC_DIRICHLET");
    if (o.deterministic != 0)
      throw std::invalid_argument("deterministic: single-problem handles only (the batch scatters patches with atomics)");
    B->vt = o.precision == RM_FP32 ? 1 : 0;
    B->nprob = nprob;
    B->sc = o.static_condensation != 0;
    B->ph = o.decomposition == RM_PH;
    for (int i = 0; i < nprob; ++i) {
      if (space[i] < 0 || space[i] > 2 || p[i] < 1 || p[i] > 15 || meshes[i].nx < 2 || meshes[i].ny < 2 ||
          meshes[i].nz < 2)
        throw std::invalid_argument("problem " + std::to_string(i) + ": bad space, degree or mesh");
      if (B->ph && space[i] != RM_HCURL) throw std::invalid_argument("RM_PH needs H(curl) problems");
    }
    if (B->ph && !B->sc) throw std::invalid_argument("RM_PH needs static_condensation = 1");
    BK(cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking));
    BK(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
    for (int i = 0; i < rm_batch::kBranches; ++i) {
      BK(cudaStreamCreateWithFlags(&B->br[i], cudaStreamNonBlocking));
      BK(cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming));
    }
    // ---- host setup of every problem, offsets ----
    std::vector<HostProb> H;
    H.reserve(nprob);
    B->off.assign(nprob + 1, 0);
    B->off0.assign(nprob + 1, 0);
    B->coff.assign(nprob + 1, 0);
    for (int i = 0; i < nprob; ++i) {
      H.push_back(build_prob(space[i], meshes[i], p[i], alpha ? alpha[i] : nullptr, beta ? beta[i] : nullptr, o));
      B->off[i + 1] = B->off[i] + H[i].L.size;
      B->off0[i + 1] = B->off0[i] + (B->ph ? H[i].L0.size : 0);
      B->coff[i + 1] = B->coff[i] + H[i].cd.nc;
      B->size.push_back(H[i].L.size);
    }
    B->N = B->off[nprob];
    B->N0 = B->off0[nprob];
    B->NC = B->coff[nprob];
    if (B->N > 2147483647LL || B->N0 > 2147483647LL) throw std::invalid_argument("batch too large for int32 indices");
    // ---- mask ----
    {
      std::vector<uint8_t> mask(B->N, 1);
      for (int i = 0; i < nprob; ++i)
        for (int l : H[i].fm.free2lat) mask[B->off[i] + l] = 0;
      B->mask = B->upload(mask);
    }
    // ---- the Cartesian apply of every problem, grouped by (space, p) ----
    {
      std::map<std::pair<int, int>, std::vector<int>> byp;
      for (int i = 0; i < nprob; ++i) byp[{H[i].k, H[i].p}].push_back(i);
      for (auto &kv : byp) {
        ApplyGroup g;
        g.k = kv.first.first;
        g.p = kv.first.second;
        g.probs = kv.second;
        B->groups.push_back(g);
      }
      B->capply.resize(nprob);
      for (int i = 0; i < nprob; ++i) {
        const HostProb &P = H[i];
        ApplyDev A{};
        Layout L1(P.k + 1, P.n, P.p);
        A.k = P.k;
        A.p = P.p;
        A.q = quad_points(P.p);
        A.prob = i;
        A.arith = o.arith == RM_ARITH_DF64 ? 1 : 0;
        for (int d = 0; d < 3; ++d) A.n[d] = P.n[d];
        A.nc0 = P.L.ncomp;
        A.nc1 = L1.ncomp;
        for (int m = 0; m < 3; ++m)
          for (int d = 0; d < 3; ++d) A.N[m][d] = (int)P.L.N[m][d];
        for (int m = 0; m < 3; ++m) A.off[m] = P.L.off[m] + B->off[i];
        A.nloc0 = P.L.nloc;
        A.nloc1 = L1.nloc;
        // the Cartesian kernel reads D-hat at offset q(p+1) + qp of tabs
        std::vector<double> tabs((size_t)A.q * (P.p + 1) + (size_t)A.q * P.p, 0.0);
        tabs.insert(tabs.end(), P.D1.begin(), P.D1.end());
        A.tabs = B->upload(tabs);
        A.cartesian = 1;
        A.bh_a = P.bh_a;
        A.bh_b = P.bh_b;
        const int ncell = P.n[0] * P.n[1] * P.n[2];
        // per cell: beta x the box metric of each V^k component, alpha x that
        // of each V^{k+1} component (J = diag(h/2); the pullbacks of Sec. 3.1)
        std::vector<double> cc((size_t)ncell * 8, 0.0);
        auto box_metric = [](int kk, int m, const double *hh) {
          const double det = 0.125 * hh[0] * hh[1] * hh[2];
          if (kk == 0) return det;
          if (kk == 3) return 1.0 / det;
          if (kk == 1) return det * 4.0 / (hh[m] * hh[m]);
          return 0.25 * hh[m] * hh[m] / det;
        };
        const int nc0 = P.k == 0 ? 1 : 3, nc1 = P.k == 2 ? 1 : 3;
        for (int c = 0; c < ncell; ++c) {
          const double *hh = &P.hcell[3 * (size_t)c];
          for (int m = 0; m < nc0; ++m) cc[(size_t)c * 8 + m] = P.be[c] * box_metric(P.k, m, hh);
          for (int t = 0; t < nc1; ++t) cc[(size_t)c * 8 + 3 + t] = P.al[c] * box_metric(P.k + 1, t, hh);
        }
        A.ccoef = B->upload(cc);
        if (cart_local_smem_doubles(A.k, A.p, A.nloc0, A.nloc1) * sizeof(double) > 227 * 1024)
          throw std::invalid_argument("degree too high for the Cartesian apply kernel");
        A.Y = B->dalloc<double>((size_t)ncell * A.nloc0);  // unassembled cell products
        B->capply[i] = A;
      }
    }
    // ---- static condensation, Hiptmair gradient, coarse (concatenated) ----
    if (B->sc) {
      CsrCat cb, ce, cet, cd, cdt;
      for (int i = 0; i < nprob; ++i) {
        const HostProb &P = H[i];
        cb.prob = i;
        cb.append(P.C.Binv, &P.C.I, &P.fm.free2lat, &P.fm.free2lat, B->off[i], B->off[i]);
        ce.prob = i;
        ce.append(P.C.E, &P.C.G, &P.fm.free2lat, &P.fm.free2lat, B->off[i], B->off[i]);
        cet.prob = i;
        cet.append(P.C.Et, &P.C.I, &P.fm.free2lat, &P.fm.free2lat, B->off[i], B->off[i]);
        if (B->ph) {
          cd.prob = i;
          cd.append(P.D, &P.G1, nullptr, nullptr, B->off[i], B->off0[i]);
          cdt.prob = i;
          cdt.append(transpose(P.D), &P.G0, nullptr, nullptr, B->off0[i], B->off[i]);
        }
      }
      // the interior solve and harmonic extension in FP64 whatever the
      // precision (as in rm_setup)
      B->Binv = B->upload_cat(cb, true);
      B->E = B->upload_cat(ce, true);
      B->Et = B->upload_cat(cet, true);
      if (B->ph) {
        B->Dt = B->upload_cat(cd);
        B->DtT = B->upload_cat(cdt);
        B->u0 = B->dalloc<double>(B->N0);
        B->v0 = B->dalloc<double>(B->N0);
      }
      B->w = B->dalloc<double>(B->N);
      B->rt = B->dalloc<double>(B->N);
    }
    if (B->NC > 0) {
      CsrCat cr, crt;
      std::vector<double> A0;
      std::vector<long long> aoff;
      std::vector<int> cstart, csz, rowprob;
      for (int i = 0; i < nprob; ++i) {
        const CoarseData &c = H[i].cd;
        std::vector<int> rows(c.nc);
        for (int j = 0; j < c.nc; ++j) rows[j] = j;
        cr.prob = i;
        cr.append(c.R0, &rows, nullptr, nullptr, B->coff[i], B->off[i]);
        crt.prob = i;
        crt.append(c.R0T, nullptr, nullptr, nullptr, B->off[i], B->coff[i]);
        aoff.push_back((long long)A0.size());
        A0.insert(A0.end(), c.A0inv.begin(), c.A0inv.end());
        cstart.push_back((int)B->coff[i]);
        csz.push_back(c.nc);
        for (int j = 0; j < c.nc; ++j) rowprob.push_back(i);
      }
      B->R0 = B->upload_cat(cr, true);
      B->R0T = B->upload_cat(crt, true);
      B->A0inv = B->upload(A0);
      B->aoff = B->upload(aoff);
      B->cstart = B->upload(cstart);
      B->csz = B->upload(csz);
      B->rowprob = B->upload(rowprob);
      B->cc = B->dalloc<double>(B->NC);
      B->ce = B->dalloc<double>(B->NC);
    }
    // ---- patch families: identical templates merged ----
    auto merge = [&](bool potential) {
      std::vector<FamCat> cats;
      for (int i = 0; i < nprob; ++i) {
        const auto &fams = potential ? H[i].pfam : H[i].fam;
        const long long voff = potential ? B->off0[i] : B->off[i];
        for (const PatchFamily &F : fams) {
          FamCat *dst = nullptr;
          for (auto &c : cats)
            if (same_template(c.tmpl, F)) dst = &c;
          if (!dst) {
            cats.emplace_back();
            dst = &cats.back();
            dst->tmpl = F;
            dst->tmpl.slotmap.clear();
            dst->tmpl.val.clear();
            dst->tmpl.ival.clear();
          }
          for (int s : F.slotmap) dst->slotmap.push_back(s >= 0 ? (int)(s + voff) : -1);
          const std::vector<double> v = F.device_values();
          dst->val.insert(dst->val.end(), v.begin(), v.end());
          dst->npatch += F.npatch;
          dst->pprob.insert(dst->pprob.end(), F.npatch, i);
        }
      }
      std::vector<DevPatch> out;
      for (auto &c : cats) out.push_back(B->upload_fam(c));
      return out;
    };
    B->fam = merge(false);
    if (B->ph) B->pfam = merge(true);
    H.clear();
    // ---- vectors, CG state, chunks ----
    B->x = B->dalloc<double>(B->N);
    B->b = B->dalloc<double>(B->N);
    B->r = B->dalloc<double>(B->N);
    B->z = B->dalloc<double>(B->N);
    B->pv = B->dalloc<double>(B->N);
    B->qv = B->dalloc<double>(B->N);
    {
      const long long CH = 65536;
      std::vector<int4> chunk;
      std::vector<int> cptr{0};
      for (int i = 0; i < nprob; ++i) {
        for (long long s0 = B->off[i]; s0 < B->off[i + 1]; s0 += CH)
          chunk.push_back(make_int4(i, (int)s0, (int)std::min(s0 + CH, B->off[i + 1]), 0));
        cptr.push_back((int)chunk.size());
      }
      B->nchunk = (int)chunk.size();
      B->chunk = B->upload(chunk);
      B->cptr = B->upload(cptr);
    }
    B->partial = B->dalloc<double>(2 * (size_t)B->nchunk);
    B->scal = B->dalloc<double>((size_t)nprob * S_COUNT);
    B->done = B->dalloc<int>(nprob);
    BK(cudaMemset(B->done, 0, nprob * sizeof(int)));
    // rows and patches of converged problems are skipped by the kernels
    for (DevCsr *M : {&B->Binv, &B->E, &B->Et, &B->Dt, &B->DtT, &B->R0, &B->R0T}) M->done = B->done;
    for (auto &F : B->fam) F.done = B->done;
    for (auto &F : B->pfam) F.done = B->done;
    for (auto &A : B->capply) A.done = B->done;
    B->iters = B->dalloc<int>(nprob);
    BK(cudaMallocHost((void **)&B->hdone, nprob * sizeof(int)));
    BK(cudaMallocHost((void **)&B->hscal, (size_t)nprob * S_COUNT * sizeof(double)));
    // ---- autotuner: grid of the Cartesian assembly per (space, p) group ----
    // (the cell-product kernel's shape per degree is fixed at compile time
    // by its lane-use rule; the assembly grid is timed here: 2 to 16 CTAs
    // per SM, the fastest kept for every problem of the group)
    BK(cudaMemsetAsync(B->pv, 0, B->N * sizeof(double), B->stream));
    BK(cudaMemsetAsync(B->done, 0, nprob * sizeof(int), B->stream));
    {
      cudaEvent_t e0, e1;
      BK(cudaEventCreate(&e0));
      BK(cudaEventCreate(&e1));
      int dev = 0, nsm = 152;
      BK(cudaGetDevice(&dev));
      BK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      for (auto &g : B->groups) {
        float best = 1e30f;
        int bestg = 8 * nsm;
        for (int per : {2, 4, 8, 16}) {
          for (int i : g.probs) B->capply[i].asm_grid = per * nsm;
          for (int i : g.probs) BK(launch_apply_cart(B->capply[i], B->pv, B->qv, B->stream));
          BK(cudaEventRecord(e0, B->stream));
          for (int rep = 0; rep < 3; ++rep)
            for (int i : g.probs) BK(launch_apply_cart(B->capply[i], B->pv, B->qv, B->stream));
          BK(cudaEventRecord(e1, B->stream));
          BK(cudaEventSynchronize(e1));
          float ms = 0.f;
          BK(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) {
            best = ms;
            bestg = per * nsm;
          }
        }
        for (int i : g.probs) B->capply[i].asm_grid = bestg;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    // ---- capture one lock-step iteration in a CUDA graph ----
    batch_iteration(B.get(), 0.0);  // warm-up: sets kernel attributes before capture
    BK(cudaStreamSynchronize(B->stream));
    const long long l0 = launch_count();
    cudaGraph_t graph;
    BK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeRelaxed));
    batch_iteration(B.get(), o.rtol * o.rtol);
    BK(cudaStreamEndCapture(B->stream, &graph));
    B->graph_launches = launch_count() - l0;
    BK(cudaGraphInstantiate(&B->graph, graph, 0));
    cudaGraphDestroy(graph);
    BK(cudaStreamSynchronize(B->stream));
  } catch (const BatchError &e) {
    return bfail(nullptr, RM_ERR_CUDA, std::string("rm_batch_setup: ") + e.what());
  } catch (const std::invalid_argument &e) {
    return bfail(nullptr, RM_ERR_ARG, std::string("rm_batch_setup: ") + e.what());
  } catch (const std::bad_alloc &) {
    return bfail(nullptr, RM_ERR_OOM, "rm_batch_setup: host allocation failed");
  } catch (const std::exception &e) {
    std::string w = e.what();
    return bfail(nullptr, w.find("breakdown") != std::string::npos ? RM_ERR_BREAKDOWN : RM_ERR_ARG,
                 std::string("rm_batch_setup: ") + w);
  }
  B->setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_setup).count();
  *out = B.release();
  return RM_OK;
}

int rm_batch_ndofs(const rm_batch *b, int i, long long *lattice) {
  if (!b || i < 0 || i >= b->nprob || !lattice) return bfail(nullptr, RM_ERR_ARG, "rm_batch_ndofs: bad argument");
  *lattice = b->size[i];
  return RM_OK;
}

int rm_batch_solve(rm_batch *B, const double *const *bvec, double *const *xvec, rm_info *infos,
                   void *stream) {
  if (!B || !bvec || !xvec) return bfail(B, RM_ERR_ARG, "rm_batch_solve: NULL argument");
  cudaStream_t s = B->stream;
  int status = RM_OK;
  float ms = 0.f;
  int rounds = 0;
  try {
    BK(cudaStreamSynchronize((cudaStream_t)stream));
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    BK(cudaEventRecord(e0, s));
    const long long l0 = launch_count();
    for (int i = 0; i < B->nprob; ++i) {
      BK(cudaMemcpyAsync(B->b + B->off[i], bvec[i], B->size[i] * sizeof(double), cudaMemcpyDeviceToDevice, s));
      BK(cudaMemcpyAsync(B->x + B->off[i], xvec[i], B->size[i] * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    const double tol2 = B->opt.rtol * B->opt.rtol;
    BK(launch_mask_copy(B->N, B->mask, B->x, B->x, s));
    batch_apply(B, B->x, B->qv);
    BK(launch_sub(B->N, B->mask, B->b, B->qv, B->r, s));
    BK(launch_mask_copy(B->N, B->mask, B->b, B->z, s));
    BK(cudaMemsetAsync(B->done, 0, B->nprob * sizeof(int), s));
    BK(cudaMemsetAsync(B->iters, 0, B->nprob * sizeof(int), s));
    BK(launch_seg_dot(B->chunk, B->nchunk, B->cptr, B->nprob, B->z, B->z, B->partial, B->scal, B->done,
                      B->iters, S_BB, 0, tol2, s));
    BK(launch_seg_dot(B->chunk, B->nchunk, B->cptr, B->nprob, B->r, B->r, B->partial, B->scal, B->done,
                      B->iters, S_RR, 0, tol2, s));
    BK(cudaMemcpyAsync(B->hscal, B->scal, (size_t)B->nprob * S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    BK(cudaStreamSynchronize(s));
    int ndone = 0;
    for (int i = 0; i < B->nprob; ++i) {
      const double *sc = B->hscal + i * S_COUNT;
      B->hdone[i] = !std::isfinite(sc[S_RR]) ? 2 : (sc[S_RR] <= tol2 * sc[S_BB]) ? 1 : 0;
      ndone += B->hdone[i] != 0;
    }
    BK(cudaMemcpyAsync(B->done, B->hdone, B->nprob * sizeof(int), cudaMemcpyHostToDevice, s));
    batch_precondition(B, B->r, B->z);
    BK(launch_seg_dot(B->chunk, B->nchunk, B->cptr, B->nprob, B->r, B->z, B->partial, B->scal, B->done,
                      B->iters, S_RZ, 0, tol2, s));
    BK(cudaMemcpyAsync(B->pv, B->z, B->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int it = 0;
    const int every = std::max(1, B->opt.check_every);
    while (ndone < B->nprob && it < B->opt.max_it) {
      const int m = std::min(every, B->opt.max_it - it);
      for (int j = 0; j < m; ++j) BK(cudaGraphLaunch(B->graph, s));
      it += m;
      ++rounds;
      BK(cudaMemcpyAsync(B->hdone, B->done, B->nprob * sizeof(int), cudaMemcpyDeviceToHost, s));
      BK(cudaStreamSynchronize(s));
      ndone = 0;
      for (int i = 0; i < B->nprob; ++i) ndone += B->hdone[i] != 0;
    }
    for (int i = 0; i < B->nprob; ++i)
      BK(cudaMemcpyAsync(xvec[i], B->x + B->off[i], B->size[i] * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BK(cudaEventRecord(e1, s));
    BK(cudaEventSynchronize(e1));
    BK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const long long launches = launch_count() - l0 + (long long)it * B->graph_launches;
    std::vector<int> hit(B->nprob);
    BK(cudaMemcpy(hit.data(), B->iters, B->nprob * sizeof(int), cudaMemcpyDeviceToHost));
    BK(cudaMemcpy(B->hscal, B->scal, (size_t)B->nprob * S_COUNT * sizeof(double), cudaMemcpyDeviceToHost));
    for (int i = 0; i < B->nprob; ++i) {
      const double *sc = B->hscal + i * S_COUNT;
      const double rel = sc[S_BB] > 0 ? std::sqrt(sc[S_RR] / sc[S_BB]) : 0.0;
      // the problem's flag: 1 converged, 2 NaN/Inf residual, 3 CG breakdown
      const int st = B->hdone[i] == 1   ? RM_OK
                     : B->hdone[i] == 2 ? RM_ERR_NAN
                     : B->hdone[i] == 3 ? RM_ERR_BREAKDOWN
                                        : (std::isfinite(rel) ? RM_ERR_NOT_CONVERGED : RM_ERR_NAN);
      if (st != RM_OK) status = st;
      if (infos) {
        infos[i].iterations = hit[i];
        infos[i].status = st;
        infos[i].rel_res_l2 = rel;
        infos[i].rel_res_natural = -1.0;  // the lock step stops on the l2 residual only
        infos[i].iterations_natural = -1;
        infos[i].history_len = 0;
        infos[i].setup_s = B->setup_s;
        infos[i].solve_ms = ms;
        infos[i].apply_ms = 0.0;
        infos[i].apply_calls = 0;
        infos[i].precond_ms = 0.0;
        infos[i].precond_calls = rounds;
        infos[i].kernel_launches = launches;
        infos[i].learned_calls = 0;
        infos[i].judge_calls = 0;
        infos[i].fallback_at = -1;
        infos[i].judge_eta = -1.0;
      }
    }
  } catch (const std::exception &e) {
    return bfail(B, RM_ERR_CUDA, e.what());
  }
  if (status != RM_OK) bfail(B, status, "rm_batch_solve: not every problem converged (see infos[i].status)");
  return status;
}

void rm_batch_destroy(rm_batch *b) { delete b; }

const char *rm_batch_last_error(const rm_batch *b) {
  if (b) return b->err.c_str();
  return g_batch_error.c_str();
}

}  // extern "C"
