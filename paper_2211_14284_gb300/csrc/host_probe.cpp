// Host-only inspection entry points for the FP64 setup (no CUDA): the test
// suite compares these intermediate objects with the CPU oracle without a
// GPU.  Not part of the solver ABI in include/rm.h.
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "host_basis.h"
#include "host_setup.h"

using namespace rm;

namespace {
struct Probe {
  Layout L, L0;
  FreeMap fm, fm0;
  Csr P, S, E, Binv, S0, R0, Dt;
  std::vector<PatchFamily> fams;
  CoarseData coarse;
  std::string err;
};
std::unique_ptr<Probe> g;
std::string g_err;

const Csr *pick(int which) {
  switch (which) {
    case 0: return &g->P;
    case 1: return &g->S;
    case 2: return &g->E;
    case 3: return &g->Binv;
    case 4: return &g->coarse.R0;
    case 5: return &g->S0;
    case 6: return &g->Dt;
    default: return nullptr;
  }
}
}  // namespace

extern "C" {

const char *rmh_error() { return g_err.c_str(); }

int rmh_basis(int p, double *S, double *lam, double *Bhat, double *Ahat, double *D, double *Js) {
  try {
    Basis1D B(p);
    std::memcpy(S, B.S.data(), B.S.size() * sizeof(double));
    std::memcpy(lam, B.lam.data(), B.lam.size() * sizeof(double));
    std::memcpy(Bhat, B.Bhat.data(), B.Bhat.size() * sizeof(double));
    std::memcpy(Ahat, B.Ahat.data(), B.Ahat.size() * sizeof(double));
    std::memcpy(D, B.D.data(), B.D.size() * sizeof(double));
    std::memcpy(Js, B.Js.data(), B.Js.size() * sizeof(double));
  } catch (const std::exception &e) {
    g_err = e.what();
    return 1;
  }
  return 0;
}

int rmh_gll(int q, double *x, double *w) {
  std::vector<double> xx, ww;
  gll_rule(q, xx, ww);
  std::memcpy(x, xx.data(), q * sizeof(double));
  std::memcpy(w, ww.data(), q * sizeof(double));
  return 0;
}

// Builds P, the Schur complement and the patch families as rm_setup would.
// mode & 15: 0 non-condensed PAFW, 1 SC-PAFW, 2 SC-PH (k = 1, 2); mode & 16:
// Gamma_D empty (natural boundary conditions).
int rmh_build(int k, const int n[3], int p, const double *X, const double *alpha,
              const double *beta, int mode, int factor, int coarse) {
  try {
    g.reset(new Probe());
    const bool natural = (mode & 16) != 0;
    mode &= 15;
    g->L = Layout(k, n, p, natural);
    g->fm = FreeMap(g->L);
    Geometry geo;
    for (int d = 0; d < 3; ++d) geo.n[d] = n[d];
    size_t nv = (size_t)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
    geo.X.assign(X, X + 3 * nv);
    const int ncell = n[0] * n[1] * n[2];
    g->P = assemble_aux(g->L, geo, beta, alpha, g->fm);
    if (mode == 0) {
      g->fams.push_back(build_patches(g->L, g->fm, g->P, 0, false, factor));
    } else {
      Condensed C = condense(g->L, g->fm, g->P);
      g->S = C.S;
      g->E = C.E;
      g->Binv = C.Binv;
      if (mode == 1) {
        g->fams.push_back(build_patches(g->L, g->fm, C.S, 0, true, factor));
      } else {
        for (int m = 0; m < 3; ++m)
          g->fams.push_back(build_patches(g->L, g->fm, C.S, k == 1 ? (1 << m) : (7 & ~(1 << m)), true, 0));
        g->L0 = Layout(k - 1, n, p, natural);
        g->fm0 = FreeMap(g->L0);
        std::vector<double> pmass(ncell, 0.0);
        if (k == 2)
          for (int c = 0; c < ncell; ++c) pmass[c] = kHdivPotentialEps * beta[c];
        Csr B = assemble_aux(g->L0, geo, pmass.data(), beta, g->fm0);
        Condensed C0 = condense(g->L0, g->fm0, B);
        g->S0 = C0.S;
        if (k == 1)
          g->fams.push_back(build_patches(g->L0, g->fm0, C0.S, 0, true, factor));
        else
          for (int m = 0; m < 3; ++m) g->fams.push_back(build_patches(g->L0, g->fm0, C0.S, 1 << m, true, factor));
        std::vector<int> G1, G0;
        for (int f : C.G) G1.push_back(g->fm.free2lat[f]);
        for (int f : C0.G) G0.push_back(g->fm0.free2lat[f]);
        g->Dt = discrete_derivative(g->L0, g->L, G1, G0);
      }
    }
    if (coarse) g->coarse = build_coarse(g->L, geo, alpha, beta);
  } catch (const std::exception &e) {
    g_err = e.what();
    return 1;
  }
  return 0;
}

int rmh_csr_size(int which, int *nrows, long long *nnz) {
  const Csr *A = g ? pick(which) : nullptr;
  if (!A) return 1;
  *nrows = A->nrows;
  *nnz = A->nnz();
  return 0;
}

int rmh_csr_get(int which, long long *ptr, int *col, double *val) {
  const Csr *A = g ? pick(which) : nullptr;
  if (!A) return 1;
  for (int i = 0; i <= A->nrows; ++i) ptr[i] = A->ptr.empty() ? 0 : A->ptr[i];
  std::memcpy(col, A->col.data(), A->col.size() * sizeof(int));
  std::memcpy(val, A->val.data(), A->val.size() * sizeof(double));
  return 0;
}

int rmh_nfamilies() { return g ? (int)g->fams.size() : 0; }

int rmh_family_size(int f, int *nslots, int *npatch, int *nnz) {
  if (!g || f < 0 || f >= (int)g->fams.size()) return 1;
  *nslots = g->fams[f].nslots;
  *npatch = g->fams[f].npatch;
  *nnz = g->fams[f].nnz();
  return 0;
}

int rmh_family_get(int f, int *slotmap, int *rowptr, int *col, double *val) {
  if (!g || f < 0 || f >= (int)g->fams.size()) return 1;
  const PatchFamily &F = g->fams[f];
  std::memcpy(slotmap, F.slotmap.data(), F.slotmap.size() * sizeof(int));
  std::memcpy(rowptr, F.rowptr.data(), F.rowptr.size() * sizeof(int));
  std::memcpy(col, F.col.data(), F.col.size() * sizeof(int));
  std::memcpy(val, F.val.data(), F.val.size() * sizeof(double));
  return 0;
}

// Block-inverse form of a family: is_inverse, number of blocks, values per patch.
int rmh_family_inverse_size(int f, int *is_inverse, int *nblocks, int *nvals) {
  if (!g || f < 0 || f >= (int)g->fams.size()) return 1;
  const PatchFamily &F = g->fams[f];
  *is_inverse = F.inverse;
  *nblocks = F.inverse ? (int)F.bptr.size() - 1 : 0;
  *nvals = F.ivals();
  return 0;
}

int rmh_family_inverse_get(int f, int *bptr, int *pos_slot, int *boff, double *ival) {
  if (!g || f < 0 || f >= (int)g->fams.size()) return 1;
  const PatchFamily &F = g->fams[f];
  std::memcpy(bptr, F.bptr.data(), F.bptr.size() * sizeof(int));
  std::memcpy(pos_slot, F.pos_slot.data(), F.pos_slot.size() * sizeof(int));
  std::memcpy(boff, F.boff.data(), F.boff.size() * sizeof(int));
  std::memcpy(ival, F.ival.data(), F.ival.size() * sizeof(double));
  return 0;
}

int rmh_coarse_size() { return g ? g->coarse.nc : 0; }

int rmh_coarse_inverse(double *A0inv) {
  if (!g) return 1;
  std::memcpy(A0inv, g->coarse.A0inv.data(), g->coarse.A0inv.size() * sizeof(double));
  return 0;
}

}  // extern "C"
