// Host FP64 setup: lattice layout (Sec. 2.4), the sparse auxiliary operator
// P (Sec. 3.2), static condensation (Eqs. LDU, schur), star patches with
// exact / incomplete Cholesky factors on a slot template shared by all
// patches of one entity kind (Sec. 4.1, 4.3, 4.5), and the p = 1 coarse
// space (Sec. 4.3, Eq. asm-afw).
#include "host_setup.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <stdexcept>
#include <unordered_map>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace rm {

static const char *kTypes[4][3] = {
    {"sss", nullptr, nullptr}, {"rss", "srs", "ssr"}, {"srr", "rsr", "rrs"}, {"rrr", nullptr, nullptr}};

// d^k as (source component, direction, sign) terms per target component.
struct DTerm {
  int src, dir, sgn;
};
static const int kNumTerms[3][3] = {{1, 1, 1}, {2, 2, 2}, {3, 0, 0}};
static const DTerm kTerms[3][3][3] = {
    {{{0, 0, 1}}, {{0, 1, 1}}, {{0, 2, 1}}},
    {{{2, 1, 1}, {1, 2, -1}}, {{0, 2, 1}, {2, 0, -1}}, {{1, 0, 1}, {0, 1, -1}}},
    {{{0, 0, 1}, {1, 1, 1}, {2, 2, 1}}, {}, {}}};

Layout::Layout(int k_, const int n_[3], int p_, bool natural_) : k(k_), p(p_), natural(natural_) {
  if (k < 0 || k > 3) throw std::runtime_error("Layout: k in 0..3");
  for (int d = 0; d < 3; ++d) n[d] = n_[d];
  ncomp = (k == 0 || k == 3) ? 1 : 3;
  off[0] = 0;
  loff[0] = 0;
  for (int m = 0; m < ncomp; ++m) {
    long long sz = 1;
    int lsz = 1;
    for (int d = 0; d < 3; ++d) {
      t[m][d] = kTypes[k][m][d];
      N[m][d] = (long long)n[d] * p + (t[m][d] == 's' ? 1 : 0);
      ld[m][d] = t[m][d] == 's' ? p + 1 : p;
      sz *= N[m][d];
      lsz *= ld[m][d];
    }
    off[m + 1] = off[m] + sz;
    loff[m + 1] = loff[m] + lsz;
  }
  size = off[ncomp];
  nloc = loff[ncomp];
}

void Layout::coords(long long idx, int &m, long long g[3]) const {
  m = 0;
  while (m + 1 < ncomp && idx >= off[m + 1]) ++m;
  long long r = idx - off[m];
  g[0] = r % N[m][0];
  r /= N[m][0];
  g[1] = r % N[m][1];
  g[2] = r / N[m][1];
}

// A key whose integer order is the numeric order of doubles (a total order,
// NaNs included).
static inline int64_t total_order_key(double v) {
  int64_t k;
  std::memcpy(&k, &v, sizeof k);
  return k < 0 ? (int64_t)((uint64_t)k ^ 0x7fffffffffffffffULL) : k;
}

// CSR from lists of triplets (duplicates summed).  The triplets are counted
// and scattered in parallel, in no particular order; each row is then sorted
// by column and its duplicates are merged in value order, so the result does
// not depend on the order of the triplets or on the thread count.  The lists
// are freed.
static Csr csr_from_parts(int nrows, int ncols, std::vector<std::vector<Trip>> &parts) {
  Csr A;
  A.nrows = nrows;
  A.ncols = ncols;
  // chunks of at most 1 << 20 triplets, so that even one list keeps every
  // thread busy
  struct Span {
    const Trip *p;
    size_t n;
  };
  std::vector<Span> spans;
  for (auto &t : parts)
    for (size_t a = 0; a < t.size(); a += (size_t)1 << 20)
      spans.push_back({t.data() + a, std::min(t.size() - a, (size_t)1 << 20)});
  const int ns = (int)spans.size();
  std::vector<int64_t> cnt(nrows + 1, 0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < ns; ++q)
    for (size_t a = 0; a < spans[q].n; ++a) {
      const int r = spans[q].p[a].r;
#pragma omp atomic
      cnt[r + 1]++;
    }
  for (int i = 0; i < nrows; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> cc(cnt[nrows]);
  std::vector<double> vv(cnt[nrows]);
  {
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < ns; ++q)
      for (size_t a = 0; a < spans[q].n; ++a) {
        const Trip &x = spans[q].p[a];
        int64_t at;
#pragma omp atomic capture
        at = pos[x.r]++;
        cc[at] = x.c;
        vv[at] = x.v;
      }
  }
  for (auto &t : parts) std::vector<Trip>().swap(t);
  A.ptr.assign(nrows + 1, 0);
  std::vector<int64_t> rowlen(nrows, 0);
  // sort & merge per row
#pragma omp parallel
  {
    std::vector<int> ord;
    std::vector<int> c2;
    std::vector<double> v2;
#pragma omp for schedule(dynamic, 256)
    for (int i = 0; i < nrows; ++i) {
      int64_t b = cnt[i], e = cnt[i + 1];
      int len = (int)(e - b);
      if (len == 0) continue;
      ord.resize(len);
      std::iota(ord.begin(), ord.end(), 0);
      // duplicates merge in value order, so the sums do not depend on the
      // order the (multithreaded) producers emitted them in
      std::sort(ord.begin(), ord.end(), [&](int a, int c) {
        if (cc[b + a] != cc[b + c]) return cc[b + a] < cc[b + c];
        return total_order_key(vv[b + a]) < total_order_key(vv[b + c]);
      });
      c2.clear();
      v2.clear();
      for (int a : ord) {
        if (!c2.empty() && c2.back() == cc[b + a])
          v2.back() += vv[b + a];
        else {
          c2.push_back(cc[b + a]);
          v2.push_back(vv[b + a]);
        }
      }
      for (size_t a = 0; a < c2.size(); ++a) {
        cc[b + a] = c2[a];
        vv[b + a] = v2[a];
      }
      rowlen[i] = (int64_t)c2.size();
    }
  }
  for (int i = 0; i < nrows; ++i) A.ptr[i + 1] = A.ptr[i] + rowlen[i];
  A.col.resize(A.ptr[nrows]);
  A.val.resize(A.ptr[nrows]);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int i = 0; i < nrows; ++i) {
    std::copy(cc.begin() + cnt[i], cc.begin() + cnt[i] + rowlen[i], A.col.begin() + A.ptr[i]);
    std::copy(vv.begin() + cnt[i], vv.begin() + cnt[i] + rowlen[i], A.val.begin() + A.ptr[i]);
  }
  return A;
}

Csr csr_from_triplets(int nrows, int ncols, std::vector<Trip> &t) {
  std::vector<std::vector<Trip>> parts(1);
  parts[0].swap(t);
  return csr_from_parts(nrows, ncols, parts);
}

Csr transpose(const Csr &A) {
  Csr T;
  T.nrows = A.ncols;
  T.ncols = A.nrows;
  T.ptr.assign(T.nrows + 1, 0);
  for (int64_t e = 0; e < A.nnz(); ++e) T.ptr[A.col[e] + 1]++;
  for (int i = 0; i < T.nrows; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.nnz());
  T.val.resize(A.nnz());
  std::vector<int64_t> pos(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < A.nrows; ++i)
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      int64_t p = pos[A.col[e]]++;
      T.col[p] = i;
      T.val[p] = A.val[e];
    }
  return T;
}

void Geometry::cell_vertices(int e1, int e2, int e3, double out[24]) const {
  for (int c3 = 0; c3 < 2; ++c3)
    for (int c2 = 0; c2 < 2; ++c2)
      for (int c1 = 0; c1 < 2; ++c1) {
        long long a = (e1 + c1) + (long long)(n[0] + 1) * ((e2 + c2) + (long long)(n[1] + 1) * (e3 + c3));
        int c = c1 + 2 * c2 + 4 * c3;
        for (int x = 0; x < 3; ++x) out[3 * c + x] = X[3 * a + x];
      }
}

FreeMap::FreeMap(const Layout &L) {
  lat2free.assign(L.size, -1);
  for (int m = 0; m < L.ncomp; ++m)
    for (long long g3 = 0; g3 < L.N[m][2]; ++g3)
      for (long long g2 = 0; g2 < L.N[m][1]; ++g2)
        for (long long g1 = 0; g1 < L.N[m][0]; ++g1) {
          long long g[3] = {g1, g2, g3};
          if (!L.dirichlet(m, g)) {
            long long idx = L.index(m, g1, g2, g3);
            lat2free[idx] = (int)free2lat.size();
            free2lat.push_back((int)idx);
          }
        }
}

// ---------------------------------------------------------------------------
// geometry at a reference point
// ---------------------------------------------------------------------------
static void jacobian(const double X8[24], const double xi[3], double J[9]) {
  double N[3][2], dN[2] = {-0.5, 0.5};
  for (int d = 0; d < 3; ++d) {
    N[d][0] = 0.5 * (1.0 - xi[d]);
    N[d][1] = 0.5 * (1.0 + xi[d]);
  }
  for (int i = 0; i < 9; ++i) J[i] = 0.0;
  for (int c3 = 0; c3 < 2; ++c3)
    for (int c2 = 0; c2 < 2; ++c2)
      for (int c1 = 0; c1 < 2; ++c1) {
        const double *v = X8 + 3 * (c1 + 2 * c2 + 4 * c3);
        double g0 = dN[c1] * N[1][c2] * N[2][c3];
        double g1 = N[0][c1] * dN[c2] * N[2][c3];
        double g2 = N[0][c1] * N[1][c2] * dN[c3];
        for (int a = 0; a < 3; ++a) {
          J[3 * a + 0] += v[a] * g0;
          J[3 * a + 1] += v[a] * g1;
          J[3 * a + 2] += v[a] * g2;
        }
      }
}

static double det3(const double J[9]) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
         J[2] * (J[3] * J[7] - J[4] * J[6]);
}

// full pullback weight of kk-forms (Sec. 3.1): out 3x3 (or [0] for scalars)
static void form_weight(int kk, const double J[9], double W[9]) {
  double det = det3(J);
  if (!(det > 0)) throw std::runtime_error("inverted or degenerate cell");
  if (kk == 0) { W[0] = det; return; }
  if (kk == 3) { W[0] = 1.0 / det; return; }
  if (kk == 2) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double s = 0.0;
        for (int c = 0; c < 3; ++c) s += J[3 * c + a] * J[3 * c + b];
        W[3 * a + b] = s / det;
      }
    return;
  }
  // kk == 1: det J^-1 J^-T = adj adj^T / det, adj = det J^-1
  double A[9];
  A[0] = J[4] * J[8] - J[5] * J[7];
  A[1] = J[2] * J[7] - J[1] * J[8];
  A[2] = J[1] * J[5] - J[2] * J[4];
  A[3] = J[5] * J[6] - J[3] * J[8];
  A[4] = J[0] * J[8] - J[2] * J[6];
  A[5] = J[2] * J[3] - J[0] * J[5];
  A[6] = J[3] * J[7] - J[4] * J[6];
  A[7] = J[1] * J[6] - J[0] * J[7];
  A[8] = J[0] * J[4] - J[1] * J[3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int c = 0; c < 3; ++c) s += A[3 * a + c] * A[3 * b + c];
      W[3 * a + b] = s / det;
    }
}

// ---------------------------------------------------------------------------
// auxiliary operator
// ---------------------------------------------------------------------------
namespace {

struct SparseVec {
  std::vector<int> idx;
  std::vector<double> val;
  void clear() { idx.clear(); val.clear(); }
};

struct AuxCtx {
  Layout Lk, Lk1;
  int p = 0, q = 0;
  std::vector<double> xq, wq;
  std::vector<double> Tsb, Tr;   // broken s-tabulation q x (p+1), r-tabulation q x p
  std::vector<double> D1;        // p x (p+1)
  double h = 1.0 / std::sqrt(2.0);
};

// entries of row j of the 1D broken transform G for type ty
inline int grow(char ty, int j, int p, double h, int *ii, double *vv) {
  if (ty == 'r' || (j > 0 && j < p)) { ii[0] = j; vv[0] = 1.0; return 1; }
  ii[0] = 0; vv[0] = h;
  ii[1] = p; vv[1] = (j == 0) ? h : -h;
  return 2;
}

// diag of the broken weighted mass of V^kk (layout Lx) with per-point weight
// F[m][q] (already including w_q and the coefficient): sum-factorised
// d[m](i1,i2,i3) = sum_q F[m][q] Tb1[q1,i1]^2 Tb2[q2,i2]^2 Tb3[q3,i3]^2.
void broken_diag(const AuxCtx &C, const Layout &Lx, const std::vector<double> *F,
                 std::vector<double> &d) {
  const int q = C.q, p = C.p;
  d.assign(Lx.nloc, 0.0);
  std::vector<double> t1, t2;
  for (int m = 0; m < Lx.ncomp; ++m) {
    const int l1 = Lx.ld[m][0], l2 = Lx.ld[m][1], l3 = Lx.ld[m][2];
    auto sq = [&](int d, int qq, int i) {
      double v = Lx.t[m][d] == 's' ? C.Tsb[qq * (p + 1) + i] : C.Tr[qq * p + i];
      return v * v;
    };
    // contract q1 -> i1: t1[q3][q2][i1]
    t1.assign((size_t)q * q * l1, 0.0);
    for (int q3 = 0; q3 < q; ++q3)
      for (int q2 = 0; q2 < q; ++q2)
        for (int i1 = 0; i1 < l1; ++i1) {
          double s = 0.0;
          for (int q1 = 0; q1 < q; ++q1) s += F[m][q1 + q * (q2 + q * q3)] * sq(0, q1, i1);
          t1[(q3 * q + q2) * l1 + i1] = s;
        }
    // contract q2 -> i2: t2[q3][i2][i1]
    t2.assign((size_t)q * l2 * l1, 0.0);
    for (int q3 = 0; q3 < q; ++q3)
      for (int i2 = 0; i2 < l2; ++i2)
        for (int i1 = 0; i1 < l1; ++i1) {
          double s = 0.0;
          for (int q2 = 0; q2 < q; ++q2) s += t1[(q3 * q + q2) * l1 + i1] * sq(1, q2, i2);
          t2[(q3 * l2 + i2) * l1 + i1] = s;
        }
    for (int i3 = 0; i3 < l3; ++i3)
      for (int i2 = 0; i2 < l2; ++i2)
        for (int i1 = 0; i1 < l1; ++i1) {
          double s = 0.0;
          for (int q3 = 0; q3 < q; ++q3) s += t2[(q3 * l2 + i2) * l1 + i1] * sq(2, q3, i3);
          d[Lx.loff[m] + i1 + l1 * (i2 + l2 * i3)] = s;
        }
  }
}

}  // namespace

Csr assemble_aux(const Layout &L, const Geometry &geo, const double *mcoef,
                 const double *scoef, const FreeMap &fm) {
  if (L.k > 2) throw std::runtime_error("assemble_aux: k in 0..2");
  AuxCtx C;
  C.p = L.p;
  C.Lk = L;
  C.Lk1 = Layout(L.k + 1, L.n, L.p, L.natural);
  const int p = L.p;
  Basis1D B(p);
  C.q = quad_points(p);
  gll_rule(C.q, C.xq, C.wq);
  const int q = C.q;
  std::vector<double> Ts(q * (p + 1));
  B.tab_s(C.xq.data(), q, Ts.data());
  C.Tr.resize(q * p);
  B.tab_r(C.xq.data(), q, C.Tr.data());
  C.Tsb = Ts;
  for (int a = 0; a < q; ++a) {
    double s0 = Ts[a * (p + 1) + 0], sp = Ts[a * (p + 1) + p];
    C.Tsb[a * (p + 1) + 0] = C.h * (s0 + sp);
    C.Tsb[a * (p + 1) + p] = C.h * (s0 - sp);
  }
  C.D1 = B.D;
  const int k = L.k;
  const Layout &Lk1 = C.Lk1;
  const int nloc = L.nloc, nloc1 = Lk1.nloc;
  const int ncell = L.n[0] * L.n[1] * L.n[2];
  const int nq = q * q * q;
  const int nfree = (int)fm.free2lat.size();

  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  std::vector<std::vector<Trip>> trips(nthreads);
  // a cell whose Jacobian is not positive somewhere; reported after the
  // parallel region (an exception must not leave it)
  int bad_cell = -1;

#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    // local entries of P_K as (i * nloc + j, value), merged after the cell
    std::vector<std::pair<long long, double>> ent;
    std::vector<double> Fk[3], Fk1[3], dk, dk1;
    std::vector<int> l2f(nloc);
    std::vector<double> acc(nloc, 0.0);
    std::vector<char> accm(nloc, 0);
    SparseVec row, drow;
    auto add_outer = [&](const SparseVec &v, double w) {
      for (size_t a = 0; a < v.idx.size(); ++a)
        for (size_t b = 0; b < v.idx.size(); ++b)
          ent.push_back({(long long)v.idx[a] * nloc + v.idx[b], w * v.val[a] * v.val[b]});
    };
#pragma omp for schedule(dynamic, 1)
    for (int c = 0; c < ncell; ++c) {
      const int e1 = c % L.n[0], e2 = (c / L.n[0]) % L.n[1], e3 = c / (L.n[0] * L.n[1]);
      double X8[24];
      geo.cell_vertices(e1, e2, e3, X8);
      // per-point diagonal weights of V^k and V^{k+1}
      for (int m = 0; m < 3; ++m) {
        Fk[m].assign(nq, 0.0);
        Fk1[m].assign(nq, 0.0);
      }
      for (int q3 = 0; q3 < q; ++q3)
        for (int q2 = 0; q2 < q; ++q2)
          for (int q1 = 0; q1 < q; ++q1) {
            double xi[3] = {C.xq[q1], C.xq[q2], C.xq[q3]};
            double J[9], W[9];
            jacobian(X8, xi, J);
            if (!(det3(J) > 0)) {
#pragma omp critical
              bad_cell = c;
              for (int a = 0; a < 9; ++a) J[a] = (a % 4 == 0) ? 1.0 : 0.0;  // placeholder, discarded
            }
            double w = C.wq[q1] * C.wq[q2] * C.wq[q3];
            int qi = q1 + q * (q2 + q * q3);
            form_weight(k, J, W);
            for (int m = 0; m < L.ncomp; ++m)
              Fk[m][qi] = mcoef[c] * w * (L.ncomp == 1 ? W[0] : W[4 * m]);
            form_weight(k + 1, J, W);
            for (int m = 0; m < Lk1.ncomp; ++m)
              Fk1[m][qi] = scoef[c] * w * (Lk1.ncomp == 1 ? W[0] : W[4 * m]);
          }
      broken_diag(C, L, Fk, dk);
      broken_diag(C, Lk1, Fk1, dk1);
      // mass part: G^T diag(dk) G
      for (int m = 0; m < L.ncomp; ++m) {
        const int l1 = L.ld[m][0], l2 = L.ld[m][1], l3 = L.ld[m][2];
        for (int j3 = 0; j3 < l3; ++j3)
          for (int j2 = 0; j2 < l2; ++j2)
            for (int j1 = 0; j1 < l1; ++j1) {
              double db = dk[L.loff[m] + j1 + l1 * (j2 + l2 * j3)];
              if (db == 0.0) continue;
              int i1[2], i2[2], i3[2];
              double v1[2], v2[2], v3[2];
              int n1 = grow(L.t[m][0], j1, p, C.h, i1, v1);
              int n2 = grow(L.t[m][1], j2, p, C.h, i2, v2);
              int n3 = grow(L.t[m][2], j3, p, C.h, i3, v3);
              row.clear();
              for (int a3 = 0; a3 < n3; ++a3)
                for (int a2 = 0; a2 < n2; ++a2)
                  for (int a1 = 0; a1 < n1; ++a1) {
                    row.idx.push_back(L.loff[m] + i1[a1] + l1 * (i2[a2] + l2 * i3[a3]));
                    row.val.push_back(v1[a1] * v2[a2] * v3[a3]);
                  }
              add_outer(row, db);
            }
      }
      // derivative part: Dbar^T diag(dk1) Dbar, Dbar = G' D-hat
      for (int t = 0; t < Lk1.ncomp; ++t) {
        const int l1 = Lk1.ld[t][0], l2 = Lk1.ld[t][1], l3 = Lk1.ld[t][2];
        for (int j3 = 0; j3 < l3; ++j3)
          for (int j2 = 0; j2 < l2; ++j2)
            for (int j1 = 0; j1 < l1; ++j1) {
              double db = dk1[Lk1.loff[t] + j1 + l1 * (j2 + l2 * j3)];
              if (db == 0.0) continue;
              int i1[2], i2[2], i3[2];
              double v1[2], v2[2], v3[2];
              int n1 = grow(Lk1.t[t][0], j1, p, C.h, i1, v1);
              int n2 = grow(Lk1.t[t][1], j2, p, C.h, i2, v2);
              int n3 = grow(Lk1.t[t][2], j3, p, C.h, i3, v3);
              drow.clear();
              for (int a3 = 0; a3 < n3; ++a3)
                for (int a2 = 0; a2 < n2; ++a2)
                  for (int a1 = 0; a1 < n1; ++a1) {
                    double g = v1[a1] * v2[a2] * v3[a3];
                    int ii[3] = {i1[a1], i2[a2], i3[a3]};
                    // row (t, ii) of D-hat
                    for (int s = 0; s < kNumTerms[k][t]; ++s) {
                      const DTerm &T = kTerms[k][t][s];
                      const int sm = T.src, dd = T.dir;
                      const int s1 = L.ld[sm][0], s2 = L.ld[sm][1];
                      for (int l = 0; l <= p; ++l) {
                        double dv = C.D1[ii[dd] * (p + 1) + l];
                        if (dv == 0.0) continue;
                        int jj[3] = {ii[0], ii[1], ii[2]};
                        jj[dd] = l;
                        int src = L.loff[sm] + jj[0] + s1 * (jj[1] + s2 * jj[2]);
                        if (!accm[src]) {
                          accm[src] = 1;
                          drow.idx.push_back(src);
                          acc[src] = 0.0;
                        }
                        acc[src] += g * T.sgn * dv;
                      }
                    }
                  }
              for (size_t a = 0; a < drow.idx.size(); ++a) {
                drow.val.push_back(acc[drow.idx[a]]);
                accm[drow.idx[a]] = 0;
              }
              add_outer(drow, db);
            }
      }
      // local -> free
      for (int m = 0; m < L.ncomp; ++m) {
        const int l1 = L.ld[m][0], l2 = L.ld[m][1], l3 = L.ld[m][2];
        for (int i3 = 0; i3 < l3; ++i3)
          for (int i2 = 0; i2 < l2; ++i2)
            for (int i1 = 0; i1 < l1; ++i1) {
              long long idx = L.index(m, (long long)e1 * p + i1, (long long)e2 * p + i2,
                                      (long long)e3 * p + i3);
              l2f[L.loff[m] + i1 + l1 * (i2 + l2 * i3)] = fm.lat2free[idx];
            }
      }
      std::sort(ent.begin(), ent.end(),
                [](const std::pair<long long, double> &x, const std::pair<long long, double> &y) {
                  return x.first < y.first;
                });
      for (size_t a = 0; a < ent.size();) {
        const long long key = ent[a].first;
        double v = 0.0;
        for (; a < ent.size() && ent[a].first == key; ++a) v += ent[a].second;
        const int i = (int)(key / nloc), j = (int)(key % nloc);
        if (l2f[i] >= 0 && l2f[j] >= 0) trips[tid].push_back({l2f[i], l2f[j], v});
      }
      ent.clear();
    }
  }
  if (bad_cell >= 0) throw std::runtime_error("inverted or degenerate cell " + std::to_string(bad_cell));
  (void)nloc1;
  return csr_from_parts(nfree, nfree, trips);
}

// ---------------------------------------------------------------------------
// static condensation
// ---------------------------------------------------------------------------
static bool is_interior(const Layout &L, long long lat) {
  int m;
  long long g[3];
  L.coords(lat, m, g);
  for (int d = 0; d < 3; ++d)
    if (L.t[m][d] == 's' && g[d] % L.p == 0) return false;
  return true;
}

// The inverse Cholesky factor of a small SPD block (row-major, n x n):
// A = L L^T, returns L^-1 (lower triangular).  A non-positive pivot is an
// error (the interior block of the auxiliary operator is SPD).
static std::vector<double> inverse_cholesky_small(const std::vector<double> &A, int n) {
  std::vector<double> L(n * n, 0.0), Li(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) throw std::runtime_error("interior block not positive definite");
    L[j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = v / L[j * n + j];
    }
  }
  for (int c = 0; c < n; ++c) {  // columns of L^-1 by forward substitution
    for (int i = c; i < n; ++i) {
      double v = i == c ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v -= L[i * n + k] * Li[k * n + c];
      Li[i * n + c] = v / L[i * n + i];
    }
  }
  return Li;
}

// CSR from rows computed independently: row_fn(i, cols, vals) fills row i
// (columns in any order, no duplicates).  The listed rows (increasing) are
// split into one contiguous range per chunk, computed and column-sorted in
// parallel and copied into place; every other row is empty.
template <class RowFn>
static Csr csr_from_rows(int nrows, int ncols, const std::vector<int> &rows, RowFn row_fn) {
  Csr A;
  A.nrows = nrows;
  A.ncols = ncols;
  const int nr = (int)rows.size();
  int nch = 1;
#ifdef _OPENMP
  nch = 4 * omp_get_max_threads();
#endif
  std::vector<std::vector<int>> tc(nch);
  std::vector<std::vector<double>> tv(nch);
  std::vector<int64_t> len(nr, 0);
  auto lo = [&](int t) { return (int)((int64_t)nr * t / nch); };
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < nch; ++t) {
    std::vector<int> c, ord;
    std::vector<double> v;
    for (int r = lo(t); r < lo(t + 1); ++r) {
      c.clear();
      v.clear();
      row_fn(rows[r], c, v);
      ord.resize(c.size());
      std::iota(ord.begin(), ord.end(), 0);
      std::sort(ord.begin(), ord.end(), [&](int a, int b) { return c[a] < c[b]; });
      for (int a : ord) {
        tc[t].push_back(c[a]);
        tv[t].push_back(v[a]);
      }
      len[r] = (int64_t)c.size();
    }
  }
  A.ptr.assign(nrows + 1, 0);
  for (int r = 0; r < nr; ++r) A.ptr[rows[r] + 1] = len[r];
  for (int i = 0; i < nrows; ++i) A.ptr[i + 1] += A.ptr[i];
  A.col.resize(A.ptr[nrows]);
  A.val.resize(A.ptr[nrows]);
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < nch; ++t) {
    if (lo(t) == lo(t + 1)) continue;
    const int64_t at = A.ptr[rows[lo(t)]];
    std::copy(tc[t].begin(), tc[t].end(), A.col.begin() + at);
    std::copy(tv[t].begin(), tv[t].end(), A.val.begin() + at);
    std::vector<int>().swap(tc[t]);
    std::vector<double>().swap(tv[t]);
  }
  return A;
}

Condensed condense(const Layout &L, const FreeMap &fm, const Csr &P) {
  Condensed R;
  const int nf = P.nrows;
  std::vector<char> inI(nf, 0);
  for (int f = 0; f < nf; ++f) {
    if (is_interior(L, fm.free2lat[f])) {
      inI[f] = 1;
      R.I.push_back(f);
    } else {
      R.G.push_back(f);
    }
  }
  // blocks of P_II by union-find
  std::vector<int> parent(nf);
  std::iota(parent.begin(), parent.end(), 0);
  std::function<int(int)> find = [&](int x) {
    while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
    return x;
  };
  for (int i : R.I)
    for (int64_t e = P.ptr[i]; e < P.ptr[i + 1]; ++e) {
      int j = P.col[e];
      if (inI[j] && P.val[e] != 0.0) {
        int a = find(i), b = find(j);
        if (a != b) parent[a] = b;
      }
    }
  std::unordered_map<int, std::vector<int>> blocks;
  for (int i : R.I) blocks[find(i)].push_back(i);
  std::vector<int> blk_of(nf, -1);
  std::vector<std::vector<int>> blist;
  for (auto &kv : blocks) {
    std::sort(kv.second.begin(), kv.second.end());
    if (kv.second.size() > 8) throw std::runtime_error("interior block larger than 8");
    for (int i : kv.second) blk_of[i] = (int)blist.size();
    blist.push_back(kv.second);
  }
  auto getP = [&](int i, int j) {
    auto b = P.col.begin() + P.ptr[i], e = P.col.begin() + P.ptr[i + 1];
    auto it = std::lower_bound(b, e, j);
    return (it != e && *it == j) ? P.val[it - P.col.begin()] : 0.0;
  };
  // P_II = L L^T blockwise; P_II^-1 = L^-T L^-1 formed as that product, so it
  // is symmetric to the last bit and positive definite
  std::vector<std::vector<double>> binv(blist.size()), linv(blist.size());
  std::vector<Trip> tb;
  for (size_t b = 0; b < blist.size(); ++b) {
    const auto &ix = blist[b];
    int n = (int)ix.size();
    std::vector<double> A(n * n);
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) A[a * n + c] = getP(ix[a], ix[c]);
    linv[b] = inverse_cholesky_small(A, n);
    const std::vector<double> &Li = linv[b];
    std::vector<double> Bi(n * n, 0.0);
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) {
        double v = 0.0;
        for (int k = std::max(a, c); k < n; ++k) v += Li[k * n + a] * Li[k * n + c];
        Bi[a * n + c] = v;
      }
    binv[b] = Bi;
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) tb.push_back({ix[a], ix[c], Bi[a * n + c]});
  }
  R.Binv = csr_from_triplets(nf, nf, tb);
  // E = P_GI Binv, row by row (each entry summed in the order of P's row)
  {
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    std::vector<std::vector<double>> accs(nth);
    std::vector<std::vector<char>> marks(nth);
    R.E = csr_from_rows(nf, nf, R.G, [&](int g, std::vector<int> &cols, std::vector<double> &vals) {
      int t = 0;
#ifdef _OPENMP
      t = omp_get_thread_num();
#endif
      std::vector<double> &acc = accs[t];
      std::vector<char> &m = marks[t];
      if (acc.empty()) {
        acc.assign(nf, 0.0);
        m.assign(nf, 0);
      }
      for (int64_t e = P.ptr[g]; e < P.ptr[g + 1]; ++e) {
        int i = P.col[e];
        if (!inI[i] || P.val[e] == 0.0) continue;
        int b = blk_of[i];
        const auto &ix = blist[b];
        int n = (int)ix.size();
        int a = (int)(std::find(ix.begin(), ix.end(), i) - ix.begin());
        for (int c = 0; c < n; ++c) {
          const int j = ix[c];
          if (!m[j]) {
            m[j] = 1;
            acc[j] = 0.0;
            cols.push_back(j);
          }
          acc[j] += P.val[e] * binv[b][a * n + c];
        }
      }
      for (int j : cols) {
        vals.push_back(acc[j]);
        m[j] = 0;
      }
    });
  }
  R.Et = transpose(R.E);
  // S = P_GG - W^T W with W = L^-1 P_IG (blockwise): the Schur complement of
  // Eq. schur in a form that stays symmetric positive definite in floating
  // point when P_II is ill conditioned (beta << alpha makes the interior
  // gradients (curls) nearly singular): the product E P_IG through an
  // explicit inverse loses both properties there.  Per block: its interface
  // columns (sorted) and W_b = L_b^-1 P_{b,cols}.
  std::vector<std::vector<int>> wcols(blist.size());
  std::vector<std::vector<double>> wval(blist.size());
  {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long long bb = 0; bb < (long long)blist.size(); ++bb) {
      const auto &ix = blist[bb];
      const int n = (int)ix.size();
      std::vector<int> &cols = wcols[bb];
      for (int i : ix)
        for (int64_t e = P.ptr[i]; e < P.ptr[i + 1]; ++e)
          if (!inI[P.col[e]] && P.val[e] != 0.0) cols.push_back(P.col[e]);
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      const int nc = (int)cols.size();
      std::vector<double> PB(n * nc, 0.0);
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < nc; ++c) PB[a * nc + c] = getP(ix[a], cols[c]);
      const std::vector<double> &Li = linv[bb];
      std::vector<double> &W = wval[bb];
      W.assign(n * nc, 0.0);
      for (int k = 0; k < n; ++k)
        for (int c = 0; c < nc; ++c) {
          double v = 0.0;
          for (int a = 0; a <= k; ++a) v += Li[k * n + a] * PB[a * nc + c];
          W[k * nc + c] = v;
        }
    }
  }
  {
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    std::vector<std::vector<double>> accs(nth);
    std::vector<std::vector<char>> marks(nth), bmarks(nth);
    R.S = csr_from_rows(nf, nf, R.G, [&](int g, std::vector<int> &cols, std::vector<double> &vals) {
      int t = 0;
#ifdef _OPENMP
      t = omp_get_thread_num();
#endif
      std::vector<double> &acc = accs[t];
      std::vector<char> &m = marks[t];
      std::vector<char> &bm = bmarks[t];
      if (acc.empty()) {
        acc.assign(nf, 0.0);
        m.assign(nf, 0);
        bm.assign(blist.size(), 0);
      }
      for (int64_t e = P.ptr[g]; e < P.ptr[g + 1]; ++e) {
        int c = P.col[e];
        if (inI[c]) continue;
        if (!m[c]) { m[c] = 1; cols.push_back(c); acc[c] = 0.0; }
        acc[c] += P.val[e];
      }
      // the blocks coupled to g, in the order of P's row g
      std::vector<int> bl;
      for (int64_t e = P.ptr[g]; e < P.ptr[g + 1]; ++e) {
        int i = P.col[e];
        if (!inI[i] || P.val[e] == 0.0) continue;
        const int b = blk_of[i];
        if (!bm[b]) { bm[b] = 1; bl.push_back(b); }
      }
      for (int b : bl) {
        bm[b] = 0;
        const std::vector<int> &wc = wcols[b];
        const std::vector<double> &W = wval[b];
        const int n = (int)blist[b].size(), nc = (int)wc.size();
        const int gi = (int)(std::lower_bound(wc.begin(), wc.end(), g) - wc.begin());
        if (gi == nc || wc[gi] != g) continue;  // P_{b,g} = 0: no contribution
        for (int c = 0; c < nc; ++c) {
          double v = 0.0;
          for (int k = 0; k < n; ++k) v += W[k * nc + gi] * W[k * nc + c];
          const int cc = wc[c];
          if (!m[cc]) { m[cc] = 1; cols.push_back(cc); acc[cc] = 0.0; }
          acc[cc] -= v;
        }
      }
      for (int c : cols) {
        vals.push_back(acc[c]);
        m[c] = 0;
      }
    });
  }
  return R;
}

// ---------------------------------------------------------------------------
// patches
// ---------------------------------------------------------------------------
namespace {
struct Slot {
  int m, o[3], dim;
};
}  // namespace

static const double kDrop = 1e-12;  // ICC pattern: |A_ij| > kDrop sqrt(|A_ii A_jj|)

PatchFamily build_patches(const Layout &L, const FreeMap &fm, const Csr &M, int span,
                          bool interface_only, int factor) {
  const int p = L.p;
  // slot template
  std::vector<Slot> slots;
  for (int m = 0; m < L.ncomp; ++m) {
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      bool cell = (span >> d) & 1;
      bool s = L.t[m][d] == 's';
      if (cell) { lo[d] = s ? 1 : 0; hi[d] = p - 1; }
      else { lo[d] = s ? -(p - 1) : -p; hi[d] = p - 1; }
    }
    for (int o3 = lo[2]; o3 <= hi[2]; ++o3)
      for (int o2 = lo[1]; o2 <= hi[1]; ++o2)
        for (int o1 = lo[0]; o1 <= hi[0]; ++o1) {
          int o[3] = {o1, o2, o3};
          int nv = 0;
          for (int d = 0; d < 3; ++d)
            if (!((span >> d) & 1) && L.t[m][d] == 's' && o[d] == 0) ++nv;
          if (interface_only && nv == 0) continue;
          slots.push_back({m, {o1, o2, o3}, 3 - nv});
        }
  }
  std::stable_sort(slots.begin(), slots.end(), [](const Slot &a, const Slot &b) {
    if (a.dim != b.dim) return a.dim > b.dim;
    if (a.m != b.m) return a.m < b.m;
    if (a.o[2] != b.o[2]) return a.o[2] < b.o[2];
    if (a.o[1] != b.o[1]) return a.o[1] < b.o[1];
    return a.o[0] < b.o[0];
  });
  const int ns = (int)slots.size();
  if (ns > 6000)
    throw std::runtime_error("patch template of " + std::to_string(ns) +
                             " slots is too large (> 6000): use static condensation");
  PatchFamily F;
  F.nslots = ns;
  // entities
  int hi[3];
  for (int d = 0; d < 3; ++d) hi[d] = L.n[d] - (((span >> d) & 1) ? 1 : 0);
  std::vector<int> smap;
  for (int a3 = 0; a3 <= hi[2]; ++a3)
    for (int a2 = 0; a2 <= hi[1]; ++a2)
      for (int a1 = 0; a1 <= hi[0]; ++a1) {
        int a[3] = {a1, a2, a3};
        std::vector<int> row(ns, -1);
        int nvalid = 0;
        for (int s = 0; s < ns; ++s) {
          const Slot &S = slots[s];
          long long g[3];
          bool ok = true;
          for (int d = 0; d < 3; ++d) {
            g[d] = (long long)a[d] * p + S.o[d];
            if (g[d] < 0 || g[d] >= L.N[S.m][d]) ok = false;
          }
          if (!ok) continue;
          long long idx = L.index(S.m, g[0], g[1], g[2]);
          if (fm.lat2free[idx] < 0) continue;
          row[s] = (int)idx;
          ++nvalid;
        }
        if (nvalid == 0) continue;
        smap.insert(smap.end(), row.begin(), row.end());
      }
  F.npatch = (int)(smap.size() / (ns ? ns : 1));
  F.slotmap.swap(smap);
  const int np = F.npatch;
  const int nf = M.nrows;

  auto extract = [&](int pi, std::vector<int> &pos, std::vector<double> &A) {
    A.assign((size_t)ns * ns, 0.0);
    const int *sm = &F.slotmap[(size_t)pi * ns];
    for (int s = 0; s < ns; ++s)
      if (sm[s] >= 0) pos[fm.lat2free[sm[s]]] = s;
    for (int s = 0; s < ns; ++s) {
      if (sm[s] < 0) { A[(size_t)s * ns + s] = 1.0; continue; }
      int f = fm.lat2free[sm[s]];
      for (int64_t e = M.ptr[f]; e < M.ptr[f + 1]; ++e) {
        int t = pos[M.col[e]];
        if (t >= 0) A[(size_t)s * ns + t] = M.val[e];
      }
    }
    for (int s = 0; s < ns; ++s)
      if (sm[s] >= 0) pos[fm.lat2free[sm[s]]] = -1;
  };
  auto own = [&](const std::vector<double> &A, int i, int j) {
    if (i == j) return true;
    double a = A[(size_t)i * ns + j];
    return std::fabs(a) > kDrop * std::sqrt(std::fabs(A[(size_t)i * ns + i] * A[(size_t)j * ns + j]));
  };
  // pass 1: union of the thresholded lower patterns
  std::vector<char> uni((size_t)ns * ns, 0);
#pragma omp parallel
  {
    std::vector<int> pos(nf, -1);
    std::vector<double> A;
    std::vector<char> mine((size_t)ns * ns, 0);
#pragma omp for schedule(dynamic, 4)
    for (int pi = 0; pi < np; ++pi) {
      extract(pi, pos, A);
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j <= i; ++j)
          if (own(A, i, j)) mine[(size_t)i * ns + j] = 1;
    }
#pragma omp critical
    for (size_t x = 0; x < mine.size(); ++x) uni[x] |= mine[x];
  }
  // Exact factorisation: the patch matrix splits into decoupled blocks (the
  // connected components of the union pattern; p blocks for H(curl) edge
  // stars, fig. spy_feec(e)).  Store the dense inverse of each block, so the
  // device applies L^-T L^-1 as one parallel product with no level chain.
  if (factor == 0) {
    std::vector<int> comp(ns, -1);
    std::vector<std::vector<int>> adj(ns);
    for (int i = 0; i < ns; ++i)
      for (int j = 0; j < i; ++j)
        if (uni[(size_t)i * ns + j]) {
          adj[i].push_back(j);
          adj[j].push_back(i);
        }
    int nblk = 0;
    std::vector<std::vector<int>> blocks;
    for (int s0 = 0; s0 < ns; ++s0) {
      if (comp[s0] >= 0) continue;
      std::vector<int> stack{s0}, members;
      comp[s0] = nblk;
      while (!stack.empty()) {
        int u = stack.back();
        stack.pop_back();
        members.push_back(u);
        for (int v : adj[u])
          if (comp[v] < 0) {
            comp[v] = nblk;
            stack.push_back(v);
          }
      }
      std::sort(members.begin(), members.end());
      blocks.push_back(members);
      ++nblk;
    }
    F.inverse = 1;
    F.bptr.assign(1, 0);
    F.boff.assign(1, 0);
    for (int b = 0; b < nblk; ++b) {
      for (int s : blocks[b]) {
        F.pos_slot.push_back(s);
        F.pos_blk.push_back(b);
      }
      const int nb = (int)blocks[b].size();
      F.bptr.push_back(F.bptr.back() + nb);
      F.boff.push_back(F.boff.back() + nb * nb);
    }
    const int nv = F.boff.back();
    F.ival.assign((size_t)np * nv, 0.0);
    int bad = -1;
#pragma omp parallel
    {
      std::vector<int> pos(nf, -1);
      std::vector<double> A, Bk;
#pragma omp for schedule(dynamic, 4)
      for (int pi = 0; pi < np; ++pi) {
        extract(pi, pos, A);
        double *out = &F.ival[(size_t)pi * nv];
        for (int b = 0; b < nblk; ++b) {
          const std::vector<int> &m = blocks[b];
          const int nb = (int)m.size();
          Bk.assign((size_t)nb * nb, 0.0);
          for (int x = 0; x < nb; ++x)
            for (int y = 0; y < nb; ++y)
              if (own(A, m[x], m[y])) Bk[(size_t)x * nb + y] = A[(size_t)m[x] * ns + m[y]];
          // Cholesky, then the inverse L^-T L^-1
          bool ok = true;
          for (int j = 0; j < nb && ok; ++j) {
            double d = Bk[(size_t)j * nb + j];
            for (int kk = 0; kk < j; ++kk) d -= Bk[(size_t)j * nb + kk] * Bk[(size_t)j * nb + kk];
            if (!(d > 0.0)) { ok = false; break; }
            d = std::sqrt(d);
            Bk[(size_t)j * nb + j] = d;
            for (int i = j + 1; i < nb; ++i) {
              double s = Bk[(size_t)i * nb + j];
              for (int kk = 0; kk < j; ++kk) s -= Bk[(size_t)i * nb + kk] * Bk[(size_t)j * nb + kk];
              Bk[(size_t)i * nb + j] = s / d;
            }
          }
          if (!ok) {
#pragma omp critical
            bad = pi;
            continue;
          }
          std::vector<double> Linv((size_t)nb * nb, 0.0);  // lower, L^-1
          for (int c = 0; c < nb; ++c) {
            Linv[(size_t)c * nb + c] = 1.0 / Bk[(size_t)c * nb + c];
            for (int i = c + 1; i < nb; ++i) {
              double s = 0.0;
              for (int kk = c; kk < i; ++kk) s -= Bk[(size_t)i * nb + kk] * Linv[(size_t)kk * nb + c];
              Linv[(size_t)i * nb + c] = s / Bk[(size_t)i * nb + i];
            }
          }
          double *ob = out + F.boff[b];
          for (int x = 0; x < nb; ++x)
            for (int y = 0; y <= x; ++y) {
              double s = 0.0;
              for (int kk = x; kk < nb; ++kk) s += Linv[(size_t)kk * nb + x] * Linv[(size_t)kk * nb + y];
              ob[(size_t)y * nb + x] = s;
              ob[(size_t)x * nb + y] = s;
            }
        }
      }
    }
    if (bad >= 0)
      throw std::runtime_error("patch factorisation breakdown (non-positive pivot) in patch " +
                               std::to_string(bad));
    return F;
  }
  // symbolic fill for exact Cholesky
  if (factor == 0) {
    for (int j = 0; j < ns; ++j) {
      std::vector<int> below;
      for (int i = j + 1; i < ns; ++i)
        if (uni[(size_t)i * ns + j]) below.push_back(i);
      for (size_t a = 0; a < below.size(); ++a)
        for (size_t b = 0; b <= a; ++b) uni[(size_t)below[a] * ns + below[b]] = 1;
    }
  }
  F.rowptr.assign(ns + 1, 0);
  for (int i = 0; i < ns; ++i) {
    for (int j = 0; j < i; ++j)
      if (uni[(size_t)i * ns + j]) F.col.push_back(j);
    F.col.push_back(i);
    F.rowptr[i + 1] = (int)F.col.size();
  }
  const int nnz = F.nnz();
  // pass 2: numeric factorisation on the template pattern (left-looking)
  F.val.assign((size_t)np * nnz, 0.0);
  int breakdown = -1;
#pragma omp parallel
  {
    std::vector<int> pos(nf, -1);
    std::vector<double> A, Ld((size_t)ns * ns, 0.0);
#pragma omp for schedule(dynamic, 4)
    for (int pi = 0; pi < np; ++pi) {
      extract(pi, pos, A);
      for (int i = 0; i < ns; ++i) {
        double *Li = &Ld[(size_t)i * ns];
        for (int e = F.rowptr[i]; e < F.rowptr[i + 1] - 1; ++e) {
          int j = F.col[e];
          double v = 0.0;
          if (factor == 0 || own(A, i, j)) {
            double s = A[(size_t)i * ns + j];
            const double *Lj = &Ld[(size_t)j * ns];
            for (int f = F.rowptr[j]; f < F.rowptr[j + 1] - 1; ++f) s -= Lj[F.col[f]] * Li[F.col[f]];
            v = s / Lj[j];
          }
          Li[j] = v;
        }
        double s = A[(size_t)i * ns + i];
        for (int e = F.rowptr[i]; e < F.rowptr[i + 1] - 1; ++e) s -= Li[F.col[e]] * Li[F.col[e]];
        if (!(s > 0.0)) {
#pragma omp critical
          breakdown = pi;
          s = 1.0;
        }
        Li[i] = std::sqrt(s);
      }
      double *out = &F.val[(size_t)pi * nnz];
      for (int i = 0; i < ns; ++i)
        for (int e = F.rowptr[i]; e < F.rowptr[i + 1]; ++e) {
          out[e] = Ld[(size_t)i * ns + F.col[e]];
          Ld[(size_t)i * ns + F.col[e]] = 0.0;
        }
    }
  }
  if (breakdown >= 0)
    throw std::runtime_error("patch factorisation breakdown (non-positive pivot) in patch " +
                             std::to_string(breakdown));
  // transposed pattern (strictly lower entries grouped by column)
  F.tptr.assign(ns + 1, 0);
  for (int i = 0; i < ns; ++i)
    for (int e = F.rowptr[i]; e < F.rowptr[i + 1] - 1; ++e) F.tptr[F.col[e] + 1]++;
  for (int j = 0; j < ns; ++j) F.tptr[j + 1] += F.tptr[j];
  F.trow.resize(F.tptr[ns]);
  F.tpos.resize(F.tptr[ns]);
  {
    std::vector<int> cur(F.tptr.begin(), F.tptr.end() - 1);
    for (int i = 0; i < ns; ++i)
      for (int e = F.rowptr[i]; e < F.rowptr[i + 1] - 1; ++e) {
        int c = cur[F.col[e]]++;
        F.trow[c] = i;
        F.tpos[c] = e;
      }
  }
  // level schedules
  std::vector<int> lev(ns, 0);
  int nlev = 0;
  for (int i = 0; i < ns; ++i) {
    int l = 0;
    for (int e = F.rowptr[i]; e < F.rowptr[i + 1] - 1; ++e) l = std::max(l, lev[F.col[e]] + 1);
    lev[i] = l;
    nlev = std::max(nlev, l + 1);
  }
  auto bucket = [&](const std::vector<int> &lv, int nl, std::vector<int> &ptr, std::vector<int> &rows) {
    ptr.assign(nl + 1, 0);
    for (int i = 0; i < ns; ++i) ptr[lv[i] + 1]++;
    for (int l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
    rows.assign(ns, 0);
    std::vector<int> cur(ptr.begin(), ptr.end() - 1);
    for (int i = 0; i < ns; ++i) rows[cur[lv[i]]++] = i;
  };
  bucket(lev, nlev, F.flev, F.frows);
  std::vector<int> blv(ns, 0);
  int nbl = 0;
  for (int j = ns - 1; j >= 0; --j) {
    int l = 0;
    for (int e = F.tptr[j]; e < F.tptr[j + 1]; ++e) l = std::max(l, blv[F.trow[e]] + 1);
    blv[j] = l;
    nbl = std::max(nbl, l + 1);
  }
  bucket(blv, nbl, F.blev, F.brows);
  return F;
}

// ---------------------------------------------------------------------------
// coarse space
// ---------------------------------------------------------------------------
// Element matrix of a^k at p = 1 on a trilinear cell (3-point GLL rule).
static void element_p1(int k, const double X8[24], double alpha, double beta,
                       std::vector<double> &A, const Layout &L1) {
  const int nl = L1.nloc;
  Layout L2;
  int nn[3] = {1, 1, 1};
  if (k < 3) L2 = Layout(k + 1, nn, 1);
  std::vector<double> xq, wq;
  gll_rule(3, xq, wq);
  const double h = 1.0 / std::sqrt(2.0);
  auto tab = [&](char ty, int i, double x) {
    if (ty == 'r') return h;
    return i == 0 ? 0.5 * (1.0 - x) : 0.5 * (1.0 + x);
  };
  const double D1[2] = {-h, h};  // p = 1: D-hat = (r_0, s_j')
  A.assign((size_t)nl * nl, 0.0);
  // values of each basis function (and of its reference derivative) at a point
  std::vector<double> val((size_t)nl * 3), dval((size_t)nl * 3);
  for (int q3 = 0; q3 < 3; ++q3)
    for (int q2 = 0; q2 < 3; ++q2)
      for (int q1 = 0; q1 < 3; ++q1) {
        double xi[3] = {xq[q1], xq[q2], xq[q3]};
        double w = wq[q1] * wq[q2] * wq[q3];
        double J[9], Wk[9], Wk1[9];
        jacobian(X8, xi, J);
        form_weight(k, J, Wk);
        form_weight(k + 1, J, Wk1);
        std::fill(val.begin(), val.end(), 0.0);
        std::fill(dval.begin(), dval.end(), 0.0);
        for (int m = 0; m < L1.ncomp; ++m)
          for (int i3 = 0; i3 < L1.ld[m][2]; ++i3)
            for (int i2 = 0; i2 < L1.ld[m][1]; ++i2)
              for (int i1 = 0; i1 < L1.ld[m][0]; ++i1) {
                int b = L1.loff[m] + i1 + L1.ld[m][0] * (i2 + L1.ld[m][1] * i3);
                int ii[3] = {i1, i2, i3};
                double v = 1.0;
                for (int d = 0; d < 3; ++d) v *= tab(L1.t[m][d], ii[d], xi[d]);
                val[3 * b + (L1.ncomp == 1 ? 0 : m)] = v;
                // d^k of this basis function: D-hat maps s-index i_d to the r-index 0
                for (int t = 0; t < L2.ncomp; ++t)
                  for (int s = 0; s < kNumTerms[k][t]; ++s) {
                    const DTerm &T = kTerms[k][t][s];
                    if (T.src != m) continue;
                    double dv = T.sgn * D1[ii[T.dir]];
                    for (int d = 0; d < 3; ++d)
                      dv *= (d == T.dir) ? h : tab(L2.t[t][d], ii[d], xi[d]);
                    dval[3 * b + (L2.ncomp == 1 ? 0 : t)] += dv;
                  }
              }
        const int c0 = L1.ncomp == 1 ? 1 : 3, c1 = L2.ncomp == 1 ? 1 : 3;
        for (int a = 0; a < nl; ++a)
          for (int b = 0; b < nl; ++b) {
            double s = 0.0;
            for (int x = 0; x < c0; ++x)
              for (int y = 0; y < c0; ++y) s += beta * val[3 * a + x] * Wk[3 * x + y] * val[3 * b + y];
            for (int x = 0; x < c1; ++x)
              for (int y = 0; y < c1; ++y) s += alpha * dval[3 * a + x] * Wk1[3 * x + y] * dval[3 * b + y];
            A[(size_t)a * nl + b] += w * s;
          }
      }
}

// Triplets of A_0 (a^k at p = 1, Sec. 4.3) over the coarse free DOFs.
static std::vector<Trip> coarse_triplets(const Layout &Lf, const Layout &Lc, const FreeMap &fc,
                                         const Geometry &geo, const double *alpha,
                                         const double *beta) {
  const int k = Lf.k;
  const int ncell = Lf.n[0] * Lf.n[1] * Lf.n[2];
  std::vector<Trip> t;
  std::vector<double> AK;
  for (int c = 0; c < ncell; ++c) {
    int e[3] = {c % Lf.n[0], (c / Lf.n[0]) % Lf.n[1], c / (Lf.n[0] * Lf.n[1])};
    double X8[24];
    geo.cell_vertices(e[0], e[1], e[2], X8);
    element_p1(k, X8, alpha[c], beta[c], AK, Lc);
    std::vector<int> l2f(Lc.nloc);
    for (int m = 0; m < Lc.ncomp; ++m)
      for (int i3 = 0; i3 < Lc.ld[m][2]; ++i3)
        for (int i2 = 0; i2 < Lc.ld[m][1]; ++i2)
          for (int i1 = 0; i1 < Lc.ld[m][0]; ++i1)
            l2f[Lc.loff[m] + i1 + Lc.ld[m][0] * (i2 + Lc.ld[m][1] * i3)] =
                fc.lat2free[Lc.index(m, e[0] + i1, e[1] + i2, e[2] + i3)];
    for (int a = 0; a < Lc.nloc; ++a)
      for (int b = 0; b < Lc.nloc; ++b)
        if (l2f[a] >= 0 && l2f[b] >= 0) t.push_back({l2f[a], l2f[b], AK[(size_t)a * Lc.nloc + b]});
  }
  return t;
}

// R_0 (coarse free rows, fine lattice columns): closed-form injection
// coefficients per direction (dual functionals of Eq. fdmdualbasis applied
// to the p = 1 basis).
static void restriction_R0(const Layout &Lf, const Layout &Lc, const FreeMap &fc, CoarseData &C) {
  const int p = Lf.p;
  Basis1D B(p);
  std::vector<Trip> t;
  FreeMap ff(Lf);
  for (int f = 0; f < (int)ff.free2lat.size(); ++f) {
    long long lat = ff.free2lat[f];
    int m;
    long long g[3];
    Lf.coords(lat, m, g);
    long long ci[3][2];
    double cv[3][2];
    int cn[3];
    bool zero = false;
    for (int d = 0; d < 3; ++d) {
      long long e = g[d] / p;
      int i = (int)(g[d] % p);
      if (Lf.t[m][d] == 's') {
        if (i == 0) { ci[d][0] = e; cv[d][0] = 1.0; cn[d] = 1; }
        else {
          ci[d][0] = e; cv[d][0] = B.Js[i * 2 + 0];
          ci[d][1] = e + 1; cv[d][1] = B.Js[i * 2 + 1];
          cn[d] = 2;
        }
      } else {
        if (i != 0) { zero = true; break; }
        ci[d][0] = e; cv[d][0] = 1.0; cn[d] = 1;
      }
    }
    if (zero) continue;
    for (int a3 = 0; a3 < cn[2]; ++a3)
      for (int a2 = 0; a2 < cn[1]; ++a2)
        for (int a1 = 0; a1 < cn[0]; ++a1) {
          double v = cv[0][a1] * cv[1][a2] * cv[2][a3];
          if (v == 0.0) continue;
          int cf = fc.lat2free[Lc.index(m, ci[0][a1], ci[1][a2], ci[2][a3])];
          if (cf < 0) continue;
          t.push_back({cf, (int)lat, v});
        }
  }
  C.R0 = csr_from_triplets(C.nc, (int)Lf.size, t);
  C.R0T = transpose(C.R0);
}

// Dense SPD inverse by Cholesky (n x n row-major), OpenMP over columns.
static std::vector<double> dense_spd_inverse(std::vector<double> Lm, int nc) {
  for (int j = 0; j < nc; ++j) {
    double d = Lm[(size_t)j * nc + j];
    for (int kk = 0; kk < j; ++kk) d -= Lm[(size_t)j * nc + kk] * Lm[(size_t)j * nc + kk];
    if (!(d > 0)) throw std::runtime_error("coarse matrix not SPD");
    d = std::sqrt(d);
    Lm[(size_t)j * nc + j] = d;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < nc; ++i) {
      double s = Lm[(size_t)i * nc + j];
      for (int kk = 0; kk < j; ++kk) s -= Lm[(size_t)i * nc + kk] * Lm[(size_t)j * nc + kk];
      Lm[(size_t)i * nc + j] = s / d;
    }
  }
  // Y = L^-1 stored transposed (row c of Yt = column c of Y), so both the
  // substitution and the product A^-1 = Y^T Y run over contiguous rows.
  std::vector<double> Yt((size_t)nc * nc, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int c = 0; c < nc; ++c) {
    double *y = &Yt[(size_t)c * nc];
    for (int i = c; i < nc; ++i) {
      const double *Li = &Lm[(size_t)i * nc];
      double s = (i == c) ? 1.0 : 0.0;
      for (int kk = c; kk < i; ++kk) s -= Li[kk] * y[kk];
      y[i] = s / Li[i];
    }
  }
  std::vector<double>().swap(Lm);
  std::vector<double> inv((size_t)nc * nc, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int a = 0; a < nc; ++a) {
    const double *ya = &Yt[(size_t)a * nc];
    for (int b = 0; b <= a; ++b) {
      const double *yb = &Yt[(size_t)b * nc];
      double s = 0.0;
      for (int i = a; i < nc; ++i) s += ya[i] * yb[i];
      inv[(size_t)a * nc + b] = s;
      inv[(size_t)b * nc + a] = s;
    }
  }
  return inv;
}

CoarseData build_coarse(const Layout &Lf, const Geometry &geo, const double *alpha,
                        const double *beta) {
  CoarseData C;
  Layout Lc(Lf.k, Lf.n, 1, Lf.natural);
  FreeMap fc(Lc);
  const int nc = (int)fc.free2lat.size();
  C.nc = nc;
  if (nc > 16384)
    throw std::runtime_error("coarse space too large for the dense coarse solve (> 16384 DOFs): "
                             "use RM_COARSE_GMG");
  std::vector<double> A0((size_t)nc * nc, 0.0);
  std::vector<Trip> t = coarse_triplets(Lf, Lc, fc, geo, alpha, beta);
  for (const Trip &x : t) A0[(size_t)x.r * nc + x.c] += x.v;
  C.A0inv = dense_spd_inverse(A0, nc);
  C.A0 = csr_from_triplets(nc, nc, t);
  C.free2lat = fc.free2lat;
  restriction_R0(Lf, Lc, fc, C);
  return C;
}

// Sparse product A B (rows of A, columns of B).
static Csr spgemm(const Csr &A, const Csr &B) {
  std::vector<Trip> t;
  std::vector<double> acc(B.ncols, 0.0);
  std::vector<char> m(B.ncols, 0);
  std::vector<int> touched;
  for (int i = 0; i < A.nrows; ++i) {
    touched.clear();
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      const int j = A.col[e];
      for (int64_t f = B.ptr[j]; f < B.ptr[j + 1]; ++f) {
        const int c = B.col[f];
        if (!m[c]) { m[c] = 1; acc[c] = 0.0; touched.push_back(c); }
        acc[c] += A.val[e] * B.val[f];
      }
    }
    for (int c : touched) { t.push_back({i, c, acc[c]}); m[c] = 0; }
  }
  return csr_from_triplets(A.nrows, B.ncols, t);
}

// 1 / diag(M) / ||diag(M)^-1 M||_inf: damped Jacobi weights
static std::vector<double> jacobi_weights(const Csr &M, const char *what) {
  std::vector<double> dinv(M.nrows);
  double norm = 0.0;
  for (int i = 0; i < M.nrows; ++i) {
    double diag = 0.0, rs = 0.0;
    for (int64_t e = M.ptr[i]; e < M.ptr[i + 1]; ++e) {
      rs += std::fabs(M.val[e]);
      if (M.col[e] == i) diag = M.val[e];
    }
    if (!(diag > 0)) throw std::runtime_error(std::string(what) + ": non-positive diagonal");
    dinv[i] = 1.0 / diag;
    norm = std::max(norm, rs / diag);
  }
  for (double &v : dinv) v /= norm;
  return dinv;
}

// M with rows and columns renumbered by rmap / cmap (lattice -> compact, -1
// dropped), nrows x ncols
static Csr compact_csr(const Csr &M, const std::vector<int> &rmap, const std::vector<int> &cmap, int nrows,
                       int ncols) {
  std::vector<Trip> t;
  for (int i = 0; i < M.nrows; ++i) {
    if (rmap[i] < 0) continue;
    for (int64_t e = M.ptr[i]; e < M.ptr[i + 1]; ++e)
      if (cmap[M.col[e]] >= 0) t.push_back({rmap[i], cmap[M.col[e]], M.val[e]});
  }
  return csr_from_triplets(nrows, ncols, t);
}

CoarseData build_coarse_gmg(const Layout &Lf, const Geometry &geo, const double *alpha,
                            const double *beta, CoarseGMG &mg, bool hiptmair) {
  CoarseData C;
  const int k = Lf.k;
  Layout Lc(k, Lf.n, 1, Lf.natural);
  FreeMap fc(Lc);
  C.nc = (int)fc.free2lat.size();
  std::vector<Trip> t = coarse_triplets(Lf, Lc, fc, geo, alpha, beta);
  Csr A = csr_from_triplets(C.nc, C.nc, t);
  restriction_R0(Lf, Lc, fc, C);
  C.A0 = A;
  C.free2lat = fc.free2lat;
  mg = CoarseGMG();
  mg.hiptmair = hiptmair && k >= 1;
  int n[3] = {Lf.n[0], Lf.n[1], Lf.n[2]};
  Layout L = Lc;
  FreeMap fm = fc;
  while (true) {
    const bool can = n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0 && n[0] >= 4 && n[1] >= 4 &&
                     n[2] >= 4 && A.nrows > 512;
    if (!can) break;
    int nh[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    Layout Lh(k, nh, 1, Lf.natural);
    FreeMap fh(Lh);
    // P: level l+1 (mesh nh) -> level l (mesh n), per direction
    // s-type: fine index g from coarse g/2 (even) or (g-1)/2, (g+1)/2 with 1/2
    // r-type: fine cell g from coarse cell g/2 with weight 1/2
    std::vector<Trip> pt;
    for (int f = 0; f < (int)fm.free2lat.size(); ++f) {
      int m;
      long long g[3];
      L.coords(fm.free2lat[f], m, g);
      long long ci[3][2];
      double cv[3][2];
      int cn[3];
      for (int d = 0; d < 3; ++d) {
        if (L.t[m][d] == 's') {
          if (g[d] % 2 == 0) { ci[d][0] = g[d] / 2; cv[d][0] = 1.0; cn[d] = 1; }
          else { ci[d][0] = (g[d] - 1) / 2; ci[d][1] = (g[d] + 1) / 2; cv[d][0] = cv[d][1] = 0.5; cn[d] = 2; }
        } else {
          ci[d][0] = g[d] / 2; cv[d][0] = 0.5; cn[d] = 1;
        }
      }
      for (int a3 = 0; a3 < cn[2]; ++a3)
        for (int a2 = 0; a2 < cn[1]; ++a2)
          for (int a1 = 0; a1 < cn[0]; ++a1) {
            int cf = fh.lat2free[Lh.index(m, ci[0][a1], ci[1][a2], ci[2][a3])];
            if (cf < 0) continue;
            pt.push_back({f, cf, cv[0][a1] * cv[1][a2] * cv[2][a3]});
          }
    }
    Csr P = csr_from_triplets((int)fm.free2lat.size(), (int)fh.free2lat.size(), pt);
    Csr PT = transpose(P);
    Csr Ah = spgemm(PT, spgemm(A, P));
    // smoother weights
    mg.A.push_back(A);
    mg.P.push_back(P);
    mg.PT.push_back(PT);
    mg.dinv.push_back(jacobi_weights(A, "coarse multigrid"));
    if (mg.hiptmair) {
      // Hiptmair-Jacobi: the level's lowest-order d^{k-1} from the potential
      // space V^{k-1}_{h,1} and the Jacobi weights of B = G^T A G
      Layout L0(k - 1, n, 1, Lf.natural);
      FreeMap f0(L0);
      Csr D = discrete_derivative(L0, L, fm.free2lat, f0.free2lat);
      Csr G = compact_csr(D, fm.lat2free, f0.lat2free, (int)fm.free2lat.size(), (int)f0.free2lat.size());
      Csr GT = transpose(G);
      Csr B = spgemm(GT, spgemm(A, G));
      mg.dinvB.push_back(jacobi_weights(B, "coarse multigrid potential"));
      mg.G.push_back(std::move(G));
      mg.GT.push_back(std::move(GT));
    } else if (k >= 1) {
      // vertex stars of the level (exact, block inverses); slot maps renumbered
      // to the level's compact free numbering
      PatchFamily F = build_patches(L, fm, A, 0, false, 0);
      for (int &s : F.slotmap)
        if (s >= 0) s = fm.lat2free[s];
      mg.star.push_back(std::move(F));
    }
    A = Ah;
    L = Lh;
    fm = fh;
    for (int d = 0; d < 3; ++d) n[d] = nh[d];
  }
  mg.levels = (int)mg.A.size();
  mg.ncoarsest = A.nrows;
  if (mg.ncoarsest > 8192) throw std::runtime_error("coarse multigrid: coarsest level too large");
  std::vector<double> dense((size_t)A.nrows * A.nrows, 0.0);
  for (int i = 0; i < A.nrows; ++i)
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) dense[(size_t)i * A.nrows + A.col[e]] += A.val[e];
  mg.Ainv = dense_spd_inverse(dense, A.nrows);
  mg.A.push_back(A);
  return C;
}

Csr discrete_derivative(const Layout &La, const Layout &Lb, const std::vector<int> &rows,
                        const std::vector<int> &cols) {
  const int p = La.p, kk = La.k;
  if (kk < 0 || kk > 2 || Lb.k != kk + 1) throw std::runtime_error("discrete_derivative: V^k -> V^{k+1}");
  Basis1D B(p);
  std::vector<char> okc(La.size, 0);
  for (int c : cols) okc[c] = 1;
  std::vector<Trip> t;
  for (int r : rows) {
    int m;
    long long g[3];
    Lb.coords(r, m, g);
    // target component m of V^{k+1}: each term reads source component src,
    // s-type along dr where the target is r-type, equal in the other directions
    for (int s = 0; s < kNumTerms[kk][m]; ++s) {
      const DTerm &T = kTerms[kk][m][s];
      const long long e = g[T.dir] / p;
      const int i = (int)(g[T.dir] % p);
      for (int l = 0; l <= p; ++l) {
        const double v = B.D[i * (p + 1) + l];
        if (v == 0.0) continue;
        long long h[3] = {g[0], g[1], g[2]};
        h[T.dir] = e * p + l;
        const long long c = La.index(T.src, h[0], h[1], h[2]);
        if (!okc[c]) continue;
        t.push_back({r, (int)c, T.sgn * v});
      }
    }
  }
  return csr_from_triplets((int)Lb.size, (int)La.size, t);
}

Csr discrete_gradient(const Layout &L0, const Layout &L1, const std::vector<int> &rows1,
                      const std::vector<int> &cols0) {
  return discrete_derivative(L0, L1, rows1, cols0);
}

Csr mass_v3(const Layout &L3, const Geometry &geo, const double *coef) {
  if (L3.k != 3) throw std::runtime_error("mass_v3: a V^3 layout");
  const int p = L3.p, q = quad_points(p);
  Basis1D B(p);
  std::vector<double> xq, wq;
  gll_rule(q, xq, wq);
  std::vector<double> R(q * p);  // R[o * p + i] = r_i(x_o)
  B.tab_r(xq.data(), q, R.data());
  const int n0 = L3.n[0], n1 = L3.n[1], n2 = L3.n[2];
  const int ncell = n0 * n1 * n2, nl = p * p * p;
  std::vector<std::vector<Trip>> parts(ncell);
  int inverted = -1;  // an inverted cell, reported after the parallel region
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8)
#endif
  for (int c = 0; c < ncell; ++c) {
    const int e0 = c % n0, e1 = (c / n0) % n1, e2 = c / (n0 * n1);
    bool bad = false;
    double X8[24];
    geo.cell_vertices(e0, e1, e2, X8);
    // weight per point: w / det J (the 3-form pullback) times the coefficient
    std::vector<double> W(q * q * q);
    for (int a3 = 0; a3 < q; ++a3)
      for (int a2 = 0; a2 < q; ++a2)
        for (int a1 = 0; a1 < q; ++a1) {
          const double xi[3] = {xq[a1], xq[a2], xq[a3]};
          double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          for (int cn = 0; cn < 8; ++cn) {
            const int c1 = cn & 1, c2 = (cn >> 1) & 1, c3 = cn >> 2;
            const double N[3] = {c1 ? 0.5 * (1 + xi[0]) : 0.5 * (1 - xi[0]),
                                 c2 ? 0.5 * (1 + xi[1]) : 0.5 * (1 - xi[1]),
                                 c3 ? 0.5 * (1 + xi[2]) : 0.5 * (1 - xi[2])};
            const double dN[3] = {c1 ? 0.5 : -0.5, c2 ? 0.5 : -0.5, c3 ? 0.5 : -0.5};
            const double g[3] = {dN[0] * N[1] * N[2], N[0] * dN[1] * N[2], N[0] * N[1] * dN[2]};
            for (int r = 0; r < 3; ++r)
              for (int d = 0; d < 3; ++d) J[3 * r + d] += X8[3 * cn + r] * g[d];
          }
          const double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                             J[2] * (J[3] * J[7] - J[4] * J[6]);
          if (!(det > 0)) bad = true;
          W[a1 + q * (a2 + q * a3)] = wq[a1] * wq[a2] * wq[a3] * coef[c] / det;
        }
    if (bad) {
#ifdef _OPENMP
#pragma omp critical(rm_mass_v3_inverted)
#endif
      inverted = c;
      continue;
    }
    std::vector<Trip> &t = parts[c];
    for (int i3 = 0; i3 < p; ++i3)
      for (int i2 = 0; i2 < p; ++i2)
        for (int i1 = 0; i1 < p; ++i1)
          for (int j3 = 0; j3 < p; ++j3)
            for (int j2 = 0; j2 < p; ++j2)
              for (int j1 = 0; j1 < p; ++j1) {
                double v = 0.0;
                for (int a3 = 0; a3 < q; ++a3)
                  for (int a2 = 0; a2 < q; ++a2) {
                    const double f = R[a3 * p + i3] * R[a3 * p + j3] * R[a2 * p + i2] * R[a2 * p + j2];
                    for (int a1 = 0; a1 < q; ++a1)
                      v += f * R[a1 * p + i1] * R[a1 * p + j1] * W[a1 + q * (a2 + q * a3)];
                  }
                const long long gi = L3.index(0, (long long)e0 * p + i1, (long long)e1 * p + i2, (long long)e2 * p + i3);
                const long long gj = L3.index(0, (long long)e0 * p + j1, (long long)e1 * p + j2, (long long)e2 * p + j3);
                t.push_back({(int)gi, (int)gj, v});
              }
  }
  (void)nl;
  if (inverted >= 0) throw std::runtime_error("mass_v3: inverted cell " + std::to_string(inverted));
  std::vector<Trip> all;
  for (auto &pt : parts) all.insert(all.end(), pt.begin(), pt.end());
  return csr_from_triplets((int)L3.size, (int)L3.size, all);
}

}  // namespace rm
