// Host FP64 setup of the Riesz-map solvers: lattice layout, auxiliary
// operator, static condensation, patch factors, coarse space.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "host_basis.h"

namespace rm {

// Per-component lattice of V^k (k = 0..3) on an n1 x n2 x n3 mesh, Sec. 2.4.
struct Layout {
  int k = 0, p = 0, n[3] = {0, 0, 0}, ncomp = 0;
  char t[3][3] = {};       // 's' / 'r' per component and direction
  long long N[3][3] = {};  // lattice points per component and direction
  long long off[4] = {};   // component offsets
  int ld[3][3] = {};       // local (cell) dims
  int loff[4] = {};
  long long size = 0;
  int nloc = 0;
  // Gamma_D empty (natural boundary conditions everywhere): no entry is
  // Dirichlet; otherwise Gamma_D is the whole boundary of the cube
  bool natural = false;
  Layout() = default;
  Layout(int k, const int n[3], int p, bool natural = false);
  long long index(int m, long long g1, long long g2, long long g3) const {
    return off[m] + g1 + N[m][0] * (g2 + N[m][1] * g3);
  }
  bool dirichlet(int m, const long long g[3]) const {
    if (natural) return false;
    for (int d = 0; d < 3; ++d)
      if (t[m][d] == 's' && (g[d] == 0 || g[d] == (long long)n[d] * p)) return true;
    return false;
  }
  // decode a lattice index
  void coords(long long idx, int &m, long long g[3]) const;
};

struct Csr {
  int nrows = 0, ncols = 0;
  std::vector<int64_t> ptr;
  std::vector<int> col;
  std::vector<double> val;
  int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

struct Trip {
  int r, c;
  double v;
};
// Sums duplicates; columns sorted within rows.
Csr csr_from_triplets(int nrows, int ncols, std::vector<Trip> &t);
Csr transpose(const Csr &A);

struct Geometry {
  int n[3];
  std::vector<double> X;  // (n1+1)(n2+1)(n3+1) x 3
  void cell_vertices(int e1, int e2, int e3, double out[24]) const;
};

struct FreeMap {
  std::vector<int> lat2free;  // -1 for Dirichlet
  std::vector<int> free2lat;
  explicit FreeMap(const Layout &L);
  FreeMap() = default;
};

// Sparse auxiliary operator P (Sec. 3.2, Eq. sum-factorization_approx) on
// the free DOFs, with mass coefficient mcoef and derivative coefficient
// scoef per cell.
Csr assemble_aux(const Layout &L, const Geometry &geo, const double *mcoef,
                 const double *scoef, const FreeMap &fm);

// Interior / interface split and Schur complement (Eqs. LDU, schur).
struct Condensed {
  std::vector<int> I, G;   // free indices
  Csr Binv;                // P_II^{-1}, free x free (rows in I)
  Csr E;                   // P_GI P_II^{-1}, free x free (rows in G, cols in I)
  Csr Et;                  // E^T (rows in I, cols in G)
  Csr S;                   // interface Schur complement, free x free (rows/cols in G)
};
Condensed condense(const Layout &L, const FreeMap &fm, const Csr &P);

// A family of patches sharing one slot template (stars of one entity kind).
struct PatchFamily {
  int nslots = 0, npatch = 0;
  std::vector<int> slotmap;           // npatch x nslots lattice indices, -1 = absent
  std::vector<int> rowptr, col;       // template lower pattern, diagonal last per row
  std::vector<int> tptr, trow, tpos;  // transposed pattern: strictly-lower entries by column
  std::vector<int> flev, frows;       // forward level schedule (level ptr, rows)
  std::vector<int> blev, brows;       // backward level schedule
  std::vector<double> val;            // npatch x nnz
  int nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
  // Block-inverse form (exact factorisation only): the template pattern
  // splits into decoupled blocks; each patch stores the dense inverse of
  // every block (column-major, nb x nb), applied as one parallel product.
  int inverse = 0;
  std::vector<int> bptr;              // block b = positions bptr[b]..bptr[b+1]
  std::vector<int> pos_slot;          // slot at position t (blocks contiguous)
  std::vector<int> pos_blk;           // block of position t
  std::vector<int> boff;              // value offset of block b within a patch
  std::vector<double> ival;           // npatch x boff.back()
  int ivals() const { return boff.empty() ? 0 : boff.back(); }
  // The values the device kernels read: the block inverses, or the
  // triangular factor with every diagonal entry replaced by its reciprocal.
  std::vector<double> device_values() const {
    if (inverse) return ival;
    std::vector<double> v = val;
    const int nz = nnz();
    for (int pi = 0; pi < npatch; ++pi)
      for (size_t i = 0; i + 1 < rowptr.size(); ++i) {
        double &d = v[(size_t)pi * nz + rowptr[i + 1] - 1];
        d = 1.0 / d;
      }
    return v;
  }
};
// span: bit d set = the entity spans direction d (0: vertex, 1 bit: edge, ...)
// interface_only: slots restricted to interface DOFs (static condensation).
// factor: 0 exact Cholesky, 1 ICC(0) on the patch matrix pattern.
PatchFamily build_patches(const Layout &L, const FreeMap &fm, const Csr &M,
                          int span, bool interface_only, int factor);

// p = 1 coarse space (Sec. 4.3): restriction R_0 (coarse free x fine
// lattice) and the dense inverse of the rediscretised A_0.
struct CoarseData {
  int nc = 0;
  Csr R0;    // rows: coarse free, cols: fine lattice index
  Csr R0T;   // rows: fine lattice index (only free), cols: coarse free
  std::vector<double> A0inv;
  Csr A0;                      // the p = 1 operator on the coarse free DOFs
  std::vector<int> free2lat;   // coarse free index -> coarse lattice index
};
CoarseData build_coarse(const Layout &Lf, const Geometry &geo, const double *alpha,
                        const double *beta);

// Multigrid hierarchy for the p = 1 coarse problem when it is too large for
// a dense inverse: level 0 is A_0 (sparse); level l+1 is the Galerkin
// product P^T A_l P with the lowest-order refinement P from the mesh n_l/2 to
// n_l (hat weights along s-type directions, 1/2 per r-type direction);
// damped point Jacobi (omega = 1 / ||D^-1 A||_inf) pre- and post-smoothing;
// dense inverse on the coarsest level.
struct CoarseGMG {
  int levels = 0;               // smoothed levels; level `levels` is solved densely
  std::vector<Csr> A;           // A[l], compact free numbering of level l
  std::vector<Csr> P, PT;       // P[l]: level l+1 -> level l
  std::vector<std::vector<double>> dinv;  // omega / diag(A_l)  (k = 0)
  // k = 1, 2: additive vertex-star smoother omega sum_v R_v^T A_v^-1 R_v with
  // omega = 1/8 (at most 8 stars overlap a DOF); slot maps in the level's
  // compact numbering
  std::vector<PatchFamily> star;
  double star_omega = 0.125;
  // k = 1, 2 with the Hiptmair-Jacobi smoother: per level the lowest-order
  // discrete gradient / curl G (level free x potential free), G^T, and the
  // damped Jacobi weights of the potential operator B = G^T A G
  bool hiptmair = false;
  std::vector<Csr> G, GT;
  std::vector<std::vector<double>> dinvB;
  std::vector<double> Ainv;     // coarsest dense inverse
  int ncoarsest = 0;
};
// R_0 and the multigrid hierarchy of the coarse problem.  hiptmair (k = 1,
// 2): Hiptmair-Jacobi smoothing data instead of the vertex stars.
CoarseData build_coarse_gmg(const Layout &Lf, const Geometry &geo, const double *alpha,
                            const double *beta, CoarseGMG &mg, bool hiptmair = false);

// Discrete exterior derivative d^k: V^k (La) -> V^{k+1} (Lb) in FDM
// coefficients (cellwise D-hat, Sec. 2.3), restricted to the given rows
// (V^{k+1} lattice ids) and columns (V^k lattice ids).
Csr discrete_derivative(const Layout &La, const Layout &Lb, const std::vector<int> &rows,
                        const std::vector<int> &cols);
// H(div) SC-PH potential operator: (curl phi, beta curl psi) + eps (phi, beta
// psi), eps = the small mass multiple the paper adds to its singular patch
// matrices (Remark after Eq. ph); 1e-2, iteration counts flat for eps in
// [1e-4, 1e-1].
constexpr double kHdivPotentialEps = 1e-2;
// Discrete gradient V^0 -> V^1 restricted to free rows/cols (lattice ids).
Csr discrete_gradient(const Layout &L0, const Layout &L1, const std::vector<int> &rows1,
                      const std::vector<int> &cols0);

// Mass matrix of V^3 (DQ_{p-1}, the FDM r-basis, Sec. 2.4) with the 3-form
// pullback weight 1/det J and a per-cell coefficient, by the GLL rule of
// quad_points(p): block diagonal (every entry lives in one cell), rows and
// columns lattice indices of L3 (k = 3).
Csr mass_v3(const Layout &L3, const Geometry &geo, const double *coef);

// Quadrature points per direction: ceil(3(p+1)/2) (Sec. 5).
inline int quad_points(int p) { return (3 * (p + 1) + 1) / 2; }

}  // namespace rm
