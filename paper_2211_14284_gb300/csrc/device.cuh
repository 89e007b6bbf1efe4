// Device-side data structures shared by the kernels and the C ABI.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace rmd {

// general-cell apply: 512 threads, two CTAs (32 warps) per SM to hide the
// shared-memory latency of the contraction chains
constexpr int kApplyThreadsGeneral = 512;

// Operator apply (Eq. sum-factorization) on trilinear cells.
struct ApplyDev {
  int k, p, q;
  int n[3];
  int nc0, nc1;            // components of V^k and V^{k+1}
  int N[3][3];             // lattice dims of V^k per component
  long long off[3];        // component offsets of V^k
  int ld0[3][3], loff0[4]; // local dims of V^k
  int ld1[3][3], loff1[4]; // local dims of V^{k+1}
  char t0[3][3], t1[3][3];
  int nloc0, nloc1;
  const double *X;         // vertices, 3 per vertex
  const double *alpha, *beta;
  const double *tabs;      // Ts q(p+1) | Tr qp | D1 p(p+1) | xq q | wq q | reflection-split
                           // tables of Ts then Tr (eo_tables; general cells)
  const void *G;           // pullback weights per cell and point (metric_kernel),
                           // in the general apply's number type (double-float)
  int nA, nAB;             // entries of stage A, of both stages (1 or 6 each)
  // Cartesian fast path (every cell an axis-aligned box): the 1D factors
  // of B-hat (a = B_00 = B_pp, b = B_0p)
  int cartesian;
  double bh_a, bh_b;
  double *Y;               // unassembled cell products, [component][cell][local entry] (Cartesian apply)
  const double *ccoef;     // per cell: beta x box metric of V^k (3), alpha x box metric
                           // of V^{k+1} (3), 2 unused (Cartesian apply; setup-time FP64)
  int prob;                // batched solves: the problem's index
  int arith;               // number type of the apply: 0 double, 1 double-float (DF)
  int natural;             // 1: Gamma_D empty (no Dirichlet entries)
  const int *done = nullptr;  // batched solves: convergence flags (problem prob skipped
                              // by the Cartesian apply once set; its y entries are 0)
  int asm_grid = 0;        // CTAs of the Cartesian assembly (0: 8 per SM)
};

// s-type test of component m of V^kk in direction d (Sec. 2.4): H(grad) all
// s; NCE component m r-type along m; NCF component m s-type along m only.
__host__ __device__ constexpr bool styp(int kk, int m, int d) {
  return kk == 0 ? true : (kk == 3 ? false : (kk == 1 ? d != m : d == m));
}
__host__ __device__ constexpr int ncomp(int kk) { return (kk == 0 || kk == 3) ? 1 : 3; }

// Reflection split of a 1D tabulation T (q points x n functions, row-major)
// at the symmetric GLL points x_{q-1-o} = -x_o.  Each function reflects
// into plus or minus itself or one partner (the interface pair), so
//   E[o][i] = (T[o][i] + T[q-1-o][i]) / 2   (o < he = ceil(q/2)),
//   Od[o][i] = (T[o][i] - T[q-1-o][i]) / 2  (o < ho = floor(q/2))
// vanish for whole columns (odd functions in E, even ones in Od).  Then
//   T u at o and q-1-o = E u +- Od u       (forward: n + 2 FMAs per pair
//                                            of points instead of 2n),
//   T^T w = E^T w+ + Od^T w-,  w+- = w_o +- w_{q-1-o}  (backward).
// Header per table (kEoHeader ints): n, he, ho, nse, nso, double offset,
// se[16] (columns with an even part), so[16] (with an odd part), fl[16]
// (bit 0 even, bit 1 odd).  Doubles: Ec[he][nse], Oc[ho][nso] (compressed
// columns), ET[n][he], OT[n][ho].
constexpr int kEoHeader = 6 + 3 * 16;

// The column lists follow from the parity of the FDM bases under x -> -x:
// the s-type interface pair {0, p} swaps (s_p(x) = s_0(-x), both parts
// present), the interior s_j is even for odd j and odd for even j, and r_i
// is even for even i.  The general apply takes the lists as compile-time
// constants for 1 <= p <= kMaxGeneralP; eo_rule_holds() checks the host
// tables against them.
constexpr int kMaxGeneralP = 8;
__host__ __device__ constexpr int quad_q(int p) { return (3 * (p + 1) + 1) / 2; }
__host__ __device__ constexpr int eo_n(bool s, int p) { return s ? p + 1 : p; }
__host__ __device__ constexpr int eo_nse(bool s, int p) { return s ? 2 + p / 2 : (p + 1) / 2; }
__host__ __device__ constexpr int eo_nso(bool s, int p) { return s ? 2 + (p - 1) / 2 : p / 2; }
// k-th column with an even (se) or odd (so) part
__host__ __device__ constexpr int eo_se(bool s, int p, int k) {
  return s ? (k == 0 ? 0 : (k == eo_nse(s, p) - 1 ? p : 2 * k - 1)) : 2 * k;
}
__host__ __device__ constexpr int eo_so(bool s, int p, int k) {
  return s ? (k == 0 ? 0 : (k == eo_nso(s, p) - 1 ? p : 2 * k)) : 2 * k + 1;
}
__host__ __device__ constexpr int eo_fl(bool s, int p, int i) {
  return s ? ((i == 0 || i == p) ? 3 : ((i & 1) ? 1 : 2)) : ((i & 1) ? 2 : 1);
}
// doubles of one table (Ec, Oc, ET, OT)
__host__ __device__ constexpr int eo_size(bool s, int p) {
  return ((quad_q(p) + 1) / 2) * (eo_nse(s, p) + eo_n(s, p)) + (quad_q(p) / 2) * (eo_nso(s, p) + eo_n(s, p));
}
// The host tables (s-type header then r-type header, doubles dbl) match the
// rule, and the interface pair has E[o][p] = E[o][0], Od[o][p] = -Od[o][0].
inline bool eo_rule_holds(int p, const std::vector<int> &hdr, const std::vector<double> &dbl) {
  if (p < 1 || p > kMaxGeneralP || (int)hdr.size() != 2 * kEoHeader) return false;
  const int q = quad_q(p), he = (q + 1) / 2, ho = q / 2;
  for (int t = 0; t < 2; ++t) {
    const bool s = t == 0;
    const int *h = hdr.data() + t * kEoHeader;
    if (h[0] != eo_n(s, p) || h[1] != he || h[2] != ho || h[3] != eo_nse(s, p) || h[4] != eo_nso(s, p) ||
        h[5] != (s ? 0 : eo_size(true, p)))
      return false;
    for (int k = 0; k < h[3]; ++k)
      if (h[6 + k] != eo_se(s, p, k)) return false;
    for (int k = 0; k < h[4]; ++k)
      if (h[22 + k] != eo_so(s, p, k)) return false;
    for (int i = 0; i < h[0]; ++i)
      if (h[38 + i] != eo_fl(s, p, i)) return false;
  }
  if ((int)dbl.size() != eo_size(true, p) + eo_size(false, p)) return false;
  const int n = p + 1, oET = he * eo_nse(true, p) + ho * eo_nso(true, p), oOT = oET + n * he;
  double tmax = 0.0;
  for (double v : dbl) tmax = v > tmax ? v : (-v > tmax ? -v : tmax);
  const double tol = 1e-13 * tmax;
  for (int o = 0; o < he; ++o) {
    const double d = dbl[oET + p * he + o] - dbl[oET + o];
    if (d > tol || -d > tol) return false;
  }
  for (int o = 0; o < ho; ++o) {
    const double d = dbl[oOT + p * ho + o] + dbl[oOT + o];
    if (d > tol || -d > tol) return false;
  }
  return true;
}

// Shared memory of the general apply (doubles): both split tables, D-hat
// and its transpose, the V^k and V^{k+1} cell blocks (input, output), the
// point values (3 components) and the two staging buffers.
__host__ __device__ constexpr int general_smem_doubles(int k, int p) {
  return eo_size(true, p) + eo_size(false, p) + 2 * p * (p + 1) +
         2 * ncomp(k) * (styp(k, 0, 0) ? p + 1 : p) * (styp(k, 0, 1) ? p + 1 : p) * (styp(k, 0, 2) ? p + 1 : p) +
         2 * ncomp(k + 1) * (styp(k + 1, 0, 0) ? p + 1 : p) * (styp(k + 1, 0, 1) ? p + 1 : p) *
             (styp(k + 1, 0, 2) ? p + 1 : p) +
         3 * quad_q(p) * quad_q(p) * quad_q(p) + quad_q(p) * (p + 1) * (p + 1) + quad_q(p) * quad_q(p) * (p + 1);
}
inline bool eo_tables(const double *T, int q, int n, std::vector<double> &dbl,
                      std::vector<int> &hdr) {
  if (n > 16) return false;
  double tmax = 0.0;
  for (int i = 0; i < q * n; ++i) tmax = T[i] > tmax ? T[i] : (-T[i] > tmax ? -T[i] : tmax);
  const double tol = 1e-10 * tmax;
  std::vector<int> partner(n, -1), sig(n, 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n && partner[i] < 0; ++j)
      for (int sg = 1; sg >= -1 && partner[i] < 0; sg -= 2) {
        bool ok = true;
        for (int o = 0; o < q && ok; ++o) {
          const double d = T[(q - 1 - o) * n + i] - sg * T[o * n + j];
          ok = (d <= tol && -d <= tol);
        }
        if (ok) {
          partner[i] = j;
          sig[i] = sg;
        }
      }
  for (int i = 0; i < n; ++i)
    if (partner[i] < 0) return false;
  const int he = (q + 1) / 2, ho = q / 2;
  std::vector<int> se, so, fl(16, 0);
  for (int i = 0; i < n; ++i) {
    const bool ev = partner[i] != i || sig[i] > 0, od = partner[i] != i || sig[i] < 0;
    if (ev) se.push_back(i);
    if (od) so.push_back(i);
    fl[i] = (ev ? 1 : 0) | (od ? 2 : 0);
  }
  auto E = [&](int o, int i) { return 0.5 * (T[o * n + i] + T[(q - 1 - o) * n + i]); };
  auto O = [&](int o, int i) { return 0.5 * (T[o * n + i] - T[(q - 1 - o) * n + i]); };
  const int off = (int)dbl.size();
  for (int o = 0; o < he; ++o)
    for (int i : se) dbl.push_back(E(o, i));
  for (int o = 0; o < ho; ++o)
    for (int i : so) dbl.push_back(O(o, i));
  for (int i = 0; i < n; ++i)
    for (int o = 0; o < he; ++o) dbl.push_back((fl[i] & 1) ? E(o, i) : 0.0);
  for (int i = 0; i < n; ++i)
    for (int o = 0; o < ho; ++o) dbl.push_back((fl[i] & 2) ? O(o, i) : 0.0);
  const size_t h0 = hdr.size();
  hdr.resize(h0 + kEoHeader, 0);
  int *hh = hdr.data() + h0;
  hh[0] = n;
  hh[1] = he;
  hh[2] = ho;
  hh[3] = (int)se.size();
  hh[4] = (int)so.size();
  hh[5] = off;
  for (size_t k = 0; k < se.size(); ++k) hh[6 + k] = se[k];
  for (size_t k = 0; k < so.size(); ++k) hh[22 + k] = so[k];
  for (int i = 0; i < 16; ++i) hh[38 + i] = fl[i];
  return true;
}

// Launch shape of the per-handle Cartesian apply (cart_local_kernel): a
// thread owns one line of a cell, a cell has at most (p + 1)^2 lines per
// component, so a CTA takes CPB cells (CPB (p + 1)^2 <= 256) and as many
// threads, rounded up to whole warps; CPB is the count that leaves the
// fewest idle lanes in that rounding (the smallest such).
__host__ __device__ constexpr int cart_cpb(int p) {
  const int nl = (p + 1) * (p + 1);
  int best = 1, bnum = 0, bden = 1;  // best lane use bnum / bden
  for (int c = 1; c <= 32 && c * nl <= 256; ++c) {
    const int nt = (c * nl + 31) / 32 * 32;
    if ((long long)c * nl * bden > (long long)bnum * nt) {
      best = c;
      bnum = c * nl;
      bden = nt;
    }
  }
  return best;
}
__host__ __device__ constexpr int cart_threads(int p) { return (cart_cpb(p) * (p + 1) * (p + 1) + 31) / 32 * 32; }
// its shared memory (doubles): D-hat, then per cell 8 coefficients, x on
// V^k (at the end the cell's product, staged for coalesced stores), d (later
// dy) on V^{k+1} and the interface line sums of every D-hat term
__host__ __device__ constexpr size_t cart_local_smem_doubles(int k, int p, int nloc0, int nloc1) {
  return (size_t)p * (p + 1) +
         (size_t)cart_cpb(p) * (8 + (size_t)nloc0 + (size_t)nloc1 + (size_t)(k == 1 ? 6 : 3) * 2 * (p + 1) * (p + 1));
}

// Compressed sparse rows with explicit row ids (lattice or compact).
// Threads per row of the CSR SpMV for an average row length avg: each
// lane takes about four entries (their loads in flight together), few warps
// per wave of dependent loads; rows of more than 256 entries get a CTA of
// 256 threads each.
inline int spmv_tpr(double avg) {
  return avg > 256 ? 256 : avg > 128 ? 32 : avg > 64 ? 16 : avg > 32 ? 8 : avg > 16 ? 4 : avg > 8 ? 2 : 1;
}

struct DevCsr {
  int nrows = 0;
  int tpr = 1;             // threads per row (spmv_tpr: 1..32 or 256, power of two)
  int *rid = nullptr;
  int *ptr = nullptr;
  int *col = nullptr;
  void *val = nullptr;     // double or float (vt)
  int vt = 0;
  // batched solves: the problem of every row and the device convergence
  // flags; rows of converged problems are skipped (null: no skipping)
  const int *rprob = nullptr, *done = nullptr;
};

// A family of patches with a shared slot template.
struct DevPatch {
  int nslots = 0, npatch = 0, nnz = 0;
  int nflev = 0, nblev = 0;
  const int *slotmap = nullptr;  // npatch x nslots
  const int *rowptr = nullptr, *col = nullptr;
  const int *tptr = nullptr, *trow = nullptr, *tpos = nullptr;
  const int *flev = nullptr, *frows = nullptr, *blev = nullptr, *brows = nullptr;
  const void *val = nullptr;     // npatch x nnz, double or float
  int vt = 0;
  // block-inverse form (exact factorisations): per patch the dense inverse
  // of every decoupled block, column-major, concatenated (ivals values)
  int inverse = 0, ivals = 0;
  const int *pos_slot = nullptr, *pos_blk = nullptr, *bptr = nullptr, *boff = nullptr;
  // batched solves: the problem of every patch and the convergence flags
  const int *pprob = nullptr, *done = nullptr;
  // elements between consecutive patches' factor values (>= nnz; padded to
  // 16 bytes when the warp kernel stages them with bulk copies)
  int vstride = 0;
  // warp-per-patch substitution (patch_warp_kernel): the template as one
  // 16-byte aligned blob of 16-bit arrays -- rowptr[ns+1], col[nnz],
  // flev[nflev+1], frows[ns], blev[nblev+1], brows[ns], tptr[ns+1],
  // trow[nstrict], tpos[nstrict] at element offsets toff[0..8] -- or null
  const unsigned short *tmpl = nullptr;
  int tmpl_bytes = 0;
  int toff[9] = {};
  int wpb = 0;  // patches (warps) per CTA of patch_warp_kernel; 0: the CTA-per-patch kernels
  // deterministic relaxation: the kernels store patch p's slot s value at
  // zp[p * nslots + s] instead of adding it into z; launch_patch_gather then
  // adds, for each of the family's ng lattice entries grow[i], the values
  // zp[gidx[gptr[i] .. gptr[i + 1])] in that (fixed) order
  double *zp = nullptr;
  int ng = 0;
  const int *grow = nullptr, *gptr = nullptr, *gidx = nullptr;
};

// launchers (kernels.cu); launch_count() = kernels launched so far in this process
long long launch_count();
void add_launches(long long k);  // for launchers in other files (learned.cu)
cudaError_t launch_apply(const ApplyDev &A, const double *x, double *y, cudaStream_t s);
// general cells (apply_general.cu)
cudaError_t launch_apply_general(const ApplyDev &A, const double *x, double *y, cudaStream_t s);
cudaError_t launch_metric(const ApplyDev &A, void *G, cudaStream_t s);
// Cartesian cells (apply_cart.cu): cell products into A.Y, then assembled;
// writes every entry of y (no zeroing needed)
cudaError_t launch_apply_cart(const ApplyDev &A, const double *x, double *y, cudaStream_t s);
// spmv modes: 0 y = a A x; 1 y += a A x; 2 y = u + a A x; 3 y += a A x with
// atomic adds (rows shared with other kernels adding concurrently)
cudaError_t launch_spmv(const DevCsr &M, const double *x, double *y, const double *u, int mode,
                        double a, cudaStream_t s);
cudaError_t launch_patches(const DevPatch &F, const double *r, double *z, cudaStream_t s);
// z[grow[i]] += the family's stored patch values of that entry, in a fixed order
cudaError_t launch_patch_gather(const DevPatch &F, double *z, cudaStream_t s);
// the warp-per-patch kernel's bounded waits: 1 if any gave up since the last
// call (the flag is cleared), 0 otherwise; a CUDA error code on failure
int patch_timeouts(cudaError_t *err);
// testing aid: 1 makes the warp kernel's bounded waits give up (see
// rm_debug_patch_timeout), 0 restores normal operation
cudaError_t patch_inject_timeout(int on);
// patches per CTA of the warp kernel for a family on the current device,
// chosen for the fewest waves (0: it does not fit)
int patch_warps_per_block(const DevPatch &F);
cudaError_t launch_gemv(int n, const void *A, int vt, const double *x, double *y, cudaStream_t s);
// coarse multigrid: x_out = x_in + w (b - A x_in) (A FP64, rows compact); x = w b
cudaError_t launch_jacobi(const DevCsr &A, const double *b, const double *xin, const double *w,
                          double *xout, cudaStream_t s);
cudaError_t launch_diag_scale(int n, const double *w, const double *b, double *x, cudaStream_t s);
cudaError_t launch_axpy(int n, double a, const double *x, double *y, int acc, cudaStream_t s);
cudaError_t launch_mask_copy(long long n, const uint8_t *mask, const double *b, double *r,
                             cudaStream_t s);
cudaError_t launch_sub(long long n, const uint8_t *mask, const double *b, const double *q,
                       double *r, cudaStream_t s);

// CG scalars in device memory
enum { S_RZ = 0, S_PQ, S_RR, S_BB, S_ALPHA, S_BETA, S_RZNEW, S_ZQ, S_COUNT };
constexpr int kDotBlocks = 592;  // 4 x 148 SMs-worth, fixed for deterministic sums
// partial buffer of the reductions below: 2 kDotBlocks partial sums and a
// ticket counter (zero-initialised; the finishing CTA resets it)
constexpr int kPartialDoubles = 2 * kDotBlocks + 1;
// hist (may be null): the reduction's sum is also stored at *hist
cudaError_t launch_dot(long long n, const double *a, const double *b, double *partial,
                       double *scal, int slot, cudaStream_t s, double *hist = nullptr);
cudaError_t launch_dot2(long long n, const double *r, const double *z, const double *q,
                        double *partial, double *scal, int flexible, cudaStream_t s,
                        double *hist = nullptr);
cudaError_t launch_alpha(long long n, const double *p, const double *q, double *partial,
                         double *scal, cudaStream_t s);
cudaError_t launch_update_xr(long long n, double *x, double *r, const double *p, const double *q,
                             double *partial, double *scal, cudaStream_t s, double *hist = nullptr);
cudaError_t launch_update_p(long long n, double *p, const double *z, const double *scal,
                            cudaStream_t s);

// batched solver (batch.cu)
cudaError_t launch_seg_dot(const int4 *chunk, int nchunk, const int *cptr, int nprob, const double *a,
                           const double *b, double *partial, double *scal, int *done, int *iters,
                           int slot, int op, double tol2, cudaStream_t s);
cudaError_t launch_seg_update_xr(const int4 *chunk, int nchunk, const int *cptr, int nprob, double *x,
                                 double *r, const double *p, const double *q, double *partial,
                                 double *scal, int *done, int *iters, double tol2, cudaStream_t s);
cudaError_t launch_seg_dot2(const int4 *chunk, int nchunk, const int *cptr, int nprob, const double *r,
                            const double *z, const double *q, double *partial, double *scal, int *done,
                            int *iters, int flexible, cudaStream_t s);
cudaError_t launch_seg_update_p(const int4 *chunk, int nchunk, double *p, const double *z,
                                const double *scal, cudaStream_t s);
cudaError_t launch_gemv_batch(int nrows, const int *rowprob, const long long *aoff, const int *cstart,
                              const int *csz, const double *A, const double *x, double *y,
                              cudaStream_t s);

}  // namespace rmd
