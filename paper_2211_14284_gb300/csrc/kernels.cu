// Device kernels of the Riesz-map solvers (sm_103a).
//
// (The operator applies are in apply_general.cuh, general cells, and
// apply_cart.cuh, axis-aligned cells and the shared assembly.)
// * patch_warp_kernel / patch_kernel: z += sum_j R_j^T L_j^-T L_j^-1 R_j r
//   over a patch family (Eqs. asm-afw, sc-asm-afw, sc-asm-hiptmair):
//   level-scheduled sparse forward/backward substitutions on the template
//   pattern shared by all patches of the family, a warp per patch with the
//   factors staged by bulk copies, or a CTA per patch for factors too large
//   to stage; patch_inv_kernel for exact factors stored as block inverses.
// * SpMV / GEMV for static condensation (Eq. schur), the Hiptmair gradient
//   and the p = 1 coarse correction; fused CG updates with deterministic
//   fixed-order FP64 reductions finished by the last CTA.
#include <algorithm>
#include <atomic>

#include "df.cuh"
#include "mbarrier.cuh"

namespace rmd {

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void add_launches(long long k) { g_launches += k; }

namespace {

// One damped Jacobi sweep of the coarse multigrid: x_out = x_in + w (b - A x_in),
// w = omega / diag(A) (FP64 CSR, TPR threads per row).
template <int TPR>
__global__ void jacobi_kernel(int nrows, const int *__restrict__ ptr, const int *__restrict__ col,
                              const double *__restrict__ val, const double *__restrict__ b,
                              const double *__restrict__ xin, const double *__restrict__ w,
                              double *__restrict__ xout) {
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = (int)(gt / TPR), lane = (int)(gt % TPR);
  double s = 0.0;
  if (row < nrows)
    for (int e = ptr[row] + lane; e < ptr[row + 1]; e += TPR) s = fma(val[e], xin[col[e]], s);
#pragma unroll
  for (int off = TPR / 2; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off, TPR);
  if (lane == 0 && row < nrows) xout[row] = fma(w[row], b[row] - s, xin[row]);
}

__global__ void diag_scale_kernel(int n, const double *__restrict__ w, const double *__restrict__ b,
                                  double *__restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = w[i] * b[i];
}

// y = a x (acc = 0) or y += a x (acc = 1)
__global__ void axpy_kernel(int n, double a, const double *__restrict__ x, double *__restrict__ y,
                            int acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = acc ? fma(a, x[i], y[i]) : a * x[i];
}

template <typename VT, int TPR>
__global__ void spmv_kernel(int nrows, const int *__restrict__ rid, const int *__restrict__ ptr,
                            const int *__restrict__ col, const VT *__restrict__ val,
                            const double *x, double *y, const double *u, int mode, double a,
                            const int *__restrict__ rprob, const int *__restrict__ done) {
  // x, y and u may alias (z_I = w_I - E^T z_G reads and writes z on
  // disjoint rows), so they are not declared __restrict__.
  // Products accumulate in the matrix's precision VT (FP32 data: the
  // mixed-precision preconditioner; the coarse path is always FP64).
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = (int)(gt / TPR), lane = (int)(gt % TPR);
  // rows of converged problems (batched solves) are skipped; their lanes
  // still take part in the shuffles
  const bool live = row < nrows && !(rprob && done[rprob[row]]);
  VT s = 0;
  if (live) {
    const int e1 = ptr[row + 1];
#pragma unroll 4
    for (int e = ptr[row] + lane; e < e1; e += TPR) s = fma(val[e], (VT)x[col[e]], s);
  }
#pragma unroll
  for (int off = TPR / 2; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off, TPR);
  if (lane == 0 && live) {
    const int r = rid[row];
    const double v = a * (double)s;
    if (mode == 0) y[r] = v;
    else if (mode == 1) y[r] += v;
    else if (mode == 3) atomicAdd(y + r, v);  // y += a A x beside concurrent atomic adders
    else y[r] = u[r] + v;
  }
}

// The same product with one CTA of kSpmvRowBlock threads per row (rows of
// hundreds to thousands of entries: the p -> 1 restriction R_0).
constexpr int kSpmvRowBlock = 256;
template <typename VT>
__global__ void __launch_bounds__(kSpmvRowBlock) spmv_row_block_kernel(
    int nrows, const int *__restrict__ rid, const int *__restrict__ ptr, const int *__restrict__ col,
    const VT *__restrict__ val, const double *x, double *y, const double *u, int mode, double a,
    const int *__restrict__ rprob, const int *__restrict__ done) {
  __shared__ VT part[kSpmvRowBlock / 32];
  const int row = blockIdx.x;
  if (rprob && done[rprob[row]]) return;  // uniform over the CTA
  VT s = 0;
  const int e1 = ptr[row + 1];
#pragma unroll 4
  for (int e = ptr[row] + threadIdx.x; e < e1; e += kSpmvRowBlock) s = fma(val[e], (VT)x[col[e]], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    VT t = 0;
#pragma unroll
    for (int w = 0; w < kSpmvRowBlock / 32; ++w) t += part[w];
    const int r = rid[row];
    const double v = a * (double)t;
    if (mode == 0) y[r] = v;
    else if (mode == 1) y[r] += v;
    else if (mode == 3) atomicAdd(y + r, v);
    else y[r] = u[r] + v;
  }
}

// xs[s] = r[sm[s]] (0 for slots outside the problem, sm[s] < 0): the slot
// indices of four rounds are loaded before their gathers.
template <typename VT>
__device__ __forceinline__ void gather_slots(const int *__restrict__ sm, int ns, const double *__restrict__ r,
                                             VT *xs) {
  const int nt = blockDim.x;
  int s = threadIdx.x;
  for (; s + 3 * nt < ns; s += 4 * nt) {
    int g[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) g[u] = sm[s + u * nt];
#pragma unroll
    for (int u = 0; u < 4; ++u) xs[s + u * nt] = g[u] >= 0 ? (VT)r[g[u]] : (VT)0;
  }
  for (; s < ns; s += nt) {
    const int g = sm[s];
    xs[s] = g >= 0 ? (VT)r[g] : (VT)0;
  }
}

// Level-scheduled forward/backward substitution with the template factor.
// STAGE: the patch's factor values are first copied to shared memory with
// coalesced loads, so the dependency chain reads only shared memory.  The
// arithmetic runs in the factor's precision VT (FP32 for the mixed-precision
// preconditioner: GB300's FP64 pipe is 1/64 of its FP32 rate), and the
// factor's diagonal entries are stored as their reciprocals (no division).
template <typename VT, bool STAGE>
__global__ void patch_kernel(DevPatch F, const double *__restrict__ r, double *__restrict__ z) {
  if (F.pprob && F.done[F.pprob[blockIdx.x]]) return;  // converged problem (batched solves)
  extern __shared__ double smem_raw[];
  VT *xs = reinterpret_cast<VT *>(smem_raw);
  const int ns = F.nslots;
  const int *sm = F.slotmap + (size_t)blockIdx.x * ns;
  const VT *Lg = reinterpret_cast<const VT *>(F.val) + (size_t)blockIdx.x * (F.vstride ? F.vstride : F.nnz);
  // the factor follows x (ns values of VT, padded to whole doubles)
  VT *Ls = reinterpret_cast<VT *>(smem_raw + (ns * sizeof(VT) + sizeof(double) - 1) / sizeof(double));
  gather_slots(sm, ns, r, xs);
  if (STAGE) {
    // coalesced copy, eight loads per thread in flight
    const int nnz = F.nnz, nt = blockDim.x;
    int e = threadIdx.x;
    for (; e + 7 * nt < nnz; e += 8 * nt) {
      VT t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = Lg[e + u * nt];
#pragma unroll
      for (int u = 0; u < 8; ++u) Ls[e + u * nt] = t[u];
    }
    for (; e < nnz; e += nt) Ls[e] = Lg[e];
  }
  const VT *L = STAGE ? Ls : Lg;
  __syncthreads();
  for (int lv = 0; lv < F.nflev; ++lv) {
    for (int t = F.flev[lv] + threadIdx.x; t < F.flev[lv + 1]; t += blockDim.x) {
      const int i = F.frows[t];
      const int b = F.rowptr[i], d = F.rowptr[i + 1] - 1;
      VT v = xs[i];
#pragma unroll 4
      for (int e = b; e < d; ++e) v = fma(-L[e], xs[F.col[e]], v);
      xs[i] = v * L[d];
    }
    __syncthreads();
  }
  for (int lv = 0; lv < F.nblev; ++lv) {
    for (int t = F.blev[lv] + threadIdx.x; t < F.blev[lv + 1]; t += blockDim.x) {
      const int j = F.brows[t];
      VT v = xs[j];
      const int e1 = F.tptr[j + 1];
#pragma unroll 4
      for (int e = F.tptr[j]; e < e1; ++e) v = fma(-L[F.tpos[e]], xs[F.trow[e]], v);
      xs[j] = v * L[F.rowptr[j + 1] - 1];
    }
    __syncthreads();
  }
  if (F.zp) {  // deterministic relaxation: the values, summed later in a fixed order
    for (int s = threadIdx.x; s < ns; s += blockDim.x) F.zp[(size_t)blockIdx.x * ns + s] = (double)xs[s];
    return;
  }
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    const int g = sm[s];
    if (g >= 0) atomicAdd(&z[g], (double)xs[s]);
  }
}

// ---- warp-per-patch substitution --------------------------------------------
// WPB patches per CTA, one warp each.  The family's template (16-bit index
// arrays, shared by every patch) and the CTA's factors are staged into
// shared memory by bulk copies (cp.async.bulk, the TMA unit) completing on
// one mbarrier, while the warps gather their patch residuals; each warp then
// runs its patch's level-scheduled forward and backward substitutions with
// __syncwarp between levels instead of CTA barriers.  Every wait on the
// mbarrier is bounded: on timeout the CTA records it in g_patch_timeout,
// waits once more (bounded) for its copies and returns without touching z.
__device__ int g_patch_timeout = 0;
// testing aid (rm_debug_patch_timeout): when set, every CTA of the warp
// kernel expects 16 bytes more than its copies deliver, so its bounded wait
// gives up as a wait on a lost copy would
__device__ int g_patch_inject = 0;

constexpr int kPatchWarpMaxWPB = 8;
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
// shared memory of the warp kernel: mbarrier, template, then per warp the
// factor and the slot values
template <typename VT>
__host__ __device__ inline size_t patch_warp_smem(const DevPatch &F, int wpb) {
  return 16 + align16((size_t)F.tmpl_bytes) +
         (size_t)wpb * (align16((size_t)F.vstride * sizeof(VT)) + align16((size_t)F.nslots * sizeof(VT)));
}

template <typename VT, int WPB>
__global__ void __launch_bounds__(WPB * 32) patch_warp_kernel(DevPatch F, const double *__restrict__ r,
                                                              double *__restrict__ z) {
  extern __shared__ __align__(16) unsigned char psm[];
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(psm);
  const unsigned short *T = reinterpret_cast<const unsigned short *>(psm + 16);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p0 = blockIdx.x * WPB;
  const int nblk = min(WPB, F.npatch - p0);
  const size_t fbytes = align16((size_t)F.vstride * sizeof(VT)), xbytes = align16((size_t)F.nslots * sizeof(VT));
  unsigned char *wbase = psm + 16 + align16((size_t)F.tmpl_bytes) + (size_t)warp * (fbytes + xbytes);
  const VT *L = reinterpret_cast<const VT *>(wbase);
  VT *xs = reinterpret_cast<VT *>(wbase + fbytes);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned extra = g_patch_inject ? 16u : 0u;
    mbar_expect_tx(bar, (unsigned)(F.tmpl_bytes + (size_t)nblk * F.vstride * sizeof(VT)) + extra);
    bulk_g2s(psm + 16, F.tmpl, (unsigned)F.tmpl_bytes, bar);
    for (int w = 0; w < nblk; ++w)
      bulk_g2s(psm + 16 + align16((size_t)F.tmpl_bytes) + (size_t)w * (fbytes + xbytes),
               reinterpret_cast<const VT *>(F.val) + (size_t)(p0 + w) * F.vstride,
               (unsigned)((size_t)F.vstride * sizeof(VT)), bar);
  }
  const int patch = p0 + warp;
  const bool live = warp < nblk && !(F.pprob && F.done[F.pprob[patch]]);
  const int ns = F.nslots;
  const int *sm = F.slotmap + (size_t)(live ? patch : 0) * ns;
  if (live)
    for (int s = lane; s < ns; s += 32) {
      const int g = sm[s];
      xs[s] = g >= 0 ? (VT)r[g] : (VT)0;
    }
  if (!mbar_wait_bounded(bar, 0)) {
    if (threadIdx.x == 0) atomicExch(&g_patch_timeout, 1);
    mbar_wait_bounded(bar, 0);  // the copies in flight still target this CTA's memory
    return;
  }
  __syncwarp();
  if (!live) return;
  const unsigned short *rowptr = T + F.toff[0], *col = T + F.toff[1], *flev = T + F.toff[2],
                       *frows = T + F.toff[3], *blev = T + F.toff[4], *brows = T + F.toff[5],
                       *tptr = T + F.toff[6], *trow = T + F.toff[7], *tpos = T + F.toff[8];
  for (int lv = 0; lv < F.nflev; ++lv) {
    for (int t = flev[lv] + lane; t < flev[lv + 1]; t += 32) {
      const int i = frows[t];
      const int b = rowptr[i], d = rowptr[i + 1] - 1;
      VT v = xs[i];
#pragma unroll 4
      for (int e = b; e < d; ++e) v = fma(-L[e], xs[col[e]], v);
      xs[i] = v * L[d];
    }
    __syncwarp();
  }
  for (int lv = 0; lv < F.nblev; ++lv) {
    for (int t = blev[lv] + lane; t < blev[lv + 1]; t += 32) {
      const int j = brows[t];
      VT v = xs[j];
      const int e1 = tptr[j + 1];
#pragma unroll 4
      for (int e = tptr[j]; e < e1; ++e) v = fma(-L[tpos[e]], xs[trow[e]], v);
      xs[j] = v * L[rowptr[j + 1] - 1];
    }
    __syncwarp();
  }
  if (F.zp) {  // deterministic relaxation: the values, summed later in a fixed order
    for (int s = lane; s < ns; s += 32) F.zp[(size_t)patch * ns + s] = (double)xs[s];
    return;
  }
  for (int s = lane; s < ns; s += 32) {
    const int g = sm[s];
    if (g >= 0) atomicAdd(&z[g], (double)xs[s]);
  }
}

// Block-inverse patches: y_block = (A_block)^{-1} x_block for every decoupled
// block of the patch, one row per thread, the column-major inverse read with
// coalesced loads; no level chain.  Arithmetic in the data's precision VT.
template <typename VT>
__global__ void patch_inv_kernel(DevPatch F, const double *__restrict__ r, double *__restrict__ z) {
  if (F.pprob && F.done[F.pprob[blockIdx.x]]) return;  // converged problem (batched solves)
  extern __shared__ double smem_raw[];
  VT *xs = reinterpret_cast<VT *>(smem_raw);
  const int ns = F.nslots;
  VT *ys = xs + ns;
  const int *sm = F.slotmap + (size_t)blockIdx.x * ns;
  const VT *V = reinterpret_cast<const VT *>(F.val) + (size_t)blockIdx.x * F.ivals;
  gather_slots(sm, ns, r, xs);
  __syncthreads();
  for (int t = threadIdx.x; t < ns; t += blockDim.x) {
    const int b = F.pos_blk[t];
    const int p0 = F.bptr[b], nb = F.bptr[b + 1] - p0, i = t - p0;
    const VT *Vb = V + F.boff[b] + i;
    const int *ps = F.pos_slot + p0;
    VT acc = 0;
    int j = 0;
    // eight column loads in flight before their multiply-adds (same order)
    for (; j + 8 <= nb; j += 8) {
      VT v[8];
      int c[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        v[u] = Vb[(size_t)(j + u) * nb];
        c[u] = ps[j + u];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) acc = fma(v[u], xs[c[u]], acc);
    }
    for (; j < nb; ++j) acc = fma(Vb[(size_t)j * nb], xs[ps[j]], acc);
    ys[t] = acc;
  }
  __syncthreads();
  if (F.zp) {  // deterministic relaxation: the values, summed later in a fixed order
    for (int t = threadIdx.x; t < ns; t += blockDim.x)
      F.zp[(size_t)blockIdx.x * ns + F.pos_slot[t]] = (double)ys[t];
    return;
  }
  for (int t = threadIdx.x; t < ns; t += blockDim.x) {
    const int g = sm[F.pos_slot[t]];
    if (g >= 0) atomicAdd(&z[g], (double)ys[t]);
  }
}

// z[grow[i]] += sum of zp[gidx[k]], k = gptr[i] .. gptr[i + 1] - 1, in that
// order: the deterministic form of a patch family's scatter (one thread per
// lattice entry the family touches; the entries are distinct)
__global__ void patch_gather_kernel(int ng, const int *__restrict__ grow, const int *__restrict__ gptr,
                                    const int *__restrict__ gidx, const double *__restrict__ zp,
                                    double *__restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ng) return;
  double acc = 0.0;
  for (int k = gptr[i]; k < gptr[i + 1]; ++k) acc += zp[gidx[k]];
  z[grow[i]] += acc;
}

template <typename VT>
__global__ void gemv_kernel(int n, const VT *__restrict__ A, const double *__restrict__ x,
                            double *__restrict__ y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
  if (warp < n)
    for (int j = lane; j < n; j += 32) s = fma((double)A[(size_t)warp * n + j], x[j], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0 && warp < n) y[warp] = s;
}

__global__ void mask_copy_kernel(long long n, const uint8_t *__restrict__ mask,
                                 const double *__restrict__ b, double *__restrict__ r) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = mask[i] ? 0.0 : b[i];
}
__global__ void sub_kernel(long long n, const uint8_t *__restrict__ mask, const double *__restrict__ b,
                           const double *__restrict__ q, double *__restrict__ r) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = mask[i] ? 0.0 : b[i] - q[i];
}

// ---- reductions -------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (w == 0)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// The CTA that finishes last (a ticket counter after the 2 kDotBlocks
// partials) sums the partials in fixed order -- the order of one CTA of
// blockDim threads, so the result does not depend on which CTA finishes
// last -- applies op and resets the counter.  No CTA waits for another.
// op 0: scal[slot] = sum; op 1: pq -> alpha; op 2: (rz_new, zq) -> beta, rz.
// hist (may be null): the sum is also stored there (residual histories).
__device__ __forceinline__ void finish_reduction(double *partial, double *scal, int slot, int op, int flexible,
                                                 double *hist = nullptr) {
  __shared__ bool last;
  unsigned int *count = reinterpret_cast<unsigned int *>(partial + 2 * kDotBlocks);
  __threadfence();  // this CTA's partials before its ticket
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += blockDim.x) {
    s += __ldcg(partial + i);
    if (op == 2) t += __ldcg(partial + kDotBlocks + i);
  }
  s = block_sum(s);
  if (op == 2) t = block_sum(t);
  if (threadIdx.x == 0) {
    if (hist) *hist = s;
    if (op == 0) {
      scal[slot] = s;
    } else if (op == 1) {
      scal[S_PQ] = s;
      scal[S_ALPHA] = scal[S_RZ] / s;
    } else {
      const double rz = scal[S_RZ];
      scal[S_RZNEW] = s;
      scal[S_ZQ] = t;
      scal[S_BETA] = flexible ? -t / scal[S_PQ] : s / rz;
      scal[S_RZ] = s;
    }
    *count = 0u;
  }
}

__global__ void dot_kernel(long long n, const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ partial, double *__restrict__ scal, int slot, int op,
                           double *hist) {
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  finish_reduction(partial, scal, slot, op, 0, hist);
}

__global__ void dot2_kernel(long long n, const double *__restrict__ r, const double *__restrict__ z,
                            const double *__restrict__ q, double *__restrict__ partial, double *__restrict__ scal,
                            int flexible, double *hist) {
  double s = 0.0, t = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double zi = z[i];
    s = fma(r[i], zi, s);
    t = fma(q[i], zi, t);
  }
  s = block_sum(s);
  t = block_sum(t);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    partial[kDotBlocks + blockIdx.x] = t;
  }
  finish_reduction(partial, scal, S_RZNEW, 2, flexible, hist);
}

__global__ void update_xr_kernel(long long n, double *__restrict__ x, double *__restrict__ r,
                                 const double *__restrict__ p, const double *__restrict__ q,
                                 double *__restrict__ partial, double *__restrict__ scal, double *hist) {
  const double a = scal[S_ALPHA];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  finish_reduction(partial, scal, S_RR, 0, 0, hist);
}

__global__ void update_p_kernel(long long n, double *__restrict__ p, const double *__restrict__ z,
                                const double *__restrict__ scal) {
  const double b = scal[S_BETA];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(b, p[i], z[i]);
}

// ---- batched (segmented) CG: block b works on chunk[b] = (problem, begin,
// end) of the concatenated vectors; per-problem scalars scal[prob * S_COUNT];
// done[prob] freezes a converged problem (alpha = beta = 0) --------------------
__global__ void seg_dot_kernel(const int4 *__restrict__ chunk, const double *__restrict__ a,
                               const double *__restrict__ b, double *__restrict__ partial) {
  const int4 c = chunk[blockIdx.x];
  double s = 0.0;
  for (int i = c.y + threadIdx.x; i < c.z; i += blockDim.x) s = fma(a[i], b[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}
__global__ void seg_dot2_kernel(const int4 *__restrict__ chunk, int nchunk, const double *__restrict__ r,
                                const double *__restrict__ z, const double *__restrict__ q,
                                double *__restrict__ partial) {
  const int4 c = chunk[blockIdx.x];
  double s = 0.0, t = 0.0;
  for (int i = c.y + threadIdx.x; i < c.z; i += blockDim.x) {
    s = fma(r[i], z[i], s);
    t = fma(q[i], z[i], t);
  }
  s = block_sum(s);
  t = block_sum(t);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    partial[nchunk + blockIdx.x] = t;
  }
}
__global__ void seg_update_xr_kernel(const int4 *__restrict__ chunk, double *__restrict__ x,
                                     double *__restrict__ r, const double *__restrict__ p,
                                     const double *__restrict__ q, const double *__restrict__ scal,
                                     double *__restrict__ partial) {
  const int4 c = chunk[blockIdx.x];
  const double a = scal[c.x * S_COUNT + S_ALPHA];
  double s = 0.0;
  for (int i = c.y + threadIdx.x; i < c.z; i += blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}
__global__ void seg_update_p_kernel(const int4 *__restrict__ chunk, double *__restrict__ p,
                                    const double *__restrict__ z, const double *__restrict__ scal) {
  const int4 c = chunk[blockIdx.x];
  const double b = scal[c.x * S_COUNT + S_BETA];
  for (int i = c.y + threadIdx.x; i < c.z; i += blockDim.x) p[i] = fma(b, p[i], z[i]);
}
// One block per problem: fixed-order sum of its chunks' partials.
// op 0: scal[slot] = s; op 1: pq -> alpha; op 2: rr -> convergence test;
// op 3: (rz_new, zq) -> beta.  done[prob]: 0 running, 1 converged, 2 NaN/Inf
// residual, 3 breakdown (p^T A p <= 0); a nonzero flag freezes the problem
// (alpha = beta = 0) and its cells, patches and rows are skipped.
__global__ void seg_finalize_kernel(const int *__restrict__ cptr, int nchunk,
                                    const double *__restrict__ partial, double *__restrict__ scal,
                                    int *__restrict__ done, int *__restrict__ iters, int slot, int op,
                                    int flexible, double tol2) {
  const int prob = blockIdx.x;
  double s = 0.0, t = 0.0;
  for (int i = cptr[prob] + threadIdx.x; i < cptr[prob + 1]; i += blockDim.x) {
    s += partial[i];
    if (op == 3) t += partial[nchunk + i];
  }
  s = block_sum(s);
  if (op == 3) t = block_sum(t);
  if (threadIdx.x != 0) return;
  double *sc = scal + prob * S_COUNT;
  const bool dn = done[prob] != 0;
  if (op == 0) {
    sc[slot] = s;
  } else if (op == 1) {
    sc[S_PQ] = s;
    const bool brk = !dn && !(s > 0.0);
    if (brk) done[prob] = 3;
    sc[S_ALPHA] = (dn || brk) ? 0.0 : sc[S_RZ] / s;
  } else if (op == 2) {
    if (!dn) {
      sc[S_RR] = s;
      iters[prob] += 1;
      if (!isfinite(s)) done[prob] = 2;
      else if (s <= tol2 * sc[S_BB]) done[prob] = 1;
    }
  } else {
    sc[S_RZNEW] = s;
    sc[S_ZQ] = t;
    sc[S_BETA] = dn ? 0.0 : (flexible ? -t / sc[S_PQ] : s / sc[S_RZ]);
    sc[S_RZ] = s;
  }
}

// Batched dense GEMV of the per-problem coarse inverses: one warp per coarse
// row of the concatenation; rowprob maps it to its problem.
__global__ void gemv_batch_kernel(int nrows, const int *__restrict__ rowprob,
                                  const long long *__restrict__ aoff, const int *__restrict__ cstart,
                                  const int *__restrict__ csz, const double *__restrict__ A,
                                  const double *__restrict__ x, double *__restrict__ y) {
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
  int pr = 0, lr = 0, n = 0;
  if (g < nrows) {
    pr = rowprob[g];
    n = csz[pr];
    lr = g - cstart[pr];
    const double *Ar = A + aoff[pr] + (long long)lr * n;
    const double *xp = x + cstart[pr];
    for (int j = lane; j < n; j += 32) s = fma(Ar[j], xp[j], s);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0 && g < nrows) y[g] = s;
}

inline int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 1184 ? 1184 : g));
}

}  // namespace

cudaError_t launch_apply(const ApplyDev &A, const double *x, double *y, cudaStream_t s) {
  if (A.cartesian) return launch_apply_cart(A, x, y, s);
  return launch_apply_general(A, x, y, s);
}

template <typename VT>
static void spmv_dispatch(const DevCsr &M, const double *x, double *y, const double *u, int mode,
                          double a, cudaStream_t s) {
  const int threads = 256;
  const long long tot = (long long)M.nrows * M.tpr;
  const int grid = (int)((tot + threads - 1) / threads);
  const VT *v = reinterpret_cast<const VT *>(M.val);
  switch (M.tpr) {
    case 1: spmv_kernel<VT, 1><<<grid, threads, 0, s>>>(M.nrows, M.rid, M.ptr, M.col, v, x, y, u, mode, a, M.rprob, M.done); break;
    case 2: spmv_kernel<VT, 2><<<grid, threads, 0, s>>>(M.nrows, M.rid, M.ptr, M.col, v, x, y, u, mode, a, M.rprob, M.done); break;
    case 4: spmv_kernel<VT, 4><<<grid, threads, 0, s>>>(M.nrows, M.rid, M.ptr, M.col, v, x, y, u, mode, a, M.rprob, M.done); break;
    case 8: spmv_kernel<VT, 8><<<grid, threads, 0, s>>>(M.nrows, M.rid, M.ptr, M.col, v, x, y, u, mode, a, M.rprob, M.done); break;
    case 16: spmv_kernel<VT, 16><<<grid, threads, 0, s>>>(M.nrows, M.rid, M.ptr, M.col, v, x, y, u, mode, a, M.rprob, M.done); break;
    case kSpmvRowBlock:
      spmv_row_block_kernel<VT><<<M.nrows, kSpmvRowBlock, 0, s>>>(M.nrows, M.rid, M.ptr, M.col, v, x, y, u, mode, a,
                                                                  M.rprob, M.done);
      break;
    default: spmv_kernel<VT, 32><<<grid, threads, 0, s>>>(M.nrows, M.rid, M.ptr, M.col, v, x, y, u, mode, a, M.rprob, M.done); break;
  }
}

cudaError_t launch_spmv(const DevCsr &M, const double *x, double *y, const double *u, int mode,
                        double a, cudaStream_t s) {
  if (M.nrows == 0) return cudaSuccess;
  if (M.vt == 0) spmv_dispatch<double>(M, x, y, u, mode, a, s);
  else spmv_dispatch<float>(M, x, y, u, mode, a, s);
  g_launches += 1;
  return cudaGetLastError();
}

template <typename VT, int... W>
static const void *warp_kernel_at(int w, std::integer_sequence<int, W...>) {
  const void *k = nullptr;
  ((w == W + 1 ? (k = (const void *)patch_warp_kernel<VT, W + 1>, 0) : 0), ...);
  return k;
}
template <typename VT>
static const void *warp_kernel(int w) {
  return warp_kernel_at<VT>(w, std::make_integer_sequence<int, kPatchWarpMaxWPB>{});
}

// Patches per CTA of the warp kernel: the fewest waves over the SMs (CTAs
// resident per SM from the occupancy calculator at that CTA's shared
// memory), then the fewest patches on the busiest SM, then the most patches
// per CTA (one template copy for more of them).  0: it does not fit.
template <typename VT>
static int warps_per_block(const DevPatch &F) {
  if (!F.tmpl || F.inverse) return 0;
  int dev = 0, nsm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  long long best[3] = {0, 0, 0};
  int wbest = 0;
  for (int w = 1; w <= kPatchWarpMaxWPB; ++w) {
    const size_t smem = patch_warp_smem<VT>(F, w);
    if (smem > 227 * 1024) break;
    const void *kern = warp_kernel<VT>(w);
    int cps = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cps, kern, 32 * w, smem) != cudaSuccess || cps < 1)
      continue;
    const long long ncta = (F.npatch + w - 1) / w;
    const long long waves = (ncta + (long long)nsm * cps - 1) / ((long long)nsm * cps);
    const long long load = (ncta + nsm - 1) / nsm * w;
    const long long key[3] = {waves, load, -w};
    if (wbest == 0 || std::lexicographical_compare(key, key + 3, best, best + 3)) {
      std::copy(key, key + 3, best);
      wbest = w;
    }
  }
  cudaGetLastError();  // a refused configuration above is not an error of the caller
  return wbest;
}

template <typename VT>
static void patch_dispatch(const DevPatch &F, const double *r, double *z, cudaStream_t s) {
  if (F.wpb > 0) {
    const size_t smem = patch_warp_smem<VT>(F, F.wpb);
    const int grid = (F.npatch + F.wpb - 1) / F.wpb;
    const void *kern = warp_kernel<VT>(F.wpb);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    DevPatch Fa = F;
    const double *ra = r;
    double *za = z;
    void *args[] = {&Fa, &ra, &za};
    cudaLaunchKernel(kern, dim3(grid), dim3(32 * F.wpb), args, smem, s);
    return;
  }
  if (F.inverse) {
    const size_t smem = 2 * (size_t)F.nslots * sizeof(VT);
    cudaFuncSetAttribute(patch_inv_kernel<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    patch_inv_kernel<VT><<<F.npatch, 256, smem, s>>>(F, r, z);
    return;
  }
  // x in VT, padded to whole doubles so the staged factor stays aligned
  const size_t base = ((size_t)F.nslots * sizeof(VT) + sizeof(double) - 1) / sizeof(double) * sizeof(double);
  const size_t staged = base + (size_t)F.nnz * sizeof(VT);
  if (staged <= 220 * 1024) {
    cudaFuncSetAttribute(patch_kernel<VT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)staged);
    patch_kernel<VT, true><<<F.npatch, 128, staged, s>>>(F, r, z);
  } else {
    cudaFuncSetAttribute(patch_kernel<VT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base);
    patch_kernel<VT, false><<<F.npatch, 128, base, s>>>(F, r, z);
  }
}

cudaError_t launch_patch_gather(const DevPatch &F, double *z, cudaStream_t s) {
  if (!F.zp || F.ng == 0) return cudaSuccess;
  patch_gather_kernel<<<(F.ng + 255) / 256, 256, 0, s>>>(F.ng, F.grow, F.gptr, F.gidx, F.zp, z);
  g_launches += 1;
  return cudaGetLastError();
}

int patch_warps_per_block(const DevPatch &F) {
  return F.vt == 0 ? warps_per_block<double>(F) : warps_per_block<float>(F);
}

cudaError_t patch_inject_timeout(int on) {
  const int v = on ? 1 : 0;
  return cudaMemcpyToSymbol(g_patch_inject, &v, sizeof(int));
}

int patch_timeouts(cudaError_t *err) {
  int v = 0;
  const int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_patch_timeout, sizeof(int));
  if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_patch_timeout, &zero, sizeof(int));
  if (err) *err = e;
  return v;
}

cudaError_t launch_patches(const DevPatch &F, const double *r, double *z, cudaStream_t s) {
  if (F.npatch == 0) return cudaSuccess;
  if (F.vt == 0) patch_dispatch<double>(F, r, z, s);
  else patch_dispatch<float>(F, r, z, s);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const DevCsr &A, const double *b, const double *xin, const double *w,
                          double *xout, cudaStream_t s) {
  const int threads = 256;
  const int tpr = A.tpr > 32 ? 32 : A.tpr;
  const long long tot = (long long)A.nrows * tpr;
  const int grid = (int)((tot + threads - 1) / threads);
  const double *v = reinterpret_cast<const double *>(A.val);
  switch (tpr) {
    case 1: jacobi_kernel<1><<<grid, threads, 0, s>>>(A.nrows, A.ptr, A.col, v, b, xin, w, xout); break;
    case 2: jacobi_kernel<2><<<grid, threads, 0, s>>>(A.nrows, A.ptr, A.col, v, b, xin, w, xout); break;
    case 4: jacobi_kernel<4><<<grid, threads, 0, s>>>(A.nrows, A.ptr, A.col, v, b, xin, w, xout); break;
    case 8: jacobi_kernel<8><<<grid, threads, 0, s>>>(A.nrows, A.ptr, A.col, v, b, xin, w, xout); break;
    case 16: jacobi_kernel<16><<<grid, threads, 0, s>>>(A.nrows, A.ptr, A.col, v, b, xin, w, xout); break;
    default: jacobi_kernel<32><<<grid, threads, 0, s>>>(A.nrows, A.ptr, A.col, v, b, xin, w, xout); break;
  }
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_axpy(int n, double a, const double *x, double *y, int acc, cudaStream_t s) {
  axpy_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, a, x, y, acc);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_diag_scale(int n, const double *w, const double *b, double *x, cudaStream_t s) {
  diag_scale_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, w, b, x);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_gemv(int n, const void *A, int vt, const double *x, double *y, cudaStream_t s) {
  const int threads = 256;
  const int grid = (int)(((long long)n * 32 + threads - 1) / threads);
  if (vt == 0) gemv_kernel<double><<<grid, threads, 0, s>>>(n, (const double *)A, x, y);
  else gemv_kernel<float><<<grid, threads, 0, s>>>(n, (const float *)A, x, y);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_mask_copy(long long n, const uint8_t *mask, const double *b, double *r, cudaStream_t s) {
  mask_copy_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, mask, b, r);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_sub(long long n, const uint8_t *mask, const double *b, const double *q, double *r,
                       cudaStream_t s) {
  sub_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, mask, b, q, r);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_dot(long long n, const double *a, const double *b, double *partial, double *scal,
                       int slot, cudaStream_t s, double *hist) {
  dot_kernel<<<kDotBlocks, 256, 0, s>>>(n, a, b, partial, scal, slot, 0, hist);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_alpha(long long n, const double *p, const double *q, double *partial, double *scal,
                         cudaStream_t s) {
  dot_kernel<<<kDotBlocks, 256, 0, s>>>(n, p, q, partial, scal, S_PQ, 1, nullptr);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_dot2(long long n, const double *r, const double *z, const double *q, double *partial,
                        double *scal, int flexible, cudaStream_t s, double *hist) {
  dot2_kernel<<<kDotBlocks, 256, 0, s>>>(n, r, z, q, partial, scal, flexible, hist);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_update_xr(long long n, double *x, double *r, const double *p, const double *q,
                             double *partial, double *scal, cudaStream_t s, double *hist) {
  update_xr_kernel<<<kDotBlocks, 256, 0, s>>>(n, x, r, p, q, partial, scal, hist);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_update_p(long long n, double *p, const double *z, const double *scal, cudaStream_t s) {
  update_p_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, p, z, scal);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_seg_dot(const int4 *chunk, int nchunk, const int *cptr, int nprob, const double *a,
                           const double *b, double *partial, double *scal, int *done, int *iters,
                           int slot, int op, double tol2, cudaStream_t s) {
  seg_dot_kernel<<<nchunk, 256, 0, s>>>(chunk, a, b, partial);
  seg_finalize_kernel<<<nprob, 128, 0, s>>>(cptr, nchunk, partial, scal, done, iters, slot, op, 0, tol2);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_seg_update_xr(const int4 *chunk, int nchunk, const int *cptr, int nprob, double *x,
                                 double *r, const double *p, const double *q, double *partial,
                                 double *scal, int *done, int *iters, double tol2, cudaStream_t s) {
  seg_update_xr_kernel<<<nchunk, 256, 0, s>>>(chunk, x, r, p, q, scal, partial);
  seg_finalize_kernel<<<nprob, 128, 0, s>>>(cptr, nchunk, partial, scal, done, iters, S_RR, 2, 0, tol2);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_seg_dot2(const int4 *chunk, int nchunk, const int *cptr, int nprob, const double *r,
                            const double *z, const double *q, double *partial, double *scal, int *done,
                            int *iters, int flexible, cudaStream_t s) {
  seg_dot2_kernel<<<nchunk, 256, 0, s>>>(chunk, nchunk, r, z, q, partial);
  seg_finalize_kernel<<<nprob, 128, 0, s>>>(cptr, nchunk, partial, scal, done, iters, S_RZNEW, 3, flexible,
                                            0.0);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_seg_update_p(const int4 *chunk, int nchunk, double *p, const double *z,
                                const double *scal, cudaStream_t s) {
  seg_update_p_kernel<<<nchunk, 256, 0, s>>>(chunk, p, z, scal);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_gemv_batch(int nrows, const int *rowprob, const long long *aoff, const int *cstart,
                              const int *csz, const double *A, const double *x, double *y,
                              cudaStream_t s) {
  const int threads = 256;
  const int grid = (int)(((long long)nrows * 32 + threads - 1) / threads);
  gemv_batch_kernel<<<grid, threads, 0, s>>>(nrows, rowprob, aoff, cstart, csz, A, x, y);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace rmd

