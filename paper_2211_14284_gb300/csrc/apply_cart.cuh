// Operator apply on axis-aligned (Cartesian) cells, y = A x, where the cell
// matrix of Eq. sum-factorization is a Kronecker sum of the 1D FDM factors
// (Sec. 2.2-2.4): the mass of V^k is c_m (x)_d F_d per component m (F_d =
// B-hat along an s-type direction, I along an r-type one; c_m the box
// metric times beta), the derivative term D-hat^T (alpha M^{k+1}) D-hat.
// B-hat is the identity on the interior functions plus a 2x2 block on the
// interface pair {0, p}; a row of D-hat has at most three nonzeros (columns
// 0, p and its own index).  No quadrature: ~30 flops per DOF.
//
// Two launches, no atomics, bitwise reproducible:
//  * cart_local_kernel<K, P, R>: the cell products y_K = A_K x_K, one CTA per
//    CPB cells with one thread per line of a cell (cart_cpb, cart_threads),
//    every shape and loop bound a compile-time constant of (K, P); written
//    unassembled, with coalesced stores, to the scratch Y (cart_y_index) in
//    the number type R;
//  * cart_assemble_kernel<K, P, R>: every lattice entry sums its (at most 8)
//    cell contributions from Y in a fixed order, in R, and converts once to
//    FP64; Dirichlet entries get 0.
// The double-float instances convert between FP64 and pairs of FP32 by
// integer operations on the bit patterns (df_split, df_to_double), off the
// FP64 pipe.
// R = double (FP64) or DF (double-float, df.cuh), chosen per handle.
//
// This header holds the templates; apply_cart_part.cu instantiates them for
// one space k (P = 1..15, both number types), compiled once per k.
#pragma once
#include "df.cuh"

namespace rmd {
// launch the (K, A.p) instantiation (apply_cart_part.cu); writes every entry of y
template <int K>
cudaError_t launch_cart_part(const ApplyDev &A, const double *x, double *y, cudaStream_t s);
// the assembly alone (the general apply's second kernel): y from the cell
// products in A.Y; writes every entry of y
template <int K>
cudaError_t launch_cart_assemble_part(const ApplyDev &A, double *y, cudaStream_t s);

namespace {

constexpr int kCartMaxP = 15;

template <int K, int P>
struct CartShape {
  static constexpr int NC0 = ncomp(K), NC1 = ncomp(K + 1);
  static constexpr int S0 = csize(K, P), S1 = csize(K + 1, P);  // per component
  static constexpr int L0 = NC0 * S0, L1 = NC1 * S1;
  static constexpr int NTERMS = K == 1 ? 6 : 3;                 // signed D-hat terms
  static constexpr int LMAX = (P + 1) * (P + 1);                // lines per term (bound)
  static constexpr int LS = NTERMS * LMAX * 2;                  // interface line sums
  // cells per CTA and threads: one thread per line of the largest phase
  static constexpr int CPB = cart_cpb(P), NT = cart_threads(P);
  static_assert(CPB * LMAX <= NT, "every thread owns at most one line of a component");
  // shared memory in units of R (8 bytes): D-hat, per cell 8 coefficients,
  // x, d (later dy), line sums
  static constexpr int SMEM = P * (P + 1) + CPB * (8 + L0 + L1 + LS);
  static_assert(SMEM == cart_local_smem_doubles(K, P, L0, L1), "host and device agree on the layout");
};

// (t, s) of the ts-th signed D-hat term: two per target component for the
// curl, one per target for the gradient, three into the one divergence target
__host__ __device__ constexpr int term_t(int k, int ts) { return k == 1 ? ts >> 1 : (k == 0 ? ts : 0); }
__host__ __device__ constexpr int term_s(int k, int ts) { return k == 1 ? ts & 1 : (k == 0 ? 0 : ts); }

// (x)_d F_d at local index (i0, i1, i2) of one component block `in` with
// local sizes (L0, L1, .) and s-type flags (T0, T1, T2): an s-type index on
// the interface {0, P} couples to itself with weight a and to the opposite
// index P - i with weight b; every other index only to itself.
template <bool T0, bool T1, bool T2, int LL0, int LL1, int P, typename R>
__device__ __forceinline__ R kron_mass(const R *in, int i0, int i1, int i2, R a, R b) {
  const bool f0 = T0 && (i0 == 0 || i0 == P), f1 = T1 && (i1 == 0 || i1 == P),
             f2 = T2 && (i2 == 0 || i2 == P);
  auto line = [&](int base) -> R {
    const R v = in[base + i0];
    return f0 ? rfma(b, in[base + P - i0], rmul(a, v)) : v;
  };
  auto plane = [&](int j2) -> R {
    const int b2 = LL0 * LL1 * j2;
    const R v = line(b2 + LL0 * i1);
    return f1 ? rfma(b, line(b2 + LL0 * (P - i1)), rmul(a, v)) : v;
  };
  const R v = plane(i2);
  return f2 ? rfma(b, plane(P - i2), rmul(a, v)) : v;
}


// Lines along direction 0 of a component block with local sizes (., L1, L2),
// in the CTA's CPB cells: f(cb, i1, i2) for the calling thread's line, if it
// owns one (CPB L1 L2 <= NT: at most one line per thread).
template <int CPB, int NT, int LL1, int LL2, typename F>
__device__ __forceinline__ void for_lines(F &&f) {
  constexpr int NL = LL1 * LL2;
  static_assert(CPB * NL <= NT, "one line per thread");
  const int u = threadIdx.x;
  if (u < CPB * NL) {
    const int cb = u / NL, r = u - cb * NL;
    f(cb, r % LL1, r / LL1);
  }
}

// (x)_d F_d on the whole line (i1, i2) of a component block `in` (local sizes
// LL0, LL1, .): the lines at P - i1 and P - i2 enter where i1, i2 lie on the
// s-type interface {0, P} (weights a on the own index, b on the opposite
// one), then the same along direction 0 at the compile-time ends.
template <bool T0, bool T1, bool T2, int LL0, int LL1, int P, typename R>
__device__ __forceinline__ void line_mass(const R *in, int i1, int i2, R a, R b, R (&u)[LL0]) {
  const bool f1 = T1 && (i1 == 0 || i1 == P), f2 = T2 && (i2 == 0 || i2 == P);
  const R *l00 = in + LL0 * (i1 + LL1 * i2);
  R w[LL0];
#pragma unroll
  for (int i0 = 0; i0 < LL0; ++i0) w[i0] = l00[i0];
  if (f1) {
    const R *l10 = in + LL0 * ((P - i1) + LL1 * i2);
#pragma unroll
    for (int i0 = 0; i0 < LL0; ++i0) w[i0] = rfma(b, l10[i0], rmul(a, w[i0]));
  }
  if (f2) {
    const R *l01 = in + LL0 * (i1 + LL1 * (P - i2));
    R v[LL0];
#pragma unroll
    for (int i0 = 0; i0 < LL0; ++i0) v[i0] = l01[i0];
    if (f1) {
      const R *l11 = in + LL0 * ((P - i1) + LL1 * (P - i2));
#pragma unroll
      for (int i0 = 0; i0 < LL0; ++i0) v[i0] = rfma(b, l11[i0], rmul(a, v[i0]));
    }
#pragma unroll
    for (int i0 = 0; i0 < LL0; ++i0) w[i0] = rfma(b, v[i0], rmul(a, w[i0]));
  }
  if constexpr (T0) {
#pragma unroll
    for (int i0 = 0; i0 < LL0; ++i0) u[i0] = (i0 == 0 || i0 == P) ? rfma(b, w[P - i0], rmul(a, w[i0])) : w[i0];
  } else {
#pragma unroll
    for (int i0 = 0; i0 < LL0; ++i0) u[i0] = w[i0];
  }
}

// Position of entry (i0, i1, i2) of component m of cell c in the scratch Y
// of unassembled cell products: component-major, then cell, then the local
// entry ([m][cell][i2][i1][i0]), so that the CPB consecutive cells of a CTA
// own one contiguous run of every component.
template <int K, int P>
__device__ __forceinline__ size_t cart_y_index(int ncell, int m, size_t c, int i0, int i1, int i2) {
  using Sh = CartShape<K, P>;
  const bool s0 = m == 0 ? styp(K, 0, 0) : (m == 1 ? styp(K, 1, 0) : styp(K, 2, 0));
  const bool s1 = m == 0 ? styp(K, 0, 1) : (m == 1 ? styp(K, 1, 1) : styp(K, 2, 1));
  const int l0 = s0 ? P + 1 : P, l1 = s1 ? P + 1 : P;
  return ((size_t)m * ncell + c) * Sh::S0 + i0 + l0 * (i1 + l1 * i2);
}

template <int K, int P, typename R>
__global__ void __launch_bounds__(cart_threads(P)) cart_local_kernel(ApplyDev A, const double *__restrict__ x,
                                                                    R *__restrict__ Y) {
  using Sh = CartShape<K, P>;
  constexpr int NC0 = Sh::NC0, NC1 = Sh::NC1, S0 = Sh::S0, S1 = Sh::S1, L0 = Sh::L0, L1 = Sh::L1;
  constexpr int CPB = Sh::CPB, LMAX = Sh::LMAX, LS = Sh::LS, NT = Sh::NT;
  constexpr int Q1 = P + 1;
  extern __shared__ double smd[];
  R *sm = reinterpret_cast<R *>(smd);
  R *D1 = sm;                    // D-hat, P x (P + 1)
  R *coef = D1 + P * Q1;         // per cell: beta c_m (NC0), then alpha c'_t (NC1)
  R *xl = coef + CPB * 8;        // CPB x L0
  R *dl = xl + CPB * L0;         // CPB x L1: d = D-hat x, then dy in place
  R *ls = dl + CPB * L1;         // CPB x LS: interface line sums
  __shared__ long long cbase[32][3];  // lattice index of local (0,0,0) per component
  __shared__ int cdir[32];            // Dirichlet faces: bit 2d low side, 2d+1 high side
  if (A.done && A.done[A.prob]) return;  // a converged problem of a batch (uniform per CTA)
  const int tid = threadIdx.x;
  const int ncell = A.n[0] * A.n[1] * A.n[2];
  const int c0 = blockIdx.x * CPB;
  // every FP64 value enters through the integer split (to_r): the FP64 pipe
  // runs at 1/64 of the FP32 rate on GB300
  {
    const double *g = A.tabs + A.q * Q1 + A.q * P;
    for (int i = tid; i < P * Q1; i += NT) D1[i] = to_r<R>(g[i]);
  }
  for (int i = tid; i < CPB * 8; i += NT) {
    const int c = c0 + i / 8;
    coef[i] = c < ncell ? to_r<R>(A.ccoef[(size_t)c * 8 + (i & 7)]) : rzero(R());
  }
  if (tid < CPB) {
    const int c = c0 + tid;
    if (c < ncell) {
      const int e0 = c % A.n[0], e1 = (c / A.n[0]) % A.n[1], e2 = c / (A.n[0] * A.n[1]);
      for (int m = 0; m < NC0; ++m)
        cbase[tid][m] = A.off[m] + (long long)e0 * P +
                        (long long)A.N[m][0] * ((long long)e1 * P + (long long)A.N[m][1] * e2 * P);
      int f = 0;
      if (!A.natural) {
        if (e0 == 0) f |= 1;
        if (e0 == A.n[0] - 1) f |= 2;
        if (e1 == 0) f |= 4;
        if (e1 == A.n[1] - 1) f |= 8;
        if (e2 == 0) f |= 16;
        if (e2 == A.n[2] - 1) f |= 32;
      }
      cdir[tid] = f;
    } else {
      for (int m = 0; m < NC0; ++m) cbase[tid][m] = -1;
      cdir[tid] = 0;
    }
  }
  __syncthreads();
  const R ba = to_r<R>(A.bh_a), bb = to_r<R>(A.bh_b);
  // Every phase runs over lines along direction 0: a thread takes one line
  // (cell cb, indices i1, i2) and walks its l0 entries with a compile-time
  // unrolled loop, so index decoding happens once per line and the
  // interface tests along direction 0 fold into constants.
  // ---- gather x (Dirichlet entries and padding cells read as 0) ----
  sfor<NC0>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    constexpr bool t0 = styp(K, m, 0), t1 = styp(K, m, 1), t2 = styp(K, m, 2);
    constexpr int l0 = sld(K, P, m, 0), l1 = sld(K, P, m, 1), l2 = sld(K, P, m, 2);
    for_lines<CPB, NT, l1, l2>([&](int cb, int i1, int i2) {
      const int f = cdir[cb];
      const long long b0 = cbase[cb][m];
      const bool dl_ = (t1 && (((f & 4) && i1 == 0) || ((f & 8) && i1 == P))) ||
                       (t2 && (((f & 16) && i2 == 0) || ((f & 32) && i2 == P)));
      const double *src = x + (b0 >= 0 ? b0 + (long long)A.N[m][0] * (i1 + (long long)A.N[m][1] * i2) : 0);
      R *dst = xl + cb * L0 + m * S0 + l0 * (i1 + l1 * i2);
#pragma unroll
      for (int i0 = 0; i0 < l0; ++i0) {
        const bool d = dl_ || (t0 && (((f & 1) && i0 == 0) || ((f & 2) && i0 == P)));
        dst[i0] = to_r<R>((b0 >= 0 && !d) ? src[i0] : 0.0);
      }
    });
  });
  __syncthreads();
  // ---- d = D-hat x ----
  sfor<NC1>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    constexpr int l0 = sld(K + 1, P, t, 0), l1 = sld(K + 1, P, t, 1), l2 = sld(K + 1, P, t, 2);
    for_lines<CPB, NT, l1, l2>([&](int cb, int j1, int j2) {
      Acc<R> acc[l0];
      sfor<dterm_count(K, t)>([&](auto sc) {
        constexpr DTerm T = dterm(K, t, decltype(sc)::value);
        // the source is s-type along T.dir (P + 1 entries), equal elsewhere
        constexpr int sl0 = T.dir == 0 ? Q1 : l0, sl1 = T.dir == 1 ? Q1 : l1;
        const R *src = xl + cb * L0 + T.src * S0;
        auto sg = [&](R v) { return T.sgn > 0 ? v : rneg(v); };
        if constexpr (T.dir == 0) {
          const R *in = src + sl0 * (j1 + sl1 * j2);
#pragma unroll
          for (int j = 0; j < l0; ++j) {
            acc[j].add(D1[j * Q1], sg(in[0]));
            acc[j].add(D1[j * Q1 + P], sg(in[P]));
            if (j >= 1) acc[j].add(D1[j * Q1 + j], sg(in[j]));
          }
        } else {
          const int j = T.dir == 1 ? j1 : j2;
          // the three source lines at index 0, P and j along T.dir
          auto line_at = [&](int i) {
            return T.dir == 1 ? src + sl0 * (i + sl1 * j2) : src + sl0 * (j1 + sl1 * i);
          };
          const R *s0 = line_at(0), *sp = line_at(P), *sj = line_at(j);
          const R d0 = D1[j * Q1], dp = D1[j * Q1 + P], dj = D1[j * Q1 + j];
#pragma unroll
          for (int i0 = 0; i0 < l0; ++i0) {
            acc[i0].add(d0, sg(s0[i0]));
            acc[i0].add(dp, sg(sp[i0]));
            if (j >= 1) acc[i0].add(dj, sg(sj[i0]));
          }
        }
      });
      R *dst = dl + cb * L1 + t * S1 + l0 * (j1 + l1 * j2);
#pragma unroll
      for (int i0 = 0; i0 < l0; ++i0) dst[i0] = acc[i0].val();
    });
  });
  __syncthreads();
  // ---- dy = alpha M^{K+1} d, in place: per component, every thread reads
  // its line's mass into registers, then (after a barrier) overwrites the
  // line; the next component's block is disjoint ----
  sfor<NC1>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    constexpr bool t0 = styp(K + 1, t, 0), t1 = styp(K + 1, t, 1), t2 = styp(K + 1, t, 2);
    constexpr int l0 = sld(K + 1, P, t, 0), l1 = sld(K + 1, P, t, 1), l2 = sld(K + 1, P, t, 2);
    R u[l0];
    for_lines<CPB, NT, l1, l2>([&](int cb, int j1, int j2) {
      line_mass<t0, t1, t2, l0, l1, P>(dl + cb * L1 + t * S1, j1, j2, ba, bb, u);
    });
    __syncthreads();
    for_lines<CPB, NT, l1, l2>([&](int cb, int j1, int j2) {
      R *dst = dl + cb * L1 + t * S1 + l0 * (j1 + l1 * j2);
      const R cm = coef[cb * 8 + 3 + t];
#pragma unroll
      for (int i0 = 0; i0 < l0; ++i0) dst[i0] = rmul(cm, u[i0]);
    });
  });
  __syncthreads();
  // ---- line sums of D-hat^T's interface rows, into the d region: for every
  // term and every line of its target component along the term's direction,
  // (sum_j D[j][0] dy_j, sum_j D[j][P] dy_j) ----
  sfor<Sh::NTERMS>([&](auto tsc) {
    constexpr int ts = decltype(tsc)::value;
    constexpr int t = term_t(K, ts);
    constexpr DTerm T = dterm(K, t, term_s(K, ts));
    constexpr int l0 = sld(K + 1, P, t, 0), l1 = sld(K + 1, P, t, 1), l2 = sld(K + 1, P, t, 2);
    constexpr int la = T.dir == 0 ? l1 : l0, lb = T.dir == 2 ? l1 : l2;
    constexpr int str = T.dir == 0 ? 1 : (T.dir == 1 ? l0 : l0 * l1);
    for (int u = tid; u < CPB * la * lb; u += NT) {
      const int cb = u / (la * lb), line = u - cb * (la * lb);
      const int a = line % la, b = line / la;
      const int c0i = T.dir == 0 ? 0 : a, c1i = T.dir == 0 ? a : (T.dir == 1 ? 0 : b), c2i = T.dir == 2 ? 0 : b;
      const R *in = dl + cb * L1 + t * S1 + c0i + l0 * (c1i + l1 * c2i);
      Acc<R> v0, vp;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const R dj = in[j * str];
        v0.add(D1[j * Q1], dj);
        vp.add(D1[j * Q1 + P], dj);
      }
      ls[cb * LS + 2 * (ts * LMAX + line)] = v0.val();
      ls[cb * LS + 2 * (ts * LMAX + line) + 1] = vp.val();
    }
  });
  __syncthreads();
  // ---- y = beta M^K x + D-hat^T dy; the cell's unassembled product to Y,
  // per component: the lines in registers, then (after every thread has read
  // the component's x block) written over that block, then copied out as
  // one coalesced run per component ----
  sfor<NC0>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    constexpr bool t0 = styp(K, m, 0), t1 = styp(K, m, 1), t2 = styp(K, m, 2);
    constexpr int l0 = sld(K, P, m, 0), l1 = sld(K, P, m, 1), l2 = sld(K, P, m, 2);
    R out[l0];
    for_lines<CPB, NT, l1, l2>([&](int cb, int i1, int i2) {
      Acc<R> acc[l0];
      {
        R u[l0];
        line_mass<t0, t1, t2, l0, l1, P>(xl + cb * L0 + m * S0, i1, i2, ba, bb, u);
        const R cm = coef[cb * 8 + m];
#pragma unroll
        for (int i0 = 0; i0 < l0; ++i0) acc[i0] = Acc<R>(rmul(cm, u[i0]));
      }
      sfor<Sh::NTERMS>([&](auto tsc) {
        constexpr int ts = decltype(tsc)::value;
        constexpr int t = term_t(K, ts);
        constexpr DTerm T = dterm(K, t, term_s(K, ts));
        if constexpr (T.src == m) {
          // the target is r-type along T.dir (P entries), equal elsewhere
          constexpr int tl0 = T.dir == 0 ? P : l0, tl1 = T.dir == 1 ? P : l1;
          const R *lsum = ls + cb * LS + 2 * ts * LMAX;
          const R *dyt = dl + cb * L1 + t * S1;
          auto sg = [&](R v) { return T.sgn > 0 ? v : rneg(v); };
          if constexpr (T.dir == 0) {
            const R *dline = dyt + tl0 * (i1 + tl1 * i2);
#pragma unroll
            for (int i0 = 0; i0 < l0; ++i0) {
              if (i0 == 0 || i0 == P) acc[i0].add_value(sg(lsum[2 * (i1 + tl1 * i2) + (i0 == 0 ? 0 : 1)]));
              else acc[i0].add(D1[i0 * Q1 + i0], sg(dline[i0]));
            }
          } else {
            // one instruction stream for interface and interior lines (a
            // branch would diverge within most warps): an interface line
            // adds its line sums (weight 1, stride 2), an interior line
            // D[i][i] times its dy line
            const int i = T.dir == 1 ? i1 : i2;
            const bool itf = i == 0 || i == P;
            const int b = T.dir == 1 ? i2 : i1;
            const R *src = itf ? lsum + 2 * tl0 * b + (i == 0 ? 0 : 1) : dyt + tl0 * (i1 + tl1 * i2);
            const int stride = itf ? 2 : 1;
            const int id = itf ? 0 : i;
            const R co = itf ? rone(R()) : D1[id * Q1 + id];
#pragma unroll
            for (int i0 = 0; i0 < l0; ++i0) acc[i0].add(co, sg(src[i0 * stride]));
          }
        }
      });
#pragma unroll
      for (int i0 = 0; i0 < l0; ++i0) out[i0] = acc[i0].val();
    });
    __syncthreads();
    for_lines<CPB, NT, l1, l2>([&](int cb, int i1, int i2) {
      R *st = xl + cb * L0 + m * S0 + l0 * (i1 + l1 * i2);
#pragma unroll
      for (int i0 = 0; i0 < l0; ++i0) st[i0] = out[i0];
    });
    __syncthreads();
    // the CTA's cells hold one contiguous run of component m in Y
    const int nv = (ncell - c0 < CPB ? ncell - c0 : CPB) * S0;
    R *dst = Y + cart_y_index<K, P>(ncell, m, c0, 0, 0, 0);
    for (int i = tid; i < nv; i += NT) {
      const int cb = i / S0;
      dst[i] = xl[cb * L0 + m * S0 + (i - cb * S0)];
    }
  });
}

// y[g] = sum over the cells holding lattice entry g of their contribution in
// Y, in a fixed order (cells lexicographic, direction 2 outermost);
// Dirichlet entries 0.  A warp takes one lattice row (m, g1, g2) at a
// time (grid-stride over the rows of all components): the cells and local indices along
// directions 1 and 2 are the row's, decoded once; the lanes walk g0, whose
// consecutive entries are consecutive local indices of a cell in Y and
// consecutive entries of y; an entry inside a cell along g0 reads one
// value per run, an interface entry two.
template <int K, int P, typename R>
__global__ void __launch_bounds__(256) cart_assemble_kernel(ApplyDev A, const R *__restrict__ Y,
                                                            double *__restrict__ y) {
  using Sh = CartShape<K, P>;
  constexpr int NC0 = Sh::NC0;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int ncell = A.n[0] * A.n[1] * A.n[2];
  const bool frozen = A.done && A.done[A.prob];  // a converged problem of a batch: y = 0
  // the rows of every component form one range of work items, so a small
  // lattice's components are assembled in one pass of the warps
  int total = 0;
  for (int m = 0; m < NC0; ++m) total += A.N[m][1] * A.N[m][2];
  for (int w = gw; w < total; w += nw) {
    int start = 0;
    sfor<NC0>([&](auto mc) {
      constexpr int m = decltype(mc)::value;
      constexpr bool st0 = styp(K, m, 0), st1 = styp(K, m, 1), st2 = styp(K, m, 2);
      const int N0 = A.N[m][0], N1 = A.N[m][1], rows = A.N[m][1] * A.N[m][2];
      const int row = w - start;
      start += rows;
      if (row >= 0 && row < rows) {
        const int g1 = row % N1, g2 = row / N1;
        // (cell, local index) pairs along a direction: two on an interior
        // s-type interface plane, else one; dir: a Dirichlet plane
        bool dir = false;
        auto pairs = [&](bool st, int g, int nd, int (&ce)[2], int (&ci)[2], int &nc) {
          const int e = g / P, i = g - e * P;
          if (st && i == 0) {
            if (!A.natural && (g == 0 || e == nd)) dir = true;
            const bool lo = e >= 1, hi = e < nd;
            ce[0] = lo ? e - 1 : e;
            ci[0] = lo ? P : 0;
            ce[1] = e;
            ci[1] = 0;
            nc = (lo && hi) ? 2 : 1;
          } else {
            ce[0] = ce[1] = e;
            ci[0] = ci[1] = i;
            nc = 1;
          }
        };
        int ce1[2], ci1[2], n1, ce2[2], ci2[2], n2;
        pairs(st1, g1, A.n[1], ce1, ci1, n1);
        pairs(st2, g2, A.n[2], ce2, ci2, n2);
        const bool rowdir = dir || frozen;
        // the row's (up to 4) runs in Y: cell (0, e1, e2) at local (0, i1, i2)
        // for each pair along directions 1 and 2 (warp-uniform)
        const R *base[2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int b = 0; b < 2; ++b)
            base[c][b] = Y + cart_y_index<K, P>(ncell, m, (size_t)A.n[0] * (ce1[b] + (size_t)A.n[1] * ce2[c]), 0,
                                                ci1[b], ci2[c]);
        double *yrow = y + A.off[m] + (long long)N0 * row;
        for (int g0 = lane; g0 < N0; g0 += 32) {
          int ce0[2], ci0[2], n0;
          dir = rowdir;
          pairs(st0, g0, A.n[0], ce0, ci0, n0);
          const int o0 = ce0[0] * Sh::S0 + ci0[0], o1 = ce0[1] * Sh::S0 + ci0[1];
          R s = rzero(R());
          if (!dir) {
            // fixed order: direction 2 outermost, then 1, then 0
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
              for (int b = 0; b < 2; ++b)
                if (c < n2 && b < n1) {
                  const R v0 = base[c][b][o0];
                  s = (c == 0 && b == 0) ? v0 : radd(s, v0);
                  if (n0 == 2) s = radd(s, base[c][b][o1]);
                }
          }
          yrow[g0] = to_double(s);
        }
      }
    });
  }
}

template <int K, int P, typename R>
cudaError_t launch_assemble_kpr(const ApplyDev &A, double *y, cudaStream_t s) {
  // a grid of resident CTAs (by default 8 per SM), each warp striding over the rows
  int grid = A.asm_grid;
  if (grid <= 0) {
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    grid = 8 * nsm;
  }
  cart_assemble_kernel<K, P, R><<<grid, 256, 0, s>>>(A, reinterpret_cast<const R *>(A.Y), y);
  return cudaGetLastError();
}
template <int K, int P, typename R>
cudaError_t launch_cart_kpr(const ApplyDev &A, const double *x, double *y, cudaStream_t s) {
  using Sh = CartShape<K, P>;
  const size_t smem = (size_t)Sh::SMEM * sizeof(double);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t err =
      cudaFuncSetAttribute(cart_local_kernel<K, P, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int ncell = A.n[0] * A.n[1] * A.n[2];
  cart_local_kernel<K, P, R><<<(ncell + Sh::CPB - 1) / Sh::CPB, Sh::NT, smem, s>>>(A, x, reinterpret_cast<R *>(A.Y));
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_assemble_kpr<K, P, R>(A, y, s);
}
template <int K, int P>
cudaError_t launch_cart_kp(const ApplyDev &A, const double *x, double *y, cudaStream_t s) {
  return A.arith ? launch_cart_kpr<K, P, DF>(A, x, y, s) : launch_cart_kpr<K, P, double>(A, x, y, s);
}
template <int K, int... PS>
cudaError_t launch_cart_range(const ApplyDev &A, const double *x, double *y, cudaStream_t s,
                              std::integer_sequence<int, PS...>) {
  cudaError_t err = cudaErrorInvalidValue;
  ((A.p == PS + 1 ? (err = launch_cart_kp<K, PS + 1>(A, x, y, s), 0) : 0), ...);
  return err;
}
template <int K, int... PS>
cudaError_t launch_assemble_range(const ApplyDev &A, double *y, cudaStream_t s, std::integer_sequence<int, PS...>) {
  cudaError_t err = cudaErrorInvalidValue;
  ((A.p == PS + 1 ? (err = A.arith ? launch_assemble_kpr<K, PS + 1, DF>(A, y, s)
                                   : launch_assemble_kpr<K, PS + 1, double>(A, y, s),
    0)
                  : 0),
   ...);
  return err;
}

}  // namespace
}  // namespace rmd
