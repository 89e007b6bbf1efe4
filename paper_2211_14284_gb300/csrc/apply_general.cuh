// Operator apply on general (trilinear) cells, y = A x with
// A_K = M^k_beta + D-hat^T M^{k+1}_alpha D-hat (Eq. sum-factorization): one
// CTA per cell; the V^k coefficients and their reference exterior
// derivative D-hat x are interpolated to the q^3 GLL points, q =
// ceil(3(p+1)/2), by three 1D contractions staged in shared memory,
// weighted by the pullback metric of the trilinear map (Sec. 3.1),
// contracted back and scatter-added.  Arithmetic in double-float (df.cuh).
//
// The kernel is instantiated per space k and degree p (1 <= p <= 8, the
// shared-memory limit), so every shape, loop count, divisor and table
// offset is a constant.  Each 1D interpolation is split into its even and
// odd halves at the mirrored GLL points x_{q-1-o} = -x_o (eo_tables in
// device.cuh): forward, one thread per mirror pair of points; backward, one
// thread per pair of functions (one with an even part, one with an odd
// part, or the interface pair {0, p}), so all threads of a pass run the same
// instruction stream.
//
// This header holds the kernel templates; apply_general_part.cu instantiates
// them for one space k and a range of four degrees per object (compiled in
// parallel), apply_general.cu dispatches.
#pragma once
#include <type_traits>
#include <utility>

#include "df.cuh"

namespace rmd {
// launch the (K, p) instantiation for p in [PLO, PLO + 3] (apply_general_part.cu)
template <int K, int PLO>
cudaError_t launch_general_part(int p, const ApplyDev &A, const double *x, double *y, cudaStream_t s);

namespace {

// ---- compile-time shapes (sld, csize in df.cuh) --------------------------------
// pullback-metric entries of kk-forms: scalar or symmetric 3x3
__host__ __device__ constexpr int nweights(int kk) { return (kk == 0 || kk == 3) ? 1 : 6; }

template <bool S, int PP>
struct Tab {  // one reflection-split table: Ec[he][nse] Oc[ho][nso] ET[n][he] OT[n][ho]
  static constexpr int q = quad_q(PP), he = (q + 1) / 2, ho = q / 2, n = eo_n(S, PP);
  static constexpr int nse = eo_nse(S, PP), nso = eo_nso(S, PP);
  static constexpr int oOc = he * nse, oET = oOc + ho * nso, oOT = oET + n * he;
  // backward units: s-type unit 0 is the interface pair {0, p}, unit u >= 1
  // the interior pair (2u - 1 even part, 2u odd part); r-type unit u the
  // pair (2u even part, 2u + 1 odd part).  A missing member is -1.
  static constexpr int nu = S ? 1 + PP / 2 : (PP + 1) / 2;
};
template <bool S, int PP>
__device__ __forceinline__ int unit_even(int u) {
  return S ? (u == 0 ? 0 : (2 * u - 1 <= PP - 1 ? 2 * u - 1 : -1)) : (2 * u < PP ? 2 * u : -1);
}
template <bool S, int PP>
__device__ __forceinline__ int unit_odd(int u) {
  return S ? (u == 0 ? 0 : (2 * u <= PP - 1 ? 2 * u : -1)) : (2 * u + 1 < PP ? 2 * u + 1 : -1);
}

constexpr int NT = kApplyThreadsGeneral;

// out[c][o][a] (op)= sum_i T[o][i] in[c][i][a]  (i < n functions, o < q
// points): one thread per mirror pair (o, q-1-o), the even and odd halves
// as two interleaved chains.
template <int MODE, bool S, int PP, int C, int A, typename R>
__device__ __forceinline__ void fwd(const R *__restrict__ in, R *__restrict__ out, const R *__restrict__ tab) {
  using T = Tab<S, PP>;
  constexpr int q = T::q, he = T::he, ho = T::ho, n = T::n, nse = T::nse, nso = T::nso;
  constexpr int nm = nse > nso ? nse : nso;
  for (int idx = threadIdx.x; idx < C * he * A; idx += NT) {
    const int a = idx % A, o = (idx / A) % he, c = idx / (A * he);
    const R *xv = in + (c * n) * A + a;
    const R *er = tab + o * nse;
    R *yv = out + (c * q) * A + a;
    Acc<R> ea;
    if (o < ho) {
      const R *orow = tab + T::oOc + o * nso;
      Acc<R> oa;
#pragma unroll
      for (int k = 0; k < nm; ++k) {
        if (k < nse) ea.add(er[k], xv[eo_se(S, PP, k) * A]);
        if (k < nso) oa.add(orow[k], xv[eo_so(S, PP, k) * A]);
      }
      const R ev = ea.val(), od = oa.val();
      put<MODE>(yv[o * A], radd(ev, od));
      put<MODE>(yv[(q - 1 - o) * A], rsub(ev, od));
    } else {  // the middle point of an odd q
#pragma unroll
      for (int k = 0; k < nse; ++k) ea.add(er[k], xv[eo_se(S, PP, k) * A]);
      put<MODE>(yv[o * A], ea.val());
    }
  }
}

// A folded point index o of w[c][o][a] holds w_o + w_{q-1-o} and its mirror
// q-1-o holds w_o - w_{q-1-o} (o < ho); the middle point of an odd q stays.
// Backward unit u at wv = w + c q A + a: the even-part sum of its first
// member, sum_o E[o][i] w+_o, and the odd-part sum of its second, sum_o
// Od[o][j] w-_o; for the interface pair (E, Od columns of 0, with E[.][p] =
// E[.][0], Od[.][p] = -Od[.][0]) the values at 0 and p are their sum and
// difference.  v[0], v[1] are the values of the unit's two functions.
template <bool S, int PP, int A, typename R>
__device__ __forceinline__ void bwd_unit(const R *__restrict__ wv, const R *__restrict__ tab, int u, R v[2]) {
  using T = Tab<S, PP>;
  constexpr int q = T::q, he = T::he, ho = T::ho;
  const int ie = unit_even<S, PP>(u), io = unit_odd<S, PP>(u);
  const R *er = tab + T::oET + (ie < 0 ? 0 : ie) * he;
  const R *orow = tab + T::oOT + (io < 0 ? 0 : io) * ho;
  Acc<R> se, so;
#pragma unroll
  for (int o = 0; o < he; ++o) {
    se.add(er[o], wv[o * A]);
    if (o < ho) so.add(orow[o], wv[(q - 1 - o) * A]);
  }
  const R e = se.val(), d = so.val();
  if (S && u == 0) {
    v[0] = radd(e, d);
    v[1] = rsub(e, d);
  } else {
    v[0] = e;
    v[1] = d;
  }
}
// the functions of unit u (-1: none)
template <bool S, int PP>
__device__ __forceinline__ void unit_members(int u, int &i0, int &i1) {
  if (S && u == 0) {
    i0 = 0;
    i1 = PP;
  } else {
    i0 = unit_even<S, PP>(u);
    i1 = unit_odd<S, PP>(u);
  }
}

// out[c][i][a] (op)= sum_o T[o][i] w[c][o][a] for a folded w.
template <int MODE, bool S, int PP, int C, int A, typename R>
__device__ __forceinline__ void bwd(const R *__restrict__ w, R *__restrict__ out, const R *__restrict__ tab) {
  using T = Tab<S, PP>;
  constexpr int q = T::q, n = T::n, nu = T::nu;
  for (int idx = threadIdx.x; idx < C * nu * A; idx += NT) {
    const int a = idx % A, u = (idx / A) % nu, c = idx / (A * nu);
    R v[2];
    bwd_unit<S, PP, A>(w + (c * q) * A + a, tab, u, v);
    int i0, i1;
    unit_members<S, PP>(u, i0, i1);
    R *ov = out + (c * n) * A + a;
    if (i0 >= 0) put<MODE>(ov[i0 * A], v[0]);
    if (i1 >= 0) put<MODE>(ov[i1 * A], v[1]);
  }
}
// bwd (SET) storing the result folded along its point index of stride
// A / q (the slowest part of a = o' (A / q) + r): one thread per unit and
// mirror pair (o', q-1-o').
template <bool S, int PP, int C, int A, typename R>
__device__ __forceinline__ void bwd_fold(const R *__restrict__ w, R *__restrict__ out, const R *__restrict__ tab) {
  using T = Tab<S, PP>;
  constexpr int q = T::q, n = T::n, nu = T::nu, he = T::he, ho = T::ho, SS = A / q;
  for (int idx = threadIdx.x; idx < C * nu * he * SS; idx += NT) {
    const int r = idx % SS, of = (idx / SS) % he, u = (idx / (SS * he)) % nu, c = idx / (SS * he * nu);
    const R *wv = w + (c * q) * A + r;
    int i0, i1;
    unit_members<S, PP>(u, i0, i1);
    R *o0 = out + (c * n + (i0 < 0 ? 0 : i0)) * A + r, *o1 = out + (c * n + (i1 < 0 ? 0 : i1)) * A + r;
    R x[2];
    bwd_unit<S, PP, A>(wv + of * SS, tab, u, x);
    if (of < ho) {
      R y[2];
      bwd_unit<S, PP, A>(wv + (q - 1 - of) * SS, tab, u, y);
      if (i0 >= 0) {
        o0[of * SS] = radd(x[0], y[0]);
        o0[(q - 1 - of) * SS] = rsub(x[0], y[0]);
      }
      if (i1 >= 0) {
        o1[of * SS] = radd(x[1], y[1]);
        o1[(q - 1 - of) * SS] = rsub(x[1], y[1]);
      }
    } else {
      if (i0 >= 0) o0[of * SS] = x[0];
      if (i1 >= 0) o1[of * SS] = x[1];
    }
  }
}

// The metric weights at point pt (NW = 1 scalar, NW = 6 symmetric 3x3).
template <int NW, typename R>
__device__ __forceinline__ void weight_at(const R *__restrict__ Gc, const R *U, int q3, int pt, R v[3]) {
  if (NW == 1) {
    v[0] = rmul(U[pt], Gc[pt]);
  } else {
    const R w00 = Gc[pt], w11 = Gc[q3 + pt], w22 = Gc[2 * q3 + pt];
    const R w01 = Gc[3 * q3 + pt], w02 = Gc[4 * q3 + pt], w12 = Gc[5 * q3 + pt];
    const R u0 = U[pt], u1 = U[q3 + pt], u2 = U[2 * q3 + pt];
    v[0] = rfma(w00, u0, rfma(w01, u1, rmul(w02, u2)));
    v[1] = rfma(w01, u0, rfma(w11, u1, rmul(w12, u2)));
    v[2] = rfma(w02, u0, rfma(w12, u1, rmul(w22, u2)));
  }
}
// The weights at every point, every component stored folded along the
// slowest point index (stride q^2): one thread per mirror pair of points.
template <int NW, int PP, typename R>
__device__ __forceinline__ void weight_fold(const R *__restrict__ Gc, R *U) {
  constexpr int q = quad_q(PP), q2 = q * q, q3 = q2 * q, he = (q + 1) / 2, ho = q / 2;
  constexpr int nc = NW == 1 ? 1 : 3;
  for (int idx = threadIdx.x; idx < he * q2; idx += NT) {
    const int r = idx % q2, of = idx / q2;
    const int p1 = of * q2 + r, p2 = (q - 1 - of) * q2 + r;
    R u[3], v[3];
    weight_at<NW>(Gc, U, q3, p1, u);
    if (of < ho) {
      weight_at<NW>(Gc, U, q3, p2, v);
#pragma unroll
      for (int m = 0; m < nc; ++m) {
        U[m * q3 + p1] = radd(u[m], v[m]);
        U[m * q3 + p2] = rsub(u[m], v[m]);
      }
    } else {
#pragma unroll
      for (int m = 0; m < nc; ++m) U[m * q3 + p1] = u[m];
    }
  }
}

// out[c][o][a] (op)= sum_i M[o][i] in[c][i][a] for a dense O x I matrix M
// (the signed D-hat terms).  Output element idx belongs to thread idx mod
// NT in every call of the same output shape, so terms accumulating into the
// same output need no barrier between them.
template <int MODE, int O, int I, int C, int A, typename R>
__device__ __forceinline__ void contract(const R *__restrict__ in, R *__restrict__ out, const R *__restrict__ M) {
  for (int idx = threadIdx.x; idx < C * O * A; idx += NT) {
    const int a = idx % A, o = (idx / A) % O, c = idx / (A * O);
    const R *mi = M + o * I;
    const R *xi = in + c * I * A + a;
    Acc<R> s;
#pragma unroll
    for (int i = 0; i < I; ++i) s.add(mi[i], xi[i * A]);
    put<MODE>(out[idx], s.val());
  }
}
// One signed term along direction DIR of an input block with local sizes
// (L0, L1, L2): C x I x A with I the DIR extent.
template <int MODE, int DIR, int O, int I, int L0, int L1, int L2, typename R>
__device__ __forceinline__ void dterm_pass(const R *in, R *out, const R *M) {
  if (DIR == 0) contract<MODE, O, I, L1 * L2, 1>(in, out, M);
  else if (DIR == 1) contract<MODE, O, I, L2, L0>(in, out, M);
  else contract<MODE, O, I, 1, L0 * L1>(in, out, M);
}

// Interpolate component block `in` (local sizes of V^KK component m) to the
// points: U[o2][o1][o0].
template <int KK, int PP, int m, typename R>
__device__ __forceinline__ void to_points(const R *in, R *SA, R *SB, R *Um, const R *tS, const R *tR) {
  constexpr int q = quad_q(PP);
  constexpr bool s0 = styp(KK, m, 0), s1 = styp(KK, m, 1), s2 = styp(KK, m, 2);
  constexpr int l1 = sld(KK, PP, m, 1), l2 = sld(KK, PP, m, 2);
  fwd<SET, s0, PP, l1 * l2, 1>(in, SA, s0 ? tS : tR);
  __syncthreads();
  fwd<SET, s1, PP, l2, q>(SA, SB, s1 ? tS : tR);
  __syncthreads();
  fwd<SET, s2, PP, 1, q * q>(SB, Um, s2 ? tS : tR);
  __syncthreads();
}
// Contract the folded point values Um back onto component m: out (op)= .
template <int MODE, int KK, int PP, int m, typename R>
__device__ __forceinline__ void from_points(const R *Um, R *SA, R *SB, R *out, const R *tS, const R *tR) {
  constexpr int q = quad_q(PP);
  constexpr bool s0 = styp(KK, m, 0), s1 = styp(KK, m, 1), s2 = styp(KK, m, 2);
  constexpr int l1 = sld(KK, PP, m, 1), l2 = sld(KK, PP, m, 2);
  bwd_fold<s2, PP, 1, q * q>(Um, SB, s2 ? tS : tR);
  __syncthreads();
  bwd_fold<s1, PP, l2, q>(SB, SA, s1 ? tS : tR);
  __syncthreads();
  bwd<MODE, s0, PP, l1 * l2, 1>(SA, out, s0 ? tS : tR);
  __syncthreads();
}

// Gather (SCATTER = false: xl = x on the cell, Dirichlet entries 0, yl = 0)
// or store (SCATTER = true: the cell's product yl to its run of the scratch
// P.Y, [component][cell][local entry], coalesced; the assembly kernel sums
// the contributions of every lattice entry in a fixed order, no atomics).
template <bool SCATTER, int KK, int PP, typename R>
__device__ __forceinline__ void cell_io(const ApplyDev &P, const int e[3], const double *__restrict__ x,
                                        double *__restrict__ y, R *xl, R *yl) {
  constexpr int CS = csize(KK, PP);
  if constexpr (SCATTER) {
    const size_t ncell = (size_t)P.n[0] * P.n[1] * P.n[2];
    const size_t c = e[0] + (size_t)P.n[0] * (e[1] + (size_t)P.n[1] * e[2]);
    R *Yr = reinterpret_cast<R *>(P.Y);
    sfor<ncomp(KK)>([&](auto mc) {
      constexpr int m = decltype(mc)::value;
      R *dst = Yr + ((size_t)m * ncell + c) * CS;
      for (int l = threadIdx.x; l < CS; l += NT) dst[l] = yl[m * CS + l];
    });
    return;
  }
  sfor<ncomp(KK)>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    constexpr int l0 = sld(KK, PP, m, 0), l1 = sld(KK, PP, m, 1);
    for (int l = threadIdx.x; l < CS; l += NT) {
      const int i1 = l % l0, i2 = (l / l0) % l1, i3 = l / (l0 * l1);
      const int g1 = e[0] * PP + i1, g2 = e[1] * PP + i2, g3 = e[2] * PP + i3;
      const bool dir = !P.natural && ((styp(KK, m, 0) && (g1 == 0 || g1 == P.n[0] * PP)) ||
                       (styp(KK, m, 1) && (g2 == 0 || g2 == P.n[1] * PP)) ||
                       (styp(KK, m, 2) && (g3 == 0 || g3 == P.n[2] * PP)));
      const long long gi = P.off[m] + g1 + (long long)P.N[m][0] * (g2 + (long long)P.N[m][1] * g3);
      xl[m * CS + l] = to_r<R>(dir ? 0.0 : x[gi]);
      yl[m * CS + l] = rzero(R());
    }
  });
}

template <int K, int PP, typename R>
__global__ void __launch_bounds__(kApplyThreadsGeneral) apply_kernel(ApplyDev P, const double *__restrict__ x,
                                                              double *__restrict__ y) {
  constexpr int p = PP, q = quad_q(PP), q3 = q * q * q;
  constexpr int NC0 = ncomp(K), NC1 = ncomp(K + 1), CS0 = csize(K, PP), CS1 = csize(K + 1, PP);
  constexpr int EOS = eo_size(true, PP), EOD = EOS + eo_size(false, PP);
  extern __shared__ double smd[];
  R *sm = reinterpret_cast<R *>(smd);
  R *tS = sm, *tR = sm + EOS;
  R *D1 = sm + EOD;
  R *D1T = D1 + p * (p + 1);
  R *xl = D1T + p * (p + 1);
  R *yl = xl + NC0 * CS0;
  R *dl = yl + NC0 * CS0;
  R *dyl = dl + NC1 * CS1;
  R *U = dyl + NC1 * CS1;
  R *SA = U + 3 * q3;
  R *SB = SA + q * (p + 1) * (p + 1);
  const int tid = threadIdx.x;
  const int c = blockIdx.x;
  const int e[3] = {c % P.n[0], (c / P.n[0]) % P.n[1], c / (P.n[0] * P.n[1])};
  {
    const double *g = P.tabs + q * (p + 1) + q * p;
    for (int i = tid; i < p * (p + 1); i += NT) {
      D1[i] = to_r<R>(g[i]);
      D1T[(i % (p + 1)) * p + i / (p + 1)] = to_r<R>(g[i]);
    }
    g += p * (p + 1) + 2 * q;
    for (int i = tid; i < EOD; i += NT) sm[i] = to_r<R>(g[i]);
  }
  cell_io<false, K, PP>(P, e, x, y, xl, yl);
  __syncthreads();
  const R *Gc = static_cast<const R *>(P.G) + (size_t)c * (nweights(K) + nweights(K + 1)) * q3;
  // ---- stage A: (v, beta u) on V^k ----
  sfor<NC0>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    to_points<K, PP, m>(xl + m * CS0, SA, SB, U + m * q3, tS, tR);
  });
  weight_fold<nweights(K), PP>(Gc, U);
  __syncthreads();
  sfor<NC0>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    from_points<ADD, K, PP, m>(U + m * q3, SA, SB, yl + m * CS0, tS, tR);
  });
  // ---- stage B: (d v, alpha d u) on V^{k+1}, d = D-hat ----
  sfor<NC1>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    sfor<dterm_count(K, t)>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      constexpr DTerm T = dterm(K, t, s);
      constexpr int mode = s == 0 ? (T.sgn > 0 ? SET : NEG) : (T.sgn > 0 ? ADD : SUB);
      dterm_pass<mode, T.dir, p, p + 1, sld(K, PP, T.src, 0), sld(K, PP, T.src, 1), sld(K, PP, T.src, 2)>(
          xl + T.src * CS0, dl + t * CS1, D1);
    });
  });
  __syncthreads();
  sfor<NC1>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    to_points<K + 1, PP, t>(dl + t * CS1, SA, SB, U + t * q3, tS, tR);
  });
  weight_fold<nweights(K + 1), PP>(Gc + nweights(K) * q3, U);
  __syncthreads();
  sfor<NC1>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    from_points<SET, K + 1, PP, t>(U + t * q3, SA, SB, dyl + t * CS1, tS, tR);
  });
  sfor<NC1>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    sfor<dterm_count(K, t)>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      constexpr DTerm T = dterm(K, t, s);
      constexpr int mode = T.sgn > 0 ? ADD : SUB;
      dterm_pass<mode, T.dir, p + 1, p, sld(K + 1, PP, t, 0), sld(K + 1, PP, t, 1),
                 sld(K + 1, PP, t, 2)>(dyl + t * CS1, yl + T.src * CS0, D1T);
    });
  });
  __syncthreads();
  cell_io<true, K, PP>(P, e, x, y, xl, yl);
}

template <int K, int PP, typename R>
cudaError_t launch_kpr(const ApplyDev &A, const double *x, double *y, cudaStream_t s) {
  const size_t smem = general_smem_doubles(K, PP) * sizeof(double);  // sizeof(R) == sizeof(double)
  cudaError_t err =
      cudaFuncSetAttribute(apply_kernel<K, PP, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  apply_kernel<K, PP, R><<<A.n[0] * A.n[1] * A.n[2], kApplyThreadsGeneral, smem, s>>>(A, x, y);
  return cudaGetLastError();
}
template <int K, int PP>
cudaError_t launch_kp(const ApplyDev &A, const double *x, double *y, cudaStream_t s) {
  return A.arith ? launch_kpr<K, PP, DF>(A, x, y, s) : launch_kpr<K, PP, double>(A, x, y, s);
}
template <int K, int PLO, int... PS>
cudaError_t launch_range(int p, const ApplyDev &A, const double *x, double *y, cudaStream_t s,
                         std::integer_sequence<int, PS...>) {
  cudaError_t err = cudaErrorInvalidValue;
  ((p == PLO + PS ? (err = launch_kp<K, PLO + PS>(A, x, y, s), 0) : 0), ...);
  return err;
}

}  // namespace
}  // namespace rmd
