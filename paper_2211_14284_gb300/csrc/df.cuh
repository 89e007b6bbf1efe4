// Number types and helpers shared by the operator-apply kernels (general
// and Cartesian cells): the signed D-hat term tables, double-float
// arithmetic and the dot-product accumulator.
#pragma once

#include <type_traits>
#include <utility>

#include "device.cuh"

namespace rmd {
namespace {

// Reference exterior derivative D-hat of V^k into component t of V^{k+1}
// as a sum of signed 1D derivative terms: term s reads component src of V^k
// and differentiates along direction dir with sign sgn (grad, curl, div).
struct DTerm {
  int src, dir, sgn;
};
__constant__ int c_nterms[3][3] = {{1, 1, 1}, {2, 2, 2}, {3, 0, 0}};
__constant__ DTerm c_terms[3][3][3] = {
    {{{0, 0, 1}}, {{0, 1, 1}}, {{0, 2, 1}}},
    {{{2, 1, 1}, {1, 2, -1}}, {{0, 2, 1}, {2, 0, -1}}, {{1, 0, 1}, {0, 1, -1}}},
    {{{0, 0, 1}, {1, 1, 1}, {2, 2, 1}}, {}, {}}};
// The same table as constant expressions (compile-time kernels).
__host__ __device__ constexpr int dterm_count(int k, int t) {
  return k == 0 ? 1 : (k == 1 ? 2 : (t == 0 ? 3 : 0));
}
__host__ __device__ constexpr DTerm dterm(int k, int t, int s) {
  return k == 0   ? DTerm{0, t, 1}
         : k == 1 ? (s == 0 ? DTerm{(t + 2) % 3, (t + 1) % 3, 1} : DTerm{(t + 1) % 3, (t + 2) % 3, -1})
                  : DTerm{s, s, 1};
}

// ---- compile-time shapes and loops ---------------------------------------------
// local size per direction of a component of V^kk on a cell of degree p
__host__ __device__ constexpr int sld(int kk, int p, int m, int d) { return styp(kk, m, d) ? p + 1 : p; }
// every component of V^kk has the same local size on a cell
__host__ __device__ constexpr int csize(int kk, int p) {
  return sld(kk, p, 0, 0) * sld(kk, p, 0, 1) * sld(kk, p, 0, 2);
}
template <int... I, typename F>
__device__ __forceinline__ void sfor_seq(std::integer_sequence<int, I...>, F &&f) {
  (f(std::integral_constant<int, I>{}), ...);
}
// f(integral_constant<int, i>) for i = 0 .. N-1, unrolled at compile time
template <int N, typename F>
__device__ __forceinline__ void sfor(F &&f) {
  sfor_seq(std::make_integer_sequence<int, N>{}, f);
}

// ---- number types of the general apply --------------------------------------
// The general apply runs in "double-float" arithmetic: a value is the
// unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi) / 2, about 48
// significant bits), operated on with the error-free transformations of
// Knuth (two-sum) and Dekker (two-product, here through one FMA).  On GB300
// the FP32 pipe runs 64x the FP64 rate, so a double-float FMA (~15 FP32
// instructions) beats one FP64 FMA by ~4x, at ~1e-14 relative accuracy.
// The same templates instantiate with double.
struct DF {
  float hi, lo;
};
static_assert(sizeof(DF) == sizeof(double), "DF arrays share the double layout");

// s + e = a + b exactly
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// s + e = a + b exactly when |a| >= |b| or a = 0
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ double rzero(double) { return 0.0; }
__device__ __forceinline__ DF rzero(DF) { return {0.f, 0.f}; }
__device__ __forceinline__ double rone(double) { return 1.0; }
__device__ __forceinline__ DF rone(DF) { return {1.f, 0.f}; }
__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ DF rfma(DF a, DF b, DF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);  // a.hi b.hi = p + e exactly
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const DF s = two_sum(p, c.hi);
  return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, c.lo), e));
}
__device__ __forceinline__ double radd(double a, double b) { return a + b; }
__device__ __forceinline__ DF radd(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo));
}
__device__ __forceinline__ double rneg(double a) { return -a; }
__device__ __forceinline__ DF rneg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ double rsub(double a, double b) { return a - b; }
__device__ __forceinline__ DF rsub(DF a, DF b) { return radd(a, rneg(b)); }
__device__ __forceinline__ double rmul(double a, double b) { return a * b; }
__device__ __forceinline__ DF rmul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
template <typename R>
__device__ __forceinline__ R rfrom(double x);
template <>
__device__ __forceinline__ double rfrom<double>(double x) { return x; }
template <>
__device__ __forceinline__ DF rfrom<DF>(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double rto(double a) { return a; }
__device__ __forceinline__ double rto(DF a) { return (double)a.hi + (double)a.lo; }

// The conversions between FP64 and double-float without the FP64 pipe
// (1/64 of the FP32 rate on GB300), by integer operations on the bit
// patterns.  df_split: hi = the leading 24 significand bits of x (truncated),
// lo = the next 24 (truncated), so hi + lo agrees with x to 2^-48 relative;
// zero maps to zero.  |x| < 2^-70 (lo would leave the FP32 range) and
// |x| >= 2^127 take the FP64 conversion rfrom<DF> in a function of its own,
// so that the common path is a real branch around it: an inlined rare path
// would be predicated and its FP64 instructions issued for every element.
__device__ __noinline__ DF df_split_rare(double x) { return rfrom<DF>(x); }
__device__ __forceinline__ DF df_split(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  if ((bits << 1) == 0ULL) return {__uint_as_float((unsigned)(bits >> 32)), 0.f};  // +-0
  const int e = (int)((bits >> 52) & 0x7FF) - 1023;  // unbiased exponent
  if (e < -70 || e > 126) return df_split_rare(x);   // tiny, huge, inf, nan: rare
  const unsigned sign = (unsigned)(bits >> 32) & 0x80000000u;
  const unsigned long long frac = bits & 0xFFFFFFFFFFFFFULL;
  const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(frac >> 29));
  const unsigned r = (unsigned)(frac & 0x1FFFFFFFu);  // the 29 bits below hi, weight 2^(e - 52)
  if (r == 0u) return {hi, 0.f};
  const int lead = 31 - __clz(r);                     // 0 .. 28
  const unsigned m = lead >= 23 ? (r >> (lead - 23)) : (r << (23 - lead));
  const float lo = __uint_as_float(sign | ((unsigned)(e - 52 + lead + 127) << 23) | (m & 0x7FFFFFu));
  return {hi, lo};
}
// FP64 <-> the apply's number type: the integer split for double-float
template <typename R>
__device__ __forceinline__ R to_r(double x);
template <>
__device__ __forceinline__ double to_r<double>(double x) { return x; }
template <>
__device__ __forceinline__ DF to_r<DF>(double x) { return df_split(x); }
// an FP32 value as FP64, by its bits (exact): normal numbers and zeros
// inline; subnormals, infinities and NaN in a function of its own (as for
// df_split, so that the common path does not issue FP64 instructions)
__device__ __noinline__ double f2d_rare(float f) { return (double)f; }
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFFu;
  if ((u << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));  // +-0
  if (ex == 0u || ex == 0xFFu) return f2d_rare(f);
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(ex - 127 + 1023) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}
// hi + lo in FP64: the two exact conversions by bits and one FP64 add
__device__ __forceinline__ double df_to_double(DF a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(DF a) { return df_to_double(a); }

// Dot-product accumulator: for double-float, the compensated scheme of
// Ogita, Rump and Oishi (Dot2): the running sum h and a compensation l take
// every exact product a.hi b.hi = p + e (plus the cross terms) through one
// two-sum of h and p, and the pair is renormalised once at the end -- about
// 12 FP32 instructions per term instead of a full double-float FMA's 15.
template <typename R>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  Acc() = default;
  __device__ __forceinline__ explicit Acc(double v) : s(v) {}
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void add_value(double v) { s += v; }
  __device__ __forceinline__ double val() const { return s; }
};
template <>
struct Acc<DF> {
  float h = 0.f, l = 0.f;
  Acc() = default;
  __device__ __forceinline__ explicit Acc(DF v) : h(v.hi), l(v.lo) {}
  // the pair v.hi + v.lo taken in like a product's p + e
  __device__ __forceinline__ void add_value(DF v) {
    const DF t = two_sum(h, v.hi);
    h = t.hi;
    l = __fadd_rn(l, __fadd_rn(t.lo, v.lo));
  }
  __device__ __forceinline__ void add(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const DF t = two_sum(h, p);
    h = t.hi;
    l = __fadd_rn(l, __fadd_rn(t.lo, e));
  }
  __device__ __forceinline__ DF val() const { return fast_two_sum(h, l); }
};

// Store modes of the 1D contractions: out = s, out += s, out -= s, out = -s
// (the D-hat terms carry signs +-1; no multiply is spent on them).
enum { SET = 0, ADD = 1, SUB = 2, NEG = 3 };
template <int MODE, typename R>
__device__ __forceinline__ void put(R &o, R s) {
  if (MODE == SET) o = s;
  else if (MODE == ADD) o = radd(o, s);
  else if (MODE == SUB) o = rsub(o, s);
  else o = rneg(s);
}

}  // namespace
}  // namespace rmd
