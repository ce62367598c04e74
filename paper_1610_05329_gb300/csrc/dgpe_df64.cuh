// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  The operations run on the
// FP32 pipe, which GB300 issues 64 times as fast as FP64; they follow the classical
// error-free transformations (Dekker 1971; Knuth's TwoSum, TAOCP vol. 2 4.2.2) with the
// FMA-based exact product, as used by double-double libraries (Hida, Li & Bailey 2001):
//   two_sum(a, b):      s = a + b, e = the exact rounding error of s (6 flops);
//   fast_two_sum(a, b): the same for |a| >= |b| (3 flops);
//   two_prod(a, b):     p = a b, e = fma(a, b, -p) exactly.
// Addition is the "sloppy" variant (one two_sum on the high parts, the low parts added in
// FP32): its error is bounded by about 2^-44 of the operands' magnitude, which is what a
// transform or a recurrence needs (errors relative to the data, not to each output).
// Every FP32 operation is an explicit round-to-nearest intrinsic, so nothing is contracted
// or reassociated by the compiler.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace dgpe {

// the global overloads stay visible next to the df ones declared in this namespace
using ::fabs;
using ::fma;

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // A double split into hi = fl32(d) and lo = fl32(d - hi): exact to 48 bits.  constexpr, so
  // the literals of the kernels fold at compile time (at run time it issues FP64 instructions).
  __host__ __device__ explicit constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit constexpr df(float f) : hi(f), lo(0.0f) {}
  // small integers (grid indices, |i| < 2^24) are exact in the high part
  __host__ __device__ explicit constexpr df(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

#ifdef __CUDACC__
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// a b + c with one renormalisation: the exact product's two parts and c are summed with a
// two_sum on the leading terms.
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  const df s = df_two_sum(p, c.hi);
  e = __fadd_rn(e, __fadd_rn(s.lo, c.lo));
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df &operator+=(df &a, df b) { return a = a + b; }
__device__ __forceinline__ df &operator*=(df &a, df b) { return a = a * b; }
__device__ __forceinline__ bool operator==(df a, df b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df a, df b) { return !(a == b); }
__device__ __forceinline__ bool operator>(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(df a, df b) { return b > a; }
__device__ __forceinline__ df fabs(df a) { return a.hi < 0.0f ? -a : a; }
// 2^k a, exact
__device__ __forceinline__ df df_ldexp(df a, int k) { return {ldexpf(a.hi, k), ldexpf(a.lo, k)}; }
// the exact product of two floats as a pair
__device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// Sine and cosine in double-float: r = x - k pi/2 with k = rint(2x/pi), the products k P_i
// of the three-float split of pi/2 taken exactly (two_prod); then Taylor series in r
// (coefficients (-1)^j/(2j+1)! and (-1)^j/(2j)!), through r^15 and r^16 on |r| <= pi/4
// (first omitted terms below 5e-17), or through r^11 and r^10 when |x| <= 1/4 (below 6e-15
// and 1.2e-16 there; the pair itself carries about 2^-48 = 3.6e-15).  |x| >= 4096 and
// non-finite x take the FP64 routine.
__device__ __forceinline__ void sin_cos(df x, df *s, df *c) {
  const float ax = fabsf(x.hi);
  if (ax <= 0.25f) {
    const df u = x * x;
    df ps = df(-2.505210838544172e-08);
    ps = fma(ps, u, df(2.7557319223985893e-06));
    ps = fma(ps, u, df(-0.0001984126984126984));
    ps = fma(ps, u, df(0.008333333333333333));
    ps = fma(ps, u, df(-0.16666666666666666));
    *s = fma(x * u, ps, x);
    df pc = df(-2.755731922398589e-07);
    pc = fma(pc, u, df(2.48015873015873e-05));
    pc = fma(pc, u, df(-0.001388888888888889));
    pc = fma(pc, u, df(0.041666666666666664));
    pc = fma(pc, u, df(-0.5));
    *c = fma(u, pc, df(1.0f));
    return;
  }
  if (!(ax < 4096.0f)) {
    double sd, cd;
    sincos((double)x, &sd, &cd);
    *s = df(sd);
    *c = df(cd);
    return;
  }
  const float k = rintf(__fmul_rn(x.hi, 0.6366197466850281f));
  const int q = ((int)k) & 3;
  df r = x - df_two_prod(k, 1.5707963705062866f);
  r = r - df_two_prod(k, -4.371138828673793e-08f);
  r = r - df{__fmul_rn(k, -1.7151245100058819e-15f), 0.0f};
  const df u = r * r;
  df ps = df(7.647163731819816e-13);
  ps = fma(ps, u, df(-1.6059043836821613e-10));
  ps = fma(ps, u, df(2.505210838544172e-08));
  ps = fma(ps, u, df(-2.7557319223985893e-06));
  ps = fma(ps, u, df(0.0001984126984126984));
  ps = fma(ps, u, df(-0.008333333333333333));
  ps = fma(ps, u, df(0.16666666666666666));
  const df sr = r - (r * u) * ps;
  df pc = df(4.779477332387385e-14);
  pc = fma(pc, u, df(-1.1470745597729725e-11));
  pc = fma(pc, u, df(2.08767569878681e-09));
  pc = fma(pc, u, df(-2.755731922398589e-07));
  pc = fma(pc, u, df(2.48015873015873e-05));
  pc = fma(pc, u, df(-0.001388888888888889));
  pc = fma(pc, u, df(0.041666666666666664));
  pc = fma(pc, u, df(-0.5));
  const df cr = fma(u, pc, df(1.0f));
  switch (q) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
  }
}

// e^x in double-float: x = k ln2 + r, k = rint(x / ln2), k ln2 subtracted through the
// exact products of a three-float split of ln2; e^r by its Taylor series through r^12 on
// |r| <= ln2/2 (first omitted term below 2e-16); then 2^k exactly.
__device__ __forceinline__ df exp_r(df x) {
  if (!(x.hi > -100.0f)) return x.hi < 0.0f ? df{0.0f, 0.0f} : df{x.hi, 0.0f};   // underflow, or NaN
  if (x.hi > 88.0f) return df{INFINITY, 0.0f};
  const float k = rintf(__fmul_rn(x.hi, 1.4426950216293335f));
  df r = x - df_two_prod(k, 0.6931471824645996f);
  r = r - df_two_prod(k, -1.9046542121259336e-09f);
  r = r - df{__fmul_rn(k, -8.78318373858934e-17f), 0.0f};
  // coefficients 1/j!, j = 12 .. 0
  df p = df(2.08767569878681e-09);
  p = fma(p, r, df(2.505210838544172e-08));
  p = fma(p, r, df(2.755731922398589e-07));
  p = fma(p, r, df(2.7557319223985893e-06));
  p = fma(p, r, df(2.48015873015873e-05));
  p = fma(p, r, df(0.0001984126984126984));
  p = fma(p, r, df(0.001388888888888889));
  p = fma(p, r, df(0.008333333333333333));
  p = fma(p, r, df(0.041666666666666664));
  p = fma(p, r, df(0.16666666666666666));
  p = fma(p, r, df(0.5));
  p = fma(p, r, df(1.0f));
  p = fma(p, r, df(1.0f));
  return df_ldexp(p, (int)k);
}
#endif

}  // namespace dgpe
