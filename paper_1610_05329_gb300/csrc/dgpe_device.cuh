// Device code of the SSCN step: complex arithmetic, shared-memory Stockham FFT stages,
// the chunked Thomas solver of the Crank-Nicolson sweeps, and the kernel templates.
// Instantiated once per real type by kernels_f64.cu (double), kernels_f32.cu (float) and
// kernels_df64.cu (df, the double-float pair of dgpe_df64.cuh).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "dgpe_df64.cuh"
#include "dgpe_internal.h"

namespace dgpe {

// FP64-class real types (double and df) take the FP64 design choices: the dipolar kernel
// from a table, FP64-accuracy copies of the scalars.
template <typename R>
struct Fp64Class {
  static constexpr bool value = false;
};
template <>
struct Fp64Class<double> {
  static constexpr bool value = true;
};
template <>
struct Fp64Class<df> {
  static constexpr bool value = true;
};

// ---------------------------------------------------------------------------------------
// Complex arithmetic
// ---------------------------------------------------------------------------------------
template <typename R>
struct alignas(2 * sizeof(R)) cplx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * conj(b)
template <typename R>
__device__ __forceinline__ cplx<R> mul_conj(cplx<R> a, cplx<R> b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// double-float: one product and one fused product-sum per component (the builtin types get
// the same from the compiler's contraction)
__device__ __forceinline__ cplx<df> operator*(cplx<df> a, cplx<df> b) {
  return {fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cplx<df> mul_conj(cplx<df> a, cplx<df> b) {
  return {fma(a.re, b.re, a.im * b.im), fma(a.im, b.re, -(a.re * b.im))};
}
// 2 a - b (doubling is exact; for a pair it scales both parts)
template <typename R>
__device__ __forceinline__ R twice_minus(R a, R b) { return fma(R(2), a, -b); }
__device__ __forceinline__ df twice_minus(df a, df b) { return df{2.0f * a.hi, 2.0f * a.lo} - b; }
template <typename R>
__device__ __forceinline__ cplx<R> scale(cplx<R> a, R s) { return {a.re * s, a.im * s}; }
template <typename R>
__device__ __forceinline__ cplx<R> mul_i(cplx<R> a) { return {-a.im, a.re}; }
template <typename R>
__device__ __forceinline__ cplx<R> mul_mi(cplx<R> a) { return {a.im, -a.re}; }
template <typename R>
__device__ __forceinline__ cplx<R> czero() { return {R(0), R(0)}; }

// Coefficients of the Crank-Nicolson solve: complex (real time) or real (imaginary time).
template <typename R>
__device__ __forceinline__ cplx<R> mul(R a, cplx<R> v) { return {a * v.re, a * v.im}; }
template <typename R>
__device__ __forceinline__ cplx<R> mul(cplx<R> a, cplx<R> v) { return a * v; }
// a b + d as a chain of FMAs (2 per component for complex a, 1 for real a).
template <typename R>
__device__ __forceinline__ cplx<R> cfma(R a, cplx<R> b, cplx<R> d) { return {fma(a, b.re, d.re), fma(a, b.im, d.im)}; }
template <typename R>
__device__ __forceinline__ cplx<R> cfma(cplx<R> a, cplx<R> b, cplx<R> d) {
  return {fma(a.re, b.re, fma(-a.im, b.im, d.re)), fma(a.re, b.im, fma(a.im, b.re, d.im))};
}
template <typename R>
__device__ __forceinline__ R neg_coef(R a) { return -a; }
template <typename R>
__device__ __forceinline__ cplx<R> neg_coef(cplx<R> a) { return {-a.re, -a.im}; }
// c v + d for the Crank-Nicolson coefficient c: real r (imaginary time) or i r (real time;
// the complex Coef holds {0, r}, so only its imaginary part enters).
template <typename R>
__device__ __forceinline__ cplx<R> cfma_c(R c, cplx<R> v, cplx<R> d) { return cfma(c, v, d); }
template <typename R>
__device__ __forceinline__ cplx<R> cfma_c(cplx<R> c, cplx<R> v, cplx<R> d) {
  return {fma(-c.im, v.im, d.re), fma(c.im, v.re, d.im)};
}

__device__ __forceinline__ double shfl_up(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float shfl_up(float v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float shfl_down(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ df shfl_up(df v, int d) { return {shfl_up(v.hi, d), shfl_up(v.lo, d)}; }
__device__ __forceinline__ df shfl_down(df v, int d) { return {shfl_down(v.hi, d), shfl_down(v.lo, d)}; }
__device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ df shfl_xor(df v, int m) { return {shfl_xor(v.hi, m), shfl_xor(v.lo, m)}; }
template <typename R>
__device__ __forceinline__ cplx<R> shfl_xor(cplx<R> v, int m) { return {shfl_xor(v.re, m), shfl_xor(v.im, m)}; }
template <typename R>
__device__ __forceinline__ cplx<R> shfl_up(cplx<R> v, int d) { return {shfl_up(v.re, d), shfl_up(v.im, d)}; }
template <typename R>
__device__ __forceinline__ cplx<R> shfl_down(cplx<R> v, int d) { return {shfl_down(v.re, d), shfl_down(v.im, d)}; }

// FP64 sine and cosine: Taylor series (coefficients (-1)^k/(2k+1)! and (-1)^k/(2k)!) on
// |r| <= pi/4 after Cody & Waite (1980) reduction r = x - k pi/2, with pi/2 split into
// three doubles (two of 32 significant bits, so k * part is exact for |k| < 2^21).  The
// first omitted terms, r^19/19! and r^20/20!, are below 1e-19.  The phase step's angles
// are usually small: for |x| <= 1/4 the sine series stops at x^11 (first omitted term below
// 3e-18) and the cosine is a fitted polynomial in x^2 (below), 12 FP64 instructions in all
// (GB300 issues 2 FP64 instructions per clock per SM).
__device__ __forceinline__ void sin_cos(double x, double *s, double *c) {
  // the range tests compare the bit pattern of |x| as an integer (positive doubles order as
  // their bits), which keeps them off the FP64 pipe; NaN fails both
  const unsigned long long ab = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
  if (ab <= 0x3fc0000000000000ULL) {   // |x| <= 1/8
    // least-squares fits of (sin x / x - 1)/x^2 and (cos x - 1)/x^2 as cubics in u = x^2
    // at 64 Chebyshev nodes of [0, 1/64] (40-digit arithmetic, coefficients rounded to
    // double: fit_sincos.py; errors below 2e-19 relative for the sine and 2e-18 absolute for
    // the cosine on |x| <= 1/8): two FMAs fewer than the |x| <= 1/4 branch
    const double u = x * x;
    double ps = 2.75494915427022e-06;
    ps = fma(ps, u, -0.0001984126907688373);
    ps = fma(ps, u, 0.008333333333309446);
    ps = fma(ps, u, -0.16666666666666666);
    *s = fma(x * u, ps, x);
    double pc = 2.4792977072672542e-05;
    pc = fma(pc, u, -0.0013888888048092878);
    pc = fma(pc, u, 0.04166666666640392);
    pc = fma(pc, u, -0.4999999999999999);
    *c = fma(u, pc, 1.0);
    return;
  }
  if (ab <= 0x3fd0000000000000ULL) {   // |x| <= 1/4
    const double u = x * x;
    double ps = -2.505210838544172e-08;
    ps = fma(ps, u, 2.7557319223985893e-06);
    ps = fma(ps, u, -0.0001984126984126984);
    ps = fma(ps, u, 0.008333333333333333);
    ps = fma(ps, u, -0.16666666666666666);
    *s = fma(x * u, ps, x);
    // cosine: the same least-squares fit of (cos x - 1)/x^2 as a quartic in u = x^2 on
    // [0, 1/16] (fit_sincos.py; error below 5.2e-19 on |x| <= 1/4), one term fewer than the
    // Taylor series for the same accuracy
    double pc = -2.7524717767692497e-07;
    pc = fma(pc, u, 2.48015694760334e-05);
    pc = fma(pc, u, -0.0013888888884910347);
    pc = fma(pc, u, 0.041666666666663556);
    pc = fma(pc, u, -0.5);
    *c = fma(u, pc, 1.0);
    return;
  }
  double r = x;
  int q = 0;
  if (fabs(x) > 0.7853981633974483) {
    if (!(fabs(x) < 1.0e6)) {   // huge or non-finite: the general routine
      sincos(x, s, c);
      return;
    }
    const double k = rint(x * 0.6366197723675814);
    r = fma(-k, 1.5707963267341256, x);
    r = fma(-k, 6.077100506303966e-11, r);
    r = fma(-k, 2.0222662487959506e-21, r);
    q = ((int)k) & 3;
  }
  const double u = r * r;
  double ps = 2.8114572543455206e-15;
  ps = fma(ps, u, -7.647163731819816e-13);
  ps = fma(ps, u, 1.6059043836821613e-10);
  ps = fma(ps, u, -2.505210838544172e-08);
  ps = fma(ps, u, 2.7557319223985893e-06);
  ps = fma(ps, u, -0.0001984126984126984);
  ps = fma(ps, u, 0.008333333333333333);
  ps = fma(ps, u, -0.16666666666666666);
  const double sr = fma(r * u, ps, r);
  double pc = -1.5619206968586225e-16;
  pc = fma(pc, u, 4.779477332387385e-14);
  pc = fma(pc, u, -1.1470745597729725e-11);
  pc = fma(pc, u, 2.08767569878681e-09);
  pc = fma(pc, u, -2.755731922398589e-07);
  pc = fma(pc, u, 2.48015873015873e-05);
  pc = fma(pc, u, -0.001388888888888889);
  pc = fma(pc, u, 0.041666666666666664);
  pc = fma(pc, u, -0.5);
  const double cr = fma(u, pc, 1.0);
  switch (q) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
  }
}
// FP32 sine and cosine by the same method (a short Taylor branch for |x| <= 1/4, then):
// r = x - k pi/2 with k = rint(2x/pi) taken from
// the low bits of the FP32 sum 2x/pi + 1.5 * 2^23 (no conversion instruction), pi/2 split
// into three floats and subtracted by FMAs; Taylor series through r^9 (sine) and r^10
// (cosine) on |r| <= pi/4, first omitted terms below 2e-9.  |x| >= 2^16 and non-finite x
// go to the general routine.
__device__ __forceinline__ void sin_cos(float x, float *s, float *c) {
  if (fabsf(x) <= 0.25f) {
    // short angles (nearly every point of the phase step): Taylor series through x^7 and
    // x^6, first omitted terms below 1.1e-11 and 3.8e-10 at |x| = 1/4, no reduction
    const float u = x * x;
    float ps = -1.9841269841269841e-4f;
    ps = fmaf(ps, u, 8.3333333333333333e-3f);
    ps = fmaf(ps, u, -0.16666666666666666f);
    *s = fmaf(x * u, ps, x);
    float pc = -1.3888888888888889e-3f;
    pc = fmaf(pc, u, 4.1666666666666667e-2f);
    pc = fmaf(pc, u, -0.5f);
    *c = fmaf(u, pc, 1.0f);
    return;
  }
  if (!(fabsf(x) < 65536.0f)) {
    sincosf(x, s, c);
    return;
  }
  const float kb = fmaf(x, 0.63661974668502808f, 12582912.0f);
  const int q = __float_as_int(kb) & 3;
  const float k = kb - 12582912.0f;
  float r = fmaf(-k, 1.5707963705062866f, x);
  r = fmaf(-k, -4.371138828673793e-08f, r);
  r = fmaf(-k, -1.7151245100058819e-15f, r);
  const float u = r * r;
  float ps = 2.7557319223985893e-06f;
  ps = fmaf(ps, u, -0.0001984126984126984f);
  ps = fmaf(ps, u, 0.008333333333333333f);
  ps = fmaf(ps, u, -0.16666666666666666f);
  const float sr = fmaf(r * u, ps, r);
  float pc = -2.755731922398589e-07f;
  pc = fmaf(pc, u, 2.48015873015873e-05f);
  pc = fmaf(pc, u, -0.001388888888888889f);
  pc = fmaf(pc, u, 0.041666666666666664f);
  pc = fmaf(pc, u, -0.5f);
  const float cr = fmaf(u, pc, 1.0f);
  const float ss = (q & 1) ? cr : sr, cc = (q & 1) ? sr : cr;
  *s = (q & 2) ? -ss : ss;
  *c = ((q + 1) & 2) ? -cc : cc;
}
__device__ __forceinline__ double exp_r(double x) { return exp(x); }
__device__ __forceinline__ float exp_r(float x) { return expf(x); }

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }
template <>
__device__ __forceinline__ cplx<double> ldg(const cplx<double> *p) {
  double2 v = __ldg(reinterpret_cast<const double2 *>(p));
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ cplx<float> ldg(const cplx<float> *p) {
  float2 v = __ldg(reinterpret_cast<const float2 *>(p));
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ df ldg(const df *p) {
  float2 v = __ldg(reinterpret_cast<const float2 *>(p));
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ cplx<df> ldg(const cplx<df> *p) {
  float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  return {df{v.x, v.y}, df{v.z, v.w}};
}

// ---------------------------------------------------------------------------------------
// Tile shapes per precision.  Rows of strided tiles are 128 B (8 complex128 or 16
// complex64) so every global access of a tile row is one full cache line.
// ---------------------------------------------------------------------------------------
template <typename R>
struct Tiles;
template <>
struct Tiles<double> {
  static constexpr int kZLines = 8;       // z-lines per CTA in K1/K5 (4 pairs)
  static constexpr int kZThreads = 256;   // 8 warps: one z-line per warp in the CN-z solve
  static constexpr int kZMinBlocks = 2;   // K5: two CTAs per SM (at most 128 registers)
  static constexpr int kXCols = 4;        // consecutive y columns per K3 tile
  static constexpr int kCnCols = 8;       // consecutive z columns per K6/K7 tile (128 B rows)
  static constexpr int kCnThreads = 128;  // 4 warps, two lines per warp
  static constexpr int kYBudget = 1024;   // K2/K4: lines per CTA ~ budget / ny
};
template <>
struct Tiles<df> : Tiles<double> {};   // the 16-byte complex values of FP64
template <>
struct Tiles<float> {
  static constexpr int kZLines = 16;
  static constexpr int kZThreads = 256;
  static constexpr int kZMinBlocks = 2;
  static constexpr int kXCols = 8;
  static constexpr int kCnCols = 16;
  static constexpr int kCnThreads = 512;  // 16 warps, one line per warp
  static constexpr int kYBudget = 4096;
};
// z-lines per K1 and K5 tile: 32 for the FP32 compile-time lengths of at most 128 points
// (twice the points per CTA over its fixed costs; in K5 every warp busy in the 8-lane z
// solve), else kZLines
template <typename R>
__host__ __device__ constexpr int ztile_lines(int n) {
  return std::is_same<R, float>::value && (n == 64 || n == 96 || n == 128) ? 32 : Tiles<R>::kZLines;
}
constexpr int kFftThreads = 256;
constexpr int kUnroll = 8;  // loads in flight per thread in the register-staged load loops

// K2/K4 lines per CTA: a power of two in [2, 32] (it must divide the block size).
template <typename R>
__host__ __device__ constexpr int y_lines_per_cta(int ny) {
  int l = 2;
  while (l * 2 <= 32 && l * 2 * ny <= Tiles<R>::kYBudget) l *= 2;
  return l;
}

// Walks the flat index e = b * n + k of contiguous lines of length n in steps of `step`
// (the block size), keeping (b, k) up to date without an integer division per step.
struct LinePos {
  int b, k, sb, sk, n;
  __device__ __forceinline__ LinePos(int e0, int n_, int step) : n(n_) {
    b = e0 / n;
    k = e0 - b * n;
    sb = step / n;
    sk = step - sb * n;
  }
  __device__ __forceinline__ void next() {
    k += sk;
    b += sb;
    if (k >= n) {
      k -= n;
      ++b;
    }
  }
};

// ---------------------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async): every copy of a tile is in flight at
// once instead of one dependent load per loop iteration.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
template <typename C>
__device__ __forceinline__ void cp_async(C *dst, const C *src) {
  static_assert(sizeof(C) == 4 || sizeof(C) == 8 || sizeof(C) == 16, "4-, 8- or 16-byte elements");
  if constexpr (sizeof(C) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else if constexpr (sizeof(C) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Bulk prefetch of bytes [p, p + n) into L2 (no destination, no completion to wait for):
// p 16-byte aligned, n a multiple of 16.  The tile kernels that run in waves of CTAs use it
// to fetch the rows of the tile that a CTA one resident wave later will load.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned n) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(__cvta_generic_to_global(p)), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Double-float accumulator (Knuth's TwoSum): FP64-quality running sums from FP32 terms
// without FP64 instructions per term.
struct DFAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = __fadd_rn(hi, v);
    const float bp = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    hi = t;
    lo = __fadd_rn(lo, err);
  }
  // a v for an FP32 a, exactly: the product p = fl(a v) and its error fma(a, v, -p)
  __device__ __forceinline__ void add_prod(float a, float v) {
    const float p = __fmul_rn(a, v);
    add(p);
    lo = __fadd_rn(lo, fmaf(a, v, -p));
  }
  // a (x.hi + x.lo) for an FP32 a
  __device__ __forceinline__ void add_scaled(float a, const DFAcc &x) {
    add_prod(a, x.hi);
    lo = fmaf(a, x.lo, lo);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Slot of grid point n of a line in a Crank-Nicolson tile: one padding slot after every
// chunk = 2^lchunk interior points, so that the 32 lanes solving one line hit distinct
// banks.  cn_slots = slots of a line of n points.
__host__ __device__ inline int cn_slot(int n, int lchunk) { return n + (max(n - 1, 0) >> lchunk); }
__host__ __device__ inline int cn_slots(int n, int lchunk) { return n + ((n - 2) >> lchunk); }

// K5's tile stride (slots per line) at a compile-time length n (FP32): the padded line of
// 32 k5_chunk(n) + 2 points with one pad slot per chunk, rounded up to an odd stride.
__host__ __device__ constexpr int k5_tile_stride(int n) { return kWarp * k5_chunk(n) + 35; }

// Points n = k0 + W j (j = 0, 1, ...) of a line in a Crank-Nicolson tile, for W a multiple of
// the chunk: their slots cn_slot(n) = n + ((n - 1) >> lchunk) advance by the constant
// W + (W >> lchunk), from k0 + ((k0 - 1) >> lchunk) (an arithmetic shift: -1 for k0 = 0,
// where the wall n = 0 itself is slot 0).  The tile loops of the compile-time line lengths
// walk their points this way instead of recomputing the slot and the line of every point.
// The same for any chunk CH (K5's z solve at 12 points per lane): period P = lcm(W, CH);
// a thread at offset o < P walks n = o + P j, slot n + (n - 1)/CH = base + j (P + P/CH),
// base = o + (o - 1)/CH (-1 for o = 0, with the wall n = 0 at slot 0).
template <int P, int CH>
struct SlotWalkP {
  static_assert(P % CH == 0, "whole chunks per period");
  int base;
  static constexpr int step = P + P / CH;
  __device__ __forceinline__ explicit SlotWalkP(int o) : base(o == 0 ? -1 : o + (o - 1) / CH) {}
  __device__ __forceinline__ int operator()(int j, int o) const { return (o | j) == 0 ? 0 : base + j * step; }
};
__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

template <int W>
struct SlotWalk {
  int base, step;
  __device__ __forceinline__ SlotWalk(int k0, int lchunk) : base(k0 + ((k0 - 1) >> lchunk)), step(W + (W >> lchunk)) {}
  __device__ __forceinline__ int operator()(int j, int k0) const { return (k0 | j) == 0 ? 0 : base + j * step; }
};

// ---------------------------------------------------------------------------------------
// FFT: radix-2/3/4/5/7/8 butterflies (DIR = -1 forward e^{-i..}, +1 inverse, unnormalised)
// ---------------------------------------------------------------------------------------
template <typename R, int DIR>
__device__ __forceinline__ void bf2(cplx<R> *v) {
  const cplx<R> a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}

template <typename R, int DIR>
__device__ __forceinline__ void bf4(cplx<R> &a0, cplx<R> &a1, cplx<R> &a2, cplx<R> &a3) {
  const cplx<R> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3;
  const cplx<R> d = a1 - a3;
  const cplx<R> t3 = DIR < 0 ? mul_mi(d) : mul_i(d);
  a0 = t0 + t2;
  a2 = t0 - t2;
  a1 = t1 + t3;
  a3 = t1 - t3;
}

template <typename R, int DIR>
__device__ __forceinline__ void bf8(cplx<R> *v) {
  cplx<R> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cplx<R> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  bf4<R, DIR>(e0, e1, e2, e3);
  bf4<R, DIR>(o0, o1, o2, o3);
  const R h = R(0.70710678118654752440084436210485);
  // o_k *= w8^k, w8 = e^{DIR 2 pi i / 8}
  cplx<R> p1, p2, p3;
  if (DIR < 0) {
    p1 = {(o1.re + o1.im) * h, (o1.im - o1.re) * h};
    p2 = mul_mi(o2);
    p3 = {(o3.im - o3.re) * h, -(o3.re + o3.im) * h};
  } else {
    p1 = {(o1.re - o1.im) * h, (o1.re + o1.im) * h};
    p2 = mul_i(o2);
    p3 = {-(o3.re + o3.im) * h, (o3.re - o3.im) * h};
  }
  v[0] = e0 + o0;
  v[4] = e0 - o0;
  v[1] = e1 + p1;
  v[5] = e1 - p1;
  v[2] = e2 + p2;
  v[6] = e2 - p2;
  v[3] = e3 + p3;
  v[7] = e3 - p3;
}

template <typename R, int DIR>
__device__ __forceinline__ void bf3(cplx<R> *v) {
  const R s3 = R(0.86602540378443864676372317075294);
  const cplx<R> t = v[1] + v[2];
  const cplx<R> u = scale(v[1] - v[2], s3);
  const cplx<R> m = {v[0].re - R(0.5) * t.re, v[0].im - R(0.5) * t.im};
  v[0] = v[0] + t;
  if (DIR < 0) {
    v[1] = m + mul_mi(u);
    v[2] = m + mul_i(u);
  } else {
    v[1] = m + mul_i(u);
    v[2] = m + mul_mi(u);
  }
}

// Radix 5 and 7 (odd primes): with t_k = v_k + v_{P-k}, u_k = v_k - v_{P-k},
// X_m = v_0 + sum_k cos(2 pi k m / P) t_k  -/+  i sum_k sin(2 pi k m / P) u_k  (m, P - m),
// the sign of i being DIR's.
template <typename R, int DIR>
__device__ __forceinline__ void bf5(cplx<R> *v) {
  const R c1 = R(0.30901699437494745), c2 = R(-0.8090169943749475);
  const R s1 = R(0.9510565162951535), s2 = R(0.5877852522924731);
  const cplx<R> t1 = v[1] + v[4], t2 = v[2] + v[3], t3 = v[1] - v[4], t4 = v[2] - v[3];
  const cplx<R> a = {v[0].re + c1 * t1.re + c2 * t2.re, v[0].im + c1 * t1.im + c2 * t2.im};
  const cplx<R> b = {v[0].re + c2 * t1.re + c1 * t2.re, v[0].im + c2 * t1.im + c1 * t2.im};
  const cplx<R> d = {s1 * t3.re + s2 * t4.re, s1 * t3.im + s2 * t4.im};
  const cplx<R> e = {s2 * t3.re - s1 * t4.re, s2 * t3.im - s1 * t4.im};
  const cplx<R> id = DIR < 0 ? mul_mi(d) : mul_i(d), ie = DIR < 0 ? mul_mi(e) : mul_i(e);
  v[0] = v[0] + t1 + t2;
  v[1] = a + id;
  v[4] = a - id;
  v[2] = b + ie;
  v[3] = b - ie;
}

template <typename R, int DIR>
__device__ __forceinline__ void bf7(cplx<R> *v) {
  const R C1 = R(0.6234898018587335), C2 = R(-0.2225209339563144), C3 = R(-0.9009688679024191);
  const R S1 = R(0.7818314824680298), S2 = R(0.9749279121818236), S3 = R(0.4338837391175581);
  const cplx<R> t1 = v[1] + v[6], t2 = v[2] + v[5], t3 = v[3] + v[4];
  const cplx<R> u1 = v[1] - v[6], u2 = v[2] - v[5], u3 = v[3] - v[4];
  auto lin3 = [](R p, cplx<R> x, R q, cplx<R> y, R r, cplx<R> z) {
    return cplx<R>{p * x.re + q * y.re + r * z.re, p * x.im + q * y.im + r * z.im};
  };
  const cplx<R> a1 = v[0] + lin3(C1, t1, C2, t2, C3, t3);
  const cplx<R> a2 = v[0] + lin3(C2, t1, C3, t2, C1, t3);
  const cplx<R> a3 = v[0] + lin3(C3, t1, C1, t2, C2, t3);
  const cplx<R> d1 = lin3(S1, u1, S2, u2, S3, u3);
  const cplx<R> d2 = lin3(S2, u1, -S3, u2, -S1, u3);
  const cplx<R> d3 = lin3(S3, u1, -S1, u2, S2, u3);
  const cplx<R> i1 = DIR < 0 ? mul_mi(d1) : mul_i(d1);
  const cplx<R> i2 = DIR < 0 ? mul_mi(d2) : mul_i(d2);
  const cplx<R> i3 = DIR < 0 ? mul_mi(d3) : mul_i(d3);
  v[0] = v[0] + t1 + t2 + t3;
  v[1] = a1 + i1;
  v[6] = a1 - i1;
  v[2] = a2 + i2;
  v[5] = a2 - i2;
  v[3] = a3 + i3;
  v[4] = a3 - i3;
}

template <typename R, int DIR, int P>
__device__ __forceinline__ void butterfly(cplx<R> *v) {
  if constexpr (P == 2) bf2<R, DIR>(v);
  else if constexpr (P == 3) bf3<R, DIR>(v);
  else if constexpr (P == 4) bf4<R, DIR>(v[0], v[1], v[2], v[3]);
  else if constexpr (P == 5) bf5<R, DIR>(v);
  else if constexpr (P == 7) bf7<R, DIR>(v);
  else bf8<R, DIR>(v);
}

// Tangent-form twiddles (FP64, radix 2, 4 and 8).  GB300 issues FP64 arithmetic at 1/64
// of the FP32 rate, so the FP64 transforms count FP64 instructions, not memory traffic or
// integer work.  A twiddle w = e^{-i phi} is stored as w = sigma i^q (1 + i t) with |t| <= 1
// (q = 1 where |sin phi| > |cos phi|, so |sigma| >= 1/sqrt 2): v w = sigma u with
// u = (1 + i t) i^q v, two FMAs, and sigma enters the butterfly's additions, which become
// FMAs (the multiply-add FFT of Linzer & Feig 1993 and Goedecker 1997).  q follows from the
// twiddle's index, so only (t, sigma) is stored.  A radix-8 butterfly with its seven
// twiddles takes 67 FP64 instructions instead of 80, a radix-4 one 22 instead of 28, a
// radix-2 one 6 instead of 8.  Entry r - 1 of index k holds {t_r, S_r}: S = sigma_1 for
// radix 2; (sigma_1, sigma_2, sigma_3/sigma_1) for radix 4; (sigma_1, sigma_2,
// sigma_3/sigma_1, sigma_4, sigma_5/sigma_1, sigma_6/sigma_2, sigma_7/sigma_3) for radix 8 --
// the scales the butterflies below fold in (all between 1/sqrt 2 and sqrt 2 in magnitude).
template <typename R, int P>
struct TangentTw {
  static constexpr bool value = std::is_same<R, double>::value && (P == 2 || P == 4 || P == 8);
};
// q of the twiddle e^{-2 pi i a / M}, 0 <= a < M: the angle lies within pi/4 of +-pi/2
__host__ __device__ __forceinline__ bool tw_rot(int a, int M) {
  int c = 8 * a;
  if (c >= 4 * M) c -= 4 * M;
  return c > M && c < 3 * M;
}
// u = (1 + i t) i^q v for the forward twiddle, (1 - i t) (-i)^q v for its conjugate; the
// rotation and its sign are integer selects on the two FMA results
template <int DIR>
__device__ __forceinline__ cplx<double> tw_u(cplx<double> v, double t, bool q) {
  constexpr unsigned long long kSign = 0x8000000000000000ULL;
  const double tt = DIR < 0 ? t : -t;
  const double x = fma(tt, v.re, v.im), y = fma(-tt, v.im, v.re);
  const unsigned long long xb = (unsigned long long)__double_as_longlong(x);
  const unsigned long long yb = (unsigned long long)__double_as_longlong(y);
  if (DIR < 0) return {q ? __longlong_as_double((long long)(xb ^ kSign)) : y, q ? y : x};
  return {q ? x : y, q ? __longlong_as_double((long long)(yb ^ kSign)) : x};
}
// a + s b for real s
__device__ __forceinline__ cplx<double> fma_s(double s, cplx<double> b, cplx<double> a) {
  return {fma(s, b.re, a.re), fma(s, b.im, a.im)};
}
template <int DIR>
__device__ __forceinline__ cplx<double> mul_dir_i(cplx<double> d) { return DIR < 0 ? mul_mi(d) : mul_i(d); }

// twiddles of index k (table entries w[0..P-2], M = ns P) and the butterfly, in place
template <int DIR, int P>
__device__ __forceinline__ void butterfly_tangent(cplx<double> *v, const cplx<double> *__restrict__ w, int k, int M) {
  cplx<double> u[P];
  double sg[P];
#pragma unroll
  for (int r = 1; r < P; ++r) {
    const cplx<double> e = ldg(w + r - 1);
    u[r] = tw_u<DIR>(v[r], e.re, tw_rot(r * k, M));
    sg[r] = e.im;
  }
  if constexpr (P == 2) {
    const cplx<double> a = v[0];
    v[0] = fma_s(sg[1], u[1], a);
    v[1] = fma_s(-sg[1], u[1], a);
  } else if constexpr (P == 4) {
    const cplx<double> t0 = fma_s(sg[2], u[2], v[0]), t1 = fma_s(-sg[2], u[2], v[0]);
    const cplx<double> p = fma_s(sg[3], u[3], u[1]);
    const cplx<double> d = mul_dir_i<DIR>(fma_s(-sg[3], u[3], u[1]));
    v[0] = fma_s(sg[1], p, t0);
    v[2] = fma_s(-sg[1], p, t0);
    v[1] = fma_s(sg[1], d, t1);
    v[3] = fma_s(-sg[1], d, t1);
  } else {
    // even inputs (v0, sigma_2 u2, sigma_4 u4, sigma_6 u6): a radix-4 butterfly
    const cplx<double> et0 = fma_s(sg[4], u[4], v[0]), et1 = fma_s(-sg[4], u[4], v[0]);
    const cplx<double> ep = fma_s(sg[6], u[6], u[2]);
    const cplx<double> ed = mul_dir_i<DIR>(fma_s(-sg[6], u[6], u[2]));
    const cplx<double> e0 = fma_s(sg[2], ep, et0), e2 = fma_s(-sg[2], ep, et0);
    const cplx<double> e1 = fma_s(sg[2], ed, et1), e3 = fma_s(-sg[2], ed, et1);
    // odd inputs over sigma_1: (u1, rho_3 u3, rho_5 u5, rho_7 u7), rho_j = sigma_j / sigma_1
    const cplx<double> ot0 = fma_s(sg[5], u[5], u[1]), ot1 = fma_s(-sg[5], u[5], u[1]);
    const cplx<double> op = fma_s(sg[7], u[7], u[3]);
    const cplx<double> od = mul_dir_i<DIR>(fma_s(-sg[7], u[7], u[3]));
    const cplx<double> o0 = fma_s(sg[3], op, ot0), o2 = fma_s(-sg[3], op, ot0);
    const cplx<double> o1 = fma_s(sg[3], od, ot1), o3 = fma_s(-sg[3], od, ot1);
    // out_j = e_j + sigma_1 w8^j o_j, out_{j+4} = e_j - sigma_1 w8^j o_j, w8 = e^{DIR 2 pi i / 8}
    const double h1 = sg[1] * 0.70710678118654752440084436210485;
    cplx<double> z1, z3;
    if (DIR < 0) {
      z1 = {o1.re + o1.im, o1.im - o1.re};
      z3 = {o3.im - o3.re, -(o3.re + o3.im)};
    } else {
      z1 = {o1.re - o1.im, o1.re + o1.im};
      z3 = {-(o3.re + o3.im), o3.re - o3.im};
    }
    const cplx<double> r2 = mul_dir_i<DIR>(o2);
    v[0] = fma_s(sg[1], o0, e0);
    v[4] = fma_s(-sg[1], o0, e0);
    v[1] = fma_s(h1, z1, e1);
    v[5] = fma_s(-h1, z1, e1);
    v[2] = fma_s(sg[1], r2, e2);
    v[6] = fma_s(-sg[1], r2, e2);
    v[3] = fma_s(h1, z3, e3);
    v[7] = fma_s(-h1, z3, e3);
  }
}

// The twiddles of index k of a stage (M = ns P) and the butterfly, for every precision; the
// complex-twiddle form keeps one inlined butterfly per stage (twiddled or not), which the
// double-float code, many instructions per operation, needs for its instruction cache.
template <typename R, int DIR, int P>
__device__ __forceinline__ void stage_butterfly(cplx<R> *v, bool twiddled, const cplx<R> *__restrict__ w, int k,
                                                int M) {
  if constexpr (TangentTw<R, P>::value) {
    if (twiddled) butterfly_tangent<DIR, P>(v, w, k, M);
    else butterfly<R, DIR, P>(v);
  } else {
    if (twiddled) {
#pragma unroll
      for (int r = 1; r < P; ++r) {
        const cplx<R> t = ldg(w + r - 1);
        v[r] = DIR < 0 ? v[r] * t : mul_conj(v[r], t);
      }
    }
    butterfly<R, DIR, P>(v);
  }
}

// One Stockham autosort stage of radix P over `nlines` lines held in shared memory,
// element e of line l at [e * sb + l].  ns = product of the radices of earlier stages.
// Butterfly j reads x[j + r n/P], twiddles by w_n^{r (j mod ns) n/(ns P)}, and writes the
// P outputs to (j div ns) ns P + (j mod ns) + s ns.  Thread t works on line t mod lw
// (lw divides the block size) and on every (blockDim/lw)-th butterfly of it.
template <typename R, int DIR, int P>
__device__ __forceinline__ void fft_stage(const cplx<R> *__restrict__ src, cplx<R> *__restrict__ dst, int n,
                                          int ns, int lw, int nlines, int sb, const cplx<R> *__restrict__ tw) {
  const int nbf = n / P;
  const int line = threadIdx.x % lw;
  if (line >= nlines) return;
  const int jstep = blockDim.x / lw;
  const bool pow2 = (ns & (ns - 1)) == 0;
  // strides (in elements) between the P inputs and between the P outputs of a butterfly
  const int in_stride = nbf * sb, out_stride = ns * sb;
  const cplx<R> *s0 = src + line;
  cplx<R> *d0 = dst + line;
  for (int j = threadIdx.x / lw; j < nbf; j += jstep) {
    const int k = pow2 ? (j & (ns - 1)) : (j % ns);
    const cplx<R> *in = s0 + j * sb;
    cplx<R> v[P];
#pragma unroll
    for (int r = 0; r < P; ++r) v[r] = in[r * in_stride];
    stage_butterfly<R, DIR, P>(v, ns > 1, tw + k * (P - 1), k, ns * P);   // the P-1 twiddles of k
    cplx<R> *out = d0 + ((j - k) * P + k) * sb;
#pragma unroll
    for (int s = 0; s < P; ++s) out[s * out_stride] = v[s];
  }
}

// Full transform of `nlines` (<= lw) lines (ping-pong between a and b); returns the
// buffer holding the result.  The caller synchronises before the call (input written).
template <typename R, int DIR>
__device__ cplx<R> *fft_lines(cplx<R> *a, cplx<R> *b, const FftPlan &pl, int lw, int nlines, int sb,
                              const cplx<R> *tw) {
  int ns = 1;
  for (int st = 0; st < pl.nstages; ++st) {
    const int p = pl.radix[st];
    const cplx<R> *tws = tw + pl.twoff[st];
    if (p == 8) fft_stage<R, DIR, 8>(a, b, pl.n, ns, lw, nlines, sb, tws);
    else if (p == 4) fft_stage<R, DIR, 4>(a, b, pl.n, ns, lw, nlines, sb, tws);
    else if (p == 3) fft_stage<R, DIR, 3>(a, b, pl.n, ns, lw, nlines, sb, tws);
    else if (p == 5) fft_stage<R, DIR, 5>(a, b, pl.n, ns, lw, nlines, sb, tws);
    else if (p == 7) fft_stage<R, DIR, 7>(a, b, pl.n, ns, lw, nlines, sb, tws);
    else fft_stage<R, DIR, 2>(a, b, pl.n, ns, lw, nlines, sb, tws);
    __syncthreads();
    cplx<R> *t = a;
    a = b;
    b = t;
    ns *= p;
  }
  return a;
}

// The same transform with the length, the line layout and the block size fixed at compile
// time (the radix order is make_plan's default: radix 8 first, then 4, 2, 3, 5, 7): every
// stride, trip count and twiddle offset is a constant, the loops unroll, and the shared-
// memory accesses of a butterfly share one base address.
__host__ __device__ constexpr int ct_radix(int n, int st) {
  int m = n, k = 0;
  while (m % 8 == 0) {
    if (k++ == st) return 8;
    m /= 8;
  }
  while (m % 4 == 0) {
    if (k++ == st) return 4;
    m /= 4;
  }
  if (m % 2 == 0) {
    if (k++ == st) return 2;
    m /= 2;
  }
  const int odd[3] = {3, 5, 7};
  for (int q = 0; q < 3; ++q)
    while (m % odd[q] == 0) {
      if (k++ == st) return odd[q];
      m /= odd[q];
    }
  return 0;
}
__host__ __device__ constexpr int ct_ns(int n, int st) {
  int ns = 1;
  for (int s = 0; s < st; ++s) ns *= ct_radix(n, s);
  return ns;
}
__host__ __device__ constexpr int ct_twoff(int n, int st) {
  int off = 0;
  for (int s = 0; s < st; ++s) off += ct_ns(n, s) * (ct_radix(n, s) - 1);
  return off;
}

template <typename R, int DIR, int P, int N, int NS, int LW, int SB, int NT>
__device__ __forceinline__ void fft_stage_ct(const cplx<R> *__restrict__ src, cplx<R> *__restrict__ dst, int nlines,
                                             const cplx<R> *__restrict__ tw) {
  constexpr int NBF = N / P, JSTEP = NT / LW;
  static_assert(NT % LW == 0, "the line count divides the block size");
  const int line = threadIdx.x % LW;
  if (line >= nlines) return;
  const int j0 = threadIdx.x / LW;
#pragma unroll
  for (int it = 0; it < (NBF + JSTEP - 1) / JSTEP; ++it) {
    const int j = j0 + it * JSTEP;
    if (NBF % JSTEP != 0 && j >= NBF) break;
    const int k = j % NS;
    const cplx<R> *in = src + j * SB + line;
    cplx<R> v[P];
#pragma unroll
    for (int r = 0; r < P; ++r) v[r] = in[r * NBF * SB];
    stage_butterfly<R, DIR, P>(v, NS > 1, tw + k * (P - 1), k, NS * P);
    cplx<R> *out = dst + ((j - k) * P + k) * SB + line;
#pragma unroll
    for (int s = 0; s < P; ++s) out[s * NS * SB] = v[s];
  }
}

// Two consecutive stages (radix P1 at ns = NS, then radix P2 at ns = NS P1) in one pass, the
// intermediate values in registers: the P2 stage-1 butterflies j1 = (q2 + r Q) NS + k1
// (r < P2, Q = N / (P1 P2 NS)) produce exactly the inputs of the P1 stage-2 butterflies
// j2 = q2 NS P1 + s NS + k1 (s < P1), output s of the r-th feeding input r of the s-th.  The
// same butterflies and twiddles as the two stages, in the same order per element: only the
// round trip through shared memory and one barrier go.
template <typename R, int DIR, int P1, int P2, int N, int NS, int LW, int SB, int NT>
__device__ __forceinline__ void fft_stage_ct2(const cplx<R> *__restrict__ src, cplx<R> *__restrict__ dst, int nlines,
                                              const cplx<R> *__restrict__ tw1, const cplx<R> *__restrict__ tw2) {
  constexpr int NS2 = NS * P1, Q = N / (P1 * P2 * NS), NU = N / (P1 * P2), JSTEP = NT / LW;
  static_assert(NT % LW == 0 && Q * P1 * P2 * NS == N, "whole fused units");
  const int line = threadIdx.x % LW;
  if (line >= nlines) return;
  const int u0 = threadIdx.x / LW;
#pragma unroll
  for (int it = 0; it < (NU + JSTEP - 1) / JSTEP; ++it) {
    const int u = u0 + it * JSTEP;
    if (NU % JSTEP != 0 && u >= NU) break;
    const int k1 = u % NS, q2 = u / NS;
    cplx<R> w[P2][P1];
#pragma unroll
    for (int r = 0; r < P2; ++r) {
      const int j1 = (q2 + r * Q) * NS + k1;
      cplx<R> v[P1];
#pragma unroll
      for (int r1 = 0; r1 < P1; ++r1) v[r1] = src[(j1 + r1 * (N / P1)) * SB + line];
      stage_butterfly<R, DIR, P1>(v, NS > 1, tw1 + k1 * (P1 - 1), k1, NS * P1);
#pragma unroll
      for (int q = 0; q < P1; ++q) w[r][q] = v[q];
    }
#pragma unroll
    for (int q = 0; q < P1; ++q) {
      const int k2 = q * NS + k1, j2 = q2 * NS2 + k2;
      cplx<R> v[P2];
#pragma unroll
      for (int r = 0; r < P2; ++r) v[r] = w[r][q];
      stage_butterfly<R, DIR, P2>(v, NS2 > 1, tw2 + k2 * (P2 - 1), k2, NS2 * P2);
      cplx<R> *out = dst + ((j2 - k2) * P2 + k2) * SB + line;
#pragma unroll
      for (int s2 = 0; s2 < P2; ++s2) out[s2 * NS2 * SB] = v[s2];
    }
  }
}

// FP32: a radix-2 or radix-4 stage followed by a radix-3 stage runs as one fused pass
template <typename R, int N, int ST>
__host__ __device__ constexpr bool ct_fuse(int p) {
  return std::is_same<R, float>::value && (p == 2 || p == 4) && ct_radix(N, ST + 1) == 3;
}

template <typename R, int DIR, int N, int LW, int SB, int NT, int ST = 0>
__device__ __forceinline__ cplx<R> *fft_lines_ct(cplx<R> *a, cplx<R> *b, int nlines, const cplx<R> *tw) {
  constexpr int P = ct_radix(N, ST);
  if constexpr (P == 0) {
    return a;
  } else if constexpr (ct_fuse<R, N, ST>(P)) {
    fft_stage_ct2<R, DIR, P, 3, N, ct_ns(N, ST), LW, SB, NT>(a, b, nlines, tw + ct_twoff(N, ST), tw + ct_twoff(N, ST + 1));
    __syncthreads();
    return fft_lines_ct<R, DIR, N, LW, SB, NT, ST + 2>(b, a, nlines, tw);
  } else {
    fft_stage_ct<R, DIR, P, N, ct_ns(N, ST), LW, SB, NT>(a, b, nlines, tw + ct_twoff(N, ST));
    __syncthreads();
    return fft_lines_ct<R, DIR, N, LW, SB, NT, ST + 1>(b, a, nlines, tw);
  }
}

// The compile-time transform when N > 0 (the caller checked that the plan is the default
// one of length N and that the block has NT threads), else the runtime plan.
template <typename R, int DIR, int N, int LW, int SB, int NT>
__device__ __forceinline__ cplx<R> *fft_lines_n(cplx<R> *a, cplx<R> *b, const FftPlan &pl, int nlines,
                                                const cplx<R> *tw) {
  if constexpr (N > 0) return fft_lines_ct<R, DIR, N, LW, SB, NT>(a, b, nlines, tw);
  else return fft_lines<R, DIR>(a, b, pl, LW, nlines, SB, tw);
}

// ---------------------------------------------------------------------------------------
// Crank-Nicolson along one line: solve (1 - cD) chi = psi on the m interior points
// (Dirichlet walls), then psi' = 2 chi - psi = (1 - cD)^{-1} (1 + cD) psi.
//
// Chunked Thomas algorithm, one warp per line, lane t owns interior points
// [t C, t C + C).  With the LU factors alpha_i = c / e_{i-1}, beta_i = 1 / e_i,
//   forward  y_i = psi_i + alpha_i y_{i-1},   backward chi_i = beta_i (y_i + c chi_{i+1}),
// each lane runs both recurrences on its chunk from zero boundary values, and the exact
// solution follows by linearity:
//   y_i   = y0_i + P_i Y_t,                   Y_t = y at the point before the chunk,
//   chi_i = chi0_i + Y_t H_i + X_{t+1} G_i,   X_{t+1} = chi at the point after the chunk,
// with P, H, G precomputed per position (see k_cn_tables).  The carries Y_t and X_t are
// affine recurrences across lanes, resolved by warp-shuffle scans of (A, B) pairs; the A
// factors of every lane and scan step depend only on the position, so they come from the
// tables as well (only B is scanned).
// Element n of the line is at buf[cn_slot(n, lchunk) * es].
// Table layout (lane-interleaved, mp = 32 * chunk): [alpha | beta | H | G] at q * mp + e * 32
// + t for interior point t * chunk + e, then the scan factors: forward step k (offset
// 2^k) at 4 mp + k * 32 + t, backward step k at 4 mp + (5 + k) * 32 + t.
// ---------------------------------------------------------------------------------------
// FULL: the line is padded to 32 CH unknowns (m = 32 CH; the padded slots hold zeros and the
// tables decouple them), so every lane has a whole chunk and no per-point guard.
// L: lanes per line (32, or 8 for the short lines: four lines per warp, lanes 8g .. 8g + 7,
// log2(L) scan steps; the tables in the L-lane layout).
template <typename R, typename Coef, int CH, bool SHARED_TAB, bool FULL = false, int L = kWarp>
__device__ __forceinline__ void cn_line(cplx<R> *__restrict__ buf, int es, int m, int lchunk,
                                        const Coef *__restrict__ tab, const Coef *__restrict__ scan_s, Coef c) {
  static_assert(L == kWarp || L == 8, "32 or 8 lanes per line");
  constexpr int LG = L == kWarp ? 5 : 3;
  const int t = threadIdx.x & (L - 1);
  constexpr int chunk = CH;
  const int s0 = t * chunk;
  const int len = FULL ? CH : max(0, min(chunk, m - s0));
  constexpr int mp = L * CH;
  const Coef *alpha = tab + t;
  const Coef *beta = tab + mp + t;
  const Coef *H = tab + 2 * mp + t;
  const Coef *G = tab + 3 * mp + t;
  const Coef *scan = scan_s + t;   // the scan factors, staged in shared memory by the caller

  cplx<R> y[CH];
  cplx<R> acc = czero<R>();
  // factor tables: shared memory (plain loads) or global memory (read-only path)
  auto T = [](const Coef *q) -> Coef {
    if constexpr (SHARED_TAB) return *q;
    else return ldg(q);
  };
#pragma unroll
  for (int e = 0; e < CH; ++e) {
    if (e < len) {
      const int i = s0 + e;
      acc = cfma(T(alpha + e * L), acc, buf[(i + 1 + t) * es]);
      y[e] = acc;
    }
  }
  // forward carries: Y_{t+1} = A_t Y_t + B_t, Y_0 = 0 (the shuffles span the warp; a lane
  // takes a neighbour's value only within its own line's L lanes)
  cplx<R> B = acc;
#pragma unroll
  for (int k = 0; k < LG; ++k) {
    const cplx<R> Bp = shfl_up(B, 1 << k);
    if (t >= (1 << k)) B = cfma(scan[k * L], Bp, B);
  }
  cplx<R> Y = shfl_up(B, 1);
  if (t == 0) Y = czero<R>();

  acc = czero<R>();
#pragma unroll
  for (int e = CH - 1; e >= 0; --e) {
    if (e < len) {
      acc = mul(T(beta + e * L), cfma_c(c, acc, y[e]));
      y[e] = acc;
    }
  }
  // backward carries: X_t = G_{s0} X_{t+1} + (chi0_{s0} + H_{s0} Y_t), X_32 = 0
  cplx<R> B2 = len > 0 ? cfma(T(H), Y, acc) : czero<R>();
#pragma unroll
  for (int k = 0; k < LG; ++k) {
    const cplx<R> Bn = shfl_down(B2, 1 << k);
    if (t + (1 << k) < L) B2 = cfma(scan[(LG + k) * L], Bn, B2);
  }
  cplx<R> X = shfl_down(B2, 1);
  if (t == L - 1) X = czero<R>();

#pragma unroll
  for (int e = 0; e < CH; ++e) {
    if (e < len) {
      const int i = s0 + e;
      const cplx<R> chi = cfma(T(H + e * L), Y, cfma(T(G + e * L), X, y[e]));
      const int q = (i + 1 + t) * es;
      const cplx<R> v = buf[q];
      buf[q] = {twice_minus(chi.re, v.re), twice_minus(chi.im, v.im)};
    }
  }
  if (t == 0) {
    buf[0] = czero<R>();
    if (!FULL) buf[(m + 1 + (m >> lchunk)) * es] = czero<R>();   // (FULL: the padding already holds 0)
  }
}

// Two lines of the same factor tables (and the same padded length, FULL) solved by one warp
// in lockstep: each table and scan-factor value is read from shared memory once for both
// lines, and the two recurrences interleave.  The arithmetic of each line is cn_line's.
template <typename R, typename Coef, int CH>
__device__ __forceinline__ void cn_line2(cplx<R> *__restrict__ b1, cplx<R> *__restrict__ b2, int es,
                                         const Coef *__restrict__ tab, const Coef *__restrict__ scan_s, Coef c) {
  const int t = threadIdx.x & (kWarp - 1);
  constexpr int mp = kWarp * CH;
  const Coef *alpha = tab + t, *beta = tab + mp + t, *H = tab + 2 * mp + t, *G = tab + 3 * mp + t;
  const Coef *scan = scan_s + t;
  cplx<R> y1[CH], y2[CH];
  cplx<R> a1 = czero<R>(), a2 = czero<R>();
#pragma unroll
  for (int e = 0; e < CH; ++e) {
    const Coef al = alpha[e * kWarp];
    const int q = (t * CH + e + 1 + t) * es;
    a1 = cfma(al, a1, b1[q]);
    a2 = cfma(al, a2, b2[q]);
    y1[e] = a1;
    y2[e] = a2;
  }
  cplx<R> B1 = a1, B2 = a2;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const Coef f = scan[k * kWarp];
    const cplx<R> p1 = shfl_up(B1, 1 << k), p2 = shfl_up(B2, 1 << k);
    if (t >= (1 << k)) {
      B1 = cfma(f, p1, B1);
      B2 = cfma(f, p2, B2);
    }
  }
  cplx<R> Y1 = shfl_up(B1, 1), Y2 = shfl_up(B2, 1);
  if (t == 0) Y1 = Y2 = czero<R>();
  a1 = a2 = czero<R>();
#pragma unroll
  for (int e = CH - 1; e >= 0; --e) {
    const Coef be = beta[e * kWarp];
    a1 = mul(be, cfma_c(c, a1, y1[e]));
    a2 = mul(be, cfma_c(c, a2, y2[e]));
    y1[e] = a1;
    y2[e] = a2;
  }
  const Coef h0 = H[0];
  cplx<R> C1 = cfma(h0, Y1, a1), C2 = cfma(h0, Y2, a2);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const Coef f = scan[(5 + k) * kWarp];
    const cplx<R> n1 = shfl_down(C1, 1 << k), n2 = shfl_down(C2, 1 << k);
    if (t + (1 << k) < kWarp) {
      C1 = cfma(f, n1, C1);
      C2 = cfma(f, n2, C2);
    }
  }
  cplx<R> X1 = shfl_down(C1, 1), X2 = shfl_down(C2, 1);
  if (t == kWarp - 1) X1 = X2 = czero<R>();
#pragma unroll
  for (int e = 0; e < CH; ++e) {
    const Coef h = H[e * kWarp], g = G[e * kWarp];
    const int q = (t * CH + e + 1 + t) * es;
    const cplx<R> chi1 = cfma(h, Y1, cfma(g, X1, y1[e])), chi2 = cfma(h, Y2, cfma(g, X2, y2[e]));
    const cplx<R> v1 = b1[q], v2 = b2[q];
    b1[q] = {twice_minus(chi1.re, v1.re), twice_minus(chi1.im, v1.im)};
    b2[q] = {twice_minus(chi2.re, v2.re), twice_minus(chi2.im, v2.im)};
  }
  if (t == 0) {
    b1[0] = czero<R>();
    b2[0] = czero<R>();
  }
}

// cn_line with the chunk length as a compile-time constant (every unrolled iteration live).
template <typename R, typename Coef, bool SHARED_TAB, bool FULL = false>
__device__ __forceinline__ void cn_line_any(cplx<R> *__restrict__ buf, int es, int m, int lchunk,
                                            const Coef *__restrict__ tab, const Coef *__restrict__ scan_s, Coef c) {
  switch (lchunk) {
    case 1: cn_line<R, Coef, 2, SHARED_TAB, FULL>(buf, es, m, lchunk, tab, scan_s, c); break;
    case 2: cn_line<R, Coef, 4, SHARED_TAB, FULL>(buf, es, m, lchunk, tab, scan_s, c); break;
    case 3: cn_line<R, Coef, 8, SHARED_TAB, FULL>(buf, es, m, lchunk, tab, scan_s, c); break;
    default: cn_line<R, Coef, 16, SHARED_TAB, FULL>(buf, es, m, lchunk, tab, scan_s, c); break;
  }
}
// cn_line2 (two lines in lockstep, padded to 32 whole chunks) at the chunk 2^lchunk
template <typename R, typename Coef>
__device__ __forceinline__ void cn_line2_any(cplx<R> *b1, cplx<R> *b2, int es, int lchunk, const Coef *tab,
                                             const Coef *scan_s, Coef c) {
  switch (lchunk) {
    case 1: cn_line2<R, Coef, 2>(b1, b2, es, tab, scan_s, c); break;
    case 2: cn_line2<R, Coef, 4>(b1, b2, es, tab, scan_s, c); break;
    case 3: cn_line2<R, Coef, 8>(b1, b2, es, tab, scan_s, c); break;
    default: cn_line2<R, Coef, 16>(b1, b2, es, tab, scan_s, c); break;
  }
}

template <typename R, typename Coef>
struct CnCoef;
template <typename R>
struct CnCoef<R, R> {
  __device__ static R make(R r) { return r; }
};
template <typename R>
struct CnCoef<R, cplx<R>> {
  __device__ static cplx<R> make(R r) { return {R(0), r}; }
};

// A host-precomputed constant in the kernel precision (no FP64 work per thread in FP32 and
// double-float): the double d, its FP32 rounding f and the FP32 remainder l = fl32(d - f).
template <typename R>
__device__ __forceinline__ R pick(double d, float f, float l);
template <>
__device__ __forceinline__ double pick<double>(double d, float, float) { return d; }
template <>
__device__ __forceinline__ float pick<float>(double, float f, float) { return f; }
template <>
__device__ __forceinline__ df pick<df>(double, float f, float l) { return {f, l}; }

// The pending renormalisation factor s of the device state (and s^2) in the kernel
// precision; the FP32 kernels read the FP32 copies, so they issue no FP64 instruction.
__device__ __forceinline__ void set_scale(DevState *st, double s) {
  st->s = s;
  st->sf = (float)s;
  st->sl = (float)(s - (double)st->sf);
  const double s2 = s * s;
  st->s2f = (float)s2;
  st->s2l = (float)(s2 - (double)st->s2f);
}
template <typename R>
__device__ __forceinline__ R scale_of(const DevState *st) {
  if constexpr (std::is_same<R, double>::value) return st->s;
  else if constexpr (std::is_same<R, df>::value) return df{st->sf, st->sl};
  else return st->sf;
}
template <typename R>
__device__ __forceinline__ R scale_sq_of(const DevState *st) {
  if constexpr (std::is_same<R, double>::value) return st->s * st->s;
  else if constexpr (std::is_same<R, df>::value) return df{st->s2f, st->s2l};
  else return st->s2f;
}

// ---------------------------------------------------------------------------------------
// Reductions (FP64): warp shuffle, then across warps; deterministic order.
// ---------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*red)[NV]) {
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
  const int nwarps = (blockDim.x + kWarp - 1) / kWarp;
#pragma unroll
  for (int q = 0; q < NV; ++q)
    for (int d = kWarp / 2; d > 0; d >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], d);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) red[warp][q] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      v[q] = lane < nwarps ? red[lane][q] : 0.0;
      for (int d = kWarp / 2; d > 0; d >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], d);
    }
  }
}

// Store this block's partial sums; the last block to finish adds all partials in block
// order and returns true (in every thread of that block) with the totals in thread 0.
template <int NV>
__device__ bool reduce_across_blocks(double (&v)[NV], double *partials, unsigned int *ticket) {
  __shared__ double red[32][NV];
  __shared__ bool last;
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  block_sum<NV>(v, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[(size_t)bid * NV + q] = v[q];
    __threadfence();
    const unsigned int prev = atomicAdd(ticket, 1u);
    last = (prev == (unsigned int)nblocks - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __ldcg(partials + (size_t)b * NV + q);
  block_sum<NV>(v, red);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

__device__ __forceinline__ double coordinate(int i, int n, double h) { return (double)(i - n / 2) * h; }

// Quadrature weight (times h) of index i on an axis of n points: 1 (rectangle rule), or
// composite Simpson (1, 4, 2, ..., 4, 1)/3 on indices 0..n-2 and 0 on the last point (a wall).
__device__ __forceinline__ double quad_weight(int i, int n, int simpson) {
  if (!simpson) return 1.0;
  if (i > n - 2) return 0.0;
  if (i == 0 || i == n - 2) return 1.0 / 3.0;
  return (i & 1) ? 4.0 / 3.0 : 2.0 / 3.0;
}

// 3 x the quadrature weight: 1 (rectangle rule: the factor 3 is not applied), or Simpson's
// 1, 4, 2, ..., 4, 1 and 0 on the last point, all exact small integers.
__device__ __forceinline__ int quad_weight3(int i, int n, int simpson) {
  if (!simpson) return 1;
  if (i > n - 2) return 0;
  if (i == 0 || i == n - 2) return 1;
  return (i & 1) ? 4 : 2;
}

template <typename R>
__device__ __forceinline__ R quad_weight_r(int i, int n, int simpson) {
  if (!simpson) return R(1);
  if (i > n - 2) return R(0);
  if (i == 0 || i == n - 2) return R(1.0 / 3.0);
  return (i & 1) ? R(4.0 / 3.0) : R(2.0 / 3.0);
}

// ---------------------------------------------------------------------------------------
// Set-up kernels
// ---------------------------------------------------------------------------------------
// Per-stage twiddle tables of a plan (layout in FftPlan): entry twoff[s] + k (P-1) + r - 1
// = e^{-2 pi i r k / (ns P)}, or its tangent form {t_r, S_r} (see TangentTw) for the FP64
// radix-2/4/8 stages.
// sigma and t of the tangent form of e^{-2 pi i a / M}
__device__ inline void tangent_twiddle(int a, int M, double *sigma, double *t) {
  double s, c;
  sincospi(2.0 * (double)a / (double)M, &s, &c);
  if (tw_rot(a, M)) {   // e^{-i phi} = -sin phi * i * (1 + i cot phi)
    *sigma = -s;
    *t = c / s;
  } else {              // e^{-i phi} = cos phi * (1 - i tan phi)
    *sigma = c;
    *t = -s / c;
  }
}
template <typename R>
__global__ void k_twiddles(cplx<R> *tw, FftPlan pl) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= pl.n - 1) return;
  int st = 0, ns = 1;
  while (st + 1 < pl.nstages && t >= pl.twoff[st + 1]) {
    ns *= pl.radix[st];
    ++st;
  }
  const int p = pl.radix[st];
  const int q = t - pl.twoff[st];
  const int k = q / (p - 1), r = q - k * (p - 1) + 1;
  const int M = ns * p;
  if (std::is_same<R, double>::value && (p == 2 || p == 4 || p == 8)) {
    // the scale stored with t_r: sigma_r, or sigma_r over the scale it is folded against
    const int den = (p == 4 && r == 3) || (p == 8 && (r == 3 || r == 5)) ? 1
                    : p == 8 && r == 6                                   ? 2
                    : p == 8 && r == 7                                   ? 3
                                                                         : 0;
    double sg, tr, sd = 1.0, td;
    tangent_twiddle(r * k, M, &sg, &tr);
    if (den) tangent_twiddle(den * k, M, &sd, &td);
    tw[t] = {R(tr), R(sg / sd)};
    return;
  }
  double s, c;
  sincospi(2.0 * (double)(r * k) / (double)M, &s, &c);
  tw[t] = {R(c), R(-s)};
}

// LU factors of tridiag(-c, 1 + 2c, -c) (order m) and the chunk response tables P, H, G
// of the chunked Thomas solve (see cn_line), computed in FP64 by one thread in one pass:
//   e_0 = 1 + 2c, e_i = 1 + 2c - c alpha_i, alpha_i = c / e_{i-1}, beta_i = 1 / e_i;
//   per chunk [s0, end]: P_s0 = alpha_s0, P_i = alpha_i P_{i-1};
//   H_end = beta_end P_end, H_i = beta_i (P_i + c H_{i+1});
//   G_end = beta_end c,     G_i = beta_i c G_{i+1};
// alpha, beta, H and G are stored; P only enters the forward scan factors (P at each chunk
// end, then the running products of the scan), stored after them with the backward ones.
struct Z64 {
  double re, im;
};
__device__ __forceinline__ Z64 zmul(Z64 a, Z64 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Z64 zadd(Z64 a, Z64 b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Z64 zdiv(Z64 a, Z64 b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

template <typename R, typename Coef>
__device__ __forceinline__ void store_coef(Coef *tab, int k, Z64 v) {
  if constexpr (sizeof(Coef) == sizeof(R)) tab[k] = Coef(v.re);
  else tab[k] = Coef{R(v.re), R(v.im)};
}

template <typename R, typename Coef>
__global__ void k_cn_tables(CnJobs jobs) {
  if (threadIdx.x != 0 || (int)blockIdx.x >= jobs.n) return;
  const CnJob &jb = jobs.job[blockIdx.x];
  Coef *tab = static_cast<Coef *>(jb.tab);
  const int m = jb.m, chunk = jb.chunk, imag = jobs.imag;
  const int L = jb.lanes == 8 ? 8 : kWarp, lg = L == 8 ? 3 : 5;   // lanes per line, log2
  const double r = jb.r;
  // lane-interleaved layout: interior point i = t*chunk + e of table q at q*mp + e*L + t
  const int mp = L * chunk;
  auto at = [&](int q, int i) { return q * mp + (i % chunk) * L + i / chunk; };
  const Z64 c = imag ? Z64{r, 0.0} : Z64{0.0, r};
  const Z64 diag = {1.0 + 2.0 * c.re, 2.0 * c.im};
  const Z64 one = {1.0, 0.0};
  Z64 al[kCnMaxChunk], be[kCnMaxChunk], pv[kCnMaxChunk];
  Z64 fa[kWarp], ba[kWarp];   // per lane: P at the chunk end, G at the chunk start
  for (int t = 0; t < kWarp; ++t) fa[t] = ba[t] = one;
  Z64 e_prev = diag;
  const int h = m / 2;   // the twist point of the two-thread (twisted) sweeps
  Z64 e_h = diag, e_hm = diag;
  // all L chunks: positions i >= m are padding, decoupled (alpha = 0, e = 1), so a solve
  // over the padded length with zero values there gives zero there and leaves the m real
  // unknowns exactly as they are (the padding only ever multiplies zeros)
  for (int s0 = 0; s0 < L * chunk; s0 += chunk) {
    const int end = s0 + chunk - 1;
    for (int i = s0; i <= end; ++i) {
      Z64 a = {0.0, 0.0}, e = diag;
      if (i >= m) {
        e = one;
      } else if (i > 0) {
        a = zdiv(c, e_prev);
        const Z64 ca = zmul(c, a);
        e = Z64{diag.re - ca.re, diag.im - ca.im};
      }
      if (i == h) e_h = e;
      if (i == m - 1 - h) e_hm = e;
      al[i - s0] = a;
      be[i - s0] = zdiv(one, e);
      e_prev = e;
      store_coef<R>(tab, at(0, i), a);
      store_coef<R>(tab, at(1, i), be[i - s0]);
    }
    Z64 p = al[0];
    pv[0] = p;
    for (int i = s0 + 1; i <= end; ++i) {
      p = zmul(p, al[i - s0]);
      pv[i - s0] = p;
    }
    Z64 h = zmul(be[end - s0], pv[end - s0]);
    Z64 gg = zmul(be[end - s0], c);
    store_coef<R>(tab, at(2, end), h);
    store_coef<R>(tab, at(3, end), gg);
    for (int i = end - 1; i >= s0; --i) {
      h = zmul(be[i - s0], zadd(pv[i - s0], zmul(c, h)));
      gg = zmul(be[i - s0], zmul(c, gg));
      store_coef<R>(tab, at(2, i), h);
      store_coef<R>(tab, at(3, i), gg);
    }
    fa[s0 / chunk] = pv[end - s0];
    ba[s0 / chunk] = gg;
  }
  // Kogge-Stone scan factors: before step k (offset d = 2^k) lane t holds the product of
  // the factors of lanes t - 2^k + 1 .. t (forward) or t .. t + 2^k - 1 (backward).
  // Layout: forward step k at 4 mp + k L + t, backward step k at 4 mp + (lg + k) L + t.
  for (int k = 0, d = 1; d < L; ++k, d <<= 1) {
    for (int t = 0; t < L; ++t) {
      store_coef<R>(tab, 4 * mp + k * L + t, fa[t]);
      store_coef<R>(tab, 4 * mp + (lg + k) * L + t, ba[t]);
    }
    for (int t = L - 1; t >= d; --t) fa[t] = zmul(fa[t], fa[t - d]);
    for (int t = 0; t + d < L; ++t) ba[t] = zmul(ba[t], ba[t + d]);
  }
  // 1/gamma, gamma = e_h + e_{m-1-h} - (1 + 2c): the pivot of the twist point
  store_coef<R>(tab, 4 * mp + 2 * lg * L, zdiv(one, Z64{e_h.re + e_hm.re - diag.re, e_h.im + e_hm.im - diag.im}));
}

// dt v_d x_i^2 on one axis, x_i = (i - n/2) h (the potential-step angle, per axis).
template <typename R>
__global__ void k_axis_potential(R *out, int n, double h, double v, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double x = (double)(i - n / 2) * h;
    out[i] = R(dt * v * x * x);
  }
}

// Cutoff factor c(x) = 1 + 3 cos x / x^2 - 3 sin x / x^3 = 3 int_0^x j_2(t)/t dt of the
// spherically truncated dipolar interaction; below x = 0.5 its Taylor series
// sum_{n>=2} (-1)^n 6n x^(2n-2) / (2n+1)!, where the closed form cancels.
template <typename R>
__device__ __forceinline__ R cutoff_factor(R x) {
  if (x >= R(0.5)) {
    R sn, cs;
    sin_cos(x, &sn, &cs);
    const R ix2 = R(1) / (x * x);
    return R(1) + R(3) * cs * ix2 - R(3) * sn * ix2 / x;
  }
  const R u = x * x;
  // coefficients 6n/(2n+1)! for n = 2..9 (alternating signs)
  R p = R(6.0 * 9 / 121645100408832000.0);
  p = fma(p, -u, R(6.0 * 8 / 355687428096000.0));
  p = fma(p, -u, R(6.0 * 7 / 1307674368000.0));
  p = fma(p, -u, R(6.0 * 6 / 6227020800.0));
  p = fma(p, -u, R(6.0 * 5 / 39916800.0));
  p = fma(p, -u, R(6.0 * 4 / 362880.0));
  p = fma(p, -u, R(6.0 * 3 / 5040.0));
  p = fma(p, -u, R(6.0 * 2 / 120.0));
  return p * u;
}

// Ut(k) = 3 kz^2 / |k|^2 - 1 (Ut(0) = 0), times the cutoff factor when a cutoff is set, on
// the half spectrum [m][i][j] (kz index m <= nz/2, kx index i, ky index j), computed in
// FP64: k_d = 2 pi q / (n_d h_d) with the signed frequency q (q <= n/2: q, else q - n).
template <typename R>
__global__ void k_dipolar_table(R *ut, KArgs a) {
  const size_t total = (size_t)a.nzh * a.nx * a.ny;
  const double two_pi = 6.283185307179586476925286766559;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % a.ny);
    const size_t r = e / a.ny;
    const int i = (int)(r % a.nx), m = (int)(r / a.nx);
    const int qx = i <= a.nx / 2 ? i : i - a.nx, qy = j <= a.ny / 2 ? j : j - a.ny;
    const double kx = two_pi * qx / (a.nx * a.hx), ky = two_pi * qy / (a.ny * a.hy), kz = two_pi * m / (a.nz * a.hz);
    const double k2 = kx * kx + ky * ky + kz * kz;
    double u = k2 > 0.0 ? 3.0 * kz * kz / k2 - 1.0 : 0.0;
    if (a.cutoff > 0.0 && k2 > 0.0) u *= cutoff_factor<double>(sqrt(k2) * a.cutoff);
    ut[e] = R(u);
  }
}

// Double-float boundary: complex128 values split into (hi, lo) pairs (in place allowed:
// each thread reads its 16 bytes before writing them), and pairs summed back to complex128
// (after the pending renormalisation has been applied by k_materialize).
template <typename R>
__global__ void k_c128_to_pair(const double2 *src, cplx<R> *psi, size_t n) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const double2 v = src[q];
    psi[q] = {R(v.x), R(v.y)};
  }
}
template <typename R>
__global__ void k_pair_to_c128(const cplx<R> *psi, double2 *dst, size_t n) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const cplx<R> v = psi[q];
    dst[q] = make_double2((double)v.re, (double)v.im);
  }
}

template <typename R>
__global__ void k_reset_state(DevState *st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    set_scale(st, 1.0);
    st->norm = 0.0;
    st->norm_in = 0.0;
    st->norm_ref = 0.0;
    st->flags = 0u;
    st->ticket = 0u;
    st->steps = 0ull;
  }
}

// d / 2 for a density d >= 0, exactly and off the FP64 pipe: the exponent field minus one
// for 2^-1021 <= d < inf; 0 below (the half would be subnormal, under 2.3e-308: flushed);
// inf and NaN unchanged.  Other types multiply.
template <typename R>
__device__ __forceinline__ R half_density(R d) { return R(0.5) * d; }
template <>
__device__ __forceinline__ double half_density(double d) {
  const long long b = __double_as_longlong(d);
  const long long h = b < (2LL << 52) ? 0LL : (b >= 0x7ff0000000000000LL ? b : b - (1LL << 52));
  return __longlong_as_double(h);
}

// The CTA `ahead` positions after this one in launch order (x fastest, then y, then the
// member z of a grouped launch), for the L2 prefetch of the tile kernels: its tile (x-row
// i2, j-tile bx2) and its member's arguments (ga + z2 for grouped launches, else a).  False
// past the end of the grid.
struct AheadTile {
  int i2, bx2;
  const KArgs *b;
};
__device__ __forceinline__ bool ahead_tile(const KArgs &a, const KArgs *ga, int ahead, AheadTile &t) {
  // (32-bit: a grid of these kernels holds far fewer than 2^31 CTAs)
  const unsigned gx = gridDim.x, gxy = gx * gridDim.y;
  const unsigned L = (blockIdx.z * gridDim.y + blockIdx.y) * gx + blockIdx.x + (unsigned)ahead;
  if (ahead <= 0 || L >= gxy * gridDim.z) return false;
  const unsigned z2 = ga ? L / gxy : 0u, rem = L - z2 * gxy;
  t.i2 = (int)(rem / gx);
  t.bx2 = (int)(rem - (unsigned)t.i2 * gx);
  t.b = ga ? ga + z2 : &a;
  return true;
}

// ---------------------------------------------------------------------------------------
// K1: n = s^2 |psi|^2 of kZLines consecutive z-lines (i, j0..), packed in pairs as the
// real and imaginary parts of one complex line, forward FFT along z, then the two real
// spectra are separated (X1 = (Z_m + conj Z_{N-m})/2, X2 = (Z_m - conj Z_{N-m})/2i; the 1/2
// is applied exactly to the packed density instead) and
// the half spectrum m = 0..nz/2 is stored to spec[m][i][j].
// ---------------------------------------------------------------------------------------
template <typename R, int N>
__device__ __forceinline__ void k1_density_r2cz_body(const KArgs &a, const KArgs *ga) {
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int BZ = ztile_lines<R>(N);
  constexpr int PZ = BZ / 2;
  constexpr int SB = PZ + 1;
  const int nz = N > 0 ? N : a.nz, i = blockIdx.y, j0 = blockIdx.x * BZ;
  const int nl = min(BZ, a.ny - j0), np = nl >> 1;
  C *za = reinterpret_cast<C *>(smem_raw);
  C *zb = za + nz * SB;
  // the packed density carries a factor 1/2 (exact), so the separation below needs none
  const R s2 = R(0.5) * (a.unit_scale ? R(1) : scale_sq_of<R>(a.state));
  const C *psi = reinterpret_cast<const C *>(a.psi) + ((size_t)i * a.ny + j0) * nz;
  const int total = nl * nz;
  // kHalve: s = 1 (real time), so the factor is the 1/2 alone, applied to FP64 densities by
  // the exponent (half_density) instead of a multiply on the FP64 pipe
  auto fill = [&](auto halve) {
    constexpr bool kHalve = decltype(halve)::value;
    if constexpr (N > 0 && !Fp64Class<R>::value) {
      // FP32, compile-time length: thread (line b, offset k0 < W) takes the points k0 + W j of
      // line b (W consecutive points of a line per W lanes: coalesced loads; at W = 16 the
      // 4-byte stores into the pair-interleaved buffer, stride SB = 9 pairs, fall on 16 distinct
      // banks per line, at W = 8 (32-line tiles) on two-way shared banks)
      constexpr int W = Tiles<R>::kZThreads / BZ;
      const int b = threadIdx.x / W, k0 = threadIdx.x % W;
      if (b < nl) {
        const C *src = psi + (size_t)b * nz + k0;
        R *z = reinterpret_cast<R *>(za + k0 * SB + (b >> 1)) + (b & 1);
#pragma unroll 8
        for (int j = 0; j < N / W; ++j) {
          const C v = src[W * j];
          z[2 * SB * W * j] = s2 * (v.re * v.re + v.im * v.im);
        }
      }
      // the psi rows of the CTA one resident wave ahead into L2 (residency: the CTAs whose
      // two transform buffers fit the SM's shared memory, at most 6 by registers)
      constexpr int kRes = (228 * 1024) / (2 * N * SB * (int)sizeof(C) + 1024) < 6 ? (228 * 1024) / (2 * N * SB * (int)sizeof(C) + 1024) : 6;
      AheadTile t;
      if (threadIdx.x == 0 && ahead_tile(a, ga, kRes * a.nsm, t)) {
        const int j2 = t.bx2 * BZ;
        prefetch_l2(reinterpret_cast<const C *>(t.b->psi) + ((size_t)t.i2 * a.ny + j2) * nz, min(BZ, a.ny - j2) * nz * (unsigned)sizeof(C));
      }
      return;
    }
    LinePos pos(threadIdx.x, nz, blockDim.x);
    for (int e0 = threadIdx.x; e0 < total; e0 += kUnroll * blockDim.x) {
      C v[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < total) v[u] = psi[e];
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < total) {
          R *z = reinterpret_cast<R *>(za + pos.k * SB + (pos.b >> 1));
          const R d = v[u].re * v[u].re + v[u].im * v[u].im;
          if constexpr (kHalve) z[pos.b & 1] = half_density(d);
          else z[pos.b & 1] = s2 * d;
        }
        pos.next();
      }
    }
  };
  if (std::is_same<R, double>::value && s2 == R(0.5)) fill(std::true_type{});
  else fill(std::false_type{});
  __syncthreads();
  const C *res = fft_lines_n<R, -1, N, PZ, SB, Tiles<R>::kZThreads>(za, zb, a.plan[2], np,
                                                                   reinterpret_cast<const C *>(a.tw[2]));
  C *spec = reinterpret_cast<C *>(a.spec) + (size_t)i * a.ny + j0;
  const size_t plane = (size_t)a.nx * a.ny;
  const int p = threadIdx.x % PZ;
  if (p < np) {
    for (int m = threadIdx.x / PZ; m < a.nzh; m += blockDim.x / PZ) {
      const C zm = res[m * SB + p];
      const C zc = res[((nz - m) % nz) * SB + p];
      const C x1 = {zm.re + zc.re, zm.im - zc.im};
      const C x2 = {zm.im + zc.im, zc.re - zm.re};
      C *dst = spec + m * plane + 2 * p;
      dst[0] = x1;
      dst[1] = x2;
    }
  }
}
// one condensate (G = false, its arguments passed by value), or condensate blockIdx.z of
// a group of same-shaped condensates (G = true, the arguments from the device array ga)
template <typename R, int N, bool G = false>
__global__ void __launch_bounds__(Tiles<R>::kZThreads) k1_density_r2cz(KArgs a, const KArgs *ga) {
  if constexpr (G) k1_density_r2cz_body<R, N>(ga[blockIdx.z], ga);
  else k1_density_r2cz_body<R, N>(a, nullptr);
}

// ---------------------------------------------------------------------------------------
// K2 / K4: FFT along y of the contiguous lines spec[m][i][:].
// ---------------------------------------------------------------------------------------
template <typename R, int DIR, int N>
__device__ __forceinline__ void k_ffty_body(const KArgs &a) {
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // N > 0: ny = N with the default lines per CTA and 256 threads, fixed at compile time
  constexpr int LC = N > 0 ? y_lines_per_cta<R>(N) : 0;
  const int n = N > 0 ? N : a.ny;
  const int L = N > 0 ? LC : a.ylines;
  const int SB = L + 1;
  const size_t total = (size_t)a.nzh * a.nx;
  const size_t l0 = (size_t)blockIdx.x * L;
  const int nl = (int)min((size_t)L, total - l0);
  C *za = reinterpret_cast<C *>(smem_raw);
  C *zb = za + n * SB;
  C *spec = reinterpret_cast<C *>(a.spec) + l0 * n;
  {
    LinePos pos(threadIdx.x, n, blockDim.x);
    for (int e = threadIdx.x; e < nl * n; e += blockDim.x, pos.next()) cp_async(za + pos.k * SB + pos.b, spec + e);
  }
  cp_async_wait_all();
  __syncthreads();
  const C *res;
  if constexpr (N > 0)
    res = fft_lines_ct<R, DIR, N, LC, LC + 1, kFftThreads>(za, zb, nl, reinterpret_cast<const C *>(a.tw[1]));
  else
    res = fft_lines<R, DIR>(za, zb, a.plan[1], L, nl, SB, reinterpret_cast<const C *>(a.tw[1]));
  LinePos pos(threadIdx.x, n, blockDim.x);
#pragma unroll 4
  for (int e = threadIdx.x; e < nl * n; e += blockDim.x, pos.next()) spec[e] = res[pos.k * SB + pos.b];
}
// one condensate (G = false, its arguments passed by value), or condensate blockIdx.z of
// a group of same-shaped condensates (G = true, the arguments from the device array ga)
template <typename R, int DIR, int N, bool G = false>
__global__ void __launch_bounds__(kFftThreads) k_ffty(KArgs a, const KArgs *ga) {
  if constexpr (G) k_ffty_body<R, DIR, N>(ga[blockIdx.z]);
  else k_ffty_body<R, DIR, N>(a);
}

// ---------------------------------------------------------------------------------------
// K3: for the plane kz = m, lines along x (stride ny), kXCols consecutive ky per CTA:
// forward FFT along x, multiply by Ut(kx, ky, kz) = 3 kz^2 / |k|^2 - 1 (Ut(0) = 0),
// inverse FFT along x.
// ---------------------------------------------------------------------------------------
template <typename R, int N>
__device__ __forceinline__ void k3_fftx_dipolar_body(const KArgs &a) {
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int BX = Tiles<R>::kXCols;
  constexpr int SB = BX;
  const int n = N > 0 ? N : a.nx, m = blockIdx.y, j0 = blockIdx.x * BX;
  const int nb = min(BX, a.ny - j0);
  C *za = reinterpret_cast<C *>(smem_raw);
  C *zb = za + n * SB;
  C *spec = reinterpret_cast<C *>(a.spec) + (size_t)m * a.nx * a.ny + j0;
  for (int e = threadIdx.x; e < n * BX; e += blockDim.x) {
    const int b = e % BX, k = e / BX;
    if (b < nb) cp_async(za + k * SB + b, spec + (size_t)k * a.ny + b);
  }
  cp_async_wait_all();
  __syncthreads();
  const C *tw = reinterpret_cast<const C *>(a.tw[0]);
  C *res = fft_lines_n<R, -1, N, BX, SB, kFftThreads>(za, zb, a.plan[0], nb, tw);
  const int b = threadIdx.x % BX;
  if (b < nb) {
    if constexpr (Fp64Class<R>::value) {
      // FP64 (and double-float): the table (the division and the cutoff factor would cost
      // more than the read)
      const R *ut = reinterpret_cast<const R *>(a.utab) + (size_t)m * a.nx * a.ny + j0;
      for (int k = threadIdx.x / BX; k < n; k += blockDim.x / BX)
        res[k * SB + b] = scale(res[k * SB + b], ldg(ut + (size_t)k * a.ny + b));
    } else {
      // FP32: in place, k_d = q_d * (2 pi / (n_d h_d)) with the signed frequency q_d
      const R fx = a.kf[0], fy = a.kf[1], fz = a.kf[2];
      const int jy = j0 + b;
      const R ky = R(jy <= a.ny / 2 ? jy : jy - a.ny) * fy, kz = R(m) * fz;
      const R kz2 = kz * kz, kyz2 = fma(ky, ky, kz2);
      for (int k = threadIdx.x / BX; k < n; k += blockDim.x / BX) {
        const R kx = R(k <= n / 2 ? k : k - n) * fx;
        const R k2 = fma(kx, kx, kyz2);
        R u = k2 > R(0) ? __fdividef(R(3) * kz2, k2) - R(1) : R(0);
        if (a.has_cutoff && k2 > R(0)) u *= cutoff_factor<R>(sqrt(k2) * a.cutoff_f);
        res[k * SB + b] = scale(res[k * SB + b], u);
      }
    }
  }
  __syncthreads();
  C *other = (res == za) ? zb : za;
  const C *out = fft_lines_n<R, +1, N, BX, SB, kFftThreads>(res, other, a.plan[0], nb, tw);
#pragma unroll 4
  for (int e = threadIdx.x; e < n * BX; e += blockDim.x) {
    const int b = e % BX, k = e / BX;
    if (b < nb) spec[(size_t)k * a.ny + b] = out[k * SB + b];
  }
}
// one condensate (G = false, its arguments passed by value), or condensate blockIdx.z of
// a group of same-shaped condensates (G = true, the arguments from the device array ga)
template <typename R, int N, bool G = false>
__global__ void __launch_bounds__(kFftThreads) k3_fftx_dipolar(KArgs a, const KArgs *ga) {
  if constexpr (G) k3_fftx_dipolar_body<R, N>(ga[blockIdx.z]);
  else k3_fftx_dipolar_body<R, N>(a);
}

// ---------------------------------------------------------------------------------------
// Register-resident transforms (FP32) of lines of N = 64 Q points (Q = 2, 4 or 8) with
// T = N/8 threads per line: thread t holds elements t + T r (r = 0..7) of its line before
// and after the transform.  Three Stockham stages of the default plan (radix 8, 8, Q): the
// first and the last in registers, two exchanges through shared memory between them.  The
// callers load the registers straight from global memory and store them straight back
// (consecutive t on consecutive lanes: coalesced), so a transform costs two shared-memory
// round trips instead of a staging copy and one round trip per stage; and a forward
// transform leaves its output in the layout the inverse transform's input needs.
// Stage 1 (ns = 1):  butterfly t on x[t + T r]             -> y[8 t + s]
// Stage 2 (ns = 8):  butterfly t on y[t + T r], k = t mod 8 -> z[8 (t - k) + k + 8 s]
// Stage 3 (ns = 64): butterflies j = t + T u (u < 8/Q) on z[j + 64 r], k = j -> o[j + 64 s]
//                    = o[t + T (u + (8/Q) s)]
// Shared memory: element i of a line at pad(i) * LS (+ the caller's column offset),
// pad(i) = i + i/8.  With LS = 1 (one line per buffer) or LS = 8 (eight columns
// interleaved, lanes spanning the columns), every access above is free of bank conflicts
// within a half-warp.
// ---------------------------------------------------------------------------------------
template <int N>
struct RegFft {
  static_assert(N == 128 || N == 256 || N == 512, "N = 64 Q, Q = 2, 4 or 8");
  static constexpr int Q = N / 64;
  static constexpr int T = N / 8;
  static constexpr int SLOTS = N + N / 8;
  __device__ static __forceinline__ int pad(int i) { return i + (i >> 3); }
};

template <int DIR>
__device__ __forceinline__ cplx<float> twiddle(cplx<float> v, cplx<float> w) {
  return DIR < 0 ? v * w : mul_conj(v, w);
}

// One transform of the registers v (see RegFft).  sa, sb: this line's two shared buffers
// (element i at pad(i) * LS); tw: the per-stage twiddle table of the default plan of length
// N (stage 2 at offset 7, stage 3 at offset 63); sync: the barrier that spans the threads
// of the line (and of every line that shares them).
template <int DIR, int N, int LS, typename Sync>
__device__ __forceinline__ void reg_fft(cplx<float> (&v)[8], cplx<float> *__restrict__ sa, cplx<float> *__restrict__ sb,
                                        int t, const cplx<float> *__restrict__ tw, Sync sync) {
  using F = RegFft<N>;
  using C = cplx<float>;
  constexpr int T = F::T, Q = F::Q, U = 8 / Q;
  // the padded indices, pad(i) = i + i/8, are linear in the unrolled counters (T and 64 are
  // multiples of 8): computed once per thread, the rest are immediate offsets
  //   stage 1 writes pad(8 t + s)             = 9 t + s (s < 8)
  //   stage 2 reads  pad(t + T r)             = (t + t/8) + r (9 T / 8)
  //   stage 2 writes pad(8 (t - k) + k + 8 s) = 72 (t/8) + k + 9 s,  k = t mod 8
  //   stage 3 reads  pad(j + 64 r)            = (j + j/8) + 72 r,    j = t + T u
  const int rd = t + (t >> 3);
  butterfly<float, DIR, 8>(v);
#pragma unroll
  for (int s = 0; s < 8; ++s) sa[(9 * t + s) * LS] = v[s];
  sync();
  {
    const int k = t & 7;
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = sa[(rd + r * (9 * T / 8)) * LS];
#pragma unroll
    for (int r = 1; r < 8; ++r) v[r] = twiddle<DIR>(v[r], ldg(tw + 7 + k * 7 + r - 1));
    butterfly<float, DIR, 8>(v);
    const int wr = 72 * (t >> 3) + k;
#pragma unroll
    for (int s = 0; s < 8; ++s) sb[(wr + 9 * s) * LS] = v[s];
  }
  sync();
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int j = t + T * u;
    const int rj = rd + T * u + (T / 8) * u;   // pad(j): T u is a multiple of 8
    C w[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) w[r] = sb[(rj + 72 * r) * LS];
#pragma unroll
    for (int r = 1; r < Q; ++r) w[r] = twiddle<DIR>(w[r], ldg(tw + 63 + j * (Q - 1) + r - 1));
    butterfly<float, DIR, Q>(w);
#pragma unroll
    for (int s = 0; s < Q; ++s) v[u + U * s] = w[s];
  }
}

// K2 / K4 in FP32 for ny = 128, 256 or 512 with the default plan: 256 / T lines per CTA,
// each line's registers loaded from and stored to global memory directly.
template <int DIR, int N>
__device__ __forceinline__ void k_ffty_reg_body(const KArgs &a) {
  using C = cplx<float>;
  using F = RegFft<N>;
  constexpr int T = F::T, LPC = 256 / T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = threadIdx.x / T, t = threadIdx.x % T;
  const size_t line = (size_t)blockIdx.x * LPC + l;
  const bool active = line < (size_t)a.nzh * a.nx;
  C *sa = reinterpret_cast<C *>(smem_raw) + (size_t)l * 2 * F::SLOTS;
  C *g = reinterpret_cast<C *>(a.spec) + (active ? line : 0) * N;
  C v[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = active ? g[t + T * r] : czero<float>();
  auto sync = [] {
    if constexpr (T > kWarp) __syncthreads();
    else __syncwarp();
  };
  reg_fft<DIR, N, 1>(v, sa, sa + F::SLOTS, t, reinterpret_cast<const C *>(a.tw[1]), sync);
  if (active) {
#pragma unroll
    for (int r = 0; r < 8; ++r) g[t + T * r] = v[r];
  }
}
// one condensate (G = false, its arguments passed by value), or condensate blockIdx.z of
// a group of same-shaped condensates (G = true, the arguments from the device array ga)
template <int DIR, int N, bool G = false>
__global__ void __launch_bounds__(256, 4) k_ffty_reg(KArgs a, const KArgs *ga) {
  if constexpr (G) k_ffty_reg_body<DIR, N>(ga[blockIdx.z]);
  else k_ffty_reg_body<DIR, N>(a);
}

// K3 in FP32 for nx = 128, 256 or 512 with the default plan: the forward transform along x,
// the product with Ut(k) in registers (each thread's outputs are exactly its inputs of the
// inverse transform), the inverse transform; 8 consecutive ky columns per CTA, the lanes of
// a warp spanning them (64-byte rows), the columns interleaved in shared memory.
template <int N>
__device__ __forceinline__ void k3_reg_body(const KArgs &a) {
  using C = cplx<float>;
  using F = RegFft<N>;
  constexpr int T = F::T, B = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = threadIdx.x % B, t = threadIdx.x / B;
  const int m = blockIdx.y, j0 = blockIdx.x * B;
  const int jy = j0 + b;
  const bool active = jy < a.ny;
  C *sa = reinterpret_cast<C *>(smem_raw) + b;
  C *sb = sa + (size_t)B * F::SLOTS;
  C *g = reinterpret_cast<C *>(a.spec) + (size_t)m * a.nx * a.ny + (active ? jy : 0);
  const size_t sx = (size_t)a.ny;
  C v[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = active ? g[(size_t)(t + T * r) * sx] : czero<float>();
  const C *tw = reinterpret_cast<const C *>(a.tw[0]);
  auto sync = [] { __syncthreads(); };
  reg_fft<-1, N, B>(v, sa, sb, t, tw, sync);
  // Ut(k) = 3 kz^2 / |k|^2 - 1 (Ut(0) = 0) at kx index t + T q, k_d = q_d 2 pi / (n_d h_d)
  {
    const float fx = a.kf[0], fy = a.kf[1], fz = a.kf[2];
    const float ky = (float)(jy <= a.ny / 2 ? jy : jy - a.ny) * fy, kz = (float)m * fz;
    const float kz2 = kz * kz, kyz2 = fmaf(ky, ky, kz2);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = t + T * q;
      const float kx = (float)(i <= N / 2 ? i : i - N) * fx;
      const float k2 = fmaf(kx, kx, kyz2);
      float u = k2 > 0.0f ? __fdividef(3.0f * kz2, k2) - 1.0f : 0.0f;
      if (a.has_cutoff && k2 > 0.0f) u *= cutoff_factor<float>(sqrtf(k2) * a.cutoff_f);
      v[q] = scale(v[q], u);
    }
  }
  __syncthreads();   // the inverse transform's first exchange reuses sa
  reg_fft<+1, N, B>(v, sa, sb, t, tw, sync);
  if (active) {
#pragma unroll
    for (int r = 0; r < 8; ++r) g[(size_t)(t + T * r) * sx] = v[r];
  }
}
// one condensate (G = false, its arguments passed by value), or condensate blockIdx.z of
// a group of same-shaped condensates (G = true, the arguments from the device array ga)
template <int N, bool G = false>
__global__ void __launch_bounds__(8 * RegFft<N>::T, 1024 / (8 * RegFft<N>::T)) k3_reg(KArgs a, const KArgs *ga) {
  if constexpr (G) k3_reg_body<N>(ga[blockIdx.z]);
  else k3_reg_body<N>(a);
}

// ---------------------------------------------------------------------------------------
// K5: the z-line kernel.  For kZLines lines (i, j0..): inverse half-spectrum transform
// along z (C2R, two real lines per complex FFT; the imaginary parts of the kz = 0 and
// kz = nz/2 bins are dropped), Phi = result / (nx ny nz); then, per zmode, the potential
// step psi <- s psi e^{-i theta} (real time) or s psi e^{-theta} (imaginary time) with
// theta = dt (V + g s^2 |psi|^2 + gdd Phi), and the Crank-Nicolson solve along z.
// The FP64 phase-only pass runs three CTAs per SM (80 registers and a few spills beat two).
// ---------------------------------------------------------------------------------------
template <typename R, typename Coef, int ZM, int N>
__device__ __forceinline__ void k5_zline_body(const KArgs &a, const KArgs *ga) {
  constexpr int zmode = ZM;   // one instance per mode: each gets its own register allocation
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int BZ = ztile_lines<R>(N);
  constexpr int PZ = BZ / 2;
  constexpr int SB = PZ;   // unpadded: the butterflies (pair fastest) and the line-fastest phase loop are conflict-free
  const int nz = N > 0 ? N : a.nz, i = blockIdx.y, j0 = blockIdx.x * BZ;
  const int nl = min(BZ, a.ny - j0), np = nl >> 1;
  const int lc = a.cn[2].lchunk;
  // Compile-time lengths (FP32, the fused step): the z solve takes CHZ = k5_chunk(N) points
  // per lane on a line padded to 32 CHZ unknowns (every lane busy, no per-point guard), the
  // tile one pad slot per CHZ points, lines kept at an odd stride (distinct banks across
  // lines); the tile loops walk period PW = lcm(W, CHZ) (W = threads / lines).
  constexpr int W = Tiles<R>::kZThreads / BZ;
  constexpr bool kWalk = N > 0 && !Fp64Class<R>::value;
  // lines of 64, 96, 128: the z solve on 8 lanes per line (8, 12, 16 points each, three scan
  // steps), the tables in the 8-lane layout; longer lines on 32 lanes
  constexpr int LZ = kWalk && k5_short_z(N) ? 8 : kWarp;
  constexpr int CHZ = kWalk ? (LZ == 8 ? N / 8 : k5_chunk(N)) : 1;
  constexpr int PW = kWalk ? W / gcd_c(W, CHZ) * CHZ : W;
  constexpr int SUBS = PW / W;
  static_assert(!kWalk || (N % PW == 0 && zmode == kZStep), "compile-time FP32 instances: the fused step");
  const int LS = kWalk ? k5_tile_stride(N) : cn_slots(nz, lc);
  C *za = reinterpret_cast<C *>(smem_raw);
  C *zb = za + nz * SB;
  C *tile = zb + nz * SB;
  const R s = scale_of<R>(a.state);
  const R inv_ntot = pick<R>(a.inv_ntot, a.inv_ntot_f, a.inv_ntot_l);
  const size_t line0 = (size_t)i * a.ny + j0;
  C *psi = reinterpret_cast<C *>(a.psi) + line0 * nz;
  const C *res = nullptr;

  // the CN-z scan factors, staged after the per-CTA potential tables (dt V_z per point of a
  // line, dt V_y per line; dt V_x of this CTA's x index is a register).  For the compile-time
  // lengths (nz a multiple of 4: every piece 16-byte aligned) they are cp.async copies in the
  // psi tile's group, so their latency hides behind the spectrum load and the transform.
  R *tz = reinterpret_cast<R *>(tile + BZ * LS);
  R *ty = tz + nz;
  Coef *scan_s = reinterpret_cast<Coef *>(ty + BZ);
  constexpr bool kAsyncTabs = N > 0 && !Fp64Class<R>::value;   // (FP64-class: pipe bound, unchanged)
  static_assert(N % 4 == 0, "16-byte aligned pieces");
  const bool phase = zmode == kZStep || zmode == kZPhaseOnly;
  R dtvx = R(0);
  if (phase) dtvx = reinterpret_cast<const R *>(a.dtv[0])[i];
  // the z solve's tables: K5's own at CHZ points per lane where that is not the sweeps' chunk
  const Coef *ztab_g = reinterpret_cast<const Coef *>(
      LZ == 8 ? a.cn8_tab[2] : (kWalk && a.cnz_tab ? a.cnz_tab : a.cn[2].tab));
  const int zmp = kWalk ? LZ * CHZ : (kWarp << lc);
  if (zmode == kZStep || zmode == kZCnOnly) {
    const Coef *gscan = ztab_g + 4 * zmp;
    if constexpr (kAsyncTabs) {
      constexpr int chunks = (LZ == 8 ? 6 : 10) * LZ * (int)sizeof(Coef) / 16;   // the scan factors
      for (int q = threadIdx.x; q < chunks; q += blockDim.x)
        cp_async(reinterpret_cast<uint4 *>(scan_s) + q, reinterpret_cast<const uint4 *>(gscan) + q);
    } else {
      for (int q = threadIdx.x; q < 10 * kWarp; q += blockDim.x) scan_s[q] = gscan[q];
    }
  }
  if (kAsyncTabs && phase) {
    const R *dtv_y = reinterpret_cast<const R *>(a.dtv[1]) + j0;
    const R *dtv_z = reinterpret_cast<const R *>(a.dtv[2]);
    for (int q = threadIdx.x; q < nz * (int)sizeof(R) / 16; q += blockDim.x)
      cp_async(reinterpret_cast<uint4 *>(tz) + q, reinterpret_cast<const uint4 *>(dtv_z) + q);
    if (threadIdx.x < nl) cp_async(ty + threadIdx.x, dtv_y + threadIdx.x);
  }

  // psi tile: asynchronous copies, overlapped with the spectrum load and the C2R transform.
  // Compile-time lengths: thread (line b, offset k0 < W) copies the points k0 + W j of its
  // line (W = threads / lines: 16 consecutive points of a line per half-warp, coalesced).
  static_assert(N % W == 0 && Tiles<R>::kZThreads % BZ == 0, "the walk covers whole lines");
  // issued after the first batch of spectrum loads: the transform needs those first, so they
  // go out ahead of the tile's copies
  bool psi_issued = false;
  auto issue_psi = [&]() {
    if (psi_issued) return;
    psi_issued = true;
    if (zmode != kZPhi) {
      if constexpr (kWalk) {
        const int b = threadIdx.x / W, k0 = threadIdx.x % W;
        if (b < nl) {
          C *dst = tile + b * LS;
#pragma unroll
          for (int sub = 0; sub < SUBS; ++sub) {
            const int o = k0 + W * sub;
            const SlotWalkP<PW, CHZ> w(o);
            const C *src = psi + (size_t)b * nz + o;
#pragma unroll 8
            for (int j = 0; j < N / PW; ++j) cp_async(dst + w(j, o), src + PW * j);
          }
        }
      } else {
        LinePos pos(threadIdx.x, nz, blockDim.x);
        for (int e = threadIdx.x; e < nl * nz; e += blockDim.x, pos.next())
          cp_async(tile + pos.b * LS + cn_slot(pos.k, lc), psi + e);
      }
    }
    cp_async_commit();
  };

  if (zmode == kZCnOnly) issue_psi();
  if (zmode != kZCnOnly) {
    const C *spec = reinterpret_cast<const C *>(a.spec) + line0;
    const size_t plane = (size_t)a.nx * a.ny;
    const int half = nz / 2;
    const int p = threadIdx.x % PZ;
    const int mstep = blockDim.x / PZ;
    if constexpr (kWalk) {
      // the unpacking and the C2R's first stage (radix 8, untwiddled) in one pass: its
      // butterfly j reads z[j + r J] (r < 8, J = N / 8), z[q] = x1 + i x2 of half-spectrum
      // row q for q <= N / 2 (D) and the mirror of row N - q beyond (M); butterflies u and
      // J - u read the same rows u + r J and (r + 1) J - u (r < 4), so one thread takes both
      // (u = 0 and J / 2 alone; rows 0 and N / 2 with their imaginary parts dropped, where D and
      // M agree).  The outputs go to zb at 8 j + s, as the stage writes them.
      constexpr int J = N / 8;
      static_assert(ct_radix(N, 0) == 8, "the first stage is radix 8");
      auto D = [](float4 q) { return C{q.x - q.w, q.y + q.z}; };
      auto M = [](float4 q) { return C{q.x + q.w, q.z - q.y}; };
      if (p < np) {
        for (int u = threadIdx.x / PZ; u <= J / 2; u += mstep) {
          float4 ra[4], rb[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            ra[r] = *reinterpret_cast<const float4 *>(spec + (u + r * J) * plane + 2 * p);
            rb[r] = *reinterpret_cast<const float4 *>(spec + ((r + 1) * J - u) * plane + 2 * p);
          }
          issue_psi();
          if (u == 0) {   // rows 0 and N / 2: the kz = 0 and Nyquist bins are real
            ra[0].y = ra[0].w = 0.0f;
            rb[3].y = rb[3].w = 0.0f;
          }
          C v[8];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            v[r] = D(ra[r]);
            v[r + 4] = M(rb[3 - r]);
          }
          butterfly<R, +1, 8>(v);
#pragma unroll
          for (int q = 0; q < 8; ++q) zb[(8 * u + q) * SB + p] = v[q];
          if (u > 0 && u < J / 2) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              v[r] = D(rb[r]);
              v[r + 4] = M(ra[3 - r]);
            }
            butterfly<R, +1, 8>(v);
#pragma unroll
            for (int q = 0; q < 8; ++q) zb[(8 * (J - u) + q) * SB + p] = v[q];
          }
        }
      }
    } else if (p < np) {
      for (int m0 = threadIdx.x / PZ; m0 < a.nzh; m0 += kUnroll * mstep) {
        C x1[kUnroll], x2[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int m = m0 + u * mstep;
          if (m < a.nzh) {
            if constexpr (std::is_same<R, float>::value) {
              // the pair's two values are adjacent and 16-byte aligned (ny even): one load
              const float4 q = *reinterpret_cast<const float4 *>(spec + m * plane + 2 * p);
              x1[u] = {q.x, q.y};
              x2[u] = {q.z, q.w};
            } else {
              x1[u] = spec[m * plane + 2 * p];
              x2[u] = spec[m * plane + 2 * p + 1];
            }
          }
        }
        issue_psi();
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int m = m0 + u * mstep;
          if (m < a.nzh) {
            if (m == 0 || m == half) {
              x1[u].im = R(0);
              x2[u].im = R(0);
            }
            za[m * SB + p] = {x1[u].re - x2[u].im, x1[u].im + x2[u].re};
            if (m > 0 && m < half) za[(nz - m) * SB + p] = {x1[u].re + x2[u].im, x2[u].re - x1[u].im};
          }
        }
      }
    }
    issue_psi();   // (threads without spectrum rows)
    if constexpr (kWalk) {
      // the rows of tile L + ahead (L the linear CTA index, ahead the CTAs resident at once):
      // that CTA starts about when this one ends and finds its spectrum and psi rows in L2
      // (grouped launches: across the members, each from its own buffers)
      AheadTile t;
      if (ahead_tile(a, ga, Tiles<R>::kZMinBlocks * a.nsm, t)) {
        const int j2 = t.bx2 * BZ;
        const int nl2 = min(BZ, a.ny - j2);   // even: 16-byte multiples
        const size_t l2 = (size_t)t.i2 * a.ny + j2;
        const C *sp2 = reinterpret_cast<const C *>(t.b->spec) + l2;
        for (int m = threadIdx.x; m < a.nzh; m += blockDim.x) prefetch_l2(sp2 + m * plane, nl2 * (unsigned)sizeof(C));
        if (threadIdx.x == blockDim.x - 1)
          prefetch_l2(reinterpret_cast<const C *>(t.b->psi) + l2 * nz, nl2 * nz * (unsigned)sizeof(C));
      }
    }
    __syncthreads();
    if constexpr (kWalk)   // (the first stage done: from zb, at stage 1)
      res = fft_lines_ct<R, +1, N, PZ, SB, Tiles<R>::kZThreads, 1>(zb, za, np, reinterpret_cast<const C *>(a.tw[2]));
    else
      res = fft_lines_n<R, +1, N, PZ, SB, Tiles<R>::kZThreads>(za, zb, a.plan[2], np,
                                                               reinterpret_cast<const C *>(a.tw[2]));
  }

  // the CN-z factor tables (alpha, beta, H, G; 4 * 32 * chunk values), staged into the
  // transform buffer that does not hold the result: they arrive during the phase loop, and
  // the solve reads them from shared memory.  They take 128 chunk sizeof(Coef) bytes, the
  // buffer nz PZ sizeof(C): with chunk the least power of two >= max(2, (nz - 2)/32) they fit
  // for the compile-time lengths (128 to 512); the runtime-length instance reads them from
  // global memory.
  const Coef *ztab = reinterpret_cast<const Coef *>(a.cn[2].tab);
  if constexpr (N > 0) {
    static_assert(N >= 64, "the staged tables fit the spare transform buffer");
    if (zmode == kZStep || zmode == kZCnOnly) {
      C *spare = (zmode == kZCnOnly || res != za) ? za : zb;
      const int bytes = 4 * zmp * (int)sizeof(Coef);
      const uint4 *src = reinterpret_cast<const uint4 *>(ztab_g);
      uint4 *dst = reinterpret_cast<uint4 *>(spare);
      for (int q = threadIdx.x; q < bytes / 16; q += blockDim.x) cp_async(dst + q, src + q);
      ztab = reinterpret_cast<const Coef *>(spare);
    }
  }
  cp_async_commit();

  if (zmode == kZPhi) {
    // Phi in the kernel precision; double for double-float
    using O = typename std::conditional<std::is_same<R, df>::value, double, R>::type;
    O *out = reinterpret_cast<O *>(a.out) + line0 * nz;
    LinePos pos(threadIdx.x, nz, blockDim.x);
    for (int e = threadIdx.x; e < nl * nz; e += blockDim.x, pos.next()) {
      const C z = res[pos.k * SB + (pos.b >> 1)];
      out[e] = O(((pos.b & 1) ? z.im : z.re) * inv_ntot);
    }
    return;
  }
  cp_async_wait_group<1>();   // the psi tile (the tables may still be in flight)
  __syncthreads();

  if (zmode == kZObs) {
    // the sums are taken over the stored values; the pending scale enters in FP64 at the end
    // (s^2 for the quadratic sums, s^4 for the contact term; Phi already carries s^2 through
    // K1's density), so FP32 data are not rounded again by the scaling
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const R sr = R(1);
    const double x = coordinate(i, a.nx, a.hx);
    const double wxi = quad_weight(i, a.nx, a.simpson);
    const R ihx2 = R(1.0 / (a.hx * a.hx)), ihy2 = R(1.0 / (a.hy * a.hy)), ihz2 = R(1.0 / (a.hz * a.hz));
    const C *gpsi = reinterpret_cast<const C *>(a.psi);
    const size_t sx = (size_t)a.ny * nz;
    if constexpr (std::is_same<R, float>::value) {
      // FP32 data: each per-point term in FP32 (the state's precision); the weights exact small
      // integers (3 x the Simpson weights per axis) and the squared coordinates exact integers
      // (the signed index squared), every product by them exact (FMA exact product) and every
      // sum in double-float per thread, as the x sweep's norm; h^2, (1/3)^3 and the physical
      // factors applied in FP64 to the thread's totals.  The trap term needs no sum of its own:
      // sum w V n = vx sum w x^2 n + vy sum w y^2 n + vz sum w z^2 n.  (FP64 work per point
      // would bound this pass on GB300's FP64 pipe.)
      DFAcc t[7];   // n, the kinetic term, n^2, Phi n, i'^2 n, j'^2 n, k'^2 n
      const int wx = quad_weight3(i, a.nx, a.simpson), ii = i - a.nx / 2;
      LinePos pos(threadIdx.x, nz, blockDim.x);
      for (int e = threadIdx.x; e < nl * nz; e += blockDim.x, pos.next()) {
        const int b = pos.b, n = pos.k;
        const int j = j0 + b;
        const int W = wx * quad_weight3(j, a.ny, a.simpson) * quad_weight3(n, nz, a.simpson);
        if (W == 0) continue;
        const C *row = tile + b * LS;
        const C c = row[cn_slot(n, lc)];
        const C zm = n > 0 ? row[cn_slot(n - 1, lc)] : czero<R>();
        const C zp = n < nz - 1 ? row[cn_slot(n + 1, lc)] : czero<R>();
        const size_t q = (line0 + b) * nz + n;
        const C ym = j > 0 ? gpsi[q - nz] : czero<R>();
        const C yp = j < a.ny - 1 ? gpsi[q + nz] : czero<R>();
        const C xm = i > 0 ? gpsi[q - sx] : czero<R>();
        const C xp = i < a.nx - 1 ? gpsi[q + sx] : czero<R>();
        float kin;   // c . Lap c (the kinetic energy is -1/2 its sum), or |grad c|^2 (+1/2)
        if (!a.kinetic5) {
          const float lre = (xm.re - 2.0f * c.re + xp.re) * ihx2 + (ym.re - 2.0f * c.re + yp.re) * ihy2 +
                            (zm.re - 2.0f * c.re + zp.re) * ihz2;
          const float lim = (xm.im - 2.0f * c.im + xp.im) * ihx2 + (ym.im - 2.0f * c.im + yp.im) * ihy2 +
                            (zm.im - 2.0f * c.im + zp.im) * ihz2;
          kin = fmaf(c.re, lre, c.im * lim);
        } else {
          // 4th-order first derivatives (f(-2) - 8 f(-1) + 8 f(1) - f(2)) / (12 h), zero outside
          const C zm2 = n > 1 ? row[cn_slot(n - 2, lc)] : czero<R>();
          const C zp2 = n < nz - 2 ? row[cn_slot(n + 2, lc)] : czero<R>();
          const C ym2 = j > 1 ? gpsi[q - 2 * nz] : czero<R>();
          const C yp2 = j < a.ny - 2 ? gpsi[q + 2 * nz] : czero<R>();
          const C xm2 = i > 1 ? gpsi[q - 2 * sx] : czero<R>();
          const C xp2 = i < a.nx - 2 ? gpsi[q + 2 * sx] : czero<R>();
          auto d1 = [](C m2, C m1, C p1, C p2, float f) {
            const float re = (m2.re - 8.0f * m1.re + 8.0f * p1.re - p2.re) * f;
            const float im = (m2.im - 8.0f * m1.im + 8.0f * p1.im - p2.im) * f;
            return fmaf(re, re, im * im);
          };
          kin = d1(xm2, xm, xp, xp2, float(1.0 / (12.0 * a.hx))) + d1(ym2, ym, yp, yp2, float(1.0 / (12.0 * a.hy))) +
                d1(zm2, zm, zp, zp2, float(1.0 / (12.0 * a.hz)));
        }
        const C z = res[n * SB + (b >> 1)];
        const float phi = ((b & 1) ? z.im : z.re) * inv_ntot;
        const float d = fmaf(c.re, c.re, c.im * c.im);
        const int jj = j - a.ny / 2, kk = n - nz / 2;
        const float wf = (float)W;
        t[0].add_prod(wf, d);
        t[1].add_prod(wf, kin);
        t[2].add_prod(wf, d * d);
        t[3].add_prod(wf, phi * d);
        t[4].add_prod((float)(ii * ii * W), d);   // <= 256^2 x 64 = 2^22: exact
        t[5].add_prod((float)(jj * jj * W), d);
        t[6].add_prod((float)(kk * kk * W), d);
      }
      const double ws = a.simpson ? 1.0 / 27.0 : 1.0;
      const double X = t[4].value() * ws * a.hx * a.hx, Y = t[5].value() * ws * a.hy * a.hy,
                   Z = t[6].value() * ws * a.hz * a.hz;
      v[0] = t[0].value() * ws;
      v[1] = (a.kinetic5 ? 0.5 : -0.5) * t[1].value() * ws;
      v[2] = a.vx * X + a.vy * Y + a.vz * Z;
      v[3] = a.g * t[2].value() * ws;
      v[4] = a.gdd * t[3].value() * ws;
      v[5] = X;
      v[6] = Y;
      v[7] = Z;
    } else {
      LinePos pos(threadIdx.x, nz, blockDim.x);
      for (int e = threadIdx.x; e < nl * nz; e += blockDim.x, pos.next()) {
        const int b = pos.b, n = pos.k;
        const int j = j0 + b;
        const C *row = tile + b * LS;
        const C c = scale(row[cn_slot(n, lc)], sr);
        const C zm = n > 0 ? scale(row[cn_slot(n - 1, lc)], sr) : czero<R>();
        const C zp = n < nz - 1 ? scale(row[cn_slot(n + 1, lc)], sr) : czero<R>();
        const size_t q = (line0 + b) * nz + n;
        const C ym = j > 0 ? scale(gpsi[q - nz], sr) : czero<R>();
        const C yp = j < a.ny - 1 ? scale(gpsi[q + nz], sr) : czero<R>();
        const C xm = i > 0 ? scale(gpsi[q - sx], sr) : czero<R>();
        const C xp = i < a.nx - 1 ? scale(gpsi[q + sx], sr) : czero<R>();
        double ekin;
        if (!a.kinetic5) {
          const C lap = {(xm.re - R(2) * c.re + xp.re) * ihx2 + (ym.re - R(2) * c.re + yp.re) * ihy2 +
                             (zm.re - R(2) * c.re + zp.re) * ihz2,
                         (xm.im - R(2) * c.im + xp.im) * ihx2 + (ym.im - R(2) * c.im + yp.im) * ihy2 +
                             (zm.im - R(2) * c.im + zp.im) * ihz2};
          ekin = -0.5 * ((double)c.re * (double)lap.re + (double)c.im * (double)lap.im);
        } else {
          // 4th-order first derivatives (f(-2) - 8 f(-1) + 8 f(1) - f(2)) / (12 h), zero outside
          const C zm2 = n > 1 ? scale(row[cn_slot(n - 2, lc)], sr) : czero<R>();
          const C zp2 = n < nz - 2 ? scale(row[cn_slot(n + 2, lc)], sr) : czero<R>();
          const C ym2 = j > 1 ? scale(gpsi[q - 2 * nz], sr) : czero<R>();
          const C yp2 = j < a.ny - 2 ? scale(gpsi[q + 2 * nz], sr) : czero<R>();
          const C xm2 = i > 1 ? scale(gpsi[q - 2 * sx], sr) : czero<R>();
          const C xp2 = i < a.nx - 2 ? scale(gpsi[q + 2 * sx], sr) : czero<R>();
          auto d1 = [](C m2, C m1, C p1, C p2, double h) {
            const double f = 1.0 / (12.0 * h);
            const double re = ((double)m2.re - 8.0 * (double)m1.re + 8.0 * (double)p1.re - (double)p2.re) * f;
            const double im = ((double)m2.im - 8.0 * (double)m1.im + 8.0 * (double)p1.im - (double)p2.im) * f;
            return re * re + im * im;
          };
          ekin = 0.5 * (d1(xm2, xm, xp, xp2, a.hx) + d1(ym2, ym, yp, yp2, a.hy) + d1(zm2, zm, zp, zp2, a.hz));
        }
        const C z = res[n * SB + (b >> 1)];
        const double phi = (double)(((b & 1) ? z.im : z.re) * inv_ntot);
        const double dens = (double)c.re * (double)c.re + (double)c.im * (double)c.im;
        const double y = coordinate(j, a.ny, a.hy), zc = coordinate(n, nz, a.hz);
        const double w = wxi * quad_weight(j, a.ny, a.simpson) * quad_weight(n, nz, a.simpson);
        v[0] += w * dens;
        v[1] += w * ekin;
        v[2] += w * (a.vx * x * x + a.vy * y * y + a.vz * zc * zc) * dens;
        v[3] += w * a.g * dens * dens;
        v[4] += w * a.gdd * phi * dens;
        v[5] += w * x * x * dens;
        v[6] += w * y * y * dens;
        v[7] += w * zc * zc * dens;
      }
    }
    if (reduce_across_blocks<8>(v, a.partials, &a.state->ticket) && threadIdx.x == 0) {
      const double dv = a.hx * a.hy * a.hz;
      DevState *st = a.state;
      const double s2 = st->s * st->s;
      for (int q = 0; q < 8; ++q) v[q] *= q == 3 ? s2 * s2 : s2;
      for (int q = 0; q < 8; ++q) st->sums[q] = v[q];
      const double norm = dv * v[0];
      const double ekin = dv * v[1], etrap = dv * v[2], econ = 0.5 * dv * v[3], edd = 0.5 * dv * v[4];
      st->obs[0] = norm;
      st->obs[1] = dv * (v[1] + v[2] + v[3] + v[4]) / norm;
      st->obs[2] = ekin + etrap + econ + edd;
      st->obs[3] = sqrt(v[5] / v[0]);
      st->obs[4] = sqrt(v[6] / v[0]);
      st->obs[5] = sqrt(v[7] / v[0]);
      st->obs[6] = ekin;
      st->obs[7] = etrap;
      st->obs[8] = econ;
      st->obs[9] = edd;
      bool finite = true;
      for (int q = 0; q < 10; ++q) finite = finite && isfinite(st->obs[q]);
      if (!finite) st->flags |= kFlagNonFinite;
    }
    return;
  }

  if (zmode == kZStep || zmode == kZPhaseOnly) {
    // theta = dt (V + g n + gdd Phi): dt V_z per n and dt (V_x + V_y) per line come from
    // small per-CTA tables; the 1/(nx ny nz) of the inverse transform is folded into gdd.
    if constexpr (!kAsyncTabs) {
      const R *dtv_y = reinterpret_cast<const R *>(a.dtv[1]);
      const R *dtv_z = reinterpret_cast<const R *>(a.dtv[2]);
      for (int n = threadIdx.x; n < nz; n += blockDim.x) tz[n] = dtv_z[n];
      if (threadIdx.x < nl) ty[threadIdx.x] = dtvx + dtv_y[j0 + threadIdx.x];   // dt (V_x + V_y) per line
      __syncthreads();
    }
    const R sr = R(s);
    const bool scaled = s != R(1);
    const R dtg = pick<R>(a.dtg, a.dtg_f, a.dtg_l), dtgdd = pick<R>(a.dtgdd_n, a.dtgdd_n_f, a.dtgdd_n_l);
    // lines fastest: the padded tile rows (odd stride LS) and the pair-interleaved Phi are
    // read without bank conflicts
    auto phase_at = [&](int n, int b, int q) {
      C v = tile[q];
      if (scaled) v = scale(v, sr);
      const C z = res[n * SB + (b >> 1)];
      const R phi = (b & 1) ? z.im : z.re;
      const R dens = v.re * v.re + v.im * v.im;
      // dt (V_x + V_y): the async path copied dt V_y and adds dt V_x here (one FP32 add); the
      // other path summed them per line
      const R vxy = kAsyncTabs ? ty[b] + dtvx : ty[b];
      const R theta = fma(dtg, dens, fma(dtgdd, phi, vxy + tz[n]));
      if (a.imag) {
        tile[q] = scale(v, exp_r(-theta));
      } else {
        R sn, cs;
        sin_cos(theta, &sn, &cs);
        tile[q] = {v.re * cs + v.im * sn, v.im * cs - v.re * sn};
      }
    };
    if constexpr (kWalk) {
      // thread (line b, offset n0 < W): the points n0 + W sub + PW i of line b, lines fastest;
      // the line's dt (V_x + V_y) read once, its Phi (.re or .im of pair b/2) through its own
      // float pointer
      const int b = threadIdx.x % BZ, n0 = threadIdx.x / BZ;
      if (b < nl) {
        const R vxy = ty[b] + dtvx;
        const R *phib = reinterpret_cast<const R *>(res + (b >> 1)) + (b & 1);
        C *row = tile + b * LS;
#pragma unroll
        for (int sub = 0; sub < SUBS; ++sub) {
          const int o = n0 + W * sub;
          const SlotWalkP<PW, CHZ> w(o);
#pragma unroll 4
          for (int i = 0; i < N / PW; ++i) {
            const int n = o + PW * i;
            C v = row[w(i, o)];
            if (scaled) v = scale(v, sr);
            const R dens = v.re * v.re + v.im * v.im;
            const R theta = fma(dtg, dens, fma(dtgdd, phib[2 * SB * n], vxy + tz[n]));
            if (a.imag) {
              row[w(i, o)] = scale(v, exp_r(-theta));
            } else {
              R sn, cs;
              sin_cos(theta, &sn, &cs);
              row[w(i, o)] = {v.re * cs + v.im * sn, v.im * cs - v.re * sn};
            }
          }
        }
      }
    } else {
      LinePos pos(threadIdx.x, nl, blockDim.x);   // pos.b = z index n, pos.k = line b
      for (int e = threadIdx.x; e < nl * nz; e += blockDim.x, pos.next())
        phase_at(pos.b, pos.k, pos.k * LS + cn_slot(pos.b, lc));
    }
    __syncthreads();
  }

  if (zmode == kZStep || zmode == kZCnOnly) {
    if constexpr (kWalk) {
      // the padded solve: the far wall (grid N - 1, which the phase loop has written) and the
      // points beyond it, up to the padded length 32 CHZ, hold zero; after the phase loop's
      // barrier, before the solve's
      constexpr int kPad = LZ * CHZ + 2 - N;
      static_assert(kPad >= 1 && kPad * BZ <= Tiles<R>::kZThreads, "a thread per padded slot");
      if (threadIdx.x < BZ * kPad) {
        const int b = threadIdx.x / kPad, g = N - 1 + threadIdx.x % kPad;
        tile[b * LS + g + (g - 1) / CHZ] = czero<R>();
      }
    }
    cp_async_wait_group<0>();
    __syncthreads();
    const Coef c = CnCoef<R, Coef>::make(pick<R>(a.cn_r[2], a.cn_rf[2], a.cn_rl[2]));
    if constexpr (LZ == 8) {
      // four lines per warp, two per half-warp 8 apart (at the odd line stride they fall on
      // distinct banks): 32 lines on the 8 warps (w + 8 g), or 16 on warps 0-3 (w, w + 8, w + 4,
      // w + 12).  Lines past nl are solved too (all lanes take part in the scans), not stored.
      static_assert((BZ == 32 || BZ == 16) && Tiles<R>::kZThreads == 256, "32 or 16 lines on 256 threads");
      const int w = threadIdx.x / kWarp, g = (threadIdx.x & (kWarp - 1)) >> 3;
      if constexpr (BZ == 32)
        cn_line<R, Coef, CHZ, true, true, 8>(tile + (w + 8 * g) * LS, 1, 8 * CHZ, lc, ztab, scan_s, c);
      else if (w < 4)
        cn_line<R, Coef, CHZ, true, true, 8>(tile + (w + 8 * (g & 1) + 4 * (g >> 1)) * LS, 1, 8 * CHZ, lc, ztab, scan_s, c);
    } else if constexpr (kWalk && BZ == 2 * (Tiles<R>::kZThreads / kWarp) && CHZ <= 12) {
      // two lines per warp in lockstep (w and w + BZ / 2): each table value read once for
      // both (chunks up to 12 points: at 16 the two lines' values no longer fit the registers).
      // Lines past nl are solved too (their padding is zero), not stored.
      const int w = threadIdx.x / kWarp;
      cn_line2<R, Coef, CHZ>(tile + w * LS, tile + (w + BZ / 2) * LS, 1, ztab, scan_s, c);
    } else {
      for (int b = threadIdx.x / kWarp; b < nl; b += blockDim.x / kWarp) {
        if constexpr (kWalk) cn_line<R, Coef, CHZ, true, true>(tile + b * LS, 1, kWarp * CHZ, lc, ztab, scan_s, c);
        else cn_line_any<R, Coef, (N > 0)>(tile + b * LS, 1, a.cn[2].m, lc, ztab, scan_s, c);
      }
    }
    __syncthreads();
  }

  if constexpr (kWalk) {
    const int b = threadIdx.x / W, k0 = threadIdx.x % W;
    if (b < nl) {
      const C *src = tile + b * LS;
#pragma unroll
      for (int sub = 0; sub < SUBS; ++sub) {
        const int o = k0 + W * sub;
        const SlotWalkP<PW, CHZ> w(o);
        C *dst = psi + (size_t)b * nz + o;
#pragma unroll 8
        for (int j = 0; j < N / PW; ++j) dst[PW * j] = src[w(j, o)];
      }
    }
  } else {
    LinePos pos(threadIdx.x, nz, blockDim.x);
#pragma unroll 4
    for (int e = threadIdx.x; e < nl * nz; e += blockDim.x, pos.next()) psi[e] = tile[pos.b * LS + cn_slot(pos.k, lc)];
  }
}
// one condensate (G = false, its arguments passed by value), or condensate blockIdx.z of
// a group of same-shaped condensates (G = true, the arguments from the device array ga)
template <typename R, typename Coef, int ZM, int N, bool G = false>
__global__ void __launch_bounds__(Tiles<R>::kZThreads,
                                  ZM == kZObs ? 1 : (ZM == kZPhaseOnly && std::is_same<R, double>::value ? 3 : Tiles<R>::kZMinBlocks)) k5_zline(KArgs a, const KArgs *ga) {
  if constexpr (G) k5_zline_body<R, Coef, ZM, N>(ga[blockIdx.z], ga);
  else k5_zline_body<R, Coef, ZM, N>(a, nullptr);
}

// ---------------------------------------------------------------------------------------
// K6 / K7: Crank-Nicolson along y (AXIS = 1, lines psi[i][:][k]) or x (AXIS = 0, lines
// psi[:][j][k]) for kCnCols consecutive k per CTA (one warp per line).  K7 (x) also sums
// n, x^2 n, y^2 n, z^2 n (FP64 totals) and, in the last block, sets the norm and the pending
// renormalisation factor s = 1/sqrt(norm) (imaginary time) or 1 (real time).  The x^2 n
// sum is not taken (nothing reads it: the observables take their own FP64 sums).  FP64
// data: FP64 sums per thread.  FP32 data (k_cn): the terms n = |psi|^2 in FP32 (the state's
// own precision), and from there every product exact and every sum in double-float, point
// by point (error about 2^-44 of the total): the weights are exact small integers (3 x the
// Simpson weights per axis, the squared signed index instead of the squared coordinate),
// the products by them exact (FMA exact product), the sums Knuth's TwoSum; the factors
// h_d^2 and (1/3)^3 (Simpson) are applied in FP64 at the end.
// ---------------------------------------------------------------------------------------
// Running sums of the reduction of the FP64-class per-line sweeps: FP64 for FP64 data,
// double-float pairs for double-float data.
template <typename R>
struct SumAcc;
template <>
struct SumAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double t) { v += t; }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct SumAcc<df> {
  df v{0.0f, 0.0f};
  __device__ __forceinline__ void add(df t) { v = v + t; }
  __device__ __forceinline__ double value() const { return (double)v; }
};

// Block sums of n, x^2 n, y^2 n, z^2 n -> across blocks; the last block sets the norm and
// the pending scale s of the state.  renorm: kRenormNone (real time: s = 1), kRenormUnit
// (imaginary time: s = 1/sqrt(norm)), kRenormRestore (real time, FP32-mixed: s restores the
// norm the state had when the real-time run began, the true norm of the state the first
// real-time step started from, or its own output's norm if that is unknown).  The exact
// real-time step conserves the norm; the FP32-rounded Crank-Nicolson factor tables make
// each sweep non-unitary by about 1e-7 (the same rounding at every point of a line, so it
// adds up instead of averaging out), and this undoes that drift from the FP64-class sum.
__device__ __forceinline__ void finish_sweep_sums(const KArgs &a, double (&v)[4], int renorm) {
  if (reduce_across_blocks<4>(v, a.partials, &a.state->ticket) && threadIdx.x == 0) {
    DevState *st = a.state;
    const double norm = a.hx * a.hy * a.hz * v[0];
    for (int q = 0; q < 4; ++q) st->sums[q] = v[q];
    st->norm = norm;
    // a zero state is a state (real time keeps it zero); only the renormalisation of
    // imaginary time needs a positive norm
    const bool ok = isfinite(norm) && (norm > 0.0 || renorm != kRenormUnit);
    if (!ok) st->flags |= kFlagNonFinite;
    double s = 1.0;
    if (renorm == kRenormUnit) {
      if (ok) s = 1.0 / sqrt(norm);
      st->norm_ref = 0.0;   // a later real-time run takes its own reference
    } else if (renorm == kRenormRestore && ok && norm > 0.0) {
      if (!(st->norm_ref > 0.0)) st->norm_ref = st->norm_in > 0.0 ? st->norm_in : norm;
      s = sqrt(st->norm_ref / norm);
    }
    set_scale(st, s);
    st->norm_in = norm * s * s;
    st->steps += 1ull;
  }
}

// Persistent, double-buffered: each CTA walks the tiles (fixed index, k-tile)
// blockIdx.x, blockIdx.x + gridDim.x, ...; the cp.async copies of the next tile are in
// flight while the current tile is solved and stored.
// B columns (z) per tile, NT threads (B divides NT; one or two lines per warp).
template <typename R, typename Coef, int AXIS, int B = Tiles<R>::kCnCols, int NT = Tiles<R>::kCnThreads,
          bool FULL = false>
__device__ __forceinline__ void k_cn_body(const KArgs &a, int reduce, int renorm) {
  static_assert(std::is_same<R, float>::value, "the chunked sweeps serve FP32 data");
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int SB = B + 1;
  const int N = AXIS == 0 ? a.nx : a.ny;
  const int nfixed = AXIS == 0 ? a.ny : a.nx;
  const int nkt = (a.nz + B - 1) / B;
  const int ntiles = nfixed * nkt;
  const int lc = a.cn[AXIS].lchunk;
  // FULL: the lines padded to 32 chunks of unknowns (grid indices up to m_pad + 1)
  const int m_pad = kWarp << lc;
  const int slots = FULL ? cn_slots(m_pad + 2, lc) : cn_slots(N, lc);
  C *cur = reinterpret_cast<C *>(smem_raw);
  C *nxt = cur + slots * SB;
  Coef *stab = reinterpret_cast<Coef *>(nxt + slots * SB);     // factor tables, staged once
  const int ntab = 4 * (kWarp << lc) + 10 * kWarp;
  float *wxtab = reinterpret_cast<float *>(stab + ntab);        // W_x(i) = 3 x the weight (or 1)
  const size_t stride = AXIS == 1 ? (size_t)a.nz : (size_t)a.ny * a.nz;
  C *gpsi = reinterpret_cast<C *>(a.psi);
  const int b = threadIdx.x % B;   // B divides the block size: the column is fixed per thread
  const int n0 = threadIdx.x / B;
  constexpr int nstep = NT / B;   // the launch has NT threads
  const bool do_reduce = AXIS == 0 && reduce;

  auto tile_origin = [&](int tile, int &fixed, int &k0) -> size_t {
    fixed = tile / nkt;
    k0 = (tile - fixed * nkt) * B;
    return AXIS == 1 ? (size_t)fixed * a.ny * a.nz + k0 : (size_t)fixed * a.nz + k0;
  };
  auto issue = [&](int tile, C *buf) {
    int fixed, k0;
    const size_t base = tile_origin(tile, fixed, k0);
    if (b < min(B, a.nz - k0)) {
      const C *src = gpsi + base + b + (size_t)n0 * stride;
      const SlotWalk<NT / B> w(n0, lc);
      // (FULL: not the far wall, whose slot stays zero, as the padding's do)
      const int nload = FULL ? N - 1 : N;
#pragma unroll 4
      for (int j = 0; n0 + (NT / B) * j < nload; ++j, src += (NT / B) * stride) cp_async(buf + w(j, n0) * SB + b, src);
    }
    cp_async_commit();
  };

  if (do_reduce)
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
      wxtab[n] = (float)quad_weight3(n, a.nx, a.simpson);
    }
  const Coef c = CnCoef<R, Coef>::make(pick<R>(a.cn_r[AXIS], a.cn_rf[AXIS], a.cn_rl[AXIS]));
  {
    const Coef *gtab = reinterpret_cast<const Coef *>(a.cn[AXIS].tab);
    for (int q = threadIdx.x; q < ntab; q += blockDim.x) stab[q] = gtab[q];
  }
  const Coef *tab = stab;
  DFAcc acc[4];
  if constexpr (FULL) {   // the far wall and the padding: zero in both buffers, once
    for (int q = threadIdx.x; q < (m_pad + 2 - N) * SB; q += blockDim.x) {
      const int g = N - 1 + q / SB, col = q % SB;
      cur[cn_slot(g, lc) * SB + col] = czero<R>();
      nxt[cn_slot(g, lc) * SB + col] = czero<R>();
    }
  }

  int tile = blockIdx.x;
  if (tile < ntiles) issue(tile, cur);
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    if (next < ntiles) {
      issue(next, nxt);
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_group<0>();
    }
    __syncthreads();
    int fixed, k0;
    const size_t base = tile_origin(tile, fixed, k0);
    const int nb = min(B, a.nz - k0);
    if constexpr (FULL && NT == 8 * kWarp && B == 16) {
      // 8 warps, two columns each in lockstep (w, w + 8): each table value read once for both;
      // columns past nb are solved too (their padding is zero) and not stored
      const int w = threadIdx.x / kWarp;
      cn_line2_any<R, Coef>(cur + w, cur + w + 8, SB, lc, tab, tab + 4 * (kWarp << lc), c);
    } else {
      for (int l = threadIdx.x / kWarp; l < nb; l += blockDim.x / kWarp)
        cn_line_any<R, Coef, true, FULL>(cur + l, SB, FULL ? m_pad : a.cn[AXIS].m, lc, tab, tab + 4 * (kWarp << lc), c);
    }
    __syncthreads();
    if (b < nb) {
      DFAcc s0;   // this thread's share of the column: sum W_x n
      C *dst = gpsi + base + b + (size_t)n0 * stride;
      const SlotWalk<NT / B> walk(n0, lc);
#pragma unroll 4
      for (int j = 0, n = n0; n < N; ++j, n += nstep, dst += nstep * stride) {
        const C w = cur[walk(j, n0) * SB + b];
        *dst = w;
        if (do_reduce) {
          const float d = fmaf(w.re, w.re, w.im * w.im);
          s0.add(a.simpson ? wxtab[n] * d : d);   // exact: W_x is 0, 1, 2 or 4 (1 without Simpson)
        }
      }
      if (do_reduce) {
        // W_y W_z is 0 or a power of two up to 16; j'^2 W_y W_z <= 2^20: exact floats
        const int jj = fixed - a.ny / 2, kk = k0 + b - a.nz / 2;
        const int wyz = quad_weight3(fixed, a.ny, a.simpson) * quad_weight3(k0 + b, a.nz, a.simpson);
        acc[0].add_scaled((float)wyz, s0);
        acc[2].add_scaled((float)(jj * jj * wyz), s0);
        acc[3].add_scaled((float)(kk * kk * wyz), s0);
      }
    }
    __syncthreads();   // `cur` is refilled by the prefetch two tiles ahead
    C *t = cur;
    cur = nxt;
    nxt = t;
  }
  if (do_reduce) {
    const double w = a.simpson ? 1.0 / 27.0 : 1.0;   // (1/3)^3 of the integer Simpson weights
    double v[4] = {acc[0].value() * w, 0.0, acc[2].value() * (w * a.hy * a.hy), acc[3].value() * (w * a.hz * a.hz)};
    finish_sweep_sums(a, v, renorm);
  }
}
// one condensate (G = false, its arguments passed by value), or condensate blockIdx.z of
// a group of same-shaped condensates (G = true, the arguments from the device array ga)
template <typename R, typename Coef, int AXIS, int B = Tiles<R>::kCnCols, int NT = Tiles<R>::kCnThreads, bool G = false,
          bool FULL = false>
__global__ void __launch_bounds__(NT, (FULL && NT == 256) ? 1 : 512 / NT) k_cn(KArgs a, const KArgs *ga, int reduce, int renorm) {
  if constexpr (G) k_cn_body<R, Coef, AXIS, B, NT, FULL>(ga[blockIdx.z], reduce, renorm);
  else k_cn_body<R, Coef, AXIS, B, NT, FULL>(a, reduce, renorm);
}

// K6 / K7 for short FP32 lines of n = 8 CH points (CH = short_cn_chunk(n) = 4 .. 16): the
// chunked solve on 8 lanes per line, CH points each (three scan steps instead of five, whose
// cost per point on 32 lanes of 4 points outweighed the solve), four lines per warp, 4 warps
// and 16 columns per tile, up to four CTAs per SM; persistent and double-buffered as k_cn.
// The line is padded to the 8 CH unknowns of grid indices 1 .. n: the far wall n - 1 and the
// slot n beyond it hold zero, and the tables (8-lane layout) decouple them.  Slot of grid
// index g: g + (g - 1) / CH (slot 0 the wall g = 0).  The four lines of warp w are the columns
// 2w, 2w + 8, 2w + 1 and 2w + 9: the two lines of a half-warp fall on distinct banks.
template <typename Coef, int AXIS, int CH>
__device__ __forceinline__ void k_cn_short_body(const KArgs &a, int reduce, int renorm) {
  using R = float;
  using C = cplx<float>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int L = 8, B = 16, NT = 128, SB = B + 1;
  constexpr int N = L * CH;                     // the line length
  constexpr int SLOTS = N + 2 + N / CH;         // grid indices 0 .. N + 1
  constexpr int W = NT / B;                     // rows per pass of the tile loops
  constexpr int P = W / gcd_c(W, CH) * CH;      // lcm(W, CH): the rows' slot walk period
  constexpr int NTAB = 4 * L * CH + 6 * L;      // alpha, beta, H, G, then the scan factors
  static_assert(N % P == 0 && P % W == 0, "whole periods per line");
  const int nkt = (a.nz + B - 1) / B;
  const int ntiles = (AXIS == 0 ? a.ny : a.nx) * nkt;
  C *cur = reinterpret_cast<C *>(smem_raw);
  C *nxt = cur + SLOTS * SB;
  Coef *stab = reinterpret_cast<Coef *>(nxt + SLOTS * SB);
  float *wxtab = reinterpret_cast<float *>(stab + NTAB);   // W_x(i) = 3 x the weight (or 1)
  const size_t stride = AXIS == 1 ? (size_t)a.nz : (size_t)a.ny * a.nz;
  C *gpsi = reinterpret_cast<C *>(a.psi);
  const int b = threadIdx.x % B, n0 = threadIdx.x / B;
  const bool do_reduce = AXIS == 0 && reduce;

  auto tile_origin = [&](int tile, int &fixed, int &k0) -> size_t {
    fixed = tile / nkt;
    k0 = (tile - fixed * nkt) * B;
    return AXIS == 1 ? (size_t)fixed * a.ny * a.nz + k0 : (size_t)fixed * a.nz + k0;
  };
  // rows 0 .. N - 2 (not the far wall, whose slot stays zero)
  auto issue = [&](int tile, C *buf) {
    int fixed, k0;
    const size_t base = tile_origin(tile, fixed, k0);
    if (b < min(B, a.nz - k0)) {
      const C *src = gpsi + base + b;
#pragma unroll
      for (int sub = 0; sub < P / W; ++sub) {
        const int o = n0 + W * sub;
        const SlotWalkP<P, CH> w(o);
#pragma unroll
        for (int j = 0; j < N / P; ++j)
          if (o + P * j < N - 1) cp_async(buf + w(j, o) * SB + b, src + (size_t)(o + P * j) * stride);
      }
    }
    cp_async_commit();
  };

  for (int q = threadIdx.x; q < 3 * SB; q += NT) {   // grid indices N - 1 .. N + 1: zero, once
    const int g = N - 1 + q / SB, col = q % SB;
    cur[(g + (g - 1) / CH) * SB + col] = czero<R>();
    nxt[(g + (g - 1) / CH) * SB + col] = czero<R>();
  }
  {
    const Coef *gtab = reinterpret_cast<const Coef *>(a.cn8_tab[AXIS]);
    for (int q = threadIdx.x; q < NTAB; q += NT) stab[q] = gtab[q];
  }
  if (do_reduce)
    for (int n = threadIdx.x; n < N; n += NT) wxtab[n] = (float)quad_weight3(n, a.nx, a.simpson);
  const Coef c = CnCoef<R, Coef>::make(a.cn_rf[AXIS]);
  const int warp = threadIdx.x / kWarp, grp = (threadIdx.x & (kWarp - 1)) >> 3;
  const int col = 2 * warp + (grp >> 1) + 8 * (grp & 1);
  DFAcc acc[4];

  int tile = blockIdx.x;
  if (tile < ntiles) issue(tile, cur);
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    if (next < ntiles) {
      issue(next, nxt);
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_group<0>();
    }
    __syncthreads();
    int fixed, k0;
    const size_t base = tile_origin(tile, fixed, k0);
    const int nb = min(B, a.nz - k0);
    // every column is solved (all lanes take part in the scans); those past nb are not stored
    cn_line<R, Coef, CH, true, true, L>(cur + col, SB, N, 0, stab, stab + 4 * L * CH, c);
    __syncthreads();
    if (b < nb) {
      DFAcc s0;   // this thread's share of the column: sum W_x n
      C *dst = gpsi + base + b;
#pragma unroll
      for (int sub = 0; sub < P / W; ++sub) {
        const int o = n0 + W * sub;
        const SlotWalkP<P, CH> w(o);
#pragma unroll
        for (int j = 0; j < N / P; ++j) {
          const int n = o + P * j;
          const C v = cur[w(j, o) * SB + b];
          dst[(size_t)n * stride] = v;
          if (do_reduce) {
            const float d = fmaf(v.re, v.re, v.im * v.im);
            s0.add(a.simpson ? wxtab[n] * d : d);   // exact: W_x is 0, 1, 2 or 4 (1 without Simpson)
          }
        }
      }
      if (do_reduce) {
        const int jj = fixed - a.ny / 2, kk = k0 + b - a.nz / 2;
        const int wyz = quad_weight3(fixed, a.ny, a.simpson) * quad_weight3(k0 + b, a.nz, a.simpson);
        acc[0].add_scaled((float)wyz, s0);
        acc[2].add_scaled((float)(jj * jj * wyz), s0);
        acc[3].add_scaled((float)(kk * kk * wyz), s0);
      }
    }
    __syncthreads();   // `cur` is refilled by the prefetch two tiles ahead
    C *t = cur;
    cur = nxt;
    nxt = t;
  }
  if (do_reduce) {
    const double w = a.simpson ? 1.0 / 27.0 : 1.0;   // (1/3)^3 of the integer Simpson weights
    double v[4] = {acc[0].value() * w, 0.0, acc[2].value() * (w * a.hy * a.hy), acc[3].value() * (w * a.hz * a.hz)};
    finish_sweep_sums(a, v, renorm);
  }
}
template <typename Coef, int AXIS, int CH, bool G = false>
__global__ void __launch_bounds__(128, 4) k_cn_short(KArgs a, const KArgs *ga, int reduce, int renorm) {
  if constexpr (G) k_cn_short_body<Coef, AXIS, CH>(ga[blockIdx.z], reduce, renorm);
  else k_cn_short_body<Coef, AXIS, CH>(a, reduce, renorm);
}
// shared memory of k_cn_short at chunk CH: two tile buffers, the tables, the x weights
__host__ __device__ constexpr size_t smem_cn_short(int ch) {
  return 2 * (size_t)(8 * ch + 2 + 8) * 17 * 8 + (size_t)(4 * 8 * ch + 48) * 8 + (size_t)8 * ch * 4;
}

// FP64-class sweeps: two threads per line, the twisted ("burn at both ends") factorization.
// The matrix tridiag(-c, 1 + 2c, -c) reads the same from either end, so its UL factors are
// its LU factors mirrored: the top thread eliminates points 0 .. h-1 downwards
// (y_i = psi_i + alpha_i y_{i-1}), the bottom thread points m-1 .. h+1 upwards
// (z_i = psi_i + alpha_{m-1-i} z_{i+1}), both with table entry s at their s-th step.  They
// meet at the twist point h = m/2:
//   gamma x_h = psi_h + alpha_h y_{h-1} + alpha_{m-1-h} z_{h+1},
//   gamma = e_h + e_{m-1-h} - (1 + 2c)   (e_i = 1/beta_i, the LU pivots; 1/gamma is stored
// after the scan factors), then substitute back away from h: chi_i = beta_i (y_i + c chi_{i+1})
// above, chi_i = beta_{m-1-i} (z_i + c chi_{i-1}) below, psi'_i = 2 chi_i - psi_i.  Twice the
// threads of one thread per line: at 256^3 a sweep is 4096 warps, 6.7 per SM sub-partition
// instead of 3.4, so the last partial round of warps idles a sub-partition for about 1/28 of
// the sweep instead of 1/6.  A warp holds 16 lines: lanes 0-15 their top halves, lanes 16-31
// their bottom halves.
// FP64 (12 FP64 instructions per point) writes y and z to the scratch buffer and reads them
// and psi back; double-float, whose step leans on HBM more, writes them over psi and
// recovers psi_i = y_i - alpha_i y_{i-1} (z_i - alpha_{m-1-i} z_{i+1}) on the way back.
template <typename R, typename Coef, int AXIS>
__global__ void __launch_bounds__(128, 7) k_cn_twisted(KArgs a, int reduce, int renorm) {
  using C = cplx<R>;
  constexpr bool kScratch = std::is_same<R, double>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = AXIS == 0 ? a.nx : AXIS == 1 ? a.ny : a.nz;
  const int nfixed = AXIS == 0 ? a.ny : a.nx;
  const long long nlines = AXIS == 2 ? (long long)a.nx * a.ny : (long long)nfixed * a.nz;
  const int lane = threadIdx.x & (kWarp - 1);
  const bool bottom = lane >= kWarp / 2;
  const long long line = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kWarp * (kWarp / 2) + (lane & 15);
  const bool active = line < nlines;
  const bool do_reduce = AXIS == 0 && reduce;
  R *wxtab = reinterpret_cast<R *>(smem_raw);   // quadrature weights along x
  if (do_reduce) {
    for (int n = threadIdx.x; n < N; n += blockDim.x) wxtab[n] = R(quad_weight(n, a.nx, a.simpson));
    __syncthreads();
  }
  SumAcc<R> acc[4];
  const long long ln = active ? line : 0;
  const int k = (int)(ln % a.nz), fixed = (int)(ln / a.nz);
  const size_t stride = AXIS == 2 ? (size_t)1 : AXIS == 1 ? (size_t)a.nz : (size_t)a.ny * a.nz;
  // grid index i + 1 of interior point i
  C *p = reinterpret_cast<C *>(a.psi) +
         (AXIS == 2 ? (size_t)ln * a.nz : (AXIS == 1 ? (size_t)fixed * a.ny * a.nz : (size_t)fixed * a.nz) + k) + stride;
  // FP64: y_i (z_i) of this line at yb[i * nlines], consecutive lines side by side
  C *yb = kScratch ? reinterpret_cast<C *>(a.ybuf) + ln : nullptr;
  auto elim = [&](int i) -> C & { return kScratch ? yb[(size_t)i * (size_t)nlines] : p[(size_t)i * stride]; };
  const Coef *tab = reinterpret_cast<const Coef *>(a.cn[AXIS].tab);
  const int lc = a.cn[AXIS].lchunk, chunk = 1 << lc, mp = kWarp << lc, m = a.cn[AXIS].m, h = m / 2;
  const Coef c = CnCoef<R, Coef>::make(pick<R>(a.cn_r[AXIS], a.cn_rf[AXIS], a.cn_rl[AXIS]));
  // table slot of interior point s (lane-interleaved layout)
  auto slot = [&](int s) { return ((s & (chunk - 1)) << 5) + (s >> lc); };
  const int dir = bottom ? -1 : 1;
  const int nf = active ? (bottom ? m - 1 - h : h) : 0;   // elimination steps
  const int i0 = bottom ? m - 1 : 0;                       // first point eliminated
  constexpr int kPf = 4;
  C ring[kPf];
  C y = czero<R>();
#pragma unroll
  for (int j = 0; j < kPf; ++j) ring[j] = j < nf ? p[(ptrdiff_t)(i0 + dir * j) * (ptrdiff_t)stride] : czero<R>();
  for (int s0 = 0; s0 < nf; s0 += kPf) {
#pragma unroll
    for (int j = 0; j < kPf; ++j) {
      const int s = s0 + j;
      if (s < nf) {
        const C v = ring[j];
        if (s + kPf < nf) ring[j] = p[(ptrdiff_t)(i0 + dir * (s + kPf)) * (ptrdiff_t)stride];
        y = cfma(ldg(tab + slot(s)), y, v);
        elim(i0 + dir * s) = y;
      }
    }
  }
  // the twist point: the bottom thread takes y_{h-1} from its partner and solves for x_h
  const C yt = shfl_xor(y, kWarp / 2);
  C xh = czero<R>(), ph = czero<R>();
  if (bottom && active) {
    ph = p[(size_t)h * stride];
    const Coef ginv = ldg(tab + 4 * mp + 10 * kWarp);
    // alpha_{m-1-h} multiplies z_{h+1} (zero when the bottom half eliminated nothing)
    const C rhs = cfma(ldg(tab + slot(m - 1 - h)), y, cfma(ldg(tab + slot(h)), yt, ph));
    xh = mul(ginv, rhs);
  }
  const C xt = shfl_xor(xh, kWarp / 2);
  if (!bottom) xh = xt;
  R s0 = R(0);
  auto emit = [&](int i, C out) {
    p[(size_t)i * stride] = out;
    if (do_reduce) {
      R d = out.re * out.re + out.im * out.im;
      if (a.simpson) d *= wxtab[i + 1];
      s0 += d;
    }
  };
  if (bottom && active) emit(h, C{twice_minus(xh.re, ph.re), twice_minus(xh.im, ph.im)});
  // back-substitution away from h: point ib0 - dir j, table entry tb0 - j
  {
    const int ib0 = bottom ? h + 1 : h - 1;
    const int tb0 = bottom ? m - 2 - h : h - 1;
    // FP64: y_i and psi_i of the coming points; double-float: the eliminated value one point
    // further on (psi_i is recovered from it), the current one carried in `cur`
    C yr[kPf], pr[kScratch ? kPf : 1];
#pragma unroll
    for (int j = 0; j < kPf; ++j) {
      if constexpr (kScratch) {
        const int i = ib0 - dir * j;
        yr[j] = j < nf ? elim(i) : czero<R>();
        pr[j] = j < nf ? p[(ptrdiff_t)i * (ptrdiff_t)stride] : czero<R>();
      } else {
        yr[j] = j + 1 < nf ? elim(ib0 - dir * (j + 1)) : czero<R>();
      }
    }
    C chi = xh, cur = y;
    for (int j0 = 0; j0 < nf; j0 += kPf) {
#pragma unroll
      for (int jj = 0; jj < kPf; ++jj) {
        const int j = j0 + jj;
        if (j < nf) {
          const int i = ib0 - dir * j;
          const int q = slot(tb0 - j);
          C yi, ps;
          if constexpr (kScratch) {
            yi = yr[jj];
            ps = pr[jj];
            if (j + kPf < nf) {
              const int in = ib0 - dir * (j + kPf);
              yr[jj] = elim(in);
              pr[jj] = p[(ptrdiff_t)in * (ptrdiff_t)stride];
            }
          } else {
            const C nxt = yr[jj];
            if (j + 1 + kPf < nf) yr[jj] = elim(ib0 - dir * (j + 1 + kPf));
            yi = cur;
            ps = cfma(neg_coef(ldg(tab + q)), nxt, cur);
            cur = nxt;
          }
          chi = mul(ldg(tab + mp + q), cfma_c(c, chi, yi));
          emit(i, C{twice_minus(chi.re, ps.re), twice_minus(chi.im, ps.im)});
        }
      }
    }
  }
  if (active) {
    // the walls (grid points 0 and N-1)
    if (!bottom) p[-(ptrdiff_t)stride] = czero<R>();
    else p[(size_t)m * stride] = czero<R>();
    if (do_reduce) {
      const R wyz = quad_weight_r<R>(fixed, a.ny, a.simpson) * quad_weight_r<R>(k, a.nz, a.simpson);
      const R yv = R(fixed - a.ny / 2) * R(a.hy), zv = R(k - a.nz / 2) * R(a.hz);
      const R tt = wyz * s0;
      acc[0].add(tt);
      acc[2].add(yv * yv * tt);
      acc[3].add(zv * zv * tt);
    }
  }
  if (do_reduce) {
    double v[4] = {acc[0].value(), acc[1].value(), acc[2].value(), acc[3].value()};
    finish_sweep_sums(a, v, renorm);
  }
}

// ---------------------------------------------------------------------------------------
// Adjoint of the real-time potential step (the paper has no adjoint; this differentiates
// the step above by hand).  With P(psi) = e^{-i theta} psi, theta = dt (V + g n + gdd Phi[n])
// and the cotangent gbar1 of P's output:
//   u = e^{+i theta} gbar1,  s = Im(conj(gbar1) P(psi)) = Im(conj(u) psi),
//   gbar = u + 2 dt (g s + gdd Phi[s]) psi,
//   dL/dg = dt sum s n,  dL/dgdd = dt sum s Phi[n],  dL/dnu_z = dt nu_z sum s z^2.
// k5_adj_phase: C2R of the spectrum of n -> Phi[n]; theta; u (written over gbar); the three
// sums; then s is transformed along z (R2C, as in K1) and written back to the same
// spectrum column (each CTA owns its (i, j0..) column, so reading and writing it is safe).
// k5_adj_combine: C2R of the spectrum of s (after the y/x passes) -> Phi[s]; final gbar.
// ---------------------------------------------------------------------------------------
template <typename R>
struct AdjSums;
template <>
struct AdjSums<double> {
  double v[3] = {0, 0, 0};
  __device__ __forceinline__ void add(double sg, double sdd, double snu) {
    v[0] += sg;
    v[1] += sdd;
    v[2] += snu;
  }
  __device__ __forceinline__ double get(int q) const { return v[q]; }
};
template <>
struct AdjSums<df> {
  df v[3] = {df{0.0f, 0.0f}, df{0.0f, 0.0f}, df{0.0f, 0.0f}};
  __device__ __forceinline__ void add(df sg, df sdd, df snu) {
    v[0] = v[0] + sg;
    v[1] = v[1] + sdd;
    v[2] = v[2] + snu;
  }
  __device__ __forceinline__ double get(int q) const { return (double)v[q]; }
};
template <>
struct AdjSums<float> {
  DFAcc v[3];
  __device__ __forceinline__ void add(float sg, float sdd, float snu) {
    v[0].add(sg);
    v[1].add(sdd);
    v[2].add(snu);
  }
  __device__ __forceinline__ double get(int q) const { return v[q].value(); }
};

template <typename R>
__device__ __forceinline__ void load_half_spectrum_column(const KArgs &a, cplx<R> *za, int i, int j0, int np) {
  using C = cplx<R>;
  constexpr int PZ = Tiles<R>::kZLines / 2;
  constexpr int SB = PZ + 1;
  const int nz = a.nz, half = nz / 2;
  const C *spec = reinterpret_cast<const C *>(a.spec) + (size_t)i * a.ny + j0;
  const size_t plane = (size_t)a.nx * a.ny;
  const int p = threadIdx.x % PZ;
  if (p >= np) return;
  for (int m = threadIdx.x / PZ; m < a.nzh; m += blockDim.x / PZ) {
    C x1 = spec[m * plane + 2 * p];
    C x2 = spec[m * plane + 2 * p + 1];
    if (m == 0 || m == half) {
      x1.im = R(0);
      x2.im = R(0);
    }
    za[m * SB + p] = {x1.re - x2.im, x1.im + x2.re};
    if (m > 0 && m < half) za[(nz - m) * SB + p] = {x1.re + x2.im, x2.re - x1.im};
  }
}

template <typename R>
__device__ __forceinline__ void store_half_spectrum_column(const KArgs &a, const cplx<R> *res, int i, int j0, int np) {
  using C = cplx<R>;
  constexpr int PZ = Tiles<R>::kZLines / 2;
  constexpr int SB = PZ + 1;
  const int nz = a.nz;
  C *spec = reinterpret_cast<C *>(a.spec) + (size_t)i * a.ny + j0;
  const size_t plane = (size_t)a.nx * a.ny;
  const int p = threadIdx.x % PZ;
  if (p >= np) return;
  for (int m = threadIdx.x / PZ; m < a.nzh; m += blockDim.x / PZ) {
    const C zm = res[m * SB + p];
    const C zc = res[((nz - m) % nz) * SB + p];
    C *dst = spec + m * plane + 2 * p;
    dst[0] = {zm.re + zc.re, zm.im - zc.im};   // the packed input carries the factor 1/2
    dst[1] = {zm.im + zc.im, zc.re - zm.re};
  }
}

// N > 0: the compile-time transforms of that length (FP32, the default z plan)
template <typename R, int N = 0>
__global__ void __launch_bounds__(Tiles<R>::kZThreads) k5_adj_phase(KArgs a) {
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int BZ = Tiles<R>::kZLines;
  constexpr int PZ = BZ / 2;
  constexpr int SB = PZ + 1;
  const int nz = N > 0 ? N : a.nz, i = blockIdx.y, j0 = blockIdx.x * BZ;
  const int nl = min(BZ, a.ny - j0), np = nl >> 1;
  C *za = reinterpret_cast<C *>(smem_raw);
  C *zb = za + nz * SB;
  C *pk = zb + nz * SB;      // psi_k tile [b][n]
  C *gt = pk + BZ * nz;      // gbar tile [b][n]
  R *tz = reinterpret_cast<R *>(gt + BZ * nz);
  R *z2 = tz + nz;
  R *txy = z2 + nz;
  const size_t line0 = (size_t)i * a.ny + j0;
  const C *psi = reinterpret_cast<const C *>(a.psi) + line0 * nz;
  C *gb = reinterpret_cast<C *>(a.gbar) + line0 * nz;
  for (int e = threadIdx.x; e < nl * nz; e += blockDim.x) {
    cp_async(pk + e, psi + e);
    cp_async(gt + e, gb + e);
  }
  const R *dtv_x = reinterpret_cast<const R *>(a.dtv[0]);
  const R *dtv_y = reinterpret_cast<const R *>(a.dtv[1]);
  const R *dtv_z = reinterpret_cast<const R *>(a.dtv[2]);
  for (int n = threadIdx.x; n < nz; n += blockDim.x) {
    tz[n] = dtv_z[n];
    const double zc = coordinate(n, nz, a.hz);
    z2[n] = R(zc * zc);
  }
  if (threadIdx.x < nl) txy[threadIdx.x] = dtv_x[i] + dtv_y[j0 + threadIdx.x];
  load_half_spectrum_column<R>(a, za, i, j0, np);
  __syncthreads();
  C *res = fft_lines_n<R, +1, N, PZ, SB, Tiles<R>::kZThreads>(za, zb, a.plan[2], np, reinterpret_cast<const C *>(a.tw[2]));
  C *sbuf = (res == za) ? zb : za;
  cp_async_wait_all();
  __syncthreads();
  const R dtg = pick<R>(a.dtg, a.dtg_f, a.dtg_l), dtgdd = pick<R>(a.dtgdd_n, a.dtgdd_n_f, a.dtgdd_n_l);
  const R inv_ntot = pick<R>(a.inv_ntot, a.inv_ntot_f, a.inv_ntot_l);
  AdjSums<R> acc;
  LinePos pos(threadIdx.x, nz, blockDim.x);
  for (int e = threadIdx.x; e < nl * nz; e += blockDim.x, pos.next()) {
    const int b = pos.b, n = pos.k;
    const C v = pk[e];
    const C g1 = gt[e];
    const C z = res[n * SB + (b >> 1)];
    const R phi = (b & 1) ? z.im : z.re;
    const R dens = v.re * v.re + v.im * v.im;
    const R theta = fma(dtg, dens, fma(dtgdd, phi, txy[b] + tz[n]));
    R sn, cs;
    sin_cos(theta, &sn, &cs);
    const C u = {g1.re * cs - g1.im * sn, g1.re * sn + g1.im * cs};
    const R sv = u.re * v.im - u.im * v.re;
    gt[e] = u;
    reinterpret_cast<R *>(sbuf + n * SB + (b >> 1))[b & 1] = R(0.5) * sv;   // 1/2 of the R2C separation
    acc.add(sv * dens, sv * phi * inv_ntot, sv * z2[n]);
  }
  __syncthreads();
  const C *res2 = fft_lines_n<R, -1, N, PZ, SB, Tiles<R>::kZThreads>(sbuf, res, a.plan[2], np, reinterpret_cast<const C *>(a.tw[2]));
  store_half_spectrum_column<R>(a, res2, i, j0, np);
  for (int e = threadIdx.x; e < nl * nz; e += blockDim.x) gb[e] = gt[e];
  double v3[3] = {acc.get(0), acc.get(1), acc.get(2)};
  if (reduce_across_blocks<3>(v3, a.partials, &a.state->ticket) && threadIdx.x == 0) {
    a.state->grads[0] += a.dt * v3[0];
    a.state->grads[1] += a.dt * v3[1];
    a.state->grads[2] += a.dt_nuz * v3[2];
    if (a.grad_nu_slot) *a.grad_nu_slot += a.dt_nuz * v3[2];
  }
}

template <typename R, int N = 0>
__global__ void __launch_bounds__(Tiles<R>::kZThreads) k5_adj_combine(KArgs a) {
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int BZ = Tiles<R>::kZLines;
  constexpr int PZ = BZ / 2;
  constexpr int SB = PZ + 1;
  const int nz = N > 0 ? N : a.nz, i = blockIdx.y, j0 = blockIdx.x * BZ;
  const int nl = min(BZ, a.ny - j0), np = nl >> 1;
  C *za = reinterpret_cast<C *>(smem_raw);
  C *zb = za + nz * SB;
  C *pk = zb + nz * SB;
  C *gt = pk + BZ * nz;
  const size_t line0 = (size_t)i * a.ny + j0;
  const C *psi = reinterpret_cast<const C *>(a.psi) + line0 * nz;
  C *gb = reinterpret_cast<C *>(a.gbar) + line0 * nz;
  for (int e = threadIdx.x; e < nl * nz; e += blockDim.x) {
    cp_async(pk + e, psi + e);
    cp_async(gt + e, gb + e);
  }
  load_half_spectrum_column<R>(a, za, i, j0, np);
  __syncthreads();
  const C *res = fft_lines_n<R, +1, N, PZ, SB, Tiles<R>::kZThreads>(za, zb, a.plan[2], np, reinterpret_cast<const C *>(a.tw[2]));
  cp_async_wait_all();
  __syncthreads();
  const R dtg = pick<R>(a.dtg, a.dtg_f, a.dtg_l), dtgdd = pick<R>(a.dtgdd_n, a.dtgdd_n_f, a.dtgdd_n_l);
  LinePos pos(threadIdx.x, nz, blockDim.x);
  for (int e = threadIdx.x; e < nl * nz; e += blockDim.x, pos.next()) {
    const int b = pos.b, n = pos.k;
    const C v = pk[e];
    const C u = gt[e];
    const C z = res[n * SB + (b >> 1)];
    const R phis = (b & 1) ? z.im : z.re;
    const R sv = u.re * v.im - u.im * v.re;
    const R coef = R(2) * fma(dtg, sv, dtgdd * phis);
    gb[e] = {fma(coef, v.re, u.re), fma(coef, v.im, u.im)};
  }
}

// Cotangent of L = hx hy hz sum z^2 |psi|^2: gbar = 2 hx hy hz z^2 psi.
template <typename R>
__global__ void k_loss_z2(KArgs a, size_t count) {
  using C = cplx<R>;
  const C *psi = reinterpret_cast<const C *>(a.psi);
  C *gb = reinterpret_cast<C *>(a.gbar);
  const R w = R(2.0 * a.hx * a.hy * a.hz);
  const R hz = R(a.hz);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count; q += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(q % a.nz);
    const R z = R(k - a.nz / 2) * hz;
    gb[q] = scale(psi[q], w * z * z);
  }
}

// psi <- s psi, then s <- 1 (set by the last block).
template <typename R>
__global__ void k_materialize(KArgs a, size_t count) {
  using C = cplx<R>;
  const R s = scale_of<R>(a.state);
  C *psi = reinterpret_cast<C *>(a.psi);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count; q += (size_t)gridDim.x * blockDim.x)
    psi[q] = scale(psi[q], s);
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&a.state->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    set_scale(a.state, 1.0);
    a.state->ticket = 0u;
  }
}

// ---------------------------------------------------------------------------------------
// Host launchers of one precision.
// ---------------------------------------------------------------------------------------
template <typename R>
struct Impl {
  using C = cplx<R>;
  using T = Tiles<R>;
  static constexpr size_t E = sizeof(C);
  // compile-time transforms of lengths 128-512 (not for double-float: its kernels take many
  // times longer to compile)
  static constexpr bool kCtSizes = !std::is_same<R, df>::value;
  // FP32 also at nz = 96 and 64 (K1, K5; the batched small grids)
  static constexpr bool kShortCt = std::is_same<R, float>::value;
  // the padded (FULL) chunked sweeps: the y sweep on 8 warps, two columns each in lockstep
  // (one CTA per SM); the x sweep, whose store also takes the norm sums (a longer serial chain
  // per thread at half the threads), on 16 warps of one column each
  template <int AXIS>
  static constexpr int cn_full_threads() { return AXIS == 1 ? 256 : T::kCnThreads; }
  // the FP64-class sweeps run a Thomas solve per line on two threads (k_cn_twisted), the
  // FP32 ones the chunked solver in persistent tiles (k_cn)
  static constexpr bool kCnThread = Fp64Class<R>::value;
  // and the z sweep too, after a phase-only K5 pass: the per-line solve's fewer arithmetic
  // instructions win over the extra pass through HBM
  static constexpr bool kZSplit = Fp64Class<R>::value;

  static size_t smem_z_fft(const KArgs &a, int bz = T::kZLines) { return 2 * (size_t)a.nz * (bz / 2 + 1) * E; }
  // K5's grid and shared memory for tiles of bz lines
  static dim3 grid_z5(const KArgs &a, int bz) { return dim3((a.ny + bz - 1) / bz, a.nx); }
  static size_t smem_k5(const KArgs &a, int bz = T::kZLines) {
    // the tile: the sweeps' layout, or (FP32, compile-time lengths) K5's padded one
    int ls = cn_slots(a.nz, a.cn[2].lchunk);
    if (std::is_same<R, float>::value &&
        (a.nz == 64 || a.nz == 96 || a.nz == 128 || a.nz == 256 || a.nz == 384 || a.nz == 512))
      ls = std::max(ls, k5_tile_stride(a.nz));
    return 2 * (size_t)a.nz * (bz / 2) * E + (size_t)bz * ls * E + (size_t)(a.nz + bz) * sizeof(R) +
           (size_t)10 * kWarp * E;
  }
  static size_t smem_y(const KArgs &a) { return 2 * (size_t)a.ny * (a.ylines + 1) * E; }
  static size_t smem_x(const KArgs &a) { return 2 * (size_t)a.nx * T::kXCols * E; }
  static size_t smem_cn(int n, int lchunk, int cols = T::kCnCols) {
    return 2 * (size_t)cn_slots(n, lchunk) * (cols + 1) * E + (size_t)(4 * (kWarp << lchunk) + 10 * kWarp) * E +
           2 * (size_t)n * sizeof(R);
  }


  static dim3 grid_z(const KArgs &a) { return dim3((a.ny + T::kZLines - 1) / T::kZLines, a.nx); }
  // persistent grid of the CN kernels: all tiles, capped at the number of co-resident CTAs
  static int sm_count() {
    static int n = 0;
    if (!n) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      if (n <= 0) n = 1;
    }
    return n;
  }
  // the chunked sweeps pad a line to 32 whole chunks (no per-point guard) when that adds at
  // most two unknowns (the power-of-two lengths); the tile line then has 32 chunk + 2 points
  static bool cn_full(const KArgs &a, int axis) { return (kWarp << a.cn[axis].lchunk) <= a.cn[axis].m + 2; }
  static int cn_len(const KArgs &a, int axis) {
    return cn_full(a, axis) ? (kWarp << a.cn[axis].lchunk) + 2 : a.cn[axis].m + 2;
  }
  static dim3 grid_cn(const KArgs &a, int axis, int cols = T::kCnCols) {
    const int tiles = ((a.nz + cols - 1) / cols) * (axis == 0 ? a.ny : a.nx);
    const int n = cn_len(a, axis);
    const size_t sm = smem_cn(n, a.cn[axis].lchunk, cols);
    // co-resident CTAs per SM: by shared memory, and by registers (NT threads of up to 128)
    const int fit_regs = 65536 / (T::kCnThreads * 128) < 1 ? 1 : 65536 / (T::kCnThreads * 128);
    const int fit = std::min(sm * 2 + 4096 <= 227 * 1024 ? 2 : 1, fit_regs);
    const int per_sm = a.cn_per_sm < fit ? (a.cn_per_sm < 1 ? 1 : a.cn_per_sm) : fit;
    const int cap = sm_count() * per_sm;
    return dim3(tiles < cap ? tiles : cap);
  }

  // Allow each kernel the device's opt-in shared memory minus its static shared memory.
  template <typename K>
  static cudaError_t allow_smem(K kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
  }

  // (a member of the class template: instantiated only where it is called, FP32)
  static cudaError_t init_reg() {
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) {
      if (e == cudaSuccess) e = r;
    };
    using K = void (*)(KArgs, const KArgs *);
    chk(allow_smem(static_cast<K>(k_ffty_reg<-1, 512>)));
    chk(allow_smem(static_cast<K>(k_ffty_reg<+1, 512>)));
    chk(allow_smem(static_cast<K>(k_ffty_reg<-1, 256>)));
    chk(allow_smem(static_cast<K>(k_ffty_reg<+1, 256>)));
    chk(allow_smem(static_cast<K>(k_ffty_reg<-1, 128>)));
    chk(allow_smem(static_cast<K>(k_ffty_reg<+1, 128>)));
    chk(allow_smem(static_cast<K>(k3_reg<512>)));
    chk(allow_smem(static_cast<K>(k3_reg<256>)));
    chk(allow_smem(static_cast<K>(k3_reg<128>)));
    return e;
  }

  static cudaError_t init() {
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) {
      if (e == cudaSuccess) e = r;
    };
    chk(allow_smem(k1_density_r2cz<R, 0>));
    chk(allow_smem(k_ffty<R, -1, 0>));
    chk(allow_smem(k_ffty<R, +1, 0>));
    chk(allow_smem(k3_fftx_dipolar<R, 0>));
    chk(allow_smem(k5_zline<R, R, kZFast, 0>));
    chk(allow_smem(k5_zline<R, C, kZFast, 0>));
    if constexpr (!kZSplit) {
      chk(allow_smem(k5_zline<R, R, kZPhaseOnly, 0>));
      chk(allow_smem(k5_zline<R, C, kZPhaseOnly, 0>));
      chk(allow_smem(k5_zline<R, R, kZCnOnly, 0>));
      chk(allow_smem(k5_zline<R, C, kZCnOnly, 0>));
    }
    chk(allow_smem(k5_zline<R, R, kZPhi, 0>));
    chk(allow_smem(k5_zline<R, R, kZObs, 0>));
    if constexpr (kCtSizes) {
      chk(allow_smem(k1_density_r2cz<R, 512>));
      chk(allow_smem(k1_density_r2cz<R, 384>));
      chk(allow_smem(k1_density_r2cz<R, 256>));
      chk(allow_smem(k1_density_r2cz<R, 128>));
      chk(allow_smem(k_ffty<R, -1, 512>));
      chk(allow_smem(k_ffty<R, +1, 512>));
      chk(allow_smem(k_ffty<R, -1, 384>));
      chk(allow_smem(k_ffty<R, +1, 384>));
      chk(allow_smem(k_ffty<R, -1, 256>));
      chk(allow_smem(k_ffty<R, +1, 256>));
      chk(allow_smem(k_ffty<R, -1, 128>));
      chk(allow_smem(k_ffty<R, +1, 128>));
      chk(allow_smem(k3_fftx_dipolar<R, 512>));
      chk(allow_smem(k3_fftx_dipolar<R, 384>));
      chk(allow_smem(k3_fftx_dipolar<R, 256>));
      chk(allow_smem(k3_fftx_dipolar<R, 128>));
      chk(allow_smem(k5_zline<R, R, kZFast, 512>));
      chk(allow_smem(k5_zline<R, C, kZFast, 512>));
      chk(allow_smem(k5_zline<R, R, kZFast, 384>));
      chk(allow_smem(k5_zline<R, C, kZFast, 384>));
      chk(allow_smem(k5_zline<R, R, kZFast, 256>));
      chk(allow_smem(k5_zline<R, C, kZFast, 256>));
      chk(allow_smem(k5_zline<R, R, kZFast, 128>));
      chk(allow_smem(k5_zline<R, C, kZFast, 128>));
      if constexpr (kShortCt) {
        chk(allow_smem(k1_density_r2cz<R, 96>));
        chk(allow_smem(k1_density_r2cz<R, 64>));
        chk(allow_smem(k5_zline<R, R, kZFast, 96>));
        chk(allow_smem(k5_zline<R, C, kZFast, 96>));
        chk(allow_smem(k5_zline<R, R, kZFast, 64>));
        chk(allow_smem(k5_zline<R, C, kZFast, 64>));
      }
    }
    if constexpr (!kCnThread) {
      constexpr int B = T::kCnCols, NT = T::kCnThreads;
      chk(allow_smem(k_cn<R, R, 0>));
      chk(allow_smem(k_cn<R, R, 1>));
      chk(allow_smem(k_cn<R, C, 0>));
      chk(allow_smem(k_cn<R, C, 1>));
      chk(allow_smem(k_cn<R, R, 0, B, cn_full_threads<0>(), false, true>));
      chk(allow_smem(k_cn<R, R, 1, B, cn_full_threads<1>(), false, true>));
      chk(allow_smem(k_cn<R, C, 0, B, cn_full_threads<0>(), false, true>));
      chk(allow_smem(k_cn<R, C, 1, B, cn_full_threads<1>(), false, true>));
    }
    if constexpr (kRegFft) chk(init_reg());
    if constexpr (kAdjoint) chk(allow_smem(k5_adj_phase<R>));
    if constexpr (kAdjoint) chk(allow_smem(k5_adj_combine<R>));
    if constexpr (kAdjoint && kShortCt) {
      chk(allow_smem(k5_adj_phase<R, 128>));
      chk(allow_smem(k5_adj_phase<R, 256>));
      chk(allow_smem(k5_adj_phase<R, 384>));
      chk(allow_smem(k5_adj_phase<R, 512>));
      chk(allow_smem(k5_adj_combine<R, 128>));
      chk(allow_smem(k5_adj_combine<R, 256>));
      chk(allow_smem(k5_adj_combine<R, 384>));
      chk(allow_smem(k5_adj_combine<R, 512>));
    }
    return e;
  }

  static cudaError_t twiddles(void *tw, const FftPlan &pl, cudaStream_t st) {
    k_twiddles<R><<<(pl.n + 127) / 128, 128, 0, st>>>(reinterpret_cast<C *>(tw), pl);
    return cudaGetLastError();
  }

  static cudaError_t cn_tables(const CnJobs &jobs, cudaStream_t st) {
    if (jobs.n <= 0) return cudaSuccess;
    if (jobs.imag) k_cn_tables<R, R><<<jobs.n, 32, 0, st>>>(jobs);
    else k_cn_tables<R, C><<<jobs.n, 32, 0, st>>>(jobs);
    return cudaGetLastError();
  }

  static cudaError_t axis_potential(void *out, int n, double h, double v, double dt, cudaStream_t st) {
    k_axis_potential<R><<<(n + 127) / 128, 128, 0, st>>>(reinterpret_cast<R *>(out), n, h, v, dt);
    return cudaGetLastError();
  }

  static cudaError_t dipolar_table(const KArgs &a, cudaStream_t st) {
    if (!Fp64Class<R>::value) return cudaSuccess;   // FP32 evaluates the kernel in K3
    const size_t total = (size_t)a.nzh * a.nx * a.ny;
    const size_t want = (total + 255) / 256, cap = (size_t)sm_count() * 8;
    const int blocks = (int)(want < cap ? want : cap);
    k_dipolar_table<R><<<blocks, 256, 0, st>>>(reinterpret_cast<R *>(const_cast<void *>(a.utab)), a);
    return cudaGetLastError();
  }

  static cudaError_t from_c128(const void *src, void *psi, size_t n, cudaStream_t st) {
    if constexpr (!std::is_same<R, df>::value) {
      return cudaErrorNotSupported;
    } else {
      const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 16);
      k_c128_to_pair<R><<<blocks, 256, 0, st>>>(static_cast<const double2 *>(src), static_cast<C *>(psi), n);
      return cudaGetLastError();
    }
  }
  static cudaError_t to_c128(const void *psi, void *dst, size_t n, cudaStream_t st) {
    if constexpr (!std::is_same<R, df>::value) {
      return cudaErrorNotSupported;
    } else {
      const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 16);
      k_pair_to_c128<R><<<blocks, 256, 0, st>>>(static_cast<const C *>(psi), static_cast<double2 *>(dst), n);
      return cudaGetLastError();
    }
  }

  static cudaError_t reset_state(DevState *s, cudaStream_t st) {
    k_reset_state<R><<<1, 32, 0, st>>>(s);
    return cudaGetLastError();
  }

  // the plan of length n is make_plan's default (the compile-time transforms follow it)
  static bool plan_ct(const FftPlan &pl, int n) {
    if (pl.n != n) return false;
    for (int st = 0; st < kMaxStages; ++st) {
      const int p = st < pl.nstages ? pl.radix[st] : 0;
      if (p != ct_radix(n, st)) return false;
      if (p == 0) break;
    }
    return true;
  }
  static cudaError_t k1(const KArgs &a, cudaStream_t st) {
    // (instances of other tile heights, ztile_lines, get their own grid and shared memory)
    auto go = [&](auto len) {
      constexpr int N = decltype(len)::value;
      constexpr int bz = ztile_lines<R>(N);
      k1_density_r2cz<R, N><<<grid_z5(a, bz), T::kZThreads, smem_z_fft(a, bz), st>>>(a, nullptr);
    };
    using std::integral_constant;
    if constexpr (kCtSizes) {
      if (plan_ct(a.plan[2], 512)) go(integral_constant<int, 512>{});
      else if (plan_ct(a.plan[2], 384)) go(integral_constant<int, 384>{});
      else if (plan_ct(a.plan[2], 256)) go(integral_constant<int, 256>{});
      else if (plan_ct(a.plan[2], 128)) go(integral_constant<int, 128>{});
      else if (kShortCt && plan_ct(a.plan[2], 96)) go(integral_constant<int, kShortCt ? 96 : 0>{});
      else if (kShortCt && plan_ct(a.plan[2], 64)) go(integral_constant<int, kShortCt ? 64 : 0>{});
      else go(integral_constant<int, 0>{});
    } else {
      go(integral_constant<int, 0>{});
    }
    return cudaGetLastError();
  }
  // the compile-time transform applies when the y plan, lines per CTA and block size are
  // the defaults for that length
  static bool y_fixed(const KArgs &a, int n) {
    return a.ylines == y_lines_per_cta<R>(n) && a.fft_threads == kFftThreads && plan_ct(a.plan[1], n);
  }
  // the register-resident FP32 transforms (default plans of length 128, 256, 512)
  static constexpr bool kRegFft = std::is_same<R, float>::value;
  static constexpr size_t kRegYSmem = 2 * (256 / 64) * (size_t)RegFft<512>::SLOTS * sizeof(cplx<float>);
  template <int N>
  static constexpr size_t reg_x_smem() { return 2 * 8 * (size_t)RegFft<N>::SLOTS * sizeof(cplx<float>); }
  template <int DIR, int N>
  static void ffty_reg(const KArgs &a, cudaStream_t st) {
    const size_t lines = (size_t)a.nzh * a.nx, lpc = 256 / RegFft<N>::T;
    k_ffty_reg<DIR, N><<<(unsigned)((lines + lpc - 1) / lpc), 256, kRegYSmem, st>>>(a, nullptr);
  }
  template <int N>
  static void k3_reg_launch(const KArgs &a, cudaStream_t st) {
    const dim3 grid((a.ny + 7) / 8, a.nzh);
    k3_reg<N><<<grid, 8 * RegFft<N>::T, reg_x_smem<N>(), st>>>(a, nullptr);
  }
  template <int DIR>
  static cudaError_t ffty(const KArgs &a, cudaStream_t st) {
    if constexpr (kRegFft) {
      if (plan_ct(a.plan[1], 512)) return ffty_reg<DIR, 512>(a, st), cudaGetLastError();
      if (plan_ct(a.plan[1], 256)) return ffty_reg<DIR, 256>(a, st), cudaGetLastError();
      if (plan_ct(a.plan[1], 128)) return ffty_reg<DIR, 128>(a, st), cudaGetLastError();
    }
    const size_t lines = (size_t)a.nzh * a.nx;
    const int L = a.ylines;
    const dim3 g((unsigned)((lines + L - 1) / L));
    const size_t sm = smem_y(a);
    if constexpr (kCtSizes) {
      if (y_fixed(a, 512)) k_ffty<R, DIR, 512><<<g, kFftThreads, sm, st>>>(a, nullptr);
      else if (y_fixed(a, 384)) k_ffty<R, DIR, 384><<<g, kFftThreads, sm, st>>>(a, nullptr);
      else if (y_fixed(a, 256)) k_ffty<R, DIR, 256><<<g, kFftThreads, sm, st>>>(a, nullptr);
      else if (y_fixed(a, 128)) k_ffty<R, DIR, 128><<<g, kFftThreads, sm, st>>>(a, nullptr);
      else k_ffty<R, DIR, 0><<<g, a.fft_threads, sm, st>>>(a, nullptr);
    } else {
      k_ffty<R, DIR, 0><<<g, a.fft_threads, sm, st>>>(a, nullptr);
    }
    return cudaGetLastError();
  }
  static cudaError_t k2(const KArgs &a, cudaStream_t st) { return ffty<-1>(a, st); }
  static cudaError_t k3(const KArgs &a, cudaStream_t st) {
    if constexpr (kRegFft) {
      if (plan_ct(a.plan[0], 512)) return k3_reg_launch<512>(a, st), cudaGetLastError();
      if (plan_ct(a.plan[0], 256)) return k3_reg_launch<256>(a, st), cudaGetLastError();
      if (plan_ct(a.plan[0], 128)) return k3_reg_launch<128>(a, st), cudaGetLastError();
    }
    dim3 grid((a.ny + T::kXCols - 1) / T::kXCols, a.nzh);
    const size_t sm = smem_x(a);
    const bool fixed = a.fft_threads == kFftThreads;
    if constexpr (kCtSizes) {
      if (fixed && plan_ct(a.plan[0], 512)) k3_fftx_dipolar<R, 512><<<grid, kFftThreads, sm, st>>>(a, nullptr);
      else if (fixed && plan_ct(a.plan[0], 384)) k3_fftx_dipolar<R, 384><<<grid, kFftThreads, sm, st>>>(a, nullptr);
      else if (fixed && plan_ct(a.plan[0], 256)) k3_fftx_dipolar<R, 256><<<grid, kFftThreads, sm, st>>>(a, nullptr);
      else if (fixed && plan_ct(a.plan[0], 128)) k3_fftx_dipolar<R, 128><<<grid, kFftThreads, sm, st>>>(a, nullptr);
      else k3_fftx_dipolar<R, 0><<<grid, a.fft_threads, sm, st>>>(a, nullptr);
    } else {
      k3_fftx_dipolar<R, 0><<<grid, a.fft_threads, sm, st>>>(a, nullptr);
    }
    return cudaGetLastError();
  }
  static cudaError_t k4(const KArgs &a, cudaStream_t st) { return ffty<+1>(a, st); }
  // K5 in mode ZM with coefficient type Co: the compile-time transform when the z plan is
  // the default one of a supported length.
  template <int ZM, typename Co>
  static void k5_launch(const KArgs &a, dim3 g, size_t sm, cudaStream_t st) {
    // (instances of other tile heights, ztile_lines, get their own grid and shared memory)
    auto go = [&](auto len) {
      constexpr int N = decltype(len)::value;
      constexpr int bz = ztile_lines<R>(N);
      if constexpr (bz == T::kZLines) k5_zline<R, Co, ZM, N><<<g, T::kZThreads, sm, st>>>(a, nullptr);
      else k5_zline<R, Co, ZM, N><<<grid_z5(a, bz), T::kZThreads, smem_k5(a, bz), st>>>(a, nullptr);
    };
    using std::integral_constant;
    if constexpr (kCtSizes) {
      if (plan_ct(a.plan[2], 512)) go(integral_constant<int, 512>{});
      else if (plan_ct(a.plan[2], 384)) go(integral_constant<int, 384>{});
      else if (plan_ct(a.plan[2], 256)) go(integral_constant<int, 256>{});
      else if (plan_ct(a.plan[2], 128) && (!kShortCt || a.cn8_tab[2])) go(integral_constant<int, 128>{});
      else if (kShortCt && plan_ct(a.plan[2], 96) && a.cn8_tab[2]) go(integral_constant<int, kShortCt ? 96 : 0>{});
      else if (kShortCt && plan_ct(a.plan[2], 64) && a.cn8_tab[2]) go(integral_constant<int, kShortCt ? 64 : 0>{});
      else go(integral_constant<int, 0>{});
    } else {
      go(integral_constant<int, 0>{});
    }
  }
  // the mode whose compile-time instances exist: the fused step (FP32), or the phase-only
  // pass that precedes the per-line z sweep (FP64-class)
  static constexpr int kZFast = kZSplit ? kZPhaseOnly : kZStep;
  static cudaError_t k5(const KArgs &a, int zmode, cudaStream_t st) {
    if constexpr (kZSplit) {
      // the z sweep runs per line (two threads each) after the phase-only pass
      if (zmode == kZCnOnly) return cn<2>(a, 0, 0, st);
      if (zmode == kZStep) {
        const cudaError_t e = k5(a, kZPhaseOnly, st);
        return e != cudaSuccess ? e : cn<2>(a, 0, 0, st);
      }
    }
    const dim3 g = grid_z(a);
    const size_t sm = smem_k5(a);
    if (zmode == kZFast) {
      if (a.imag) k5_launch<kZFast, R>(a, g, sm, st);
      else k5_launch<kZFast, C>(a, g, sm, st);
      return cudaGetLastError();
    }
    switch (zmode) {
      case kZPhaseOnly:
        if constexpr (!kZSplit) {
          if (a.imag) k5_zline<R, R, kZPhaseOnly, 0><<<g, T::kZThreads, sm, st>>>(a, nullptr);
          else k5_zline<R, C, kZPhaseOnly, 0><<<g, T::kZThreads, sm, st>>>(a, nullptr);
        }
        break;
      case kZCnOnly:
        if constexpr (!kZSplit) {
          if (a.imag) k5_zline<R, R, kZCnOnly, 0><<<g, T::kZThreads, sm, st>>>(a, nullptr);
          else k5_zline<R, C, kZCnOnly, 0><<<g, T::kZThreads, sm, st>>>(a, nullptr);
        }
        break;
      case kZPhi: k5_zline<R, R, kZPhi, 0><<<g, T::kZThreads, sm, st>>>(a, nullptr); break;
      case kZObs: k5_zline<R, R, kZObs, 0><<<g, T::kZThreads, sm, st>>>(a, nullptr); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  // The short-line sweep (FP32, x or y lines of short_cn_chunk(n) != 0 with their 8-lane
  // tables): launched for `members` condensates (blockIdx.z; ga their arguments when GRP) on
  // one resident wave of persistent CTAs, four per SM.  False when the line takes k_cn.
  template <int AXIS, bool GRP>
  static bool cn_short(const KArgs &a, const KArgs *ga, unsigned members, int reduce, int renorm, cudaStream_t st) {
    if constexpr (!std::is_same<R, float>::value) {
      return false;
    } else {
      const int n = AXIS == 0 ? a.nx : a.ny;
      const int ch = short_cn_chunk(n);
      if (!ch || !a.cn8_tab[AXIS]) return false;
      const int tiles = ((a.nz + 15) / 16) * (AXIS == 0 ? a.ny : a.nx);
      const int per = std::max(1, sm_count() * 4 / (int)members);
      const dim3 g(std::min(tiles, per), 1, members);
      const size_t sm = smem_cn_short(ch);
      auto go = [&](auto chc) {
        constexpr int CH = decltype(chc)::value;
        if (a.imag) k_cn_short<R, AXIS, CH, GRP><<<g, 128, sm, st>>>(a, ga, reduce, renorm);
        else k_cn_short<C, AXIS, CH, GRP><<<g, 128, sm, st>>>(a, ga, reduce, renorm);
      };
      switch (ch) {
        case 4: go(std::integral_constant<int, 4>{}); break;
        case 6: go(std::integral_constant<int, 6>{}); break;
        case 8: go(std::integral_constant<int, 8>{}); break;
        case 12: go(std::integral_constant<int, 12>{}); break;
        default: go(std::integral_constant<int, 16>{}); break;
      }
      return true;
    }
  }
  template <int AXIS>
  static cudaError_t cn(const KArgs &a, int reduce, int renorm, cudaStream_t st) {
    const int n = AXIS == 0 ? a.nx : AXIS == 1 ? a.ny : a.nz;
    if constexpr (kCnThread) {
      const long long lines = AXIS == 2 ? (long long)a.nx * a.ny : (long long)(AXIS == 0 ? a.ny : a.nx) * a.nz;
      const size_t sm = AXIS == 0 ? (size_t)n * sizeof(R) : 0;
      const unsigned blocks = (unsigned)((lines + 63) / 64);   // 64 lines, two threads each
      if (a.imag) k_cn_twisted<R, R, AXIS><<<blocks, 128, sm, st>>>(a, reduce, renorm);
      else k_cn_twisted<R, C, AXIS><<<blocks, 128, sm, st>>>(a, reduce, renorm);
    } else {
      if constexpr (AXIS < 2) {
        if (cn_short<AXIS, false>(a, nullptr, 1, reduce, renorm, st)) return cudaGetLastError();
      }
      constexpr int B = T::kCnCols, NT = T::kCnThreads;
      const size_t sm = smem_cn(cn_len(a, AXIS), a.cn[AXIS].lchunk);
      const dim3 g = grid_cn(a, AXIS);
      if (cn_full(a, AXIS)) {
        constexpr int NF = cn_full_threads<AXIS>();
        if (a.imag) k_cn<R, R, AXIS, B, NF, false, true><<<g, NF, sm, st>>>(a, nullptr, reduce, renorm);
        else k_cn<R, C, AXIS, B, NF, false, true><<<g, NF, sm, st>>>(a, nullptr, reduce, renorm);
      } else {
        if (a.imag) k_cn<R, R, AXIS><<<g, NT, sm, st>>>(a, nullptr, reduce, renorm);
        else k_cn<R, C, AXIS><<<g, NT, sm, st>>>(a, nullptr, reduce, renorm);
      }
    }
    return cudaGetLastError();
  }
  static cudaError_t k6(const KArgs &a, cudaStream_t st) { return cn<1>(a, 0, 0, st); }
  static cudaError_t k7(const KArgs &a, int reduce, int renorm, cudaStream_t st) { return cn<0>(a, reduce, renorm, st); }
  static cudaError_t materialize(const KArgs &a, cudaStream_t st) {
    const size_t count = (size_t)a.nx * a.ny * a.nz;
    size_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_materialize<R><<<(unsigned)blocks, 256, 0, st>>>(a, count);
    return cudaGetLastError();
  }
  // Host-only bound (no device query): the CN grid never exceeds its tile count.
  // the adjoint's phase (PHASE) or combining pass, at a compile-time length where the z plan
  // is the default one (FP32)
  template <bool PHASE>
  static void adj_launch(const KArgs &a, cudaStream_t st) {
    auto go = [&](auto len) {
      constexpr int N = decltype(len)::value;
      if constexpr (PHASE) k5_adj_phase<R, N><<<grid_z(a), T::kZThreads, smem_adj(a), st>>>(a);
      else k5_adj_combine<R, N><<<grid_z(a), T::kZThreads, smem_adj(a), st>>>(a);
    };
    using std::integral_constant;
    if constexpr (kShortCt) {
      if (plan_ct(a.plan[2], 512)) return go(integral_constant<int, 512>{});
      if (plan_ct(a.plan[2], 384)) return go(integral_constant<int, 384>{});
      if (plan_ct(a.plan[2], 256)) return go(integral_constant<int, 256>{});
      if (plan_ct(a.plan[2], 128)) return go(integral_constant<int, 128>{});
    }
    go(integral_constant<int, 0>{});
  }
  static size_t smem_adj(const KArgs &a) {
    return smem_z_fft(a) + 2 * (size_t)T::kZLines * a.nz * E + (size_t)(2 * a.nz + T::kZLines) * sizeof(R);
  }
  // the differentiation kernels exist for FP64 and FP32 only
  static constexpr bool kAdjoint = !std::is_same<R, df>::value;
  static cudaError_t adj_phase(const KArgs &a, cudaStream_t st) {
    if constexpr (!kAdjoint) {
      return cudaErrorNotSupported;
    } else {
      adj_launch<true>(a, st);
      return cudaGetLastError();
    }
  }
  static cudaError_t adj_combine(const KArgs &a, cudaStream_t st) {
    if constexpr (!kAdjoint) {
      return cudaErrorNotSupported;
    } else {
      adj_launch<false>(a, st);
      return cudaGetLastError();
    }
  }
  static cudaError_t loss_z2(const KArgs &a, cudaStream_t st) {
    if constexpr (!kAdjoint) {
      return cudaErrorNotSupported;
    } else {
      const size_t count = (size_t)a.nx * a.ny * a.nz;
      size_t blocks = (count + 255) / 256;
      if (blocks > 8192) blocks = 8192;
      k_loss_z2<R><<<(unsigned)blocks, 256, 0, st>>>(a, count);
      return cudaGetLastError();
    }
  }

  static int default_ylines(int ny) { return y_lines_per_cta<R>(ny); }
  static size_t y_smem(int ny, int ylines) { return 2 * (size_t)ny * (ylines + 1) * E; }

  static int max_blocks(const KArgs &a) {
    const dim3 z = grid_z(a);
    const int bz = (int)(z.x * z.y);
    const int bx = ((a.nz + T::kCnCols - 1) / T::kCnCols) * a.ny;
    const int bt = (int)(((long long)a.ny * a.nz + 63) / 64);   // the two-thread sweep along x
    return std::max(bz, std::max(bx, bt));
  }

  static const KernelSet *set() {
    // groups of same-shaped condensates launched together: FP32 only (kernels_f32_group.cu)
    constexpr bool kGroup = std::is_same<R, float>::value;
    static const KernelSet ks = {(int)E, &init,          &twiddles,   &cn_tables, &axis_potential, &dipolar_table, &from_c128, &to_c128, &reset_state,
                                 &k1,        &k2,            &k3,         &k4,        &k5,             &k6,
                                 &k7,        &materialize,   &adj_phase,  &adj_combine, &loss_z2,
                                 &max_blocks, kZSplit ? 2 : 1, &default_ylines, &y_smem,
                                 kGroup ? &group_init_f32 : nullptr, kGroup ? &group_step_f32 : nullptr};
    return &ks;
  }
};

// ---------------------------------------------------------------------------------------
// One step of a group of same-shaped condensates (same shape, precision, mode and launch
// shape; their own psi, physics and device state): every kernel of the step is launched
// once for all of them, condensate z = blockIdx.z with its arguments ga[z] in device
// memory.  a is one member's arguments, for the launch configuration.  A group of 16
// condensates of 128^3 then runs each kernel as one grid of 16 times the blocks, instead of
// 16 small grids whose launch latency and last partial waves dominate.  The arithmetic per
// condensate is that of its own step, so the results are bitwise the same.
// ---------------------------------------------------------------------------------------
template <typename R>
struct GroupLaunch {
  using I = Impl<R>;
  using C = cplx<R>;
  using T = Tiles<R>;
  static_assert(std::is_same<R, float>::value, "grouped steps serve the FP32-mixed path");

  template <typename K>
  static void attr(K k, cudaError_t &e) {
    if (e == cudaSuccess) e = I::allow_smem(k);
  }
  static cudaError_t init() {
    cudaError_t e = cudaSuccess;
    attr(k1_density_r2cz<R, 512, true>, e);
    attr(k1_density_r2cz<R, 384, true>, e);
    attr(k1_density_r2cz<R, 256, true>, e);
    attr(k1_density_r2cz<R, 128, true>, e);
    attr(k1_density_r2cz<R, 96, true>, e);
    attr(k1_density_r2cz<R, 64, true>, e);
    attr(k1_density_r2cz<R, 0, true>, e);
    attr(k_ffty<R, -1, 0, true>, e);
    attr(k_ffty<R, +1, 0, true>, e);
    attr(k_ffty<R, -1, 384, true>, e);
    attr(k_ffty<R, +1, 384, true>, e);
    attr(k3_fftx_dipolar<R, 384, true>, e);
    attr(k3_fftx_dipolar<R, 0, true>, e);
    using K = void (*)(KArgs, const KArgs *);
    attr(static_cast<K>(k_ffty_reg<-1, 512, true>), e);
    attr(static_cast<K>(k_ffty_reg<+1, 512, true>), e);
    attr(static_cast<K>(k_ffty_reg<-1, 256, true>), e);
    attr(static_cast<K>(k_ffty_reg<+1, 256, true>), e);
    attr(static_cast<K>(k_ffty_reg<-1, 128, true>), e);
    attr(static_cast<K>(k_ffty_reg<+1, 128, true>), e);
    attr(static_cast<K>(k3_reg<512, true>), e);
    attr(static_cast<K>(k3_reg<256, true>), e);
    attr(static_cast<K>(k3_reg<128, true>), e);
    attr(k5_zline<R, R, kZStep, 512, true>, e);
    attr(k5_zline<R, C, kZStep, 512, true>, e);
    attr(k5_zline<R, R, kZStep, 384, true>, e);
    attr(k5_zline<R, C, kZStep, 384, true>, e);
    attr(k5_zline<R, R, kZStep, 256, true>, e);
    attr(k5_zline<R, C, kZStep, 256, true>, e);
    attr(k5_zline<R, R, kZStep, 96, true>, e);
    attr(k5_zline<R, C, kZStep, 96, true>, e);
    attr(k5_zline<R, R, kZStep, 64, true>, e);
    attr(k5_zline<R, C, kZStep, 64, true>, e);
    attr(k5_zline<R, R, kZStep, 128, true>, e);
    attr(k5_zline<R, C, kZStep, 128, true>, e);
    attr(k5_zline<R, R, kZStep, 0, true>, e);
    attr(k5_zline<R, C, kZStep, 0, true>, e);
    attr(k_cn<R, R, 0, T::kCnCols, T::kCnThreads, true>, e);
    attr(k_cn<R, R, 1, T::kCnCols, T::kCnThreads, true>, e);
    attr(k_cn<R, C, 0, T::kCnCols, T::kCnThreads, true>, e);
    attr(k_cn<R, C, 1, T::kCnCols, T::kCnThreads, true>, e);
    attr(k_cn<R, R, 0, T::kCnCols, I::template cn_full_threads<0>(), true, true>, e);
    attr(k_cn<R, R, 1, T::kCnCols, I::template cn_full_threads<1>(), true, true>, e);
    attr(k_cn<R, C, 0, T::kCnCols, I::template cn_full_threads<0>(), true, true>, e);
    attr(k_cn<R, C, 1, T::kCnCols, I::template cn_full_threads<1>(), true, true>, e);
    return e;
  }

  template <int DIR>
  static void ffty(const KArgs &a, const KArgs *ga, unsigned n, cudaStream_t st) {
    const size_t lines = (size_t)a.nzh * a.nx;
    auto reg = [&](auto len) {
      constexpr int N = decltype(len)::value;
      const size_t lpc = 256 / RegFft<N>::T;
      k_ffty_reg<DIR, N, true><<<dim3((unsigned)((lines + lpc - 1) / lpc), 1, n), 256, I::kRegYSmem, st>>>(a, ga);
    };
    if (I::plan_ct(a.plan[1], 512)) return reg(std::integral_constant<int, 512>{});
    if (I::plan_ct(a.plan[1], 256)) return reg(std::integral_constant<int, 256>{});
    if (I::plan_ct(a.plan[1], 128)) return reg(std::integral_constant<int, 128>{});
    const int L = a.ylines;
    const dim3 g((unsigned)((lines + L - 1) / L), 1, n);
    const size_t sm = I::smem_y(a);
    if (I::y_fixed(a, 384)) k_ffty<R, DIR, 384, true><<<g, kFftThreads, sm, st>>>(a, ga);
    else k_ffty<R, DIR, 0, true><<<g, a.fft_threads, sm, st>>>(a, ga);
  }
  static void k3(const KArgs &a, const KArgs *ga, unsigned n, cudaStream_t st) {
    auto reg = [&](auto len) {
      constexpr int N = decltype(len)::value;
      k3_reg<N, true><<<dim3((a.ny + 7) / 8, a.nzh, n), 8 * RegFft<N>::T, I::template reg_x_smem<N>(), st>>>(a, ga);
    };
    if (I::plan_ct(a.plan[0], 512)) return reg(std::integral_constant<int, 512>{});
    if (I::plan_ct(a.plan[0], 256)) return reg(std::integral_constant<int, 256>{});
    if (I::plan_ct(a.plan[0], 128)) return reg(std::integral_constant<int, 128>{});
    const dim3 g((a.ny + T::kXCols - 1) / T::kXCols, a.nzh, n);
    const size_t sm = I::smem_x(a);
    if (a.fft_threads == kFftThreads && I::plan_ct(a.plan[0], 384))
      k3_fftx_dipolar<R, 384, true><<<g, kFftThreads, sm, st>>>(a, ga);
    else
      k3_fftx_dipolar<R, 0, true><<<g, a.fft_threads, sm, st>>>(a, ga);
  }
  template <typename Co>
  static void k5(const KArgs &a, const KArgs *ga, unsigned n, cudaStream_t st) {
    auto go = [&](auto len) {
      constexpr int N = decltype(len)::value;
      constexpr int bz = ztile_lines<R>(N);
      dim3 g = I::grid_z5(a, bz);
      g.z = n;
      k5_zline<R, Co, kZStep, N, true><<<g, T::kZThreads, I::smem_k5(a, bz), st>>>(a, ga);
    };
    using std::integral_constant;
    if (I::plan_ct(a.plan[2], 512)) go(integral_constant<int, 512>{});
    else if (I::plan_ct(a.plan[2], 384)) go(integral_constant<int, 384>{});
    else if (I::plan_ct(a.plan[2], 256)) go(integral_constant<int, 256>{});
    else if (I::plan_ct(a.plan[2], 128) && a.cn8_tab[2]) go(integral_constant<int, 128>{});
    else if (I::plan_ct(a.plan[2], 96) && a.cn8_tab[2]) go(integral_constant<int, 96>{});
    else if (I::plan_ct(a.plan[2], 64) && a.cn8_tab[2]) go(integral_constant<int, 64>{});
    else go(integral_constant<int, 0>{});
  }
  template <typename Co, int AXIS>
  static void cn(const KArgs &a, const KArgs *ga, unsigned n, int reduce, int renorm, cudaStream_t st) {
    if (I::template cn_short<AXIS, true>(a, ga, n, reduce, renorm, st)) return;
    // one resident wave for the whole group: each member's share of the persistent CTAs,
    // so that every CTA stages the factor tables once for many tiles and prefetches
    dim3 g = I::grid_cn(a, AXIS);
    g.x = g.x / n < 1 ? 1 : g.x / n;
    g.z = n;
    const size_t sm = I::smem_cn(I::cn_len(a, AXIS), a.cn[AXIS].lchunk);
    if (I::cn_full(a, AXIS))
      k_cn<R, Co, AXIS, T::kCnCols, I::template cn_full_threads<AXIS>(), true, true><<<g, I::template cn_full_threads<AXIS>(), sm, st>>>(a, ga, reduce, renorm);
    else
      k_cn<R, Co, AXIS, T::kCnCols, T::kCnThreads, true><<<g, T::kCnThreads, sm, st>>>(a, ga, reduce, renorm);
  }
  static cudaError_t step(const KArgs &a, const KArgs *ga, int count, int renorm, cudaStream_t st) {
    if (count < 1 || count > 65535) return cudaErrorInvalidValue;
    const unsigned n = (unsigned)count;
    {
      auto go = [&](auto len) {
        constexpr int N = decltype(len)::value;
        constexpr int bz = ztile_lines<R>(N);
        dim3 g = I::grid_z5(a, bz);
        g.z = n;
        k1_density_r2cz<R, N, true><<<g, T::kZThreads, I::smem_z_fft(a, bz), st>>>(a, ga);
      };
      using std::integral_constant;
      if (I::plan_ct(a.plan[2], 512)) go(integral_constant<int, 512>{});
      else if (I::plan_ct(a.plan[2], 384)) go(integral_constant<int, 384>{});
      else if (I::plan_ct(a.plan[2], 256)) go(integral_constant<int, 256>{});
      else if (I::plan_ct(a.plan[2], 128)) go(integral_constant<int, 128>{});
      else if (I::plan_ct(a.plan[2], 96)) go(integral_constant<int, 96>{});
      else if (I::plan_ct(a.plan[2], 64)) go(integral_constant<int, 64>{});
      else go(integral_constant<int, 0>{});
    }
    ffty<-1>(a, ga, n, st);
    k3(a, ga, n, st);
    ffty<+1>(a, ga, n, st);
    if (a.imag) {
      k5<R>(a, ga, n, st);
      cn<R, 1>(a, ga, n, 0, 0, st);
      cn<R, 0>(a, ga, n, 1, renorm, st);
    } else {
      k5<C>(a, ga, n, st);
      cn<C, 1>(a, ga, n, 0, 0, st);
      cn<C, 0>(a, ga, n, 1, renorm, st);
    }
    return cudaGetLastError();
  }
};

}  // namespace dgpe
