// Arithmetic policies of the TSQR kernels.
//
// ArithF64: native IEEE binary64 everywhere.
// ArithDF : "double-float": every value is an unevaluated sum hi + lo of two binary32 numbers
//           (|lo| <= ulp(hi)/2), about 48 significant bits, computed on the FP32 pipe.  On GB300
//           the FP64 pipe issues one warp instruction per ~20 SM cycles while the FP32 pipe
//           issues ~4 per cycle, so a double-float multiply-add of 12-15 FP32 instructions is
//           still several times cheaper than one native FP64 FMA.  The error-free transformations
//           are the published ones: Knuth's TwoSum, Dekker's Fast2Sum (|a| >= |b|) and the
//           FMA-based TwoProduct; sums follow the "sloppy" double-float addition, whose error
//           is bounded relative to |a| + |b|, the model Householder QR's backward-error analysis
//           needs (each operation accurate relative to its operands, unit roundoff ~2^-46).
//           Every FP32 operation is a non-contractible _rn intrinsic so the compiler cannot
//           fuse the steps the transformations rely on.
//           Range: magnitudes within about [2^-100, 2^100] keep full accuracy (FP32 exponent
//           range); sums of squares are taken after a power-of-two rescaling.
//
// ArithF32: IEEE binary32 arithmetic for FP32 storage (A, R, Q and B are float): each value is
//           the hi half of a pair whose lo half stays zero, so that it shares the 8-byte
//           element of the other policies.
//
// All store an element in 8 bytes, so the shared-memory tile layout, the TMA descriptors and
// the workspace are shared; in double-float mode the workspace holds (hi, lo) pairs.  Out is the
// type of the caller's R, Q and B.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tsqr {

struct ArithF64 {
  using E = double;
  using Out = double;
  static constexpr int kPrecision = 0;
  __device__ __forceinline__ static E from_f64(double x) { return x; }
  __device__ __forceinline__ static double to_f64(E x) { return x; }
  __device__ __forceinline__ static E from_out(Out x) { return x; }
  __device__ __forceinline__ static Out to_out(E x) { return x; }
  __device__ __forceinline__ static E zero() { return 0.0; }
  __device__ __forceinline__ static E from_int(int v) { return (double)v; }
  // an accumulated value in its final form (the double-float sums end unnormalised)
  __device__ __forceinline__ static E fin(E x) { return x; }
  // s += a * b
  __device__ __forceinline__ static void fma_acc(E& s, E a, E b) { s = fma(a, b, s); }
  __device__ __forceinline__ static E add(E a, E b) { return a + b; }
  __device__ __forceinline__ static E sub(E a, E b) { return a - b; }
  __device__ __forceinline__ static E mul(E a, E b) { return a * b; }
  __device__ __forceinline__ static E neg(E a) { return -a; }
  // a - w * y
  __device__ __forceinline__ static E axpy(E a, E w, E y) { return fma(-w, y, a); }
  __device__ __forceinline__ static E shfl_xor(E v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
  __device__ __forceinline__ static bool is_zero(E x) { return x == 0.0; }
  __device__ __forceinline__ static bool is_neg(E x) { return x < 0.0; }
};

struct __align__(8) f32x2 {
  float hi, lo;
};

struct ArithDF {
  using E = f32x2;
  using Out = double;
  static constexpr int kPrecision = 1;

  // Knuth TwoSum: a + b = s + e exactly.
  __device__ __forceinline__ static void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }
  // Dekker Fast2Sum, |a| >= |b| (or a == 0): a + b = s + e exactly.
  __device__ __forceinline__ static E fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return E{s, __fsub_rn(b, __fsub_rn(s, a))};
  }
  // hi*hi' exactly plus the cross terms: the unnormalised product (p, e) of two pairs.
  __device__ __forceinline__ static void prod(E a, E b, float& p, float& e) {
    p = __fmul_rn(a.hi, b.hi);
    e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
  }

  __device__ __forceinline__ static E from_f64(double x) {
    const float h = __double2float_rn(x);
    return E{h, __double2float_rn(x - (double)h)};
  }
  __device__ __forceinline__ static double to_f64(E x) { return (double)x.hi + (double)x.lo; }
  __device__ __forceinline__ static E from_out(Out x) { return from_f64(x); }
  __device__ __forceinline__ static Out to_out(E x) { return to_f64(x); }
  __device__ __forceinline__ static E zero() { return E{0.f, 0.f}; }
  __device__ __forceinline__ static E from_int(int v) { return E{(float)v, 0.f}; }
  // s += a * b, with s left unnormalised (hi carries the running TwoSum, lo the errors)
  __device__ __forceinline__ static void fma_acc(E& s, E a, E b) {
    float p, e, t, err;
    prod(a, b, p, e);
    two_sum(s.hi, p, t, err);
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
  }
  __device__ __forceinline__ static E norm(E a) { return fast_two_sum(a.hi, a.lo); }
  __device__ __forceinline__ static E add(E a, E b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
  }
  __device__ __forceinline__ static E neg(E a) { return E{-a.hi, -a.lo}; }
  __device__ __forceinline__ static E sub(E a, E b) { return add(a, neg(b)); }
  __device__ __forceinline__ static E fin(E x) { return add(x, zero()); }
  __device__ __forceinline__ static E mul(E a, E b) {
    float p, e;
    prod(a, b, p, e);
    return fast_two_sum(p, e);
  }
  // a - w * y
  __device__ __forceinline__ static E axpy(E a, E w, E y) {
    float p, e, t, err;
    prod(w, y, p, e);
    two_sum(a.hi, -p, t, err);
    return fast_two_sum(t, __fadd_rn(__fsub_rn(a.lo, e), err));
  }
  __device__ __forceinline__ static E shfl_xor(E v, int o) {
    return E{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
  }
  __device__ __forceinline__ static bool is_zero(E x) { return x.hi == 0.f && x.lo == 0.f; }
  __device__ __forceinline__ static bool is_neg(E x) { return x.hi < 0.f || (x.hi == 0.f && x.lo < 0.f); }

  // sqrt(x) for x > 0: the FP32 root refined by one Newton step, s = s0 + (x - s0^2) / (2 s0).
  __device__ static E sqrt_df(E x) {
    const float s0 = __fsqrt_rn(x.hi);
    float p, e;
    p = __fmul_rn(s0, s0);
    e = __fmaf_rn(s0, s0, -p);
    // r = x - s0^2, small: its leading bits cancel
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), e), x.lo);
    return fast_two_sum(s0, __fdiv_rn(r, __fmul_rn(2.f, s0)));
  }
  // a / b for b != 0: the FP32 quotient plus one correction term from the residual a - q0 b.
  __device__ static E div_df(E a, E b) {
    const float q0 = __fdiv_rn(a.hi, b.hi);
    float p, e, t, err;
    p = __fmul_rn(q0, b.hi);
    e = __fmaf_rn(q0, b.hi, -p);
    e = __fmaf_rn(q0, b.lo, e);
    two_sum(a.hi, -p, t, err);
    const float r = __fadd_rn(t, __fadd_rn(__fsub_rn(a.lo, e), err));
    return fast_two_sum(q0, __fdiv_rn(r, b.hi));
  }
  // x * 2^k exactly (both halves), k chosen so no under/overflow occurs
  __device__ __forceinline__ static E ldexp(E x, int k) {
    const float s = __int_as_float((127 + k) << 23);
    return E{__fmul_rn(x.hi, s), __fmul_rn(x.lo, s)};
  }
};

struct ArithF32 {
  using E = f32x2;  // lo == 0
  using Out = float;
  static constexpr int kPrecision = 16;
  __device__ __forceinline__ static E mk(float v) { return E{v, 0.f}; }
  __device__ __forceinline__ static E from_f64(double x) { return mk(__double2float_rn(x)); }
  __device__ __forceinline__ static double to_f64(E x) { return (double)x.hi; }
  __device__ __forceinline__ static E from_out(Out x) { return mk(x); }
  __device__ __forceinline__ static Out to_out(E x) { return x.hi; }
  __device__ __forceinline__ static E zero() { return mk(0.f); }
  __device__ __forceinline__ static E from_int(int v) { return mk((float)v); }
  __device__ __forceinline__ static E fin(E x) { return x; }
  __device__ __forceinline__ static void fma_acc(E& s, E a, E b) { s.hi = __fmaf_rn(a.hi, b.hi, s.hi); }
  __device__ __forceinline__ static E add(E a, E b) { return mk(__fadd_rn(a.hi, b.hi)); }
  __device__ __forceinline__ static E sub(E a, E b) { return mk(__fsub_rn(a.hi, b.hi)); }
  __device__ __forceinline__ static E mul(E a, E b) { return mk(__fmul_rn(a.hi, b.hi)); }
  __device__ __forceinline__ static E neg(E a) { return mk(-a.hi); }
  // a - w * y
  __device__ __forceinline__ static E axpy(E a, E w, E y) { return mk(__fmaf_rn(-w.hi, y.hi, a.hi)); }
  __device__ __forceinline__ static E shfl_xor(E v, int o) { return mk(__shfl_xor_sync(0xffffffffu, v.hi, o)); }
  __device__ __forceinline__ static bool is_zero(E x) { return x.hi == 0.f; }
  __device__ __forceinline__ static bool is_neg(E x) { return x.hi < 0.f; }
  // x * 2^k exactly, k chosen so no under/overflow occurs
  __device__ __forceinline__ static E ldexp(E x, int k) { return mk(__fmul_rn(x.hi, __int_as_float((127 + k) << 23))); }
};

}  // namespace tsqr
