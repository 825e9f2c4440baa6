// Arithmetic policies of the tile kernels.
//
//   PREC_F64: native FP64.
//   PREC_DD : "double-float" -- a value is the unevaluated sum hi + lo of two
//             FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits,
//             computed on the FP32 pipes with the error-free transformations
//             TwoSum (Knuth), FastTwoSum (Dekker) and the FMA-based TwoProduct;
//             every operation below uses the non-contracting round-to-nearest
//             intrinsics so the compiler cannot fuse or reorder the
//             compensation terms.
//   PREC_F32: plain FP32 (inner solver of the defect-correction form).
//
// Accumulations of products (the 1D contractions and the inner products) keep
// an unnormalised pair (s, t): s collects the rounded leading parts by TwoSum,
// t the exact rounding errors and the cross terms; one FastTwoSum normalises.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace mfcg {

//   PREC_F64TC: FP64 like PREC_F64 (every stored value, update and inner
//             product in FP64), with the contractions of the Cartesian cell
//             operator on the FP16 tensor cores by an exact 8-bit digit split
//             of 64-bit fixed-point data (tc_operator.cuh); only the affine
//             operator passes and the fused CG iterations use it.
enum Prec { PREC_F64 = 0, PREC_DD = 1, PREC_F32 = 2, PREC_F64TC = 3 };

// FP64 arithmetic in the vector work (PREC_F64 and PREC_F64TC)
__host__ __device__ constexpr bool is_f64(int prec) { return prec == PREC_F64 || prec == PREC_F64TC; }

// bytes of one stored value
inline size_t prec_bytes(int prec) { return prec == PREC_F32 ? 4 : 8; }

struct __align__(8) dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| or a = 0
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s, e);
}

__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, {-b.hi, -b.lo}); }

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

struct dd_acc {
  float s, t;
};

// a = x * y
__device__ __forceinline__ void acc_set(dd_acc& a, dd x, dd y) {
  a.s = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -a.s);
  e = __fmaf_rn(x.hi, y.lo, e);
  a.t = __fmaf_rn(x.lo, y.hi, e);
}

// a += x * y
__device__ __forceinline__ void acc_madd(dd_acc& a, dd x, dd y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  float s, err;
  two_sum(a.s, p, s, err);
  a.s = s;
  a.t = __fadd_rn(a.t, __fadd_rn(err, e));
}

// a += x
__device__ __forceinline__ void acc_add(dd_acc& a, dd x) {
  float s, err;
  two_sum(a.s, x.hi, s, err);
  a.s = s;
  a.t = __fadd_rn(a.t, __fadd_rn(err, x.lo));
}

__device__ __forceinline__ dd acc_get(const dd_acc& a) { return fast_two_sum(a.s, a.t); }

__device__ __forceinline__ double acc_to_double(const dd_acc& a) { return (double)a.s + (double)a.t; }

// ------------------------------------------------------------------------------------
// policy
// ------------------------------------------------------------------------------------
template <int PREC>
struct Num;
template <>
struct Num<PREC_F64> {
  using T = double;
};
template <>
struct Num<PREC_DD> {
  using T = dd;
};
template <>
struct Num<PREC_F32> {
  using T = float;
};
template <>
struct Num<PREC_F64TC> {
  using T = double;
};

template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T t_zero() {
  if constexpr (PREC == PREC_DD)
    return dd{0.f, 0.f};
  else
    return typename Num<PREC>::T(0);
}

template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T t_from_double(double x) {
  if constexpr (PREC == PREC_DD)
    return dd_from_double(x);
  else
    return (typename Num<PREC>::T)x;
}

template <int PREC>
__device__ __forceinline__ double t_to_double(typename Num<PREC>::T x) {
  if constexpr (PREC == PREC_DD)
    return dd_to_double(x);
  else
    return (double)x;
}

template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T t_add(typename Num<PREC>::T a, typename Num<PREC>::T b) {
  if constexpr (PREC == PREC_DD)
    return dd_add(a, b);
  else
    return a + b;
}

template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T t_sub(typename Num<PREC>::T a, typename Num<PREC>::T b) {
  if constexpr (PREC == PREC_DD)
    return dd_sub(a, b);
  else
    return a - b;
}

template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T t_neg(typename Num<PREC>::T a) {
  if constexpr (PREC == PREC_DD)
    return dd{-a.hi, -a.lo};
  else
    return -a;
}

template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T t_mul(typename Num<PREC>::T a, typename Num<PREC>::T b) {
  if constexpr (PREC == PREC_DD)
    return dd_mul(a, b);
  else
    return a * b;
}

// a * x + b * y
template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T t_axby(typename Num<PREC>::T a, typename Num<PREC>::T x,
                                                       typename Num<PREC>::T b, typename Num<PREC>::T y) {
  if constexpr (PREC == PREC_DD) {
    dd_acc s;
    acc_set(s, a, x);
    acc_madd(s, b, y);
    return acc_get(s);
  } else {
    return fma(a, x, b * y);
  }
}

// a * x + y
template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T t_axpy(typename Num<PREC>::T a, typename Num<PREC>::T x,
                                                       typename Num<PREC>::T y) {
  if constexpr (PREC == PREC_DD) {
    dd_acc s;
    acc_set(s, a, x);
    acc_add(s, y);
    return acc_get(s);
  } else {
    return fma(a, x, y);
  }
}

// Per-thread accumulator of inner products: FP64 for PREC_F64, a double-float
// pair for PREC_DD, FP32 for PREC_F32 (the per-CTA and grid stages are FP64).
template <int PREC>
struct DotAcc;
template <>
struct DotAcc<PREC_F64> {
  double v = 0.0;
  __device__ void madd(double x, double y) { v = fma(x, y, v); }
  __device__ double get() const { return v; }
};
template <>
struct DotAcc<PREC_F64TC> : DotAcc<PREC_F64> {};
template <>
struct DotAcc<PREC_F32> {
  float v = 0.f;
  __device__ void madd(float x, float y) { v = fmaf(x, y, v); }
  __device__ double get() const { return (double)v; }
};
template <>
struct DotAcc<PREC_DD> {
  dd_acc a{0.f, 0.f};
  __device__ void madd(dd x, dd y) { acc_madd(a, x, y); }
  __device__ double get() const { return acc_to_double(a); }
};

}  // namespace mfcg
