// Element types of the Krylov basis and their arithmetic.
//
//   double  FP64 storage and FP64 arithmetic (DFMA).
//   float   FP32 storage; SpMV and updates in FP32 with FP32 accumulation;
//           dot products of FP32 vectors summed in FP32 over chunks of four
//           products and accumulated across chunks as float pairs.
//   df32    "float pair": x = hi + lo with |lo| <= ulp(hi)/2, 8 bytes, about
//           48 significant bits.  Every product and sum runs on the FP32 pipe
//           through error-free transforms: TwoProduct by FMA (x*y = p + e
//           exactly) and Knuth's TwoSum (a + b = s + t exactly).  On GB300 the
//           FP64 pipe issues about 2 FMA/clk/SM against about 128 FP32 FMA/clk/SM,
//           so this keeps FP64-class accuracy without the FP64 pipe.
#pragma once
#include <cuda_runtime.h>

struct df32 {
  float hi, lo;
};

// ---- error-free transforms --------------------------------------------------------
__device__ __forceinline__ void ef_two_sum(float a, float b, float& s, float& t) {
  s = a + b;
  const float z = s - a;
  t = (a - (s - z)) + (b - z);
}
__device__ __forceinline__ void ef_fast_two_sum(float a, float b, float& s, float& t) {   // |a| >= |b|
  s = a + b;
  t = b - (s - a);
}

struct F2Acc {   // running sum as an unevaluated float pair
  float hi, lo;
};
__device__ __forceinline__ F2Acc f2_zero() { F2Acc a; a.hi = 0.f; a.lo = 0.f; return a; }
__device__ __forceinline__ double f2_value(const F2Acc& a) { return (double)a.hi + (double)a.lo; }
// a += x*y for FP32 x, y (the product is exact as p + e)
__device__ __forceinline__ void f2_add_prod(F2Acc& a, float x, float y) {
  const float p = x * y;
  const float e = fmaf(x, y, -p);
  float s, t;
  ef_two_sum(a.hi, p, s, t);
  a.lo += t + e;
  a.hi = s;
}
// a += x*y for float pairs (the lo*lo term, about 2^-48 relative, is dropped)
__device__ __forceinline__ void f2_add_prod(F2Acc& a, df32 x, df32 y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  float s, t;
  ef_two_sum(a.hi, p, s, t);
  a.lo += t + e;
  a.hi = s;
}
// a += q for an FP32 value q (TwoSum of the high parts)
__device__ __forceinline__ void f2_add_float(F2Acc& a, float q) {
  float s, t;
  ef_two_sum(a.hi, q, s, t);
  a.lo += t;
  a.hi = s;
}
__device__ __forceinline__ df32 f2_round(const F2Acc& a) {
  df32 r;
  ef_two_sum(a.hi, a.lo, r.hi, r.lo);
  return r;
}
// Partial sums are combined across lanes, warps and CTAs as normalised float pairs
// (for the FP32 and float-pair bases): on GB300 every FP64 warp instruction holds the
// FP64 pipe for about 64 cycles however few lanes are active, so FP64 shuffle-adds
// would dominate a reduction tree.  f2_add is Dekker's pair addition (TwoSum of the
// high parts, the low parts added to the error, renormalised by TwoSum); it is exact
// up to about 2^-47 of |a| + |b| and commutative bit for bit.
__device__ __forceinline__ F2Acc f2_norm(const F2Acc& a) {
  F2Acc r;
  ef_two_sum(a.hi, a.lo, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ F2Acc f2_add(const F2Acc& a, const F2Acc& b) {
  float s, e;
  ef_two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  F2Acc r;
  ef_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ F2Acc f2_split(double x) {   // x to about 48 bits
  F2Acc r;
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ df32 df_from_d(double x) {
  df32 r;
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ double df_to_d(df32 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df32 df_sub(df32 a, df32 b) {
  float s, t;
  ef_two_sum(a.hi, -b.hi, s, t);
  t += a.lo - b.lo;
  df32 r;
  ef_two_sum(s, t, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  df32 r;
  ef_fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// ---- traits -------------------------------------------------------------------------
// kind: 0 FP64, 1 FP32 basis, 2 float-pair basis (FP64 mode)
template <class S> struct Elem;

template <> struct Elem<double> {
  static constexpr int kind = 0;
  typedef double Acc;   // dot accumulator
  typedef double Red;   // partial sum as combined across lanes, warps and CTAs
  typedef double Coef;  // Gram-Schmidt coefficient as used in updates
  __device__ static __forceinline__ Acc zero() { return 0.0; }
  __device__ static __forceinline__ Red red_of(const Acc& a, const Acc& b) { return a + b; }
  __device__ static __forceinline__ Red red_add(const Red& a, const Red& b) { return a + b; }
  __device__ static __forceinline__ Red red_zero() { return 0.0; }
  __device__ static __forceinline__ double red_val(const Red& a) { return a; }
  __device__ static __forceinline__ void dot(Acc& a, double x, double y) { a = fma(x, y, a); }
  __device__ static __forceinline__ void dot4(Acc& a, const double* x, const double* y) {
#pragma unroll
    for (int k = 0; k < 4; ++k) a = fma(x[k], y[k], a);
  }
  __device__ static __forceinline__ double val(const Acc& a) { return a; }
  __device__ static __forceinline__ double from_d(double x) { return x; }
  __device__ static __forceinline__ double to_d(double x) { return x; }
  __device__ static __forceinline__ Coef coef(double c) { return c; }
  __device__ static __forceinline__ double scale(double x, Coef s) { return x * s; }
  __device__ static __forceinline__ double zero_elem() { return 0.0; }
};

template <> struct Elem<float> {
  static constexpr int kind = 1;
  typedef F2Acc Acc;
  typedef F2Acc Red;
  typedef float Coef;
  __device__ static __forceinline__ Acc zero() { return f2_zero(); }
  __device__ static __forceinline__ Red red_of(const Acc& a, const Acc& b) { return f2_add(f2_norm(a), f2_norm(b)); }
  __device__ static __forceinline__ Red red_add(const Red& a, const Red& b) { return f2_add(a, b); }
  __device__ static __forceinline__ Red red_zero() { return f2_zero(); }
  __device__ static __forceinline__ double red_val(const Red& a) { return f2_value(a); }
  __device__ static __forceinline__ void dot(Acc& a, float x, float y) { f2_add_prod(a, x, y); }
  // four products summed by an FP32 multiply-add chain, the chunk added to the float
  // pair by TwoSum: the sum is exact to about 4 u32 of sum |x_k y_k| (Higham's bound for
  // recursive summation), the size of the FP32 basis's own rounding, at a quarter of the
  // FP32 instructions of four exact products
  __device__ static __forceinline__ void dot4(Acc& a, const float* x, const float* y) {
    float q = x[0] * y[0];
    q = fmaf(x[1], y[1], q);
    q = fmaf(x[2], y[2], q);
    q = fmaf(x[3], y[3], q);
    f2_add_float(a, q);
  }
  __device__ static __forceinline__ double val(const Acc& a) { return f2_value(a); }
  __device__ static __forceinline__ float from_d(double x) { return (float)x; }
  __device__ static __forceinline__ double to_d(float x) { return (double)x; }
  __device__ static __forceinline__ Coef coef(double c) { return (float)c; }
  __device__ static __forceinline__ float scale(float x, Coef s) { return x * s; }
  __device__ static __forceinline__ float zero_elem() { return 0.f; }
};

template <> struct Elem<df32> {
  static constexpr int kind = 2;
  typedef F2Acc Acc;
  typedef F2Acc Red;
  typedef df32 Coef;
  __device__ static __forceinline__ Acc zero() { return f2_zero(); }
  __device__ static __forceinline__ Red red_of(const Acc& a, const Acc& b) { return f2_add(f2_norm(a), f2_norm(b)); }
  __device__ static __forceinline__ Red red_add(const Red& a, const Red& b) { return f2_add(a, b); }
  __device__ static __forceinline__ Red red_zero() { return f2_zero(); }
  __device__ static __forceinline__ double red_val(const Red& a) { return f2_value(a); }
  __device__ static __forceinline__ void dot(Acc& a, df32 x, df32 y) { f2_add_prod(a, x, y); }
  __device__ static __forceinline__ void dot4(Acc& a, const df32* x, const df32* y) {
#pragma unroll
    for (int k = 0; k < 4; ++k) f2_add_prod(a, x[k], y[k]);
  }
  __device__ static __forceinline__ double val(const Acc& a) { return f2_value(a); }
  __device__ static __forceinline__ df32 from_d(double x) { return df_from_d(x); }
  __device__ static __forceinline__ double to_d(df32 x) { return df_to_d(x); }
  __device__ static __forceinline__ Coef coef(double c) { return df_from_d(c); }
  __device__ static __forceinline__ df32 scale(df32 x, Coef s) { return df_mul(x, s); }
  __device__ static __forceinline__ df32 zero_elem() { df32 z; z.hi = 0.f; z.lo = 0.f; return z; }
};

// Four consecutive elements moved with 16-byte accesses (addresses 16-byte aligned).
template <class S> struct Quad;
template <> struct Quad<float> {
  float x[4];
  __device__ __forceinline__ void load(const float* p) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
  }
  __device__ __forceinline__ void load_cg(const float* p) {   // through L2 (data other SMs wrote)
    const float4 q = __ldcg(reinterpret_cast<const float4*>(p));
    x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
  }
  __device__ __forceinline__ void store(float* p) const {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  }
};
template <> struct Quad<double> {
  double x[4];
  __device__ __forceinline__ void load(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  }
  __device__ __forceinline__ void load_cg(const double* p) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p)), b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  }
  __device__ __forceinline__ void store(double* p) const {
    reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
  }
};
template <> struct Quad<df32> {
  df32 x[4];
  __device__ __forceinline__ void load(const df32* p) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    x[0].hi = a.x; x[0].lo = a.y; x[1].hi = a.z; x[1].lo = a.w;
    x[2].hi = b.x; x[2].lo = b.y; x[3].hi = b.z; x[3].lo = b.w;
  }
  __device__ __forceinline__ void load_cg(const df32* p) {
    const float4 a = __ldcg(reinterpret_cast<const float4*>(p)), b = __ldcg(reinterpret_cast<const float4*>(p) + 1);
    x[0].hi = a.x; x[0].lo = a.y; x[1].hi = a.z; x[1].lo = a.w;
    x[2].hi = b.x; x[2].lo = b.y; x[3].hi = b.z; x[3].lo = b.w;
  }
  __device__ __forceinline__ void store(df32* p) const {
    reinterpret_cast<float4*>(p)[0] = make_float4(x[0].hi, x[0].lo, x[1].hi, x[1].lo);
    reinterpret_cast<float4*>(p)[1] = make_float4(x[2].hi, x[2].lo, x[3].hi, x[3].lo);
  }
};
