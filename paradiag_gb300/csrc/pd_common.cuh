// Shared device helpers for the ParaDiag-II kernels: complex arithmetic in
// FP32/FP64, double-float ("df") arithmetic on pairs of FP32 numbers, and the
// conversions between FP64 storage and df registers done with integer
// operations (on GB300 the FP64 pipe, which also performs FP64<->FP32
// conversions, runs at about 1/70 of the FP32 rate, so the mixed path keeps
// FP64 instructions off its inner loops).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#define PD_HD __host__ __device__ __forceinline__
#define PD_D __device__ __forceinline__

// ----------------------------------------------------------------------------
// complex helpers (float2 / double2), templated on the real type
// ----------------------------------------------------------------------------
template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename R> using cplx_t = typename cplx_of<R>::type;

PD_HD float2 mk(float a, float b) { return make_float2(a, b); }
PD_HD double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> PD_HD C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> PD_HD C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> PD_HD C cmul(C a, C b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> PD_HD C cconj(C a) { return mk(a.x, -a.y); }
template <typename C, typename R> PD_HD C cscale(C a, R s) { return mk(a.x * s, a.y * s); }
// a * conj(b)
template <typename C> PD_HD C cmulc(C a, C b) { return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
// multiply by -i / +i
template <typename C> PD_HD C cmul_mi(C a) { return mk(a.y, -a.x); }
template <typename C> PD_HD C cmul_pi(C a) { return mk(-a.y, a.x); }

PD_D float2 crcp(float2 a) {
  float s = __frcp_rn(fmaf(a.x, a.x, a.y * a.y));
  return make_float2(a.x * s, -a.y * s);
}
PD_D double2 crcp(double2 a) {
  double s = 1.0 / fma(a.x, a.x, a.y * a.y);
  return make_double2(a.x * s, -a.y * s);
}

template <typename C> PD_HD C czero() { C z; z.x = 0; z.y = 0; return z; }

// ----------------------------------------------------------------------------
// double-float arithmetic (value = hi + lo, |lo| <= ulp(hi)/2).
// Error-free transformations: Knuth's two-sum, Dekker's fast-two-sum and the
// FMA-based two-product.
// ----------------------------------------------------------------------------
struct df { float hi, lo; };

PD_D df df_make(float h, float l) { df r; r.hi = h; r.lo = l; return r; }
PD_D df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}
PD_D df fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}
PD_D df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  float e = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, e);
  e = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, e);
}
PD_D df df_neg(df a) { return df_make(-a.hi, -a.lo); }
PD_D df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
PD_D df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
PD_D df df_scale2(df a, float pow2) { return df_make(a.hi * pow2, a.lo * pow2); }

// The same compensated arithmetic on two independent values at once (the
// lanes of a float2), with the paired FP32 instructions of sm_100+.
PD_D float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
PD_D float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
PD_D float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
PD_D float2 f2sub(float2 a, float2 b) {
  unsigned long long x = *reinterpret_cast<unsigned long long*>(&a);
  unsigned long long y = *reinterpret_cast<unsigned long long*>(&b);
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
  return *reinterpret_cast<float2*>(&d);
}
struct DF2 {    // two double-float values: (hi_A, hi_B), (lo_A, lo_B)
  float2 hi, lo;
};
struct Acc2 {   // two compensated sums
  float2 s, e;
};
PD_D DF2 df2_pack(float2 a, float2 b) { return DF2{make_float2(a.x, b.x), make_float2(a.y, b.y)}; }
// A += h + l (two-sum on the high parts)
PD_D void acc2_add(Acc2& A, float2 h, float2 l) {
  const float2 t = f2add(A.s, h);
  const float2 bb = f2sub(t, A.s);
  const float2 err = f2add(f2sub(A.s, f2sub(t, bb)), f2sub(h, bb));
  A.s = t;
  A.e = f2add(A.e, f2add(err, l));
}
// A -= h + l
PD_D void acc2_sub(Acc2& A, float2 h, float2 l) {
  const float2 t = f2sub(A.s, h);
  const float2 bb = f2sub(t, A.s);
  const float2 err = f2sub(f2sub(A.s, f2sub(t, bb)), f2add(h, bb));
  A.s = t;
  A.e = f2sub(f2add(A.e, err), l);
}
// coefficient k = kh + kl broadcast to both lanes, with its negation
struct K2 {
  float2 h, nh, nl;
};
// A += k u (two-product of the high parts, the cross terms into the error)
PD_D void acc2_add_prod(Acc2& A, const K2& k, const DF2& u) {
  const float2 p = f2mul(u.hi, k.h);
  float2 npe = f2fma(u.hi, k.nh, p);   // p - u.hi k.hi = -(rounding error of p)
  npe = f2fma(u.hi, k.nl, npe);
  npe = f2fma(u.lo, k.nh, npe);
  const float2 t = f2add(A.s, p);
  const float2 bb = f2sub(t, A.s);
  const float2 err = f2add(f2sub(A.s, f2sub(t, bb)), f2sub(p, bb));
  A.s = t;
  A.e = f2sub(f2add(A.e, err), npe);
}

// the sum k u started from nothing: the product and its rounding error
PD_D Acc2 acc2_of_prod(const K2& k, const DF2& u) {
  const float2 p = f2mul(u.hi, k.h);
  float2 npe = f2fma(u.hi, k.nh, p);
  npe = f2fma(u.hi, k.nl, npe);
  npe = f2fma(u.lo, k.nh, npe);
  return Acc2{p, f2mul(npe, make_float2(-1.f, -1.f))};
}

// Split an FP64 value into hi + lo FP32 parts with integer operations only.
// hi keeps the leading 24 significand bits (truncated), lo the next 24 bits
// (rounded by the integer-to-float conversion), so |x - hi - lo| <= 2^-47 |x|.
// Magnitudes below 2^-126 are flushed to zero, the low part is dropped below
// 2^-74 (an absolute error under 2^-97), and magnitudes of 2^128 and more
// (and NaN) become a signed infinity.
PD_D df df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);       // biased FP64 exponent
  const int fe = e - 1023 + 127;                // biased FP32 exponent of hi
  if (fe <= 0) return df_make(0.f, 0.f);
  if (fe >= 255) return df_make(__uint_as_float(sign | 0x7F800000u), 0.f);
  const unsigned int mhi = (unsigned int)((b >> 29) & 0x7FFFFFu);
  const float hi = __uint_as_float(sign | ((unsigned int)fe << 23) | mhi);
  float lo = 0.f;
  if (fe > 52) {
    // the 29 low significand bits have weight 2^(e-1075) = 2^((fe-52)-127)
    const unsigned int mlo = (unsigned int)(b & 0x1FFFFFFFu);
    lo = __uint2float_rn(mlo) * __uint_as_float((unsigned int)(fe - 52) << 23);
    lo = __uint_as_float(__float_as_uint(lo) | sign);
  }
  return df_make(hi, lo);
}

// FP32 value to FP64 bits with integer operations (exact; FP32 subnormals and
// zeros map to a signed zero).
PD_D double double_from_float(float f) {
  unsigned int u = __float_as_uint(f);
  unsigned int sign = u & 0x80000000u;
  unsigned int e = (u >> 23) & 0xFF;
  if (e == 0) return __longlong_as_double((long long)((unsigned long long)sign << 32));
  unsigned long long de = (e == 0xFF) ? 0x7FFull : (unsigned long long)(e - 127 + 1023);
  unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(((unsigned long long)sign << 32) | (de << 52) | m));
}

// ----------------------------------------------------------------------------
// misc
// ----------------------------------------------------------------------------
PD_HD int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
PD_HD bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
PD_HD int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
