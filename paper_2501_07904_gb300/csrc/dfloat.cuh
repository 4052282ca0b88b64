// Double-float arithmetic: a value carried as an unevaluated sum h + l of two
// FP32 words (|l| <= ulp(h) / 2), about 48 significant bits, computed with
// FP32 instructions only.  GB300 issues FP64 at 1/64 of its FP32 rate, so a
// factorization that needs more than FP32 but far less than FP64's 53 bits
// (the tight steps' small factors: tails resolved to ~1e-10 of the trace)
// runs several times faster in this form.
//
// Building blocks (error-free transformations):
//   two_sum   Knuth's TwoSum: s + e = a + b exactly, any magnitudes;
//   fast_two_sum  Dekker's Fast2Sum: the same when |a| >= |b| (or a = 0);
//   two_prod  p + e = a b exactly, e by one fused multiply-add.
// Compound operations follow Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic" (ACM TOMS
// 2017): the accurate sum of two double-words (their AccurateDWPlusDW) and
// the product DWTimesDW; fma_df fuses a product and a sum with the high parts
// added by TwoSum, so its error stays ~u^2 (|a b| + |c|) under cancellation
// (u = 2^-24).  The reciprocal square root refines the FP32 estimate by one
// Newton step x (3 - a x^2) / 2 carried out in double-float.
//
// On the device the FP32 operations are the _rn intrinsics, which the
// compiler never contracts into fused multiply-adds; host code (the unit
// tests) must be compiled with -ffp-contract=off.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace ttk {

#if defined(__CUDA_ARCH__)
DF_HD float df_add_(float a, float b) { return __fadd_rn(a, b); }
DF_HD float df_sub_(float a, float b) { return __fsub_rn(a, b); }
DF_HD float df_mul_(float a, float b) { return __fmul_rn(a, b); }
DF_HD float df_fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
DF_HD float df_add_(float a, float b) { return a + b; }
DF_HD float df_sub_(float a, float b) { return a - b; }
DF_HD float df_mul_(float a, float b) { return a * b; }
DF_HD float df_fma_(float a, float b, float c) { return fmaf(a, b, c); }
#endif

struct df32 {
  float h, l;
  df32() = default;
  DF_HD constexpr df32(float x) : h(x), l(0.f) {}
  DF_HD constexpr df32(int x) : h((float)x), l(0.f) {}
  DF_HD constexpr df32(float hi, float lo) : h(hi), l(lo) {}
  // nearest double-float to x (its high word, then the rounded remainder)
  DF_HD df32(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
  DF_HD explicit operator double() const { return (double)h + (double)l; }
  DF_HD explicit operator float() const { return df_add_(h, l); }
};

DF_HD void two_sum(float a, float b, float& s, float& e) {
  s = df_add_(a, b);
  const float bv = df_sub_(s, a);
  e = df_add_(df_sub_(a, df_sub_(s, bv)), df_sub_(b, bv));
}
DF_HD void fast_two_sum(float a, float b, float& s, float& e) {
  s = df_add_(a, b);
  e = df_sub_(b, df_sub_(s, a));
}
DF_HD void two_prod(float a, float b, float& p, float& e) {
  p = df_mul_(a, b);
  e = df_fma_(a, b, -p);
}

DF_HD df32 operator-(df32 a) { return df32(-a.h, -a.l); }

DF_HD df32 operator+(df32 a, df32 b) {
  float sh, sl, th, tl, vh, vl, zh, zl;
  two_sum(a.h, b.h, sh, sl);
  two_sum(a.l, b.l, th, tl);
  fast_two_sum(sh, df_add_(sl, th), vh, vl);
  fast_two_sum(vh, df_add_(tl, vl), zh, zl);
  return df32(zh, zl);
}
DF_HD df32 operator-(df32 a, df32 b) { return a + (-b); }

DF_HD df32 operator*(df32 a, df32 b) {
  float ch, cl;
  two_prod(a.h, b.h, ch, cl);
  const float t = df_fma_(a.h, b.l, df_mul_(a.l, b.h));
  float zh, zl;
  fast_two_sum(ch, df_add_(cl, t), zh, zl);
  return df32(zh, zl);
}

// a b + c
DF_HD df32 fma_df(df32 a, df32 b, df32 c) {
  float ph, pe, sh, se;
  two_prod(a.h, b.h, ph, pe);
  two_sum(ph, c.h, sh, se);
  // low-order terms: the product's error, the cross products, c's low word
  float t = df_add_(pe, c.l);
  t = df_fma_(a.h, b.l, t);
  t = df_fma_(a.l, b.h, t);
  float zh, zl;
  fast_two_sum(sh, df_add_(se, t), zh, zl);
  return df32(zh, zl);
}

DF_HD df32& operator+=(df32& a, df32 b) { return a = a + b; }
DF_HD df32& operator-=(df32& a, df32 b) { return a = a - b; }

DF_HD bool operator>(df32 a, df32 b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }
DF_HD bool operator<(df32 a, df32 b) { return b > a; }
DF_HD bool operator<=(df32 a, df32 b) { return !(a > b); }
DF_HD bool operator>=(df32 a, df32 b) { return !(b > a); }
DF_HD bool operator==(df32 a, df32 b) { return a.h == b.h && a.l == b.l; }
DF_HD bool operator!=(df32 a, df32 b) { return !(a == b); }

DF_HD df32 fmax_df(df32 a, df32 b) { return (b > a) ? b : a; }

// 1 / sqrt(a) for a > 0: x0 ~ 1/sqrt(a.h) in FP32, then one Newton step
// x0 + x0 (1 - a x0^2) / 2 with the residual in double-float (quadratic
// convergence: ~2^-44 from an estimate good to a few ulp of FP32).
DF_HD df32 rsqrt_df(df32 a, float x0) {
  const df32 x(x0);
  const df32 r = df32(1.0f) - a * (x * x);
  return fma_df(x, df32(df_mul_(0.5f, r.h), df_mul_(0.5f, r.l)), x);
}

}  // namespace ttk
