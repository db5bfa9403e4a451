// frmg_dfmath.cuh -- double-float ("float-float") arithmetic, FP64 <-> pair
// conversion with integer operations, and division by invariant integers.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, so the quantities that need
// FP64 accuracy in the mixed-precision outer loop (the fine-grid defect, the
// update u += delta and the convergence test) are carried as unevaluated sums
// of two floats, hi + lo with |lo| <= ulp(hi)/2: about 48 significant bits,
// evaluated on the FP32 pipes.  The building blocks are the error-free
// transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the FMA form of
// Dekker's TwoProduct; every operation below states its error.
#pragma once

#include <cuda_runtime.h>

namespace frmg {

struct df {
  float h, l;
};

// s + e = a + b exactly (Knuth's TwoSum, no ordering requirement).
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker's FastTwoSum).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}

// p + e = a * b exactly (FMA form of Dekker's TwoProduct).
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  return {p, e};
}

// a + b with absolute error about eps^2 (|a| + |b|), eps = 2^-24: enough
// whenever the result is measured against the size of the terms, as a residual is.
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.h, b);
  s.l += a.l;
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.h, b.h);
  p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
  return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.h, b);
  p.l = fmaf(a.l, b, p.l);
  return fast_two_sum(p.h, p.l);
}

// 1/sqrt(a) for a > 0: FP32 estimate refined by one Newton step in double-float
// (the step doubles the number of correct bits).
__device__ __forceinline__ df df_rsqrt(df a) {
  float y = rsqrtf(a.h);
  // y' = y + y (1 - a y^2) / 2
  df y2 = two_prod(y, y);
  df ay2 = df_mul(a, y2);
  df r = df_add_f(df_neg(ay2), 1.0f);
  return df_add_f({0.5f * y * r.h, 0.0f}, y);
}

// e^u for u = (h, l) (|u| < 80): u = n ln2 + r, e^r from its Taylor series at
// r/16 (degree 7, truncation below 1e-17 relative) squared four times, scaled
// by 2^n.  ln2 enters as the double-float pair (ln2h, ln2l) supplied by the host.
__device__ __forceinline__ df df_exp(df u, float ln2h, float ln2l) {
  float n = rintf(u.h * 1.44269504f);  // nearest integer to u / ln2
  df nl = df_add(two_prod(n, ln2h), two_prod(n, ln2l));
  df r = df_sub(u, nl);
  r.h *= 0.0625f;  // exact scaling by 2^-4
  r.l *= 0.0625f;
  // Horner: 1 + r (1 + r/2 (1 + r/3 (... (1 + r/7))))
  df t = {1.0f, 0.0f};
#pragma unroll
  for (int k = 7; k >= 1; k--) {
    t = df_mul(t, r);
    // t = 1 + t / k: q = t.h (1/k) rounded, then the remainder t - q k (exact
    // by FMA) divided by k gives the low part (two-step division by a float)
    const float rk = 1.0f / (float)k;  // a constant after unrolling
    const float q = t.h * rk;
    const float rem = fmaf(-q, (float)k, t.h) + t.l;
    df tq = {q, rem * rk};
    t = df_add_f(tq, 1.0f);
  }
  for (int k = 0; k < 4; k++) t = df_mul(t, t);
  int ni = (int)n;
  return {ldexpf(t.h, ni), ldexpf(t.l, ni)};
}

// ---- the same arithmetic on two independent values at once ----
// Blackwell's packed FP32 instructions (PTX add/sub/fma .rn.f32x2) round each
// lane to nearest exactly as the scalar instruction does, so the error-free
// transformations above hold lane by lane.  A float2 here holds one
// quantity of two cells (lane x: the first cell, lane y: the second).
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// Products stay per lane (mul.rn.f32): with the packed multiply, a product
// followed by packed sums did not reproduce the scalar error-free
// transformations lane by lane (measured: two_prod's error term and the sums
// built on it came out different, and less accurate, in kernels; alone, the
// same sequence agreed), while per-lane products under the packed sums agree
// bit for bit with the scalar sequence.
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pc, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "mov.b64 pc, {%6, %7};\n\tfma.rn.f32x2 pr, pa, pb, pc;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

// a double-float value of two cells: hi and lo lanes
struct df2 {
  float2 h, l;
};

__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  const float2 bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}
// p + e = a b: the error term as fma(a, b, -p), -p formed as 0 - p
__device__ __forceinline__ df2 two_prod2(float2 a, float2 b) {
  const float2 p = mul2(a, b);
  return {p, fma2(a, b, sub2(splat2(0.0f), p))};
}
__device__ __forceinline__ df2 df_add2(df2 a, df2 b) {
  df2 s = two_sum2(a.h, b.h);
  s.l = add2(s.l, add2(a.l, b.l));
  return fast_two_sum2(s.h, s.l);
}
__device__ __forceinline__ df2 df_sub2(df2 a, df2 b) {
  // a + (-b): the two sums of df_add with b's lanes negated, as subtractions
  const float2 s = sub2(a.h, b.h);
  const float2 bb = sub2(s, a.h);
  float2 e = sub2(sub2(a.h, sub2(s, bb)), add2(b.h, bb));
  e = add2(e, sub2(a.l, b.l));
  return fast_two_sum2(s, e);
}
__device__ __forceinline__ df2 df_add_f2(df2 a, float b) {
  df2 s = two_sum2(a.h, splat2(b));
  s.l = add2(s.l, a.l);
  return fast_two_sum2(s.h, s.l);
}
__device__ __forceinline__ df2 df_mul2(df2 a, df2 b) {
  df2 p = two_prod2(a.h, b.h);
  p.l = fma2(a.h, b.l, fma2(a.l, b.h, p.l));
  return fast_two_sum2(p.h, p.l);
}
// u_j - u_i of two cells' faces (df_diff lane by lane)
__device__ __forceinline__ df2 df_diff2(df2 ui, df2 uj) {
  const float2 s = sub2(uj.h, ui.h);
  const float2 bb = sub2(s, uj.h);
  float2 e = sub2(sub2(uj.h, sub2(s, bb)), add2(ui.h, bb));
  e = add2(e, sub2(uj.l, ui.l));
  return fast_two_sum2(s, e);
}
// df_rsqrt lane by lane: the FP32 estimate per lane, the Newton step packed
__device__ __forceinline__ df2 df_rsqrt2(df2 a) {
  const float2 y = make_float2(rsqrtf(a.h.x), rsqrtf(a.h.y));
  const df2 y2 = two_prod2(y, y);
  const df2 ay2 = df_mul2(a, y2);
  // r = 1 - a y^2
  df2 r = two_sum2(splat2(1.0f), sub2(splat2(0.0f), ay2.h));
  r.l = sub2(r.l, ay2.l);
  r = fast_two_sum2(r.h, r.l);
  // y + (y / 2) r
  const float2 c = mul2(mul2(splat2(0.5f), y), r.h);
  const df2 t = two_sum2(c, y);
  return fast_two_sum2(t.h, t.l);
}

// n / d for 0 <= n < 2^31, 1 <= d < 2^31, by one widening multiply and a
// shift (division by an invariant integer, Granlund and Montgomery 1994):
// with l = ceil(log2 d), p = 31 + l and m = ceil(2^p / d) (< 2^32),
// m = 2^p / d + e with 0 <= e < 1, so n m / 2^p = n / d + n e / 2^p where
// n e / 2^p < 2^-l <= 1 / d: the floor is that of n / d.
struct FastDiv {
  unsigned m;
  int p;
};

inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) l++;
  const int p = 31 + l;
  const unsigned long long num = 1ull << p;
  return {(unsigned)((num + d - 1) / d), p};
}

__device__ __forceinline__ unsigned fdiv(unsigned n, FastDiv f) {
  return (unsigned)(((unsigned long long)n * f.m) >> f.p);
}

// Splits an FP64 value into a double-float pair through the FP64 pipe.
__device__ __forceinline__ df split_d(double v) {
  float h = (float)v;
  return {h, (float)(v - (double)h)};
}

// The same split with integer operations (the FP64 pipe is narrow): the
// 53-bit significand m of v = +-m 2^(e-1075) is rounded to its top 24 bits
// h (hi = h 2^(e-1046)) and the remainder r = m - h 2^29 (|r| <= 2^28) gives
// lo = r 2^(e-1075), rounded to 24 bits.  Values outside 2^-70 <= |v| < 2^100
// (zero, tiny, huge, non-finite) take the FP64 route.
__device__ __forceinline__ df split_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ffu);
  if (e < 1023 - 70 || e >= 1023 + 100) return split_d(v);
  const unsigned sgn = (unsigned)(b >> 63) << 31;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned long long h = (m + (1ull << 28)) >> 29;
  const int r = (int)((long long)m - (long long)(h << 29));
  int eh = e - 1023;
  if (h == (1ull << 24)) {
    h >>= 1;
    eh += 1;
  }
  const float hi = __uint_as_float(sgn | ((unsigned)(eh + 127) << 23) | ((unsigned)h & 0x7fffffu));
  const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);  // 2^(e-1075), exact
  const float lo = __uint_as_float(__float_as_uint((float)r * scale) ^ sgn);
  return {hi, lo};
}

// hi + lo as an FP64 value with integer operations: the significands are
// aligned (|lo| <= ulp(hi) / 2, so lo sits at least 24 binary places below
// hi), added as integers and renormalised; rounding is to nearest at the last
// step only.  Pairs with hi outside 2^-70 <= |hi| < 2^100 use FP64 arithmetic.
__device__ __forceinline__ double join_bits(float hi, float lo) {
  const unsigned hb = __float_as_uint(hi), lb = __float_as_uint(lo);
  const int eh = (int)((hb >> 23) & 0xffu), el = (int)((lb >> 23) & 0xffu);
  const bool lzero = (lb << 1) == 0;
  if (eh < 127 - 70 || eh >= 127 + 100 || (!lzero && (el == 0 || eh - el < 24)))
    return (double)hi + (double)lo;
  // significands: hi at bit 52 of a 64-bit integer (scaled 2^29), lo below it
  long long M = (long long)((hb & 0x7fffffu) | 0x800000u) << 29;
  const long long ml = (long long)((lb & 0x7fffffu) | 0x800000u);
  const int d = eh - el;  // >= 24
  long long L;
  if (lzero) {
    L = 0;
  } else if (d <= 29) {
    L = ml << (29 - d);
  } else if (d < 64) {
    const int sh = d - 29;
    L = (ml + (1ll << (sh - 1))) >> sh;
  } else {
    L = 0;
  }
  M = ((hb ^ lb) >> 31) ? M - L : M + L;
  int E = eh - 127 + 1023;
  if (M >= (1ll << 53)) {
    M = (M + 1) >> 1;
    E += 1;
  } else if (M < (1ll << 52)) {
    M <<= 1;
    E -= 1;
  }
  const unsigned long long bits = ((unsigned long long)(hb >> 31) << 63) |
                                  ((unsigned long long)E << 52) |
                                  ((unsigned long long)M & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

}  // namespace frmg
