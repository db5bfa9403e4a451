// frmg_df.cuh -- double-float ("float-float") arithmetic and the FP64-accurate
// fine-grid defect of the mixed-precision loop.
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
// whenever the result is judged against the size of the terms, as a residual is.
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

}  // namespace frmg

namespace frmg {

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

// Fine-grid state of the double-float outer loop of one grid.
struct DFGrid {
  float2 *u;             // u = (hi, lo)
  float2 *B;             // e^u
  float2 *r;             // gamma (rho - 1)
  const double *bnd;     // packed Dirichlet faces (FP64) or null
  long long foff[6];
  long long ncell;
  int n0, n1, n2;
  FastDiv fd0, fd1;      // division by n0 and n1 (grids below 2^31 cells)
  float ahh, ahl;        // alpha / 2
  float beh, bel;        // beta
  float gah, gal;        // gamma
};

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

// State set-up: u (FP64, or zero), e^u and gamma (rho - 1) as double-float.
__global__ void k_df_init(DFGrid G, const double *u64, const double *rho, int zero_u,
                          float ln2h, float ln2l) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  df u = zero_u ? df{0.f, 0.f} : split_bits(u64[t]);
  G.u[t] = make_float2(u.h, u.l);
  df B = zero_u ? df{1.f, 0.f} : df_exp(u, ln2h, ln2l);
  G.B[t] = make_float2(B.h, B.l);
  const df r = df_mul(df_add_f(split_bits(rho[t]), -1.0f), df{G.gah, G.gal});
  G.r[t] = make_float2(r.h, r.l);
}

// u += delta, e^u recomputed from u (no drift across outer steps).
__global__ void k_df_update(DFGrid G, const float *delta, float ln2h, float ln2l) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  const float2 uo = G.u[t];
  df s = two_sum(uo.x, delta[t]);
  s.l += uo.y;
  df u = fast_two_sum(s.h, s.l);
  G.u[t] = make_float2(u.h, u.l);
  df B = df_exp(u, ln2h, ln2l);
  G.B[t] = make_float2(B.h, B.l);
}

__global__ void k_df_final(DFGrid G, double *u64) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  const float2 v = G.u[t];
  u64[t] = join_bits(v.x, v.y);
}

// One face of the double-float operator: (B_i + B_j)(u_j - u_i).
__device__ __forceinline__ df df_face(df ui, df Bi, df uj, df Bj) {
  df dd = two_sum(uj.h, -ui.h);
  dd.l += uj.l - ui.l;
  dd = fast_two_sum(dd.h, dd.l);
  df sB = two_sum(Bi.h, Bj.h);
  sB.l += Bi.l + Bj.l;
  sB = fast_two_sum(sB.h, sB.l);
  return df_mul(sB, dd);
}

// FP64-accurate defect d = A(u) - gamma (rho - 1) of the fine grid in
// double-float, and the set-up of the FP32 correction problem that follows:
// r32 = -d, background ub32 = hi(u) with E32 = e^{ub32}, delta = x = 0.
// Block partials (sum d^2, max |d|) go to partial[2 (base + block)].
template <bool BIG>
__global__ void __launch_bounds__(256)
    k_df_defect(DFGrid G, float *r32, float *ub32, float *E32, float *delta, float *x32,
                double *partial, int base, float ln2h, float ln2l, double *dout = nullptr) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float s2 = 0.0f, mx = 0.0f;
  if (t < G.ncell) {
    int i, j, k;
    if (BIG) {
      i = (int)(t % G.n0);
      const long long rr = t / G.n0;
      j = (int)(rr % G.n1);
      k = (int)(rr / G.n1);
    } else {
      const unsigned tu = (unsigned)t, q = fdiv(tu, G.fd0), q2 = fdiv(q, G.fd1);
      i = (int)(tu - q * (unsigned)G.n0);
      j = (int)(q - q2 * (unsigned)G.n1);
      k = (int)q2;
    }
    const float2 uv = G.u[t], Bv = G.B[t];
    const df ui = {uv.x, uv.y};
    const df Bi = {Bv.x, Bv.y};
    df acc = {0.f, 0.f};
    const bool dir = G.bnd != nullptr;
    const long long sx = 1, sy = G.n0, sz = (long long)G.n0 * G.n1;
    auto reg = [&](long long cj) {
      const float2 uj = G.u[cj], Bj = G.B[cj];
      acc = df_add(acc, df_face(ui, Bi, df{uj.x, uj.y}, df{Bj.x, Bj.y}));
    };
    auto ghost = [&](int f) {
      long long o;
      if (f < 2) o = (long long)k * G.n1 + j;
      else if (f < 4) o = (long long)k * G.n0 + i;
      else o = (long long)j * G.n0 + i;
      const df ub = split_bits(G.bnd[G.foff[f] + o]);
      // u_g = 2 u_b - u_i (mask ratio r = -1), b_g = exp(u_g)
      const df ug = df_sub(df{2.f * ub.h, 2.f * ub.l}, ui);
      acc = df_add(acc, df_face(ui, Bi, ug, df_exp(ug, ln2h, ln2l)));
    };
    if (i > 0) reg(t - sx); else if (!dir) reg(t + (G.n0 - 1) * sx); else ghost(0);
    if (i < G.n0 - 1) reg(t + sx); else if (!dir) reg(t - (G.n0 - 1) * sx); else ghost(1);
    if (j > 0) reg(t - sy); else if (!dir) reg(t + (G.n1 - 1) * sy); else ghost(2);
    if (j < G.n1 - 1) reg(t + sy); else if (!dir) reg(t - (G.n1 - 1) * sy); else ghost(3);
    if (k > 0) reg(t - sz); else if (!dir) reg(t + (G.n2 - 1) * sz); else ghost(4);
    if (k < G.n2 - 1) reg(t + sz); else if (!dir) reg(t - (G.n2 - 1) * sz); else ghost(5);
    // beta (e^{-u/2} - 1) with e^{-u/2} = 1/sqrt(e^u)
    const df y = df_add_f(df_rsqrt(Bi), -1.0f);
    df d = df_add(df_mul(acc, df{G.ahh, G.ahl}), df_mul(y, df{G.beh, G.bel}));
    const float2 rv = G.r[t];
    d = df_sub(d, df{rv.x, rv.y});
    const float dv = d.h + d.l;
    r32[t] = -dv;
    ub32[t] = ui.h;
    E32[t] = expf(ui.h);
    delta[t] = 0.0f;
    x32[t] = 0.0f;
    if (dout) dout[t] = join_bits(d.h, d.l);
    s2 = dv * dv;
    mx = fabsf(dv);
  }
  block_reduce2f<256>(s2, mx, &partial[2 * (base + blockIdx.x)],
                      &partial[2 * (base + blockIdx.x) + 1]);
}

}  // namespace frmg
