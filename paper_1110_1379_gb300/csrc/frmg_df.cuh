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
  for (int k = 7; k >= 1; k--) {
    t = df_mul(t, r);
    // t = 1 + t / k
    float q = t.h / (float)k;
    float rem = fmaf(-q, (float)k, t.h) + t.l;  // t - q k
    df tq = {q, rem / (float)k};
    t = df_add_f(tq, 1.0f);
  }
  for (int k = 0; k < 4; k++) t = df_mul(t, t);
  int ni = (int)n;
  return {ldexpf(t.h, ni), ldexpf(t.l, ni)};
}

}  // namespace frmg

namespace frmg {

// Fine-grid state of the double-float outer loop of one grid.
struct DFGrid {
  float *uh, *ul;        // u = uh + ul
  float *Bh, *Bl;        // e^u
  float *rh, *rl;        // gamma (rho - 1)
  const double *bnd;     // packed Dirichlet faces (FP64) or null
  long long foff[6];
  long long ncell;
  int n0, n1, n2;
  float ahh, ahl;        // alpha / 2
  float beh, bel;        // beta
};

// Splits an FP64 value into a double-float pair.
__device__ __forceinline__ df split_d(double v) {
  float h = (float)v;
  return {h, (float)(v - (double)h)};
}

// State set-up: u (FP64, or zero), e^u and gamma (rho - 1) as double-float.
__global__ void k_df_init(DFGrid G, const double *u64, const double *rho, double gamma,
                          int zero_u, float ln2h, float ln2l) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  df u = zero_u ? df{0.f, 0.f} : split_d(u64[t]);
  G.uh[t] = u.h;
  G.ul[t] = u.l;
  df B = zero_u ? df{1.f, 0.f} : df_exp(u, ln2h, ln2l);
  G.Bh[t] = B.h;
  G.Bl[t] = B.l;
  df r = split_d(gamma * (rho[t] - 1.0));
  G.rh[t] = r.h;
  G.rl[t] = r.l;
}

// u += delta, e^u recomputed from u (no drift across outer steps).
__global__ void k_df_update(DFGrid G, const float *delta, float ln2h, float ln2l) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  df s = two_sum(G.uh[t], delta[t]);
  s.l += G.ul[t];
  df u = fast_two_sum(s.h, s.l);
  G.uh[t] = u.h;
  G.ul[t] = u.l;
  df B = df_exp(u, ln2h, ln2l);
  G.Bh[t] = B.h;
  G.Bl[t] = B.l;
}

__global__ void k_df_final(DFGrid G, double *u64) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  u64[t] = (double)G.uh[t] + (double)G.ul[t];
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
__global__ void __launch_bounds__(256)
    k_df_defect(DFGrid G, float *r32, float *ub32, float *E32, float *delta, float *x32,
                double *partial, int base, float ln2h, float ln2l, double *dout = nullptr) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float s2 = 0.0f, mx = 0.0f;
  if (t < G.ncell) {
    const int i = (int)(t % G.n0);
    const long long rr = t / G.n0;
    const int j = (int)(rr % G.n1);
    const int k = (int)(rr / G.n1);
    const df ui = {G.uh[t], G.ul[t]};
    const df Bi = {G.Bh[t], G.Bl[t]};
    df acc = {0.f, 0.f};
    const bool dir = G.bnd != nullptr;
    const long long sx = 1, sy = G.n0, sz = (long long)G.n0 * G.n1;
    auto reg = [&](long long cj) {
      acc = df_add(acc, df_face(ui, Bi, df{G.uh[cj], G.ul[cj]}, df{G.Bh[cj], G.Bl[cj]}));
    };
    auto ghost = [&](int f) {
      long long o;
      if (f < 2) o = (long long)k * G.n1 + j;
      else if (f < 4) o = (long long)k * G.n0 + i;
      else o = (long long)j * G.n0 + i;
      const df ub = split_d(G.bnd[G.foff[f] + o]);
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
    d = df_sub(d, df{G.rh[t], G.rl[t]});
    const float dv = d.h + d.l;
    r32[t] = -dv;
    ub32[t] = ui.h;
    E32[t] = expf(ui.h);
    delta[t] = 0.0f;
    x32[t] = 0.0f;
    if (dout) dout[t] = (double)d.h + (double)d.l;
    s2 = dv * dv;
    mx = fabsf(dv);
  }
  block_reduce2f<256>(s2, mx, &partial[2 * (base + blockIdx.x)],
                      &partial[2 * (base + blockIdx.x) + 1]);
}

}  // namespace frmg
