// frmg_df.cuh -- the FP64-accurate fine-grid state, defect and update of the
// mixed-precision loop of the f(R) solve, in double-float arithmetic
// (frmg_dfmath.cuh).
#pragma once

#include <cuda_runtime.h>

#include "frmg_dfmath.cuh"

namespace frmg {

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

// u += delta and e^u.  For |delta| < 2^-5 (the correction steps) e^u is the
// old e^u times e^delta, e^delta by its Taylor series to degree 7 in
// double-float (truncation below 2^-40 delta^8 / 8!, far under the pair's
// rounding); larger steps (the first update after the full-variable phase)
// recompute e^u from u.
__global__ void k_df_update(DFGrid G, const float *delta, float ln2h, float ln2l) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  const float2 uo = G.u[t];
  const float dl = delta[t];
  df s = two_sum(uo.x, dl);
  s.l += uo.y;
  df u = fast_two_sum(s.h, s.l);
  G.u[t] = make_float2(u.h, u.l);
  df B;
  if (fabsf(dl) < 0.03125f) {
    // Horner: e^d = 1 + d (1 + d/2 (1 + d/3 (... (1 + d/7))))
    df q = {1.0f, 0.0f};
#pragma unroll
    for (int k = 7; k >= 1; k--) {
      q = df_mul_f(q, dl);
      const float rk = 1.0f / (float)k;  // a constant after unrolling
      const float qh = q.h * rk;
      const float rem = fmaf(-qh, (float)k, q.h) + q.l;
      q = df_add_f(df{qh, rem * rk}, 1.0f);
    }
    const float2 Bo = G.B[t];
    B = df_mul(df{Bo.x, Bo.y}, q);
  } else {
    B = df_exp(u, ln2h, ln2l);
  }
  G.B[t] = make_float2(B.h, B.l);
}

__global__ void k_df_final(DFGrid G, double *u64) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  const float2 v = G.u[t];
  u64[t] = join_bits(v.x, v.y);
}

// u_j - u_i of one face in double-float.
__device__ __forceinline__ df df_diff(df ui, df uj) {
  df dd = two_sum(uj.h, -ui.h);
  dd.l += uj.l - ui.l;
  return fast_two_sum(dd.h, dd.l);
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
    // sum over the faces of (B_i + B_j)(u_j - u_i) = B_i S1 + S2 with
    // S1 = sum (u_j - u_i) and S2 = sum B_j (u_j - u_i)
    df fs1 = {0.f, 0.f}, fs2 = {0.f, 0.f};
    const bool dir = G.bnd != nullptr;
    const long long sx = 1, sy = G.n0, sz = (long long)G.n0 * G.n1;
    auto face = [&](df uj, df Bj) {
      const df dd = df_diff(ui, uj);
      fs1 = df_add(fs1, dd);
      fs2 = df_add(fs2, df_mul(Bj, dd));
    };
    auto reg = [&](long long cj) {
      const float2 uj = G.u[cj], Bj = G.B[cj];
      face(df{uj.x, uj.y}, df{Bj.x, Bj.y});
    };
    auto ghost = [&](int f) {
      long long o;
      if (f < 2) o = (long long)k * G.n1 + j;
      else if (f < 4) o = (long long)k * G.n0 + i;
      else o = (long long)j * G.n0 + i;
      const df ub = split_bits(G.bnd[G.foff[f] + o]);
      // u_g = 2 u_b - u_i (mask ratio r = -1), b_g = exp(u_g)
      const df ug = df_sub(df{2.f * ub.h, 2.f * ub.l}, ui);
      face(ug, df_exp(ug, ln2h, ln2l));
    };
    if (i > 0) reg(t - sx); else if (!dir) reg(t + (G.n0 - 1) * sx); else ghost(0);
    if (i < G.n0 - 1) reg(t + sx); else if (!dir) reg(t - (G.n0 - 1) * sx); else ghost(1);
    if (j > 0) reg(t - sy); else if (!dir) reg(t + (G.n1 - 1) * sy); else ghost(2);
    if (j < G.n1 - 1) reg(t + sy); else if (!dir) reg(t - (G.n1 - 1) * sy); else ghost(3);
    if (k > 0) reg(t - sz); else if (!dir) reg(t + (G.n2 - 1) * sz); else ghost(4);
    if (k < G.n2 - 1) reg(t + sz); else if (!dir) reg(t - (G.n2 - 1) * sz); else ghost(5);
    const df acc = df_add(df_mul(Bi, fs1), fs2);
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
