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
  FastDiv fdh, fd1;      // division by n0 / 2 (x-pairs) and n1 (grids below 2^31 cells)
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

// u += delta and e^u, two cells (an x-pair) per thread.  For |delta| < 2^-5
// (the correction steps) e^u is the old e^u times e^delta, e^delta by its
// Taylor series to degree 7 in double-float (truncation below 2^-40 delta^8 /
// 8!, far under the pair's rounding), on packed FP32 pairs, when every cell
// of the warp takes it; otherwise (the first update after the full-variable
// phase) e^u is recomputed from u.
__global__ void __launch_bounds__(128) k_df_update(DFGrid G, const float *delta, float ln2h,
                                                   float ln2l) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = t < (G.ncell >> 1);
  float4 *U4 = reinterpret_cast<float4 *>(G.u);
  float4 *B4 = reinterpret_cast<float4 *>(G.B);
  const float2 dl = in ? reinterpret_cast<const float2 *>(delta)[t] : make_float2(0.f, 0.f);
  // the path is chosen per warp: every lane recomputes e^u from u when one
  // cell of the warp has a large step (one path executed, not both)
  const bool smallw = __all_sync(0xffffffffu, fabsf(dl.x) < 0.03125f && fabsf(dl.y) < 0.03125f);
  if (!in) return;
  const float4 uo = U4[t];
  // u + delta: TwoSum of the hi parts, the lo part added, renormalised
  df2 s = two_sum2(make_float2(uo.x, uo.z), dl);
  s.l = add2(s.l, make_float2(uo.y, uo.w));
  const df2 u = fast_two_sum2(s.h, s.l);
  U4[t] = make_float4(u.h.x, u.l.x, u.h.y, u.l.y);
  float4 Bn;
  if (smallw) {
    const float4 Bo = B4[t];
    df2 q = {splat2(1.0f), splat2(0.0f)};
#pragma unroll
    for (int k = 7; k >= 1; k--) {
      // q *= d (df_mul_f lane by lane)
      df2 p = two_prod2(q.h, dl);
      p.l = fma2(q.l, dl, p.l);
      q = fast_two_sum2(p.h, p.l);
      // q = 1 + q / k: quotient of the hi part, remainder by FMA, low part
      const float rk = 1.0f / (float)k;
      const float2 qh = mul2(q.h, splat2(rk));
      const float2 rem = add2(fma2(qh, splat2(-(float)k), q.h), q.l);
      q = df_add_f2(df2{qh, mul2(rem, splat2(rk))}, 1.0f);
    }
    const df2 B = df_mul2(df2{make_float2(Bo.x, Bo.z), make_float2(Bo.y, Bo.w)}, q);
    Bn = make_float4(B.h.x, B.l.x, B.h.y, B.l.y);
  } else {
    const df b0 = df_exp(df{u.h.x, u.l.x}, ln2h, ln2l);
    const df b1 = df_exp(df{u.h.y, u.l.y}, ln2h, ln2l);
    Bn = make_float4(b0.h, b0.l, b1.h, b1.l);
  }
  B4[t] = Bn;
}

__global__ void k_df_final(DFGrid G, double *u64) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  const float2 v = G.u[t];
  u64[t] = join_bits(v.x, v.y);
}

// FP64-accurate defect d = A(u) - gamma (rho - 1) of the fine grid in
// double-float, and the set-up of the FP32 correction problem that follows:
// r32 = -d, background ub32 = hi(u) with E32 = e^{ub32}, delta = x = 0.
// Block partials (sum d^2, max |d|) go to partial[2 (base + block)].
// Two cells per thread (every grid has an even n0): the x-pair (2p, 2p + 1)
// of a row, every double-float operation on packed FP32 pairs (lane x: cell
// 2p, lane y: cell 2p + 1).  The face sum (B_i + B_j)(u_j - u_i) is taken as
// B_i S1 + S2 with S1 = sum (u_j - u_i) and S2 = sum B_j (u_j - u_i); the
// first face initialises the sums (adding a normalised pair to zero returns
// it).  256 cells per block of 128 threads.
template <bool BIG>
__global__ void __launch_bounds__(128)
    k_df_defect(DFGrid G, float *r32, float *ub32, float *E32, float *delta, float *x32,
                 double *partial, int base, float ln2h, float ln2l, double *dout = nullptr) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long np = G.ncell >> 1;
  float s2 = 0.0f, mx = 0.0f;
  if (t < np) {
    const int h0 = G.n0 >> 1;
    int i, j, k;
    if (BIG) {
      i = 2 * (int)(t % h0);
      const long long rr = t / h0;
      j = (int)(rr % G.n1);
      k = (int)(rr / G.n1);
    } else {
      const unsigned tu = (unsigned)t, q = fdiv(tu, G.fdh), q2 = fdiv(q, G.fd1);
      i = 2 * (int)(tu - q * (unsigned)h0);
      j = (int)(q - q2 * (unsigned)G.n1);
      k = (int)q2;
    }
    const long long c = 2 * t;
    const float4 *U4 = reinterpret_cast<const float4 *>(G.u);
    const float4 *B4 = reinterpret_cast<const float4 *>(G.B);
    const float4 uv = U4[t], Bv = B4[t];
    const df2 ui = {make_float2(uv.x, uv.z), make_float2(uv.y, uv.w)};
    const df2 Bi = {make_float2(Bv.x, Bv.z), make_float2(Bv.y, Bv.w)};
    const bool dir = G.bnd != nullptr;
    const long long sy = G.n0, sz = (long long)G.n0 * G.n1;
    // one lane's ghost value across face f (u_g = 2 u_b - u_i, b_g = e^{u_g})
    auto ghost = [&](int f, int lane, float &gh, float &gl, float &bh, float &bl) {
      const int ii = i + lane;
      long long o;
      if (f < 2) o = (long long)k * G.n1 + j;
      else if (f < 4) o = (long long)k * G.n0 + ii;
      else o = (long long)j * G.n0 + ii;
      const df ub = split_bits(G.bnd[G.foff[f] + o]);
      const df uil = lane ? df{uv.z, uv.w} : df{uv.x, uv.y};
      const df ug = df_sub(df{2.f * ub.h, 2.f * ub.l}, uil);
      const df bg = df_exp(ug, ln2h, ln2l);
      gh = ug.h;
      gl = ug.l;
      bh = bg.h;
      bl = bg.l;
    };
    df2 fs1, fs2;
    bool first = true;
    auto face = [&](const df2 &uj, const df2 &Bj) {
      const df2 dd = df_diff2(ui, uj);
      const df2 pr = df_mul2(Bj, dd);
      if (first) {
        fs1 = dd;
        fs2 = pr;
        first = false;
      } else {
        fs1 = df_add2(fs1, dd);
        fs2 = df_add2(fs2, pr);
      }
    };
    // a whole neighbouring pair (y and z faces): the pair at cell index cj
    auto pair_face = [&](long long cj) {
      const float4 a = U4[cj >> 1], b = B4[cj >> 1];
      face(df2{make_float2(a.x, a.z), make_float2(a.y, a.w)},
           df2{make_float2(b.x, b.z), make_float2(b.y, b.w)});
    };
    auto ghost_face = [&](int f) {
      float g0h, g0l, b0h, b0l, g1h, g1l, b1h, b1l;
      ghost(f, 0, g0h, g0l, b0h, b0l);
      ghost(f, 1, g1h, g1l, b1h, b1l);
      face(df2{make_float2(g0h, g1h), make_float2(g0l, g1l)},
           df2{make_float2(b0h, b1h), make_float2(b0l, b1l)});
    };
    // -x: cells (2p - 1, 2p); the left cell of the pair wraps or is a ghost at i = 0
    {
      float lh, ll, lbh, lbl;
      if (i > 0 || !dir) {
        const long long cl = i > 0 ? c - 1 : c + G.n0 - 1;
        const float2 a = G.u[cl], b = G.B[cl];
        lh = a.x; ll = a.y; lbh = b.x; lbl = b.y;
      } else {
        ghost(0, 0, lh, ll, lbh, lbl);
      }
      face(df2{make_float2(lh, uv.x), make_float2(ll, uv.y)},
           df2{make_float2(lbh, Bv.x), make_float2(lbl, Bv.y)});
    }
    // +x: cells (2p + 1, 2p + 2)
    {
      float rh, rl, rbh, rbl;
      if (i + 2 < G.n0 || !dir) {
        const long long cr = i + 2 < G.n0 ? c + 2 : c + 2 - G.n0;
        const float2 a = G.u[cr], b = G.B[cr];
        rh = a.x; rl = a.y; rbh = b.x; rbl = b.y;
      } else {
        ghost(1, 1, rh, rl, rbh, rbl);
      }
      face(df2{make_float2(uv.z, rh), make_float2(uv.w, rl)},
           df2{make_float2(Bv.z, rbh), make_float2(Bv.w, rbl)});
    }
    if (j > 0) pair_face(c - sy); else if (!dir) pair_face(c + (G.n1 - 1) * sy); else ghost_face(2);
    if (j < G.n1 - 1) pair_face(c + sy); else if (!dir) pair_face(c - (G.n1 - 1) * sy); else ghost_face(3);
    if (k > 0) pair_face(c - sz); else if (!dir) pair_face(c + (G.n2 - 1) * sz); else ghost_face(4);
    if (k < G.n2 - 1) pair_face(c + sz); else if (!dir) pair_face(c - (G.n2 - 1) * sz); else ghost_face(5);
    const df2 acc = df_add2(df_mul2(Bi, fs1), fs2);
    const df2 y = df_add_f2(df_rsqrt2(Bi), -1.0f);
    const df2 ah = {splat2(G.ahh), splat2(G.ahl)}, be = {splat2(G.beh), splat2(G.bel)};
    df2 d = df_add2(df_mul2(acc, ah), df_mul2(y, be));
    const float4 rv = reinterpret_cast<const float4 *>(G.r)[t];
    d = df_sub2(d, df2{make_float2(rv.x, rv.z), make_float2(rv.y, rv.w)});
    const float2 dv = add2(d.h, d.l);
    reinterpret_cast<float2 *>(r32)[t] = make_float2(-dv.x, -dv.y);
    reinterpret_cast<float2 *>(ub32)[t] = ui.h;
    reinterpret_cast<float2 *>(E32)[t] = make_float2(expf(ui.h.x), expf(ui.h.y));
    reinterpret_cast<float2 *>(delta)[t] = make_float2(0.0f, 0.0f);
    reinterpret_cast<float2 *>(x32)[t] = make_float2(0.0f, 0.0f);
    if (dout)
      reinterpret_cast<double2 *>(dout)[t] =
          make_double2(join_bits(d.h.x, d.l.x), join_bits(d.h.y, d.l.y));
    s2 = fmaf(dv.y, dv.y, dv.x * dv.x);
    mx = fmaxf(fabsf(dv.x), fabsf(dv.y));
  }
  block_reduce2f<128>(s2, mx, &partial[2 * (base + blockIdx.x)],
                      &partial[2 * (base + blockIdx.x) + 1]);
}

}  // namespace frmg
