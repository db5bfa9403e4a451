// frmg_kernels.cuh -- device code of the f(R) FAS multigrid solver (sm_103a).
//
// Operator (Sec. IV Eq. discrete_fR times c~^2, Sec. V.B.1 Eq. bc_modified_fR_op)
// in u = ln(f_R/fbar_R), as a nonlinear operator A with right-hand side f:
//
//   A_i(u) = (alpha/2) sum_j (e^{u_i} + e^{u_j}) (u_j - u_i) + beta (e^{-u_i/2} - 1)
//   finest level:  A(u) = gamma (rho - 1);  coarse levels: A^H(u^H) = f^H (FAS).
//
// Two evaluation modes share one code path:
//  * plain (BG = false): u is the unknown itself.  Cache x = expm1(u), so
//    B = e^u = 1 + x.
//  * background (BG = true, FP32 inside the mixed-precision loop): the unknown
//    is a correction delta on a fixed FP32 background ub (E = e^{ub}), and the
//    kernels evaluate N(delta) = A(ub + delta) - A(ub) in a form where every
//    term carries a factor of delta:
//      (alpha/2) sum_j [ (E_i x_i + E_j x_j)(ub_j - ub_i) + (B_i + B_j)(d_j - d_i) ]
//      + beta e^{-ub_i/2} (e^{-d_i/2} - 1),    x = expm1(delta), B = E (1 + x).
//    so that FP32 rounding is relative to the correction, not to u.
// Both modes give the same Newton derivative (Eq. bc_modified_fR_dop):
//   dA_i/du_i = (alpha/2) sum_j [ B_i (u_j - u_i) - (B_i + B_j) ] - (beta/2) e^{-u_i/2}.
//
// Refinement patches: a ghost neighbour outside the patch takes
//   u_g = u_b - r u_b + r u_i with r = -1, b_g = exp(u_g)     (Eq. u_i-1jk),
// so its face contributes (B_i + B_g)(u_g - u_i) and, because u_g depends on
// u_i, (B_i - B_g)(u_g - u_i) - 2 (B_i + B_g) to the derivative.
//
// Red-black ordering: colour = (i + j + k) & 1, red (0) first.
// Layout: [n2][n1][n0], x fastest.  Packed boundary faces: -x,+x,-y,+y,-z,+z,
// face normal to axis a indexed by the other axes p < q as c[q]*n[p] + c[p].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "frmg_dfmath.cuh"

namespace frmg {

template <typename T>
struct Grid {
  T *u;            // unknown (delta in background mode), buffer 0
  T *u2;           // buffer 1: the tiled smoother reads one buffer and writes the other
  T *x2;           // buffer 1 of the x cache (ping-pongs with u)
  T *x;            // cache: expm1(u)
  const T *f;      // right-hand side storage; f_i = fs * (f[i] - fo); null = 0
                   // (FP32 grids store f_i itself: fs = 1, fo = 0)
  T *uR;           // R u^h saved for the FAS correction (coarse levels)
  const float *ubg;  // background (BG mode), null otherwise
  const float *Ebg;  // exp(background)
  const T *bnd;    // packed Dirichlet faces (null: periodic)
  long long foff[6];
  long long ncell;
  int n0, n1, n2;
  int field;       // index into the active-flag array
  T ah;            // alpha / 2
  T beta;
  T fs, fo;
  T cap;           // Newton step cap
  T relax;         // relaxation factor of the Newton update (1: plain Newton-GS)
  FastDiv fd0, fd1;  // division by n0 and n1 (cell index -> (i, j, k))
};

// (i, j, k) of the linear cell index c < ncell: 32-bit multiply-shift division
// below 2^31 cells, 64-bit division above.
template <typename T>
__device__ __forceinline__ void cell_ijk(const Grid<T> &G, long long c, int &i, int &j, int &k) {
  if (G.ncell < (1ll << 31)) {
    const unsigned cu = (unsigned)c, q = fdiv(cu, G.fd0), q2 = fdiv(q, G.fd1);
    i = (int)(cu - q * (unsigned)G.n0);
    j = (int)(q - q2 * (unsigned)G.n1);
    k = (int)q2;
  } else {
    i = (int)(c % G.n0);
    const long long r = c / G.n0;
    j = (int)(r % G.n1);
    k = (int)(r / G.n1);
  }
}

// ----------------------------------------------------------------------------
// math wrappers (library functions; no re-derived constants)
__device__ __forceinline__ float m_exp(float v) { return expf(v); }
__device__ __forceinline__ double m_exp(double v) { return exp(v); }
// FP32 e^d - 1 used by every FP32 kernel (so all of them see the same cache
// values): the Taylor series to degree 6 for |d| < 1/16 (truncation below
// 1e-12 relative, which keeps small corrections exact to FP32 rounding), and
// the correctly rounded-to-1-ulp exponential minus one otherwise (strongly
// screened cells reach |u| ~ 10, where the SFU approximation's error of a few
// ulp per unit of |u| would set the FP32 residual floor).
// Every FP32 operation of the shared operator code is written out as an
// explicit rounding (fmaf, __fadd_rn, __fmul_rn, ...), so that no kernel's
// compiler contraction can change it: the scalar and the packed (two cells per
// instruction, below) evaluations are then the same bit for bit.
__device__ __forceinline__ float m_expm1_taylor(float d) {
  float p = fmaf(d, 1.0f / 720.0f, 1.0f / 120.0f);
  p = fmaf(d, p, 1.0f / 24.0f);
  p = fmaf(d, p, 1.0f / 6.0f);
  p = fmaf(d, p, 0.5f);
  p = fmaf(d, p, 1.0f);
  return __fmul_rn(d, p);
}
__device__ __forceinline__ float m_expm1(float d) {
  if (fabsf(d) < 0.0625f) return m_expm1_taylor(d);
  return __fsub_rn(expf(d), 1.0f);
}
__device__ __forceinline__ double m_expm1(double v) { return expm1(v); }
__device__ __forceinline__ float m_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double m_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float m_rsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double m_rsqrt(double v) { return rsqrt(v); }

__device__ __forceinline__ int wrapmod(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ int find_grid(const int *off, int ngrid, int b) {
  int lo = 0, hi = ngrid;  // off[lo] <= b < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= b)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Grid view whose u is the current buffer (par selects buffer 0 or 1).
template <typename T>
__device__ __forceinline__ Grid<T> view(const Grid<T> *grids, int g, int par) {
  Grid<T> G = grids[g];
  if (par) {
    G.u = G.u2;
    G.x = G.x2;
  }
  return G;
}

__device__ __forceinline__ bool grid_active(const int *active, int field) {
  return active == nullptr || active[field] != 0;
}

template <typename T>
__device__ __forceinline__ long long idx3(const Grid<T> &G, int i, int j, int k) {
  return ((long long)k * G.n1 + j) * G.n0 + i;
}

// Boundary value of the face f (0..5) at the boundary cell (i,j,k).
template <typename T>
__device__ __forceinline__ T face_value(const Grid<T> &G, int f, int i, int j, int k) {
  long long o;
  if (f < 2)
    o = (long long)k * G.n1 + j;
  else if (f < 4)
    o = (long long)k * G.n0 + i;
  else
    o = (long long)j * G.n0 + i;
  return G.bnd[G.foff[f] + o];
}

// Contribution of one regular face (neighbour values given).
template <typename T, bool BG>
__device__ __forceinline__ void face_vals(T dj, T xj, T ubj, T Ej, T di, T Ei, T xi, T Bi, T ubi,
                                          T &acc, T &dacc) {
  T Bj = BG ? Ej + Ej * xj : T(1) + xj;
  T dd = dj - di;
  T w;
  if (BG) {
    T gd = ubj - ubi;
    acc += (Ei * xi + Ej * xj) * gd + (Bi + Bj) * dd;
    w = gd + dd;
  } else {
    acc += (Bi + Bj) * dd;
    w = dd;
  }
  dacc += Bi * w - (Bi + Bj);
}

template <typename T, bool BG>
__device__ __forceinline__ void face_ghost(T ubf, T di, T Ei, T xi, T Bi, T ubi, T &acc,
                                           T &dacc) {
  T w, Bg;
  if (BG) {
    T ubgh = T(2) * ubf - ubi;   // background ghost
    T Eg = m_exp(ubgh);
    T xg = -xi / (T(1) + xi);    // expm1(-delta_i)
    T gd = ubgh - ubi;
    T dd = T(-2) * di;           // delta_g - delta_i
    Bg = Eg + Eg * xg;
    acc += (Ei * xi + Eg * xg) * gd + (Bi + Bg) * dd;
    w = gd + dd;
  } else {
    T ug = T(2) * ubf - di;
    Bg = m_exp(ug);
    w = ug - di;
    acc += (Bi + Bg) * w;
  }
  dacc += (Bi - Bg) * w - T(2) * (Bi + Bg);
}

// Face-sum accumulator of one cell: own values at construction, one call per
// face (regular neighbour or patch ghost), then the two sums
//   acc  = sum_faces (flux term),   dacc = sum_faces d(flux term)/du_i.
// The generic form adds (B_i + B_j)(u_j - u_i) face by face.  The plain FP32
// form (the bulk of the mixed-precision work) regroups the same sum as
//   acc  = (B_i + 1) S1 + S2,   dacc = B_i S1 - n (B_i + 1) - S3,
//   S1 = sum (u_j - u_i),  S2 = sum x_j (u_j - u_i),  S3 = sum x_j,
// over the n regular faces (B_j = 1 + x_j), four operations per face instead
// of six; every FP32 kernel uses this one accumulator, so all of them evaluate
// the same discrete operator.
template <typename T, bool BG>
struct OpAcc {
  T di, Ei, xi, Bi, ubi;
  T acc = T(0), dacc = T(0);
  __device__ __forceinline__ OpAcc(T d, T E, T x, T B, T ub) : di(d), Ei(E), xi(x), Bi(B), ubi(ub) {}
  __device__ __forceinline__ void reg(T dj, T xj, T ubj, T Ej) {
    face_vals<T, BG>(dj, xj, ubj, Ej, di, Ei, xi, Bi, ubi, acc, dacc);
  }
  __device__ __forceinline__ void ghost(T ubf) {
    face_ghost<T, BG>(ubf, di, Ei, xi, Bi, ubi, acc, dacc);
  }
  __device__ __forceinline__ void done(T &a, T &da) const {
    a = acc;
    da = dacc;
  }
};

template <>
struct OpAcc<float, false> {
  float di, Ei, xi, Bi, ubi;
  float S1 = 0.f, S2 = 0.f, S3 = 0.f, ga = 0.f, gd = 0.f;
  int n = 0;
  __device__ __forceinline__ OpAcc(float d, float E, float x, float B, float ub)
      : di(d), Ei(E), xi(x), Bi(B), ubi(ub) {}
  __device__ __forceinline__ void reg(float dj, float xj, float, float) {
    const float dd = __fsub_rn(dj, di);
    S1 = __fadd_rn(S1, dd);
    S2 = fmaf(xj, dd, S2);
    S3 = __fadd_rn(S3, xj);
    n++;
  }
  __device__ __forceinline__ void ghost(float ubf) {
    face_ghost<float, false>(ubf, di, Ei, xi, Bi, ubi, ga, gd);
  }
  __device__ __forceinline__ void done(float &a, float &da) const {
    const float nf = (float)n;
    const float b1 = __fadd_rn(Bi, 1.0f);
    a = __fadd_rn(fmaf(b1, S1, S2), ga);
    da = __fadd_rn(__fsub_rn(fmaf(Bi, S1, __fmul_rn(-nf, b1)), S3), gd);
  }
};

// The FP32 correction form regroups its face sum the same way: with
// P = E x (so B = E + P) and g_j = ub_j - ub_i,
//   acc  = sum (P_i + P_j) g_j + (B_i + B_j)(d_j - d_i)
//        = P_i G1 + G2 + B_i S1 + S2,
//   dacc = sum B_i (g_j + d_j - d_i) - (B_i + B_j) = B_i (G1 + S1) - n B_i - S3,
//   G1 = sum g_j, G2 = sum P_j g_j, S1 = sum (d_j - d_i), S2 = sum B_j (d_j - d_i),
//   S3 = sum B_j,
// nine operations per face instead of about twelve, every rounding explicit.
template <>
struct OpAcc<float, true> {
  float di, Ei, xi, Bi, ubi;
  float G1 = 0.f, G2 = 0.f, S1 = 0.f, S2 = 0.f, S3 = 0.f, ga = 0.f, gd = 0.f;
  int n = 0;
  __device__ __forceinline__ OpAcc(float d, float E, float x, float B, float ub)
      : di(d), Ei(E), xi(x), Bi(B), ubi(ub) {}
  __device__ __forceinline__ void reg(float dj, float xj, float ubj, float Ej) {
    const float Pj = __fmul_rn(Ej, xj);
    const float Bj = __fadd_rn(Ej, Pj);
    const float dd = __fsub_rn(dj, di), g = __fsub_rn(ubj, ubi);
    G1 = __fadd_rn(G1, g);
    G2 = fmaf(Pj, g, G2);
    S1 = __fadd_rn(S1, dd);
    S2 = fmaf(Bj, dd, S2);
    S3 = __fadd_rn(S3, Bj);
    n++;
  }
  __device__ __forceinline__ void ghost(float ubf) {
    face_ghost<float, true>(ubf, di, Ei, xi, Bi, ubi, ga, gd);
  }
  __device__ __forceinline__ void done(float &a, float &da) const {
    const float nf = (float)n;
    const float Pi = __fmul_rn(Ei, xi);
    a = __fadd_rn(__fadd_rn(fmaf(Pi, G1, G2), fmaf(Bi, S1, S2)), ga);
    da = __fadd_rn(__fsub_rn(fmaf(Bi, __fadd_rn(G1, S1), __fmul_rn(-nf, Bi)), S3), gd);
  }
};

// Mass term and final assembly:  N = (alpha/2) acc + beta F (e^{-d/2} - 1),
// dN = (alpha/2) dacc - (beta/2) F e^{-d/2},  F = e^{-ub/2}.
// FP64 uses IEEE sqrt and division; FP32 uses the SFU reciprocal square root
// and reciprocal (the same expression in every FP32 kernel, so all of them
// see one and the same discrete operator).
__device__ __forceinline__ void finish_op(double xi, double Ei, double acc, double dacc,
                                          double ah, double beta, bool bg, double &N,
                                          double &dN) {
  double B1 = 1.0 + xi;
  double s = sqrt(B1);
  double y = -xi / (B1 + s);
  double F = bg ? rsqrt(Ei) : 1.0;
  N = ah * acc + beta * F * y;
  dN = ah * dacc - 0.5 * beta * F / s;
}

// SFU reciprocal and reciprocal square root (PTX rcp.approx / rsqrt.approx,
// subnormals flushed: every FP32 quantity here is far from the subnormal range).
__device__ __forceinline__ float sfu_rcp(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float sfu_rsqrt(float v) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ void finish_op(float xi, float Ei, float acc, float dacc, float ah,
                                          float beta, bool bg, float &N, float &dN) {
  const float B1 = __fadd_rn(1.0f, xi);
  const float rs = sfu_rsqrt(B1);  // e^{-d/2}
  const float s = __fmul_rn(B1, rs);  // e^{d/2}
  const float y = __fmul_rn(-xi, sfu_rcp(__fadd_rn(B1, s)));
  const float bF = bg ? __fmul_rn(beta, sfu_rsqrt(Ei)) : beta;  // beta F
  N = fmaf(ah, acc, __fmul_rn(bF, y));
  dN = fmaf(ah, dacc, -__fmul_rn(__fmul_rn(0.5f, bF), rs));
}

__device__ __forceinline__ double newton_step(double r, double dN) { return -r / dN; }
__device__ __forceinline__ float newton_step(float r, float dN) {
  return __fmul_rn(-r, sfu_rcp(dN));
}
// relaxed Newton step w (N - f) / -dN of a cell
__device__ __forceinline__ double newton_du(double N, double f, double dN, double w) {
  return w * newton_step(N - f, dN);
}
__device__ __forceinline__ float newton_du(float N, float f, float dN, float w) {
  return __fmul_rn(w, newton_step(__fsub_rn(N, f), dN));
}

// ---- packed FP32 pairs (add2, sub2, fma2, mul2, splat2 of frmg_dfmath.cuh)
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// m_expm1 of two values: the Taylor branch packed, the exponential branch per lane
__device__ __forceinline__ float2 m_expm1_2(float2 d) {
  float2 p = fma2(d, splat2(1.0f / 720.0f), splat2(1.0f / 120.0f));
  p = fma2(d, p, splat2(1.0f / 24.0f));
  p = fma2(d, p, splat2(1.0f / 6.0f));
  p = fma2(d, p, splat2(0.5f));
  p = fma2(d, p, splat2(1.0f));
  float2 r = mul2(d, p);
  if (!(fabsf(d.x) < 0.0625f)) r.x = __fsub_rn(expf(d.x), 1.0f);
  if (!(fabsf(d.y) < 0.0625f)) r.y = __fsub_rn(expf(d.y), 1.0f);
  return r;
}

// The plain-form Newton update of two cells at once, operation for operation
// the scalar OpAcc<float, false> (six regular faces), finish_op and newton_du:
// own (u, x), right-hand side f, neighbour u and x in the face order -x, +x,
// -y, +y, -z, +z; returns the two new u.
__device__ __forceinline__ float2 newton2_plain(float2 di, float2 xi, float2 fi, const float2 *nu,
                                                const float2 *nx, float ah, float beta, float cap,
                                                float relax) {
  const float2 Bi = add2(splat2(1.0f), xi);
  float2 S1 = sub2(nu[0], di), S2, S3 = nx[0];
  S2 = mul2(nx[0], S1);  // fmaf(x, dd, 0) rounds as the product
#pragma unroll
  for (int f = 1; f < 6; f++) {
    const float2 dd = sub2(nu[f], di);
    S1 = add2(S1, dd);
    S2 = fma2(nx[f], dd, S2);
    S3 = add2(S3, nx[f]);
  }
  const float2 b1 = add2(Bi, splat2(1.0f));
  const float2 acc = fma2(b1, S1, S2);
  const float2 dacc = sub2(fma2(Bi, S1, mul2(splat2(-6.0f), b1)), S3);
  // finish_op
  const float2 B1 = add2(splat2(1.0f), xi);
  const float2 rs = make_float2(sfu_rsqrt(B1.x), sfu_rsqrt(B1.y));
  const float2 sv = mul2(B1, rs);
  const float2 den = add2(B1, sv);
  const float2 y = mul2(neg2(xi), make_float2(sfu_rcp(den.x), sfu_rcp(den.y)));
  const float2 N = fma2(splat2(ah), acc, mul2(splat2(beta), y));
  const float2 dN = fma2(splat2(ah), dacc, neg2(mul2(splat2(0.5f * beta), rs)));
  // newton_du, clamp, update
  const float2 r = sub2(N, fi);
  const float2 q = make_float2(sfu_rcp(dN.x), sfu_rcp(dN.y));
  float2 du = mul2(splat2(relax), mul2(neg2(r), q));
  du.x = fminf(fmaxf(du.x, -cap), cap);
  du.y = fminf(fmaxf(du.y, -cap), cap);
  return add2(di, du);
}

// A_i (or N_i) and its derivative at cell (i,j,k) from global memory.
template <typename T, bool BG>
__device__ __forceinline__ void cell_eval(const Grid<T> &G, int i, int j, int k, long long c,
                                          T &N, T &dN) {
  const T di = G.u[c];
  const T xi = G.x[c];
  const T Ei = BG ? (T)G.Ebg[c] : T(1);
  const T ubi = BG ? (T)G.ubg[c] : T(0);
  const T Bi = BG ? Ei + Ei * xi : T(1) + xi;
  OpAcc<T, BG> A(di, Ei, xi, Bi, ubi);
  const bool dir = G.bnd != nullptr;
  const long long sx = 1, sy = G.n0, sz = (long long)G.n0 * G.n1;
  auto nb = [&](long long cj) {
    A.reg(G.u[cj], G.x[cj], BG ? (T)G.ubg[cj] : T(0), BG ? (T)G.Ebg[cj] : T(1));
  };
  // -x, +x
  if (i > 0) nb(c - sx);
  else if (!dir) nb(c + (G.n0 - 1) * sx);
  else A.ghost(face_value(G, 0, i, j, k));
  if (i < G.n0 - 1) nb(c + sx);
  else if (!dir) nb(c - (G.n0 - 1) * sx);
  else A.ghost(face_value(G, 1, i, j, k));
  // -y, +y
  if (j > 0) nb(c - sy);
  else if (!dir) nb(c + (G.n1 - 1) * sy);
  else A.ghost(face_value(G, 2, i, j, k));
  if (j < G.n1 - 1) nb(c + sy);
  else if (!dir) nb(c - (G.n1 - 1) * sy);
  else A.ghost(face_value(G, 3, i, j, k));
  // -z, +z
  if (k > 0) nb(c - sz);
  else if (!dir) nb(c + (G.n2 - 1) * sz);
  else A.ghost(face_value(G, 4, i, j, k));
  if (k < G.n2 - 1) nb(c + sz);
  else if (!dir) nb(c - (G.n2 - 1) * sz);
  else A.ghost(face_value(G, 5, i, j, k));
  T acc, dacc;
  A.done(acc, dacc);
  finish_op(xi, Ei, acc, dacc, G.ah, G.beta, BG, N, dN);
}

template <typename T>
__device__ __forceinline__ T rhs_at(const Grid<T> &G, long long c) {
  return G.f ? G.fs * (G.f[c] - G.fo) : T(0);
}

template <typename T, bool BG>
__device__ __forceinline__ void ngs_update(const Grid<T> &G, int i, int j, int k) {
  long long c = idx3(G, i, j, k);
  T N, dN;
  cell_eval<T, BG>(G, i, j, k, c, N, dN);
  T du = newton_du(N, rhs_at(G, c), dN, G.relax);
  du = du > G.cap ? G.cap : (du < -G.cap ? -G.cap : du);
  T unew = G.u[c] + du;
  G.u[c] = unew;
  G.x[c] = m_expm1(unew);
}

// ---------------------------------------------------------------------------
// One colour of a red-black Newton-Gauss-Seidel sweep; one thread per cell of
// that colour.  off[] maps blocks to grids (n0/2 * n1 * n2 threads per grid).
template <typename T, bool BG>
__global__ void k_smooth(const Grid<T> *grids, const int *off, int ngrid, int colour,
                         const int *active, int par) {
  int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<T> G = view(grids, g, par);
  if (!grid_active(active, G.field)) return;
  long long t = (long long)(blockIdx.x - off[g]) * blockDim.x + threadIdx.x;
  if (2 * t >= G.ncell) return;
  int i, j, k;
  cell_ijk(G, 2 * t, i, j, k);  // even cell of the pair
  i += (j + k + colour) & 1;
  ngs_update<T, BG>(G, i, j, k);
}

// Block-level (sum of squares, max |v|) partials, one pair per block.
template <int NT>
__device__ __forceinline__ void block_reduce2(double s, double m, double *out_s, double *out_m) {
  __shared__ double ss[NT / 32], sm[NT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    ss[w] = s;
    sm[w] = m;
  }
  __syncthreads();
  if (w == 0) {
    s = (l < NT / 32) ? ss[l] : 0.0;
    m = (l < NT / 32) ? sm[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, o);
      m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if (l == 0) {
      *out_s = s;
      *out_m = m;
    }
  }
}

// Block-level (sum of squares, max |v|) from FP32 per-thread values, reduced in
// FP32 (relative error ~1e-6, ample for a stopping criterion) and written as
// FP64 once per block: FP64 arithmetic runs at 1/64 of the FP32 rate here.
template <int NT>
__device__ __forceinline__ void block_reduce2f(float s, float m, double *out_s, double *out_m) {
  __shared__ float ssf[NT / 32], smf[NT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    ssf[w] = s;
    smf[w] = m;
  }
  __syncthreads();
  if (w == 0) {
    s = (l < NT / 32) ? ssf[l] : 0.0f;
    m = (l < NT / 32) ? smf[l] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, o);
      m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if (l == 0) {
      *out_s = (double)s;
      *out_m = (double)m;
    }
  }
}

// d = A(u) - f over every cell; optional output array and per-block partial
// norms (partial[2*block], partial[2*block+1]).  One thread per cell.
template <typename T, bool BG, int NT>
__global__ void __launch_bounds__(NT) k_residual(const Grid<T> *grids, const int *off, int ngrid,
                                                 T *const *dout, double *partial,
                                                 const int *active, int par) {
  int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<T> G = view(grids, g, par);
  float s = 0.0f, m = 0.0f;
  long long t = (long long)(blockIdx.x - off[g]) * NT + threadIdx.x;
  if (grid_active(active, G.field) && t < G.ncell) {
    int i, j, k;
    cell_ijk(G, t, i, j, k);
    T N, dN;
    cell_eval<T, BG>(G, i, j, k, t, N, dN);
    T d = N - rhs_at(G, t);
    if (dout && dout[g]) dout[g][t] = d;
    const float df_ = (float)d;
    s = df_ * df_;
    m = fabsf(df_);
  }
  if (partial) block_reduce2f<NT>(s, m, &partial[2 * blockIdx.x], &partial[2 * blockIdx.x + 1]);
}

// Per-grid sums of the block partials: out[2g] = sum of squares, out[2g+1] = max.
__global__ void k_reduce_partials(const double *partial, const int *off, int ngrid, double *out) {
  int g = blockIdx.x;
  if (g >= ngrid) return;
  double s = 0.0, m = 0.0;
  for (int b = off[g] + threadIdx.x; b < off[g + 1]; b += blockDim.x) {
    s += partial[2 * b];
    m = fmax(m, partial[2 * b + 1]);
  }
  block_reduce2<256>(s, m, &out[2 * g], &out[2 * g + 1]);
}

// First stage of the per-grid sums for long partial lists: block (c, g)
// reduces partials [off[g] + c CH, min(off[g] + (c + 1) CH, off[g + 1])) into
// tmp[2 (g nch + c)] (zeros when the range is empty); k_reduce_partials then
// sums each grid's nch entries (offsets g nch).
template <int CH>
__global__ void k_reduce_partials_chunks(const double *partial, const int *off, int nch,
                                         double *tmp) {
  const int g = blockIdx.y, c = blockIdx.x;
  const int b0 = off[g] + c * CH, b1 = min(b0 + CH, off[g + 1]);
  double s = 0.0, m = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
    s += partial[2 * b];
    m = fmax(m, partial[2 * b + 1]);
  }
  block_reduce2<256>(s, m, &tmp[2 * (g * nch + c)], &tmp[2 * (g * nch + c) + 1]);
}

// Second stage: out[2g] = sum, out[2g+1] = max of tmp[g nch .. (g+1) nch).
__global__ void k_reduce_chunks(const double *tmp, int nch, int ngrid, double *out) {
  const int g = blockIdx.x;
  if (g >= ngrid) return;
  double s = 0.0, m = 0.0;
  for (int c = threadIdx.x; c < nch; c += blockDim.x) {
    s += tmp[2 * (g * nch + c)];
    m = fmax(m, tmp[2 * (g * nch + c) + 1]);
  }
  block_reduce2<256>(s, m, &out[2 * g], &out[2 * g + 1]);
}

// Fused residual + restriction (Sec. V.B.2): for each coarse cell, the 8 fine
// children give  u^H = uR = mean(u^h),  x^H = expm1(u^H),  f^H <- mean(d^h)
// (the coarse operator is added by k_fas_rhs).  One thread per coarse cell;
// optionally accumulates per-block (sum d^2, max |d|) of the fine residual.
template <typename T, bool BG>
__global__ void __launch_bounds__(256)
    k_resid_restrict(const Grid<T> *fine, const Grid<T> *coarse, const int *off, int ngrid,
                     const int *active, int fpar, int cpar, double *partial) {
  int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<T> F = view(fine, g, fpar);
  const Grid<T> C = view(coarse, g, cpar);
  float ss = 0.0f, mx = 0.0f;
  long long t = (long long)(blockIdx.x - off[g]) * blockDim.x + threadIdx.x;
  if (grid_active(active, F.field) && t < C.ncell) {
    int I, J, K;
    cell_ijk(C, t, I, J, K);
    T su = T(0), sd = T(0);
#pragma unroll
    for (int cz = 0; cz < 2; cz++)
#pragma unroll
      for (int cy = 0; cy < 2; cy++)
#pragma unroll
        for (int cx = 0; cx < 2; cx++) {
          int i = 2 * I + cx, j = 2 * J + cy, k = 2 * K + cz;
          long long c = idx3(F, i, j, k);
          T N, dN;
          cell_eval<T, BG>(F, i, j, k, c, N, dN);
          T d = N - rhs_at(F, c);
          sd += d;
          const float df_ = (float)d;
          ss = fmaf(df_, df_, ss);
          mx = fmaxf(mx, fabsf(df_));
          su += F.u[c];
        }
    T uh = su * T(0.125);
    C.uR[t] = uh;
    C.u[t] = uh;
    C.x[t] = m_expm1(uh);
    const_cast<T *>(C.f)[t] = sd * T(0.125);
  }
  // fine-grid residual norm partials (the residual after pre-smoothing)
  if (partial) block_reduce2f<256>(ss, mx, &partial[2 * blockIdx.x], &partial[2 * blockIdx.x + 1]);
}

// f^H = A^H(R u^h) - R d^h, in place over the R d^h stored in f (fs = 1, fo = 0).
template <typename T, bool BG>
__global__ void k_fas_rhs(const Grid<T> *grids, const int *off, int ngrid, const int *active,
                          int par) {
  int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<T> G = view(grids, g, par);
  if (!grid_active(active, G.field)) return;
  long long t = (long long)(blockIdx.x - off[g]) * blockDim.x + threadIdx.x;
  if (t >= G.ncell) return;
  int i, j, k;
  cell_ijk(G, t, i, j, k);
  T N, dN;
  cell_eval<T, BG>(G, i, j, k, t, N, dN);
  T *f = const_cast<T *>(G.f);
  f[t] = N - f[t];
}

// Truncation-error estimate of Sec. V.B.2 on the coarse grid of a V-cycle
// level, tau = A^H(R u) - R A^h(u), after k_resid_restrict has put R u (and
// its x) into the coarse grid and R d = R(A^h(u) - f^h) into its f: then
// R A^h(u) = f^H + R f^h.  The density terms of the operator cancel between
// the two and are not part of A.  One thread per coarse cell; per-block
// partials (sum tau^2, max |tau|).
template <typename T>
__global__ void __launch_bounds__(256)
    k_tau(const Grid<T> *fine, const Grid<T> *coarse, const int *off, int ngrid, int fpar,
          int cpar, double *partial) {
  int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<T> F = view(fine, g, fpar);
  const Grid<T> C = view(coarse, g, cpar);
  float ss = 0.0f, mx = 0.0f;
  long long t = (long long)(blockIdx.x - off[g]) * blockDim.x + threadIdx.x;
  if (t < C.ncell) {
    int I, J, K;
    cell_ijk(C, t, I, J, K);
    T N, dN;
    cell_eval<T, false>(C, I, J, K, t, N, dN);
    T rf = T(0);
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
      rf += rhs_at(F, idx3(F, i, j, k));
    }
    const T tau = N - (C.f[t] + rf * T(0.125));
    const float tf = (float)tau;
    ss = tf * tf;
    mx = fabsf(tf);
  }
  block_reduce2f<256>(ss, mx, &partial[2 * blockIdx.x], &partial[2 * blockIdx.x + 1]);
}

// u^h += P (u^H - R u^h), trilinear 27/9/3/1 over 64 (Sec. V.A.3); x^h refreshed.
// One thread per coarse cell writes its 8 children: the correction
// e = u^H - R u^h of the 3x3x3 coarse neighbourhood is interpolated separably
// (weights 3/4 for the containing cell, 1/4 for the neighbour on the child's
// side, per axis; their products are the paper's 27/9/3/1 over 64).
// Patches: coarse neighbours outside the grid contribute 0.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(const Grid<T> *fine, const Grid<T> *coarse,
                                                 const int *off, int ngrid, const int *active,
                                                 int fpar, int cpar) {
  int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<T> &Fg = fine[g];
  const Grid<T> &Cg = coarse[g];
  if (!grid_active(active, Fg.field)) return;
  const int c0 = Cg.n0, c1 = Cg.n1, c2 = Cg.n2;
  long long t = (long long)(blockIdx.x - off[g]) * blockDim.x + threadIdx.x;
  if (t >= (long long)c0 * c1 * c2) return;
  const T *__restrict__ uH = cpar ? Cg.u2 : Cg.u;
  const T *__restrict__ uR = Cg.uR;
  T *__restrict__ uf = fpar ? Fg.u2 : Fg.u;
  T *__restrict__ xf = fpar ? Fg.x2 : Fg.x;
  const bool dir = Fg.bnd != nullptr;
  int I, J, K;
  cell_ijk(Cg, t, I, J, K);
  // e over the 3x3x3 neighbourhood, index [dz][dy][dx] with d = -1, 0, 1
  T e[3][3][3];
#pragma unroll
  for (int dz = 0; dz < 3; dz++) {
    int kk = K + dz - 1;
    bool vz = kk >= 0 && kk < c2;
    kk = kk < 0 ? kk + c2 : (kk >= c2 ? kk - c2 : kk);
#pragma unroll
    for (int dy = 0; dy < 3; dy++) {
      int jj = J + dy - 1;
      bool vy = jj >= 0 && jj < c1;
      jj = jj < 0 ? jj + c1 : (jj >= c1 ? jj - c1 : jj);
#pragma unroll
      for (int dx = 0; dx < 3; dx++) {
        int ii = I + dx - 1;
        bool vx = ii >= 0 && ii < c0;
        ii = ii < 0 ? ii + c0 : (ii >= c0 ? ii - c0 : ii);
        long long ci = ((long long)kk * c1 + jj) * c0 + ii;
        bool valid = !dir || (vx && vy && vz);
        e[dz][dy][dx] = valid ? uH[ci] - uR[ci] : T(0);
      }
    }
  }
  const T w3 = T(0.75), w1 = T(0.25);
  // along x: child a = 0 uses (dx = 1, 0), a = 1 uses (dx = 1, 2)
  T ex[2][3][3];
#pragma unroll
  for (int dz = 0; dz < 3; dz++)
#pragma unroll
    for (int dy = 0; dy < 3; dy++) {
      ex[0][dz][dy] = w3 * e[dz][dy][1] + w1 * e[dz][dy][0];
      ex[1][dz][dy] = w3 * e[dz][dy][1] + w1 * e[dz][dy][2];
    }
  T exy[2][2][3];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int dz = 0; dz < 3; dz++) {
      exy[a][0][dz] = w3 * ex[a][dz][1] + w1 * ex[a][dz][0];
      exy[a][1][dz] = w3 * ex[a][dz][1] + w1 * ex[a][dz][2];
    }
  const int f0 = Fg.n0, f1 = Fg.n1;
#pragma unroll
  for (int cz = 0; cz < 2; cz++)
#pragma unroll
    for (int cy = 0; cy < 2; cy++) {
      const long long fi = ((long long)(2 * K + cz) * f1 + (2 * J + cy)) * f0 + 2 * I;
#pragma unroll
      for (int a = 0; a < 2; a++) {
        const T corr = w3 * exy[a][cy][1] + w1 * exy[a][cy][cz == 0 ? 0 : 2];
        const T un = uf[fi + a] + corr;
        uf[fi + a] = un;
        xf[fi + a] = m_expm1(un);
      }
    }
}

// Tiled FP32 prolongation and correction (same interpolation as k_prolong,
// evaluated in the order z, y, x): a block owns a 64 x 16 fine tile (32 x 8
// coarse cells) and a chunk of kc coarse planes.  The correction
// e = u^H - R u^h of the coarse tile plus a one-cell halo is staged in shared
// memory for planes K-1, K, K+1 (ring of three); for each of the fine planes
// 2K and 2K+1 the z-interpolated coarse plane is formed once in shared memory,
// and each thread corrects its fine x-pairs (y- then x-interpolation,
// weights 3/4 and 1/4 per axis) with 8-byte loads and stores, refreshing
// x = expm1(u).  Patches: coarse cells outside the grid contribute 0.
constexpr int kPlTX = 64, kPlTY = 16;
template <bool DIR>
__global__ void __launch_bounds__(256)
    k_prolong_tiled(const Grid<float> *fine, const Grid<float> *coarse, const int *off, int ngrid,
                    int kc, const int *active, int fpar, int cpar) {
  constexpr int CX = kPlTX / 2 + 2, CY = kPlTY / 2 + 2, CP = CX * CY;
  constexpr int NQ = (CP + 255) / 256;
  __shared__ float se[3][CP];
  __shared__ float sz[CP];
  const int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<float> &Fg = fine[g];
  const Grid<float> &Cg = coarse[g];
  if (!grid_active(active, Fg.field)) return;
  const int n0 = Fg.n0, n1 = Fg.n1;
  const int c0 = Cg.n0, c1 = Cg.n1, c2 = Cg.n2;
  const float *__restrict__ uH = cpar ? Cg.u2 : Cg.u;
  const float *__restrict__ uR = Cg.uR;
  float *__restrict__ uf = fpar ? Fg.u2 : Fg.u;
  float *__restrict__ xf = fpar ? Fg.x2 : Fg.x;
  const int ntx = (n0 + kPlTX - 1) / kPlTX, nty = (n1 + kPlTY - 1) / kPlTY;
  int b = blockIdx.x - off[g];
  const int X0 = (b % ntx) * kPlTX;
  b /= ntx;
  const int Y0 = (b % nty) * kPlTY;
  b /= nty;
  const int K0 = b * kc, K1 = min(K0 + kc, c2);
  // coarse staging table: entry q = threadIdx.x + k 256 of the CX x CY tile
  int qoff[NQ];
  bool qok[NQ];
#pragma unroll
  for (int k = 0; k < NQ; k++) {
    const int q = threadIdx.x + k * 256;
    qoff[k] = 0;
    qok[k] = false;
    if (q < CP) {
      int I = X0 / 2 - 1 + q % CX, J = Y0 / 2 - 1 + q / CX;
      if (DIR) {
        qok[k] = I >= 0 && I < c0 && J >= 0 && J < c1;
      } else {
        I = wrapmod(I, c0);
        J = wrapmod(J, c1);
        qok[k] = true;
      }
      qoff[k] = J * c0 + I;
    }
  }
  const long long cplane = (long long)c0 * c1;
  // wrapped index of the next coarse plane to stage
  int kw = DIR ? K0 - 1 : wrapmod(K0 - 1, c2);
  auto stage = [&](int slot, int K) {
    const bool vz = !DIR || (K >= 0 && K < c2);
    const long long zo = (long long)kw * cplane;
#pragma unroll
    for (int k = 0; k < NQ; k++) {
      const int q = threadIdx.x + k * 256;
      if (q >= CP) continue;
      float e = 0.0f;
      if (qok[k] && vz) {
        const long long i = zo + qoff[k];
        e = uH[i] - uR[i];
      }
      se[slot][q] = e;
    }
    kw = DIR ? kw + 1 : (kw + 1 == c2 ? 0 : kw + 1);
  };
  const int lane = threadIdx.x & 31, r0 = threadIdx.x >> 5;  // pair, first row
  const long long fplane = (long long)n0 * n1;
  const float w3 = 0.75f, w1 = 0.25f;
  stage(0, K0 - 1);
  stage(1, K0);
  int sm = 0, sc = 1, sp = 2;  // ring slots of planes K-1, K, K+1
  for (int K = K0; K < K1; K++) {
    stage(sp, K + 1);
    __syncthreads();
#pragma unroll
    for (int cz = 0; cz < 2; cz++) {
      const int so = cz ? sp : sm;
      for (int q = threadIdx.x; q < CP; q += 256) sz[q] = w3 * se[sc][q] + w1 * se[so][q];
      __syncthreads();
      const int k = 2 * K + cz;
      const int fx = X0 + 2 * lane;
#pragma unroll
      for (int rr = 0; rr < 2; rr++) {
        const int row = r0 + 8 * rr;
        const int j = Y0 + row;
        if (j >= n1 || fx >= n0) continue;
        const int jy = row / 2 + 1, jy2 = (row & 1) ? jy + 1 : jy - 1;
        const int ix = lane + 1;
        const float *za = sz + jy * CX, *zb = sz + jy2 * CX;
        const float em = w3 * za[ix - 1] + w1 * zb[ix - 1];
        const float e0 = w3 * za[ix] + w1 * zb[ix];
        const float ep = w3 * za[ix + 1] + w1 * zb[ix + 1];
        const long long fi = (long long)k * fplane + (long long)j * n0 + fx;
        const float2 u = *reinterpret_cast<const float2 *>(uf + fi);
        const float un0 = u.x + (w3 * e0 + w1 * em);
        const float un1 = u.y + (w3 * e0 + w1 * ep);
        *reinterpret_cast<float2 *>(uf + fi) = make_float2(un0, un1);
        *reinterpret_cast<float2 *>(xf + fi) = make_float2(m_expm1(un0), m_expm1(un1));
      }
      __syncthreads();
    }
    const int t = sm;
    sm = sc;
    sc = sp;
    sp = t;
  }
}

// Block sum of two values (all threads get the result).
template <int NT, typename A>
__device__ __forceinline__ void block_sum2(A a, A b, A &ra, A &rb) {
  __shared__ A sa[NT / 32], sb[NT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  A ta = A(0), tb = A(0);
  for (int q = 0; q < NT / 32; q++) {
    ta += sa[q];
    tb += sb[q];
  }
  ra = ta;
  rb = tb;
}

// Block sum of one value per thread into *out (shared), written by thread 0.
template <int NT, typename A>
__device__ __forceinline__ void block_sum1(A a, A *out) {
  __shared__ A sa[NT / 32];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sa[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    A t = A(0);
    for (int q = 0; q < NT / 32; q++) t += sa[q];
    *out = t;
  }
}

// Coarsest level: one block per grid, Newton-Gauss-Seidel sweeps until
// rms <= max(rel * rms0, abs_floor) (at least one sweep, at most maxit).
// stop_on_stall also stops when a sweep does not lower the rms.
// meanfix (periodic grids): after every sweep, one Newton step on a constant
// shift c of the whole grid.  On a periodic grid the flux terms telescope, so
// sum_i (N_i - f_i) depends on c only through the mass term, whose derivative
// is -(beta/2) sum_i F_i e^{-d_i/2}; the step removes the error of the
// constant mode, which plain relaxation damps by only ~beta/(12 alpha) per
// sweep when the Laplacian dominates (stiff coarsest problems).
template <typename T, bool BG, int NT>
__global__ void __launch_bounds__(NT) k_coarsest(const Grid<T> *grids, int ngrid, double rel,
                                                 double abs_floor, int maxit, int stop_on_stall,
                                                 const int *active, int par, int meanfix) {
  int g = blockIdx.x;
  if (g >= ngrid) return;
  Grid<T> G = view(grids, g, par);
  if (!grid_active(active, G.field)) return;
  // sums in the precision of the grid: FP64 arithmetic runs at 1/64 of the
  // FP32 rate here, and the FP32 levels' stopping test needs no more
  using A = typename std::conditional<sizeof(T) == 4, float, double>::type;
  __shared__ A red_s;
  __shared__ int stop;
  const long long n = G.ncell;
  // a grid of up to 16 KB per array is relaxed in shared memory (u and its
  // x cache copied in and back; the same updates in the same order)
  constexpr int CAPN = 16384 / (int)sizeof(T);
  __shared__ T cs_u[CAPN], cs_x[CAPN];
  T *const gu = G.u;
  T *const gx = G.x;
  const bool local = n <= CAPN;
  if (local) {
    for (long long t = threadIdx.x; t < n; t += NT) {
      cs_u[t] = gu[t];
      cs_x[t] = gx[t];
    }
    __syncthreads();
    G.u = cs_u;
    G.x = cs_x;
  }
  const int hx = G.n0 >> 1;
  const long long nh = (long long)hx * G.n1 * G.n2;
  const bool shift = meanfix && G.bnd == nullptr;
  A thr = A(0), prev = A(0);
  for (int it = -1; it < maxit; it++) {
    if (it >= 0) {
      for (int colour = 0; colour < 2; colour++) {
        for (long long t = threadIdx.x; t < nh; t += NT) {
          int i, j, k;
          cell_ijk(G, 2 * t, i, j, k);
          ngs_update<T, BG>(G, i + ((j + k + colour) & 1), j, k);
        }
        __syncthreads();
      }
      if (shift) {
        A S = A(0), D = A(0);
        for (long long t = threadIdx.x; t < n; t += NT) {
          int i, j, k;
          cell_ijk(G, t, i, j, k);
          T N, dN;
          cell_eval<T, BG>(G, i, j, k, t, N, dN);
          S += (A)(N - rhs_at(G, t));
          const T Ei = BG ? (T)G.Ebg[t] : T(1);
          const T F = BG ? m_rsqrt(Ei) : T(1);
          D += A(0.5) * (A)G.beta * (A)(F * m_rsqrt(T(1) + G.x[t]));
        }
        A St, Dt;
        block_sum2<NT, A>(S, D, St, Dt);
        A c = Dt > A(0) ? St / Dt : A(0);
        const A cap = (A)G.cap;
        c = c > cap ? cap : (c < -cap ? -cap : c);
        __syncthreads();
        for (long long t = threadIdx.x; t < n; t += NT) {
          const T un = G.u[t] + (T)c;
          G.u[t] = un;
          G.x[t] = m_expm1(un);
        }
        __syncthreads();
      }
    }
    A s = A(0);
    for (long long t = threadIdx.x; t < n; t += NT) {
      int i, j, k;
      cell_ijk(G, t, i, j, k);
      T N, dN;
      cell_eval<T, BG>(G, i, j, k, t, N, dN);
      const A d = (A)(N - rhs_at(G, t));
      s += d * d;
    }
    block_sum1<NT, A>(s, &red_s);
    __syncthreads();
    if (threadIdx.x == 0) {
      const A rms = sqrt(red_s / (A)n);
      int st = 0;
      if (it < 0) {
        thr = fmax((A)rel * rms, (A)abs_floor);
        if (rms <= thr) st = 1;
      } else {
        if (rms <= thr) st = 1;
        if (stop_on_stall && rms >= prev) st = 1;
      }
      prev = rms;
      stop = st;
    }
    __syncthreads();
    if (stop) break;
  }
  if (local) {
    __syncthreads();
    for (long long t = threadIdx.x; t < n; t += NT) {
      gu[t] = cs_u[t];
      gx[t] = cs_x[t];
    }
  }
}

// Generic 8-child average (full weighting on cell-centred grids).
template <typename T>
__global__ void k_restrict_avg(const T *fine, int nf0, int nf1, int nf2, T *coarse) {
  int nc0 = nf0 >> 1, nc1 = nf1 >> 1, nc2 = nf2 >> 1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nc0 * nc1 * nc2) return;
  int I = (int)(t % nc0);
  long long r = t / nc0;
  int J = (int)(r % nc1);
  int K = (int)(r / nc1);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 8; c++) {
    int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
    s += fine[((long long)k * nf1 + j) * nf0 + i];
  }
  coarse[t] = s * T(0.125);
}

// ---------------------------------------------------------------------------
// Tiled FP32 smoother with temporal blocking: S full red-black sweeps per pass.
//
// A block owns a TX x TY tile of one grid and a chunk of zc planes; it marches
// along z with a ring of 2S+2 planes (tile plus a halo of 2S cells in x and y)
// in shared memory.  At the step that loads plane p, stage q (q = 0 .. 2S-1,
// colour q & 1: red first) updates plane p-1-q on the tile grown by 2S-1-q
// cells, so that plane p-2S is final and its tile cells are written out.
// Halo cells are updated redundantly by neighbouring blocks from identical
// inputs; a pass reads the current buffer and writes the other one (blocks
// load their halos from the unmodified input), which makes the result equal to
// S sweeps of k_smooth.  x = expm1(u) is recomputed from u on load and written
// in place for the kernels that follow.
template <int S, int TX, int TY>
struct TileCfg {
  static constexpr int H = 2 * S;                   // halo
  static constexpr int LX = TX + 2 * H, LY = TY + 2 * H, PL = LX * LY, NS = 2 * S + 2;
  static constexpr int PX = LX / 2;                 // x-pairs per row
  static constexpr int RPT = 2;                     // rows per thread (independent updates)
  static constexpr int NT = PX * LY / RPT;          // threads per block
  static constexpr size_t smem(bool bg) { return (size_t)NS * PL * sizeof(float) * (bg ? 5 : 3); }
  static_assert(LY % RPT == 0, "rows must split evenly over threads");
};

// ---------------------------------------------------------------------------
// Tiled FP32 smoother with temporal blocking: S full red-black sweeps per pass.
//
// A block owns a TX x TY tile of one grid and a chunk of zc planes; it marches
// along z with a ring of 2S+2 planes (tile plus a halo of 2S cells in x and y)
// in shared memory.  At the step that loads plane p, stage q (q = 0 .. 2S-1,
// colour q & 1: red first) updates plane p-1-q on the tile grown by 2S-1-q
// cells, so that plane p-2S is final and its tile cells are written out.
// Halo cells are updated redundantly by neighbouring blocks from identical
// inputs; a pass reads the current buffer and writes the other one (blocks
// load their halos from the unmodified input), which makes the result equal to
// S sweeps of k_smooth.  The x = expm1(u) cache ping-pongs with u.
//
// Each thread owns one x-pair in each of RPT rows (LY/RPT rows apart) for the
// whole pass: it loads and stores its pairs with 8-byte accesses (x-pairs
// start at even x, and n0 is even, so a pair never straddles the periodic
// seam), and at every stage it updates, in each of its rows, the one cell of
// its pair that has the stage's colour if that cell lies in the stage's
// region; the RPT updates are independent, which gives the scheduler
// instruction-level parallelism.  The right-hand side is kept in shared memory
// with the plane.  The global loads of plane p+1 are
// issued into registers before the stages of step p and stored to shared
// memory after them.
template <bool BG, bool DIR, int S, int TX, int TY>
__global__ void __launch_bounds__(TileCfg<S, TX, TY>::NT)
    k_smooth_tiled(const Grid<float> *grids, const int *off, int ngrid, int zc, const int *active,
                   int par) {
  using C = TileCfg<S, TX, TY>;
  constexpr int H = C::H, LX = C::LX, LY = C::LY, PL = C::PL, NS = C::NS, PX = C::PX;
  constexpr int RPT = C::RPT;
  extern __shared__ float smem[];
  float *sd = smem;
  float *sx = smem + NS * PL;
  float *sf = smem + 2 * NS * PL;
  float *sub = smem + 3 * NS * PL;
  float *sE = smem + 4 * NS * PL;
  const int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<float> &Gg = grids[g];
  if (!grid_active(active, Gg.field)) return;
  const float *__restrict__ uin = par ? Gg.u2 : Gg.u;
  float *__restrict__ uout = par ? Gg.u : Gg.u2;
  const float *__restrict__ xin = par ? Gg.x2 : Gg.x;
  float *__restrict__ xout = par ? Gg.x : Gg.x2;
  const float *__restrict__ fin = Gg.f;
  const float *__restrict__ ubin = Gg.ubg;
  const float *__restrict__ Ein = Gg.Ebg;
  const float fs = Gg.fs, fo = Gg.fo, ah = Gg.ah, beta = Gg.beta, cap = Gg.cap,
              relax = Gg.relax;
  const int n0 = Gg.n0, n1 = Gg.n1, n2 = Gg.n2;
  constexpr bool dir = DIR;  // patch (Dirichlet faces) or periodic grid
  const int ntx = (n0 + TX - 1) / TX, nty = (n1 + TY - 1) / TY;
  int b = blockIdx.x - off[g];
  const int X0 = (b % ntx) * TX;
  b /= ntx;
  const int Y0 = (b % nty) * TY;
  b /= nty;
  const int Z0 = b * zc;
  const int Z1 = min(Z0 + zc, n2);

  const int ly0 = threadIdx.x / PX;
  const int lx0 = 2 * (threadIdx.x - ly0 * PX);
  const int gx0 = X0 - H + lx0;
  int gxw0;
  if (dir)
    gxw0 = (gx0 < 0 || gx0 >= n0) ? -1 : gx0;
  else
    gxw0 = wrapmod(gx0, n0);
  int ly[RPT], gy[RPT], gyw[RPT], rowo[RPT];
  bool mine[RPT], writer[RPT];
#pragma unroll
  for (int r = 0; r < RPT; r++) {
    ly[r] = ly0 + r * (LY / RPT);
    gy[r] = Y0 - H + ly[r];
    if (dir)
      gyw[r] = (gy[r] < 0 || gy[r] >= n1) ? -1 : gy[r];
    else
      gyw[r] = wrapmod(gy[r], n1);
    mine[r] = gyw[r] >= 0 && gxw0 >= 0;
    rowo[r] = ly[r] * LX + lx0;
    writer[r] = mine[r] && ly[r] >= H && ly[r] < H + TY && lx0 >= H && lx0 < H + TX &&
                gx0 < n0 && gy[r] < n1;
  }

  float2 pd[RPT], px[RPT], pf[RPT], pu[RPT], pE[RPT];
#pragma unroll
  for (int r = 0; r < RPT; r++) {
    pd[r] = make_float2(0.f, 0.f);
    px[r] = pd[r];
    pf[r] = pd[r];
    pu[r] = pd[r];
    pE[r] = make_float2(1.f, 1.f);
  }
  auto fetch = [&](int p) {
    if (dir && (p < 0 || p >= n2)) return;
    const long long zo = (long long)wrapmod(p, n2) * n1;
#pragma unroll
    for (int r = 0; r < RPT; r++) {
      if (!mine[r]) continue;
      const long long gi = (zo + gyw[r]) * n0 + gxw0;
      pd[r] = *reinterpret_cast<const float2 *>(uin + gi);
      px[r] = *reinterpret_cast<const float2 *>(xin + gi);
      if (fin) pf[r] = *reinterpret_cast<const float2 *>(fin + gi);  // scaled at commit
      if (BG) {
        pu[r] = *reinterpret_cast<const float2 *>(ubin + gi);
        pE[r] = *reinterpret_cast<const float2 *>(Ein + gi);
      }
    }
  };
  auto commit = [&](int p) {
    const int base = wrapmod(p, NS) * PL;
#pragma unroll
    for (int r = 0; r < RPT; r++) {
      const int o = base + rowo[r];
      sd[o] = pd[r].x;
      sd[o + 1] = pd[r].y;
      sx[o] = px[r].x;
      sx[o + 1] = px[r].y;
      sf[o] = fin ? fs * (pf[r].x - fo) : 0.0f;
      sf[o + 1] = fin ? fs * (pf[r].y - fo) : 0.0f;
      if (BG) {
        sub[o] = pu[r].x;
        sub[o + 1] = pu[r].y;
        sE[o] = pE[r].x;
        sE[o + 1] = pE[r].y;
      }
    }
  };
  auto stage = [&](int p, int q) {
    const int m = p - 1 - q;
    const int R = 2 * S - 1 - q;
    const int colour = q & 1;
    if (m < Z0 - R || m >= Z1 + R || (dir && (m < 0 || m >= n2))) return;
    const int sl = wrapmod(m, NS), slm = wrapmod(m - 1, NS), slp = wrapmod(m + 1, NS);
#pragma unroll
    for (int r = 0; r < RPT; r++) {
      const int par01 = (X0 - H + gy[r] + m + colour) & 1;
      const int lx = lx0 + par01;
      if (!mine[r] || ly[r] < H - R || ly[r] >= H + TY + R || lx < H - R || lx >= H + TX + R)
        continue;
      const int li = rowo[r] + par01;
      const int o = sl * PL + li;
      const float di = sd[o], xi = sx[o];
      const float Ei = BG ? sE[o] : 1.0f;
      const float ubi = BG ? sub[o] : 0.0f;
      const float Bi = BG ? Ei + Ei * xi : 1.0f + xi;
      OpAcc<float, BG> A(di, Ei, xi, Bi, ubi);
      const int gxw = gxw0 + par01, gyr = gyw[r];
#define FR_NB(OFF) A.reg(sd[OFF], sx[OFF], BG ? sub[OFF] : 0.0f, BG ? sE[OFF] : 1.0f)
      if (dir && gxw == 0)
        A.ghost(face_value(Gg, 0, gxw, gyr, m));
      else
        FR_NB(o - 1);
      if (dir && gxw == n0 - 1)
        A.ghost(face_value(Gg, 1, gxw, gyr, m));
      else
        FR_NB(o + 1);
      if (dir && gyr == 0)
        A.ghost(face_value(Gg, 2, gxw, gyr, m));
      else
        FR_NB(o - LX);
      if (dir && gyr == n1 - 1)
        A.ghost(face_value(Gg, 3, gxw, gyr, m));
      else
        FR_NB(o + LX);
      if (dir && m == 0)
        A.ghost(face_value(Gg, 4, gxw, gyr, m));
      else
        FR_NB(slm * PL + li);
      if (dir && m == n2 - 1)
        A.ghost(face_value(Gg, 5, gxw, gyr, m));
      else
        FR_NB(slp * PL + li);
#undef FR_NB
      float acc, dacc;
      A.done(acc, dacc);
      float N, dN;
      finish_op(xi, Ei, acc, dacc, ah, beta, BG, N, dN);
      float du = newton_du(N, sf[o], dN, relax);
      du = fminf(fmaxf(du, -cap), cap);
      const float dn = di + du;
      sd[o] = dn;
      sx[o] = m_expm1(dn);
    }
  };

  fetch(Z0 - H);
  commit(Z0 - H);
  __syncthreads();
  for (int p = Z0 - H; p < Z1 + H; p++) {
    const bool more = p + 1 < Z1 + H;
    if (more) fetch(p + 1);
#pragma unroll
    for (int q = 0; q < 2 * S; q++) {
      stage(p, q);
      __syncthreads();
    }
    const int w = p - H;
    if (w >= Z0 && w < Z1) {
      const int base = wrapmod(w, NS) * PL;
#pragma unroll
      for (int r = 0; r < RPT; r++) {
        if (!writer[r]) continue;
        const int o = base + rowo[r];
        const long long gi = ((long long)w * n1 + gy[r]) * n0 + gx0;
        *reinterpret_cast<float2 *>(uout + gi) = make_float2(sd[o], sd[o + 1]);
        *reinterpret_cast<float2 *>(xout + gi) = make_float2(sx[o], sx[o + 1]);
      }
    }
    if (more) commit(p + 1);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Tiled FP32 smoother, one full red-black sweep per pass, rows of the tile
// distributed over warps.
//
// Same schedule as k_smooth_tiled with S = 1: a block owns a 64 x TY tile of
// one grid and an even number zc of planes and marches along z.  At the step
// that brings in plane p it updates the red cells of plane p-1 on the tile
// grown by one cell, then the black cells of plane p-2 on the tile, and
// writes plane p-2 out; the halo of two cells is loaded from the input buffer
// and the result goes to the other buffer, so the pass equals one sweep of
// k_smooth.  What differs is the layout and the work mapping:
//  * each plane is stored split by colour.  The six neighbours of a cell have
//    the other colour, so for the colour-c cell of x-pair e they are entries
//    e and e -+ 1 (x), e -+ PX (y) of the other colour's array, and entry e of
//    it in planes m -+ 1 (z); u and x = expm1(u) are interleaved, so each
//    neighbour is one 8-byte shared-memory access, stride-1 across a warp;
//  * a warp updates whole rows of pairs (lane = pair), so the position of the
//    colour-c cell inside the pair is the same for the whole warp, and only
//    the one extra cell per row of the grown red region (at the left or right
//    end of the row) is handled by two warps as a separate column task;
//  * the global loads of a plane go through fixed per-thread tables (row
//    offset, flags) built once, and the next plane's wrapped offset advances
//    by one plane per step.
template <int TY>
struct RBCfg {
  static constexpr int TX = 64, H = 2;
  static constexpr int LX = TX + 2 * H, LY = TY + 2 * H, PX = LX / 2, PP = PX * LY;
  static constexpr int NW = TY / 2, NT = 32 * NW;  // warps, threads
  static constexpr int NLD = (PP + NT - 1) / NT;   // plane-load rounds per thread
  // ring slots of (u, x) [and (ub, E)]; the right-hand side is kept per
  // colour: a red half-plane is read one step after it is loaded, a black one
  // two steps after, so two red and three black half-slots suffice
  static constexpr int NS = 4, NFR = 2, NFB = 3;
  static constexpr int NE = TY + 2;                // edge cells of the red region
  static constexpr size_t smem(bool bg) {
    return (size_t)NS * 2 * PP * sizeof(float2) * (bg ? 2 : 1) +
           (size_t)(NFR + NFB) * PP * sizeof(float);
  }
  // resident blocks per SM that shared memory allows, at most 3 (a fourth
  // block of 256 threads caps the registers at 64 per thread: measured slower)
  static constexpr int minb(bool bg) {
    const int bysm = (int)(228 * 1024 / (smem(bg) + 1024));
    const int byth = 1024 / NT < 3 ? 1024 / NT : 3;
    return bysm < 1 ? 1 : (bysm < byth ? bysm : byth);
  }
  static_assert(TY % 4 == 0 && NW >= 4 && NE <= 64, "tile height");
};

template <bool BG, bool DIR, int TY>
__global__ void __launch_bounds__(RBCfg<TY>::NT, RBCfg<TY>::minb(BG))
    k_smooth_rb(const Grid<float> *grids, const int *off, int ngrid, int zc, const int *active,
                int par) {
  using C = RBCfg<TY>;
  constexpr int TX = C::TX, H = C::H, PX = C::PX, PP = C::PP, NW = C::NW, NT = C::NT;
  constexpr int NLD = C::NLD, NS = C::NS, NFR = C::NFR, NFB = C::NFB;
  extern __shared__ float4 smem_rb[];
  // plain form: (u, x) per cell; correction form: (u, x, ub, E) per cell, so a
  // neighbour is one 16-byte access (half the shared-memory instructions)
  float2 *sux = reinterpret_cast<float2 *>(smem_rb);  // [NS][2][PP] (plain)
  float4 *s4 = smem_rb;                               // [NS][2][PP] (correction form)
  // right-hand side: red half-slots [NFR][PP], then black half-slots [NFB][PP]
  float *sfv = reinterpret_cast<float *>(sux + NS * 2 * PP * (BG ? 2 : 1));
  // cell e of a slot/colour offset: (u, x, ub, E); ub = 0, E = 1 in the plain form
  auto cell = [&](int i) -> float4 {
    if (BG) return s4[i];
    const float2 v = sux[i];
    return make_float4(v.x, v.y, 0.f, 1.f);
  };
  auto put_ux = [&](int i, float u, float x) {
    if (BG)
      *reinterpret_cast<float2 *>(&s4[i]) = make_float2(u, x);
    else
      sux[i] = make_float2(u, x);
  };
  const int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<float> &Gg = grids[g];
  if (!grid_active(active, Gg.field)) return;
  const float *__restrict__ uin = par ? Gg.u2 : Gg.u;
  float *__restrict__ uout = par ? Gg.u : Gg.u2;
  const float *__restrict__ xin = par ? Gg.x2 : Gg.x;
  float *__restrict__ xout = par ? Gg.x : Gg.x2;
  const float *__restrict__ fin = Gg.f;
  const float *__restrict__ ubin = Gg.ubg;
  const float *__restrict__ Ein = Gg.Ebg;
  const float fs = Gg.fs, fo = Gg.fo, ah = Gg.ah, beta = Gg.beta, cap = Gg.cap,
              relax = Gg.relax;
  const int n0 = Gg.n0, n1 = Gg.n1, n2 = Gg.n2;
  const int ntx = (n0 + TX - 1) / TX, nty = (n1 + TY - 1) / TY;
  int b = blockIdx.x - off[g];
  const int X0 = (b % ntx) * TX;
  b /= ntx;
  const int Y0 = (b % nty) * TY;
  b /= nty;
  const int Z0 = b * zc;  // zc is even, so plane p has the parity of its step
  const int Z1 = min(Z0 + zc, n2);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long plane = (long long)n0 * n1;

  // plane-load tables: pair q = threadIdx.x + k NT of the (TX + 4) x (TY + 4) tile
  int roff[NLD];
  unsigned ldf[NLD];  // bit 0: load, bit 1: write out, bit 2: parity of the row
#pragma unroll
  for (int k = 0; k < NLD; k++) {
    const int q = threadIdx.x + k * NT;
    roff[k] = 0;
    ldf[k] = 0;
    if (q < PP) {
      const int ly = q / PX, px = q - (q / PX) * PX;
      const int gx = X0 - H + 2 * px, gy = Y0 - H + ly;
      bool ok;
      int gxw, gyw;
      if (DIR) {
        ok = gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
        gxw = gx;
        gyw = gy;
      } else {
        ok = true;
        gxw = wrapmod(gx, n0);
        gyw = wrapmod(gy, n1);
      }
      const bool wr = ok && ly >= H && ly < H + TY && px >= 1 && px < PX - 1 && gx < n0 &&
                      gy < n1;
      roff[k] = ok ? gyw * n0 + gxw : 0;
      ldf[k] = (ok ? 1u : 0u) | (wr ? 2u : 0u) | ((unsigned)(ly & 1) << 2);
    }
  }
  float2 pd[NLD], pq[NLD], pf[NLD], pu[NLD], pE[NLD];
#pragma unroll
  for (int k = 0; k < NLD; k++) {
    pd[k] = make_float2(0.f, 0.f);
    pq[k] = pd[k];
    pf[k] = pd[k];
    pu[k] = pd[k];
    pE[k] = make_float2(1.f, 1.f);
  }
  auto fetch = [&](long long zoff) {
#pragma unroll
    for (int k = 0; k < NLD; k++) {
      if (!(ldf[k] & 1u)) continue;
      const long long gi = zoff + roff[k];
      pd[k] = *reinterpret_cast<const float2 *>(uin + gi);
      pq[k] = *reinterpret_cast<const float2 *>(xin + gi);
      // raw values: arithmetic on them here would wait for the load
      if (fin) pf[k] = *reinterpret_cast<const float2 *>(fin + gi);
      if (BG) {
        pu[k] = *reinterpret_cast<const float2 *>(ubin + gi);
        pE[k] = *reinterpret_cast<const float2 *>(Ein + gi);
      }
    }
  };
  // plane of parity pb into (u, x) slot offset so and the f half-slot offsets
  // fr (red) and fb (black); the even-x cell of a pair has colour (y + z) & 1
  auto commit = [&](int pb, int so, int fr, int fb) {
#pragma unroll
    for (int k = 0; k < NLD; k++) {
      const int q = threadIdx.x + k * NT;
      if (q >= PP) continue;
      const int c0 = (int)((ldf[k] >> 2) & 1u) ^ pb;
      const int i0 = so + c0 * PP + q, i1 = so + (c0 ^ 1) * PP + q;
      if (BG) {
        s4[i0] = make_float4(pd[k].x, pq[k].x, pu[k].x, pE[k].x);
        s4[i1] = make_float4(pd[k].y, pq[k].y, pu[k].y, pE[k].y);
      } else {
        sux[i0] = make_float2(pd[k].x, pq[k].x);
        sux[i1] = make_float2(pd[k].y, pq[k].y);
      }
      sfv[(c0 ? fb : fr) + q] = fin ? fs * (pf[k].x - fo) : 0.0f;
      sfv[(c0 ? fr : fb) + q] = fin ? fs * (pf[k].y - fo) : 0.0f;
    }
  };
  // Newton update of the colour-Q cell of pair (ly, px) of plane m; s is its x
  // position in the pair; oc, om, op are the (u, x) slot offsets of planes m,
  // m - 1, m + 1 (colour Q's array at oc + Q PP), ofq the f offset.  Split in
  // three: gather (the shared-memory reads), compute (registers and, on patch
  // faces, the boundary values) and store, so that two independent updates
  // can read all their operands before either writes (the compiler cannot
  // tell that a write of one colour never feeds a read of the other).
  struct CellIn {
    float4 own, lft, rgt, nym, nyp, nzm, nzp;
    float f;
    int e, gx, gy;
  };
  auto gather = [&](auto Qc, int ly, int px, int s, int oc, int om, int op, int ofq) {
    constexpr int Q = decltype(Qc)::value;
    CellIn c;
    c.gx = X0 - H + 2 * px + s;
    c.gy = Y0 - H + ly;
    const int e = ly * PX + px;
    c.e = e;
    const int cq = Q * PP, co = (Q ^ 1) * PP;
    const int V = oc + co;
    const int ex = s ? e + 1 : e - 1;
    c.own = cell(oc + cq + e);
    const float4 nin = cell(V + e), nxo = cell(V + ex);
    c.lft = s ? nin : nxo;
    c.rgt = s ? nxo : nin;
    c.nym = cell(V + e - PX);
    c.nyp = cell(V + e + PX);
    c.nzm = cell(om + co + e);
    c.nzp = cell(op + co + e);
    c.f = sfv[ofq + e];
    return c;
  };
  auto inside = [&](const CellIn &c) {
    return !DIR || (c.gx >= 0 && c.gx < n0 && c.gy >= 0 && c.gy < n1);
  };
  // new (u, x) of the cell
  auto compute = [&](const CellIn &c, int m) -> float2 {
    const int gx = c.gx, gy = c.gy;
    const float di = c.own.x, xi = c.own.y;
    const float Ei = BG ? c.own.w : 1.0f;
    const float ubi = BG ? c.own.z : 0.0f;
    const float Bi = BG ? Ei + Ei * xi : 1.0f + xi;
    OpAcc<float, BG> A(di, Ei, xi, Bi, ubi);
    if (DIR && gx == 0)
      A.ghost(face_value(Gg, 0, gx, gy, m));
    else
      A.reg(c.lft.x, c.lft.y, c.lft.z, c.lft.w);
    if (DIR && gx == n0 - 1)
      A.ghost(face_value(Gg, 1, gx, gy, m));
    else
      A.reg(c.rgt.x, c.rgt.y, c.rgt.z, c.rgt.w);
    if (DIR && gy == 0)
      A.ghost(face_value(Gg, 2, gx, gy, m));
    else
      A.reg(c.nym.x, c.nym.y, c.nym.z, c.nym.w);
    if (DIR && gy == n1 - 1)
      A.ghost(face_value(Gg, 3, gx, gy, m));
    else
      A.reg(c.nyp.x, c.nyp.y, c.nyp.z, c.nyp.w);
    if (DIR && m == 0)
      A.ghost(face_value(Gg, 4, gx, gy, m));
    else
      A.reg(c.nzm.x, c.nzm.y, c.nzm.z, c.nzm.w);
    if (DIR && m == n2 - 1)
      A.ghost(face_value(Gg, 5, gx, gy, m));
    else
      A.reg(c.nzp.x, c.nzp.y, c.nzp.z, c.nzp.w);
    float acc, dacc;
    A.done(acc, dacc);
    float N, dN;
    finish_op(xi, Ei, acc, dacc, ah, beta, BG, N, dN);
    float du = newton_du(N, c.f, dN, relax);
    du = fminf(fmaxf(du, -cap), cap);
    const float dn = di + du;
    return make_float2(dn, m_expm1(dn));
  };
  auto update = [&](auto Qc, int ly, int px, int s, int m, int oc, int om, int op, int ofq) {
    constexpr int Q = decltype(Qc)::value;
    const CellIn c = gather(Qc, ly, px, s, oc, om, op, ofq);
    if (!inside(c)) return;
    const float2 r = compute(c, m);
    put_ux(oc + Q * PP + c.e, r.x, r.y);
  };
  // two updates of the same colour and plane (rows lya and lyb): both gather
  // before either stores, and their arithmetic interleaves
  auto update2 = [&](auto Qc, int lya, int lyb, int px, int s, int m, int oc, int om, int op,
                     int ofq) {
    constexpr int Q = decltype(Qc)::value;
    const CellIn a = gather(Qc, lya, px, s, oc, om, op, ofq);
    const CellIn b = gather(Qc, lyb, px, s, oc, om, op, ofq);
    if (DIR) {
      if (inside(a)) {
        const float2 r = compute(a, m);
        put_ux(oc + Q * PP + a.e, r.x, r.y);
      }
      if (inside(b)) {
        const float2 r = compute(b, m);
        put_ux(oc + Q * PP + b.e, r.x, r.y);
      }
    } else {
      const float2 ra = compute(a, m), rb = compute(b, m);
      put_ux(oc + Q * PP + a.e, ra.x, ra.y);
      put_ux(oc + Q * PP + b.e, rb.x, rb.y);
    }
  };

  const int P0 = Z0 - H, PE = Z1 + H;
  constexpr int SLOT = 2 * PP;
  // wrapped index of the plane being loaded (periodic grids)
  int pw = DIR ? P0 : wrapmod(P0, n2);
  if (!DIR || (P0 >= 0 && P0 < n2)) fetch((long long)pw * plane);
  // f half-slots: red of plane m at (m & 1) PP, black at (NFR + b) PP with b
  // advancing by one per plane (mod NFB)
  commit(P0 & 1, 0, (P0 & 1) * PP, NFR * PP);
  __syncthreads();
  int cur = 0, bcur = 0;  // ring slot of plane p, black f half-slot of plane p
  for (int p = P0; p < PE; p++) {
    const int pb = p & 1;
    const bool more = p + 1 < PE;
    pw = DIR ? p + 1 : (pw + 1 == n2 ? 0 : pw + 1);
    if (more && (!DIR || (pw >= 0 && pw < n2))) fetch((long long)pw * plane);
    const int o0 = cur * SLOT, o1 = ((cur + 3) & 3) * SLOT, o2 = ((cur + 2) & 3) * SLOT,
              o3 = ((cur + 1) & 3) * SLOT;  // planes p, p-1, p-2, p-3
    const int bnx = bcur == NFB - 1 ? 0 : bcur + 1;  // black f of plane p-2, then p+1
    const int f1 = ((p - 1) & 1) * PP;  // red f of plane p-1 (then of p+1)
    const int f2 = (NFR + bnx) * PP;
    // red cells of plane p-1 on the tile grown by one
    {
      const int m = p - 1;
      if (m >= Z0 - 1 && m < Z1 + 1 && (!DIR || (m >= 0 && m < n2))) {
        const int s = (w + 1 + pb + 1) & 1;  // rows 1 + w + j NW: parity of (ly + m) = s
        update2(std::integral_constant<int, 0>{}, 1 + w, 1 + w + NW, 1 + lane, s, m, o1, o2, o0,
                f1);
        if (w < 2)
          update(std::integral_constant<int, 0>{}, 1 + w + 2 * NW, 1 + lane, s, m, o1, o2, o0,
                 f1);
        if (w == 2 || w == 3) {
          const int idx = (w - 2) * 32 + lane;
          if (idx < C::NE) {
            const int ly = 1 + idx;
            const int se = (ly + m) & 1;
            update(std::integral_constant<int, 0>{}, ly, se ? 0 : PX - 1, se, m, o1, o2, o0, f1);
          }
        }
      }
    }
    __syncthreads();
    // black cells of plane p-2 on the tile
    {
      const int m = p - 2;
      if (m >= Z0 && m < Z1 && (!DIR || (m >= 0 && m < n2))) {
        const int s = (w + m + 1) & 1;  // rows 2 + w + j NW: parity of (ly + m + 1) = s
        update2(std::integral_constant<int, 1>{}, 2 + w, 2 + w + NW, 1 + lane, s, m, o2, o3, o1,
                f2);
      }
    }
    __syncthreads();
    // plane p-2 is final: write the tile out
    {
      const int wz = p - 2;
      if (wz >= Z0 && wz < Z1) {
        const long long woff = (long long)wz * plane;
#pragma unroll
        for (int k = 0; k < NLD; k++) {
          if (!(ldf[k] & 2u)) continue;
          const int q = threadIdx.x + k * NT;
          const int c0 = (int)((ldf[k] >> 2) & 1u) ^ (wz & 1);
          const float4 a = cell(o2 + c0 * PP + q);
          const float4 bb = cell(o2 + (c0 ^ 1) * PP + q);
          *reinterpret_cast<float2 *>(uout + woff + roff[k]) = make_float2(a.x, bb.x);
          *reinterpret_cast<float2 *>(xout + woff + roff[k]) = make_float2(a.y, bb.y);
        }
      }
    }
    if (more) commit(pb ^ 1, o3, f1, f2);
    __syncthreads();
    cur = (cur + 1) & 3;
    bcur = bnx;
  }
}

// ---------------------------------------------------------------------------
// One red-black sweep per launch with register-resident z-columns (plain FP32
// form, and with BG the correction form; the same sweep, cell for cell and bit
// for bit, as k_smooth_rb).
//
// A block owns a 64 x TY tile and a chunk of zc planes and marches along z over
// the planes Z0-2 .. Z1+1.  Every x-pair of the tile plus a halo of two cells
// (34 x (TY + 4) pairs) has one owner thread for the whole march, which keeps
// the pair's red and black cell ((u, x = expm1(u)), in the correction form
// (delta, x, background ub, E = e^ub)) and right-hand sides for the last four
// planes in registers: the z neighbours of an update are the owner's
// own registers, and only the xy exchange goes through shared memory.  At the
// step that loads plane p:
//   1. the pair's u, x and f of plane p (loaded a step earlier; x from the x
//      cache that the writer of u left beside it) are split into its red and
//      black cell, and the black cell, still old, is published to the black
//      half-plane of p;
//   2. the red cells of plane p-1 on the tile grown by one cell are updated:
//      x and y neighbours are black cells of plane p-1 (the other cell of the
//      pair from registers, the rest from the black half-plane published a
//      step earlier), z neighbours are the owner's old black cells of planes
//      p-2 and p; the new values are published to the red half-plane of p-1;
//   3. the black cells of plane p-2 on the tile are updated from the new red
//      cells (red half-plane of p-2, published a step earlier, and the owner's
//      red cells of planes p-3 and p-1), and plane p-2 (u and its x cache) is
//      written out.
// Half-planes are double-buffered by step parity, so a step reads only what
// the previous step wrote and one barrier per step suffices.
// With PRL the sweep is the first one after the coarse-grid correction: every
// arriving cell first gets u += P(u^H - R u^h) from the coarser grid (the
// trilinear 27/9/3/1 prolongation of k_prolong_tiled, z then y then x, same
// arithmetic) and its x is computed from the corrected u, so the separate
// prolongation pass is saved.  The coarse
// correction of the tile, blended in z for the next plane, is staged in
// shared memory during the step before (double-buffered as the half-planes).  The ring of
// register planes is indexed by the step modulo 4, which the loop unrolls into
// compile-time indices; which cell of a pair is red is a per-slot bit flipped
// every plane, applied with selects, so an update is straight-line code and
// the updates of a thread's slots interleave.
// Thread layout (256 threads, 8 warps): warp w owns the interior pairs
// px = 1 + lane of rows 2 + w + 8 j (j < TY / 8), and thread t < NHALO also
// one halo pair: the four halo rows for t < 128, the two halo columns above.
template <int TY, bool BG = false>
struct RCCfg {
  static constexpr int TX = 64, H = 2, PX = TX / 2 + 2, LY = TY + 2 * H, PP = PX * LY;
  static constexpr int NT = 256, NW = NT / 32;
  static constexpr int NI = TY / NW;                  // interior rows per thread
  static constexpr int NSL = NI + 1;                  // pair slots per thread
  static constexpr int NHR = 4 * (TX / 2);            // halo-row pairs
  static constexpr int NHALO = NHR + 2 * LY;          // all halo pairs
#ifndef FR_RC_MINB16
#define FR_RC_MINB16 2
#endif
  // resident blocks per SM (64 x 16 tiles: 2, 124 registers; 3 would cap the
  // registers at 80 and spill)
  // (correction form: four values per cell, 64 x 8 tiles at 2 blocks per SM)
  static constexpr int MINB = BG ? 2 : (TY <= 8 ? 3 : FR_RC_MINB16);
  using Cell = typename std::conditional<BG, float4, float2>::type;
  // coarse tile of the prolongation (fine tile plus halo, +-1 coarse cell)
  static constexpr int CXE = TX / 2 + 4, CYE = TY / 2 + 4, CE = CXE * CYE;
  static constexpr size_t smem(bool prl = false) {
    return (size_t)4 * PP * sizeof(Cell) + (prl ? (size_t)2 * CE * sizeof(float) : 0);
  }
  static_assert(TY % NW == 0 && NHALO <= NT, "tile height");
};

template <bool BG, bool DIR, int TY, bool PRL = false>
__global__ void __launch_bounds__(RCCfg<TY, BG>::NT, RCCfg<TY, BG>::MINB)
    k_smooth_rc(const Grid<float> *grids, const int *off, int ngrid, int zc, const int *active,
                int par, const Grid<float> *coarse = nullptr, int cpar = 0) {
  using C = RCCfg<TY, BG>;
  using Cell = typename C::Cell;
  constexpr int TX = C::TX, PX = C::PX, PP = C::PP, NI = C::NI, NSL = C::NSL;
  constexpr int NHR = C::NHR, NHALO = C::NHALO, LY = C::LY;
  extern __shared__ float4 smem_rc4[];
  // black half-planes [2][PP] (old values), red half-planes [2][PP] (new values)
  Cell *const sbk = reinterpret_cast<Cell *>(smem_rc4);
  Cell *const srd = sbk + 2 * PP;
  float *const sez = reinterpret_cast<float *>(srd + 2 * PP);  // [2][CE] (PRL)
  constexpr int CXE = C::CXE, CE = C::CE;
  const int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<float> &Gg = grids[g];
  if (!grid_active(active, Gg.field)) return;
  const float *__restrict__ uin = par ? Gg.u2 : Gg.u;
  const float *__restrict__ xin = par ? Gg.x2 : Gg.x;  // x = expm1(u) of uin
  float *__restrict__ uout = par ? Gg.u : Gg.u2;
  float *__restrict__ xout = par ? Gg.x : Gg.x2;
  const float *__restrict__ fin = Gg.f;
  const float *__restrict__ ubin = Gg.ubg;
  const float *__restrict__ Ein = Gg.Ebg;
  const float ah = Gg.ah, beta = Gg.beta, cap = Gg.cap,
              relax = Gg.relax;
  const int n0 = Gg.n0, n1 = Gg.n1, n2 = Gg.n2;
  const int ntx = (n0 + TX - 1) / TX, nty = (n1 + TY - 1) / TY;
  int b = blockIdx.x - off[g];
  const int X0 = (b % ntx) * TX;
  b /= ntx;
  const int Y0 = (b % nty) * TY;
  b /= nty;
  const int Z0 = b * zc;
  const int Z1 = min(Z0 + zc, n2);
  const int P0 = Z0 - 2, nstep = Z1 - Z0 + 4;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long plane = (long long)n0 * n1;

  // slots: NI interior pairs, then (threads < NHALO) one halo pair.
  // fl: bit 0 load, bit 1 write out, bit 2 / 3 red update of the even / odd
  // cell; ro: 1 if the red cell of plane P0 is the odd one
  int q[NSL], roff[NSL], gyv[NSL], gxe[NSL];
  unsigned fl[NSL], ro[NSL];
#pragma unroll
  for (int s = 0; s < NSL; s++) {
    int px = -1, ly = -1;
    const bool interior = s < NI;
    if (interior) {
      px = 1 + lane;
      ly = 2 + w + C::NW * s;
    } else if ((int)threadIdx.x < NHALO) {
      const int t = threadIdx.x;
      if (t < NHR) {
        const int r = t >> 5;
        px = 1 + lane;
        ly = r < 2 ? r : TY + r;  // rows 0, 1, TY + 2, TY + 3
      } else {
        const int k = t - NHR;
        px = k < LY ? 0 : PX - 1;
        ly = k < LY ? k : k - LY;
      }
    }
    q[s] = 0;
    roff[s] = 0;
    gyv[s] = 0;
    gxe[s] = 0;
    fl[s] = 0;
    ro[s] = 0;
    if (px < 0) continue;
    const int gx = X0 - 2 + 2 * px, gy = Y0 - 2 + ly;
    q[s] = ly * PX + px;
    gyv[s] = gy;
    gxe[s] = gx;
    ro[s] = (unsigned)((gy + P0) & 1);  // gx even: colour of the even cell = (y + z) & 1
    bool ok;
    int gxw, gyw;
    if (DIR) {
      ok = gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
      gxw = gx;
      gyw = gy;
    } else {
      ok = true;
      gxw = wrapmod(gx, n0);
      gyw = wrapmod(gy, n1);
    }
    if (!ok) continue;
    roff[s] = gyw * n0 + gxw;
    unsigned f = 1u;
    // red update on the tile grown by one cell: x in [X0-1, X0+TX], y in [Y0-1, Y0+TY]
    const bool yin = gy >= Y0 - 1 && gy <= Y0 + TY;
    if (yin && gx >= X0 - 1 && gx <= X0 + TX) f |= 4u;
    if (yin && gx + 1 >= X0 - 1 && gx + 1 <= X0 + TX) f |= 8u;
    if (interior && gx < n0 && gy < n1) f |= 2u;
    fl[s] = f;
  }

  // register ring: plane P0 + k in slot k & 3; red and black cell, f
  Cell R[NSL][4], B[NSL][4];
  float FR[NSL][4], FB[NSL][4];
  // prefetched plane (u, f and, in the correction form, ub and E of the even
  // and odd cell)
  // (without the prolongation, x of the arriving u is read from the x cache
  // its writer left beside it; with it, u changes on arrival and x is computed)
  float2 pu[NSL], px[NSL], pf[NSL], pb[NSL], pe[NSL];
#pragma unroll
  for (int s = 0; s < NSL; s++) {
    pu[s] = make_float2(0.f, 0.f);
    px[s] = pu[s];
    pf[s] = pu[s];
    pb[s] = pu[s];
    pe[s] = make_float2(1.f, 1.f);
#pragma unroll
    for (int r = 0; r < 4; r++) {
      R[s][r] = Cell{};
      B[s][r] = Cell{};
      FR[s][r] = 0.f;
      FB[s][r] = 0.f;
    }
  }
  int pw = DIR ? P0 : wrapmod(P0, n2);  // wrapped index of the next plane to load
  auto fetch = [&]() {
    if (!DIR || (pw >= 0 && pw < n2)) {
      const long long zo = (long long)pw * plane;
#pragma unroll
      for (int s = 0; s < NSL; s++) {
        if (!(fl[s] & 1u)) continue;
        pu[s] = *reinterpret_cast<const float2 *>(uin + zo + roff[s]);
        if (!PRL) px[s] = *reinterpret_cast<const float2 *>(xin + zo + roff[s]);
        if (fin) pf[s] = *reinterpret_cast<const float2 *>(fin + zo + roff[s]);
        if (BG) {
          pb[s] = *reinterpret_cast<const float2 *>(ubin + zo + roff[s]);
          pe[s] = *reinterpret_cast<const float2 *>(Ein + zo + roff[s]);
        }
      }
    }
    pw = DIR ? pw + 1 : (pw + 1 == n2 ? 0 : pw + 1);
  };
  fetch();

  // prolongation (PRL): coarse correction e = u^H - R u^h of the coarse cells
  // (X0/2 - 2 + ci, Y0/2 - 2 + cj), blended in z for fine plane p, into sez[b].
  // The coarse values of the next plane are loaded into registers early in a
  // step (ez_load) and blended and stored at its end (ez_store), so that the
  // loads' latency overlaps the step's updates.
  const float w3 = 0.75f, w1 = 0.25f;
  constexpr int NEZ = PRL ? (CE + C::NT - 1) / C::NT : 1;
  float ezH[NEZ][2], ezR[NEZ][2];
  int coff[NEZ];  // offset in a coarse plane of this thread's tile entries (-1: none / zero)
  const float *__restrict__ cuH = nullptr;
  const float *__restrict__ cuR = nullptr;
  int c2 = 1;
  long long cplane = 0;
  if constexpr (PRL) {
    const Grid<float> &Cg = coarse[g];
    cuH = cpar ? Cg.u2 : Cg.u;
    cuR = Cg.uR;
    const int c0 = Cg.n0, c1 = Cg.n1;
    c2 = Cg.n2;
    cplane = (long long)c0 * c1;
#pragma unroll
    for (int r = 0; r < NEZ; r++) {
      const int q = threadIdx.x + r * C::NT;
      coff[r] = -1;
      if (q >= CE) continue;
      const int cj = q / CXE, ci = q - cj * CXE;
      int I = X0 / 2 - 2 + ci, J = Y0 / 2 - 2 + cj;
      if (DIR) {
        if (!(I >= 0 && I < c0 && J >= 0 && J < c1)) continue;
      } else {
        I = wrapmod(I, c0);
        J = wrapmod(J, c1);
      }
      coff[r] = J * c0 + I;
    }
  }
  auto ez_load = [&](int p) {
    if constexpr (PRL) {
      const int pz = DIR ? p : wrapmod(p, n2);
      const int K = pz >> 1, K2 = (pz & 1) ? K + 1 : K - 1;  // nearer, farther coarse plane
      const bool vK = !DIR || (pz >= 0 && pz < n2);
      // K is in [0, c2) for a wrapped pz; K2 wraps by one plane at most
      int K2w = K2;
      bool vK2 = vK;
      if (DIR)
        vK2 = vK && K2 >= 0 && K2 < c2;
      else
        K2w = K2 < 0 ? c2 - 1 : (K2 == c2 ? 0 : K2);
      const long long oa = (long long)K * cplane, ob = (long long)K2w * cplane;
#pragma unroll
      for (int r = 0; r < NEZ; r++) {
        ezH[r][0] = ezR[r][0] = ezH[r][1] = ezR[r][1] = 0.0f;
        if (coff[r] < 0) continue;
        if (vK) {
          ezH[r][0] = cuH[oa + coff[r]];
          ezR[r][0] = cuR[oa + coff[r]];
        }
        if (vK2) {
          ezH[r][1] = cuH[ob + coff[r]];
          ezR[r][1] = cuR[ob + coff[r]];
        }
      }
    }
  };
  auto ez_store = [&](int bsel) {
    if constexpr (PRL) {
#pragma unroll
      for (int r = 0; r < NEZ; r++) {
        const int q = threadIdx.x + r * C::NT;
        if (q >= CE) continue;
        const float ea = ezH[r][0] - ezR[r][0], eb = ezH[r][1] - ezR[r][1];
        sez[bsel * CE + q] = w3 * ea + w1 * eb;
      }
    }
  };
  if constexpr (PRL) {
    ez_load(P0);
    ez_store(0);
    __syncthreads();
  }

  // (ub, E) of a cell: (0, 1) in the plain form
  auto bgv = [](const Cell &c) -> float2 {
    if constexpr (BG)
      return make_float2(c.z, c.w);
    else
      return make_float2(0.0f, 1.0f);
  };
  // Newton update of one cell: own cell and f, neighbours -x, +x, -y, +y, -z,
  // +z; the same face order and arithmetic as k_smooth_rb
  auto newton = [&](Cell own, float fi, Cell lf, Cell rt, Cell ym, Cell yp, Cell zm, Cell zp,
                    int gx, int gy, int m) -> float {
    const float di = own.x, xi = own.y;
    const float Ei = bgv(own).y, ubi = bgv(own).x;
    const float Bi = BG ? Ei + Ei * xi : 1.0f + xi;
    OpAcc<float, BG> A(di, Ei, xi, Bi, ubi);
    auto nb = [&](const Cell &c) { A.reg(c.x, c.y, bgv(c).x, bgv(c).y); };
    if (DIR && gx == 0)
      A.ghost(face_value(Gg, 0, gx, gy, m));
    else
      nb(lf);
    if (DIR && gx == n0 - 1)
      A.ghost(face_value(Gg, 1, gx, gy, m));
    else
      nb(rt);
    if (DIR && gy == 0)
      A.ghost(face_value(Gg, 2, gx, gy, m));
    else
      nb(ym);
    if (DIR && gy == n1 - 1)
      A.ghost(face_value(Gg, 3, gx, gy, m));
    else
      nb(yp);
    if (DIR && m == 0)
      A.ghost(face_value(Gg, 4, gx, gy, m));
    else
      nb(zm);
    if (DIR && m == n2 - 1)
      A.ghost(face_value(Gg, 5, gx, gy, m));
    else
      nb(zp);
    float acc, dacc, N, dN;
    A.done(acc, dacc);
    finish_op(xi, Ei, acc, dacc, ah, beta, BG, N, dN);
    float du = newton_du(N, fi, dN, relax);
    du = fminf(fmaxf(du, -cap), cap);
    return di + du;
  };
  auto sel = [](bool c, Cell a, Cell b) { return c ? a : b; };
  // the plain form's two interior slots are updated as packed pairs
  constexpr bool PACK = !DIR && !BG && NI == 2;
  auto with_u2 = [](const Cell &c, float u, float x) -> Cell {
    Cell r = c;
    r.x = u;
    r.y = x;
    return r;
  };
  // cell of value u (x recomputed) with the background of cell c
  auto with_u = [&](const Cell &c, float u) -> Cell {
    Cell r = c;
    r.x = u;
    r.y = m_expm1(u);
    return r;
  };

  auto step = [&](auto Kc, int k) {
    constexpr int K = decltype(Kc)::value;  // ring slot of plane p
    constexpr int K1 = (K + 3) & 3, K2 = (K + 2) & 3, K3 = (K + 1) & 3;
    constexpr unsigned PK = K & 1, PK1 = K1 & 1, PK2 = K2 & 1;  // plane parities (rel. P0)
    const int p = P0 + k;
    // 1. plane p from the prefetch registers; publish its black cells
    {
      const bool inz = !DIR || (p >= 0 && p < n2);
#pragma unroll
      for (int s = 0; s < NSL; s++) {
        if (!(fl[s] & 1u)) continue;
        if constexpr (PRL) {
          // u += P(e): coarse column ci = px + 1, row cj = ly / 2 + 1 of the
          // tile; the farther row is cj + 1 for odd y, cj - 1 for even y
          const int ly = q[s] / PX, px = q[s] - ly * PX;
          const int ci = px + 1, cj = (ly >> 1) + 1, cj2 = (ly & 1) ? cj + 1 : cj - 1;
          const float *za = sez + PK * CE + cj * CXE, *zb = sez + PK * CE + cj2 * CXE;
          const float em = w3 * za[ci - 1] + w1 * zb[ci - 1];
          const float e0 = w3 * za[ci] + w1 * zb[ci];
          const float ep = w3 * za[ci + 1] + w1 * zb[ci + 1];
          pu[s].x = pu[s].x + (w3 * e0 + w1 * em);
          pu[s].y = pu[s].y + (w3 * e0 + w1 * ep);
        }
        const bool odd = (ro[s] ^ PK) != 0;  // red cell is the odd one
        const float ur = odd ? pu[s].y : pu[s].x, ub = odd ? pu[s].x : pu[s].y;
        const float xr = odd ? px[s].y : px[s].x, xb = odd ? px[s].x : px[s].y;
        // the red cell's x is needed only if this pair's red cell is updated
        const bool needr = s < NI || (fl[s] & (odd ? 8u : 4u));
        if constexpr (BG) {
          R[s][K] = make_float4(ur, needr ? (PRL ? m_expm1(ur) : xr) : 0.0f,
                                odd ? pb[s].y : pb[s].x, odd ? pe[s].y : pe[s].x);
          B[s][K] = make_float4(ub, PRL ? m_expm1(ub) : xb, odd ? pb[s].x : pb[s].y,
                                odd ? pe[s].x : pe[s].y);
        } else {
          R[s][K] = make_float2(ur, needr ? (PRL ? m_expm1(ur) : xr) : 0.0f);
          B[s][K] = make_float2(ub, PRL ? m_expm1(ub) : xb);
        }
        if (fin) {
          const float fr = odd ? pf[s].y : pf[s].x, fb = odd ? pf[s].x : pf[s].y;
          FR[s][K] = fr;  // FP32 grids: fs = 1, fo = 0, fs (f - fo) = f exactly
          FB[s][K] = fb;
        } else {
          FR[s][K] = 0.0f;
          FB[s][K] = 0.0f;
        }
        if (inz) sbk[PK * PP + q[s]] = B[s][K];
      }
    }
    if (k + 1 < nstep) {
      fetch();
      ez_load(p + 1);
    }
    // 2. red cells of plane m = p - 1 on the grown tile
    {
      const int m = p - 1;
      if (m >= Z0 - 1 && m <= Z1 && (!DIR || (m >= 0 && m < n2))) {
        if constexpr (PACK) {
          // the two interior slots (same row parity) in packed pairs
          const bool odd = (ro[0] ^ PK1) != 0;
          float2 nu[6], nxv[6];
          float2 di, xi, fi;
#pragma unroll
          for (int s = 0; s < 2; s++) {
            const Cell *bk = sbk + PK1 * PP + q[s];
            const Cell nx = bk[odd ? 1 : -1];
            const Cell in = B[s][K1];
            const Cell c6[6] = {odd ? in : nx, odd ? nx : in, bk[-PX], bk[PX], B[s][K2], B[s][K]};
#pragma unroll
            for (int f = 0; f < 6; f++) {
              (s ? nu[f].y : nu[f].x) = c6[f].x;
              (s ? nxv[f].y : nxv[f].x) = c6[f].y;
            }
            (s ? di.y : di.x) = R[s][K1].x;
            (s ? xi.y : xi.x) = R[s][K1].y;
            (s ? fi.y : fi.x) = FR[s][K1];
          }
          const float2 un = newton2_plain(di, xi, fi, nu, nxv, ah, beta, cap, relax);
          const float2 xn = m_expm1_2(un);
          R[0][K1] = with_u2(R[0][K1], un.x, xn.x);
          R[1][K1] = with_u2(R[1][K1], un.y, xn.y);
          srd[PK1 * PP + q[0]] = R[0][K1];
          srd[PK1 * PP + q[1]] = R[1][K1];
        }
#pragma unroll
        for (int s = PACK ? 2 : 0; s < NSL; s++) {
          const bool odd = (ro[s] ^ PK1) != 0;
          if (!((s < NI && !DIR) || (fl[s] & (odd ? 8u : 4u)))) continue;
          const Cell *bk = sbk + PK1 * PP + q[s];
          const Cell ym = bk[-PX], yp = bk[PX];
          const Cell nx = bk[odd ? 1 : -1];
          const float un = newton(R[s][K1], FR[s][K1], sel(odd, B[s][K1], nx),
                                  sel(odd, nx, B[s][K1]), ym, yp, B[s][K2], B[s][K],
                                  gxe[s] + (odd ? 1 : 0), gyv[s], m);
          R[s][K1] = with_u(R[s][K1], un);
          srd[PK1 * PP + q[s]] = R[s][K1];
        }
      }
    }
    // 3. black cells of plane m = p - 2 on the tile, then plane m is final
    {
      const int m = p - 2;
      if (m >= Z0 && m < Z1 && (!DIR || (m >= 0 && m < n2))) {
        float2 unp = make_float2(0.f, 0.f);
        if constexpr (PACK) {
          const bool odd = (ro[0] ^ PK2) == 0;  // black cell is the odd one
          float2 nu[6], nxv[6];
          float2 di, xi, fi;
#pragma unroll
          for (int s = 0; s < 2; s++) {
            const Cell *rd = srd + PK2 * PP + q[s];
            const Cell nx = rd[odd ? 1 : -1];
            const Cell in = R[s][K2];
            const Cell c6[6] = {odd ? in : nx, odd ? nx : in, rd[-PX], rd[PX], R[s][K3], R[s][K1]};
#pragma unroll
            for (int f = 0; f < 6; f++) {
              (s ? nu[f].y : nu[f].x) = c6[f].x;
              (s ? nxv[f].y : nxv[f].x) = c6[f].y;
            }
            (s ? di.y : di.x) = B[s][K2].x;
            (s ? xi.y : xi.x) = B[s][K2].y;
            (s ? fi.y : fi.x) = FB[s][K2];
          }
          unp = newton2_plain(di, xi, fi, nu, nxv, ah, beta, cap, relax);
        }
#pragma unroll
        for (int s = 0; s < NI; s++) {
          if (DIR && !(fl[s] & 1u)) continue;
          const bool odd = (ro[s] ^ PK2) == 0;  // black cell is the odd one
          float un;
          if constexpr (PACK) {
            un = s ? unp.y : unp.x;
          } else {
            const Cell *rd = srd + PK2 * PP + q[s];
            const Cell ym = rd[-PX], yp = rd[PX];
            const Cell nx = rd[odd ? 1 : -1];
            un = newton(B[s][K2], FB[s][K2], sel(odd, R[s][K2], nx), sel(odd, nx, R[s][K2]), ym,
                        yp, R[s][K3], R[s][K1], gxe[s] + (odd ? 1 : 0), gyv[s], m);
          }
          B[s][K2] = with_u(B[s][K2], un);
          if (fl[s] & 2u) {
            const Cell e = sel(odd, R[s][K2], B[s][K2]), o = sel(odd, B[s][K2], R[s][K2]);
            const long long oo = (long long)m * plane + roff[s];
            *reinterpret_cast<float2 *>(uout + oo) = make_float2(e.x, o.x);
            *reinterpret_cast<float2 *>(xout + oo) = make_float2(e.y, o.y);
          }
        }
      }
    }
    if (k + 1 < nstep) ez_store((int)(PK ^ 1u));
    __syncthreads();
  };
  for (int k = 0; k < nstep; k += 4) {
    step(std::integral_constant<int, 0>{}, k);
    if (k + 1 < nstep) step(std::integral_constant<int, 1>{}, k + 1);
    if (k + 2 < nstep) step(std::integral_constant<int, 2>{}, k + 2);
    if (k + 3 < nstep) step(std::integral_constant<int, 3>{}, k + 3);
  }
}

// Tiled FAS right-hand side of a coarse level, f <- A(u) - f (the same
// operator evaluation, face order and arithmetic as k_fas_rhs): a block owns a
// 64 x 16 tile and a chunk of zc planes and marches along z with a ring of
// three planes of (u, x) [and (ub, E)] in shared memory (tile plus a halo of
// one cell); at the step that has loaded plane p it evaluates plane p-1, each
// thread four cells (two rows, x = lane and lane + 32), with f read and written
// in place.  The next plane is prefetched into registers during the evaluation.
constexpr int kFrTX = 64, kFrTY = 16;
// dynamic shared memory of k_fas_rhs_tiled: three planes of the tile plus halo,
// (u, x, ub, E) per cell in the correction form, (u, x) in the plain one
constexpr size_t fas_rhs_tiled_smem(bool bg) {
  return (size_t)3 * (kFrTX + 2) * (kFrTY + 2) * (bg ? sizeof(float4) : sizeof(float2));
}
template <bool BG, bool DIR>
__global__ void __launch_bounds__(256)
    k_fas_rhs_tiled(const Grid<float> *grids, const int *off, int ngrid, int zc,
                    const int *active, int par) {
  constexpr int LX = kFrTX + 2, LY = kFrTY + 2, PC = LX * LY, NT = 256;
  constexpr int NLD = (PC + NT - 1) / NT;
  extern __shared__ float4 sfr[];
  float2 *s2 = reinterpret_cast<float2 *>(sfr);
  auto cellv = [&](int i) -> float4 {
    if (BG) return sfr[i];
    const float2 v = s2[i];
    return make_float4(v.x, v.y, 0.f, 1.f);
  };
  const int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<float> &Gg = grids[g];
  if (!grid_active(active, Gg.field)) return;
  const float *__restrict__ uin = par ? Gg.u2 : Gg.u;
  const float *__restrict__ xin = par ? Gg.x2 : Gg.x;
  const float *__restrict__ ubin = Gg.ubg;
  const float *__restrict__ Ein = Gg.Ebg;
  float *__restrict__ f = const_cast<float *>(Gg.f);
  const float ah = Gg.ah, beta = Gg.beta;
  const int n0 = Gg.n0, n1 = Gg.n1, n2 = Gg.n2;
  const int ntx = (n0 + kFrTX - 1) / kFrTX, nty = (n1 + kFrTY - 1) / kFrTY;
  int b = blockIdx.x - off[g];
  const int X0 = (b % ntx) * kFrTX;
  b /= ntx;
  const int Y0 = (b % nty) * kFrTY;
  b /= nty;
  const int Z0 = b * zc, Z1 = min(Z0 + zc, n2);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long plane = (long long)n0 * n1;
  // plane-load table: cell q = threadIdx.x + k NT of the (TX + 2) x (TY + 2) tile
  int roff[NLD];
  bool lok[NLD];
#pragma unroll
  for (int k = 0; k < NLD; k++) {
    const int q = threadIdx.x + k * NT;
    roff[k] = 0;
    lok[k] = false;
    if (q < PC) {
      const int gx = X0 - 1 + q % LX, gy = Y0 - 1 + q / LX;
      if (DIR) {
        lok[k] = gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
        roff[k] = lok[k] ? gy * n0 + gx : 0;
      } else {
        lok[k] = true;
        roff[k] = wrapmod(gy, n1) * n0 + wrapmod(gx, n0);
      }
    }
  }
  float4 pv[NLD];
  // plane at offset zoff (vz false: outside a patch, never read)
  auto fetch = [&](long long zoff, bool vz) {
#pragma unroll
    for (int k = 0; k < NLD; k++) {
      pv[k] = make_float4(0.f, 0.f, 0.f, 1.f);
      if (!vz || !lok[k]) continue;
      const long long gi = zoff + roff[k];
      pv[k].x = uin[gi];
      pv[k].y = xin[gi];
      if (BG) {
        pv[k].z = ubin[gi];
        pv[k].w = Ein[gi];
      }
    }
  };
  auto commit = [&](int so) {
#pragma unroll
    for (int k = 0; k < NLD; k++) {
      const int q = threadIdx.x + k * NT;
      if (q >= PC) continue;
      if (BG)
        sfr[so + q] = pv[k];
      else
        s2[so + q] = make_float2(pv[k].x, pv[k].y);
    }
  };
  // f <- A(u) - f at tile cell (lx, ly) of plane m; om, oc, op: slots of m-1, m, m+1
  auto eval = [&](int lx, int ly, int m, int om, int oc, int op) {
    const int gx = X0 - 1 + lx, gy = Y0 - 1 + ly;
    if (gx >= n0 || gy >= n1) return;
    const int i = ly * LX + lx;
    const float4 own = cellv(oc + i);
    const float di = own.x, xi = own.y;
    const float Ei = BG ? own.w : 1.0f;
    const float ubi = BG ? own.z : 0.0f;
    const float Bi = BG ? Ei + Ei * xi : 1.0f + xi;
    OpAcc<float, BG> A(di, Ei, xi, Bi, ubi);
    auto nb = [&](int j) {
      const float4 v = cellv(j);
      A.reg(v.x, v.y, v.z, v.w);
    };
    if (DIR && gx == 0) A.ghost(face_value(Gg, 0, gx, gy, m)); else nb(oc + i - 1);
    if (DIR && gx == n0 - 1) A.ghost(face_value(Gg, 1, gx, gy, m)); else nb(oc + i + 1);
    if (DIR && gy == 0) A.ghost(face_value(Gg, 2, gx, gy, m)); else nb(oc + i - LX);
    if (DIR && gy == n1 - 1) A.ghost(face_value(Gg, 3, gx, gy, m)); else nb(oc + i + LX);
    if (DIR && m == 0) A.ghost(face_value(Gg, 4, gx, gy, m)); else nb(om + i);
    if (DIR && m == n2 - 1) A.ghost(face_value(Gg, 5, gx, gy, m)); else nb(op + i);
    float acc, dacc, N, dN;
    A.done(acc, dacc);
    finish_op(xi, Ei, acc, dacc, ah, beta, BG, N, dN);
    const long long c = (long long)m * plane + (long long)gy * n0 + gx;
    f[c] = N - f[c];
  };
  const int P0 = Z0 - 1, PE = Z1 + 1;
  auto inr = [&](int pz) { return !DIR || (pz >= 0 && pz < n2); };
  int pw = DIR ? P0 : wrapmod(P0, n2);
  fetch((long long)pw * plane, inr(P0));
  commit(0);
  __syncthreads();
  int cur = 0;  // ring slot of plane p
  for (int p = P0; p < PE; p++) {
    const bool more = p + 1 < PE;
    pw = DIR ? p + 1 : (pw + 1 == n2 ? 0 : pw + 1);
    if (more) fetch((long long)pw * plane, inr(p + 1));
    const int o0 = cur * PC, o1 = (cur == 0 ? 2 : cur - 1) * PC,
              o2 = (cur == 2 ? 0 : cur + 1) * PC;  // planes p, p-1, p-2
    const int m = p - 1;
    if (m >= Z0 && m < Z1) {
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int h = 0; h < 2; h++) eval(1 + lane + 32 * h, 1 + w + 8 * r, m, o2, o1, o0);
    }
    __syncthreads();
    if (more) commit(o2);
    __syncthreads();
    cur = cur == 2 ? 0 : cur + 1;
  }
}

// ---------------------------------------------------------------------------
// Asynchronous global-to-shared copy of 8 bytes (PTX cp.async; both
// addresses 8-byte aligned); commit_group / wait_group track completion.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Tiled FP32 residual + restriction (same result as k_resid_restrict).
// A block owns a TX x TY fine tile and an even chunk of zc fine planes, marches
// along z with a ring of 4 planes (tile plus a halo of 2 cells in x, so that
// 8-byte x-pairs stay aligned, and 1 in y) in shared memory, and each thread
// owns one coarse column of the tile: per fine plane it evaluates the residual
// of its 2x2 fine cells from shared memory, and after every second plane it
// writes its coarse cell (u^H = uR = mean u^h, x^H = expm1(u^H),
// f^H <- mean d^h) and accumulates the fine residual norm.  Plane m+2 is
// fetched into registers while plane m is evaluated.
template <int TX, int TY>
struct RRCfg {
  // planes in flight beyond the three being read; ring of A + 4 slots (the
  // slot being refilled was last read two iterations earlier)
#ifndef FR_RR_AHEAD
#define FR_RR_AHEAD 2
#endif
  static constexpr int A = FR_RR_AHEAD;
  static constexpr int LX = TX + 4, LY = TY + 2, PL = LX * LY, NS = 4 + A;
  static constexpr int PXR = LX / 2, NPAIR = PXR * LY;
  static constexpr int CX = TX / 2, NT = (TX / 2) * (TY / 2);
  static constexpr int K = (NPAIR + NT - 1) / NT;
  static constexpr size_t smem(bool bg) { return (size_t)NS * PL * sizeof(float) * (bg ? 5 : 3); }
};

template <bool BG, bool DIR, int TX, int TY>
__global__ void __launch_bounds__(RRCfg<TX, TY>::NT)
    k_resid_restrict_tiled(const Grid<float> *fine, const Grid<float> *coarse, const int *off,
                           int ngrid, int zc, const int *active, int fpar, int cpar,
                           double *partial) {
  using C = RRCfg<TX, TY>;
  constexpr int LX = C::LX, PL = C::PL, NS = C::NS, NT = C::NT, CX = C::CX;
  constexpr int PXR = C::PXR, NPAIR = C::NPAIR, K = C::K;
  extern __shared__ float smem[];
  float *sd = smem;
  float *sx = smem + NS * PL;
  float *sf = smem + 2 * NS * PL;
  float *sub = smem + 3 * NS * PL;
  float *sE = smem + 4 * NS * PL;
  const int g = find_grid(off, ngrid, blockIdx.x);
  const Grid<float> &Fg = fine[g];
  const Grid<float> &Cg = coarse[g];
  float ss = 0.0f, mx = 0.0f;
  if (grid_active(active, Fg.field)) {
    const float *__restrict__ uin = fpar ? Fg.u2 : Fg.u;
    const float *__restrict__ xin = fpar ? Fg.x2 : Fg.x;
    const float *__restrict__ fin = Fg.f;
    const float *__restrict__ ubin = Fg.ubg;
    const float *__restrict__ Ein = Fg.Ebg;
    const float ah = Fg.ah, beta = Fg.beta;
    const int n0 = Fg.n0, n1 = Fg.n1, n2 = Fg.n2;
    const int c0 = Cg.n0, c1 = Cg.n1;
    float *__restrict__ cu = cpar ? Cg.u2 : Cg.u;
    float *__restrict__ cR = Cg.uR;
    float *__restrict__ cx = cpar ? Cg.x2 : Cg.x;
    float *__restrict__ cf = const_cast<float *>(Cg.f);
    const int ntx = (n0 + TX - 1) / TX, nty = (n1 + TY - 1) / TY;
    int b = blockIdx.x - off[g];
    const int X0 = (b % ntx) * TX;
    b /= ntx;
    const int Y0 = (b % nty) * TY;
    b /= nty;
    const int Z0 = b * zc;
    const int Z1 = min(Z0 + zc, n2);
    // the pairs this thread loads: global pair start (wrapped) per slot, -1 if none
    long long pg[K];
    int po[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      const int c = threadIdx.x + k * NT;
      pg[k] = -1;
      po[k] = 0;
      if (c < NPAIR) {
        const int yy = c / PXR, px = c - yy * PXR;
        int gxx = X0 - 2 + 2 * px, gyy = Y0 - 1 + yy;
        po[k] = yy * LX + 2 * px;
        bool in = true;
        if (DIR) {
          in = gxx >= 0 && gxx < n0 && gyy >= 0 && gyy < n1;
        } else {
          // the tile (TX + 4 wide) may span more than two periods of a small grid
          gxx = wrapmod(gxx, n0);
          gyy = wrapmod(gyy, n1);
        }
        if (in) pg[k] = (long long)gyy * n0 + gxx;
      }
    }
    // copies of plane p into ring slot (p - (Z0 - 1)) mod NS: one commit
    // group per call (empty when the plane is outside a patch)
    const bool hasf = fin != nullptr;
    int pwz = DIR ? Z0 - 1 : wrapmod(Z0 - 1, n2);  // wrapped index of the next plane
    const long long fplane = (long long)n0 * n1;
    auto issue = [&](int p, int slot) {
      if (!DIR || (p >= 0 && p < n2)) {
        const long long zo = (long long)pwz * fplane;
        const int base = slot * PL;
#pragma unroll
        for (int k = 0; k < K; k++) {
          if (pg[k] < 0) continue;
          const long long gi = zo + pg[k];
          const int o = base + po[k];
          cp_async8(sd + o, uin + gi);
          cp_async8(sx + o, xin + gi);
          if (hasf) cp_async8(sf + o, fin + gi);
          if (BG) {
            cp_async8(sub + o, ubin + gi);
            cp_async8(sE + o, Ein + gi);
          }
        }
      }
      cp_async_commit();
      pwz = DIR ? pwz + 1 : (pwz + 1 == n2 ? 0 : pwz + 1);
    };
    const int ci = threadIdx.x % CX, cj = threadIdx.x / CX;
    const int lx = 2 + 2 * ci, ly = 1 + 2 * cj;
    const int gx = X0 + 2 * ci, gy = Y0 + 2 * cj;
    const bool valid = gx < n0 && gy < n1;
    float su = 0.f, sdd = 0.f;
    constexpr int A = C::A;
    // prologue: planes Z0-1 .. Z0+A (slots 0 .. A+1)
#pragma unroll
    for (int d = 0; d < A + 2; d++) issue(Z0 - 1 + d, d);
    int sl = 1;  // ring slot of plane m
    for (int m = Z0; m < Z1; m++) {
      // plane m+1+A into the slot of plane m-3 (last read by iteration m-2,
      // before the barrier of iteration m-1); planes m-1, m, m+1 must have landed
      {
        const int pz = m + 1 + A;
        if (pz <= Z1) issue(pz, (sl + A + 1) % NS);
        else cp_async_commit();
      }
      cp_async_wait<A>();
      __syncthreads();
      if (valid) {
        const int slm = sl == 0 ? NS - 1 : sl - 1, slp = sl + 1 == NS ? 0 : sl + 1;
        // the 2 x 2 cells of this thread (rows ly, ly + 1; columns lx, lx + 1)
        // and their neighbours as aligned pairs: left, own and right pair of
        // each row, the pairs of rows ly - 1 and ly + 2, and the own pairs of
        // planes m - 1 and m + 1 (same values and face order as cell by cell)
        const int r0 = sl * PL + ly * LX + lx, r1 = r0 + LX;
        const int zm0 = slm * PL + ly * LX + lx, zp0 = slp * PL + ly * LX + lx;
        auto pr = [&](const float *a, int o) { return *reinterpret_cast<const float2 *>(a + o); };
        struct Nb {
          float2 L[2], C[2], R[2], D, U, M[2], P[2];
        };
        auto gather = [&](const float *a) {
          Nb n;
          n.L[0] = pr(a, r0 - 2);
          n.C[0] = pr(a, r0);
          n.R[0] = pr(a, r0 + 2);
          n.L[1] = pr(a, r1 - 2);
          n.C[1] = pr(a, r1);
          n.R[1] = pr(a, r1 + 2);
          n.D = pr(a, r0 - LX);
          n.U = pr(a, r1 + LX);
          n.M[0] = pr(a, zm0);
          n.M[1] = pr(a, zm0 + LX);
          n.P[0] = pr(a, zp0);
          n.P[1] = pr(a, zp0 + LX);
          return n;
        };
        const Nb nu = gather(sd), nx = gather(sx);
        Nb nb, ne;
        if (BG) {
          nb = gather(sub);
          ne = gather(sE);
        }
        const float2 f0 = hasf ? pr(sf, r0) : make_float2(0.f, 0.f);
        const float2 f1 = hasf ? pr(sf, r1) : make_float2(0.f, 0.f);
        auto lane = [](const float2 &v, int a) { return a ? v.y : v.x; };
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int ax = q & 1, ay = q >> 1;
          const int gxq = gx + ax, gyq = gy + ay;
          // value of array n at neighbour k of the cell: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z
          auto at = [&](const Nb &n, int k) -> float {
            switch (k) {
              case 0: return ax ? n.C[ay].x : n.L[ay].y;
              case 1: return ax ? n.R[ay].x : n.C[ay].y;
              case 2: return ay ? lane(n.C[0], ax) : lane(n.D, ax);
              case 3: return ay ? lane(n.U, ax) : lane(n.C[1], ax);
              case 4: return lane(n.M[ay], ax);
              default: return lane(n.P[ay], ax);
            }
          };
          const float di = lane(nu.C[ay], ax), xi = lane(nx.C[ay], ax);
          const float Ei = BG ? lane(ne.C[ay], ax) : 1.0f;
          const float ubi = BG ? lane(nb.C[ay], ax) : 0.0f;
          const float Bi = BG ? Ei + Ei * xi : 1.0f + xi;
          OpAcc<float, BG> A(di, Ei, xi, Bi, ubi);
#define FR_NB(K) A.reg(at(nu, K), at(nx, K), BG ? at(nb, K) : 0.0f, BG ? at(ne, K) : 1.0f)
          if (DIR && gxq == 0) A.ghost(face_value(Fg, 0, gxq, gyq, m));
          else FR_NB(0);
          if (DIR && gxq == n0 - 1) A.ghost(face_value(Fg, 1, gxq, gyq, m));
          else FR_NB(1);
          if (DIR && gyq == 0) A.ghost(face_value(Fg, 2, gxq, gyq, m));
          else FR_NB(2);
          if (DIR && gyq == n1 - 1) A.ghost(face_value(Fg, 3, gxq, gyq, m));
          else FR_NB(3);
          if (DIR && m == 0) A.ghost(face_value(Fg, 4, gxq, gyq, m));
          else FR_NB(4);
          if (DIR && m == n2 - 1) A.ghost(face_value(Fg, 5, gxq, gyq, m));
          else FR_NB(5);
#undef FR_NB
          float acc, dacc, N, dN;
          A.done(acc, dacc);
          finish_op(xi, Ei, acc, dacc, ah, beta, BG, N, dN);
          const float d = N - lane(ay ? f1 : f0, ax);  // FP32 grids: fs (f - fo) = f
          sdd += d;
          su += di;
          ss = fmaf(d, d, ss);
          mx = fmaxf(mx, fabsf(d));
        }
        if ((m - Z0) & 1) {
          const long long cidx = ((long long)(m >> 1) * c1 + (gy >> 1)) * c0 + (gx >> 1);
          const float uh = su * 0.125f;
          cR[cidx] = uh;
          cu[cidx] = uh;
          cx[cidx] = m_expm1(uh);
          cf[cidx] = sdd * 0.125f;
          su = 0.f;
          sdd = 0.f;
        }
      }
      sl = sl + 1 == NS ? 0 : sl + 1;
    }
    cp_async_wait<0>();
  }
  if (partial) block_reduce2f<NT>(ss, mx, &partial[2 * blockIdx.x], &partial[2 * blockIdx.x + 1]);
}

}  // namespace frmg
