// frmg_masked.cu -- the general mask scheme: FAS solve of the f(R) equation on
// a refinement region of any shape.
//
// Sec. V (the mask scheme), Sec. V.B.1 (Eqs. u_i-1jk, bc_modified_fR_op,
// bc_modified_fR_dop), Sec. V.B.2 (FAS with masked restriction, coarse masks
// and boundary values), Sec. V.A.2 (masked restriction of the residual) and
// Sec. V.A.3 (masked prolongation).  A region is a box of cells with a mask m
// in [-1, 1] per cell: m > 0 marks an active cell (relaxed), the others are
// ghosts whose values stay fixed; the box's outer layer must be ghosts.
//
// * Across the face from an active cell i to a ghost g, with r = m_g / m_i,
//   the ghost enters as u_g = u_b - r u_b + r u_i, b_g = exp(u_g), where the
//   boundary value u_b = (m_i u_g0 - m_g u_i0) / (m_i - m_g) is computed from
//   the initial values once and kept (six per cell, NaN where no ghost face).
// * L_i = (alpha/2) sum_faces (e^{u_i} + e^{u_j})(u_j - u_i)
//         + beta (e^{-u_i/2} - 1) - gamma (rho_i - 1),
//   in the solver's variable u = u~ - ubar (alpha = c~^2 |fbar~_R| / h^2);
//   with the ghost faces above this is Eq. bc_modified_fR_op, and its
//   derivative in u_i is Eq. bc_modified_fR_dop.
// * Levels: masks, densities and initial values restrict as the mean of the
//   8 children, a coarse cell is active when its mask is > 0, and its ghost
//   boundary values follow from the restricted initial values as on the
//   finest level.  R u^h is the mean of all 8 children (for active coarse
//   cells only), R d^h the sum over the active children / 8; the correction
//   u^H - R u^h is prolonged (trilinear 27/9/3/1) onto active fine cells, a
//   masked coarse cell contributing 0.  Levels halve while the sizes stay even
//   and >= 4, the next level's outer layer stays masked and it keeps an
//   active cell.
//
// FP64, or mixed (FP32 V-cycles of the full variable, then outer steps of
// FP32 V-cycles of the correction form against the FP64 residual); red-black
// Newton-Gauss-Seidel with the step clamped to |du| <= cap and optionally
// over-relaxed.  Every level keeps b = exp(u) (correction form: expm1 of the
// correction) beside u, written by each kernel that writes u, so an operator
// evaluation takes one exponential (e^{-u_i/2}) plus one per ghost face
// instead of eight.  The fine-level sweeps, residual and prolongation run
// over per-colour lists of the active cells, so that regions covering a small
// part of their box keep every warp busy.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "frmg.h"
#include "frmg_dfmath.cuh"
#include "frmg_internal.h"

using namespace frmg;

namespace {

struct MError {
  int status;
  std::string msg;
};

#define MCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw MError{FR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};       \
  } while (0)

#define MLAUNCH(ctx)                                                                    \
  do {                                                                                  \
    frmg_launch_counter(ctx)++;                                                         \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess)                                                              \
      throw MError{FR_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)};  \
  } while (0)

constexpr int kNT = 256;

long long nblk(long long n) { return (n + kNT - 1) / kNT; }

// One level of a masked region, iterate and work arrays in T (FP64, or FP32
// in a mixed-precision solve); the mask, density and ghost boundary values are
// always the FP64 level's.  BG: the correction form of the outer steps of a
// mixed solve, whose unknown is the correction v to a background (the FP64
// iterate rounded to FP32) and whose operator is L(background + v) -
// L(background), evaluated without forming either term.
template <typename T, bool BG = false>
struct MLevelT {
  T *u;             // iterate (BG: correction v) in active cells; fixed ghost values
                    // (BG: 0) elsewhere
  T *b;             // exp(u) (BG: expm1(v)) of every cell, rewritten wherever u changes
  const double *m;  // mask
  const double *rho;
  T *f;             // FAS right-hand side (0 on the finest level)
  T *uR;            // R u^h of the active cells (coarse levels)
  T *d;             // residual (fine side) or R d^h (coarse side)
  double *ub;       // [6][ncell] boundary values of the ghost faces (NaN elsewhere)
  const int *act;   // active cells in index order, colour 0 ((i+j+k) even) first
  long long na0, na;  // active cells of colour 0, of both colours
  int n0, n1, n2;
  long long ncell;
  FastDiv fd0, fd1;
  T ah;             // alpha / 2 at this level's h
  T beta, gamma;
  T *bgu, *bgE;     // BG: background value and its exponential per cell
};
using MLevel = MLevelT<double>;

__device__ __forceinline__ double m_exp(double v) { return exp(v); }
__device__ __forceinline__ float m_exp(float v) { return expf(v); }
// the per-cell cache of a new value
template <typename T, bool BG>
__device__ __forceinline__ T m_cache(T v) {
  if constexpr (BG)
    return expm1f(v);
  else
    return m_exp(v);
}

template <typename T, bool BG>
__device__ __forceinline__ void ijk(const MLevelT<T, BG> &L, long long c, int &i, int &j,
                                    int &k) {
  const unsigned cu = (unsigned)c, q = fdiv(cu, L.fd0), q2 = fdiv(q, L.fd1);
  i = (int)(cu - q * (unsigned)L.n0);
  j = (int)(q - q2 * (unsigned)L.n1);
  k = (int)q2;
}

// neighbour offset of face f (-x, +x, -y, +y, -z, +z)
template <typename T, bool BG>
__device__ __forceinline__ long long face_step(const MLevelT<T, BG> &L, int f) {
  const long long s = f < 2 ? 1 : (f < 4 ? (long long)L.n0 : (long long)L.n0 * L.n1);
  return (f & 1) ? s : -s;
}

// L_i and dL_i/du_i at active cell c (Eqs. bc_modified_fR_op / _dop); the
// exponentials of the cell and of its active neighbours come from the cache b.
// In FP32 the mass term's e^{-u/2} - 1 is formed by expm1f (no cancellation
// near u = 0).
template <typename T, bool BG>
__device__ __forceinline__ void m_cell(const MLevelT<T, BG> &L, long long c, T &N, T &dN) {
  if constexpr (BG) {
    // correction form: with B = E (1 + x) = e^{background + v}, a regular face
    // adds (E_i x_i + E_j x_j) g + (B_i + B_j) e (g, e the background and
    // correction differences); a ghost face has background value
    // u_b - r u_b + r ubg_i and correction r v_i; the mass term is
    // beta e^{-ubg_i/2} (e^{-v_i/2} - 1); the density term cancels
    const T vi = L.u[c], xi = L.b[c], mi = (T)L.m[c];
    const T gi = L.bgu[c], Ei = L.bgE[c];
    const T Bi = Ei + Ei * xi;
    T acc = T(0), dacc = T(0);
#pragma unroll
    for (int f = 0; f < 6; f++) {
      const long long cj = c + face_step(L, f);
      const double mjd = L.m[cj];
      if (mjd > 0.0) {
        const T vj = L.u[cj], xj = L.b[cj], Ej = L.bgE[cj];
        const T Bj = Ej + Ej * xj;
        const T g = L.bgu[cj] - gi, e = vj - vi;
        acc += (Ei * xi + Ej * xj) * g + (Bi + Bj) * e;
        dacc += Bi * (g + e) - (Bi + Bj);
      } else {
        const T r = (T)mjd / mi, ub = (T)L.ub[f * L.ncell + c];
        const T gg = ub - r * ub + r * gi, Eg = m_exp(gg);
        const T vg = r * vi, xg = expm1f(vg);
        const T Bg = Eg + Eg * xg;
        const T g = gg - gi, e = vg - vi;
        acc += (Ei * xi + Eg * xg) * g + (Bi + Bg) * e;
        dacc += (Bi + r * Bg) * (g + e) + (Bi + Bg) * (r - T(1));
      }
    }
    const T F = rsqrtf(Ei), em = expm1f(-0.5f * vi);
    N = L.ah * acc + L.beta * F * em;
    dN = L.ah * dacc - T(0.5) * L.beta * F * (em + T(1));
    return;
  }
  const T ui = L.u[c], mi = (T)L.m[c];
  const T bi = L.b[c];
  T acc = T(0), dacc = T(0);
#pragma unroll
  for (int f = 0; f < 6; f++) {
    const long long cj = c + face_step(L, f);
    const double mjd = L.m[cj];
    if (mjd > 0.0) {
      const T uj = L.u[cj], bj = L.b[cj];
      acc += (bi + bj) * (uj - ui);
      dacc += bi * (uj - ui) - (bi + bj);
    } else {
      const T r = (T)mjd / mi, ub = (T)L.ub[f * L.ncell + c];
      const T ug = ub - r * ub + r * ui, bg = m_exp(ug);
      acc += (bi + bg) * (ug - ui);
      dacc += (bi + r * bg) * (ug - ui) + (bi + bg) * (r - T(1));
    }
  }
  T s, sm1;
  if constexpr (sizeof(T) == 8) {
    s = exp(-0.5 * ui);
    sm1 = s - 1.0;
  } else {
    sm1 = expm1f(-0.5f * ui);
    s = sm1 + 1.0f;
  }
  N = L.ah * acc + L.beta * sm1 - L.gamma * ((T)L.rho[c] - T(1));
  dN = L.ah * dacc - T(0.5) * L.beta * s;
}

}  // namespace

namespace {

// Boundary values of the ghost faces from the current (initial) values, and
// the exponential cache of every cell.
__global__ void __launch_bounds__(kNT) k_mub(MLevel L) {
  const long long c = (long long)blockIdx.x * kNT + threadIdx.x;
  if (c >= L.ncell) return;
  const double mi = L.m[c], ui = L.u[c];
  L.b[c] = exp(ui);
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
  for (int f = 0; f < 6; f++) {
    double v = nan;
    if (mi > 0.0) {
      const long long cj = c + face_step(L, f);
      const double mg = L.m[cj];
      if (mg <= 0.0) v = (mi * L.u[cj] - mg * ui) / (mi - mg);
    }
    L.ub[f * L.ncell + c] = v;
  }
}

// Active-cell lists: per block of kNT cells, the active cells of each colour
// (k_mcount), then each cell's place in its colour's list from the scanned
// block bases (k_mlist).  A colour's cells are independent of one another, so
// a sweep over the list equals the sweep over the box; the lists keep warps
// full where the region covers a small part of the box.
__global__ void __launch_bounds__(kNT) k_mcount(MLevel L, int *cnt) {
  const long long c = (long long)blockIdx.x * kNT + threadIdx.x;
  bool a0 = false, a1 = false;
  if (c < L.ncell && L.m[c] > 0.0) {
    int i, j, k;
    ijk(L, c, i, j, k);
    a0 = ((i + j + k) & 1) == 0;
    a1 = !a0;
  }
  const int n0 = __syncthreads_count(a0), n1 = __syncthreads_count(a1);
  if (threadIdx.x == 0) {
    cnt[2 * blockIdx.x] = n0;
    cnt[2 * blockIdx.x + 1] = n1;
  }
}

__global__ void __launch_bounds__(kNT) k_mlist(MLevel L, const int *base, int *act) {
  constexpr int NWp = kNT / 32;
  __shared__ int wo[2][NWp];
  const long long c = (long long)blockIdx.x * kNT + threadIdx.x;
  bool a[2] = {false, false};
  if (c < L.ncell && L.m[c] > 0.0) {
    int i, j, k;
    ijk(L, c, i, j, k);
    a[(i + j + k) & 1] = true;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned bal[2];
  for (int q = 0; q < 2; q++) {
    bal[q] = __ballot_sync(0xffffffffu, a[q]);
    if (lane == 0) wo[q][w] = __popc(bal[q]);
  }
  __syncthreads();
  for (int q = 0; q < 2; q++) {
    if (!a[q]) continue;
    int o = base[2 * blockIdx.x + q];
    for (int v = 0; v < w; v++) o += wo[q][v];
    act[o + __popc(bal[q] & ((1u << lane) - 1u))] = (int)c;
  }
}

// One colour of a red-black Newton-Gauss-Seidel sweep over the active cells
// (one thread per active cell of the colour).
template <typename T, bool BG>
__global__ void __launch_bounds__(kNT) k_msmooth(MLevelT<T, BG> L, int colour, T cap, T relax) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  const long long n = colour ? L.na - L.na0 : L.na0;
  if (t >= n) return;
  const long long c = L.act[(colour ? L.na0 : 0) + t];
  T N, dN;
  m_cell(L, c, N, dN);
  T du = -relax * (N - L.f[c]) / dN;
  du = du > cap ? cap : (du < -cap ? -cap : du);
  const T un = L.u[c] + du;
  L.u[c] = un;
  L.b[c] = m_cache<T, BG>(un);
}

// d = L(u) - f on the active cells (one thread per active cell; ghosts' d is
// never read); per-block partials (sum d^2, max |d|).
template <typename T, bool BG>
__global__ void __launch_bounds__(kNT) k_mresid(MLevelT<T, BG> L, double *partial) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  // block sums in the level's precision (FP64 arithmetic runs at 1/64 of the
  // FP32 rate here), one FP64 pair written per block
  T s = T(0), mx = T(0);
  if (t < L.na) {
    const long long c = L.act[t];
    T N, dN;
    m_cell(L, c, N, dN);
    const T d = N - L.f[c];
    L.d[c] = d;
    s = d * d;
    mx = fabs(d);
  }
  __shared__ T ss[kNT / 32], sm[kNT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    ss[threadIdx.x >> 5] = s;
    sm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T a = T(0), b = T(0);
    for (int w = 0; w < kNT / 32; w++) {
      a += ss[w];
      b = fmax(b, sm[w]);
    }
    partial[2 * blockIdx.x] = (double)a;
    partial[2 * blockIdx.x + 1] = (double)b;
  }
}

// Setup of a coarser level: mean of the 8 children of the mask, the density
// and the (initial) values.
__global__ void __launch_bounds__(kNT) k_minit(MLevel F, MLevel C) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= C.ncell) return;
  int I, J, K;
  ijk(C, t, I, J, K);
  double sm = 0.0, sr = 0.0, su = 0.0;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const long long c = ((long long)(2 * K + (q >> 2)) * F.n1 + 2 * J + ((q >> 1) & 1)) * F.n0 +
                        2 * I + (q & 1);
    sm += F.m[c];
    sr += F.rho[c];
    su += F.u[c];
  }
  const_cast<double *>(C.m)[t] = 0.125 * sm;
  const_cast<double *>(C.rho)[t] = 0.125 * sr;
  C.u[t] = 0.125 * su;
}

// FAS restriction onto the active coarse cells: u^H = R u^h (all children),
// R d^h = sum over the active children / 8; ghosts keep their values.
template <typename T, bool BG>
__global__ void __launch_bounds__(kNT) k_mrestrict(MLevelT<T, BG> F, MLevelT<T, BG> C) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= C.ncell) return;
  if (!(C.m[t] > 0.0)) return;
  int I, J, K;
  ijk(C, t, I, J, K);
  T su = T(0), sd = T(0);
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const long long c = ((long long)(2 * K + (q >> 2)) * F.n1 + 2 * J + ((q >> 1) & 1)) * F.n0 +
                        2 * I + (q & 1);
    su += F.u[c];
    if (F.m[c] > 0.0) sd += F.d[c];
  }
  C.uR[t] = T(0.125) * su;
  C.u[t] = T(0.125) * su;
  C.b[t] = m_cache<T, BG>(T(0.125) * su);
  C.d[t] = T(0.125) * sd;
}

// f^H = L^H(R u^h) - R d^h on the active coarse cells (after k_mrestrict).
template <typename T, bool BG>
__global__ void __launch_bounds__(kNT) k_mfas(MLevelT<T, BG> C) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= C.ncell) return;
  if (!(C.m[t] > 0.0)) {
    C.f[t] = T(0);
    return;
  }
  T N, dN;
  m_cell(C, t, N, dN);
  C.f[t] = N - C.d[t];
}

// u^h += P e^H on the active fine cells (one thread per active cell), e^H =
// u^H - R u^h on active coarse cells and 0 on masked ones and outside the box
// (trilinear 27/9/3/1).
template <typename T, bool BG>
__global__ void __launch_bounds__(kNT) k_mprolong(MLevelT<T, BG> F, MLevelT<T, BG> C) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= F.na) return;
  const long long c = F.act[t];
  int i, j, k;
  ijk(F, c, i, j, k);
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const int di = (i & 1) ? 1 : -1, dj = (j & 1) ? 1 : -1, dk = (k & 1) ? 1 : -1;
  T acc = T(0);
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int ii = I + ((q & 1) ? di : 0), jj = J + (((q >> 1) & 1) ? dj : 0),
              kk = K + ((q >> 2) ? dk : 0);
    if (ii < 0 || ii >= C.n0 || jj < 0 || jj >= C.n1 || kk < 0 || kk >= C.n2) continue;
    const long long cc = ((long long)kk * C.n1 + jj) * C.n0 + ii;
    if (!(C.m[cc] > 0.0)) continue;
    const T w = T(((q & 1) ? 0.25 : 0.75) * (((q >> 1) & 1) ? 0.25 : 0.75) *
                  ((q >> 2) ? 0.25 : 0.75));
    acc += w * (C.u[cc] - C.uR[cc]);
  }
  const T un = F.u[c] + acc;
  F.u[c] = un;
  F.b[c] = m_cache<T, BG>(un);
}

// Coarsest level, one block: red-black sweeps until the rms over the active
// cells falls to max(1e-3 of its value before the first sweep, 0.1 tol), at
// most 500 sweeps.
constexpr int kCoNT = 1024;
template <typename T, bool BG>
__global__ void __launch_bounds__(kCoNT) k_mcoarsest(MLevelT<T, BG> L, long long nact, double tol,
                                                     T cap, T relax) {
  // the rms in the level's precision (FP64 arithmetic runs at 1/64 rate)
  __shared__ T red[kCoNT / 32];
  __shared__ T tot;
  auto rms = [&]() -> T {
    T s = T(0);
    for (long long c = threadIdx.x; c < L.ncell; c += kCoNT) {
      if (!(L.m[c] > 0.0)) continue;
      T N, dN;
      m_cell(L, c, N, dN);
      const T d = N - L.f[c];
      s += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      T t = T(0);
      for (int w = 0; w < kCoNT / 32; w++) t += red[w];
      tot = sqrt(t / (T)(nact > 0 ? nact : 1));
    }
    __syncthreads();
    const T r = tot;
    __syncthreads();
    return r;
  };
  const T thr = fmax(T(1e-3) * rms(), (T)(0.1 * tol));
  for (int it = 0; it < 500; it++) {
    for (int colour = 0; colour < 2; colour++) {
      for (long long c = threadIdx.x; c < L.ncell; c += kCoNT) {
        if (!(L.m[c] > 0.0)) continue;
        int i, j, k;
        ijk(L, c, i, j, k);
        if (((i + j + k) & 1) != colour) continue;
        T N, dN;
        m_cell(L, c, N, dN);
        T du = -relax * (N - L.f[c]) / dN;
        du = du > cap ? cap : (du < -cap ? -cap : du);
        const T un = L.u[c] + du;
        L.u[c] = un;
        L.b[c] = m_cache<T, BG>(un);
      }
      __syncthreads();
    }
    if (rms() <= thr) break;
  }
}

// Flags of a level's mask: [0] an outer-layer cell is active, [1] number of
// active cells.
__global__ void __launch_bounds__(kNT) k_mflags(MLevel L, unsigned long long *flags) {
  const long long c = (long long)blockIdx.x * kNT + threadIdx.x;
  if (c >= L.ncell) return;
  if (!(L.m[c] > 0.0)) return;
  int i, j, k;
  ijk(L, c, i, j, k);
  if (i == 0 || j == 0 || k == 0 || i == L.n0 - 1 || j == L.n1 - 1 || k == L.n2 - 1)
    atomicOr(&flags[0], 1ull);
  atomicAdd(&flags[1], 1ull);
}

// First phase of a mixed-precision solve: an FP32 copy of a level (iterate,
// exponential cache, zero right-hand side) ...
__global__ void __launch_bounds__(kNT) k_mto32(MLevel D, MLevelT<float> S) {
  const long long c = (long long)blockIdx.x * kNT + threadIdx.x;
  if (c >= D.ncell) return;
  const float v = (float)D.u[c];
  S.u[c] = v;
  S.b[c] = expf(v);
  S.f[c] = 0.0f;
}

// ... and its result back on the active cells of the FP64 finest level.
__global__ void __launch_bounds__(kNT) k_mto64(MLevelT<float> S, MLevel D) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= D.na) return;
  const long long c = D.act[t];
  const double v = (double)S.u[c];
  D.u[c] = v;
  D.b[c] = exp(v);
}

// Outer step of a mixed solve, finest level: background = the FP64 iterate
// rounded to FP32 (every cell), its exponential, correction 0, right-hand side
// -d (d the FP64 residual, active cells).
__global__ void __launch_bounds__(kNT) k_mbg_fine(MLevel D, MLevelT<float, true> S) {
  const long long c = (long long)blockIdx.x * kNT + threadIdx.x;
  if (c >= D.ncell) return;
  const float g = (float)D.u[c];
  S.bgu[c] = g;
  S.bgE[c] = expf(g);
  S.u[c] = 0.0f;
  S.b[c] = 0.0f;
  S.f[c] = D.m[c] > 0.0 ? -(float)D.d[c] : 0.0f;
}

// ... coarser levels: background the mean of the 8 children's, correction 0.
__global__ void __launch_bounds__(kNT) k_mbg_coarse(MLevelT<float, true> F,
                                                    MLevelT<float, true> C) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= C.ncell) return;
  int I, J, K;
  ijk(C, t, I, J, K);
  float sg = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const long long c = ((long long)(2 * K + (q >> 2)) * F.n1 + 2 * J + ((q >> 1) & 1)) * F.n0 +
                        2 * I + (q & 1);
    sg += F.bgu[c];
  }
  const float g = 0.125f * sg;
  C.bgu[t] = g;
  C.bgE[t] = expf(g);
  C.u[t] = 0.0f;
  C.b[t] = 0.0f;
}

// u += v on the active cells of the FP64 finest level, and its exponential.
__global__ void __launch_bounds__(kNT) k_madd64(MLevelT<float, true> S, MLevel D) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= D.na) return;
  const long long c = D.act[t];
  const double v = D.u[c] + (double)S.u[c];
  D.u[c] = v;
  D.b[c] = exp(v);
}

// Flags of the inputs: [0] a mask outside [-1, 1] or NaN, [1] a non-finite
// value or density (or a negative density unless allowed).
__global__ void __launch_bounds__(kNT) k_mcheck(const double *m, const double *rho,
                                                const double *u, long long n, int allow_neg,
                                                int *bad) {
  const long long c = (long long)blockIdx.x * kNT + threadIdx.x;
  if (c >= n) return;
  const double mv = m[c], r = rho[c], uv = u[c];
  if (!(mv >= -1.0 && mv <= 1.0)) atomicOr(&bad[0], 1);
  if (!isfinite(r) || !isfinite(uv) || (!allow_neg && r < 0.0)) atomicOr(&bad[1], 1);
}

}  // namespace

namespace {

bool m_on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct MArena {
  frmg_ctx *c;
  std::vector<void *> ptrs;
  explicit MArena(frmg_ctx *c_) : c(c_) {}
  template <typename T>
  T *get(size_t n) {
    void *p = nullptr;
    try {
      p = frmg_alloc(c, n * sizeof(T));
    } catch (...) {
      throw MError{FR_ENOMEM, "device allocation failed"};
    }
    ptrs.push_back(p);
    return (T *)p;
  }
  ~MArena() {
    for (void *p : ptrs) frmg_release(c, p);
  }
};

template <typename T, bool BG = false>
struct MSolver {
  frmg_ctx *ctx;
  cudaStream_t st;
  std::vector<MLevelT<T, BG>> lev;
  int pre, post;
  T cap, relax;
  double tol;
  double *partial;  // per-block (sum d^2, max |d|) of the finest level
  double *host;     // pinned staging of the partials
  long long nact0;  // active cells of the finest level

  void smooth(MLevelT<T, BG> &L, int n) {
    for (int s = 0; s < n; s++)
      for (int colour = 0; colour < 2; colour++) {
        k_msmooth<<<(unsigned)nblk(std::max(colour ? L.na - L.na0 : L.na0, 1ll)), kNT, 0, st>>>(
            L, colour, cap, relax);
        MLAUNCH(ctx);
      }
  }
  // rms over the active cells of level L (and its max |d|); host sync
  double rms(MLevelT<T, BG> &L, long long nact, double *dmax) {
    const long long nb = nblk(std::max(L.na, 1ll));
    k_mresid<<<(unsigned)nb, kNT, 0, st>>>(L, partial);
    MLAUNCH(ctx);
    MCK(cudaMemcpyAsync(host, partial, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    double s = 0.0, mx = 0.0;
    for (long long b = 0; b < nb; b++) {
      s += host[2 * b];
      mx = std::max(mx, host[2 * b + 1]);
    }
    if (dmax) *dmax = mx;
    return std::sqrt(s / (double)std::max(nact, 1ll));
  }
  void coarsest(MLevelT<T, BG> &L, long long nact) {
    k_mcoarsest<<<1, kCoNT, 0, st>>>(L, nact, tol, cap, relax);
    MLAUNCH(ctx);
  }
  std::vector<long long> nact;
  void vcycle(int l) {
    MLevelT<T, BG> &L = lev[l];
    if (l == (int)lev.size() - 1) {
      coarsest(L, nact[l]);
      return;
    }
    MLevelT<T, BG> &C = lev[l + 1];
    smooth(L, pre);
    k_mresid<<<(unsigned)nblk(std::max(L.na, 1ll)), kNT, 0, st>>>(L, partial);
    MLAUNCH(ctx);
    k_mrestrict<<<(unsigned)nblk(C.ncell), kNT, 0, st>>>(L, C);
    MLAUNCH(ctx);
    k_mfas<<<(unsigned)nblk(C.ncell), kNT, 0, st>>>(C);
    MLAUNCH(ctx);
    vcycle(l + 1);
    k_mprolong<<<(unsigned)nblk(std::max(L.na, 1ll)), kNT, 0, st>>>(L, C);
    MLAUNCH(ctx);
    smooth(L, post);
  }
};

}  // namespace

extern "C" int fr_solve_masked(frmg_ctx *ctx, const double *density, const double *mask,
                               const int dims[3], double h, double box_mpc_h, double a,
                               double omega_m, double fr0_abs, double tol, double *u_inout,
                               const fr_opts *opts, fr_stats *stats, void *stream) {
  MArena A(ctx);
  cudaStream_t st = (cudaStream_t)stream;
  try {
    const auto t0 = std::chrono::steady_clock::now();
    if (!ctx || !density || !mask || !dims || !u_inout) throw MError{FR_EINVAL, "NULL argument"};
    MCK(cudaSetDevice(frmg_device(ctx)));
    for (int d = 0; d < 3; d++)
      if (dims[d] < 3) throw MError{FR_EINVAL, "dims must be >= 3 (outer ghost layer)"};
    const long long nc = (long long)dims[0] * dims[1] * dims[2];
    if (nc >= (1ll << 31)) throw MError{FR_EINVAL, "region too large (at most 2^31 - 1 cells)"};
    if (!(h > 0) || !(tol >= 0)) throw MError{FR_EINVAL, "h must be > 0 and tol >= 0"};
    fr_opts o;
    fr_opts_default(&o);
    if (opts) o = *opts;
    if (o.pre < 0 || o.post < 0 || o.pre + o.post < 1 || o.max_vcycles < 0 ||
        !(o.newton_step_cap > 0) || !(o.relax > 0 && o.relax < 2))
      throw MError{FR_EINVAL, "invalid options"};
    double k6[6];
    if (fr_constants(box_mpc_h, 1, a, omega_m, fr0_abs, k6) != FR_OK)
      throw MError{FR_EINVAL, "box, a and |f_R0| must be > 0 and 0 < Omega_m < 1"};
    const double alpha = k6[0] / (h * h);  // alpha(h = 1) / h^2
    // inputs on the device
    auto stage_in = [&](const double *p) -> double * {
      double *d = A.get<double>(nc);
      MCK(cudaMemcpyAsync(d, p, nc * sizeof(double), m_on_device(p) ? cudaMemcpyDeviceToDevice
                                                                  : cudaMemcpyHostToDevice,
                          st));
      return d;
    };
    const bool u_dev = m_on_device(u_inout);
    double *du = stage_in(u_inout);
    const double *drho = m_on_device(density) ? density : stage_in(density);
    const double *dm = m_on_device(mask) ? mask : stage_in(mask);
    int *bad = A.get<int>(2);
    unsigned long long *flags = A.get<unsigned long long>(2);
    int hb[2];
    unsigned long long hf[2];
    MCK(cudaMemsetAsync(bad, 0, 2 * sizeof(int), st));
    k_mcheck<<<(unsigned)nblk(nc), kNT, 0, st>>>(dm, drho, du, nc, o.allow_negative_density, bad);
    MLAUNCH(ctx);
    MCK(cudaMemcpyAsync(hb, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    if (hb[0]) throw MError{FR_EINVAL, "mask values must lie in [-1, 1]"};
    if (hb[1]) throw MError{FR_EINVAL, "non-finite (or negative) density, or non-finite u"};
    // levels
    MSolver<double> S{ctx,    st,      {}, o.pre, o.post, o.newton_step_cap, o.relax, tol,
                      nullptr, nullptr, 0,  {}};
    auto make = [&](int n0, int n1, int n2, double hl, double *u, const double *m,
                    const double *rho) {
      MLevel L;
      L.n0 = n0;
      L.n1 = n1;
      L.n2 = n2;
      L.ncell = (long long)n0 * n1 * n2;
      L.fd0 = make_fastdiv((unsigned)n0);
      L.fd1 = make_fastdiv((unsigned)n1);
      L.u = u;
      L.b = A.get<double>(L.ncell);
      L.m = m;
      L.rho = rho;
      L.f = A.get<double>(L.ncell);
      L.uR = A.get<double>(L.ncell);
      L.d = A.get<double>(L.ncell);
      L.ub = A.get<double>(6 * L.ncell);
      L.act = nullptr;  // set once the level set is final
      L.na0 = L.na = 0;
      L.bgu = L.bgE = nullptr;
      L.ah = 0.5 * alpha * (h * h) / (hl * hl);
      L.beta = k6[1];
      L.gamma = k6[2];
      MCK(cudaMemsetAsync(L.f, 0, L.ncell * sizeof(double), st));
      return L;
    };
    auto level_flags = [&](MLevel &L) {
      MCK(cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned long long), st));
      k_mflags<<<(unsigned)nblk(L.ncell), kNT, 0, st>>>(L, flags);
      MLAUNCH(ctx);
      MCK(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
      MCK(cudaStreamSynchronize(st));
    };
    S.lev.push_back(make(dims[0], dims[1], dims[2], h, du, dm, drho));
    level_flags(S.lev[0]);
    if (hf[0]) throw MError{FR_EINVAL, "the outer layer of a masked region must be masked"};
    S.nact.push_back((long long)hf[1]);
    S.nact0 = (long long)hf[1];
    for (;;) {
      const MLevel &F = S.lev.back();
      if (F.n0 % 2 || F.n1 % 2 || F.n2 % 2 || F.n0 < 8 || F.n1 < 8 || F.n2 < 8) break;
      const int c0 = F.n0 / 2, c1 = F.n1 / 2, c2 = F.n2 / 2;
      const long long ncc = (long long)c0 * c1 * c2;
      MLevel C = make(c0, c1, c2, h * (double)(1 << S.lev.size()), A.get<double>(ncc),
                      A.get<double>(ncc), A.get<double>(ncc));
      k_minit<<<(unsigned)nblk(ncc), kNT, 0, st>>>(F, C);
      MLAUNCH(ctx);
      level_flags(C);
      if (hf[0] || hf[1] == 0) break;  // the level would not be a valid masked region
      S.lev.push_back(C);
      S.nact.push_back((long long)hf[1]);
    }
    for (auto &L : S.lev) {
      k_mub<<<(unsigned)nblk(L.ncell), kNT, 0, st>>>(L);
      MLAUNCH(ctx);
    }
    // active-cell lists of every level
    for (size_t l = 0; l < S.lev.size(); l++) {
      MLevel &L = S.lev[l];
      const long long nb = nblk(L.ncell);
      int *cnt = A.get<int>(2 * nb), *base = A.get<int>(2 * nb);
      int *act = A.get<int>(std::max(S.nact[l], 1ll));
      k_mcount<<<(unsigned)nb, kNT, 0, st>>>(L, cnt);
      MLAUNCH(ctx);
      std::vector<int> hc(2 * nb), hbase(2 * nb);
      MCK(cudaMemcpyAsync(hc.data(), cnt, 2 * nb * sizeof(int), cudaMemcpyDeviceToHost, st));
      MCK(cudaStreamSynchronize(st));
      long long n0 = 0, n1 = 0;  // colour 0 first, then colour 1
      for (long long b = 0; b < nb; b++) n0 += hc[2 * b];
      long long o0 = 0, o1 = n0;
      for (long long b = 0; b < nb; b++) {
        hbase[2 * b] = (int)o0;
        hbase[2 * b + 1] = (int)o1;
        o0 += hc[2 * b];
        o1 += hc[2 * b + 1];
        n1 += hc[2 * b + 1];
      }
      if (n0 + n1 != S.nact[l]) throw MError{FR_ECUDA, "active-cell count mismatch"};
      MCK(cudaMemcpyAsync(base, hbase.data(), 2 * nb * sizeof(int), cudaMemcpyHostToDevice, st));
      k_mlist<<<(unsigned)nb, kNT, 0, st>>>(L, base, act);
      MLAUNCH(ctx);
      MCK(cudaStreamSynchronize(st));
      L.act = act;
      L.na0 = n0;
      L.na = n0 + n1;
    }
    S.partial = A.get<double>(2 * nblk(nc));
    double *pin = frmg_pinned(ctx, 2 * nblk(nc));
    if (!pin) throw MError{FR_ENOMEM, "pinned host allocation failed"};
    S.host = pin;
    fr_stats sv;
    memset(&sv, 0, sizeof(sv));
    sv.tau_rms = std::nan("");
    double dmax = 0.0;
    double r = S.rms(S.lev[0], S.nact0, &dmax);
    sv.res0_rms = r;
    if (sv.nhist < FR_HIST) sv.hist[sv.nhist++] = r;
    int status = FR_OK;
    const bool mixed = o.prec == FR_MIXED;
    if (mixed && r > tol) {
      // first phase: FP32 V-cycles of the same scheme from the same start,
      // until their residual stalls (ratio >= 0.75), grows past 3x its best,
      // or falls to 1e-6 of the start or to tol
      MSolver<float> S32{ctx, st, {}, o.pre, o.post, (float)o.newton_step_cap, (float)o.relax,
                         tol, S.partial, S.host, S.nact0, S.nact};
      for (const MLevel &D : S.lev) {
        MLevelT<float> F;
        F.u = A.get<float>(D.ncell);
        F.b = A.get<float>(D.ncell);
        F.f = A.get<float>(D.ncell);
        F.uR = A.get<float>(D.ncell);
        F.d = A.get<float>(D.ncell);
        F.m = D.m;
        F.rho = D.rho;
        F.ub = D.ub;
        F.act = D.act;
        F.na0 = D.na0;
        F.na = D.na;
        F.n0 = D.n0;
        F.n1 = D.n1;
        F.n2 = D.n2;
        F.ncell = D.ncell;
        F.fd0 = D.fd0;
        F.fd1 = D.fd1;
        F.ah = (float)D.ah;
        F.beta = (float)D.beta;
        F.gamma = (float)D.gamma;
        F.bgu = F.bgE = nullptr;
        k_mto32<<<(unsigned)nblk(D.ncell), kNT, 0, st>>>(D, F);
        MLAUNCH(ctx);
        S32.lev.push_back(F);
      }
      const double r0 = r;
      double rp = r, best = r;
      bool ok = false;
      while (sv.vcycles < o.max_vcycles) {
        S32.vcycle(0);
        sv.vcycles++;
        double m32 = 0.0;
        const double rn = S32.rms(S32.lev[0], S.nact0, &m32);
        if (sv.nhist < FR_HIST) sv.hist[sv.nhist++] = rn;
        if (!(rn == rn)) {  // keep the FP64 start
          ok = false;
          break;
        }
        ok = true;
        const bool stop = rn <= tol || rn <= 1e-6 * r0 || rn >= 0.75 * rp || rn > 3.0 * best;
        rp = rn;
        best = std::min(best, rn);
        if (stop) break;
      }
      if (ok) {
        k_mto64<<<(unsigned)nblk(std::max(S.lev[0].na, 1ll)), kNT, 0, st>>>(S32.lev[0], S.lev[0]);
        MLAUNCH(ctx);
        r = S.rms(S.lev[0], S.nact0, &dmax);
        if (sv.nhist < FR_HIST) sv.hist[sv.nhist++] = -r;
        sv.outer++;
        // outer steps: opts->inner_cycles FP32 V-cycles of the correction form
        // against the FP64 residual, then u += v and the FP64 residual; a
        // step that does not halve it (or a non-finite correction) hands over
        // to FP64 V-cycles
        MSolver<float, true> SB{ctx,     st,     {}, o.pre, o.post, (float)o.newton_step_cap,
                                (float)o.relax, tol, S.partial, S.host, S.nact0, S.nact};
        for (const MLevelT<float> &F : S32.lev) {
          MLevelT<float, true> B;
          B.u = F.u;
          B.b = F.b;
          B.m = F.m;
          B.rho = F.rho;
          B.f = F.f;
          B.uR = F.uR;
          B.d = F.d;
          B.ub = F.ub;
          B.act = F.act;
          B.na0 = F.na0;
          B.na = F.na;
          B.n0 = F.n0;
          B.n1 = F.n1;
          B.n2 = F.n2;
          B.ncell = F.ncell;
          B.fd0 = F.fd0;
          B.fd1 = F.fd1;
          B.ah = F.ah;
          B.beta = F.beta;
          B.gamma = F.gamma;
          B.bgu = A.get<float>(F.ncell);
          B.bgE = A.get<float>(F.ncell);
          SB.lev.push_back(B);
        }
        const int inner = std::max(1, o.inner_cycles);
        double rp = r;
        while (r > tol && sv.vcycles < o.max_vcycles) {
          k_mbg_fine<<<(unsigned)nblk(S.lev[0].ncell), kNT, 0, st>>>(S.lev[0], SB.lev[0]);
          MLAUNCH(ctx);
          for (size_t l = 1; l < SB.lev.size(); l++) {
            k_mbg_coarse<<<(unsigned)nblk(SB.lev[l].ncell), kNT, 0, st>>>(SB.lev[l - 1],
                                                                           SB.lev[l]);
            MLAUNCH(ctx);
          }
          for (int k = 0; k < inner && sv.vcycles < o.max_vcycles; k++) {
            SB.vcycle(0);
            sv.vcycles++;
          }
          double mc = 0.0;
          const double rc = SB.rms(SB.lev[0], S.nact0, &mc);
          if (!(rc == rc)) break;
          k_madd64<<<(unsigned)nblk(std::max(S.lev[0].na, 1ll)), kNT, 0, st>>>(SB.lev[0],
                                                                                 S.lev[0]);
          MLAUNCH(ctx);
          r = S.rms(S.lev[0], S.nact0, &dmax);
          if (sv.nhist < FR_HIST) sv.hist[sv.nhist++] = -r;
          sv.outer++;
          if (!(r == r) || r > 0.5 * rp) break;
          rp = r;
        }
      }
    }
    while (r > tol) {
      if (sv.vcycles >= o.max_vcycles) {
        status = FR_ENOCONV;
        break;
      }
      S.vcycle(0);
      sv.vcycles++;
      r = S.rms(S.lev[0], S.nact0, &dmax);
      if (sv.nhist < FR_HIST) sv.hist[sv.nhist++] = mixed ? -r : r;
      if (mixed) sv.outer++;
      if (!(r == r)) {
        status = FR_EDIVERGED;
        break;
      }
    }
    sv.res_rms = r;
    sv.res_max = dmax;
    MCK(cudaMemcpyAsync(u_inout, du, nc * sizeof(double),
                        u_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    sv.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = sv;
    if (status == FR_ENOCONV) frmg_set_error("no convergence within opts->max_vcycles");
    if (status == FR_EDIVERGED) frmg_set_error("non-finite residual");
    return status;
  } catch (MError &e) {
    frmg_set_error(e.msg);
    if (st) cudaStreamSynchronize(st);
    else cudaDeviceSynchronize();
    return e.status;
  }
}
