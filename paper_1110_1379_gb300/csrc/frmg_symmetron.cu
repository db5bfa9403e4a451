// frmg_symmetron.cu -- FAS multigrid solve of the symmetron field equation on
// a periodic grid (sm_103a), the second scalar-field model on the machinery
// of the f(R) solver.
//
// The paper (Sec. I, Sec. VII) lists the symmetron (Hinterbichler & Khoury
// 2010) among the screened models whose equations its multigrid solver
// carries over to.  In chi = phi / phi_0 (phi_0 the vacuum value), with the
// vacuum range lambda_0 and the expansion factor a_SSB at which the mean
// matter density falls to the symmetry-breaking density, the quasi-static
// comoving equation is
//   laplacian chi = (a^2 / (2 lambda_0^2)) [ ((a_SSB / a)^3 rho - 1) chi + chi^3 ],
// rho the density in units of its mean.  Discretised with the 7-point
// Laplacian (Sec. IV) and divided by the bracket's coefficient, on a grid of
// cells of B h Mpc/h:
//   L_i(chi) = A sum_{6 faces} (chi_j - chi_i) - [ (s rho_i - 1) chi_i + chi_i^3 ],
//   A = 2 lambda_0^2 / (a^2 (B h)^2),  s = (a_SSB / a)^3,
// dL_i/dchi_i = -6 A - [ (s rho_i - 1) + 3 chi_i^2 ].
// The solve is the paper's (Sec. V.B.2): red-black Newton-Gauss-Seidel
// sweeps, FAS V-cycles (8-child average restriction of chi, of the residual
// and of the density; trilinear 27/9/3/1 prolongation of Sec. V.A.3), the
// coarse operator the same L with A / 4 per level.
//
// Precision: FR_FP64 runs every step in FP64.  FR_MIXED is a defect
// correction: the FP64 residual d = L(chi) and test rms(d) <= tol, and FP32
// FAS V-cycles on the correction equation
//   N(delta) = L(g + delta) - L(g) = -d,   g = fp32(chi) per level (restricted),
//   N_i = A sum (delta_j - delta_i) - delta_i [ (s rho_i - 1 + 3 g_i^2) + delta_i (3 g_i + delta_i) ],
// every term carrying a factor of delta (FP32 rounding relative to the
// correction), then chi += delta in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "frmg.h"
#include "frmg_dfmath.cuh"
#include "frmg_internal.h"

namespace {

struct SError {
  int status;
  std::string msg;
};

#define SCK(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      cudaGetLastError();                                                           \
      throw SError{FR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};   \
    }                                                                               \
  } while (0)
#define SLAUNCH(ctx)                                                                      \
  do {                                                                                    \
    frmg_launch_counter(ctx)++;                                                           \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess)                                                                \
      throw SError{FR_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)};    \
  } while (0)

constexpr int kNT = 256;

struct SArena {
  frmg_ctx *c;
  std::vector<void *> ptrs;
  explicit SArena(frmg_ctx *c_) : c(c_) {}
  template <typename T>
  T *get(size_t n) {
    void *p = nullptr;
    try {
      p = frmg_alloc(c, std::max<size_t>(n, 1) * sizeof(T));
    } catch (...) {
      throw SError{FR_ENOMEM, "device allocation failed"};
    }
    ptrs.push_back(p);
    return (T *)p;
  }
  ~SArena() {
    for (void *p : ptrs) frmg_release(c, p);
  }
};

// One level of the hierarchy.  Full form (FP64 solve): u = chi.  Correction
// form (FP32 inner solve): u = delta, g = background fp32(chi) restricted.
template <typename T>
struct SLevel {
  T *u;            // unknown (the current buffer)
  T *u2;           // second buffer of the register-column smoother (null: not used)
  int zc;          // its z-chunk
  T *uR;           // restricted fine unknown (coarse levels)
  T *f;            // right-hand side (FAS); null = 0
  const T *rho;    // density (mean 1), restricted on coarse levels
  const float *g;  // background (correction form), null otherwise
  int n0, n1, n2;
  long long nc;
  T A, s, cap, relax;
  frmg::FastDiv fd0, fd1;  // division by n0 and n1 (grids below 2^31 cells)
};

// (i, j, k) of cell c: 32-bit multiply-shift division below 2^31 cells
template <typename T>
__device__ __forceinline__ void sy_ijk(const SLevel<T> &L, long long c, int &i, int &j, int &k) {
  if (L.nc < (1ll << 31)) {
    const unsigned cu = (unsigned)c, q = frmg::fdiv(cu, L.fd0), q2 = frmg::fdiv(q, L.fd1);
    i = (int)(cu - q * (unsigned)L.n0);
    j = (int)(q - q2 * (unsigned)L.n1);
    k = (int)q2;
    return;
  }
  i = (int)(c % L.n0);
  const long long r = c / L.n0;
  j = (int)(r % L.n1);
  k = (int)(r / L.n1);
}

// N_i and dN_i/du_i at cell (i, j, k); CORR selects the correction form.
template <typename T, bool CORR>
__device__ __forceinline__ void sy_op(const SLevel<T> &L, int i, int j, int k, T &N, T &dN) {
  const long long sx = 1, sy = L.n0, sz = (long long)L.n0 * L.n1;
  const long long c = ((long long)k * L.n1 + j) * L.n0 + i;
  const T ui = L.u[c];
  const long long xm = i > 0 ? c - sx : c + (L.n0 - 1) * sx;
  const long long xp = i < L.n0 - 1 ? c + sx : c - (L.n0 - 1) * sx;
  const long long ym = j > 0 ? c - sy : c + (L.n1 - 1) * sy;
  const long long yp = j < L.n1 - 1 ? c + sy : c - (L.n1 - 1) * sy;
  const long long zm = k > 0 ? c - sz : c + (L.n2 - 1) * sz;
  const long long zp = k < L.n2 - 1 ? c + sz : c - (L.n2 - 1) * sz;
  const T lap = (L.u[xm] - ui) + (L.u[xp] - ui) + (L.u[ym] - ui) + (L.u[yp] - ui) +
                (L.u[zm] - ui) + (L.u[zp] - ui);
  const T m = L.s * L.rho[c] - T(1);
  if (CORR) {
    const T gi = (T)L.g[c];
    const T lin = m + T(3) * gi * gi;
    N = L.A * lap - ui * (lin + ui * (T(3) * gi + ui));
    const T w = gi + ui;
    dN = T(-6) * L.A - (m + T(3) * w * w);
  } else {
    N = L.A * lap - (m * ui + ui * ui * ui);
    dN = T(-6) * L.A - (m + T(3) * ui * ui);
  }
}

template <typename T>
__device__ __forceinline__ T sy_rhs(const SLevel<T> &L, long long c) {
  return L.f ? L.f[c] : T(0);
}

// One colour of a red-black Newton-Gauss-Seidel sweep (red = (i + j + k) even).
template <typename T, bool CORR>
__global__ void __launch_bounds__(kNT) k_sy_smooth(SLevel<T> L, int colour) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * t >= L.nc) return;
  int i, j, k;
  sy_ijk(L, 2 * t, i, j, k);
  i += (j + k + colour) & 1;
  T N, dN;
  sy_op<T, CORR>(L, i, j, k, N, dN);
  const long long c = ((long long)k * L.n1 + j) * L.n0 + i;
  T du = -L.relax * (N - sy_rhs(L, c)) / dN;
  du = du > L.cap ? L.cap : (du < -L.cap ? -L.cap : du);
  L.u[c] += du;
}

// Block partials (sum of squares, max |v|) into part[2 blockIdx.x ..].
template <typename T>
__device__ __forceinline__ void sy_block_norms(T v2, T vmax, double *part) {
  // reduced in the values' own precision (FP64 arithmetic runs at 1/64 of the
  // FP32 rate here; FP32 sums are ample for a stopping test), one FP64 pair
  // written per block
  __shared__ T ss[kNT / 32], sm[kNT / 32];
  T s = v2, m = vmax;
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    ss[w] = s;
    sm[w] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T ts = T(0), tm = T(0);
    for (int q = 0; q < kNT / 32; q++) {
      ts += ss[q];
      tm = fmax(tm, sm[q]);
    }
    part[2 * blockIdx.x] = (double)ts;
    part[2 * blockIdx.x + 1] = (double)tm;
  }
}

// Residual d = N(u) - f of the 8 children of each coarse cell, restricted:
// coarse uR = u^H = mean of the children's u, coarse f = mean of d (the FAS
// right-hand side is completed by k_sy_fas_rhs); optional norm partials of d.
template <typename T, bool CORR>
__global__ void __launch_bounds__(kNT) k_sy_resid_restrict(SLevel<T> F, SLevel<T> Cs,
                                                           double *part) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  T s2 = T(0), mx = T(0);
  if (t < Cs.nc) {
    int I, J, K;
    sy_ijk(Cs, t, I, J, K);
    T su = T(0), sd = T(0);
    for (int q = 0; q < 8; q++) {
      const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
      const long long c = ((long long)k * F.n1 + j) * F.n0 + i;
      T N, dN;
      sy_op<T, CORR>(F, i, j, k, N, dN);
      const T d = N - sy_rhs(F, c);
      su += F.u[c];
      sd += d;
      s2 += d * d;
      mx = fmax(mx, fabs(d));
    }
    const T uh = su * T(0.125);
    Cs.uR[t] = uh;
    Cs.u[t] = uh;
    Cs.f[t] = sd * T(0.125);
  }
  if (part) sy_block_norms<T>(s2, mx, part);
}

// FAS right-hand side of a coarse level: f <- N^H(u^H) - f (f holding R d^h).
template <typename T, bool CORR>
__global__ void __launch_bounds__(kNT) k_sy_fas_rhs(SLevel<T> Cs) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Cs.nc) return;
  int i, j, k;
  sy_ijk(Cs, t, i, j, k);
  T N, dN;
  sy_op<T, CORR>(Cs, i, j, k, N, dN);
  Cs.f[t] = N - Cs.f[t];
}

// u^h += P(u^H - R u^h): the trilinear 27/9/3/1 prolongation (Sec. V.A.3) of
// the coarse correction onto every fine cell, periodic.  One thread per
// coarse cell: the correction e = u^H - uR of its 3 x 3 x 3 coarse
// neighbourhood is read once and blended into its 8 children (the nearer
// coarse cell of a child is its parent, the farther one is the neighbour on
// the child's side), each child's x-pair row updated with one paired access.
template <typename T>
__global__ void __launch_bounds__(kNT) k_sy_prolong(SLevel<T> F, SLevel<T> Cs) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Cs.nc) return;
  int I, J, K;
  sy_ijk(Cs, t, I, J, K);
  const int Im = I == 0 ? Cs.n0 - 1 : I - 1, Ip = I + 1 == Cs.n0 ? 0 : I + 1;
  const int Jm = J == 0 ? Cs.n1 - 1 : J - 1, Jp = J + 1 == Cs.n1 ? 0 : J + 1;
  const int Km = K == 0 ? Cs.n2 - 1 : K - 1, Kp = K + 1 == Cs.n2 ? 0 : K + 1;
  const int xs[3] = {Im, I, Ip}, ys[3] = {Jm, J, Jp}, zs[3] = {Km, K, Kp};
  T e[3][3][3];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int b = 0; b < 3; b++)
#pragma unroll
      for (int a = 0; a < 3; a++) {
        const long long q = ((long long)zs[c] * Cs.n1 + ys[b]) * Cs.n0 + xs[a];
        e[c][b][a] = Cs.u[q] - Cs.uR[q];
      }
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
#pragma unroll
  for (int cz = 0; cz < 2; cz++)
#pragma unroll
    for (int cy = 0; cy < 2; cy++) {
      const int k2 = cz ? 2 : 0, j2 = cy ? 2 : 0;  // farther z and y neighbours
      T v[2];
#pragma unroll
      for (int cx = 0; cx < 2; cx++) {
        const int i2 = cx ? 2 : 0;
        v[cx] = T(27) * e[1][1][1] + T(9) * (e[1][1][i2] + e[1][j2][1] + e[k2][1][1]) +
                T(3) * (e[1][j2][i2] + e[k2][1][i2] + e[k2][j2][1]) + e[k2][j2][i2];
      }
      const long long f = ((long long)(2 * K + cz) * F.n1 + (2 * J + cy)) * F.n0 + 2 * I;
      T2 *fu = reinterpret_cast<T2 *>(F.u + f);
      T2 uu = *fu;
      uu.x += v[0] * T(1.0 / 64.0);
      uu.y += v[1] * T(1.0 / 64.0);
      *fu = uu;
    }
}

// Coarsest level: one block relaxes the whole grid until its rms residual has
// fallen by `rel` (or below `abs_`), at most maxit sweeps, or (stall != 0,
// the FP32 solve at its rounding floor) four sweeps in a row have not brought
// it below 0.9 of its best value (a single sweep may raise the rms of a
// red-black sweep's residual without the solve having stalled).
template <typename T, bool CORR>
__global__ void __launch_bounds__(kNT) k_sy_coarsest(SLevel<T> L, double rel, double abs_,
                                                     int maxit, int stall) {
  // the rms in the level's precision (FP64 arithmetic runs at 1/64 rate)
  __shared__ T red[kNT / 32];
  __shared__ T lim_s, best_s;
  __shared__ int stop_s, flat_s;
  auto rms = [&]() -> T {
    T s = T(0);
    for (long long c = threadIdx.x; c < L.nc; c += blockDim.x) {
      int i, j, k;
      sy_ijk(L, c, i, j, k);
      T N, dN;
      sy_op<T, CORR>(L, i, j, k, N, dN);
      const T d = N - sy_rhs(L, c);
      s += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    T tot = T(0);
    for (int q = 0; q < kNT / 32; q++) tot += red[q];
    return sqrt(tot / (T)L.nc);
  };
  const T r0 = rms();
  if (threadIdx.x == 0) {
    lim_s = fmax((T)rel * r0, (T)abs_);
    best_s = r0;
    flat_s = 0;
    stop_s = 0;  // at least one sweep
  }
  __syncthreads();
  for (int it = 0; it < maxit && !stop_s; it++) {
    for (int colour = 0; colour < 2; colour++) {
      for (long long t = threadIdx.x; 2 * t < L.nc; t += blockDim.x) {
        int i, j, k;
        sy_ijk(L, 2 * t, i, j, k);
        i += (j + k + colour) & 1;
        T N, dN;
        sy_op<T, CORR>(L, i, j, k, N, dN);
        const long long c = ((long long)k * L.n1 + j) * L.n0 + i;
        T du = -L.relax * (N - sy_rhs(L, c)) / dN;
        du = du > L.cap ? L.cap : (du < -L.cap ? -L.cap : du);
        L.u[c] += du;
      }
      __syncthreads();
    }
    const T r = rms();
    if (threadIdx.x == 0) {
      if (r < T(0.9) * best_s) {
        best_s = r;
        flat_s = 0;
      } else {
        flat_s++;
      }
      stop_s = r <= lim_s || !(r == r) || (stall && flat_s >= 4);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int wrapmod_sy(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// One red-black sweep of the FP32 correction form with register-resident
// z-columns (periodic grids of at least 16 cells a side): the layout and
// march of the f(R) solver's register-column smoother on 64 x 8 tiles with a
// halo of two cells.  Every x-pair of the tile plus halo has one owner
// thread that keeps, for the last four planes, the pair's red and black cell
// (delta and the cell's coefficients c1 = s rho - 1 + 3 g^2, c2 = 3 g and
// right-hand side f) in registers; only delta crosses between threads,
// through double-buffered half-planes in shared memory.  At the step that
// loads plane p: the black cells of p are published (old values), the red
// cells of p-1 on the tile grown by one cell are updated from black
// neighbours and published, and the black cells of p-2 on the tile are
// updated from the new red cells and written out (delta only; the
// coefficients are recomputed from rho and g at every load).  Reads buffer
// uin, writes uout (halos come from the unmodified input), so the sweep is
// the same as two launches of k_sy_smooth up to FP32 rounding order.
constexpr int kSyTX = 64, kSyTY = 8, kSyPX = kSyTX / 2 + 2, kSyLY = kSyTY + 4;
constexpr int kSyPP = kSyPX * kSyLY, kSyNHR = 4 * (kSyTX / 2), kSyNHALO = kSyNHR + 2 * kSyLY;
static_assert(kSyNHALO <= kNT, "halo pairs per thread");

__global__ void __launch_bounds__(kNT, 3)
    k_sy_smooth_rc(SLevel<float> L, const float *__restrict__ uin, float *__restrict__ uout,
                   int zc) {
  constexpr int NSL = 2;  // one interior pair, one halo pair
  __shared__ float sbk[2][kSyPP], srd[2][kSyPP];
  const int n0 = L.n0, n1 = L.n1, n2 = L.n2;
  const int ntx = (n0 + kSyTX - 1) / kSyTX, nty = (n1 + kSyTY - 1) / kSyTY;
  int b = blockIdx.x;
  const int X0 = (b % ntx) * kSyTX;
  b /= ntx;
  const int Y0 = (b % nty) * kSyTY;
  b /= nty;
  const int Z0 = b * zc;
  const int Z1 = min(Z0 + zc, n2);
  const int P0 = Z0 - 2, nstep = Z1 - Z0 + 4;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long plane = (long long)n0 * n1;
  const float A = L.A, s = L.s, cap = L.cap, relax = L.relax;
  const float *__restrict__ rho = L.rho;
  const float *__restrict__ gin = L.g;
  const float *__restrict__ fin = L.f;
  int q[NSL], roff[NSL];
  unsigned fl[NSL], ro[NSL];  // fl: bit 0 load, 1 write, 2 / 3 red update of even / odd cell
#pragma unroll
  for (int sl = 0; sl < NSL; sl++) {
    int px = -1, ly = -1;
    const bool interior = sl == 0;
    if (interior) {
      px = 1 + lane;
      ly = 2 + w;
    } else if ((int)threadIdx.x < kSyNHALO) {
      const int t = threadIdx.x;
      if (t < kSyNHR) {
        const int r = t >> 5;
        px = 1 + lane;
        ly = r < 2 ? r : kSyTY + r;
      } else {
        const int k = t - kSyNHR;
        px = k < kSyLY ? 0 : kSyPX - 1;
        ly = k < kSyLY ? k : k - kSyLY;
      }
    }
    q[sl] = 0;
    roff[sl] = 0;
    fl[sl] = 0;
    ro[sl] = 0;
    if (px < 0) continue;
    const int gx = X0 - 2 + 2 * px, gy = Y0 - 2 + ly;
    q[sl] = ly * kSyPX + px;
    ro[sl] = (unsigned)((gy + P0) & 1);
    roff[sl] = wrapmod_sy(gy, n1) * n0 + wrapmod_sy(gx, n0);
    unsigned f = 1u;
    const bool yin = gy >= Y0 - 1 && gy <= Y0 + kSyTY;
    if (yin && gx >= X0 - 1 && gx <= X0 + kSyTX) f |= 4u;
    if (yin && gx + 1 >= X0 - 1 && gx + 1 <= X0 + kSyTX) f |= 8u;
    if (interior && gx < n0 && gy < n1) f |= 2u;
    fl[sl] = f;
  }
  // per slot and ring plane: red and black cell (delta, c1, c2, f)
  float4 R[NSL][4], B[NSL][4];
  float2 pu[NSL], pr[NSL], pg[NSL], pf[NSL];
#pragma unroll
  for (int sl = 0; sl < NSL; sl++) {
    pu[sl] = pr[sl] = pg[sl] = pf[sl] = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < 4; r++) R[sl][r] = B[sl][r] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  int pw = wrapmod_sy(P0, n2);
  auto fetch = [&]() {
    const long long zo = (long long)pw * plane;
#pragma unroll
    for (int sl = 0; sl < NSL; sl++) {
      if (!(fl[sl] & 1u)) continue;
      const long long o = zo + roff[sl];
      pu[sl] = *reinterpret_cast<const float2 *>(uin + o);
      pr[sl] = *reinterpret_cast<const float2 *>(rho + o);
      pg[sl] = *reinterpret_cast<const float2 *>(gin + o);
      pf[sl] = fin ? *reinterpret_cast<const float2 *>(fin + o) : make_float2(0.f, 0.f);
    }
    pw = pw + 1 == n2 ? 0 : pw + 1;
  };
  fetch();
  auto cell = [&](float d, float r, float g, float f) {
    return make_float4(d, s * r - 1.0f + 3.0f * g * g, 3.0f * g, f);
  };
  // Newton update: own (delta, c1, c2, f), six neighbour deltas
  auto newton = [&](float4 c, float lf, float rt, float ym, float yp, float zm, float zp) {
    const float d = c.x;
    const float lap = (lf - d) + (rt - d) + (ym - d) + (yp - d) + (zm - d) + (zp - d);
    const float N = A * lap - d * (c.y + d * (c.z + d));
    const float dN = -6.0f * A - (c.y + d * (2.0f * c.z + 3.0f * d));
    float du = -relax * (N - c.w) / dN;
    du = fminf(fmaxf(du, -cap), cap);
    return d + du;
  };
  auto step = [&](auto Kc, int k) {
    constexpr int K = decltype(Kc)::value;
    constexpr int K1 = (K + 3) & 3, K2 = (K + 2) & 3, K3 = (K + 1) & 3;
    constexpr unsigned PK = K & 1, PK1 = K1 & 1, PK2 = K2 & 1;
    const int p = P0 + k;
#pragma unroll
    for (int sl = 0; sl < NSL; sl++) {
      if (!(fl[sl] & 1u)) continue;
      const bool odd = (ro[sl] ^ PK) != 0;  // red cell is the odd one
      const float4 e = cell(pu[sl].x, pr[sl].x, pg[sl].x, pf[sl].x);
      const float4 o = cell(pu[sl].y, pr[sl].y, pg[sl].y, pf[sl].y);
      R[sl][K] = odd ? o : e;
      B[sl][K] = odd ? e : o;
      sbk[PK][q[sl]] = B[sl][K].x;
    }
    if (k + 1 < nstep) fetch();
    {
      const int m = p - 1;
      if (m >= Z0 - 1 && m <= Z1) {
#pragma unroll
        for (int sl = 0; sl < NSL; sl++) {
          const bool odd = (ro[sl] ^ PK1) != 0;
          if (!((sl == 0) || (fl[sl] & (odd ? 8u : 4u)))) continue;
          const float *bk = &sbk[PK1][q[sl]];
          const float nx = bk[odd ? 1 : -1];
          const float in = B[sl][K1].x;
          const float dn = newton(R[sl][K1], odd ? in : nx, odd ? nx : in, bk[-kSyPX], bk[kSyPX],
                                  B[sl][K2].x, B[sl][K].x);
          R[sl][K1].x = dn;
          srd[PK1][q[sl]] = dn;
        }
      }
    }
    {
      const int m = p - 2;
      if (m >= Z0 && m < Z1) {
        const bool odd = (ro[0] ^ PK2) == 0;  // black cell is the odd one
        const float *rd = &srd[PK2][q[0]];
        const float nx = rd[odd ? 1 : -1];
        const float in = R[0][K2].x;
        const float dn = newton(B[0][K2], odd ? in : nx, odd ? nx : in, rd[-kSyPX], rd[kSyPX],
                                R[0][K3].x, R[0][K1].x);
        B[0][K2].x = dn;
        if (fl[0] & 2u) {
          const float de = odd ? R[0][K2].x : dn, dd = odd ? dn : R[0][K2].x;
          *reinterpret_cast<float2 *>(uout + (long long)m * plane + roff[0]) = make_float2(de, dd);
        }
      }
    }
    __syncthreads();
  };
  for (int k = 0; k < nstep; k += 4) {
    step(std::integral_constant<int, 0>{}, k);
    if (k + 1 < nstep) step(std::integral_constant<int, 1>{}, k + 1);
    if (k + 2 < nstep) step(std::integral_constant<int, 2>{}, k + 2);
    if (k + 3 < nstep) step(std::integral_constant<int, 3>{}, k + 3);
  }
}

// 8-child average of an array (coarse dims c0 x c1 x c2).
template <typename S, typename D>
__global__ void __launch_bounds__(kNT) k_sy_restrict(const S *fine, D *coarse, int c0, int c1,
                                                     int c2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nc = (long long)c0 * c1 * c2;
  if (t >= nc) return;
  const int I = (int)(t % c0);
  const long long r = t / c0;
  const int J = (int)(r % c1), K = (int)(r / c1);
  const int f0 = 2 * c0, f1 = 2 * c1;
  double s = 0.0;
  for (int q = 0; q < 8; q++) {
    const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
    s += (double)fine[((long long)k * f1 + j) * f0 + i];
  }
  coarse[t] = (D)(s * 0.125);
}

// FP64 residual of the full equation, d = L(chi), with norm partials.
__global__ void __launch_bounds__(kNT) k_sy_defect64(SLevel<double> L, double *d, double *part) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (t < L.nc) {
    int i, j, k;
    sy_ijk(L, t, i, j, k);
    double N, dN;
    sy_op<double, false>(L, i, j, k, N, dN);
    v = N;
    if (d) d[t] = v;
  }
  sy_block_norms<double>(v * v, fabs(v), part);
}

__global__ void __launch_bounds__(kNT) k_sy_fill(double *v, double x, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) v[t] = x;
}

template <typename S, typename D>
__global__ void __launch_bounds__(kNT) k_sy_convert(const S *in, D *out, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (D)in[t];
}

// ---- double-float outer loop of the mixed solve (FP64 accuracy on the FP32
// pipes, see frmg_dfmath.cuh): chi and rho are held as (hi, lo) pairs.
__global__ void __launch_bounds__(kNT) k_sy_split(const double *v, float2 *p, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double x = v[t];
  const float h = (float)x;
  p[t] = make_float2(h, (float)(x - (double)h));
}

__global__ void __launch_bounds__(kNT) k_sy_join(const float2 *p, double *v, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) v[t] = (double)p[t].x + (double)p[t].y;
}

// Defect of chi in double-float, two cells (an x-pair; every grid has an even
// n0) per thread on packed FP32 pairs (frmg_dfmath.cuh: add/sub/fma .f32x2,
// products per lane), and the set-up of the FP32 correction problem of the
// next outer step: g = hi(chi), f = -hi(d), delta = 0.  The six face
// differences are summed in the face order -x, +x, -y, +y, -z, +z, then
// d = A lap - chi (s rho - 1 + chi^2).  Block norms (FP32) of 2 kNT cells.
__global__ void __launch_bounds__(kNT) k_sy_defect_df(SLevel<float> L, const float2 *chi,
                                                      const float2 *rho, float Ah, float Al,
                                                      float sh, float sl, float *g, float *f,
                                                      float *delta, double *part) {
  using frmg::df2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float s2 = 0.0f, mx = 0.0f;
  if (t < (L.nc >> 1)) {
    const long long c = 2 * t;
    int i, j, k;
    sy_ijk(L, c, i, j, k);
    const long long sy = L.n0, sz = (long long)L.n0 * L.n1;
    const float4 *C4 = reinterpret_cast<const float4 *>(chi);
    const float4 cv = C4[t];
    const df2 ci = {make_float2(cv.x, cv.z), make_float2(cv.y, cv.w)};
    auto pair = [&](long long cj) {  // the neighbouring pair starting at cell cj (even)
      const float4 v = C4[cj >> 1];
      return df2{make_float2(v.x, v.z), make_float2(v.y, v.w)};
    };
    // -x: cells (2p - 1, 2p); +x: cells (2p + 1, 2p + 2), wrapping in the row
    const float2 l = chi[i > 0 ? c - 1 : c + L.n0 - 1];
    const float2 r = chi[i + 2 < L.n0 ? c + 2 : c + 2 - L.n0];
    df2 lap = frmg::df_sub2(df2{make_float2(l.x, cv.x), make_float2(l.y, cv.y)}, ci);
    lap = frmg::df_add2(lap, frmg::df_sub2(df2{make_float2(cv.z, r.x), make_float2(cv.w, r.y)}, ci));
    lap = frmg::df_add2(lap, frmg::df_sub2(pair(j > 0 ? c - sy : c + (L.n1 - 1) * sy), ci));
    lap = frmg::df_add2(lap, frmg::df_sub2(pair(j < L.n1 - 1 ? c + sy : c - (L.n1 - 1) * sy), ci));
    lap = frmg::df_add2(lap, frmg::df_sub2(pair(k > 0 ? c - sz : c + (L.n2 - 1) * sz), ci));
    lap = frmg::df_add2(lap, frmg::df_sub2(pair(k < L.n2 - 1 ? c + sz : c - (L.n2 - 1) * sz), ci));
    const float4 rv = reinterpret_cast<const float4 *>(rho)[t];
    const df2 rp = {make_float2(rv.x, rv.z), make_float2(rv.y, rv.w)};
    const df2 m = frmg::df_add_f2(frmg::df_mul2(rp, df2{frmg::splat2(sh), frmg::splat2(sl)}),
                                  -1.0f);  // s rho - 1
    const df2 loc = frmg::df_mul2(ci, frmg::df_add2(m, frmg::df_mul2(ci, ci)));  // chi (m + chi^2)
    const df2 d = frmg::df_sub2(frmg::df_mul2(lap, df2{frmg::splat2(Ah), frmg::splat2(Al)}), loc);
    const float2 v = frmg::add2(d.h, d.l);
    reinterpret_cast<float2 *>(g)[t] = ci.h;
    reinterpret_cast<float2 *>(f)[t] = make_float2(-d.h.x, -d.h.y);
    reinterpret_cast<float2 *>(delta)[t] = make_float2(0.0f, 0.0f);
    s2 = fmaf(v.y, v.y, v.x * v.x);
    mx = fmaxf(fabsf(v.x), fabsf(v.y));
  }
  sy_block_norms<float>(s2, mx, part);
}

// chi += delta in double-float
__global__ void __launch_bounds__(kNT) k_sy_update_df(float2 *chi, const float *delta,
                                                      long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float2 c = chi[t];
  const frmg::df r = frmg::df_add_f({c.x, c.y}, delta[t]);
  chi[t] = make_float2(r.h, r.l);
}

// First stage of a long partial-pair sum: block b reduces pairs
// [b 4096, (b + 1) 4096) in a fixed order.
constexpr int kSyRedCH = 4096;
__global__ void __launch_bounds__(kNT) k_sy_reduce_chunks(const double *in, long long n,
                                                          double *out) {
  const long long b0 = (long long)blockIdx.x * kSyRedCH;
  const long long b1 = b0 + kSyRedCH < n ? b0 + kSyRedCH : n;
  double s = 0.0, m = 0.0;
  for (long long i = b0 + threadIdx.x; i < b1; i += kNT) {
    s += in[2 * i];
    m = fmax(m, in[2 * i + 1]);
  }
  sy_block_norms<double>(s, m, out);
}

// density check: finite and, the model's density being a mass density, >= 0
__global__ void __launch_bounds__(kNT) k_sy_check_rho(const double *rho, long long n, int *bad) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const double r = rho[t];
    if (!(r >= 0.0) || isinf(r)) atomicOr(bad, 1);
  }
}

// sum and max of per-block partial pairs, one block, fixed order
__global__ void __launch_bounds__(kNT) k_sy_reduce(const double *part, long long nb,
                                                   double *out) {
  __shared__ double ss[kNT], sm[kNT];
  double s = 0.0, m = 0.0;
  for (long long b = threadIdx.x; b < nb; b += kNT) {
    s += part[2 * b];
    m = fmax(m, part[2 * b + 1]);
  }
  ss[threadIdx.x] = s;
  sm[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0.0, tm = 0.0;
    for (int q = 0; q < kNT; q++) {
      ts += ss[q];
      tm = fmax(tm, sm[q]);
    }
    out[0] = ts;
    out[1] = tm;
  }
}

long long nblk(long long n) { return (n + kNT - 1) / kNT; }

int sm_count_sy() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return std::max(n, 1);
}

bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int sy_levels(const int n[3]) {
  int m[3] = {n[0], n[1], n[2]};
  int nl = 1;
  while (m[0] % 2 == 0 && m[1] % 2 == 0 && m[2] % 2 == 0 && m[0] / 2 >= 4 && m[1] / 2 >= 4 &&
         m[2] / 2 >= 4) {
    for (int d = 0; d < 3; d++) m[d] /= 2;
    nl++;
  }
  return nl;
}

// The hierarchy of one precision and form, and the V-cycle on it.
template <typename T, bool CORR>
struct SHier {
  std::vector<SLevel<T>> lev;
  frmg_ctx *ctx;
  cudaStream_t st;
  int pre, post;
  double *part0;  // fine norm partials of the residual + restriction (or null)
  double crs_abs;  // absolute floor of the coarsest solve (FP64: 0.1 tol)

  void smooth(int l, int sweeps) {
    SLevel<T> &L = lev[l];
    if constexpr (CORR && sizeof(T) == 4) {
      if (L.u2) {
        const int ntx = (L.n0 + kSyTX - 1) / kSyTX, nty = (L.n1 + kSyTY - 1) / kSyTY;
        const unsigned nb = (unsigned)(ntx * nty * ((L.n2 + L.zc - 1) / L.zc));
        for (int it = 0; it < sweeps; it++) {
          k_sy_smooth_rc<<<nb, kNT, 0, st>>>(L, L.u, L.u2, L.zc);
          SLAUNCH(ctx);
          std::swap(L.u, L.u2);
        }
        return;
      }
    }
    const long long half = (L.nc + 1) / 2;
    for (int it = 0; it < sweeps; it++)
      for (int colour = 0; colour < 2; colour++) {
        k_sy_smooth<T, CORR><<<(unsigned)nblk(half), kNT, 0, st>>>(L, colour);
        SLAUNCH(ctx);
      }
  }
  void vcycle(int l) {
    const int nl = (int)lev.size();
    if (l == nl - 1) {
      k_sy_coarsest<T, CORR><<<1, kNT, 0, st>>>(lev[l], 1e-3, crs_abs, 500, CORR ? 1 : 0);
      SLAUNCH(ctx);
      return;
    }
    smooth(l, pre);
    k_sy_resid_restrict<T, CORR><<<(unsigned)nblk(lev[l + 1].nc), kNT, 0, st>>>(
        lev[l], lev[l + 1], l == 0 ? part0 : nullptr);
    SLAUNCH(ctx);
    k_sy_fas_rhs<T, CORR><<<(unsigned)nblk(lev[l + 1].nc), kNT, 0, st>>>(lev[l + 1]);
    SLAUNCH(ctx);
    vcycle(l + 1);
    k_sy_prolong<T><<<(unsigned)nblk(lev[l + 1].nc), kNT, 0, st>>>(lev[l], lev[l + 1]);
    SLAUNCH(ctx);
    smooth(l, post);
  }
};

}  // namespace

extern "C" int fr_symmetron_solve(frmg_ctx *ctx, const double *density, const int dims[3],
                                  double box, double a, double a_ssb, double lambda0, double tol,
                                  double *chi_inout, const fr_opts *opts, fr_stats *stats,
                                  void *stream) {
  const auto t_start = std::chrono::steady_clock::now();
  try {
    if (!ctx || !density || !dims || !chi_inout) throw SError{FR_EINVAL, "NULL argument"};
    for (int d = 0; d < 3; d++)
      if (dims[d] < 2 || (dims[d] & 1)) throw SError{FR_EINVAL, "dims must be even and >= 2"};
    if (!(box > 0) || !(a > 0) || !(a_ssb > 0) || !(lambda0 > 0) || !(tol >= 0))
      throw SError{FR_EINVAL, "box, a, a_ssb and lambda0 must be > 0, tol >= 0"};
    fr_opts o;
    fr_opts_default(&o);
    if (opts) o = *opts;
    if (o.pre < 0 || o.post < 0 || o.pre + o.post < 1 || !(o.newton_step_cap > 0) ||
        !(o.relax > 0 && o.relax < 2) || o.max_vcycles < 1 || o.max_outer < 1 ||
        (o.prec != FR_FP64 && o.prec != FR_MIXED))
      throw SError{FR_EINVAL, "invalid options"};
    SCK(cudaSetDevice(frmg_device(ctx)));
    cudaStream_t st = (cudaStream_t)stream;
    const long long nc = (long long)dims[0] * dims[1] * dims[2];
    if (nblk(nc) >= (1ll << 31)) throw SError{FR_EINVAL, "grid too large"};
    SArena A(ctx);
    // host arrays are staged through device buffers
    const bool rho_dev = on_device(density), chi_dev = on_device(chi_inout);
    const double *rho = density;
    if (!rho_dev) {
      double *r = A.get<double>(nc);
      SCK(cudaMemcpyAsync(r, density, nc * sizeof(double), cudaMemcpyHostToDevice, st));
      rho = r;
    }
    double *chi = chi_inout;
    if (!chi_dev) chi = A.get<double>(nc);
    const double s = std::pow(a_ssb / a, 3.0);
    if (o.initial_guess) {
      if (!chi_dev)
        SCK(cudaMemcpyAsync(chi, chi_inout, nc * sizeof(double), cudaMemcpyHostToDevice, st));
    } else {
      // the homogeneous solution on the positive branch (1 before symmetry
      // breaking, from where the field relaxes to its symmetric value 0)
      const double chib = s < 1.0 ? std::sqrt(1.0 - s) : 1.0;
      k_sy_fill<<<(unsigned)nblk(nc), kNT, 0, st>>>(chi, chib, nc);
      SLAUNCH(ctx);
    }
    {
      int *bad = A.get<int>(1);
      SCK(cudaMemsetAsync(bad, 0, sizeof(int), st));
      k_sy_check_rho<<<(unsigned)nblk(nc), kNT, 0, st>>>(rho, nc, bad);
      SLAUNCH(ctx);
      int hb = 0;
      SCK(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
      SCK(cudaStreamSynchronize(st));
      if (hb) throw SError{FR_EINVAL, "density must be finite and >= 0"};
    }
    // levels: sizes and coefficients (A quarters per level)
    const int nl = sy_levels(dims);
    std::vector<std::array<int, 3>> ns(nl);
    std::vector<double> Al(nl);
    for (int l = 0; l < nl; l++) {
      for (int d = 0; d < 3; d++) ns[l][d] = dims[d] >> l;
      const double hl = box * std::ldexp(1.0, l) / dims[0];  // cell size, Mpc/h
      Al[l] = 2.0 * lambda0 * lambda0 / (a * a * hl * hl);
    }
    auto ncell = [&](int l) { return (long long)ns[l][0] * ns[l][1] * ns[l][2]; };
    double *part = A.get<double>(2 * nblk(nc));
    double *red = A.get<double>(2);
    const long long nch_max = (nblk(nc) + kSyRedCH - 1) / kSyRedCH;
    double *red_tmp = A.get<double>(2 * nch_max);
    double *pin = frmg_pinned(ctx, 2);
    if (!pin) throw SError{FR_ENOMEM, "pinned host allocation failed"};
    // sum of squares and max over nb per-block partials (two fixed-order
    // stages for long lists), rms over n cells
    auto norms = [&](double *pp, long long nb, long long n, double &rms, double &mx) {
      if (nb > 2 * kSyRedCH) {
        const long long nch = (nb + kSyRedCH - 1) / kSyRedCH;
        k_sy_reduce_chunks<<<(unsigned)nch, kNT, 0, st>>>(pp, nb, red_tmp);
        SLAUNCH(ctx);
        pp = red_tmp;
        nb = nch;
      }
      k_sy_reduce<<<1, kNT, 0, st>>>(pp, nb, red);
      SLAUNCH(ctx);
      SCK(cudaMemcpyAsync(pin, red, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      SCK(cudaStreamSynchronize(st));
      rms = std::sqrt(pin[0] / (double)n);
      mx = pin[1];
    };
    fr_stats sv;
    memset(&sv, 0, sizeof(sv));
    sv.tau_rms = std::nan("");
    auto push = [&](double v) {
      if (sv.nhist < FR_HIST) sv.hist[sv.nhist++] = v;
    };
    auto bad_v = [](double v) { return !(v == v) || std::isinf(v); };
    int status = FR_ENOCONV;
    SLevel<double> fine64;
    memset(&fine64, 0, sizeof(fine64));
    fine64.u = chi;
    fine64.rho = rho;
    fine64.n0 = dims[0];
    fine64.n1 = dims[1];
    fine64.n2 = dims[2];
    fine64.nc = nc;
    fine64.A = Al[0];
    fine64.s = s;
    fine64.cap = o.newton_step_cap;
    fine64.relax = o.relax;
    fine64.fd0 = frmg::make_fastdiv((unsigned)dims[0]);
    fine64.fd1 = frmg::make_fastdiv((unsigned)dims[1]);
    double *d64 = nullptr;
    auto defect = [&](double &rms, double &mx) {
      k_sy_defect64<<<(unsigned)nblk(nc), kNT, 0, st>>>(fine64, d64, part);
      SLAUNCH(ctx);
      norms(part, nblk(nc), nc, rms, mx);
    };

    if (o.prec == FR_FP64) {
      SHier<double, false> H;
      H.ctx = ctx;
      H.st = st;
      H.pre = o.pre;
      H.post = o.post;
      H.part0 = nullptr;
      H.crs_abs = 0.1 * tol;
      H.lev.push_back(fine64);
      for (int l = 1; l < nl; l++) {
        SLevel<double> L = fine64;
        L.n0 = ns[l][0];
        L.n1 = ns[l][1];
        L.n2 = ns[l][2];
        L.fd0 = frmg::make_fastdiv((unsigned)L.n0);
        L.fd1 = frmg::make_fastdiv((unsigned)L.n1);
        L.nc = ncell(l);
        L.A = Al[l];
        L.u = A.get<double>(L.nc);
        L.uR = A.get<double>(L.nc);
        L.f = A.get<double>(L.nc);
        double *r = A.get<double>(L.nc);
        k_sy_restrict<double, double><<<(unsigned)nblk(L.nc), kNT, 0, st>>>(
            H.lev[l - 1].rho, r, L.n0, L.n1, L.n2);
        SLAUNCH(ctx);
        L.rho = r;
        H.lev.push_back(L);
      }
      double rms, mx;
      defect(rms, mx);
      sv.res0_rms = rms;
      push(rms);
      if (bad_v(rms)) throw SError{FR_EDIVERGED, "non-finite residual"};
      double prev = rms;
      int grow = 0;
      while (rms > tol && sv.vcycles < o.max_vcycles) {
        H.vcycle(0);
        sv.vcycles++;
        defect(rms, mx);
        push(rms);
        if (bad_v(rms)) throw SError{FR_EDIVERGED, "non-finite residual"};
        grow = rms > prev ? grow + 1 : 0;
        if (grow >= 5) throw SError{FR_EDIVERGED, "residual grew for 5 cycles"};
        prev = rms;
      }
      sv.res_rms = rms;
      sv.res_max = mx;
      status = rms <= tol ? FR_OK : FR_ENOCONV;
    } else {
      SHier<float, true> H;
      H.ctx = ctx;
      H.st = st;
      H.pre = o.pre;
      H.post = o.post;
      H.crs_abs = 0.0;
      std::vector<float *> gl(nl);
      for (int l = 0; l < nl; l++) {
        SLevel<float> L;
        memset(&L, 0, sizeof(L));
        L.n0 = ns[l][0];
        L.n1 = ns[l][1];
        L.n2 = ns[l][2];
        L.fd0 = frmg::make_fastdiv((unsigned)L.n0);
        L.fd1 = frmg::make_fastdiv((unsigned)L.n1);
        L.nc = ncell(l);
        L.A = (float)Al[l];
        L.s = (float)s;
        L.cap = (float)o.newton_step_cap;
        L.relax = (float)o.relax;
        L.u = A.get<float>(L.nc);
        L.f = A.get<float>(L.nc);
        if (l > 0) L.uR = A.get<float>(L.nc);
        // the register-column smoother on levels of at least 16 cells a side
        // with enough tiles to fill the GPU (else one colour per launch)
        if (o.tiling >= 0 && L.n0 >= 16 && L.n1 >= 16 && L.n2 >= 16) {
          const long long tiles = (long long)((L.n0 + kSyTX - 1) / kSyTX) *
                                  ((L.n1 + kSyTY - 1) / kSyTY);
          const long long slots = 3ll * sm_count_sy();
          if (o.tiling == 1 || tiles * ((L.n2 + 31) / 32) >= slots) {
            double best = 1e300;
            for (int c = 1; c <= L.n2; c++) {
              const int z = (L.n2 + c - 1) / c;
              const long long nbk = tiles * ((L.n2 + z - 1) / z);
              const double cost = std::ceil((double)nbk / slots) * (z + 4);
              if (cost < best - 1e-9) {
                best = cost;
                L.zc = z;
              }
            }
            L.u2 = A.get<float>(L.nc);
          }
        }
        float *r = A.get<float>(L.nc);
        if (l == 0) {
          k_sy_convert<double, float><<<(unsigned)nblk(L.nc), kNT, 0, st>>>(rho, r, L.nc);
        } else {
          k_sy_restrict<float, float><<<(unsigned)nblk(L.nc), kNT, 0, st>>>(
              H.lev[l - 1].rho, r, L.n0, L.n1, L.n2);
        }
        SLAUNCH(ctx);
        L.rho = r;
        gl[l] = A.get<float>(L.nc);
        L.g = gl[l];
        H.lev.push_back(L);
      }
      const long long nb1 = nl > 1 ? nblk(ncell(1)) : 0;
      double *part_in = nl > 1 ? A.get<double>(2 * nb1) : nullptr;
      H.part0 = part_in;
      // chi and rho as double-float pairs for the outer loop
      float2 *chi2 = A.get<float2>(nc), *rho2 = A.get<float2>(nc);
      k_sy_split<<<(unsigned)nblk(nc), kNT, 0, st>>>(chi, chi2, nc);
      SLAUNCH(ctx);
      k_sy_split<<<(unsigned)nblk(nc), kNT, 0, st>>>(rho, rho2, nc);
      SLAUNCH(ctx);
      const float Ah = (float)Al[0], Alo = (float)(Al[0] - (double)Ah);
      const float sh = (float)s, slo = (float)(s - (double)sh);
      // defect of chi in double-float, with the set-up of the FP32 correction
      // problem of the next outer step (g = hi(chi), f = -hi(d), delta = 0)
      auto defect_df = [&](double &rms_, double &mx_) {
        k_sy_defect_df<<<(unsigned)nblk(nc / 2), kNT, 0, st>>>(H.lev[0], chi2, rho2, Ah, Alo,
                                                               sh, slo, gl[0], H.lev[0].f,
                                                               H.lev[0].u, part);
        SLAUNCH(ctx);
        norms(part, nblk(nc / 2), nc, rms_, mx_);
      };
      double rms, mx;
      defect_df(rms, mx);
      sv.res0_rms = rms;
      push(rms);
      std::string diverged;
      if (bad_v(rms)) diverged = "non-finite residual";
      double prev = rms;
      int grow = 0;
      while (diverged.empty() && rms > tol && sv.outer < o.max_outer &&
             sv.vcycles < o.max_vcycles * o.max_outer) {
        sv.outer++;
        // correction problem of this outer step: N(delta) = -d on g = fp32(chi)
        // (fine level set up by the defect pass)
        for (int l = 1; l < nl; l++) {
          k_sy_restrict<float, float><<<(unsigned)nblk(ncell(l)), kNT, 0, st>>>(
              gl[l - 1], gl[l], ns[l][0], ns[l][1], ns[l][2]);
          SLAUNCH(ctx);
        }
        // inner V-cycles until the fine correction residual (after
        // pre-smoothing, times the last contraction) is predicted below
        // max(0.1 tol, 1e-6 rms(d)), or the contraction stalls near the FP32
        // floor, or max_vcycles cycles
        const double target = std::max(0.1 * tol, 1e-6 * rms);
        double rp = HUGE_VAL, q = 0.3;
        for (int c = 0; c < o.max_vcycles; c++) {
          H.vcycle(0);
          sv.vcycles++;
          if (nl == 1) break;
          double r, m;
          norms(part_in, nb1, nc, r, m);
          if (bad_v(r)) break;  // the defect after the update reports it
          if (c > 0) q = r / rp;
          rp = r;
          if (r * q <= target || q > 0.8) break;
        }
        k_sy_update_df<<<(unsigned)nblk(nc), kNT, 0, st>>>(chi2, H.lev[0].u, nc);
        SLAUNCH(ctx);
        defect_df(rms, mx);
        push(-rms);
        if (bad_v(rms)) diverged = "non-finite residual";
        grow = rms > prev ? grow + 1 : 0;
        if (grow >= 3) diverged = "defect grew for 3 outer steps";
        prev = rms;
      }
      sv.res_rms = rms;
      sv.res_max = mx;
      status = !diverged.empty() ? FR_EDIVERGED : (rms <= tol ? FR_OK : FR_ENOCONV);
      if (!diverged.empty()) frmg_set_error(diverged);
      k_sy_join<<<(unsigned)nblk(nc), kNT, 0, st>>>(chi2, chi, nc);
      SLAUNCH(ctx);
    }
    if (!chi_dev)
      SCK(cudaMemcpyAsync(chi_inout, chi, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    sv.seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = sv;
    if (status == FR_ENOCONV) frmg_set_error("tol not reached");
    return status;
  } catch (SError &e) {
    frmg_set_error(e.msg);
    return e.status;
  } catch (std::exception &e) {
    frmg_set_error(e.what());
    return FR_ENOMEM;
  }
}
