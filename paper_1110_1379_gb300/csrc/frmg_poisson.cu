// frmg_poisson.cu -- the modified Poisson equation for the potential Phi.
//
// Sec. III.B gives the equation in code units and Eq. (discrete_poisson) its
// 7-point discretisation,
//   (1/h^2)[sum of the six neighbours - 6 phi_i] = s_i,
//   s_i = 2 Om a (rho_i - 1) - (1/6) Om a^4 [(n a^2 xi)^(1/(n+1)) e^{-u~_i/(n+1)}
//                                            - 3 (a^-3 + 4 OL/Om)],
// which for n = 1, in the f(R) solver's variable u = u~ - ubar (ubar: the
// homogeneous solution, where the bracket vanishes), reads
//   s_i = 2 gamma (rho_i - 1) - (beta/2) (e^{-u_i/2} - 1),
//   gamma = Om a,  beta = Om a^4 (a^-3 + 4 OL/Om).
// On a refinement patch a missing neighbour is the ghost 2 phi_b - phi_i
// (Eq. phi_b with mask ratio -1), which is Eq. (bc_modified_poisson).  The
// operator is linear, so the multigrid is the correction scheme of Sec. V.A.2:
// on coarser levels L^H e^H = R(s - L phi)^h with e = 0 on patch boundaries
// (Eq. bc_modified_poisson_coarse: only the left-hand side is modified), and
// e^h += P e^H with the trilinear 27/9/3/1 weights of Sec. V.A.3 (coarse cells
// outside a patch contribute 0).
//
// Precision follows the f(R) solve: phi, the source, the fine defect and its
// norm are double-float pairs (hi + lo, ~48-bit significands) on the FP32
// pipes, and the correction equation L e = -d is solved by FP32 V-cycles;
// phi += e.  On a periodic grid the equation has a solution only for a source
// of zero mean, so the source's mean is removed (and reported) and phi is
// returned with zero mean.
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

struct PError {
  int status;
  std::string msg;
};

#define PCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw PError{FR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};       \
  } while (0)

#define PLAUNCH(ctx)                                                                    \
  do {                                                                                  \
    frmg_launch_counter(ctx)++;                                                         \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess)                                                              \
      throw PError{FR_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)};  \
  } while (0)

constexpr int kNT = 256;

long long nblk(long long n) { return (n + kNT - 1) / kNT; }

// ------------------------------------------------------------------ device
struct PLevel {
  float *e;        // correction (current buffer)
  float *e_alt;    // second buffer of the tiled smoother (null: not tiled)
  float *f;        // right-hand side of the correction equation
  int n0, n1, n2;
  long long ncell;
  FastDiv fd0, fd1;
  float h2;        // h^2
  float relax;     // relaxation factor of the smoother (1: Gauss-Seidel)
  int patch;       // 1: Dirichlet (ghost = -e on the boundary), 0: periodic
};

__device__ __forceinline__ void decomp(const PLevel &L, unsigned t, int &i, int &j, int &k) {
  const unsigned q = fdiv(t, L.fd0), q2 = fdiv(q, L.fd1);
  i = (int)(t - q * (unsigned)L.n0);
  j = (int)(q - q2 * (unsigned)L.n1);
  k = (int)q2;
}

// sum of the six neighbours of (i,j,k) and the number of missing ones (patch)
__device__ __forceinline__ float nbsum(const PLevel &L, const float *e, int i, int j, int k,
                                       long long c, int &nmiss) {
  const long long sy = L.n0, sz = (long long)L.n0 * L.n1;
  float s = 0.0f;
  nmiss = 0;
  if (L.patch) {
    if (i > 0) s += e[c - 1]; else nmiss++;
    if (i < L.n0 - 1) s += e[c + 1]; else nmiss++;
    if (j > 0) s += e[c - sy]; else nmiss++;
    if (j < L.n1 - 1) s += e[c + sy]; else nmiss++;
    if (k > 0) s += e[c - sz]; else nmiss++;
    if (k < L.n2 - 1) s += e[c + sz]; else nmiss++;
  } else {
    s += e[i > 0 ? c - 1 : c + (L.n0 - 1)];
    s += e[i < L.n0 - 1 ? c + 1 : c - (L.n0 - 1)];
    s += e[j > 0 ? c - sy : c + (L.n1 - 1) * sy];
    s += e[j < L.n1 - 1 ? c + sy : c - (L.n1 - 1) * sy];
    s += e[k > 0 ? c - sz : c + (L.n2 - 1) * sz];
    s += e[k < L.n2 - 1 ? c + sz : c - (L.n2 - 1) * sz];
  }
  return s;
}

// Gauss-Seidel value of a cell, (sum of its neighbours in the grid - h^2 f) /
// (6 + missing neighbours), with the diagonal's reciprocal as a constant (at
// most three neighbours are missing: every dimension is at least 2); every
// smoother uses this one expression.
__device__ __forceinline__ float gs_value(float sum, float h2f, int nm) {
  const float inv = nm == 0   ? 1.0f / 6.0f
                    : nm == 1 ? 1.0f / 7.0f
                    : nm == 2 ? 1.0f / 8.0f
                              : 1.0f / 9.0f;
  return (sum - h2f) * inv;
}

// Red-black Gauss-Seidel on L e = f (one colour per launch): with the ghosts
// -e_i on patch faces, e_i = (sum of the neighbours in the grid - h^2 f_i) / (6 + missing),
// over-relaxed as e_i += w (that value - e_i) when relax = w != 1.
__global__ void __launch_bounds__(kNT) k_lsmooth(PLevel L, int colour) {
  const long long half = L.ncell / 2;
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= half) return;
  // cell 2t or 2t+1 along x, whichever has the colour (n0 even)
  int i, j, k;
  decomp(L, (unsigned)(2 * t), i, j, k);
  i += (i + j + k + colour) & 1;
  const long long c = ((long long)k * L.n1 + j) * L.n0 + i;
  int nm;
  const float s = nbsum(L, L.e, i, j, k, c, nm);
  const float gs = gs_value(s, L.h2 * L.f[c], nm);
  L.e[c] = fmaf(L.relax, gs - L.e[c], L.e[c]);
}

// Tiled red-black Gauss-Seidel on L e = f, one full sweep per pass (the
// schedule of the f(R) solver's tiled smoother): a block owns a 64 x 16 tile
// and a chunk of zc planes and marches along z with a ring of four planes of e
// and f in shared memory (the tile plus a halo of two cells).  At the step for
// plane p it updates the red cells of plane p-1 on the tile grown by one cell,
// then the black cells of plane p-2 on the tile, and writes plane p-2 to the
// other buffer (the halos are read from the unmodified input, so the pass
// equals one sweep of k_lsmooth).  Each plane is stored colour-split: per
// x-pair q = (ly, px) of the tile, array c holds the pair's cell of colour c
// (the even-x cell has colour (ly + z) & 1), so the six neighbours of a cell
// are the opposite colour's entries q, q -+ 1, q -+ PX of its own and the
// adjacent planes, and a warp's accesses (lane = x-pair) are contiguous.
// Warps update whole rows of the tile; the next plane is prefetched into
// registers during the updates.
template <bool PATCH>
__global__ void __launch_bounds__(256, 4) k_lsmooth_tiled(PLevel L, int zc) {
  constexpr int TX = 64, TY = 16, H = 2, LX = TX + 2 * H, LY = TY + 2 * H, PX = LX / 2;
  constexpr int PP = PX * LY, NW = TY / 2, NT = 32 * NW, NLD = (PP + NT - 1) / NT, NS = 4;
  constexpr int NE = TY + 2, PL = 2 * PP;
  __shared__ __align__(16) float se[NS * PL];  // [slot][colour][pair]
  __shared__ __align__(16) float sf[NS * PL];
  const int n0 = L.n0, n1 = L.n1, n2 = L.n2;
  const int ntx = (n0 + TX - 1) / TX, nty = (n1 + TY - 1) / TY;
  int b = blockIdx.x;
  const int X0 = (b % ntx) * TX;
  b /= ntx;
  const int Y0 = (b % nty) * TY;
  b /= nty;
  const int Z0 = b * zc, Z1 = min(Z0 + zc, n2);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long plane = (long long)n0 * n1;
  const float *__restrict__ ein = L.e;
  float *__restrict__ eout = L.e_alt;
  const float *__restrict__ fin = L.f;
  const float h2 = L.h2, relax = L.relax;
  auto wrapm = [](int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
  };
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
      bool ok = true;
      int gxw = gx, gyw = gy;
      if (PATCH) {
        ok = gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
      } else {
        gxw = wrapm(gx, n0);
        gyw = wrapm(gy, n1);
      }
      const bool wr = ok && ly >= H && ly < H + TY && px >= 1 && px < PX - 1 && gx < n0 &&
                      gy < n1;
      roff[k] = ok ? gyw * n0 + gxw : 0;
      ldf[k] = (ok ? 1u : 0u) | (wr ? 2u : 0u) | ((unsigned)(ly & 1) << 2);
    }
  }
  float2 pe[NLD], pf[NLD];
#pragma unroll
  for (int k = 0; k < NLD; k++) {
    pe[k] = make_float2(0.f, 0.f);
    pf[k] = pe[k];
  }
  auto fetch = [&](long long zoff) {
#pragma unroll
    for (int k = 0; k < NLD; k++) {
      if (!(ldf[k] & 1u)) continue;
      pe[k] = *reinterpret_cast<const float2 *>(ein + zoff + roff[k]);
      pf[k] = *reinterpret_cast<const float2 *>(fin + zoff + roff[k]);
    }
  };
  // plane of parity pb into slot offset so
  auto commit = [&](int pb, int so) {
#pragma unroll
    for (int k = 0; k < NLD; k++) {
      const int q = threadIdx.x + k * NT;
      if (q >= PP) continue;
      const int c0 = (int)((ldf[k] >> 2) & 1u) ^ pb;
      se[so + c0 * PP + q] = pe[k].x;
      se[so + (c0 ^ 1) * PP + q] = pe[k].y;
      sf[so + c0 * PP + q] = pf[k].x;
      sf[so + (c0 ^ 1) * PP + q] = pf[k].y;
    }
  };
  // Gauss-Seidel update of the colour-Q cell of pair (ly, px) of plane m; s is
  // its x position in the pair; oc, om, op the slot offsets of planes m, m-1, m+1
  auto update = [&](int Q, int ly, int px, int s, int m, int oc, int om, int op) {
    const int gx = X0 - H + 2 * px + s, gy = Y0 - H + ly;
    if (PATCH && (gx < 0 || gx >= n0 || gy < 0 || gy >= n1)) return;
    const int e = ly * PX + px;
    const int cq = oc + Q * PP + e, V = oc + (Q ^ 1) * PP + e;
    const int o = (Q ^ 1) * PP + e;
    float sum = 0.0f;
    int nm = 0;
    if (!PATCH || gx > 0) sum += se[s ? V : V - 1]; else nm++;
    if (!PATCH || gx < n0 - 1) sum += se[s ? V + 1 : V]; else nm++;
    if (!PATCH || gy > 0) sum += se[V - PX]; else nm++;
    if (!PATCH || gy < n1 - 1) sum += se[V + PX]; else nm++;
    if (!PATCH || m > 0) sum += se[om + o]; else nm++;
    if (!PATCH || m < n2 - 1) sum += se[op + o]; else nm++;
    const float gs = gs_value(sum, h2 * sf[cq], nm);
    se[cq] = fmaf(relax, gs - se[cq], se[cq]);
  };
  const int P0 = Z0 - H, PE = Z1 + H;
  auto inr = [&](int pz) { return !PATCH || (pz >= 0 && pz < n2); };
  int pw = PATCH ? P0 : wrapm(P0, n2);
  if (inr(P0)) fetch((long long)pw * plane);
  commit(P0 & 1, 0);
  __syncthreads();
  int cur = 0;
  for (int p = P0; p < PE; p++) {
    const bool more = p + 1 < PE;
    pw = PATCH ? p + 1 : (pw + 1 == n2 ? 0 : pw + 1);
    if (more && inr(p + 1)) fetch((long long)pw * plane);
    const int o0 = cur * PL, o1 = ((cur + 3) & 3) * PL, o2 = ((cur + 2) & 3) * PL,
              o3 = ((cur + 1) & 3) * PL;  // planes p, p-1, p-2, p-3
    {
      const int m = p - 1;  // red cells, tile grown by one
      if (m >= Z0 - 1 && m < Z1 + 1 && inr(m)) {
        const int s = (w + p) & 1;  // rows 1 + w + j NW: (ly + m) & 1
#pragma unroll
        for (int j = 0; j < 3; j++) {
          if (j == 2 && w >= 2) break;
          update(0, 1 + w + j * NW, 1 + lane, s, m, o1, o2, o0);
        }
        if (w == 2 || w == 3) {
          const int idx = (w - 2) * 32 + lane;
          if (idx < NE) {
            const int ly = 1 + idx, se_ = (ly + m) & 1;
            update(0, ly, se_ ? 0 : PX - 1, se_, m, o1, o2, o0);
          }
        }
      }
    }
    __syncthreads();
    {
      const int m = p - 2;  // black cells, tile
      if (m >= Z0 && m < Z1 && inr(m)) {
        const int s = (w + m + 1) & 1;  // rows 2 + w + j NW: (ly + m + 1) & 1
#pragma unroll
        for (int j = 0; j < 2; j++) update(1, 2 + w + j * NW, 1 + lane, s, m, o2, o3, o1);
      }
    }
    __syncthreads();
    {
      const int wz = p - 2;
      if (wz >= Z0 && wz < Z1) {
        const long long woff = (long long)wz * plane;
#pragma unroll
        for (int k = 0; k < NLD; k++)
          if (ldf[k] & 2u) {
            const int q = threadIdx.x + k * NT;
            const int c0 = (int)((ldf[k] >> 2) & 1u) ^ (wz & 1);
            *reinterpret_cast<float2 *>(eout + woff + roff[k]) =
                make_float2(se[o2 + c0 * PP + q], se[o2 + (c0 ^ 1) * PP + q]);
          }
      }
    }
    if (more) commit((p + 1) & 1, o3);
    __syncthreads();
    cur = (cur + 1) & 3;
  }
}

// Residual d = f - L e of the 8 children of each coarse cell, averaged into
// the coarse right-hand side; coarse e = 0.  Optional per-block (sum d^2, max |d|).
__global__ void __launch_bounds__(kNT) k_lresid_restrict(PLevel F, PLevel C, double *partial) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  float ss = 0.0f, mx = 0.0f;
  if (t < C.ncell) {
    int I, J, K;
    decomp(C, (unsigned)t, I, J, K);
    float sd = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
      const long long c = ((long long)k * F.n1 + j) * F.n0 + i;
      int nm;
      const float s = nbsum(F, F.e, i, j, k, c, nm);
      const float d = F.f[c] - (s - (6.0f + (float)nm) * F.e[c]) / F.h2;
      sd += d;
      ss = fmaf(d, d, ss);
      mx = fmaxf(mx, fabsf(d));
    }
    C.f[t] = 0.125f * sd;
    C.e[t] = 0.0f;
  }
  if (partial) {
    for (int o = 16; o > 0; o >>= 1) {
      ss += __shfl_down_sync(0xffffffffu, ss, o);
      mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    __shared__ float a[kNT / 32], b[kNT / 32];
    if ((threadIdx.x & 31) == 0) {
      a[threadIdx.x >> 5] = ss;
      b[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s2 = 0.0;
      float m2 = 0.0f;
      for (int w = 0; w < kNT / 32; w++) {
        s2 += (double)a[w];
        m2 = fmaxf(m2, b[w]);
      }
      partial[2 * blockIdx.x] = s2;
      partial[2 * blockIdx.x + 1] = (double)m2;
    }
  }
}

// Tiled residual + restriction (the arithmetic of k_lresid_restrict): a block
// owns a 64 x 16 fine tile (32 x 8 coarse cells, one per thread) and a chunk
// of kc coarse planes, and keeps a ring of four fine planes of e (tile plus a
// one-cell halo) in shared memory: coarse plane K needs fine planes 2K-1 ..
// 2K+2, and each step loads the next two (prefetched into registers while the
// residuals of the current pair of fine planes are formed).  f is read by
// each thread for its own 2 x 2 x 2 children.  Optional per-block norm
// partials (sum d^2, max |d|).
constexpr int kLrTX = 64, kLrTY = 16;
template <bool PATCH>
__global__ void __launch_bounds__(256) k_lresid_restrict_tiled(PLevel F, PLevel C, int kc,
                                                               double *partial) {
  constexpr int LX = kLrTX + 2, LY = kLrTY + 2, PC = LX * LY, NT = 256;
  constexpr int NLD = (PC + NT - 1) / NT;
  __shared__ float se[4 * PC];
  const int n0 = F.n0, n1 = F.n1, n2 = F.n2;
  const int ntx = (n0 + kLrTX - 1) / kLrTX, nty = (n1 + kLrTY - 1) / kLrTY;
  int b = blockIdx.x;
  const int X0 = (b % ntx) * kLrTX;
  b /= ntx;
  const int Y0 = (b % nty) * kLrTY;
  b /= nty;
  const int K0 = b * kc, K1 = min(K0 + kc, C.n2);
  const long long plane = (long long)n0 * n1;
  auto wrapm = [](int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
  };
  int roff[NLD];
  bool lok[NLD];
#pragma unroll
  for (int k = 0; k < NLD; k++) {
    const int q = threadIdx.x + k * NT;
    roff[k] = 0;
    lok[k] = false;
    if (q < PC) {
      const int gx = X0 - 1 + q % LX, gy = Y0 - 1 + q / LX;
      if (PATCH) {
        lok[k] = gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
        roff[k] = lok[k] ? gy * n0 + gx : 0;
      } else {
        lok[k] = true;
        roff[k] = wrapm(gy, n1) * n0 + wrapm(gx, n0);
      }
    }
  }
  float pv[2][NLD];
  // fine plane z (may lie outside a patch: never read then) into registers
  auto fetch = [&](int r, int z) {
    const bool vz = !PATCH || (z >= 0 && z < n2);
    const long long zo = (long long)(PATCH ? z : wrapm(z, n2)) * plane;
#pragma unroll
    for (int k = 0; k < NLD; k++) pv[r][k] = (vz && lok[k]) ? F.e[zo + roff[k]] : 0.0f;
  };
  auto commit = [&](int r, int slot) {
#pragma unroll
    for (int k = 0; k < NLD; k++) {
      const int q = threadIdx.x + k * NT;
      if (q < PC) se[slot * PC + q] = pv[r][k];
    }
  };
  // this thread's coarse cell of the tile
  const int cx = threadIdx.x & 31, cy = threadIdx.x >> 5;
  const int I = X0 / 2 + cx, J = Y0 / 2 + cy;
  const bool own = 2 * I < n0 && 2 * J < n1;
  float ss = 0.0f, mx = 0.0f;
  // planes 2K0-1 .. 2K0+2 into slots 0..3 (slot of fine plane z: (z - 2K0 + 1) & 3)
  fetch(0, 2 * K0 - 1);
  fetch(1, 2 * K0);
  commit(0, 0);
  commit(1, 1);
  fetch(0, 2 * K0 + 1);
  fetch(1, 2 * K0 + 2);
  commit(0, 2);
  commit(1, 3);
  __syncthreads();
  for (int K = K0; K < K1; K++) {
    const bool more = K + 1 < K1;
    if (more) {
      fetch(0, 2 * K + 3);
      fetch(1, 2 * K + 4);
    }
    if (own) {
      float sd = 0.0f;
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int dx = q & 1, dy = (q >> 1) & 1, dz = q >> 2;
        const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
        const int lx = 1 + 2 * cx + dx, ly = 1 + 2 * cy + dy;
        const int sm = ((k - 1 - 2 * K0 + 1) & 3) * PC, sc = ((k - 2 * K0 + 1) & 3) * PC,
                  sp = ((k + 1 - 2 * K0 + 1) & 3) * PC;
        const int o = ly * LX + lx;
        float s = 0.0f;
        int nm = 0;
        if (PATCH) {
          if (i > 0) s += se[sc + o - 1]; else nm++;
          if (i < n0 - 1) s += se[sc + o + 1]; else nm++;
          if (j > 0) s += se[sc + o - LX]; else nm++;
          if (j < n1 - 1) s += se[sc + o + LX]; else nm++;
          if (k > 0) s += se[sm + o]; else nm++;
          if (k < n2 - 1) s += se[sp + o]; else nm++;
        } else {
          s += se[sc + o - 1];
          s += se[sc + o + 1];
          s += se[sc + o - LX];
          s += se[sc + o + LX];
          s += se[sm + o];
          s += se[sp + o];
        }
        const long long c = (long long)k * plane + (long long)j * n0 + i;
        const float d = F.f[c] - (s - (6.0f + (float)nm) * se[sc + o]) / F.h2;
        sd += d;
        ss = fmaf(d, d, ss);
        mx = fmaxf(mx, fabsf(d));
      }
      const long long t = ((long long)K * C.n1 + J) * C.n0 + I;
      C.f[t] = 0.125f * sd;
      C.e[t] = 0.0f;
    }
    __syncthreads();
    if (more) {
      commit(0, (2 * K + 3 - 2 * K0 + 1) & 3);
      commit(1, (2 * K + 4 - 2 * K0 + 1) & 3);
    }
    __syncthreads();
  }
  if (partial) {
    for (int o = 16; o > 0; o >>= 1) {
      ss += __shfl_down_sync(0xffffffffu, ss, o);
      mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    __shared__ float a[NT / 32], bm[NT / 32];
    if ((threadIdx.x & 31) == 0) {
      a[threadIdx.x >> 5] = ss;
      bm[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s2 = 0.0;
      float m2 = 0.0f;
      for (int w = 0; w < NT / 32; w++) {
        s2 += (double)a[w];
        m2 = fmaxf(m2, bm[w]);
      }
      partial[2 * blockIdx.x] = s2;
      partial[2 * blockIdx.x + 1] = (double)m2;
    }
  }
}

// e^h += P e^H: trilinear, per axis 3/4 on the containing coarse cell and 1/4
// on the neighbour on the child's side (products: 27/9/3/1 over 64).
__global__ void __launch_bounds__(kNT) k_lprolong(PLevel F, PLevel C) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= F.ncell) return;
  int i, j, k;
  decomp(F, (unsigned)t, i, j, k);
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const int di = (i & 1) ? 1 : -1, dj = (j & 1) ? 1 : -1, dk = (k & 1) ? 1 : -1;
  float acc = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    int ii = I + ((q & 1) ? di : 0), jj = J + (((q >> 1) & 1) ? dj : 0),
        kk = K + ((q >> 2) ? dk : 0);
    const float w = ((q & 1) ? 0.25f : 0.75f) * (((q >> 1) & 1) ? 0.25f : 0.75f) *
                    ((q >> 2) ? 0.25f : 0.75f);
    bool in = true;
    if (C.patch) {
      in = ii >= 0 && ii < C.n0 && jj >= 0 && jj < C.n1 && kk >= 0 && kk < C.n2;
    } else {
      ii = ii < 0 ? ii + C.n0 : (ii >= C.n0 ? ii - C.n0 : ii);
      jj = jj < 0 ? jj + C.n1 : (jj >= C.n1 ? jj - C.n1 : jj);
      kk = kk < 0 ? kk + C.n2 : (kk >= C.n2 ? kk - C.n2 : kk);
    }
    if (in) acc = fmaf(w, C.e[((long long)kk * C.n1 + jj) * C.n0 + ii], acc);
  }
  F.e[t] += acc;
}

// Tiled e^h += P e^H (the interpolation of k_lprolong, evaluated in the order
// z, y, x): a block owns a 64 x 16 fine tile (32 x 8 coarse cells) and a chunk
// of kc coarse planes; the coarse tile plus a one-cell halo is staged in
// shared memory for planes K-1, K, K+1 (ring of three), the z-interpolated
// plane is formed once per fine plane, and each thread corrects fine x-pairs
// with 8-byte loads and stores.  Patches: coarse cells outside the grid
// contribute 0.
constexpr int kLpTX = 64, kLpTY = 16;
template <bool PATCH>
__global__ void __launch_bounds__(256) k_lprolong_tiled(PLevel F, PLevel C, int kc) {
  constexpr int CX = kLpTX / 2 + 2, CY = kLpTY / 2 + 2, CP = CX * CY;
  constexpr int NQ = (CP + 255) / 256;
  __shared__ float se[3][CP];
  __shared__ float sz[CP];
  const int n0 = F.n0, n1 = F.n1;
  const int c0 = C.n0, c1 = C.n1, c2 = C.n2;
  const float *__restrict__ eH = C.e;
  float *__restrict__ ef = F.e;
  const int ntx = (n0 + kLpTX - 1) / kLpTX, nty = (n1 + kLpTY - 1) / kLpTY;
  int b = blockIdx.x;
  const int X0 = (b % ntx) * kLpTX;
  b /= ntx;
  const int Y0 = (b % nty) * kLpTY;
  b /= nty;
  const int K0 = b * kc, K1 = min(K0 + kc, c2);
  auto wrapm = [](int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
  };
  int qoff[NQ];
  bool qok[NQ];
#pragma unroll
  for (int k = 0; k < NQ; k++) {
    const int q = threadIdx.x + k * 256;
    qoff[k] = 0;
    qok[k] = false;
    if (q < CP) {
      int I = X0 / 2 - 1 + q % CX, J = Y0 / 2 - 1 + q / CX;
      if (PATCH) {
        qok[k] = I >= 0 && I < c0 && J >= 0 && J < c1;
      } else {
        I = wrapm(I, c0);
        J = wrapm(J, c1);
        qok[k] = true;
      }
      qoff[k] = J * c0 + I;
    }
  }
  const long long cplane = (long long)c0 * c1;
  int kw = PATCH ? K0 - 1 : wrapm(K0 - 1, c2);  // wrapped index of the next plane staged
  auto stage = [&](int slot, int K) {
    const bool vz = !PATCH || (K >= 0 && K < c2);
    const long long zo = (long long)kw * cplane;
#pragma unroll
    for (int k = 0; k < NQ; k++) {
      const int q = threadIdx.x + k * 256;
      if (q >= CP) continue;
      se[slot][q] = (qok[k] && vz) ? eH[zo + qoff[k]] : 0.0f;
    }
    kw = PATCH ? kw + 1 : (kw + 1 == c2 ? 0 : kw + 1);
  };
  const int lane = threadIdx.x & 31, r0 = threadIdx.x >> 5;
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
        const float2 v = *reinterpret_cast<const float2 *>(ef + fi);
        *reinterpret_cast<float2 *>(ef + fi) =
            make_float2(v.x + (w3 * e0 + w1 * em), v.y + (w3 * e0 + w1 * ep));
      }
      __syncthreads();
    }
    const int t = sm;
    sm = sc;
    sc = sp;
    sp = t;
  }
}

// Coarsest level: one block, red-black sweeps until the rms residual falls by
// 1e-3 of its value before the first sweep (at most maxit sweeps) or stops falling.
__global__ void __launch_bounds__(kNT) k_lcoarsest(PLevel L, int maxit) {
  __shared__ float red[kNT / 32];
  __shared__ float r0s, rprev;
  auto rms = [&]() -> float {
    float ss = 0.0f;
    for (long long c = threadIdx.x; c < L.ncell; c += kNT) {
      int i, j, k;
      decomp(L, (unsigned)c, i, j, k);
      int nm;
      const float s = nbsum(L, L.e, i, j, k, c, nm);
      const float d = L.f[c] - (s - (6.0f + (float)nm) * L.e[c]) / L.h2;
      ss = fmaf(d, d, ss);
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    float tot = 0.0f;
    for (int w = 0; w < kNT / 32; w++) tot += red[w];
    __syncthreads();
    return sqrtf(tot / (float)L.ncell);
  };
  const float r0 = rms();
  if (threadIdx.x == 0) {
    r0s = r0;
    rprev = r0;
  }
  __syncthreads();
  for (int it = 0; it < maxit; it++) {
    for (int colour = 0; colour < 2; colour++) {
      for (long long t = threadIdx.x; t < L.ncell / 2; t += kNT) {
        int i, j, k;
        decomp(L, (unsigned)(2 * t), i, j, k);
        i += (i + j + k + colour) & 1;
        const long long c = ((long long)k * L.n1 + j) * L.n0 + i;
        int nm;
        const float s = nbsum(L, L.e, i, j, k, c, nm);
        L.e[c] = gs_value(s, L.h2 * L.f[c], nm);
      }
      __syncthreads();
    }
    const float r = rms();
    const bool stop = r <= 1e-3f * r0s || !(r < rprev);
    __syncthreads();
    if (threadIdx.x == 0) rprev = r;
    __syncthreads();
    if (stop) break;
  }
}

// ---- double-float fine level

struct PFine {
  float2 *phi;         // phi (hi, lo)
  float2 *s;           // source (hi, lo)
  const double *phib;  // patch faces (FP64) or null
  long long foff[6];
  int n0, n1, n2;
  long long ncell;
  FastDiv fd0, fd1;
  float ih2h, ih2l;    // 1/h^2 as a double-float pair
};

__device__ __forceinline__ df ldf(const float2 *p, long long c) {
  const float2 v = p[c];
  return {v.x, v.y};
}

// Sum of two double-float values across a warp; lane 0 holds the total.
__device__ __forceinline__ df warp_df_sum(df v) {
  for (int o = 16; o > 0; o >>= 1) {
    df w = {__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
    v = df_add(v, w);
  }
  return v;
}

// Block (sum, max) of a double-float per-thread value: partial[2 b] = sum
// (as FP64), partial[2 b + 1] = max |value| (the max is taken on the high parts).
__device__ __forceinline__ void block_df_partial(df v, float amax, double *partial) {
  __shared__ double ws[kNT / 32];
  __shared__ float wm[kNT / 32];
  v = warp_df_sum(v);
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_down_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) {
    ws[threadIdx.x >> 5] = join_bits(v.h, v.l);
    wm[threadIdx.x >> 5] = amax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    float m = 0.0f;
    for (int w = 0; w < kNT / 32; w++) {
      s += ws[w];
      m = fmaxf(m, wm[w]);
    }
    partial[2 * blockIdx.x] = s;
    partial[2 * blockIdx.x + 1] = (double)m;
  }
}

// s = 2 gamma (rho - 1) - (beta/2)(e^{-u/2} - 1) and phi = phi0, both as
// pairs; per-block partial sums of s (for its mean).
__global__ void __launch_bounds__(kNT)
    k_psource(PFine P, const double *rho, const double *u, const double *phi0, float g2h,
              float g2l, float bh, float bl, float ln2h, float ln2l, double *partial) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  df v = {0.f, 0.f};
  float am = 0.0f;
  if (t < P.ncell) {
    const df r = split_bits(rho[t]);
    const df uu = split_bits(u[t]);
    const df e = df_exp(df{-0.5f * uu.h, -0.5f * uu.l}, ln2h, ln2l);  // exact halving
    const df s = df_sub(df_mul(df_add_f(r, -1.0f), df{g2h, g2l}),
                        df_mul(df_add_f(e, -1.0f), df{bh, bl}));
    P.s[t] = make_float2(s.h, s.l);
    const df p = phi0 ? split_bits(phi0[t]) : df{0.f, 0.f};
    P.phi[t] = make_float2(p.h, p.l);
    v = s;
    am = fabsf(s.h);
  }
  block_df_partial(v, am, partial);
}

// Fine defect d = L(phi) - (s - smean) in double-float; the FP32 correction
// problem gets f = -d and e = 0.  Per-block partials of (d^2, max |d|).
__global__ void __launch_bounds__(kNT)
    k_pdefect(PFine P, float smh, float sml, float *f32, float *e32, double *partial,
              double *dout) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  float ss = 0.0f, mx = 0.0f;
  if (t < P.ncell) {
    const unsigned tu = (unsigned)t, q = fdiv(tu, P.fd0), q2 = fdiv(q, P.fd1);
    const int i = (int)(tu - q * (unsigned)P.n0), j = (int)(q - q2 * (unsigned)P.n1),
              k = (int)q2;
    const long long sy = P.n0, sz = (long long)P.n0 * P.n1;
    const df pi = ldf(P.phi, t);
    df acc = {0.f, 0.f};
    int nb = 0;  // neighbours inside
    auto reg = [&](long long cj) {
      acc = df_add(acc, ldf(P.phi, cj));
      nb++;
    };
    auto ghost = [&](int f, long long o) {
      // ghost 2 phi_b - phi_i: phi_b enters here, -phi_i with the diagonal
      const df b = split_bits(P.phib[P.foff[f] + o]);
      acc = df_add(acc, df{2.0f * b.h, 2.0f * b.l});
    };
    const bool pat = P.phib != nullptr;
    if (i > 0) reg(t - 1); else if (!pat) reg(t + (P.n0 - 1)); else ghost(0, (long long)k * P.n1 + j);
    if (i < P.n0 - 1) reg(t + 1); else if (!pat) reg(t - (P.n0 - 1)); else ghost(1, (long long)k * P.n1 + j);
    if (j > 0) reg(t - sy); else if (!pat) reg(t + (P.n1 - 1) * sy); else ghost(2, (long long)k * P.n0 + i);
    if (j < P.n1 - 1) reg(t + sy); else if (!pat) reg(t - (P.n1 - 1) * sy); else ghost(3, (long long)k * P.n0 + i);
    if (k > 0) reg(t - sz); else if (!pat) reg(t + (P.n2 - 1) * sz); else ghost(4, (long long)j * P.n0 + i);
    if (k < P.n2 - 1) reg(t + sz); else if (!pat) reg(t - (P.n2 - 1) * sz); else ghost(5, (long long)j * P.n0 + i);
    // diagonal: -(6 + missing) phi_i = -(12 - nb) phi_i
    acc = df_sub(acc, df_mul_f(pi, (float)(12 - nb)));
    df d = df_mul(acc, df{P.ih2h, P.ih2l});
    d = df_sub(d, df_sub(ldf(P.s, t), df{smh, sml}));
    const float dv = d.h + d.l;
    f32[t] = -dv;
    e32[t] = 0.0f;
    if (dout) dout[t] = join_bits(d.h, d.l);
    ss = dv * dv;
    mx = fabsf(dv);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_down_sync(0xffffffffu, ss, o);
    mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  __shared__ float a[kNT / 32], b[kNT / 32];
  if ((threadIdx.x & 31) == 0) {
    a[threadIdx.x >> 5] = ss;
    b[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    float m2 = 0.0f;
    for (int w = 0; w < kNT / 32; w++) {
      s2 += (double)a[w];
      m2 = fmaxf(m2, b[w]);
    }
    partial[2 * blockIdx.x] = s2;
    partial[2 * blockIdx.x + 1] = (double)m2;
  }
}

// phi += e (pair arithmetic)
__global__ void __launch_bounds__(kNT) k_pupdate(PFine P, const float *e) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= P.ncell) return;
  const float2 p = P.phi[t];
  df s = two_sum(p.x, e[t]);
  s.l += p.y;
  s = fast_two_sum(s.h, s.l);
  P.phi[t] = make_float2(s.h, s.l);
}

// per-block sums of phi (for its mean)
__global__ void __launch_bounds__(kNT) k_pphisum(PFine P, double *partial) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  df v = {0.f, 0.f};
  if (t < P.ncell) v = ldf(P.phi, t);
  block_df_partial(v, fabsf(v.h), partial);
}

// phi64 = phi - mean
__global__ void __launch_bounds__(kNT) k_pfinal(PFine P, float mh, float ml, double *out) {
  const long long t = (long long)blockIdx.x * kNT + threadIdx.x;
  if (t >= P.ncell) return;
  const df p = df_sub(ldf(P.phi, t), df{mh, ml});
  out[t] = join_bits(p.h, p.l);
}

// ------------------------------------------------------------------ host
void split_host(double v, float &h, float &l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct Arena {
  frmg_ctx *c;
  std::vector<void *> ptrs;
  explicit Arena(frmg_ctx *c_) : c(c_) {}
  template <typename T>
  T *get(size_t n) {
    void *p = nullptr;
    try {
      p = frmg_alloc(c, n * sizeof(T));
    } catch (...) {
      throw PError{FR_ENOMEM, "device allocation failed"};
    }
    ptrs.push_back(p);
    return (T *)p;
  }
  ~Arena() {
    for (void *p : ptrs) frmg_release(c, p);
  }
};

// Sum and max of n (sum, max) pairs of per-block partials: block b reduces
// pairs [b kRedCH, (b + 1) kRedCH) in a fixed order (FP64) into pair b of out.
constexpr int kRedCH = 4096;
__global__ void __launch_bounds__(kNT) k_psum_pairs(const double *in, long long n, double *out) {
  __shared__ double ss[kNT / 32], sm[kNT / 32];
  const long long b0 = (long long)blockIdx.x * kRedCH;
  const long long b1 = b0 + kRedCH < n ? b0 + kRedCH : n;
  double s = 0.0, m = 0.0;
  for (long long i = b0 + threadIdx.x; i < b1; i += kNT) {
    s += in[2 * i];
    m = fmax(m, in[2 * i + 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    ss[threadIdx.x >> 5] = s;
    sm[threadIdx.x >> 5] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, mm = 0.0;
    for (int w = 0; w < kNT / 32; w++) {
      t += ss[w];
      mm = fmax(mm, sm[w]);
    }
    out[2 * blockIdx.x] = t;
    out[2 * blockIdx.x + 1] = mm;
  }
}

// Device-side sum (and max) of nb partial pairs in one or two reduction
// launches; only the final pair crosses to the host.  tmp holds at least
// 2 (ceil(nb / kRedCH) + 1) doubles; nb <= kRedCH^2.
struct PartialSum {
  frmg_ctx *ctx;
  double *tmp;
  double *pinned;
  cudaStream_t st;
  void operator()(const double *dpart, long long nb, double &sum, double &mx) const {
    const long long n2 = (nb + kRedCH - 1) / kRedCH;
    k_psum_pairs<<<(unsigned)n2, kNT, 0, st>>>(dpart, nb, tmp);
    PLAUNCH(ctx);
    const double *res = tmp;
    if (n2 > 1) {
      k_psum_pairs<<<1, kNT, 0, st>>>(tmp, n2, tmp + 2 * n2);
      PLAUNCH(ctx);
      res = tmp + 2 * n2;
    }
    PCK(cudaMemcpyAsync(pinned, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    sum = pinned[0];
    mx = pinned[1];
  }
};

int level_count(const int n[3]) {
  int L = 1, m[3] = {n[0], n[1], n[2]};
  while (true) {
    bool ok = true;
    for (int d = 0; d < 3; d++) ok = ok && (m[d] % 2 == 0) && (m[d] / 2 >= 4);
    if (!ok) break;
    for (int d = 0; d < 3; d++) m[d] /= 2;
    L++;
  }
  return L;
}

struct PoissonSolver {
  frmg_ctx *ctx;
  cudaStream_t st;
  std::vector<PLevel> lev;
  int pre = 2, post = 2;

  std::vector<int> zc, nblk_t;  // tiled smoother: z-chunk and blocks per level (0: not tiled)
  std::vector<int> kc_p, nblk_p;  // tiled prolongation onto a level: coarse planes per block
                                  // and blocks (0: one thread per fine cell)
  std::vector<int> kc_r, nblk_r;  // tiled residual + restriction from a level (same layout)

  void smooth(int l, int n) {
    for (int it = 0; it < n; it++) {
      PLevel &L = lev[l];
      if (nblk_t[l] > 0) {
        if (L.patch)
          k_lsmooth_tiled<true><<<nblk_t[l], 256, 0, st>>>(L, zc[l]);
        else
          k_lsmooth_tiled<false><<<nblk_t[l], 256, 0, st>>>(L, zc[l]);
        PLAUNCH(ctx);
        std::swap(L.e, L.e_alt);
        continue;
      }
      for (int c = 0; c < 2; c++) {
        k_lsmooth<<<nblk(L.ncell / 2), kNT, 0, st>>>(L, c);
        PLAUNCH(ctx);
      }
    }
  }
  void vcycle(int l, double *partial0) {
    if (l == (int)lev.size() - 1) {
      k_lcoarsest<<<1, kNT, 0, st>>>(lev[l], 500);
      PLAUNCH(ctx);
      return;
    }
    smooth(l, pre);
    double *part = l == 0 ? partial0 : nullptr;
    if (nblk_r[l] > 0) {
      if (lev[l].patch)
        k_lresid_restrict_tiled<true><<<nblk_r[l], 256, 0, st>>>(lev[l], lev[l + 1], kc_r[l], part);
      else
        k_lresid_restrict_tiled<false><<<nblk_r[l], 256, 0, st>>>(lev[l], lev[l + 1], kc_r[l],
                                                                  part);
    } else {
      k_lresid_restrict<<<nblk(lev[l + 1].ncell), kNT, 0, st>>>(lev[l], lev[l + 1], part);
    }
    PLAUNCH(ctx);
    vcycle(l + 1, nullptr);
    if (nblk_p[l] > 0) {
      if (lev[l].patch)
        k_lprolong_tiled<true><<<nblk_p[l], 256, 0, st>>>(lev[l], lev[l + 1], kc_p[l]);
      else
        k_lprolong_tiled<false><<<nblk_p[l], 256, 0, st>>>(lev[l], lev[l + 1], kc_p[l]);
    } else {
      k_lprolong<<<nblk(lev[l].ncell), kNT, 0, st>>>(lev[l], lev[l + 1]);
    }
    PLAUNCH(ctx);
    smooth(l, post);
  }
};

}  // namespace

extern "C" int fr_poisson_solve(frmg_ctx *ctx, const double *density, const double *u,
                                const int dims[3], double box_mpc_h, double a, double omega_m,
                                double fr0_abs, const double *phib, double h, double tol,
                                double *phi_inout, const fr_opts *opts, fr_stats *stats,
                                double *src_mean, void *stream) {
  try {
    const auto t0 = std::chrono::steady_clock::now();
    if (!ctx || !density || !u || !dims || !phi_inout)
      throw PError{FR_EINVAL, "NULL argument"};
    PCK(cudaSetDevice(frmg_device(ctx)));
    for (int d = 0; d < 3; d++)
      if (dims[d] < 2 || (dims[d] & 1)) throw PError{FR_EINVAL, "dims must be even and >= 2"};
    const long long nc = (long long)dims[0] * dims[1] * dims[2];
    if (nc >= (1ll << 31)) throw PError{FR_EINVAL, "grid too large (at most 2^31 - 1 cells)"};
    if (!(tol >= 0)) throw PError{FR_EINVAL, "tol must be >= 0"};
    fr_opts o;
    fr_opts_default(&o);
    if (opts) o = *opts;
    if (o.pre < 0 || o.post < 0 || o.pre + o.post < 1 || o.max_vcycles < 1 || o.max_outer < 1)
      throw PError{FR_EINVAL, "invalid options"};
    if (!(o.relax > 0 && o.relax < 2)) throw PError{FR_EINVAL, "relax must be in (0, 2)"};
    if (h <= 0) h = 1.0 / dims[0];
    double k6[6];
    int stc = fr_constants(box_mpc_h, dims[0], a, omega_m, fr0_abs, k6);
    if (stc != FR_OK) return stc;
    const double beta = k6[1], gamma = k6[2];
    cudaStream_t st = (cudaStream_t)stream;
    Arena A(ctx);
    // inputs on the device
    auto dev_in = [&](const double *p, long long n) -> const double * {
      if (!p) return nullptr;
      if (on_device(p)) return p;
      double *d = A.get<double>(n);
      PCK(cudaMemcpyAsync(d, p, n * sizeof(double), cudaMemcpyHostToDevice, st));
      return d;
    };
    long long nface = 2ll * dims[1] * dims[2] + 2ll * dims[0] * dims[2] + 2ll * dims[0] * dims[1];
    const double *drho = dev_in(density, nc);
    const double *du = dev_in(u, nc);
    const double *dphib = dev_in(phib, nface);
    const bool phi_dev = on_device(phi_inout);
    const double *dphi0 = dev_in(phi_inout, nc);
    double *dphi_out = phi_dev ? phi_inout : A.get<double>(nc);

    PFine P;
    memset(&P, 0, sizeof(P));
    P.n0 = dims[0];
    P.n1 = dims[1];
    P.n2 = dims[2];
    P.ncell = nc;
    P.fd0 = make_fastdiv((unsigned)P.n0);
    P.fd1 = make_fastdiv((unsigned)P.n1);
    P.phi = A.get<float2>(nc);
    P.s = A.get<float2>(nc);
    P.phib = dphib;
    {
      long long off = 0;
      const long long fs[6] = {(long long)dims[1] * dims[2], (long long)dims[1] * dims[2],
                               (long long)dims[0] * dims[2], (long long)dims[0] * dims[2],
                               (long long)dims[0] * dims[1], (long long)dims[0] * dims[1]};
      for (int f = 0; f < 6; f++) {
        P.foff[f] = off;
        off += fs[f];
      }
    }
    split_host(1.0 / (h * h), P.ih2h, P.ih2l);
    // multigrid levels of the correction equation
    PoissonSolver S{ctx, st, {}, o.pre, o.post, {}, {}, {}, {}, {}, {}};
    {
      const int nl = level_count(dims);
      int m[3] = {dims[0], dims[1], dims[2]};
      double hl = h;
      for (int l = 0; l < nl; l++) {
        PLevel L;
        L.n0 = m[0];
        L.n1 = m[1];
        L.n2 = m[2];
        L.ncell = (long long)m[0] * m[1] * m[2];
        L.fd0 = make_fastdiv((unsigned)m[0]);
        L.fd1 = make_fastdiv((unsigned)m[1]);
        L.h2 = (float)(hl * hl);
        L.relax = (float)o.relax;
        L.patch = phib != nullptr;
        L.e = A.get<float>(L.ncell);
        L.f = A.get<float>(L.ncell);
        L.e_alt = nullptr;
        PCK(cudaMemsetAsync(L.e, 0, L.ncell * sizeof(float), st));
        // tiled smoother on levels large enough to fill the GPU with 64 x 16
        // tiles; z-chunks minimise (waves of 4 resident blocks per SM) x
        // (planes per block, chunk + 4)
        int zcl = 0, nbt = 0;
        if (m[0] >= 32 && m[1] >= 16 && m[2] >= 8) {
          int sms = 0, dev = 0;
          PCK(cudaGetDevice(&dev));
          PCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
          const long long slots = 4ll * std::max(sms, 1);
          const long long tiles = (long long)((m[0] + 63) / 64) * ((m[1] + 15) / 16);
          double best = 1e300;
          for (int c = 1; c <= m[2]; c++) {
            const int z = (m[2] + c - 1) / c;
            const long long blocks = tiles * ((m[2] + z - 1) / z);
            const double cost = std::ceil((double)blocks / slots) * (z + 4);
            if (cost < best - 1e-9) {
              best = cost;
              zcl = z;
            }
          }
          const long long blocks = tiles * ((m[2] + zcl - 1) / zcl);
          if (blocks >= sms) {
            nbt = (int)blocks;
            L.e_alt = A.get<float>(L.ncell);
          } else {
            zcl = 0;
          }
        }
        S.zc.push_back(zcl);
        S.nblk_t.push_back(nbt);
        // tiled prolongation onto this level (from the next coarser one) where
        // its 64 x 16 tiles times coarse-plane chunks fill the GPU: chunks of
        // kc coarse planes minimise (waves of 8 resident blocks per SM) x (kc + 1)
        int kcp = 0, nbp = 0;
        if (l + 1 < nl && nbt > 0) {
          int sms = 0, dev = 0;
          PCK(cudaGetDevice(&dev));
          PCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
          const long long slots = 8ll * std::max(sms, 1);
          const long long tiles = (long long)((m[0] + 63) / 64) * ((m[1] + 15) / 16);
          const int c2 = m[2] / 2;
          double best = 1e300;
          for (int c = 1; c <= c2; c++) {
            const int z = (c2 + c - 1) / c;
            const long long blocks = tiles * ((c2 + z - 1) / z);
            const double cost = std::ceil((double)blocks / slots) * (z + 1);
            if (cost < best - 1e-9) {
              best = cost;
              kcp = z;
            }
          }
          nbp = (int)(tiles * ((c2 + kcp - 1) / kcp));
        }
        S.kc_p.push_back(kcp);
        S.nblk_p.push_back(nbp);
        // the residual + restriction from this level uses the same tiles and
        // coarse-plane chunks (blocks of 256 threads, one per coarse cell)
        S.kc_r.push_back(kcp);
        S.nblk_r.push_back(nbp);
        S.lev.push_back(L);
        for (int d = 0; d < 3; d++) m[d] /= 2;
        hl *= 2.0;
      }
    }
    const long long nb = nblk(nc);
    double *partial = A.get<double>(2 * nb);
    double *pin = frmg_pinned(ctx, 2);
    if (!pin) throw PError{FR_ENOMEM, "pinned host allocation failed"};
    if (nb > (long long)kRedCH * kRedCH) throw PError{FR_EINVAL, "grid too large"};
    const PartialSum psum{ctx, A.get<double>(2 * ((nb + kRedCH - 1) / kRedCH + 1)), pin, st};
    float ln2h, ln2l, g2h, g2l, bh, bl;
    split_host(std::log(2.0), ln2h, ln2l);
    split_host(2.0 * gamma, g2h, g2l);
    split_host(0.5 * beta, bh, bl);
    k_psource<<<nb, kNT, 0, st>>>(P, drho, du, dphi0, g2h, g2l, bh, bl, ln2h, ln2l, partial);
    PLAUNCH(ctx);
    double ssum, smax;
    psum(partial, nb, ssum, smax);
    const double smean = phib ? 0.0 : ssum / (double)nc;
    if (src_mean) *src_mean = smean;
    float smh, sml;
    split_host(smean, smh, sml);

    fr_stats sv;
    memset(&sv, 0, sizeof(sv));
    sv.tau_rms = std::nan("");  // not evaluated by the linear solve
    auto push = [&](double v) {
      if (sv.nhist < FR_HIST) sv.hist[sv.nhist++] = v;
    };
    double prev = HUGE_VAL;
    int status = FR_ENOCONV;
    // fine-level norm partials of the residual + restriction (one per block)
    const long long nbc = S.lev.size() > 1
                              ? (S.nblk_r[0] > 0 ? (long long)S.nblk_r[0] : nblk(S.lev[1].ncell))
                              : 0;
    double *partial0 = A.get<double>(2 * std::max<long long>(nbc, 1));
    for (int outer = 0; outer < o.max_outer; outer++) {
      k_pdefect<<<nb, kNT, 0, st>>>(P, smh, sml, S.lev[0].f, S.lev[0].e, partial, nullptr);
      PLAUNCH(ctx);
      double s2, dmax;
      psum(partial, nb, s2, dmax);
      const double r = std::sqrt(s2 / (double)nc);
      if (outer == 0) sv.res0_rms = r;
      sv.res_rms = r;
      sv.res_max = dmax;
      sv.outer = outer + 1;
      push(-r);
      if (!(r == r)) throw PError{FR_EDIVERGED, "non-finite residual"};
      if (r <= tol) {
        status = FR_OK;
        break;
      }
      if (outer > 0 && r > prev) throw PError{FR_EDIVERGED, "defect grew"};
      prev = r;
      if (sv.vcycles >= o.max_vcycles) break;
      // FP32 correction solve: stop near the FP32 floor (1e-5 of its start)
      // or when the cycle contraction stalls
      double rp = HUGE_VAL;
      for (int k = 0; k < o.max_vcycles; k++) {
        if (S.lev.size() == 1) {
          k_lcoarsest<<<1, kNT, 0, st>>>(S.lev[0], 500);
          PLAUNCH(ctx);
          sv.vcycles++;
          break;
        }
        S.vcycle(0, partial0);
        sv.vcycles++;
        double a2, am;
        psum(partial0, nbc, a2, am);
        const double rr = std::sqrt(a2 / (double)nc);  // residual after pre-smoothing
        push(rr);
        const double pred = rp < HUGE_VAL ? rr * std::sqrt(rr / rp) : rr;
        if (!(rr < 0.75 * rp) || rr <= 1e-5 * r || pred <= 0.5 * tol ||
            sv.vcycles >= o.max_vcycles)
          break;
        rp = rr;
      }
      k_pupdate<<<nb, kNT, 0, st>>>(P, S.lev[0].e);
      PLAUNCH(ctx);
    }
    // gauge (periodic): phi of zero mean
    double pmean = 0.0;
    if (!phib) {
      k_pphisum<<<nb, kNT, 0, st>>>(P, partial);
      PLAUNCH(ctx);
      double phisum, pm;
      psum(partial, nb, phisum, pm);
      pmean = phisum / (double)nc;
    }
    float mh, ml;
    split_host(pmean, mh, ml);
    k_pfinal<<<nb, kNT, 0, st>>>(P, mh, ml, dphi_out);
    PLAUNCH(ctx);
    if (!phi_dev)
      PCK(cudaMemcpyAsync(phi_inout, dphi_out, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    sv.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = sv;
    if (status != FR_OK) frmg_set_error("no convergence within the V-cycle or outer limits");
    return status;
  } catch (PError &e) {
    frmg_set_error(e.msg);
    if (stream) cudaStreamSynchronize((cudaStream_t)stream);
    return e.status;
  }
}

extern "C" int fr_poisson_source(frmg_ctx *ctx, const double *density, const double *u,
                                 const int dims[3], double box_mpc_h, double a,
                                 double omega_m, double fr0_abs, double *s_out, void *stream) {
  try {
    if (!ctx || !density || !u || !dims || !s_out) throw PError{FR_EINVAL, "NULL argument"};
    PCK(cudaSetDevice(frmg_device(ctx)));
    for (int d = 0; d < 3; d++)
      if (dims[d] < 1) throw PError{FR_EINVAL, "bad dims"};
    const long long nc = (long long)dims[0] * dims[1] * dims[2];
    double k6[6];
    int stc = fr_constants(box_mpc_h, dims[0], a, omega_m, fr0_abs, k6);
    if (stc != FR_OK) return stc;
    cudaStream_t st = (cudaStream_t)stream;
    Arena A(ctx);
    auto dev_in = [&](const double *p) -> const double * {
      if (on_device(p)) return p;
      double *d = A.get<double>(nc);
      PCK(cudaMemcpyAsync(d, p, nc * sizeof(double), cudaMemcpyHostToDevice, st));
      return d;
    };
    const double *drho = dev_in(density), *du = dev_in(u);
    const bool out_dev = on_device(s_out);
    double *ds = out_dev ? s_out : A.get<double>(nc);
    PFine P;
    memset(&P, 0, sizeof(P));
    P.ncell = nc;
    P.phi = A.get<float2>(nc);
    P.s = A.get<float2>(nc);
    const long long nb = nblk(nc);
    double *partial = A.get<double>(2 * nb);
    float ln2h, ln2l, g2h, g2l, bh, bl;
    split_host(std::log(2.0), ln2h, ln2l);
    split_host(2.0 * k6[2], g2h, g2l);
    split_host(0.5 * k6[1], bh, bl);
    k_psource<<<nb, kNT, 0, st>>>(P, drho, du, nullptr, g2h, g2l, bh, bl, ln2h, ln2l, partial);
    PLAUNCH(ctx);
    PFine Q = P;  // k_pfinal converts its phi array: point it at the source
    Q.phi = P.s;
    k_pfinal<<<nb, kNT, 0, st>>>(Q, 0.f, 0.f, ds);
    PLAUNCH(ctx);
    if (!out_dev) PCK(cudaMemcpyAsync(s_out, ds, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    return FR_OK;
  } catch (PError &e) {
    frmg_set_error(e.msg);
    return e.status;
  }
}
