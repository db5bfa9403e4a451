// frmg_solver.cu -- host driver and C ABI of the f(R) FAS multigrid solver.
//
// Method: Li, Zhao, Teyssier & Koyama (arXiv:1110.1379), Sec. V.B: FAS
// V-cycles of red-black Newton-Gauss-Seidel relaxation on the domain grid and
// on refinement patches whose Dirichlet boundary values come from the parent
// solution.  Everything that touches a grid cell runs in the kernels of
// frmg_kernels.cuh; this file builds level hierarchies, launches kernels and
// reads back per-grid residual norms.
//
// Precisions:
//  * FR_FP64: the plain method in FP64 (V-cycle, then an FP64 residual norm).
//  * FR_MIXED: iterative refinement.  Outer loop in FP64: d = A(u) - f
//    (the fine-grid defect and the convergence test), then FP32 FAS V-cycles
//    solve N(delta) = -d for a correction on the FP32 background fp32(u),
//    then u += delta in FP64.
// Batching: every launch covers all grids (fields or patches) at one depth of
// their hierarchies; a per-field active flag drops converged fields.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "frmg.h"
#include "frmg_internal.h"
#include "frmg_kernels.cuh"
#include "frmg_df.cuh"

using namespace frmg;

// ---------------------------------------------------------------------------
// errors
static thread_local std::string g_last_error;

void frmg_set_error(const std::string &s) { g_last_error = s; }

struct FrError {
  int status;
  std::string msg;
};

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw FrError{FR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};      \
  } while (0)

#define CK_LAUNCH(ctx)                                                                  \
  do {                                                                                  \
    (ctx)->launches++;                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess)                                                              \
      throw FrError{FR_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)}; \
  } while (0)

static void einval(const std::string &m) { throw FrError{FR_EINVAL, m}; }

// ---------------------------------------------------------------------------
// context: device, caching allocator, pinned readback buffer
struct ProfPending {
  const char *name;
  cudaEvent_t a, b;
};

struct frmg_ctx {
  int device = 0;
  long long launches = 0;
  std::multimap<size_t, void *> free_blocks;
  std::map<void *, size_t> sizes;
  // device workspace held by the allocator (in use or cached) and its cap
  // (0 = none; FRMG_WORKSPACE_LIMIT at creation): an allocation that would
  // pass the cap fails with FR_ENOMEM as a failed cudaMalloc does
  size_t held = 0, limit = 0;
  double *pinned = nullptr;
  size_t pinned_n = 0;
  // optional per-kernel timing with CUDA events on the launch stream
  bool prof = false;
  std::vector<ProfPending> pending;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::string> prof_names;
  std::vector<long long> prof_count;
  std::vector<double> prof_ms;
  // stream of solves issued on the legacy default stream (created on first use)
  cudaStream_t side = nullptr;
  cudaEvent_t side_in = nullptr, side_out = nullptr;
  // stream of the early device-to-host copy of a mixed solve's result
  cudaStream_t copy = nullptr;
  cudaEvent_t copy_in = nullptr, copy_out = nullptr;
};

static cudaEvent_t ev_get(frmg_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Accumulates the finished events (call after a stream synchronisation).
static void prof_harvest(frmg_ctx *c) {
  for (auto &p : c->pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.b);
    cudaEventElapsedTime(&ms, p.a, p.b);
    size_t i = 0;
    for (; i < c->prof_names.size(); i++)
      if (c->prof_names[i] == p.name) break;
    if (i == c->prof_names.size()) {
      c->prof_names.push_back(p.name);
      c->prof_count.push_back(0);
      c->prof_ms.push_back(0.0);
    }
    c->prof_count[i]++;
    c->prof_ms[i] += ms;
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
}

// Brackets one kernel launch with events when profiling is on.
struct ProfScope {
  frmg_ctx *c;
  cudaStream_t st;
  const char *name;
  cudaEvent_t a = nullptr;
  ProfScope(frmg_ctx *c_, cudaStream_t st_, const char *n) : c(c_), st(st_), name(n) {
    if (c->prof && (a = ev_get(c)) != nullptr) cudaEventRecord(a, st);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = ev_get(c);
    if (!b) return;
    cudaEventRecord(b, st);
    c->pending.push_back({name, a, b});
  }
};
#define PROF(name) ProfScope prof_scope_(ctx, st, name)

long long &frmg_launch_counter(frmg_ctx *c) { return c->launches; }
int frmg_device(frmg_ctx *c) { return c->device; }

static size_t round_bytes(size_t b) { return (b + 4095) & ~(size_t)4095; }

void *frmg_alloc(frmg_ctx *c, size_t bytes) {
  bytes = round_bytes(std::max<size_t>(bytes, 1));
  auto it = c->free_blocks.find(bytes);
  if (it != c->free_blocks.end()) {
    void *p = it->second;
    c->free_blocks.erase(it);
    return p;
  }
  auto device_malloc = [&](void **q) {
    if (c->limit && c->held + bytes > c->limit) return false;
    if (cudaMalloc(q, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  void *p = nullptr;
  if (!device_malloc(&p)) {
    // drop the cache and retry once
    for (auto &kv : c->free_blocks) {
      cudaFree(kv.second);
      c->held -= c->sizes[kv.second];
      c->sizes.erase(kv.second);
    }
    c->free_blocks.clear();
    if (!device_malloc(&p))
      throw FrError{FR_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed" +
                                   (c->limit ? " (workspace limit " + std::to_string(c->limit) +
                                                   " bytes)"
                                             : std::string())};
  }
  c->sizes[p] = bytes;
  c->held += bytes;
  return p;
}

void frmg_release(frmg_ctx *c, void *p) {
  if (!p) return;
  auto it = c->sizes.find(p);
  if (it == c->sizes.end()) return;
  c->free_blocks.emplace(it->second, p);
}

static double *pinned_buf(frmg_ctx *c, size_t n) {
  if (c->pinned_n < n) {
    if (c->pinned) cudaFreeHost(c->pinned);
    c->pinned = nullptr;
    c->pinned_n = 0;
    if (cudaMallocHost((void **)&c->pinned, n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      throw FrError{FR_ENOMEM, "cudaMallocHost failed"};
    }
    c->pinned_n = n;
  }
  return c->pinned;
}

double *frmg_pinned(frmg_ctx *c, size_t n) {
  try {
    return pinned_buf(c, n);
  } catch (...) {
    return nullptr;
  }
}

// Allocations of one call, returned to the cache on scope exit.
struct Scope {
  frmg_ctx *c;
  std::vector<void *> ptrs;
  explicit Scope(frmg_ctx *c_) : c(c_) {}
  template <typename T>
  T *get(size_t n) {
    void *p = frmg_alloc(c, n * sizeof(T));
    ptrs.push_back(p);
    return (T *)p;
  }
  ~Scope() {
    for (void *p : ptrs) frmg_release(c, p);
  }
};

// ---------------------------------------------------------------------------
// model constants (Sec. II, III.A, VI.A.1), n = 1, flat background
struct Consts {
  double alpha, beta, gamma, ct, fbar, ubar;
};

static Consts model_consts(double box, double h, double a, double om, double fr0) {
  Consts k;
  double ol = 1.0 - om;
  k.ct = 299792.458 / (100.0 * box);
  double K = 1.0 / (a * a * a) + 4.0 * ol / om;
  double K1 = 1.0 + 4.0 * ol / om;
  double xi = fr0 * (3.0 * K1) * (3.0 * K1);
  k.fbar = a * a * xi / ((3.0 * K) * (3.0 * K));
  k.alpha = k.ct * k.ct * k.fbar / (h * h);
  k.beta = om * a * a * a * a * K;
  k.gamma = om * a;
  k.ubar = std::log(k.fbar);
  return k;
}

static void check_dims(const int n[3], int minn = 2) {
  for (int d = 0; d < 3; d++)
    if (n[d] < minn || (n[d] & 1)) einval("dims must be even and >= " + std::to_string(minn));
}

static void check_model(double box, double a, double om, double fr0) {
  if (!(box > 0) || !(a > 0) || !(fr0 > 0) || !(om > 0 && om < 1))
    einval("box, a and |f_R0| must be > 0 and 0 < Omega_m < 1");
}

// Reading of the level count (the paper does not fix it): halve while every
// next size is even and >= 4.
static int count_levels(const int n[3]) {
  int m[3] = {n[0], n[1], n[2]};
  int nl = 1;
  for (;;) {
    bool ok = true;
    for (int d = 0; d < 3; d++) {
      if (m[d] & 1) ok = false;
      int nx = m[d] / 2;
      if (nx < 4 || (nx & 1)) ok = false;
    }
    if (!ok) break;
    for (int d = 0; d < 3; d++) m[d] /= 2;
    nl++;
  }
  return nl;
}

static long long face_total(const int n[3]) {
  return 2LL * n[1] * n[2] + 2LL * n[0] * n[2] + 2LL * n[0] * n[1];
}

static void face_offsets(const int n[3], long long off[6]) {
  long long sz[6] = {(long long)n[1] * n[2], (long long)n[1] * n[2], (long long)n[0] * n[2],
                     (long long)n[0] * n[2], (long long)n[0] * n[1], (long long)n[0] * n[1]};
  long long o = 0;
  for (int f = 0; f < 6; f++) {
    off[f] = o;
    o += sz[f];
  }
}

// ---------------------------------------------------------------------------
// small kernels used only by the host driver
template <typename T>
__global__ void k_expm1(const T *u, T *x, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] = m_expm1(u[t]);
}

template <typename S, typename D>
__global__ void k_convert(const S *s, D *d, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) d[t] = (D)s[t];
}

__global__ void k_expf(const float *u, float *e, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) e[t] = expf(u[t]);
}

// Mixed precision: from the FP64 defect d, the inner right-hand side -d and the
// FP32 background fp32(u) with e^{fp32(u)}; the correction restarts at 0.
__global__ void k_prep_inner(const double *d64, const double *u64, float *r32, float *ub32,
                             float *E32, float *delta, float *x32, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  r32[t] = (float)(-d64[t]);
  float ub = (float)u64[t];
  ub32[t] = ub;
  E32[t] = expf(ub);
  delta[t] = 0.0f;
  x32[t] = 0.0f;
}

// Zero-start set-up of the mixed loop: the first inner solve works on the full
// variable, u32 = 0 with right-hand side fp32(gamma (rho - 1)).
// Block partials of (sum r^2, max |r|) go to partial[2 (base + block)]: the
// initial residual is A(0) - gamma (rho - 1) = -r.
__global__ void __launch_bounds__(256) k_prep_zero(const double *rho, double gamma, float *r32,
                                                   float *u32, float *x32, long long n,
                                                   double *partial, int base) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float s = 0.0f, m = 0.0f;
  if (t < n) {
    float r = (float)(gamma * (rho[t] - 1.0));
    r32[t] = r;
    u32[t] = 0.0f;
    x32[t] = 0.0f;
    s = r * r;
    m = fabsf(r);
  }
  block_reduce2f<256>(s, m, &partial[2 * (base + blockIdx.x)], &partial[2 * (base + blockIdx.x) + 1]);
}

// Integer tests on the bit pattern (no FP64 instructions): +-0 has all bits
// but the sign clear.  One plain store per warp that saw a non-zero value
// (every writer stores 1; an atomic per cell serialises on the flag when u is
// non-zero everywhere).  Launched with a multiple of 32 threads per block.
__global__ void k_any_nonzero(const double *u, long long n, int *flag) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool nz = t < n && ((unsigned long long)__double_as_longlong(u[t]) << 1) != 0;
  if (__any_sync(0xffffffffu, nz) && (threadIdx.x & 31) == 0) *flag = 1;
}

// n doubles from device memory to page-locked host memory written by the
// kernel itself (a zero-copy read-back that does not wait behind copies
// queued on the copy engines).
__global__ void k_copy_to_host(const double *src, double *dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// u += delta in FP64, x = expm1(u).
__global__ void k_update64(double *u64, double *x64, const float *delta, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double u = u64[t] + (double)delta[t];
  u64[t] = u;
  x64[t] = expm1(u);
}

// Restriction of packed boundary faces: a coarse face value is the mean of the
// 4 fine face values covering it (reading of Sec. V.B.2, where the coarse u_B
// come from the matching cells of the coarser level).
template <typename T>
__global__ void k_restrict_faces(const T *fine, int nf0, int nf1, int nf2, T *coarse) {
  int nf[3] = {nf0, nf1, nf2};
  int nc[3] = {nf0 / 2, nf1 / 2, nf2 / 2};
  long long tot = 2LL * nc[1] * nc[2] + 2LL * nc[0] * nc[2] + 2LL * nc[0] * nc[1];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  long long offc = 0, offf = 0;
  for (int f = 0; f < 6; f++) {
    int ax = f / 2;
    int p = ax == 0 ? 1 : 0, q = ax == 2 ? 1 : 2;
    long long szc = (long long)nc[p] * nc[q], szf = (long long)nf[p] * nf[q];
    if (t < offc + szc) {
      long long r = t - offc;
      int P = (int)(r % nc[p]), Q = (int)(r / nc[p]);
      T s = T(0);
      for (int b = 0; b < 2; b++)
        for (int a = 0; a < 2; a++) s += fine[offf + (long long)(2 * Q + b) * nf[p] + 2 * P + a];
      coarse[t] = s * T(0.25);
      return;
    }
    offc += szc;
    offf += szf;
  }
}

static int nblocks(long long n, int nt = 256) { return (int)((n + nt - 1) / nt); }

// ---------------------------------------------------------------------------
// problems and level hierarchies
struct Problem {
  int n[3];
  double h, box, a, om, fr0;
  const double *rho;  // device
  double *u;          // device, in/out
  const double *bnd;  // device packed faces (patches) or null
  Consts k;
  int nl;
  int zero_u;         // 1: start from u = 0 without reading u (initial_guess = 0)
  int check_rho;      // the solve validates rho itself: 0 no, 1 yes, 2 yes, negatives allowed
  double *host_u;     // page-locked host destination of u (single-field solves with
                      // a page-locked host u), else null
  int early_copied;   // set by the mixed solve: u already copied to host_u
};

// tile of the tiled smoother (x by y cells; S = 1 and S = 2 sweeps per pass)
constexpr int kTX = 64, kTY = 16;
// tile height of k_smooth_rb: 64 x 16 tiles leave room for three resident
// blocks per SM (more loads in flight than two blocks of 64 x 32 tiles)
constexpr int kRbTY = 16;
// plain-form one-sweep smoother of the solves when fr_opts.smooth_tile = 0:
// the register-column kernel on 64 x kDefaultSmoothTile tiles (-1 = k_smooth_rb)
constexpr int kDefaultSmoothTile = 16;

template <typename T>
struct LevelSet {
  std::vector<Grid<T>> h;
  Grid<T> *d = nullptr;
  std::vector<int> off_half, off_full;
  int *d_off_half = nullptr, *d_off_full = nullptr;
  int nblk_half = 0, nblk_full = 0;
  // tiled FP32 smoother: blocks per grid for TX x TY tiles and zc-plane chunks
  bool tiled = false;     // the tiled smoother is used for this set
  bool tiled_ok = false;  // it could be used (every grid >= 16 cells a side)
  bool dirichlet = false; // patches (all grids of a set are patches or all periodic)
  int zc = 0;
  std::vector<int> off_tile;
  int *d_off_tile = nullptr;
  int nblk_tile = 0;
  // one-sweep red-black smoother (64 x kRbTY tiles); [0] plain, [1] correction
  // form (their occupancies differ, and with them the best z-chunk)
  int zc_rb[2] = {0, 0};
  std::vector<int> off_rb[2];
  int *d_off_rb[2] = {nullptr, nullptr};
  int nblk_rb[2] = {0, 0};
  // register-column one-sweep smoother: [0] plain form on 64 x rc_ty[0]
  // tiles, [1] correction form on 64 x 8 tiles (rc_ty 0: k_smooth_rb instead)
  int rc_ty[2] = {0, 0};
  int zc_rc[2] = {0, 0};
  std::vector<int> off_rc[2];
  int *d_off_rc[2] = {nullptr, nullptr};
  int nblk_rc[2] = {0, 0};
  // tiled FAS right-hand side (coarse side of a V-cycle level); [0] plain,
  // [1] correction form
  int zc_fr[2] = {0, 0};
  std::vector<int> off_fr[2];
  int *d_off_fr[2] = {nullptr, nullptr};
  int nblk_fr[2] = {0, 0};
  // tiled prolongation (fine side of a V-cycle level): chunks of coarse planes
  int kc_pl = 0;
  std::vector<int> off_pl;
  int *d_off_pl = nullptr;
  int nblk_pl = 0;
  // tiled residual + restriction (fine side of a V-cycle level)
  bool rr_tiled = false;
  int zc_rr = 0;
  std::vector<int> off_rr;
  int *d_off_rr = nullptr;
  int nblk_rr = 0;
  double *partial = nullptr;  // per-block norm partials
  int red_nch = 0;            // chunks of the two-stage sum over off_full partials
  double *red_tmp = nullptr;  // its chunk sums
  double *red = nullptr;      // per-grid (sum of squares, max)
  T **d_dout = nullptr;       // per-grid residual output pointers
  bool empty() const { return h.empty(); }
  int size() const { return (int)h.size(); }
};

// Chunks of the two-stage sum of per-block partials (0: one stage suffices).
constexpr int kRedChunk = 4096;
static int red_chunks(const std::vector<int> &off) {
  int maxc = 0;
  for (size_t g = 0; g + 1 < off.size(); g++) maxc = std::max(maxc, off[g + 1] - off[g]);
  return maxc <= 2 * kRedChunk ? 0 : (maxc + kRedChunk - 1) / kRedChunk;
}

static int sm_count() {
  static int n = 0;
  if (n <= 0) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    if (n <= 0) n = 1;
  }
  return n;
}

// Resident blocks per SM of a kernel launched with `threads` threads and
// `smem` bytes of dynamic shared memory (raises the kernel's shared-memory
// limit to `smem` first, as its launch does).
template <typename K>
static int resident_blocks(K kernel, int threads, size_t smem) {
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int nb = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem));
  return std::max(nb, 1);
}

// z-chunk length of a tiled z-marching kernel.  A block streams its chunk
// plus `halo` planes; with every block costing the same per plane, a launch
// takes about (waves of resident blocks) x (chunk + halo) plane-times.  The
// chunk (even if `even`) minimising that over the set's grids (tiles[g] tiles
// per plane, n2[g] planes) is returned; ties go to the longer chunk.
static int pick_chunk(const std::vector<long long> &tiles, const std::vector<int> &n2, long long slots,
                      int halo, bool even) {
  int maxn2 = 1;
  for (int v : n2) maxn2 = std::max(maxn2, v);
  double best = 1e300;
  int bz = maxn2, prev = -1;
  for (int c = 1; c <= maxn2; c++) {
    int zc = (maxn2 + c - 1) / c;
    if (even) zc = (zc + 1) & ~1;
    if (zc == prev) continue;
    prev = zc;
    double work = 0.0;  // block-planes of the launch
    for (size_t g = 0; g < tiles.size(); g++) {
      const long long nb = tiles[g] * ((n2[g] + zc - 1) / zc);
      work += (double)nb * (std::min(zc, n2[g]) + halo);
    }
    const double per = zc + halo;
    const double cost = std::ceil(work / ((double)slots * per)) * per;
    if (cost < best - 1e-9) {
      best = cost;
      bz = zc;
    }
  }
  return bz;
}

template <bool BG, bool DIR>
static long long rb_slots();
template <bool BG, bool DIR, int TY>
static long long rc_slots();
template <bool BG, bool DIR>
static long long fr_slots();
template <bool DIR>
static long long pl_slots();
template <bool DIR>
static long long rr_slots();

template <typename T>
static void upload_set(Scope &S, LevelSet<T> &ls, cudaStream_t st, int tiling = 0,
                       int stile = 0) {
  if (ls.empty()) return;
  int ng = ls.size();
  ls.off_half.assign(ng + 1, 0);
  ls.off_full.assign(ng + 1, 0);
  for (int g = 0; g < ng; g++) {
    long long half = (long long)(ls.h[g].n0 / 2) * ls.h[g].n1 * ls.h[g].n2;
    ls.off_half[g + 1] = ls.off_half[g] + nblocks(half);
    ls.off_full[g + 1] = ls.off_full[g] + nblocks(ls.h[g].ncell);
  }
  ls.nblk_half = ls.off_half[ng];
  ls.nblk_full = ls.off_full[ng];
  // every grid reaches the device through here: its index dividers too
  for (auto &g : ls.h) {
    g.fd0 = make_fastdiv((unsigned)g.n0);
    g.fd1 = make_fastdiv((unsigned)g.n1);
  }
  ls.d = S.get<Grid<T>>(ng);
  ls.d_off_half = S.get<int>(ng + 1);
  ls.d_off_full = S.get<int>(ng + 1);
  CK(cudaMemcpyAsync(ls.d, ls.h.data(), ng * sizeof(Grid<T>), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ls.d_off_half, ls.off_half.data(), (ng + 1) * sizeof(int),
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ls.d_off_full, ls.off_full.data(), (ng + 1) * sizeof(int),
                     cudaMemcpyHostToDevice, st));
  ls.dirichlet = ls.h[0].bnd != nullptr;
  for (int g = 1; g < ng; g++)
    if ((ls.h[g].bnd != nullptr) != ls.dirichlet)
      throw FrError{FR_EINVAL, "a level set mixes patches and periodic grids"};
  // tiled smoother for FP32 sets whose grids are all at least 16 cells a side
  ls.tiled = sizeof(T) == 4;
  int maxn2 = 0;
  long long txy = 0;
  for (int g = 0; g < ng; g++) {
    const Grid<T> &G = ls.h[g];
    if (std::min(G.n0, std::min(G.n1, G.n2)) < 16) ls.tiled = false;
    maxn2 = std::max(maxn2, G.n2);
    txy += (long long)((G.n0 + kTX - 1) / kTX) * ((G.n1 + kTY - 1) / kTY);
  }
  if (ls.tiled) {
    // chunks of z so that the set yields about 1216 blocks (several waves of
    // resident blocks), never thinner than 32 planes; sets too small to fill
    // the GPU with such blocks use the one-thread-per-cell kernel instead
    long long nz = std::max<long long>(1, (1216 + txy - 1) / txy);
    ls.zc = (int)std::max<long long>(std::min(32, maxn2), (maxn2 + nz - 1) / nz);
    ls.tiled_ok = true;
    if (tiling == 0 && txy * ((maxn2 + ls.zc - 1) / ls.zc) < 304) ls.tiled = false;
    if (tiling < 0) ls.tiled = false;
  }
  if (ls.tiled_ok) {
    ls.off_tile.assign(ng + 1, 0);
    for (int g = 0; g < ng; g++) {
      const Grid<T> &G = ls.h[g];
      int nt = ((G.n0 + kTX - 1) / kTX) * ((G.n1 + kTY - 1) / kTY) * ((G.n2 + ls.zc - 1) / ls.zc);
      ls.off_tile[g + 1] = ls.off_tile[g] + nt;
    }
    ls.nblk_tile = ls.off_tile[ng];
    ls.d_off_tile = S.get<int>(ng + 1);
    CK(cudaMemcpyAsync(ls.d_off_tile, ls.off_tile.data(), (ng + 1) * sizeof(int),
                       cudaMemcpyHostToDevice, st));
    if constexpr (sizeof(T) == 4) {
      std::vector<long long> tl(ng);
      std::vector<int> n2s(ng);
      for (int g = 0; g < ng; g++) {
        tl[g] = (long long)((ls.h[g].n0 + kTX - 1) / kTX) * ((ls.h[g].n1 + kRbTY - 1) / kRbTY);
        n2s[g] = ls.h[g].n2;
      }
      for (int v = 0; v < 2; v++) {
        const long long slots = ls.dirichlet ? (v ? rb_slots<true, true>() : rb_slots<false, true>())
                                             : (v ? rb_slots<true, false>() : rb_slots<false, false>());
        ls.zc_rb[v] = pick_chunk(tl, n2s, slots, 4, false);
        ls.off_rb[v].assign(ng + 1, 0);
        for (int g = 0; g < ng; g++)
          ls.off_rb[v][g + 1] =
              ls.off_rb[v][g] + (int)(tl[g] * ((n2s[g] + ls.zc_rb[v] - 1) / ls.zc_rb[v]));
        ls.nblk_rb[v] = ls.off_rb[v][ng];
        ls.d_off_rb[v] = S.get<int>(ng + 1);
        CK(cudaMemcpyAsync(ls.d_off_rb[v], ls.off_rb[v].data(), (ng + 1) * sizeof(int),
                           cudaMemcpyHostToDevice, st));
      }
      if (stile == 8 || stile == 16) {
        // plain form on 64 x stile tiles, correction form on 64 x 8 tiles
        for (int v = 0; v < 2; v++) {
          const int ty = v ? 8 : stile;
          ls.rc_ty[v] = ty;
          for (int g = 0; g < ng; g++)
            tl[g] = (long long)((ls.h[g].n0 + kTX - 1) / kTX) * ((ls.h[g].n1 + ty - 1) / ty);
          long long slots;
          if (v)
            slots = ls.dirichlet ? rc_slots<true, true, 8>() : rc_slots<true, false, 8>();
          else if (ty == 8)
            slots = ls.dirichlet ? rc_slots<false, true, 8>() : rc_slots<false, false, 8>();
          else
            slots = ls.dirichlet ? rc_slots<false, true, 16>() : rc_slots<false, false, 16>();
          ls.zc_rc[v] = pick_chunk(tl, n2s, slots, 4, false);
          ls.off_rc[v].assign(ng + 1, 0);
          for (int g = 0; g < ng; g++)
            ls.off_rc[v][g + 1] =
                ls.off_rc[v][g] + (int)(tl[g] * ((n2s[g] + ls.zc_rc[v] - 1) / ls.zc_rc[v]));
          ls.nblk_rc[v] = ls.off_rc[v][ng];
          ls.d_off_rc[v] = S.get<int>(ng + 1);
          CK(cudaMemcpyAsync(ls.d_off_rc[v], ls.off_rc[v].data(), (ng + 1) * sizeof(int),
                             cudaMemcpyHostToDevice, st));
        }
      }
      for (int g = 0; g < ng; g++)
        tl[g] = (long long)((ls.h[g].n0 + kFrTX - 1) / kFrTX) * ((ls.h[g].n1 + kFrTY - 1) / kFrTY);
      for (int v = 0; v < 2; v++) {
        const long long slots = ls.dirichlet ? (v ? fr_slots<true, true>() : fr_slots<false, true>())
                                             : (v ? fr_slots<true, false>() : fr_slots<false, false>());
        ls.zc_fr[v] = pick_chunk(tl, n2s, slots, 2, false);
        ls.off_fr[v].assign(ng + 1, 0);
        for (int g = 0; g < ng; g++)
          ls.off_fr[v][g + 1] =
              ls.off_fr[v][g] + (int)(tl[g] * ((n2s[g] + ls.zc_fr[v] - 1) / ls.zc_fr[v]));
        ls.nblk_fr[v] = ls.off_fr[v][ng];
        ls.d_off_fr[v] = S.get<int>(ng + 1);
        CK(cudaMemcpyAsync(ls.d_off_fr[v], ls.off_fr[v].data(), (ng + 1) * sizeof(int),
                           cudaMemcpyHostToDevice, st));
      }
    }
  }
  if (ls.tiled) {
    // tiled residual + restriction: even z-chunks (coarse planes stay whole)
    if constexpr (sizeof(T) == 4) {
      std::vector<long long> tl(ng);
      std::vector<int> n2s(ng);
      for (int g = 0; g < ng; g++) {
        tl[g] = (long long)((ls.h[g].n0 + kTX - 1) / kTX) * ((ls.h[g].n1 + kTY - 1) / kTY);
        n2s[g] = ls.h[g].n2;
      }
      ls.zc_rr = pick_chunk(tl, n2s, ls.dirichlet ? rr_slots<true>() : rr_slots<false>(), 2, true);
      // prolongation onto this set from its coarser set (every grid even-sized)
      bool even = true;
      for (int g = 0; g < ng; g++) {
        even = even && !(ls.h[g].n2 & 1);
        tl[g] = (long long)((ls.h[g].n0 + kPlTX - 1) / kPlTX) * ((ls.h[g].n1 + kPlTY - 1) / kPlTY);
        n2s[g] = ls.h[g].n2 / 2;
      }
      if (even) {
        ls.kc_pl = pick_chunk(tl, n2s, ls.dirichlet ? pl_slots<true>() : pl_slots<false>(), 2, false);
        ls.off_pl.assign(ng + 1, 0);
        for (int g = 0; g < ng; g++)
          ls.off_pl[g + 1] = ls.off_pl[g] + (int)(tl[g] * ((n2s[g] + ls.kc_pl - 1) / ls.kc_pl));
        ls.nblk_pl = ls.off_pl[ng];
        ls.d_off_pl = S.get<int>(ng + 1);
        CK(cudaMemcpyAsync(ls.d_off_pl, ls.off_pl.data(), (ng + 1) * sizeof(int),
                           cudaMemcpyHostToDevice, st));
      }
    }
    ls.off_rr.assign(ng + 1, 0);
    for (int g = 0; g < ng; g++) {
      const Grid<T> &G = ls.h[g];
      int nt = ((G.n0 + kTX - 1) / kTX) * ((G.n1 + kTY - 1) / kTY) *
               ((G.n2 + ls.zc_rr - 1) / ls.zc_rr);
      ls.off_rr[g + 1] = ls.off_rr[g] + nt;
    }
    ls.nblk_rr = ls.off_rr[ng];
    ls.d_off_rr = S.get<int>(ng + 1);
    CK(cudaMemcpyAsync(ls.d_off_rr, ls.off_rr.data(), (ng + 1) * sizeof(int),
                       cudaMemcpyHostToDevice, st));
    ls.rr_tiled = true;
  }
  ls.partial = S.get<double>(2 * (size_t)std::max(ls.nblk_full, ls.nblk_rr));
  ls.red_nch = red_chunks(ls.off_full);
  if (ls.red_nch) ls.red_tmp = S.get<double>(2 * (size_t)ls.red_nch * ng);
  ls.red = S.get<double>(2 * (size_t)ng);
  ls.d_dout = S.get<T *>(ng);
  // host vectors must stay alive until the copies finished
  CK(cudaStreamSynchronize(st));
}

// Level hierarchy of a batch of problems in precision T.  BG: background mode
// (the FP32 inner solve of the mixed loop).
template <typename T>
struct Hier {
  int depth = 0;
  std::vector<std::vector<Grid<T>>> lev;  // lev[p][l]
  std::vector<LevelSet<T>> cont, next, coarsest, all;
  std::vector<float *> bg_u, bg_E;        // fine-level background arrays per problem
  std::vector<int> par;                   // current u buffer (0/1) per depth
  T *cur_u(int pi, int l) const { return par[l] ? lev[pi][l].u2 : lev[pi][l].u; }
  T *cur_x(int pi, int l) const { return par[l] ? lev[pi][l].x2 : lev[pi][l].x; }
};

template <typename T, bool BG>
static void build_hier(Scope &S, Hier<T> &H, std::vector<Problem> &P, double cap,
                       cudaStream_t st, frmg_ctx *ctx, int tiling = 0, double relax = 1.0,
                       int stile = 0) {
  int np = (int)P.size();
  H.lev.assign(np, {});
  H.depth = 0;
  for (auto &p : P) H.depth = std::max(H.depth, p.nl);
  H.bg_u.assign(np, nullptr);
  H.bg_E.assign(np, nullptr);
  for (int pi = 0; pi < np; pi++) {
    Problem &p = P[pi];
    int n[3] = {p.n[0], p.n[1], p.n[2]};
    double h = p.h;
    const T *bnd_prev = nullptr;
    for (int l = 0; l < p.nl; l++) {
      Grid<T> G;
      memset(&G, 0, sizeof(G));
      G.n0 = n[0];
      G.n1 = n[1];
      G.n2 = n[2];
      G.ncell = (long long)n[0] * n[1] * n[2];
      G.field = pi;
      Consts k = model_consts(p.box, h, p.a, p.om, p.fr0);
      G.ah = (T)(0.5 * k.alpha);
      G.beta = (T)k.beta;
      G.cap = (T)cap;
      G.relax = (T)relax;
      face_offsets(n, G.foff);
      bool fine_fp64_plain = (l == 0 && !BG && sizeof(T) == 8);
      if (fine_fp64_plain) {
        G.u = (T *)p.u;
        G.f = (const T *)p.rho;
        G.fs = (T)k.gamma;
        G.fo = T(1);
      } else {
        G.u = S.get<T>(G.ncell);
        T *f = S.get<T>(G.ncell);
        G.f = f;
        G.fs = T(1);
        G.fo = T(0);
      }
      G.x = S.get<T>(G.ncell);
      if (sizeof(T) == 4) {
        G.u2 = S.get<T>(G.ncell);
        G.x2 = S.get<T>(G.ncell);
      }
      if (l > 0) G.uR = S.get<T>(G.ncell);
      if (BG) {
        float *ub = S.get<float>(G.ncell);
        float *E = S.get<float>(G.ncell);
        G.ubg = ub;
        G.Ebg = E;
        if (l == 0) {
          H.bg_u[pi] = ub;
          H.bg_E[pi] = E;
        }
      }
      if (p.bnd) {
        long long nf = face_total(n);
        T *b = S.get<T>(nf);
        if (l == 0) {
          if (sizeof(T) == 8)
            CK(cudaMemcpyAsync(b, p.bnd, nf * sizeof(double), cudaMemcpyDeviceToDevice, st));
          else {
            k_convert<double, float><<<nblocks(nf), 256, 0, st>>>(p.bnd, (float *)b, nf);
            CK_LAUNCH(ctx);
          }
        } else {
          int nfp[3] = {n[0] * 2, n[1] * 2, n[2] * 2};
          k_restrict_faces<T><<<nblocks(nf), 256, 0, st>>>(bnd_prev, nfp[0], nfp[1], nfp[2], b);
          CK_LAUNCH(ctx);
        }
        G.bnd = b;
        bnd_prev = b;
      }
      H.lev[pi].push_back(G);
      for (int d = 0; d < 3; d++) n[d] /= 2;
      h *= 2.0;
    }
  }
  H.par.assign(H.depth, 0);
  H.cont.assign(H.depth, {});
  H.next.assign(H.depth, {});
  H.coarsest.assign(H.depth, {});
  H.all.assign(H.depth, {});
  for (int pi = 0; pi < np; pi++) {
    int nl = P[pi].nl;
    for (int l = 0; l < nl; l++) {
      H.all[l].h.push_back(H.lev[pi][l]);
      if (l < nl - 1) {
        H.cont[l].h.push_back(H.lev[pi][l]);
        H.next[l].h.push_back(H.lev[pi][l + 1]);
      } else {
        H.coarsest[l].h.push_back(H.lev[pi][l]);
      }
    }
  }
  for (int l = 0; l < H.depth; l++) {
    upload_set(S, H.cont[l], st, tiling, stile);
    upload_set(S, H.next[l], st, tiling, stile);
    upload_set(S, H.coarsest[l], st, tiling, stile);
    upload_set(S, H.all[l], st, tiling, stile);
  }
}

// ---------------------------------------------------------------------------
// V-cycle (Sec. V.B.2), batched over the grids of each depth
struct CycleOpts {
  int pre, post;
  int tdepth;  // sweeps per tiled pass (1 or 2)
  double crs_rel, crs_abs;
  int crs_maxit, crs_stall;
  int crs_meanfix;  // constant-mode Newton step in periodic coarsest solves
  // 1: the solve records the finest-level buffer parity of every field that
  // leaves an inner solve early, so batches may also run odd numbers of
  // ping-pong passes per cycle (the parity of the grids still iterating then
  // flips each cycle while a field that left keeps its data where it was)
  int odd_ok = 0;
};

// Profiling names: kernel family, precision, fine (depth 0) or coarse level.
static const char *pname(const char *kind, bool f64, bool fine) {
  static const char *tab[][4] = {
      {"smooth_f64@fine", "smooth_f64@coarse", "smooth_f32@fine", "smooth_f32@coarse"},
      {"resid_restrict_f64@fine", "resid_restrict_f64@coarse", "resid_restrict_f32@fine",
       "resid_restrict_f32@coarse"},
      {"prolong_f64@fine", "prolong_f64@coarse", "prolong_f32@fine", "prolong_f32@coarse"},
      {"fas_rhs_f64@coarse", "fas_rhs_f64@coarse", "fas_rhs_f32@coarse", "fas_rhs_f32@coarse"},
      {"residual_f64@fine", "residual_f64@coarse", "residual_f32@fine", "residual_f32@coarse"}};
  int row = 0;
  if (!strcmp(kind, "resid_restrict")) row = 1;
  else if (!strcmp(kind, "prolong")) row = 2;
  else if (!strcmp(kind, "fas_rhs")) row = 3;
  else if (!strcmp(kind, "residual")) row = 4;
  return tab[row][(f64 ? 0 : 2) + (fine ? 0 : 1)];
}

template <bool BG, bool DIR, int S>
static void launch_tiled_k(frmg_ctx *ctx, LevelSet<float> &s, const int *active, int par,
                           cudaStream_t st) {
  using TC = TileCfg<S, kTX, kTY>;
  size_t sm = TC::smem(BG);
  static bool attr_set = false;
  if (!attr_set) {
    CK(cudaFuncSetAttribute(k_smooth_tiled<BG, DIR, S, kTX, kTY>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr_set = true;
  }
  k_smooth_tiled<BG, DIR, S, kTX, kTY><<<s.nblk_tile, TC::NT, sm, st>>>(s.d, s.d_off_tile,
                                                                        s.size(), s.zc, active, par);
}

template <bool BG, bool DIR>
static void launch_rr_k(frmg_ctx *ctx, LevelSet<float> &F, LevelSet<float> &C, const int *active,
                        int fpar, int cpar, double *partial, cudaStream_t st) {
  using RC = RRCfg<kTX, kTY>;
  size_t sm = RC::smem(BG);
  static bool attr_set = false;
  if (!attr_set) {
    CK(cudaFuncSetAttribute(k_resid_restrict_tiled<BG, DIR, kTX, kTY>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr_set = true;
  }
  k_resid_restrict_tiled<BG, DIR, kTX, kTY><<<F.nblk_rr, RC::NT, sm, st>>>(
      F.d, C.d, F.d_off_rr, F.size(), F.zc_rr, active, fpar, cpar, partial);
}

template <bool BG>
static void launch_rr_tiled(frmg_ctx *ctx, LevelSet<float> &F, LevelSet<float> &C,
                            const int *active, int fpar, int cpar, double *partial,
                            cudaStream_t st) {
  if (F.dirichlet)
    launch_rr_k<BG, true>(ctx, F, C, active, fpar, cpar, partial, st);
  else
    launch_rr_k<BG, false>(ctx, F, C, active, fpar, cpar, partial, st);
}

template <bool BG, bool DIR, int TY, bool PRL = false>
static void launch_rc_k(LevelSet<float> &s, const int *active, int par, cudaStream_t st,
                        const Grid<float> *coarse = nullptr, int cpar = 0) {
  using RC = RCCfg<TY, BG>;
  constexpr int v = BG ? 1 : 0;
  const size_t sm = RC::smem(PRL);
  static bool attr_set = false;
  if (!attr_set) {
    CK(cudaFuncSetAttribute(k_smooth_rc<BG, DIR, TY, PRL>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr_set = true;
  }
  k_smooth_rc<BG, DIR, TY, PRL><<<s.nblk_rc[v], RC::NT, sm, st>>>(
      s.d, s.d_off_rc[v], s.size(), s.zc_rc[v], active, par, coarse, cpar);
}

// The first post-smoothing sweep of a level with the prolongation from its
// coarser level applied to every arriving cell (plain-form register-column
// kernels only: the fused sweep computes x = expm1(u) of the arriving cells,
// which the plain sweep reads from the cache, and for the correction form that
// made the fused sweep slower than the prolongation and the sweep apart).
template <bool BG>
static bool can_fuse_prolong(const LevelSet<float> &F, const std::vector<int> *plan) {
  return !BG && F.tiled && plan && !plan->empty() && (*plan)[0] == 1 && F.rc_ty[0] > 0 &&
         F.rr_tiled && F.nblk_pl > 0;
}
static void launch_rc_prolong(frmg_ctx *ctx, LevelSet<float> &F, LevelSet<float> &C,
                              const int *active, int par, int cpar, cudaStream_t st) {
  const int ty = F.rc_ty[0];
  if (F.dirichlet) {
    if (ty == 8)
      launch_rc_k<false, true, 8, true>(F, active, par, st, C.d, cpar);
    else
      launch_rc_k<false, true, 16, true>(F, active, par, st, C.d, cpar);
  } else {
    if (ty == 8)
      launch_rc_k<false, false, 8, true>(F, active, par, st, C.d, cpar);
    else
      launch_rc_k<false, false, 16, true>(F, active, par, st, C.d, cpar);
  }
}

template <bool BG, bool DIR>
static void launch_rb_k(frmg_ctx *ctx, LevelSet<float> &s, const int *active, int par,
                        cudaStream_t st) {
  if (BG && s.rc_ty[1] == 8) return launch_rc_k<true, DIR, 8>(s, active, par, st);
  if (!BG && s.rc_ty[0] == 16) return launch_rc_k<false, DIR, 16>(s, active, par, st);
  if (!BG && s.rc_ty[0] == 8) return launch_rc_k<false, DIR, 8>(s, active, par, st);
  constexpr int TY = kRbTY;
  using RC = RBCfg<TY>;
  size_t sm = RC::smem(BG);
  static bool attr_set = false;
  if (!attr_set) {
    CK(cudaFuncSetAttribute(k_smooth_rb<BG, DIR, TY>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr_set = true;
  }
  constexpr int v = BG ? 1 : 0;
  k_smooth_rb<BG, DIR, TY><<<s.nblk_rb[v], RC::NT, sm, st>>>(s.d, s.d_off_rb[v], s.size(),
                                                              s.zc_rb[v], active, par);
}

template <bool BG, bool DIR>
static void launch_fas_rhs_tiled(frmg_ctx *ctx, LevelSet<float> &s, const int *active, int par,
                                 cudaStream_t st) {
  const size_t sm = fas_rhs_tiled_smem(BG);
  static bool attr_set = false;
  if (!attr_set) {
    CK(cudaFuncSetAttribute(k_fas_rhs_tiled<BG, DIR>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr_set = true;
  }
  constexpr int v = BG ? 1 : 0;
  k_fas_rhs_tiled<BG, DIR><<<s.nblk_fr[v], 256, sm, st>>>(s.d, s.d_off_fr[v], s.size(),
                                                         s.zc_fr[v], active, par);
}

template <bool BG, bool DIR>
static long long rb_slots() {
  static long long slots = 0;
  if (!slots) {
    using RC = RBCfg<kRbTY>;
    slots = (long long)sm_count() *
            resident_blocks(k_smooth_rb<BG, DIR, kRbTY>, RC::NT, RC::smem(BG));
  }
  return slots;
}

template <bool BG, bool DIR, int TY>
static long long rc_slots() {
  static long long slots = 0;
  if (!slots)
    slots = (long long)sm_count() *
            resident_blocks(k_smooth_rc<BG, DIR, TY>, RCCfg<TY, BG>::NT, RCCfg<TY, BG>::smem());
  return slots;
}

template <bool BG, bool DIR>
static long long fr_slots() {
  static long long slots = 0;
  if (!slots)
    slots = (long long)sm_count() *
            resident_blocks(k_fas_rhs_tiled<BG, DIR>, 256, fas_rhs_tiled_smem(BG));
  return slots;
}

template <bool DIR>
static long long pl_slots() {
  static long long slots = 0;
  if (!slots) slots = (long long)sm_count() * resident_blocks(k_prolong_tiled<DIR>, 256, 0);
  return slots;
}

template <bool DIR>
static long long rr_slots() {
  static long long slots = 0;
  if (!slots) {
    using RC = RRCfg<kTX, kTY>;
    slots = (long long)sm_count() *
            resident_blocks(k_resid_restrict_tiled<false, DIR, kTX, kTY>, RC::NT, RC::smem(false));
  }
  return slots;
}

template <bool BG, int S>
static void launch_tiled(frmg_ctx *ctx, LevelSet<float> &s, const int *active, int par,
                         cudaStream_t st) {
  if constexpr (S == 1) {
    if (s.dirichlet)
      launch_rb_k<BG, true>(ctx, s, active, par, st);
    else
      launch_rb_k<BG, false>(ctx, s, active, par, st);
  } else {
    if (s.dirichlet)
      launch_tiled_k<BG, true, S>(ctx, s, active, par, st);
    else
      launch_tiled_k<BG, false, S>(ctx, s, active, par, st);
  }
}

// Passes of the tiled smoother (sweeps per pass) for the pre- and post-smoothing
// of one V-cycle level.  Returns whether the total number of passes is even
// (the level's data is then back in its starting buffer at the end of the
// cycle).  An odd plan flips the depth's buffer parity once per cycle, which is
// consistent only for a single problem: in a batch, a grid that is not smoothed
// in a cycle (its coarsest level is this depth, or its field has left the
// inner solve) keeps its data in the buffer the parity has left.  A batch with
// an odd plan uses the in-place kernel instead.
static bool plan_passes(int pre, int post, int depth, std::vector<int> &a, std::vector<int> &b) {
  auto split = [depth](int n, std::vector<int> &v) {
    v.clear();
    while (n >= 2 && depth >= 2) {
      v.push_back(2);
      n -= 2;
    }
    while (n > 0) {
      v.push_back(1);
      n -= 1;
    }
  };
  split(pre, a);
  split(post, b);
  if ((a.size() + b.size()) % 2 == 0) return true;
  for (auto *v : {&b, &a}) {
    auto it = std::find(v->begin(), v->end(), 2);
    if (it != v->end()) {
      *it = 1;
      v->insert(it, 1);
      return true;
    }
  }
  return false;
}

template <typename T, bool BG>
static void smooth_set(frmg_ctx *ctx, LevelSet<T> &s, int sweeps, const std::vector<int> *plan,
                       const int *active, int &par, cudaStream_t st, bool fine = true) {
  if (s.empty() || sweeps <= 0) return;
  if constexpr (sizeof(T) == 4) {
    if (s.tiled && plan) {
      for (int S : *plan) {
        // the correction form is reported apart from the plain one (different kernel)
        PROF(BG ? (fine ? "smooth_bg_f32@fine" : "smooth_bg_f32@coarse") : pname("smooth", false, fine));
        if (S == 2)
          launch_tiled<BG, 2>(ctx, s, active, par, st);
        else
          launch_tiled<BG, 1>(ctx, s, active, par, st);
        CK_LAUNCH(ctx);
        par ^= 1;
      }
      return;
    }
  }
  for (int it = 0; it < sweeps; it++)
    for (int colour = 0; colour < 2; colour++) {
      PROF(pname("smooth", sizeof(T) == 8, fine));
      k_smooth<T, BG><<<s.nblk_half, 256, 0, st>>>(s.d, s.d_off_half, s.size(), colour, active,
                                                   par);
      CK_LAUNCH(ctx);
    }
}

// u^h += P (u^H - R u^h) from depth l + 1 onto depth l (tiled where the
// depth's sets have the tiled schedule).
template <typename T>
static void prolong_level(frmg_ctx *ctx, Hier<T> &H, int l, const int *active, cudaStream_t st) {
  auto &F = H.cont[l];
  auto &C = H.next[l];
  PROF(pname("prolong", sizeof(T) == 8, l == 0));
  bool done = false;
  if constexpr (sizeof(T) == 4) {
    if (F.rr_tiled && F.nblk_pl > 0) {
      if (F.dirichlet)
        k_prolong_tiled<true><<<F.nblk_pl, 256, 0, st>>>(F.d, C.d, F.d_off_pl, F.size(),
                                                         F.kc_pl, active, H.par[l], H.par[l + 1]);
      else
        k_prolong_tiled<false><<<F.nblk_pl, 256, 0, st>>>(F.d, C.d, F.d_off_pl, F.size(),
                                                          F.kc_pl, active, H.par[l], H.par[l + 1]);
      done = true;
    }
  }
  if (!done)
    k_prolong<T><<<C.nblk_full, 256, 0, st>>>(F.d, C.d, C.d_off_full, F.size(), active,
                                              H.par[l], H.par[l + 1]);
  CK_LAUNCH(ctx);
}

template <typename T, bool BG>
static void vcycle(frmg_ctx *ctx, Hier<T> &H, int l, const CycleOpts &o, const int *active,
                   cudaStream_t st) {
  if (!H.coarsest[l].empty()) {
    auto &c = H.coarsest[l];
    PROF(sizeof(T) == 8 ? "coarsest_f64" : "coarsest_f32");
    k_coarsest<T, BG, 256><<<c.size(), 256, 0, st>>>(c.d, c.size(), o.crs_rel, o.crs_abs,
                                                     o.crs_maxit, o.crs_stall, active, H.par[l],
                                                     o.crs_meanfix);
    CK_LAUNCH(ctx);
  }
  if (H.cont[l].empty()) return;
  auto &F = H.cont[l];
  auto &C = H.next[l];
  std::vector<int> plan_pre, plan_post;
  const bool tiled_ok = plan_passes(o.pre, o.post, o.tdepth, plan_pre, plan_post) ||
                        H.lev.size() == 1 || o.odd_ok;
  smooth_set<T, BG>(ctx, F, o.pre, tiled_ok ? &plan_pre : nullptr, active, H.par[l], st, l == 0);
  {
    PROF(pname("resid_restrict", sizeof(T) == 8, l == 0));
    if constexpr (sizeof(T) == 4) {
      if (F.rr_tiled) {
        launch_rr_tiled<BG>(ctx, F, C, active, H.par[l], H.par[l + 1],
                            l == 0 ? C.partial : nullptr, st);
      } else {
        k_resid_restrict<T, BG><<<C.nblk_full, 256, 0, st>>>(F.d, C.d, C.d_off_full, C.size(),
                                                             active, H.par[l], H.par[l + 1],
                                                             l == 0 ? C.partial : nullptr);
      }
    } else {
      k_resid_restrict<T, BG><<<C.nblk_full, 256, 0, st>>>(F.d, C.d, C.d_off_full, C.size(),
                                                           active, H.par[l], H.par[l + 1],
                                                           l == 0 ? C.partial : nullptr);
    }
    CK_LAUNCH(ctx);
  }
  {
    PROF(pname("fas_rhs", sizeof(T) == 8, false));
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (C.tiled && C.nblk_fr[BG ? 1 : 0] > 0) {
        if (C.dirichlet)
          launch_fas_rhs_tiled<BG, true>(ctx, C, active, H.par[l + 1], st);
        else
          launch_fas_rhs_tiled<BG, false>(ctx, C, active, H.par[l + 1], st);
        done = true;
      }
    }
    if (!done)
      k_fas_rhs<T, BG><<<C.nblk_full, 256, 0, st>>>(C.d, C.d_off_full, C.size(), active,
                                                    H.par[l + 1]);
    CK_LAUNCH(ctx);
  }
  vcycle<T, BG>(ctx, H, l + 1, o, active, st);
  if constexpr (sizeof(T) == 4 && !BG) {
    if (can_fuse_prolong<BG>(F, tiled_ok ? &plan_post : nullptr)) {
      // prolongation fused into the first post-smoothing sweep (reported as
      // its own kernel family)
      {
        PROF(l == 0 ? "smooth_prolong_f32@fine" : "smooth_prolong_f32@coarse");
        launch_rc_prolong(ctx, F, C, active, H.par[l], H.par[l + 1], st);
        CK_LAUNCH(ctx);
        H.par[l] ^= 1;
      }
      std::vector<int> rest(plan_post.begin() + 1, plan_post.end());
      int left = 0;
      for (int v : rest) left += v;
      smooth_set<T, BG>(ctx, F, left, &rest, active, H.par[l], st, l == 0);
      return;
    }
  }
  prolong_level<T>(ctx, H, l, active, st);
  smooth_set<T, BG>(ctx, F, o.post, tiled_ok ? &plan_post : nullptr, active, H.par[l], st,
                    l == 0);
}

// Full-multigrid start of the FP32 full-variable phase for a single field from
// u = 0 (the density term already in the finest right-hand side): the
// right-hand side is averaged down to every level, the coarsest level is
// solved, and at each finer level the coarser solution is interpolated (the
// V-cycle's trilinear prolongation applied to u^H with R u^h = 0 and u^h = 0)
// and one V-cycle is run from that level.  Ends with the V-cycle on the finest
// level.
static void fmg_start(frmg_ctx *ctx, Hier<float> &H, const CycleOpts &co, const int *active,
                      cudaStream_t st) {
  std::vector<Grid<float>> &lev = H.lev[0];
  const int L = (int)lev.size();
  for (int l = 1; l < L; l++) {
    Grid<float> &F = lev[l - 1];
    Grid<float> &C = lev[l];
    k_restrict_avg<float><<<nblocks(C.ncell), 256, 0, st>>>(F.f, F.n0, F.n1, F.n2,
                                                            const_cast<float *>(C.f));
    CK_LAUNCH(ctx);
    CK(cudaMemsetAsync(H.cur_u(0, l), 0, C.ncell * sizeof(float), st));
    CK(cudaMemsetAsync(H.cur_x(0, l), 0, C.ncell * sizeof(float), st));
  }
  vcycle<float, false>(ctx, H, L - 1, co, active, st);
  for (int l = L - 2; l >= 0; l--) {
    CK(cudaMemsetAsync(lev[l + 1].uR, 0, lev[l + 1].ncell * sizeof(float), st));
    CK(cudaMemsetAsync(H.cur_u(0, l), 0, lev[l].ncell * sizeof(float), st));
    CK(cudaMemsetAsync(H.cur_x(0, l), 0, lev[l].ncell * sizeof(float), st));
    prolong_level<float>(ctx, H, l, active, st);
    vcycle<float, false>(ctx, H, l, co, active, st);
  }
}

// Per-grid (sum, max) of per-block partials: one block per grid for short
// lists, two stages (chunks of kRedChunk partials, then the chunk sums) for
// the long lists of one-thread-per-cell kernels on fine grids.
static void reduce_partials(frmg_ctx *ctx, const double *partial, const int *d_off, int ng,
                            int nch, double *tmp, double *out, cudaStream_t st) {
  if (nch == 0) {
    k_reduce_partials<<<ng, 256, 0, st>>>(partial, d_off, ng, out);
    CK_LAUNCH(ctx);
    return;
  }
  k_reduce_partials_chunks<kRedChunk><<<dim3(nch, ng), 256, 0, st>>>(partial, d_off, nch, tmp);
  CK_LAUNCH(ctx);
  k_reduce_chunks<<<ng, 256, 0, st>>>(tmp, nch, ng, out);
  CK_LAUNCH(ctx);
}

// Residual norms of every grid of a level set: out[2g] = rms, out[2g+1] = max.
// dout (host array of ng device pointers, entries may be null) receives d.
template <typename T, bool BG>
static void level_norms(frmg_ctx *ctx, LevelSet<T> &s, T *const *dout, const int *active,
                        cudaStream_t st, std::vector<double> &out, int par = 0) {
  int ng = s.size();
  if (dout)
    CK(cudaMemcpyAsync(s.d_dout, dout, ng * sizeof(T *), cudaMemcpyHostToDevice, st));
  {
    PROF(pname("residual", sizeof(T) == 8, true));
    k_residual<T, BG, 256><<<s.nblk_full, 256, 0, st>>>(s.d, s.d_off_full, ng,
                                                        dout ? s.d_dout : nullptr, s.partial,
                                                        active, par);
    CK_LAUNCH(ctx);
  }
  reduce_partials(ctx, s.partial, s.d_off_full, ng, s.red_nch, s.red_tmp, s.red, st);
  double *hp = pinned_buf(ctx, 2 * (size_t)ng);
  CK(cudaMemcpyAsync(hp, s.red, 2 * ng * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  prof_harvest(ctx);
  out.assign(2 * ng, 0.0);
  for (int g = 0; g < ng; g++) {
    out[2 * g] = std::sqrt(hp[2 * g] / (double)s.h[g].ncell);
    out[2 * g + 1] = hp[2 * g + 1];
  }
}

// One V-cycle as a CUDA graph: the first call launches directly (it also sets
// kernel attributes), the second captures the launches on the stream and
// instantiates them, later calls replay.  A V-cycle issues the same kernels
// with the same arguments every time (the pass plan returns every level to
// its starting buffer; per-field active flags are read from device memory),
// so the replay is exact.  Not used on the legacy default stream (it cannot be
// captured) or while per-kernel profiling is on.
// Captured V-cycles, one executable graph per buffer-parity state of the
// hierarchy at the start of the cycle (a level smoothed by an odd number of
// ping-pong passes per cycle ends in its other buffer, so consecutive cycles
// alternate between two states).  A replay sets the host-side state to the
// one the captured cycle ended in.
struct CycleGraph {
  struct Entry {
    cudaGraphExec_t exec = nullptr;
    long long nlaunch = 0;
    int calls = 0;
    std::vector<int> after;
  };
  std::map<std::vector<int>, Entry> by_state;
  bool disabled = false;
  ~CycleGraph() {
    for (auto &kv : by_state)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  }
};

template <typename F>
static void run_cycle(frmg_ctx *ctx, CycleGraph &g, bool use, cudaStream_t st,
                      std::vector<int> &state, F &&launch) {
  if (!use || ctx->prof || g.disabled || st == nullptr) {
    launch();
    return;
  }
  CycleGraph::Entry &e = g.by_state[state];
  if (e.exec) {
    CK(cudaGraphLaunch(e.exec, st));
    ctx->launches += e.nlaunch;
    state = e.after;
    return;
  }
  if (e.calls++ == 0) {
    launch();
    return;
  }
  const std::vector<int> s0 = state;
  long long l0 = ctx->launches;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    g.disabled = true;
    launch();
    return;
  }
  try {
    launch();
  } catch (...) {
    cudaGraph_t gr;
    cudaStreamEndCapture(st, &gr);
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    state = s0;
    throw;
  }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamEndCapture(st, &graph));
  cudaError_t err = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (err != cudaSuccess) {
    // nothing captured ran: restore the state and run the cycle directly
    cudaGetLastError();
    e.exec = nullptr;
    g.disabled = true;
    state = s0;
    ctx->launches = l0;
    launch();
    return;
  }
  e.nlaunch = ctx->launches - l0;
  e.after = state;
  CK(cudaGraphLaunch(e.exec, st));
}

// Fine-grid residual norms accumulated by the last depth-0 residual+restriction
// (after pre-smoothing of the last V-cycle); out[p] = rms per problem (NaN for
// problems without a coarser level).
template <typename T>
static void fused_fine_norms(frmg_ctx *ctx, Hier<T> &H, int np, cudaStream_t st,
                             std::vector<double> &out) {
  out.assign(np, std::nan(""));
  LevelSet<T> &C = H.next[0];
  if (C.empty()) return;
  int ng = C.size();
  const int *offs = H.cont[0].rr_tiled ? H.cont[0].d_off_rr : C.d_off_full;
  k_reduce_partials<<<ng, 256, 0, st>>>(C.partial, offs, ng, C.red);
  CK_LAUNCH(ctx);
  double *hp = pinned_buf(ctx, 2 * (size_t)ng);
  CK(cudaMemcpyAsync(hp, C.red, 2 * ng * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  prof_harvest(ctx);
  for (int g = 0; g < ng; g++) {
    const Grid<T> &F = H.cont[0].h[g];
    out[F.field] = std::sqrt(hp[2 * g] / (double)F.ncell);
  }
}

// ---------------------------------------------------------------------------
// solve loops
struct SolveCfg {
  double tol;
  int max_vcycles, pre, post;
  double cap;
  int inner_cycles, max_outer;
  int fixed_cycles;  // > 0: exactly this many (FP64 only), no convergence test
  int tdepth;
  int tiling;
  int defect_fp64;   // mixed: 1 = native FP64 defect/update, 0 = double-float
  int use_graph;     // V-cycles replayed as CUDA graphs
  double tau_alpha;  // > 0: truncation-error stopping rule (Sec. V.B.2)
  double relax;      // relaxation factor of the Newton-GS updates
  int fmg;           // full-multigrid start (mixed, single field, u0 = 0)
  int stile;         // plain FP32 one-sweep smoother: 8/16 register-column tiles, -1 ring
};

static bool bad(double v) { return !(v == v) || std::isinf(v); }

static void hist_push(fr_stats &s, double v) {
  if (s.nhist < FR_HIST) s.hist[s.nhist++] = v;
}

// rms of the truncation-error estimate tau = A^H(R u) - R A^h(u) of every
// problem with a coarser level (NaN for the others), from the current fine
// u of the hierarchy's plain (full-variable) form.  Overwrites the first
// coarser level's u, x, uR and f (the next V-cycle restricts them again).
template <typename T>
static std::vector<double> tau_norms(frmg_ctx *ctx, Hier<T> &H, int np, cudaStream_t st) {
  std::vector<double> out(np, std::nan(""));
  if (H.cont.empty() || H.cont[0].empty()) return out;
  auto &F = H.cont[0];
  auto &C = H.next[0];
  k_resid_restrict<T, false><<<C.nblk_full, 256, 0, st>>>(F.d, C.d, C.d_off_full, C.size(),
                                                          nullptr, H.par[0], H.par[1], nullptr);
  CK_LAUNCH(ctx);
  k_tau<T><<<C.nblk_full, 256, 0, st>>>(F.d, C.d, C.d_off_full, C.size(), H.par[0], H.par[1],
                                        C.partial);
  CK_LAUNCH(ctx);
  reduce_partials(ctx, C.partial, C.d_off_full, C.size(), C.red_nch, C.red_tmp, C.red, st);
  const int ng = C.size();
  double *hp = pinned_buf(ctx, 2 * (size_t)ng);
  CK(cudaMemcpyAsync(hp, C.red, 2 * ng * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int g = 0; g < ng; g++) {
    const Grid<T> &G = C.h[g];
    out[G.field] = std::sqrt(hp[2 * g] / (double)G.ncell);
  }
  return out;
}

// Plain FP64: V-cycles until every problem has rms <= tol.
static void solve_fp64(frmg_ctx *ctx, std::vector<Problem> &P, const SolveCfg &cfg,
                       std::vector<fr_stats> &stats, cudaStream_t st) {
  Scope S(ctx);
  int np = (int)P.size();
  Hier<double> H;
  build_hier<double, false>(S, H, P, cfg.cap, st, ctx, 0, cfg.relax);
  for (int pi = 0; pi < np; pi++) {
    Grid<double> &G = H.lev[pi][0];
    k_expm1<double><<<nblocks(G.ncell), 256, 0, st>>>(G.u, G.x, G.ncell);
    CK_LAUNCH(ctx);
  }
  int *active = S.get<int>(np);
  std::vector<int> act(np, 1);
  CycleOpts co{cfg.pre, cfg.post, cfg.tdepth, 1e-3, 0.1 * cfg.tol, 500, 0, 0};
  std::vector<double> nr;
  level_norms<double, false>(ctx, H.all[0], nullptr, nullptr, st, nr);
  std::vector<double> prev(np);
  std::vector<int> grow(np, 0);
  for (int pi = 0; pi < np; pi++) {
    stats[pi].res0_rms = nr[2 * pi];
    stats[pi].res_rms = nr[2 * pi];
    stats[pi].res_max = nr[2 * pi + 1];
    stats[pi].vcycles = 0;
    stats[pi].tau_rms = std::nan("");
    prev[pi] = nr[2 * pi];
    if (cfg.fixed_cycles <= 0 && nr[2 * pi] <= cfg.tol) act[pi] = 0;
    if (bad(nr[2 * pi])) throw FrError{FR_EDIVERGED, "non-finite initial residual"};
  }
  int maxc = cfg.fixed_cycles > 0 ? cfg.fixed_cycles : cfg.max_vcycles;
  CycleGraph graph;
  for (int cyc = 0; cyc < maxc; cyc++) {
    int nact = 0;
    for (int v : act) nact += v;
    if (nact == 0) break;
    CK(cudaMemcpyAsync(active, act.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    run_cycle(ctx, graph, cfg.use_graph, st, H.par, [&]() { vcycle<double, false>(ctx, H, 0, co, active, st); });
    level_norms<double, false>(ctx, H.all[0], nullptr, nullptr, st, nr);
    std::vector<double> tau;
    if (cfg.tau_alpha > 0) tau = tau_norms<double>(ctx, H, np, st);
    for (int pi = 0; pi < np; pi++) {
      if (!act[pi]) continue;
      stats[pi].vcycles++;
      if (cfg.tau_alpha > 0) stats[pi].tau_rms = tau[pi];
      stats[pi].res_rms = nr[2 * pi];
      stats[pi].res_max = nr[2 * pi + 1];
      hist_push(stats[pi], nr[2 * pi]);
      if (bad(nr[2 * pi])) throw FrError{FR_EDIVERGED, "non-finite residual"};
      grow[pi] = nr[2 * pi] > prev[pi] ? grow[pi] + 1 : 0;
      if (grow[pi] >= 5) throw FrError{FR_EDIVERGED, "residual grew for 5 cycles"};
      prev[pi] = nr[2 * pi];
      // Sec. V.B.2: |d| <~ tau_alpha |tau| also ends the iteration
      const double lim = cfg.tau_alpha > 0 && tau[pi] == tau[pi]
                             ? std::max(cfg.tol, cfg.tau_alpha * tau[pi])
                             : cfg.tol;
      if (cfg.fixed_cycles <= 0 && nr[2 * pi] <= lim) act[pi] = 0;
    }
  }
}

// Mixed: FP64 defect / update / test around FP32 V-cycles.
// Zero initial guess: the first inner solve is a full-variable FP32 FAS solve
// (no FP64 defect needed, r = gamma (rho - 1)) run until its residual stops
// falling.  Every later inner solve is a correction solve in background mode
// on the FP32 background fp32(u), stopped once its residual is below a
// fraction of tol or stops falling.
static void solve_mixed(frmg_ctx *ctx, std::vector<Problem> &P, const SolveCfg &cfg,
                        std::vector<fr_stats> &stats, cudaStream_t st) {
  Scope S(ctx);
  int np = (int)P.size();
  Hier<double> H64;  // FP64 fine levels only (defect)
  std::vector<Problem> P1 = P;
  for (auto &p : P1) p.nl = 1;
  build_hier<double, false>(S, H64, P1, cfg.cap, st, ctx);
  Hier<float> H;
  build_hier<float, true>(S, H, P, cfg.cap, st, ctx, cfg.tiling, cfg.relax, cfg.stile);
  std::vector<double *> d64(np);
  int *flag = S.get<int>(1);
  CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
  for (int pi = 0; pi < np; pi++) {
    Grid<double> &G = H64.lev[pi][0];
    d64[pi] = S.get<double>(G.ncell);
    k_any_nonzero<<<nblocks(G.ncell), 256, 0, st>>>(G.u, G.ncell, flag);
    CK_LAUNCH(ctx);
  }
  int nonzero = 0;
  CK(cudaMemcpyAsync(&nonzero, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int *active = S.get<int>(np);
  std::vector<int> act(np, 1);
  CycleOpts co{cfg.pre, cfg.post, cfg.tdepth, 1e-3, 0.0, 500, 1, 1};
  // finest-level buffer parity of each field's FP32 data after an inner solve
  // (a field that left the solve early keeps the parity it left with)
  std::vector<int> fpar(np, 0);
  co.odd_ok = cfg.tau_alpha > 0 ? 0 : 1;  // tau reads every field at the shared parity
  auto fine_u = [&](int pi) { return fpar[pi] ? H.lev[pi][0].u2 : H.lev[pi][0].u; };
  std::vector<double> nr, inr;
  std::vector<double> prev(np, 0.0);
  std::vector<int> grow(np, 0);
  for (int pi = 0; pi < np; pi++) {
    stats[pi].vcycles = 0;
    stats[pi].outer = 0;
    stats[pi].tau_rms = std::nan("");
  }
  // truncation-error estimate of the full-variable FP32 phase (Sec. V.B.2);
  // with tau_alpha > 0, rms(d) <= tau_alpha rms(tau) also ends the solve
  std::vector<double> tau(np, std::nan(""));
  auto tol_of = [&](int pi) {
    stats[pi].tau_rms = tau[pi];
    return cfg.tau_alpha > 0 && tau[pi] == tau[pi] ? std::max(cfg.tol, cfg.tau_alpha * tau[pi])
                                                  : cfg.tol;
  };
  auto update = [&]() {
    for (int pi = 0; pi < np; pi++) {
      if (!act[pi]) continue;
      Grid<double> &G64 = H64.lev[pi][0];
      PROF("update64");
      k_update64<<<nblocks(G64.ncell), 256, 0, st>>>(G64.u, G64.x, fine_u(pi), G64.ncell);
      CK_LAUNCH(ctx);
    }
  };
  // inner V-cycles with the fused fine-residual norm as the stopping signal
  CycleGraph gr_bg, gr_plain;
  // Stopping signal: the fine residual after pre-smoothing of each cycle (fused
  // into the residual + restriction kernel).  Successive values are compared
  // (the first cycle always runs); a ratio above 0.75 means FP32 rounding has
  // taken over, or that the full-variable iteration is making little headway
  // in a strongly nonlinear field (continuing it there has run into overflow;
  // the correction form takes over instead).  The full-variable phase also
  // stops once the ratio exceeds three times the best ratio of the solve (the
  // FP32 floor is near: further cycles gain little).  A correction solve stops once
  // the residual at the end of the cycle, predicted as mid * sqrt(mid /
  // previous mid) (the rest of the cycle does about half of a cycle's
  // contraction), is below 0.7 tol.
  auto inner = [&](bool bg, const std::vector<double> &r0, double floor_rel, int kmax) {
    std::vector<double> rp(np, HUGE_VAL), rbest(np, HUGE_VAL);
    // fields leave the inner solve one by one (their active flag drops until
    // the next outer step), so a batch does not run every field as long as
    // its slowest one
    std::vector<int> iact = act;
    for (int k = 0; k < kmax; k++) {
      if (bg)
        run_cycle(ctx, gr_bg, cfg.use_graph, st, H.par,
                  [&]() { vcycle<float, true>(ctx, H, 0, co, active, st); });
      else
        run_cycle(ctx, gr_plain, cfg.use_graph, st, H.par,
                  [&]() { vcycle<float, false>(ctx, H, 0, co, active, st); });
      for (int pi = 0; pi < np; pi++)
        if (iact[pi]) fpar[pi] = H.par[0];  // this cycle moved the field's data
      bool go = false;
      for (int pi = 0; pi < np; pi++)
        if (iact[pi]) {
          stats[pi].vcycles++;
          if (stats[pi].vcycles >= cfg.max_vcycles) iact[pi] = 0;
          else go = true;
        }
      if (!go) break;
      fused_fine_norms(ctx, H, np, st, inr);
      go = false;
      for (int pi = 0; pi < np; pi++) {
        if (!iact[pi]) continue;
        double r = inr[pi];
        if (!(r == r)) { go = true; continue; }  // single-level grid: one coarsest solve per cycle
        hist_push(stats[pi], r);
        const double pred = rp[pi] < HUGE_VAL ? r * std::sqrt(r / rp[pi]) : r;
        const double ratio = rp[pi] < HUGE_VAL ? r / rp[pi] : 0.0;
        if (rp[pi] < HUGE_VAL) rbest[pi] = std::min(rbest[pi], ratio);
        if (ratio < 0.75 && (bg || ratio <= 3.0 * rbest[pi]) && r > floor_rel * r0[pi] &&
            pred > (bg ? 0.7 : 0.3) * cfg.tol)
          go = true;
        else
          iact[pi] = 0;
        rp[pi] = r;
      }
      if (!go) break;
      CK(cudaMemcpyAsync(active, iact.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(active, act.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
  };
  if (!nonzero) {
    // full-variable FP32 phase from u = 0
    for (int pi = 0; pi < np; pi++) {
      Grid<float> &G = H.lev[pi][0];
      Grid<double> &G64 = H64.lev[pi][0];
      PROF("prep_inner");
      LevelSet<double> &A0 = H64.all[0];
      k_prep_zero<<<nblocks(G.ncell), 256, 0, st>>>(G64.f, P[pi].k.gamma,
                                                    const_cast<float *>(G.f), H.cur_u(pi, 0),
                                                    H.cur_x(pi, 0), G.ncell, A0.partial,
                                                    A0.off_full[pi]);
      CK_LAUNCH(ctx);
    }
    CK(cudaMemcpyAsync(active, act.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    std::vector<double> r0(np, 0.0);
    {
      LevelSet<double> &A0 = H64.all[0];
      reduce_partials(ctx, A0.partial, A0.d_off_full, np, A0.red_nch, A0.red_tmp, A0.red, st);
      double *hp = pinned_buf(ctx, 2 * (size_t)np);
      CK(cudaMemcpyAsync(hp, A0.red, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int pi = 0; pi < np; pi++) {
        r0[pi] = std::sqrt(hp[2 * pi] / (double)A0.h[pi].ncell);
        stats[pi].res0_rms = r0[pi];
      }
    }
    if (cfg.fmg && np == 1) {
      fmg_start(ctx, H, co, active, st);
      stats[0].vcycles++;
    }
    // run to the FP32 rounding floor (1e-6 of the starting residual, or the
    // contraction stalls); the correction solves finish
    inner(false, r0, 1e-6, 40);
    if (cfg.tau_alpha > 0) tau = tau_norms<float>(ctx, H, np, st);
    update();
  } else {
    for (int pi = 0; pi < np; pi++) {
      Grid<double> &G = H64.lev[pi][0];
      k_expm1<double><<<nblocks(G.ncell), 256, 0, st>>>(G.u, G.x, G.ncell);
      CK_LAUNCH(ctx);
    }
  }
  for (int outer = 0; outer < cfg.max_outer; outer++) {
    // FP64 defect and convergence test
    CK(cudaMemcpyAsync(active, act.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    level_norms<double, false>(ctx, H64.all[0], d64.data(), active, st, nr);
    int nact = 0;
    for (int pi = 0; pi < np; pi++) {
      if (!act[pi]) continue;
      stats[pi].outer++;
      if (outer == 0 && nonzero) stats[pi].res0_rms = nr[2 * pi];
      stats[pi].res_rms = nr[2 * pi];
      stats[pi].res_max = nr[2 * pi + 1];
      if (bad(nr[2 * pi])) throw FrError{FR_EDIVERGED, "non-finite residual"};
      if (outer > 0) {
        grow[pi] = nr[2 * pi] > prev[pi] ? grow[pi] + 1 : 0;
        if (grow[pi] >= 3) throw FrError{FR_EDIVERGED, "FP64 defect grew for 3 outer steps"};
      }
      prev[pi] = nr[2 * pi];
      if (nr[2 * pi] <= tol_of(pi) || stats[pi].vcycles >= cfg.max_vcycles)
        act[pi] = 0;
      else
        nact++;
    }
    if (nact == 0) return;
    CK(cudaMemcpyAsync(active, act.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    // correction problem: rhs -d, background fp32(u) on every level, delta = 0
    std::vector<double> r0(np, 0.0);
    for (int pi = 0; pi < np; pi++) {
      if (!act[pi]) continue;
      r0[pi] = nr[2 * pi];
      Grid<float> &G = H.lev[pi][0];
      Grid<double> &G64 = H64.lev[pi][0];
      {
        PROF("prep_inner");
        k_prep_inner<<<nblocks(G.ncell), 256, 0, st>>>(d64[pi], G64.u, const_cast<float *>(G.f),
                                                       H.bg_u[pi], H.bg_E[pi], H.cur_u(pi, 0),
                                                       H.cur_x(pi, 0), G.ncell);
        CK_LAUNCH(ctx);
      }
      for (size_t l = 1; l < H.lev[pi].size(); l++) {
        Grid<float> &F = H.lev[pi][l - 1];
        Grid<float> &C = H.lev[pi][l];
        k_restrict_avg<float><<<nblocks(C.ncell), 256, 0, st>>>(F.ubg, F.n0, F.n1, F.n2,
                                                                const_cast<float *>(C.ubg));
        CK_LAUNCH(ctx);
        k_expf<<<nblocks(C.ncell), 256, 0, st>>>(C.ubg, const_cast<float *>(C.Ebg), C.ncell);
        CK_LAUNCH(ctx);
      }
    }
    inner(true, r0, 1e-6, std::max(cfg.inner_cycles, 12));
    update();
  }
}

// Zero-start set-up of the double-float loop: the FP32 right-hand side is the
// high part of gamma (rho - 1); block partials of its norm as k_prep_zero.
__global__ void __launch_bounds__(256) k_prep_zero_df(const float2 *rv, float *r32, float *u32,
                                                      float *x32, long long n, double *partial,
                                                      int base) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float s = 0.0f, m = 0.0f;
  if (t < n) {
    float r = rv[t].x;
    r32[t] = r;
    u32[t] = 0.0f;
    x32[t] = 0.0f;
    s = r * r;
    m = fabsf(r);
  }
  block_reduce2f<256>(s, m, &partial[2 * (base + blockIdx.x)], &partial[2 * (base + blockIdx.x) + 1]);
}

// Zero start of the double-float state and of the FP32 full-variable phase in
// one pass: u = 0, e^u = 1, r = gamma (rho - 1) as a pair; the FP32 right-hand
// side r32 = hi(r), u32 = x32 = 0; per-block partials of r32 (its norm is the
// residual of u = 0).  Equals k_df_init with zero_u followed by k_prep_zero_df.
// check_rho > 0: also the density validation of k_check_density (negative
// values allowed if 2), flagged in *bad.
__global__ void __launch_bounds__(256) k_df_init_zero(DFGrid G, const double *rho, float *r32,
                                                      float *u32, float *x32, double *partial,
                                                      int base, int check_rho, int *bad) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float s = 0.0f, m = 0.0f;
  if (t < G.ncell) {
    if (check_rho > 0) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(rho[t]);
      const bool nonfinite = ((b >> 52) & 0x7ffu) == 0x7ffu;
      const bool negative = (b >> 63) && (b << 1) != 0;
      if (nonfinite || (check_rho == 1 && negative)) atomicExch(bad, 1);
    }
    G.u[t] = make_float2(0.f, 0.f);
    G.B[t] = make_float2(1.f, 0.f);
    const df r = df_mul(df_add_f(split_bits(rho[t]), -1.0f), df{G.gah, G.gal});
    G.r[t] = make_float2(r.h, r.l);
    r32[t] = r.h;
    u32[t] = 0.0f;
    x32[t] = 0.0f;
    s = r.h * r.h;
    m = fabsf(r.h);
  }
  block_reduce2f<256>(s, m, &partial[2 * (base + blockIdx.x)], &partial[2 * (base + blockIdx.x) + 1]);
}

static void split_host(double v, float &h, float &l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

// Sizes and constants of a double-float fine-grid state (arrays set by the caller).
static void dfgrid_setup(DFGrid &g, const int n[3], const Consts &k, const double *bnd) {
  memset(&g, 0, sizeof(g));
  g.n0 = n[0];
  g.n1 = n[1];
  g.n2 = n[2];
  g.ncell = (long long)g.n0 * g.n1 * g.n2;
  g.fdh = make_fastdiv((unsigned)std::max(1, g.n0 / 2));
  g.fd1 = make_fastdiv((unsigned)g.n1);
  g.bnd = bnd;
  face_offsets(n, g.foff);
  split_host(0.5 * k.alpha, g.ahh, g.ahl);
  split_host(k.beta, g.beh, g.bel);
  split_host(k.gamma, g.gah, g.gal);
}

// Defect kernel for one grid (two cells per thread): 32-bit index
// decomposition below 2^31 cells.  Its blocks cover 256 cells each.
static void launch_df_defect(frmg_ctx *ctx, const DFGrid &g, float *r32, float *ub32, float *E32,
                             float *delta, float *x32, double *partial, int base, float ln2h,
                             float ln2l, double *dout, cudaStream_t st) {
  if (g.ncell < (1ll << 31))
    k_df_defect<false><<<nblocks(g.ncell), 128, 0, st>>>(g, r32, ub32, E32, delta, x32, partial,
                                                         base, ln2h, ln2l, dout);
  else
    k_df_defect<true><<<nblocks(g.ncell), 128, 0, st>>>(g, r32, ub32, E32, delta, x32, partial,
                                                        base, ln2h, ln2l, dout);
  CK_LAUNCH(ctx);
}

// Mixed precision with the FP64-accurate quantities in double-float (see
// frmg_df.cuh): the same outer loop as solve_mixed, with the defect, the
// update and the convergence test evaluated on FP32 pipes at ~48-bit accuracy.
static void solve_mixed_df(frmg_ctx *ctx, std::vector<Problem> &P, const SolveCfg &cfg,
                           std::vector<fr_stats> &stats, cudaStream_t st) {
  Scope S(ctx);
  const int np = (int)P.size();
  Hier<float> H;
  build_hier<float, true>(S, H, P, cfg.cap, st, ctx, cfg.tiling, cfg.relax, cfg.stile);
  const double ln2 = std::log(2.0);
  float ln2h, ln2l;
  split_host(ln2, ln2h, ln2l);
  std::vector<DFGrid> D(np);
  std::vector<int> boff(np + 1, 0);
  for (int pi = 0; pi < np; pi++) {
    DFGrid &g = D[pi];
    dfgrid_setup(g, P[pi].n, P[pi].k, P[pi].bnd);
    g.u = S.get<float2>(g.ncell);
    g.B = S.get<float2>(g.ncell);
    g.r = S.get<float2>(g.ncell);
    boff[pi + 1] = boff[pi] + nblocks(g.ncell);
  }
  double *partial = S.get<double>(2 * (size_t)boff[np]);
  double *red = S.get<double>(2 * (size_t)np);
  int *d_boff = S.get<int>(np + 1);
  CK(cudaMemcpyAsync(d_boff, boff.data(), (np + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  // a zero start that the caller declared (initial_guess = 0) reads no u and
  // sets the state up in one fused pass below; otherwise u is scanned for a
  // non-zero value
  bool zero_start = true;
  for (auto &p : P) zero_start = zero_start && p.zero_u;
  int *rho_bad = S.get<int>(1);
  CK(cudaMemsetAsync(rho_bad, 0, sizeof(int), st));
  int nonzero = 0;
  if (!zero_start) {
    int *flag = S.get<int>(1);
    CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
    for (int pi = 0; pi < np; pi++) {
      k_any_nonzero<<<nblocks(D[pi].ncell), 256, 0, st>>>(P[pi].u, D[pi].ncell, flag);
      CK_LAUNCH(ctx);
    }
    CK(cudaMemcpyAsync(&nonzero, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int pi = 0; pi < np; pi++) {
      PROF("df_init");
      k_df_init<<<nblocks(D[pi].ncell), 256, 0, st>>>(D[pi], P[pi].u, P[pi].rho, !nonzero, ln2h,
                                                      ln2l);
      CK_LAUNCH(ctx);
    }
  }
  const int bnch = red_chunks(boff);
  double *btmp = bnch ? S.get<double>(2 * (size_t)bnch * np) : nullptr;
  // the norms reach the host through a kernel that writes them into the
  // page-locked buffer (its device mapping), so that an early copy of the
  // result (below) does not hold them up
  auto read_norms = [&](std::vector<double> &out) {
    reduce_partials(ctx, partial, d_boff, np, bnch, btmp, red, st);
    double *hp = pinned_buf(ctx, 2 * (size_t)np);
    double *hpd = nullptr;
    if (cudaHostGetDevicePointer((void **)&hpd, hp, 0) == cudaSuccess && hpd) {
      k_copy_to_host<<<1, 256, 0, st>>>(red, hpd, 2 * np);
      CK_LAUNCH(ctx);
    } else {
      cudaGetLastError();
      CK(cudaMemcpyAsync(hp, red, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    prof_harvest(ctx);
    out.assign(2 * np, 0.0);
    for (int pi = 0; pi < np; pi++) {
      out[2 * pi] = std::sqrt(hp[2 * pi] / (double)D[pi].ncell);
      out[2 * pi + 1] = hp[2 * pi + 1];
    }
  };
  auto finalize = [&]() {
    for (int pi = 0; pi < np; pi++) {
      k_df_final<<<nblocks(D[pi].ncell), 256, 0, st>>>(D[pi], P[pi].u);
      CK_LAUNCH(ctx);
    }
  };
  int *active = S.get<int>(np);
  std::vector<int> act(np, 1);
  CycleOpts co{cfg.pre, cfg.post, cfg.tdepth, 1e-3, 0.0, 500, 1, 1};
  // finest-level buffer parity of each field's FP32 data after an inner solve
  // (a field that left the solve early keeps the parity it left with)
  std::vector<int> fpar(np, 0);
  co.odd_ok = cfg.tau_alpha > 0 ? 0 : 1;  // tau reads every field at the shared parity
  auto fine_u = [&](int pi) { return fpar[pi] ? H.lev[pi][0].u2 : H.lev[pi][0].u; };
  std::vector<double> nr, inr;
  std::vector<double> prev(np, 0.0);
  std::vector<int> grow(np, 0);
  for (int pi = 0; pi < np; pi++) {
    stats[pi].vcycles = 0;
    stats[pi].outer = 0;
    stats[pi].tau_rms = std::nan("");
  }
  // truncation-error estimate of the full-variable FP32 phase (Sec. V.B.2);
  // with tau_alpha > 0, rms(d) <= tau_alpha rms(tau) also ends the solve
  std::vector<double> tau(np, std::nan(""));
  auto tol_of = [&](int pi) {
    stats[pi].tau_rms = tau[pi];
    return cfg.tau_alpha > 0 && tau[pi] == tau[pi] ? std::max(cfg.tol, cfg.tau_alpha * tau[pi])
                                                  : cfg.tol;
  };
  auto update = [&]() {
    for (int pi = 0; pi < np; pi++) {
      if (!act[pi]) continue;
      PROF("df_update");
      k_df_update<<<nblocks(D[pi].ncell), 128, 0, st>>>(D[pi], fine_u(pi), ln2h, ln2l);
      CK_LAUNCH(ctx);
    }
  };
  CycleGraph gr_bg, gr_plain;
  // Stopping signal: the fine residual after pre-smoothing of each cycle (fused
  // into the residual + restriction kernel).  Successive values are compared
  // (the first cycle always runs); a ratio above 0.75 means FP32 rounding has
  // taken over, or that the full-variable iteration is making little headway
  // in a strongly nonlinear field (continuing it there has run into overflow;
  // the correction form takes over instead).  The full-variable phase also
  // stops once the ratio exceeds three times the best ratio of the solve (the
  // FP32 floor is near: further cycles gain little).  A correction solve stops once
  // the residual at the end of the cycle, predicted as mid * sqrt(mid /
  // previous mid) (the rest of the cycle does about half of a cycle's
  // contraction), is below 0.7 tol.
  // returns whether every field that took part stopped because its predicted
  // end-of-cycle residual fell below the tolerance (the outer step is then
  // likely the last)
  auto inner = [&](bool bg, const std::vector<double> &r0, double floor_rel, int kmax) {
    std::vector<double> rp(np, HUGE_VAL), rbest(np, HUGE_VAL);
    std::vector<int> by_pred(np, 0);
    // fields leave the inner solve one by one (their active flag drops until
    // the next outer step), so a batch does not run every field as long as
    // its slowest one
    std::vector<int> iact = act;
    for (int k = 0; k < kmax; k++) {
      if (bg)
        run_cycle(ctx, gr_bg, cfg.use_graph, st, H.par,
                  [&]() { vcycle<float, true>(ctx, H, 0, co, active, st); });
      else
        run_cycle(ctx, gr_plain, cfg.use_graph, st, H.par,
                  [&]() { vcycle<float, false>(ctx, H, 0, co, active, st); });
      for (int pi = 0; pi < np; pi++)
        if (iact[pi]) fpar[pi] = H.par[0];  // this cycle moved the field's data
      bool go = false;
      for (int pi = 0; pi < np; pi++)
        if (iact[pi]) {
          stats[pi].vcycles++;
          if (stats[pi].vcycles >= cfg.max_vcycles) iact[pi] = 0;
          else go = true;
        }
      if (!go) break;
      fused_fine_norms(ctx, H, np, st, inr);
      go = false;
      for (int pi = 0; pi < np; pi++) {
        if (!iact[pi]) continue;
        double r = inr[pi];
        if (!(r == r)) { go = true; continue; }
        hist_push(stats[pi], r);
        const double pred = rp[pi] < HUGE_VAL ? r * std::sqrt(r / rp[pi]) : r;
        const double ratio = rp[pi] < HUGE_VAL ? r / rp[pi] : 0.0;
        if (rp[pi] < HUGE_VAL) rbest[pi] = std::min(rbest[pi], ratio);
        const bool moving = ratio < 0.75 && (bg || ratio <= 3.0 * rbest[pi]) &&
                            r > floor_rel * r0[pi];
        if (moving && pred > (bg ? 0.7 : 0.3) * cfg.tol) {
          go = true;
        } else {
          iact[pi] = 0;
          by_pred[pi] = moving;
        }
        rp[pi] = r;
      }
      if (!go) break;
      CK(cudaMemcpyAsync(active, iact.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(active, act.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    bool all = true;
    for (int pi = 0; pi < np; pi++)
      if (act[pi] && !by_pred[pi]) all = false;
    return all;
  };
  // Early result copy (one field whose u is page-locked host memory): when an
  // outer step's correction solve predicts convergence, the result is formed
  // and its device-to-host copy started on the context's copy stream before
  // the FP64-accurate defect confirms it, so the copy overlaps that check; a
  // later update makes the copy stale and the result is formed and copied
  // again at the end.
  bool early = false, stale = false;
  auto early_copy = [&]() {
    if (!ctx->copy) {
      CK(cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&ctx->copy_in, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->copy_out, cudaEventDisableTiming));
    }
    if (early) CK(cudaStreamWaitEvent(st, ctx->copy_out, 0));  // the last copy has read u
    finalize();
    CK(cudaEventRecord(ctx->copy_in, st));
    CK(cudaStreamWaitEvent(ctx->copy, ctx->copy_in, 0));
    CK(cudaMemcpyAsync(P[0].host_u, P[0].u, (size_t)D[0].ncell * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->copy));
    CK(cudaEventRecord(ctx->copy_out, ctx->copy));
    stats[0].host_copies++;
    early = true;
    stale = false;
  };
  try {
    CK(cudaMemcpyAsync(active, act.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    if (!nonzero) {
      for (int pi = 0; pi < np; pi++) {
        Grid<float> &G = H.lev[pi][0];
        PROF("prep_inner");
        if (zero_start)
          k_df_init_zero<<<nblocks(G.ncell), 256, 0, st>>>(D[pi], P[pi].rho,
                                                           const_cast<float *>(G.f),
                                                           H.cur_u(pi, 0), H.cur_x(pi, 0),
                                                           partial, boff[pi], P[pi].check_rho,
                                                           rho_bad);
        else
          k_prep_zero_df<<<nblocks(G.ncell), 256, 0, st>>>(D[pi].r, const_cast<float *>(G.f),
                                                           H.cur_u(pi, 0), H.cur_x(pi, 0),
                                                           G.ncell, partial, boff[pi]);
        CK_LAUNCH(ctx);
      }
      read_norms(nr);
      if (zero_start) {
        int hb = 0;
        CK(cudaMemcpyAsync(&hb, rho_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (hb) throw FrError{FR_EINVAL, "density has NaN/Inf or negative values"};
      }
      std::vector<double> r0(np);
      for (int pi = 0; pi < np; pi++) {
        r0[pi] = nr[2 * pi];
        stats[pi].res0_rms = nr[2 * pi];
      }
      if (cfg.fmg && np == 1) {
        fmg_start(ctx, H, co, active, st);
        stats[0].vcycles++;
      }
      // run to the FP32 rounding floor (1e-6 of the starting residual, or the
      // contraction stalls); the correction solves finish
      inner(false, r0, 1e-6, 40);
      if (cfg.tau_alpha > 0) tau = tau_norms<float>(ctx, H, np, st);
      update();
    }
    for (int outer = 0; outer < cfg.max_outer; outer++) {
      CK(cudaMemcpyAsync(active, act.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
      for (int pi = 0; pi < np; pi++) {
        if (!act[pi]) continue;
        Grid<float> &G = H.lev[pi][0];
        PROF("df_defect");
        launch_df_defect(ctx, D[pi], const_cast<float *>(G.f), H.bg_u[pi], H.bg_E[pi],
                         H.cur_u(pi, 0), H.cur_x(pi, 0), partial, boff[pi], ln2h, ln2l, nullptr,
                         st);
      }
      read_norms(nr);
      int nact = 0;
      for (int pi = 0; pi < np; pi++) {
        if (!act[pi]) continue;
        stats[pi].outer++;
        if (outer == 0 && nonzero) stats[pi].res0_rms = nr[2 * pi];
        stats[pi].res_rms = nr[2 * pi];
        stats[pi].res_max = nr[2 * pi + 1];
        hist_push(stats[pi], -nr[2 * pi]);
        if (bad(nr[2 * pi])) throw FrError{FR_EDIVERGED, "non-finite residual"};
        if (outer > 0) {
          grow[pi] = nr[2 * pi] > prev[pi] ? grow[pi] + 1 : 0;
          if (grow[pi] >= 3) throw FrError{FR_EDIVERGED, "defect grew for 3 outer steps"};
        }
        prev[pi] = nr[2 * pi];
        if (nr[2 * pi] <= tol_of(pi) || stats[pi].vcycles >= cfg.max_vcycles)
          act[pi] = 0;
        else
          nact++;
      }
      if (nact == 0) break;
      CK(cudaMemcpyAsync(active, act.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
      std::vector<double> r0(np, 0.0);
      for (int pi = 0; pi < np; pi++) {
        if (!act[pi]) continue;
        r0[pi] = nr[2 * pi];
        for (size_t l = 1; l < H.lev[pi].size(); l++) {
          Grid<float> &F = H.lev[pi][l - 1];
          Grid<float> &C = H.lev[pi][l];
          k_restrict_avg<float><<<nblocks(C.ncell), 256, 0, st>>>(F.ubg, F.n0, F.n1, F.n2,
                                                                  const_cast<float *>(C.ubg));
          CK_LAUNCH(ctx);
          k_expf<<<nblocks(C.ncell), 256, 0, st>>>(C.ubg, const_cast<float *>(C.Ebg), C.ncell);
          CK_LAUNCH(ctx);
        }
      }
      const bool likely_last = inner(true, r0, 1e-6, std::max(cfg.inner_cycles, 12));
      update();
      stale = true;
      if (likely_last && np == 1 && P[0].host_u) early_copy();
    }
  } catch (...) {
    if (early) cudaStreamWaitEvent(st, ctx->copy_out, 0);
    finalize();
    cudaStreamSynchronize(st);
    throw;
  }
  if (early) CK(cudaStreamWaitEvent(st, ctx->copy_out, 0));
  if (early && !stale)
    P[0].early_copied = 1;  // u was formed after the last update and is on the host
  else
    finalize();
}

// ---------------------------------------------------------------------------
// host/device staging
static bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// page-locked (or registered) host memory: a device-to-host copy into it runs
// asynchronously
static bool is_pinned_host(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

// Device address of page-locked host memory, read by a kernel across the
// host link (null if p is not page-locked host memory).
static const double *mapped_host(const double *p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  return static_cast<const double *>(at.devicePointer);
}

struct Staged {
  void *dev = nullptr;
  const void *host_src = nullptr;
  void *host_dst = nullptr;
  size_t bytes = 0;
};

// Returns a device view of p; host memory is copied in (and back if `out`).
template <typename T>
static T *stage(Scope &S, std::vector<Staged> &back, const T *p, size_t n, bool in, bool out,
                cudaStream_t st) {
  if (!p) return nullptr;
  if (is_device_ptr(p)) return const_cast<T *>(p);
  T *d = S.get<T>(n);
  if (in) CK(cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, st));
  if (out) back.push_back({d, p, const_cast<T *>(p), n * sizeof(T)});
  return d;
}

static void unstage(std::vector<Staged> &back, cudaStream_t st) {
  for (auto &s : back) CK(cudaMemcpyAsync(s.host_dst, s.dev, s.bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

static void finish(frmg_ctx *ctx, std::vector<Staged> &back, cudaStream_t st) {
  unstage(back, st);
  prof_harvest(ctx);
}

// density validation (NaN always rejected; negative unless allowed)
// (bit tests: exponent all ones = Inf/NaN; sign set on a non-zero = negative)
__global__ void k_check_density(const double *rho, long long n, int allow_neg, int *bad) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const unsigned long long b = (unsigned long long)__double_as_longlong(rho[t]);
  const bool nonfinite = ((b >> 52) & 0x7ffu) == 0x7ffu;
  const bool negative = (b >> 63) && (b << 1) != 0;
  if (nonfinite || (!allow_neg && negative)) atomicExch(bad, 1);
}

static void validate_density(frmg_ctx *ctx, Scope &S, const double *rho, long long n,
                             int allow_neg, cudaStream_t st) {
  int *bad = S.get<int>(1);
  CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_check_density<<<nblocks(n), 256, 0, st>>>(rho, n, allow_neg, bad);
  CK_LAUNCH(ctx);
  int hb = 0;
  CK(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hb) einval("density has NaN/Inf or negative values");
}

static fr_opts resolve_opts(const fr_opts *o) {
  fr_opts r;
  fr_opts_default(&r);
  if (o) r = *o;
  return r;
}

// u of a solve: staged (host pointers) and, unless opts->initial_guess is set,
// zeroed on the device instead of read (nothing is copied in for a host u)
static double *stage_u(Scope &S, std::vector<Staged> &back, double *u, size_t n,
                       const fr_opts &o, cudaStream_t st) {
  double *d = stage(S, back, u, n, o.initial_guess != 0, true, st);
  // the double-float mixed solve of a zero start never reads u (its result
  // overwrites all of u); the other solves iterate on u itself
  const bool unread = o.prec == FR_MIXED && o.defect_precision == 0;
  if (!o.initial_guess && !unread) CK(cudaMemsetAsync(d, 0, n * sizeof(double), st));
  return d;
}

// A solve issued on the legacy default stream runs on a stream of the context
// instead, because the legacy stream cannot be captured into a graph: the side
// stream waits for the caller's earlier work and the caller's stream waits for
// the solve, so the ordering seen by the caller is unchanged.
struct SideStream {
  frmg_ctx *ctx;
  cudaStream_t caller, st;
  SideStream(frmg_ctx *c, cudaStream_t s, bool want) : ctx(c), caller(s), st(s) {
    if (s != nullptr || !want || c->prof) return;
    if (!c->side) {
      CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&c->side_in, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&c->side_out, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(c->side_in, s));
    CK(cudaStreamWaitEvent(c->side, c->side_in, 0));
    st = c->side;
  }
  ~SideStream() {
    if (st == caller) return;
    cudaEventRecord(ctx->side_out, st);
    cudaStreamWaitEvent(caller, ctx->side_out, 0);
  }
};

static void run_problems(frmg_ctx *ctx, std::vector<Problem> &P, const fr_opts &o, double tol,
                         std::vector<fr_stats> &stats, cudaStream_t st_caller, int fixed = 0) {
  SideStream side(ctx, st_caller, o.use_graph != 0);
  cudaStream_t st = side.st;
  SolveCfg cfg{tol, o.max_vcycles, o.pre, o.post, o.newton_step_cap, o.inner_cycles,
               o.max_outer, fixed, o.temporal_depth <= 0 ? 1 : o.temporal_depth, o.tiling,
               o.defect_precision, o.use_graph, o.tau_alpha, o.relax, o.fmg,
               o.smooth_tile == 0 ? kDefaultSmoothTile : o.smooth_tile};
  if (o.defect_precision < 0 || o.defect_precision > 1) einval("defect_precision must be 0 or 1");
  if (!(o.smooth_tile == 0 || o.smooth_tile == -1 || o.smooth_tile == 8 || o.smooth_tile == 16))
    einval("smooth_tile must be 0, -1, 8 or 16");
  if (cfg.tdepth > 2) einval("temporal_depth must be 0, 1 or 2");
  if (o.pre < 0 || o.post < 0 || o.max_vcycles < 0 || !(o.newton_step_cap > 0) ||
      !(tol >= 0) || o.inner_cycles < 1 || o.max_outer < 1)
    einval("invalid options");
  if (!(o.tau_alpha >= 0)) einval("tau_alpha must be >= 0");
  if (!(o.relax > 0 && o.relax < 2)) einval("relax must be in (0, 2)");
  if (o.fmg < 0 || o.fmg > 1) einval("fmg must be 0 or 1");
  if (o.initial_guess < 0 || o.initial_guess > 1) einval("initial_guess must be 0 or 1");
  for (auto &p : P) {
    p.nl = count_levels(p.n);
    p.k = model_consts(p.box, p.h, p.a, p.om, p.fr0);
  }
  if (o.prec == FR_MIXED && fixed <= 0) {
    if (cfg.defect_fp64)
      solve_mixed(ctx, P, cfg, stats, st);
    else
      solve_mixed_df(ctx, P, cfg, stats, st);
  }
  else
    solve_fp64(ctx, P, cfg, stats, st);
}

// FR_OK when every grid reached tol, or (tau_alpha > 0) tau_alpha times the
// rms of its truncation-error estimate (Sec. V.B.2).
static int status_from_stats(const std::vector<fr_stats> &stats, double tol,
                             double tau_alpha = 0.0) {
  for (auto &s : stats) {
    const double lim = tau_alpha > 0 && s.tau_rms == s.tau_rms
                           ? std::max(tol, tau_alpha * s.tau_rms)
                           : tol;
    if (!(s.res_rms <= lim)) return FR_ENOCONV;
  }
  return FR_OK;
}

template <typename F>
static int guard(F &&f) {
  try {
    return f();
  } catch (FrError &e) {
    g_last_error = e.msg;
    return e.status;
  } catch (std::exception &e) {
    g_last_error = e.what();
    return FR_ENOMEM;
  }
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// ---------------------------------------------------------------------------
// patch boundary set-up kernel (Sec. V.A.1, V.B.1, VI.B): trilinear value of
// the parent at a fine cell g (relative to the patch corner; may be -1 or n
// for ghosts).  Returns false if the stencil leaves a non-periodic parent.
__device__ bool parent_interp(const double *up, int p0, int p1, int p2, int periodic,
                              const int org[3], const int g[3], double *val) {
  const int np_[3] = {p0, p1, p2};
  int par[3], oth[3];
  for (int d = 0; d < 3; d++) {
    int fg = 2 * org[d] + g[d];
    int pc = fg >= 0 ? fg / 2 : -((-fg + 1) / 2);
    par[d] = pc;
    oth[d] = pc + ((fg - 2 * pc == 0) ? -1 : 1);
  }
  double s = 0.0;
  for (int sel = 0; sel < 8; sel++) {
    int cc[3];
    double w = 1.0;
    for (int d = 0; d < 3; d++) {
      int o = (sel >> d) & 1;
      cc[d] = o ? oth[d] : par[d];
      w *= o ? 1.0 : 3.0;
      if (cc[d] < 0 || cc[d] >= np_[d]) {
        if (!periodic) return false;
        cc[d] = ((cc[d] % np_[d]) + np_[d]) % np_[d];
      }
    }
    s += (w / 64.0) * up[((long long)cc[2] * p1 + cc[1]) * p0 + cc[0]];
  }
  *val = s;
  return true;
}

__global__ void k_patch_init(const double *up, int p0, int p1, int p2, int periodic, int o0, int o1,
                             int o2, int n0, int n1, int n2, double *u_init, int *bad) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n0 * n1 * n2) return;
  int g[3] = {(int)(t % n0), (int)((t / n0) % n1), (int)(t / ((long long)n0 * n1))};
  int org[3] = {o0, o1, o2};
  double v = 0.0;
  if (!parent_interp(up, p0, p1, p2, periodic, org, g, &v)) atomicExch(bad, 1);
  u_init[t] = v;
}

__global__ void k_patch_faces(const double *up, int p0, int p1, int p2, int periodic, int o0,
                              int o1, int o2, int n0, int n1, int n2, const double *u_init,
                              double *ub, int *bad) {
  const int n[3] = {n0, n1, n2};
  long long tot = 2LL * n1 * n2 + 2LL * n0 * n2 + 2LL * n0 * n1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  long long off = 0;
  int org[3] = {o0, o1, o2};
  for (int f = 0; f < 6; f++) {
    int ax = f / 2;
    int p = ax == 0 ? 1 : 0, q = ax == 2 ? 1 : 2;
    long long sz = (long long)n[p] * n[q];
    if (t < off + sz) {
      long long r = t - off;
      int P = (int)(r % n[p]), Q = (int)(r / n[p]);
      int inner[3], ghost[3];
      inner[p] = ghost[p] = P;
      inner[q] = ghost[q] = Q;
      inner[ax] = (f & 1) ? n[ax] - 1 : 0;
      ghost[ax] = (f & 1) ? n[ax] : -1;
      double ug = 0.0;
      if (!parent_interp(up, p0, p1, p2, periodic, org, ghost, &ug)) atomicExch(bad, 1);
      double ui = u_init[((long long)inner[2] * n1 + inner[1]) * n0 + inner[0]];
      ub[t] = 0.5 * (ug + ui);
      return;
    }
    off += sz;
  }
}

static void patch_bc_dev(frmg_ctx *ctx, Scope &S, const double *up, const int np_[3], int periodic,
                         const int org[3], const int n[3], double *u_init, double *ub,
                         cudaStream_t st) {
  int *bad = S.get<int>(1);
  CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
  long long nc = (long long)n[0] * n[1] * n[2];
  k_patch_init<<<nblocks(nc), 256, 0, st>>>(up, np_[0], np_[1], np_[2], periodic, org[0], org[1],
                                            org[2], n[0], n[1], n[2], u_init, bad);
  CK_LAUNCH(ctx);
  long long nf = face_total(n);
  k_patch_faces<<<nblocks(nf), 256, 0, st>>>(up, np_[0], np_[1], np_[2], periodic, org[0],
                                             org[1], org[2], n[0], n[1], n[2], u_init, ub, bad);
  CK_LAUNCH(ctx);
  int hb = 0;
  CK(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hb) einval("patch interpolation stencil leaves its parent (needs a 1-parent-cell margin)");
}

// y += s * x
__global__ void k_axpy(double *y, const double *x, double s, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] += s * x[t];
}

void frmg_axpy(double *y, const double *x, double s, long long n, cudaStream_t st,
               frmg_ctx *ctx) {
  k_axpy<<<nblocks(n), 256, 0, st>>>(y, x, s, n);
  CK_LAUNCH(ctx);
}

// ===========================================================================
// C ABI
extern "C" {

void fr_opts_default(fr_opts *o) {
  if (!o) return;
  o->tol = 1e-8;
  o->max_vcycles = 100;
  o->pre = 2;
  o->post = 2;
  o->prec = FR_FP64;
  o->newton_step_cap = 1.0;
  o->inner_cycles = 2;
  o->max_outer = 40;
  o->allow_negative_density = 0;
  o->use_graph = 1;
  o->temporal_depth = 0;
  o->tiling = 0;
  o->defect_precision = 0;
  o->tau_alpha = 0.0;
  o->relax = 1.0;
  o->fmg = 0;
  o->initial_guess = 1;
  o->smooth_tile = 0;
}

const char *fr_status_string(int s) {
  switch (s) {
    case FR_OK: return "FR_OK";
    case FR_EINVAL: return "FR_EINVAL: invalid argument";
    case FR_ENOMEM: return "FR_ENOMEM: allocation failed";
    case FR_ECUDA: return "FR_ECUDA: CUDA error";
    case FR_ENOCONV: return "FR_ENOCONV: tolerance not reached";
    case FR_EDIVERGED: return "FR_EDIVERGED: iteration diverged";
    case FR_ETIMEOUT: return "FR_ETIMEOUT: device wait timed out (reserved; not returned)";
    default: return "unknown status";
  }
}

const char *fr_last_error(void) { return g_last_error.c_str(); }

int fr_ctx_create(frmg_ctx **out, int device) {
  return guard([&]() {
    if (!out) einval("out is NULL");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) einval("no such device");
    CK(cudaSetDevice(device));
    frmg_ctx *c = new frmg_ctx();
    c->device = device;
    if (const char *lim = getenv("FRMG_WORKSPACE_LIMIT")) c->limit = strtoull(lim, nullptr, 10);
    *out = c;
    return FR_OK;
  });
}

void fr_ctx_destroy(frmg_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  prof_harvest(c);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
    cudaEventDestroy(c->side_in);
    cudaEventDestroy(c->side_out);
  }
  if (c->copy) {
    cudaStreamSynchronize(c->copy);
    cudaStreamDestroy(c->copy);
    cudaEventDestroy(c->copy_in);
    cudaEventDestroy(c->copy_out);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  for (auto &kv : c->sizes) cudaFree(kv.first);
  if (c->pinned) cudaFreeHost(c->pinned);
  delete c;
}

long long fr_launch_count(const frmg_ctx *c) { return c ? c->launches : 0; }

int fr_profile(frmg_ctx *c, int enable) {
  if (!c) return FR_EINVAL;
  prof_harvest(c);
  c->prof = enable != 0;
  c->prof_names.clear();
  c->prof_count.clear();
  c->prof_ms.clear();
  return FR_OK;
}

int fr_profile_entry(frmg_ctx *c, int idx, char *name, int namelen, long long *count,
                     double *total_ms) {
  if (!c || idx < 0) return FR_EINVAL;
  prof_harvest(c);
  if (idx >= (int)c->prof_names.size()) return FR_EINVAL;
  if (name && namelen > 0) {
    strncpy(name, c->prof_names[idx].c_str(), (size_t)namelen - 1);
    name[namelen - 1] = 0;
  }
  if (count) *count = c->prof_count[idx];
  if (total_ms) *total_ms = c->prof_ms[idx];
  return FR_OK;
}

int fr_constants(double box, int n0, double a, double om, double fr0, double *out6) {
  return guard([&]() {
    check_model(box, a, om, fr0);
    if (n0 <= 0 || !out6) einval("n0 <= 0 or out NULL");
    Consts k = model_consts(box, 1.0 / n0, a, om, fr0);
    out6[0] = k.alpha;
    out6[1] = k.beta;
    out6[2] = k.gamma;
    out6[3] = k.ct;
    out6[4] = k.fbar;
    out6[5] = k.ubar;
    return FR_OK;
  });
}

static int solve_impl(frmg_ctx *ctx, const double *density, const int dims[3], double box,
                      double a, double om, double fr0, double tol, double *u, const fr_opts *opts,
                      fr_stats *stats, void *stream, int fixed) {
  double t0 = now_s();
  return guard([&]() {
    if (!ctx || !density || !dims || !u) einval("NULL argument");
    check_dims(dims);
    check_model(box, a, om, fr0);
    fr_opts o = resolve_opts(opts);
    if (fixed > 0 && o.prec != FR_FP64) einval("fixed cycle counts are FP64 only");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scope S(ctx);
    std::vector<Staged> back;
    long long nc = (long long)dims[0] * dims[1] * dims[2];
    // the mixed double-float solve of a zero start validates rho in its first
    // pass; every other solve validates it here
    const bool defer = !o.initial_guess && o.prec == FR_MIXED && o.defect_precision == 0 &&
                       fixed <= 0;
    // that first pass is the only reader of rho: page-locked host density is
    // read there across the host link instead of being copied in first
    const double *drho = defer ? mapped_host(density) : nullptr;
    if (!drho) drho = stage(S, back, density, nc, true, false, st);
    double *du = stage_u(S, back, u, nc, o, st);
    if (!defer) validate_density(ctx, S, drho, nc, o.allow_negative_density, st);
    Problem p;
    memset(&p, 0, sizeof(p));
    for (int d = 0; d < 3; d++) p.n[d] = dims[d];
    p.h = 1.0 / dims[0];
    p.box = box;
    p.a = a;
    p.om = om;
    p.fr0 = fr0;
    p.rho = drho;
    p.u = du;
    p.zero_u = !o.initial_guess;
    p.check_rho = defer ? (o.allow_negative_density ? 2 : 1) : 0;
    p.host_u = du != u && is_pinned_host(u) ? u : nullptr;
    std::vector<Problem> P{p};
    std::vector<fr_stats> sv(1);
    memset(sv.data(), 0, sizeof(fr_stats));
    int status = FR_OK;
    try {
      run_problems(ctx, P, o, tol, sv, st, fixed);
      status = fixed > 0 ? FR_OK : status_from_stats(sv, tol, o.tau_alpha);
    } catch (FrError &e) {
      if (e.status != FR_EDIVERGED) throw;
      status = e.status;
      g_last_error = e.msg;
    }
    // the mixed solve may have copied its final u to the host already
    if (P[0].early_copied)
      back.erase(std::remove_if(back.begin(), back.end(),
                                [&](const Staged &b) { return b.host_dst == (void *)u; }),
                 back.end());
    for (const Staged &b : back)
      if (b.host_dst == (void *)u) sv[0].host_copies++;
    finish(ctx, back, st);
    sv[0].seconds = now_s() - t0;
    if (stats) *stats = sv[0];
    return status;
  });
}

int fr_solve(frmg_ctx *ctx, const double *density, const int dims[3], double box, double a,
             double om, double fr0, double tol, double *u, const fr_opts *opts, fr_stats *stats,
             void *stream) {
  return solve_impl(ctx, density, dims, box, a, om, fr0, tol, u, opts, stats, stream, 0);
}

int fr_autotune(frmg_ctx *ctx, const double *density, const int dims[3], double box, double a,
                double om, double fr0, double tol, const fr_opts *base, fr_opts *best,
                double *best_seconds, void *stream) {
  return guard([&]() {
    if (!ctx || !density || !dims || !best) einval("NULL argument");
    check_dims(dims);
    check_model(box, a, om, fr0);
    fr_opts o0 = resolve_opts(base);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    long long nc = (long long)dims[0] * dims[1] * dims[2];
    double *u = nullptr;
    const double *rho = density;
    {
      // scratch solution (and density, if on the host) for the trials
      u = (double *)frmg_alloc(ctx, nc * sizeof(double));
      if (!is_device_ptr(density)) {
        double *d = (double *)frmg_alloc(ctx, nc * sizeof(double));
        CK(cudaMemcpyAsync(d, density, nc * sizeof(double), cudaMemcpyHostToDevice, st));
        rho = d;
      }
    }
    const int shapes[5][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 3}};
    const double relaxes[3] = {1.0, 1.15, 1.25};
    double best_t = HUGE_VAL;
    fr_opts best_o = o0;
    int status = FR_ENOCONV;
    // best of two solves from u = 0 with options o
    auto trial = [&](const fr_opts &o) {
      double tmin = HUGE_VAL;
      for (int rep = 0; rep < 2; rep++) {
        CK(cudaMemsetAsync(u, 0, nc * sizeof(double), st));
        CK(cudaStreamSynchronize(st));
        double t0 = now_s();
        fr_stats sv;
        int r = fr_solve(ctx, rho, dims, box, a, om, fr0, tol, u, &o, &sv, stream);
        double t1 = now_s();
        if (r != FR_OK) return HUGE_VAL;
        tmin = std::min(tmin, t1 - t0);
      }
      if (tmin < best_t) {
        best_t = tmin;
        best_o = o;
        status = FR_OK;
      }
      return tmin;
    };
    // every V-cycle shape and relaxation factor with one sweep per tiled
    // pass; then, one at a time on top of the best setting so far, two sweeps
    // per tiled pass, the full-multigrid start and tiling wherever possible
    for (int sh = 0; sh < 5; sh++)
      for (double w : relaxes) {
        fr_opts o = o0;
        o.pre = shapes[sh][0];
        o.post = shapes[sh][1];
        o.temporal_depth = 1;
        o.relax = w;
        trial(o);
      }
    if (status == FR_OK) {
      fr_opts o = best_o;
      o.temporal_depth = 2;
      trial(o);
      o = best_o;
      o.fmg = 1;
      trial(o);
      o = best_o;
      o.tiling = 1;
      trial(o);
      // kernel and tile of the plain one-sweep smoother: register columns on
      // 64 x 16 (the default) or 64 x 8 tiles, or the shared-memory plane ring
      if (best_o.smooth_tile == 0) best_o.smooth_tile = kDefaultSmoothTile;
      for (int t : {16, 8, -1}) {
        if (t == best_o.smooth_tile) continue;
        o = best_o;
        o.smooth_tile = t;
        trial(o);
      }
    }
    frmg_release(ctx, u);
    if (rho != density) frmg_release(ctx, const_cast<double *>(rho));
    *best = best_o;
    if (best_seconds) *best_seconds = best_t;
    if (status != FR_OK) g_last_error = "no candidate setting reached tol";
    return status;
  });
}

int fr_autotune_batch(frmg_ctx *ctx, int nfields, const double *const *density,
                      const int (*dims)[3], const double *box, const double *a,
                      const double *fr0, double om, double tol, const fr_opts *base,
                      fr_opts *best, double *best_seconds, void *stream) {
  return guard([&]() {
    if (!ctx || nfields <= 0 || !density || !dims || !box || !a || !fr0 || !best)
      einval("NULL argument or nfields <= 0");
    fr_opts o0 = resolve_opts(base);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    // scratch solutions (every trial starts from u = 0 and never reads them)
    // and device copies of host densities
    std::vector<void *> held;
    std::vector<double *> us(nfields);
    std::vector<const double *> rhos(nfields);
    struct Release {
      frmg_ctx *c;
      std::vector<void *> &v;
      ~Release() {
        for (void *p : v) frmg_release(c, p);
      }
    } rel{ctx, held};
    for (int i = 0; i < nfields; i++) {
      if (!density[i]) einval("NULL field pointer");
      check_dims(dims[i]);
      check_model(box[i], a[i], om, fr0[i]);
      const long long nc = (long long)dims[i][0] * dims[i][1] * dims[i][2];
      us[i] = (double *)frmg_alloc(ctx, nc * sizeof(double));
      held.push_back(us[i]);
      rhos[i] = density[i];
      if (!is_device_ptr(density[i])) {
        double *d = (double *)frmg_alloc(ctx, nc * sizeof(double));
        held.push_back(d);
        CK(cudaMemcpyAsync(d, density[i], nc * sizeof(double), cudaMemcpyHostToDevice, st));
        rhos[i] = d;
      }
    }
    CK(cudaStreamSynchronize(st));
    const int shapes[5][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 3}};
    const double relaxes[3] = {1.0, 1.15, 1.25};
    double best_t = HUGE_VAL;
    fr_opts best_o = o0;
    int status = FR_ENOCONV;
    auto trial = [&](fr_opts o) {
      o.initial_guess = 0;
      double tmin = HUGE_VAL;
      for (int rep = 0; rep < 2; rep++) {
        const double t0 = now_s();
        const int r = fr_solve_batch(ctx, nfields, rhos.data(), dims, box, a, fr0, om, tol,
                                     us.data(), &o, nullptr, stream);
        const double t1 = now_s();
        if (r != FR_OK) return;
        tmin = std::min(tmin, t1 - t0);
      }
      if (tmin < best_t) {
        best_t = tmin;
        best_o = o;
        best_o.initial_guess = o0.initial_guess;
        status = FR_OK;
      }
    };
    // V-cycle shape x relaxation x tiling (the shared-memory kernels where the
    // level sets fill the GPU, or wherever possible), then the smoother's tile
    for (int tiling : {0, 1})
      for (int sh = 0; sh < 5; sh++)
        for (double w : relaxes) {
          fr_opts o = o0;
          o.pre = shapes[sh][0];
          o.post = shapes[sh][1];
          o.temporal_depth = 1;
          o.relax = w;
          o.tiling = tiling;
          trial(o);
        }
    if (status == FR_OK) {
      if (best_o.smooth_tile == 0) best_o.smooth_tile = kDefaultSmoothTile;
      const fr_opts b0 = best_o;
      for (int t : {16, 8, -1}) {
        if (t == b0.smooth_tile) continue;
        fr_opts o = b0;
        o.smooth_tile = t;
        trial(o);
      }
    }
    *best = best_o;
    if (best_seconds) *best_seconds = best_t;
    if (status != FR_OK) g_last_error = "no candidate setting reached tol";
    return status;
  });
}

int fr_vcycles(frmg_ctx *ctx, const double *density, const int dims[3], double box, double a,
               double om, double fr0, double *u, int ncycles, const fr_opts *opts,
               fr_stats *stats, void *stream) {
  if (ncycles <= 0) {
    g_last_error = "ncycles must be > 0";
    return FR_EINVAL;
  }
  return solve_impl(ctx, density, dims, box, a, om, fr0, 0.0, u, opts, stats, stream, ncycles);
}

int fr_solve_batch(frmg_ctx *ctx, int nfields, const double *const *density, const int (*dims)[3],
                   const double *box, const double *a, const double *fr0, double om, double tol,
                   double *const *u, const fr_opts *opts, fr_stats *stats, void *stream) {
  double t0 = now_s();
  return guard([&]() {
    if (!ctx || nfields <= 0 || !density || !dims || !box || !a || !fr0 || !u)
      einval("NULL argument or nfields <= 0");
    fr_opts o = resolve_opts(opts);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scope S(ctx);
    std::vector<Staged> back;
    std::vector<Problem> P(nfields);
    for (int i = 0; i < nfields; i++) {
      if (!density[i] || !u[i]) einval("NULL field pointer");
      check_dims(dims[i]);
      check_model(box[i], a[i], om, fr0[i]);
      long long nc = (long long)dims[i][0] * dims[i][1] * dims[i][2];
      Problem &p = P[i];
      memset(&p, 0, sizeof(p));
      for (int d = 0; d < 3; d++) p.n[d] = dims[i][d];
      p.h = 1.0 / dims[i][0];
      p.box = box[i];
      p.a = a[i];
      p.om = om;
      p.fr0 = fr0[i];
      p.rho = stage(S, back, density[i], nc, true, false, st);
      p.u = stage_u(S, back, u[i], nc, o, st);
      p.zero_u = !o.initial_guess;
      validate_density(ctx, S, p.rho, nc, o.allow_negative_density, st);
    }
    std::vector<fr_stats> sv(nfields);
    memset(sv.data(), 0, nfields * sizeof(fr_stats));
    int status = FR_OK;
    try {
      run_problems(ctx, P, o, tol, sv, st);
      status = status_from_stats(sv, tol, o.tau_alpha);
    } catch (FrError &e) {
      if (e.status != FR_EDIVERGED) throw;
      status = e.status;
      g_last_error = e.msg;
    }
    finish(ctx, back, st);
    double dt = now_s() - t0;
    if (stats)
      for (int i = 0; i < nfields; i++) {
        stats[i] = sv[i];
        stats[i].seconds = dt;
      }
    return status;
  });
}

int fr_solve_levels(frmg_ctx *ctx, const double *density, const int dims[3], double box, double a,
                    double om, double fr0, double tol, double tol_patch, double *u,
                    fr_patch *patches, int npatch, const fr_opts *opts, fr_stats *per_grid,
                    void *stream) {
  double t0 = now_s();
  return guard([&]() {
    if (!ctx || !density || !dims || !u || (npatch > 0 && !patches) || npatch < 0)
      einval("NULL argument");
    check_dims(dims);
    check_model(box, a, om, fr0);
    fr_opts o = resolve_opts(opts);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scope S(ctx);
    std::vector<Staged> back;
    // validate nesting on the host
    std::vector<int> level(npatch, 0);
    std::vector<std::array<int, 3>> pdims(npatch);
    for (int i = 0; i < npatch; i++) {
      fr_patch &pp = patches[i];
      if (pp.parent >= i || pp.parent < -1) einval("patch parent must precede the patch");
      if (!pp.density || !pp.u) einval("NULL patch pointer");
      check_dims(pp.n, 4);
      const int *par = pp.parent < 0 ? dims : pdims[pp.parent].data();
      level[i] = pp.parent < 0 ? 1 : level[pp.parent] + 1;
      for (int d = 0; d < 3; d++) {
        pdims[i][d] = pp.n[d];
        if (pp.parent >= 0) {
          // footprint + 1 parent cell must lie inside the parent patch
          if (pp.origin[d] < 1 || pp.origin[d] + pp.n[d] / 2 + 1 > par[d])
            einval("patch " + std::to_string(i) + " not nested with a 1-cell margin");
        } else if (pp.n[d] / 2 > par[d]) {
          einval("patch larger than the domain");
        }
      }
    }
    long long nc = (long long)dims[0] * dims[1] * dims[2];
    const double *drho = stage(S, back, density, nc, true, false, st);
    double *du = stage_u(S, back, u, nc, o, st);
    validate_density(ctx, S, drho, nc, o.allow_negative_density, st);
    std::vector<fr_stats> all(1 + npatch);
    memset(all.data(), 0, all.size() * sizeof(fr_stats));
    int status = FR_OK;
    auto run = [&](std::vector<Problem> &P, std::vector<fr_stats> &sv, double tl) {
      try {
        run_problems(ctx, P, o, tl, sv, st);
        int s2 = status_from_stats(sv, tl, o.tau_alpha);
        if (s2 != FR_OK && status == FR_OK) status = s2;
      } catch (FrError &e) {
        if (e.status != FR_EDIVERGED) throw;
        status = e.status;
        g_last_error = e.msg;
      }
    };
    {
      Problem p;
      memset(&p, 0, sizeof(p));
      for (int d = 0; d < 3; d++) p.n[d] = dims[d];
      p.h = 1.0 / dims[0];
      p.box = box;
      p.a = a;
      p.om = om;
      p.fr0 = fr0;
      p.rho = drho;
      p.u = du;
      p.zero_u = !o.initial_guess;
      std::vector<Problem> P{p};
      std::vector<fr_stats> sv(1);
      memset(sv.data(), 0, sizeof(fr_stats));
      run(P, sv, tol);
      all[0] = sv[0];
    }
    // patches level by level (one batched solve per refinement level)
    std::vector<double *> pu(npatch, nullptr);
    std::vector<double> ph(npatch, 0.0);
    int maxlev = 0;
    for (int i = 0; i < npatch; i++) maxlev = std::max(maxlev, level[i]);
    for (int lv = 1; lv <= maxlev; lv++) {
      std::vector<Problem> P;
      std::vector<int> ids;
      for (int i = 0; i < npatch; i++) {
        if (level[i] != lv) continue;
        fr_patch &pp = patches[i];
        long long pn = (long long)pp.n[0] * pp.n[1] * pp.n[2];
        const double *prho = stage(S, back, pp.density, pn, true, false, st);
        pu[i] = stage(S, back, pp.u, pn, false, true, st);
        validate_density(ctx, S, prho, pn, o.allow_negative_density, st);
        double *ub = S.get<double>(face_total(pp.n));
        const double *up = pp.parent < 0 ? du : pu[pp.parent];
        const int *pdim = pp.parent < 0 ? dims : pdims[pp.parent].data();
        double hpar = pp.parent < 0 ? 1.0 / dims[0] : ph[pp.parent];
        patch_bc_dev(ctx, S, up, pdim, pp.parent < 0, pp.origin, pp.n, pu[i], ub, st);
        ph[i] = 0.5 * hpar;
        Problem p;
        memset(&p, 0, sizeof(p));
        for (int d = 0; d < 3; d++) p.n[d] = pp.n[d];
        p.h = ph[i];
        p.box = box;
        p.a = a;
        p.om = om;
        p.fr0 = fr0;
        p.rho = prho;
        p.u = pu[i];
        p.bnd = ub;
        P.push_back(p);
        ids.push_back(i);
      }
      std::vector<fr_stats> sv(P.size());
      memset(sv.data(), 0, sv.size() * sizeof(fr_stats));
      run(P, sv, tol_patch);
      for (size_t j = 0; j < ids.size(); j++) all[1 + ids[j]] = sv[j];
    }
    finish(ctx, back, st);
    double dt = now_s() - t0;
    if (per_grid)
      for (int i = 0; i <= npatch; i++) {
        per_grid[i] = all[i];
        per_grid[i].seconds = dt;
      }
    return status;
  });
}

// ---- single-step entry points ----
static Problem one_level(const int dims[3], double h, double box, double a, double om,
                         double fr0) {
  check_dims(dims);
  check_model(box, a, om, fr0);
  if (!(h > 0)) einval("h must be > 0");
  Problem p;
  memset(&p, 0, sizeof(p));
  for (int d = 0; d < 3; d++) p.n[d] = dims[d];
  p.h = h;
  p.box = box;
  p.a = a;
  p.om = om;
  p.fr0 = fr0;
  p.nl = 1;
  return p;
}

// One FP64 level whose right-hand side is gamma(rho-1) + f.
static Grid<double> single_grid(Scope &S, frmg_ctx *ctx, Problem &p, double *u, const double *rho,
                                const double *f, const double *ub, double cap, cudaStream_t st) {
  Consts k = model_consts(p.box, p.h, p.a, p.om, p.fr0);
  Grid<double> G;
  memset(&G, 0, sizeof(G));
  G.n0 = p.n[0];
  G.n1 = p.n[1];
  G.n2 = p.n[2];
  G.ncell = (long long)p.n[0] * p.n[1] * p.n[2];
  G.ah = 0.5 * k.alpha;
  G.beta = k.beta;
  G.cap = cap;
  G.relax = 1.0;
  G.u = u;
  G.x = S.get<double>(G.ncell);
  face_offsets(p.n, G.foff);
  G.bnd = ub;
  // right-hand side gamma (rho - 1) + f, stored as rho + f/gamma with fs = gamma, fo = 1
  double *ft = S.get<double>(G.ncell);
  k_convert<double, double><<<nblocks(G.ncell), 256, 0, st>>>(rho, ft, G.ncell);
  CK_LAUNCH(ctx);
  G.f = ft;
  G.fs = k.gamma;
  G.fo = 1.0;
  if (f) frmg_axpy(ft, f, 1.0 / k.gamma, G.ncell, st, ctx);
  k_expm1<double><<<nblocks(G.ncell), 256, 0, st>>>(G.u, G.x, G.ncell);
  CK_LAUNCH(ctx);
  return G;
}

int fr_smooth(frmg_ctx *ctx, double *u, const double *density, const double *f, const int dims[3],
              double h, double box, double a, double om, double fr0, const double *ub, int nsweeps,
              double cap, void *stream) {
  return guard([&]() {
    if (!ctx || !u || !density || !dims || nsweeps < 0 || !(cap > 0)) einval("bad argument");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Problem p = one_level(dims, h, box, a, om, fr0);
    Scope S(ctx);
    std::vector<Staged> back;
    long long nc = (long long)dims[0] * dims[1] * dims[2];
    double *du = stage(S, back, u, nc, true, true, st);
    const double *dr = stage(S, back, density, nc, true, false, st);
    const double *df = stage(S, back, f, nc, true, false, st);
    const double *dub = stage(S, back, ub, ub ? face_total(dims) : 0, true, false, st);
    LevelSet<double> ls;
    ls.h.push_back(single_grid(S, ctx, p, du, dr, df, dub, cap, st));
    upload_set(S, ls, st);
    int par = 0;
    smooth_set<double, false>(ctx, ls, nsweeps, nullptr, nullptr, par, st);
    finish(ctx, back, st);
    return FR_OK;
  });
}

int fr_smooth_f32(frmg_ctx *ctx, float *u, const float *bg, const float *f, const int dims[3],
                  double h, double box, double a, double om, double fr0, const float *ub,
                  int nsweeps, double cap, int tiled, void *stream) {
  return guard([&]() {
    if (!ctx || !u || !dims || nsweeps < 0 || !(cap > 0)) einval("bad argument");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    one_level(dims, h, box, a, om, fr0);  // argument checks
    Scope S(ctx);
    std::vector<Staged> back;
    long long nc = (long long)dims[0] * dims[1] * dims[2];
    Consts k = model_consts(box, h, a, om, fr0);
    Grid<float> G;
    memset(&G, 0, sizeof(G));
    G.n0 = dims[0];
    G.n1 = dims[1];
    G.n2 = dims[2];
    G.ncell = nc;
    G.ah = (float)(0.5 * k.alpha);
    G.beta = (float)k.beta;
    G.cap = (float)cap;
    G.relax = 1.0f;
    G.fs = 1.0f;
    G.fo = 0.0f;
    face_offsets(dims, G.foff);
    float *du = stage(S, back, u, nc, true, true, st);
    G.u = S.get<float>(nc);
    G.u2 = S.get<float>(nc);
    G.x2 = S.get<float>(nc);
    CK(cudaMemcpyAsync(G.u, du, nc * sizeof(float), cudaMemcpyDeviceToDevice, st));
    G.x = S.get<float>(nc);
    k_expm1<float><<<nblocks(nc), 256, 0, st>>>(G.u, G.x, nc);
    CK_LAUNCH(ctx);
    G.f = stage(S, back, f, nc, true, false, st);
    G.bnd = stage(S, back, ub, ub ? face_total(dims) : 0, true, false, st);
    if (bg) {
      G.ubg = stage(S, back, bg, nc, true, false, st);
      float *E = S.get<float>(nc);
      k_expf<<<nblocks(nc), 256, 0, st>>>(G.ubg, E, nc);
      CK_LAUNCH(ctx);
      G.Ebg = E;
    }
    if (!(tiled == 0 || tiled == 1 || tiled == 8 || tiled == 16))
      einval("tiled must be 0, 1, 8 or 16");
    LevelSet<float> ls;
    ls.h.push_back(G);
    upload_set(S, ls, st, 0, tiled > 1 ? tiled : 0);
    if (tiled && !ls.tiled_ok) einval("tiled smoothing needs at least 16 cells a side");
    ls.tiled = tiled != 0;
    std::vector<int> plan(nsweeps, 1);  // one sweep per tiled pass, as in the solves
    int par = 0;
    if (bg)
      smooth_set<float, true>(ctx, ls, nsweeps, &plan, nullptr, par, st);
    else
      smooth_set<float, false>(ctx, ls, nsweeps, &plan, nullptr, par, st);
    CK(cudaMemcpyAsync(du, par ? G.u2 : G.u, nc * sizeof(float), cudaMemcpyDeviceToDevice, st));
    finish(ctx, back, st);
    return FR_OK;
  });
}

int fr_residual(frmg_ctx *ctx, const double *u, const double *density, const double *f,
                const int dims[3], double h, double box, double a, double om, double fr0,
                const double *ub, double *d, void *stream) {
  return guard([&]() {
    if (!ctx || !u || !density || !dims || !d) einval("bad argument");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Problem p = one_level(dims, h, box, a, om, fr0);
    Scope S(ctx);
    std::vector<Staged> back;
    long long nc = (long long)dims[0] * dims[1] * dims[2];
    double *du = S.get<double>(nc);
    const double *su = stage(S, back, u, nc, true, false, st);
    CK(cudaMemcpyAsync(du, su, nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    const double *dr = stage(S, back, density, nc, true, false, st);
    const double *df = stage(S, back, f, nc, true, false, st);
    const double *dub = stage(S, back, ub, ub ? face_total(dims) : 0, true, false, st);
    double *dd = stage(S, back, d, nc, false, true, st);
    LevelSet<double> ls;
    ls.h.push_back(single_grid(S, ctx, p, du, dr, df, dub, 1.0, st));
    upload_set(S, ls, st);
    std::vector<double> nr;
    double *outs[1] = {dd};
    level_norms<double, false>(ctx, ls, outs, nullptr, st, nr);
    finish(ctx, back, st);
    return FR_OK;
  });
}

int fr_residual_df(frmg_ctx *ctx, const double *u, const double *density, const int dims[3],
                   double h, double box, double a, double om, double fr0, const double *ub,
                   double *d, void *stream) {
  return guard([&]() {
    if (!ctx || !u || !density || !dims || !d) einval("bad argument");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Problem p = one_level(dims, h, box, a, om, fr0);
    Consts k = model_consts(box, h, a, om, fr0);
    Scope S(ctx);
    std::vector<Staged> back;
    long long nc = (long long)dims[0] * dims[1] * dims[2];
    const double *du = stage(S, back, u, nc, true, false, st);
    const double *dr = stage(S, back, density, nc, true, false, st);
    const double *dub = stage(S, back, ub, ub ? face_total(dims) : 0, true, false, st);
    double *dd = stage(S, back, d, nc, false, true, st);
    DFGrid g;
    dfgrid_setup(g, dims, k, dub);
    g.u = S.get<float2>(nc);
    g.B = S.get<float2>(nc);
    g.r = S.get<float2>(nc);
    float ln2h, ln2l;
    split_host(std::log(2.0), ln2h, ln2l);
    (void)p;
    k_df_init<<<nblocks(nc), 256, 0, st>>>(g, du, dr, 0, ln2h, ln2l);
    CK_LAUNCH(ctx);
    float *scratch = S.get<float>(5 * (size_t)nc);
    double *partial = S.get<double>(2 * (size_t)nblocks(nc));
    launch_df_defect(ctx, g, scratch, scratch + nc, scratch + 2 * nc, scratch + 3 * nc,
                     scratch + 4 * nc, partial, 0, ln2h, ln2l, dd, st);
    finish(ctx, back, st);
    return FR_OK;
  });
}

int fr_restrict(frmg_ctx *ctx, const double *fine, const int dims[3], double *coarse,
                void *stream) {
  return guard([&]() {
    if (!ctx || !fine || !dims || !coarse) einval("bad argument");
    check_dims(dims);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scope S(ctx);
    std::vector<Staged> back;
    long long nf = (long long)dims[0] * dims[1] * dims[2];
    const double *df = stage(S, back, fine, nf, true, false, st);
    double *dc = stage(S, back, coarse, nf / 8, false, true, st);
    k_restrict_avg<double><<<nblocks(nf / 8), 256, 0, st>>>(df, dims[0], dims[1], dims[2], dc);
    CK_LAUNCH(ctx);
    finish(ctx, back, st);
    return FR_OK;
  });
}

int fr_prolong_correct(frmg_ctx *ctx, double *uf, const int dims[3], const double *uH,
                       const double *uR, int dirichlet, void *stream) {
  return guard([&]() {
    if (!ctx || !uf || !dims || !uH || !uR) einval("bad argument");
    check_dims(dims);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scope S(ctx);
    std::vector<Staged> back;
    long long nf = (long long)dims[0] * dims[1] * dims[2];
    Grid<double> F, C;
    memset(&F, 0, sizeof(F));
    memset(&C, 0, sizeof(C));
    F.n0 = dims[0];
    F.n1 = dims[1];
    F.n2 = dims[2];
    F.ncell = nf;
    F.u = stage(S, back, uf, nf, true, true, st);
    F.x = S.get<double>(nf);
    // a non-null bnd marks the grid as a patch (the values are not read)
    F.bnd = dirichlet ? F.x : nullptr;
    C.n0 = dims[0] / 2;
    C.n1 = dims[1] / 2;
    C.n2 = dims[2] / 2;
    C.ncell = nf / 8;
    C.u = const_cast<double *>(stage(S, back, uH, nf / 8, true, false, st));
    C.uR = const_cast<double *>(stage(S, back, uR, nf / 8, true, false, st));
    LevelSet<double> lf, lc;
    lf.h.push_back(F);
    lc.h.push_back(C);
    upload_set(S, lf, st);
    upload_set(S, lc, st);
    k_prolong<double><<<lc.nblk_full, 256, 0, st>>>(lf.d, lc.d, lc.d_off_full, 1, nullptr, 0, 0);
    CK_LAUNCH(ctx);
    finish(ctx, back, st);
    return FR_OK;
  });
}

int fr_patch_bc(frmg_ctx *ctx, const double *uparent, const int dims_parent[3], int periodic,
                const int origin[3], const int n[3], double *u_init, double *ub, void *stream) {
  return guard([&]() {
    if (!ctx || !uparent || !dims_parent || !origin || !n || !u_init || !ub)
      einval("bad argument");
    check_dims(n);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scope S(ctx);
    std::vector<Staged> back;
    long long npar = (long long)dims_parent[0] * dims_parent[1] * dims_parent[2];
    long long nc = (long long)n[0] * n[1] * n[2];
    const double *dp = stage(S, back, uparent, npar, true, false, st);
    double *di = stage(S, back, u_init, nc, false, true, st);
    double *db = stage(S, back, ub, face_total(n), false, true, st);
    patch_bc_dev(ctx, S, dp, dims_parent, periodic, origin, n, di, db, st);
    finish(ctx, back, st);
    return FR_OK;
  });
}

}  // extern "C"

