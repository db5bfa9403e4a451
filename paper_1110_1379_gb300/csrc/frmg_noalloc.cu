// frmg_noalloc.cu -- residual norm of one grid without any device allocation.
//
// Some callers cannot allocate device memory at the moment they want to know
// how far a field is from solving the equation: code whose device memory is
// entirely owned by another allocator (a framework's caching pool that leaves
// nothing for cudaMalloc, or that must see every allocation), and
// latency-critical loops that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree.
// fr_residual_norm_noalloc serves them: the caller passes device inputs and a
// device output, and the only scratch (the per-block partial sums of the
// reduction) lives in a fixed array of this library's module that every GPU
// loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "frmg.h"
#include "frmg_internal.h"

namespace {

constexpr int kNABlocks = 1024;  // blocks of the partial-sum pass
constexpr int kNAThreads = 256;
constexpr long long kNAMaxCells = 1LL << 25;  // 33,554,432 cells (e.g. 320^3)
constexpr int kNAMaxDevices = 64;

// Scratch of the allocation-free path: (sum of squares, max) per block.
static __device__ __align__(256) double g_na_partials[2 * kNABlocks];

std::mutex g_na_mu;
double *g_na_ptr[kNAMaxDevices] = {nullptr};

// L(u) at one cell, FP64, with e^u evaluated on the fly (no cache array).
// Same operator as the library's other residual kernels: flux form of
// Eq. discrete_fR times c~^2, patch ghosts u_g = 2 u_b - u_i.
__device__ double na_cell(const double *u, const double *rho, const double *ub,
                          const long long *foff, int n0, int n1, int n2, double ah, double beta,
                          double gamma, int i, int j, int k) {
  const long long c = ((long long)k * n1 + j) * n0 + i;
  const double ui = u[c];
  const double bi = exp(ui);
  const bool dir = ub != nullptr;
  double acc = 0.0;
  const int idx[3] = {i, j, k};
  const int n[3] = {n0, n1, n2};
  const long long stride[3] = {1, n0, (long long)n0 * n1};
  for (int f = 0; f < 6; f++) {
    const int ax = f >> 1, s = (f & 1) ? 1 : -1;
    int q = idx[ax] + s;
    if (q >= 0 && q < n[ax]) {
      const double uj = u[c + s * stride[ax]];
      acc += (bi + exp(uj)) * (uj - ui);
    } else if (!dir) {
      const double uj = u[c + (q < 0 ? (n[ax] - 1) : -(n[ax] - 1)) * stride[ax]];
      acc += (bi + exp(uj)) * (uj - ui);
    } else {
      long long o;
      if (ax == 0) o = (long long)k * n1 + j;
      else if (ax == 1) o = (long long)k * n0 + i;
      else o = (long long)j * n0 + i;
      const double ug = 2.0 * ub[foff[f] + o] - ui;
      acc += (bi + exp(ug)) * (ug - ui);
    }
  }
  return ah * acc + beta * (exp(-0.5 * ui) - 1.0) - gamma * (rho[c] - 1.0);
}

struct NAGrid {
  const double *u, *rho, *ub;
  long long foff[6];
  long long ncell;
  int n0, n1, n2;
  double ah, beta, gamma;
};

// Grid-stride pass: every one of the kNABlocks blocks writes its partials,
// including blocks that own no cell, so nothing of an earlier call survives.
__global__ void __launch_bounds__(kNAThreads) k_na_partials(NAGrid G, double *partials) {
  double s = 0.0, m = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < G.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % G.n0);
    const long long r = c / G.n0;
    const int j = (int)(r % G.n1);
    const int k = (int)(r / G.n1);
    const double d = na_cell(G.u, G.rho, G.ub, G.foff, G.n0, G.n1, G.n2, G.ah, G.beta, G.gamma,
                             i, j, k);
    s += d * d;
    m = fmax(m, fabs(d));
  }
  __shared__ double ss[kNAThreads / 32], sm[kNAThreads / 32];
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
    double ts = 0.0, tm = 0.0;
    for (int q = 0; q < kNAThreads / 32; q++) {
      ts += ss[q];
      tm = fmax(tm, sm[q]);
    }
    partials[2 * blockIdx.x] = ts;
    partials[2 * blockIdx.x + 1] = tm;
  }
}

__global__ void k_na_final(const double *partials, long long ncell, double *out2) {
  __shared__ double ss[kNAThreads], sm[kNAThreads];
  double s = 0.0, m = 0.0;
  for (int b = threadIdx.x; b < kNABlocks; b += blockDim.x) {
    s += partials[2 * b];
    m = fmax(m, partials[2 * b + 1]);
  }
  ss[threadIdx.x] = s;
  sm[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0.0, tm = 0.0;
    for (int q = 0; q < kNAThreads; q++) {
      ts += ss[q];
      tm = fmax(tm, sm[q]);
    }
    out2[0] = sqrt(ts / (double)ncell);
    out2[1] = tm;
  }
}

// p is device memory of the current device `dev` (the kernels run there), or
// managed memory; device memory of another GPU is refused, since without peer
// access the kernels could not read it.
bool on_device(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

int fail(int status, const std::string &msg) {
  frmg_set_error(msg);
  return status;
}

}  // namespace

extern "C" int fr_residual_norm_noalloc(const double *u, const double *density,
                                        const int dims[3], double h, double box_mpc_h,
                                        double a, double omega_m, double fr0_abs,
                                        const double *ub, double *out2, void *stream) {
  if (!u || !density || !dims || !out2) return fail(FR_EINVAL, "NULL argument");
  for (int d = 0; d < 3; d++)
    if (dims[d] < 2 || (dims[d] & 1)) return fail(FR_EINVAL, "dims must be even and >= 2");
  if (!(h > 0)) return fail(FR_EINVAL, "h must be > 0");
  const long long ncell = (long long)dims[0] * dims[1] * dims[2];
  if (ncell > kNAMaxCells)
    return fail(FR_EINVAL, "grid of " + std::to_string(ncell) +
                               " cells exceeds the 33554432-cell limit of the allocation-free "
                               "residual norm");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(FR_ECUDA, "cudaGetDevice failed");
  }
  if (dev < 0 || dev >= kNAMaxDevices) return fail(FR_EINVAL, "device index out of range");
  if (!on_device(u, dev) || !on_device(density, dev) || !on_device(out2, dev) ||
      (ub && !on_device(ub, dev)))
    return fail(FR_EINVAL,
                "the allocation-free path takes device pointers of the current device only");
  // constants at cell size h: alpha scales as 1/h^2 from its value at h = 1
  double k6[6];
  int st = fr_constants(box_mpc_h, 1, a, omega_m, fr0_abs, k6);
  if (st != FR_OK) return st;
  NAGrid G;
  G.u = u;
  G.rho = density;
  G.ub = ub;
  G.n0 = dims[0];
  G.n1 = dims[1];
  G.n2 = dims[2];
  G.ncell = ncell;
  const long long fs[6] = {(long long)dims[1] * dims[2], (long long)dims[1] * dims[2],
                           (long long)dims[0] * dims[2], (long long)dims[0] * dims[2],
                           (long long)dims[0] * dims[1], (long long)dims[0] * dims[1]};
  long long o = 0;
  for (int f = 0; f < 6; f++) {
    G.foff[f] = o;
    o += fs[f];
  }
  G.ah = 0.5 * k6[0] / (h * h);
  G.beta = k6[1];
  G.gamma = k6[2];
  // one-time set-up per device (with that device current): device address of
  // the module's scratch array, valid for the life of the device's primary
  // context (cudaDeviceReset ends it; the header says so)
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_na_partials);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(FR_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      g_na_ptr[dev] = (double *)p;
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  k_na_partials<<<kNABlocks, kNAThreads, 0, s>>>(G, scratch);
  k_na_final<<<1, kNAThreads, 0, s>>>(scratch, ncell, out2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FR_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return FR_OK;
}
