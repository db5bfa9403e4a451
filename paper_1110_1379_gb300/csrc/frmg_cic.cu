// frmg_cic.cu -- particle-mesh steps on either side of the solvers (Sec. VI.C):
// cloud-in-cell (CIC) and triangle-shaped-cloud (TSC) density assignment, and
// force interpolation with the same scheme as the assignment.
//
// Each particle of mass n0 n1 n2 / np spreads over the nearest cell centres
// (cell centres at (i + 1/2) h), periodic, so that the mean of rho~ is 1
// (Sec. III.A; the paper checks this mean in Sec. VI.C).  In cell-centre units
// x = pos n - 1/2:
//   CIC: cells floor(x), floor(x) + 1 per axis, weights 1 - t, t (t = x - floor(x));
//   TSC: cells c - 1, c, c + 1 with c = floor(x + 1/2), d = x - c, weights
//        (1/2 - d)^2 / 2, 3/4 - d^2, (1/2 + d)^2 / 2;
// 3D weights are products over the axes.  The force on a particle is -grad Phi
// (central differences on the grid) interpolated with the assignment weights
// (the same scheme on both sides conserves momentum).
//
// GPU design: particles are processed in index order, one thread per particle.
// The deposits go to global memory with FP64 atomics; consecutive particles
// of a Zel'dovich lattice map to neighbouring cells, so the atomics of a warp
// hit few cache lines in L2.  The force pass first forms the three gradient
// components on the grid (one thread per cell), then gathers them per particle.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "frmg.h"
#include "frmg_internal.h"

namespace {

__global__ void k_zero(double *p, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) p[t] = 0.0;
}

// Per axis: first cell (unwrapped) and weights of the scheme (K = 2: CIC, 3: TSC).
template <int K>
__device__ __forceinline__ void stencil1(double x, int &c0, double w[K]) {
  if (K == 2) {
    const double fl = floor(x);
    const double t = x - fl;
    c0 = (int)fl;
    w[0] = 1.0 - t;
    w[K - 1] = t;
  } else {
    const double c = floor(x + 0.5);
    const double d = x - c;
    c0 = (int)c - 1;
    w[0] = 0.5 * (0.5 - d) * (0.5 - d);
    w[1] = 0.75 - d * d;
    w[K - 1] = 0.5 * (0.5 + d) * (0.5 + d);
  }
}

__device__ __forceinline__ int wrapc(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

template <int K>
__global__ void k_assign(const double *__restrict__ pos, long long np, int n0, int n1, int n2,
                         double mass, double *__restrict__ rho, int *bad) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int n[3] = {n0, n1, n2};
  // positions outside [0, 1) (or NaN) are reported and not deposited
#pragma unroll
  for (int d = 0; d < 3; d++) {
    double x = pos[3 * p + d];
    if (!(x >= 0.0 && x < 1.0)) {
      atomicExch(bad, 1);
      return;
    }
  }
  int c0[3];
  double w[3][K];
#pragma unroll
  for (int d = 0; d < 3; d++) stencil1<K>(pos[3 * p + d] * n[d] - 0.5, c0[d], w[d]);
#pragma unroll
  for (int c = 0; c < K; c++) {
    const int cz = wrapc(c0[2] + c, n2);
#pragma unroll
    for (int b = 0; b < K; b++) {
      const int cy = wrapc(c0[1] + b, n1);
      const double wzy = mass * w[2][c] * w[1][b];
#pragma unroll
      for (int a = 0; a < K; a++) {
        const int cx = wrapc(c0[0] + a, n0);
        atomicAdd(&rho[((long long)cz * n1 + cy) * n0 + cx], wzy * w[0][a]);
      }
    }
  }
}

// Central-difference gradient of a periodic field, box units (h_d = 1/n_d).
__global__ void k_gradient(const double *__restrict__ phi, int n0, int n1, int n2,
                           double *__restrict__ gx, double *__restrict__ gy,
                           double *__restrict__ gz) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nc = (long long)n0 * n1 * n2;
  if (t >= nc) return;
  const int i = (int)(t % n0);
  const long long r = t / n0;
  const int j = (int)(r % n1), k = (int)(r / n1);
  const long long sy = n0, sz = (long long)n0 * n1;
  const long long xm = i > 0 ? t - 1 : t + (n0 - 1), xp = i < n0 - 1 ? t + 1 : t - (n0 - 1);
  const long long ym = j > 0 ? t - sy : t + (n1 - 1) * sy, yp = j < n1 - 1 ? t + sy : t - (n1 - 1) * sy;
  const long long zm = k > 0 ? t - sz : t + (n2 - 1) * sz, zp = k < n2 - 1 ? t + sz : t - (n2 - 1) * sz;
  gx[t] = (phi[xp] - phi[xm]) * (0.5 * n0);
  gy[t] = (phi[yp] - phi[ym]) * (0.5 * n1);
  gz[t] = (phi[zp] - phi[zm]) * (0.5 * n2);
}

// -grad Phi at each particle with the assignment weights of the scheme.
template <int K>
__global__ void k_forces(const double *__restrict__ gx, const double *__restrict__ gy,
                         const double *__restrict__ gz, const double *__restrict__ pos,
                         long long np, int n0, int n1, int n2, double *__restrict__ f,
                         int *bad) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int n[3] = {n0, n1, n2};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    double x = pos[3 * p + d];
    if (!(x >= 0.0 && x < 1.0)) {
      atomicExch(bad, 1);
      f[3 * p] = f[3 * p + 1] = f[3 * p + 2] = 0.0;
      return;
    }
  }
  int c0[3];
  double w[3][K];
#pragma unroll
  for (int d = 0; d < 3; d++) stencil1<K>(pos[3 * p + d] * n[d] - 0.5, c0[d], w[d]);
  double fx = 0.0, fy = 0.0, fz = 0.0;
#pragma unroll
  for (int c = 0; c < K; c++) {
    const int cz = wrapc(c0[2] + c, n2);
#pragma unroll
    for (int b = 0; b < K; b++) {
      const int cy = wrapc(c0[1] + b, n1);
      const double wzy = w[2][c] * w[1][b];
#pragma unroll
      for (int a = 0; a < K; a++) {
        const int cx = wrapc(c0[0] + a, n0);
        const long long q = ((long long)cz * n1 + cy) * n0 + cx;
        const double ww = wzy * w[0][a];
        fx -= ww * gx[q];
        fy -= ww * gy[q];
        fz -= ww * gz[q];
      }
    }
  }
  f[3 * p] = fx;
  f[3 * p + 1] = fy;
  f[3 * p + 2] = fz;
}

bool is_dev(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

static int assign_impl(frmg_ctx *ctx, const double *pos, long long np, const int dims[3],
                       double *density_out, void *stream, int tsc) {
  if (!ctx || !pos || !dims || !density_out || np <= 0) {
    frmg_set_error("bad argument");
    return FR_EINVAL;
  }
  for (int d = 0; d < 3; d++)
    if (dims[d] <= 0) {
      frmg_set_error("dims must be positive");
      return FR_EINVAL;
    }
  if (cudaSetDevice(frmg_device(ctx)) != cudaSuccess) {
    cudaGetLastError();
    frmg_set_error("cudaSetDevice failed");
    return FR_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  long long nc = (long long)dims[0] * dims[1] * dims[2];
  const double *dpos = pos;
  double *drho = density_out;
  void *tmp_pos = nullptr, *tmp_rho = nullptr;
  int *bad = nullptr;
  int status = FR_OK;
  auto fail = [&](int s, const std::string &m) {
    status = s;
    frmg_set_error(m);
  };
  if (!is_dev(pos)) {
    tmp_pos = frmg_alloc(ctx, np * 3 * sizeof(double));
    if (cudaMemcpyAsync(tmp_pos, pos, np * 3 * sizeof(double), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      fail(FR_ECUDA, "copy of positions failed");
    dpos = (const double *)tmp_pos;
  }
  if (!is_dev(density_out)) {
    tmp_rho = frmg_alloc(ctx, nc * sizeof(double));
    drho = (double *)tmp_rho;
  }
  bad = (int *)frmg_alloc(ctx, sizeof(int));
  if (status == FR_OK) {
    cudaMemsetAsync(bad, 0, sizeof(int), st);
    k_zero<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(drho, nc);
    frmg_launch_counter(ctx)++;
    if (tsc)
      k_assign<3><<<(unsigned)((np + 255) / 256), 256, 0, st>>>(
          dpos, np, dims[0], dims[1], dims[2], (double)nc / (double)np, drho, bad);
    else
      k_assign<2><<<(unsigned)((np + 255) / 256), 256, 0, st>>>(
          dpos, np, dims[0], dims[1], dims[2], (double)nc / (double)np, drho, bad);
    frmg_launch_counter(ctx)++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(FR_ECUDA, cudaGetErrorString(e));
  }
  int hb = 0;
  if (status == FR_OK) {
    if (cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      fail(FR_ECUDA, "readback failed");
    if (tmp_rho && status == FR_OK &&
        cudaMemcpyAsync(density_out, drho, nc * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
      fail(FR_ECUDA, "copy of density failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) fail(FR_ECUDA, "stream synchronize failed");
  }
  if (status == FR_OK && hb) fail(FR_EINVAL, "particle positions must lie in [0, 1)");
  frmg_release(ctx, tmp_pos);
  frmg_release(ctx, tmp_rho);
  frmg_release(ctx, bad);
  return status;
}

extern "C" int fr_cic_assign(frmg_ctx *ctx, const double *pos, long long np, const int dims[3],
                             double *density_out, void *stream) {
  try {
    return assign_impl(ctx, pos, np, dims, density_out, stream, 0);
  } catch (...) {
    frmg_set_error("allocation failed");
    return FR_ENOMEM;
  }
}

extern "C" int fr_tsc_assign(frmg_ctx *ctx, const double *pos, long long np, const int dims[3],
                             double *density_out, void *stream) {
  try {
    return assign_impl(ctx, pos, np, dims, density_out, stream, 1);
  } catch (...) {
    frmg_set_error("allocation failed");
    return FR_ENOMEM;
  }
}

extern "C" int fr_particle_forces(frmg_ctx *ctx, const double *phi, const int dims[3],
                                  const double *pos, long long np, int scheme,
                                  double *force_out, void *stream) {
  if (!ctx || !phi || !dims || !pos || !force_out || np <= 0 ||
      (scheme != FR_SCHEME_CIC && scheme != FR_SCHEME_TSC)) {
    frmg_set_error("bad argument");
    return FR_EINVAL;
  }
  for (int d = 0; d < 3; d++)
    if (dims[d] < 3) {
      frmg_set_error("dims must be at least 3");
      return FR_EINVAL;
    }
  if (cudaSetDevice(frmg_device(ctx)) != cudaSuccess) {
    cudaGetLastError();
    frmg_set_error("cudaSetDevice failed");
    return FR_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long long nc = (long long)dims[0] * dims[1] * dims[2];
  std::vector<void *> tmp;
  int status = FR_OK;
  try {
    auto get = [&](size_t bytes) {
      void *p = frmg_alloc(ctx, bytes);
      tmp.push_back(p);
      return p;
    };
    auto fail = [&](int s, const std::string &m) {
      if (status == FR_OK) {
        status = s;
        frmg_set_error(m);
      }
    };
    const double *dphi = phi, *dpos = pos;
    if (!is_dev(phi)) {
      double *d = (double *)get(nc * sizeof(double));
      if (cudaMemcpyAsync(d, phi, nc * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
        fail(FR_ECUDA, "copy of phi failed");
      dphi = d;
    }
    if (!is_dev(pos)) {
      double *d = (double *)get(np * 3 * sizeof(double));
      if (cudaMemcpyAsync(d, pos, np * 3 * sizeof(double), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
        fail(FR_ECUDA, "copy of positions failed");
      dpos = d;
    }
    const bool fdev = is_dev(force_out);
    double *df = fdev ? force_out : (double *)get(np * 3 * sizeof(double));
    double *g = (double *)get(3 * nc * sizeof(double));
    int *bad = (int *)get(sizeof(int));
    if (status == FR_OK) {
      cudaMemsetAsync(bad, 0, sizeof(int), st);
      k_gradient<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(dphi, dims[0], dims[1], dims[2],
                                                                g, g + nc, g + 2 * nc);
      frmg_launch_counter(ctx)++;
      if (scheme == FR_SCHEME_TSC)
        k_forces<3><<<(unsigned)((np + 255) / 256), 256, 0, st>>>(
            g, g + nc, g + 2 * nc, dpos, np, dims[0], dims[1], dims[2], df, bad);
      else
        k_forces<2><<<(unsigned)((np + 255) / 256), 256, 0, st>>>(
            g, g + nc, g + 2 * nc, dpos, np, dims[0], dims[1], dims[2], df, bad);
      frmg_launch_counter(ctx)++;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) fail(FR_ECUDA, cudaGetErrorString(e));
    }
    int hb = 0;
    if (status == FR_OK) {
      if (cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        fail(FR_ECUDA, "readback failed");
      if (!fdev && status == FR_OK &&
          cudaMemcpyAsync(force_out, df, np * 3 * sizeof(double), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess)
        fail(FR_ECUDA, "copy of forces failed");
      if (cudaStreamSynchronize(st) != cudaSuccess) fail(FR_ECUDA, "stream synchronize failed");
    }
    if (status == FR_OK && hb) fail(FR_EINVAL, "particle positions must lie in [0, 1)");
  } catch (...) {
    cudaStreamSynchronize(st);
    for (void *p : tmp) frmg_release(ctx, p);
    frmg_set_error("allocation failed");
    return FR_ENOMEM;
  }
  for (void *p : tmp) frmg_release(ctx, p);
  return status;
}
