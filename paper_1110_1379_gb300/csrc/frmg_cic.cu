// frmg_cic.cu -- cloud-in-cell density assignment (Sec. VI.C) for the solver.
//
// Each particle of mass n0 n1 n2 / np spreads over the 8 nearest cell centres
// (cell centres at (i + 1/2) h) with weights prod_d (1 - |x_d - x_c,d| / h_d),
// periodic, so that the mean of rho~ is 1 (Sec. III.A; the paper checks this
// mean in Sec. VI.C).
//
// GPU design: particles are processed in index order, one thread per particle.
// The 8 deposits go to global memory with FP64 atomics; consecutive particles
// of a Zel'dovich lattice map to neighbouring cells, so the atomics of a warp
// hit few cache lines in L2.
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

__global__ void k_cic(const double *__restrict__ pos, long long np, int n0, int n1, int n2,
                      double mass, double *__restrict__ rho, int *bad) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int n[3] = {n0, n1, n2};
  int i0[3];
  double t[3];
  // positions outside [0, 1) (or NaN) are reported and not deposited
#pragma unroll
  for (int d = 0; d < 3; d++) {
    double x = pos[3 * p + d];
    if (!(x >= 0.0 && x < 1.0)) {
      atomicExch(bad, 1);
      return;
    }
  }
#pragma unroll
  for (int d = 0; d < 3; d++) {
    double x = pos[3 * p + d];
    double xc = x * n[d] - 0.5;  // position in cell-centre units
    double fl = floor(xc);
    i0[d] = (int)fl;
    t[d] = xc - fl;
  }
  int lo[3], hi[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    lo[d] = i0[d] < 0 ? i0[d] + n[d] : (i0[d] >= n[d] ? i0[d] - n[d] : i0[d]);
    hi[d] = lo[d] + 1 == n[d] ? 0 : lo[d] + 1;
  }
#pragma unroll
  for (int s = 0; s < 8; s++) {
    int cx = (s & 1) ? hi[0] : lo[0];
    int cy = (s & 2) ? hi[1] : lo[1];
    int cz = (s & 4) ? hi[2] : lo[2];
    double w = mass * ((s & 1) ? t[0] : 1.0 - t[0]) * ((s & 2) ? t[1] : 1.0 - t[1]) *
               ((s & 4) ? t[2] : 1.0 - t[2]);
    atomicAdd(&rho[((long long)cz * n1 + cy) * n0 + cx], w);
  }
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

static int cic_impl(frmg_ctx *ctx, const double *pos, long long np, const int dims[3],
                    double *density_out, void *stream) {
  if (!ctx || !pos || !dims || !density_out || np <= 0) {
    frmg_set_error("bad argument");
    return FR_EINVAL;
  }
  for (int d = 0; d < 3; d++)
    if (dims[d] <= 0) {
      frmg_set_error("dims must be positive");
      return FR_EINVAL;
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
    k_cic<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(dpos, np, dims[0], dims[1], dims[2],
                                                       (double)nc / (double)np, drho, bad);
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
    return cic_impl(ctx, pos, np, dims, density_out, stream);
  } catch (...) {
    frmg_set_error("allocation failed");
    return FR_ENOMEM;
  }
}
