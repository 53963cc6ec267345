// oecdg_noalloc.cu -- cdg_oe_damp_noalloc: the OE step for callers that cannot
// allocate device memory.  Its scratch is a file-scope __device__ array that
// lives in the library's device image; no cudaMalloc / cudaFree is ever called.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/oecdg.h"
#include "oecdg_common.cuh"
#include "oecdg_kernels.h"

namespace oecdg {

// 1 MiB of scratch, shared by every call on a device (kept until exit).
// Layout in doubles: [0] tau, [1] tau_max slot (unused by the OE kernels),
// [2, 2 + 2F) sigma, [10, 10 + 2F) avg, [24] status word (an int),
// [NA_HDR, ...) sigma partials [2][nblk][F][3].
constexpr int NA_DOUBLES = 131072;
constexpr int NA_HDR = 64;
constexpr int NA_BLOCK = 256;  // cells per partial block
static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

constexpr int NA_MAX_DEVICES = 64;
static double* g_noalloc_ptr[NA_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

// Sigma partials of a state: per block of NA_BLOCK cells of one mesh and per
// field, (sum of cell averages, max and min of the values at the cell's Gauss
// points), the same quantities the stage kernels leave behind.
template <int F, int DIM>
__global__ void __launch_bounds__(NA_BLOCK) k_sigma_partials_na(Geo g, const double* __restrict__ u,
                                                                double* __restrict__ partials, long long nblk) {
  constexpr int M = DIM == 2 ? 9 : 3;
  __shared__ double sh[96];
  const int mesh = blockIdx.y;
  const long long cell = (long long)blockIdx.x * NA_BLOCK + threadIdx.x;
  const bool active = cell < g.plane;
  const double* us = u + (long long)mesh * F * M * g.plane + (active ? cell : 0);
  const double inf = __builtin_huge_val();
#pragma unroll
  for (int f = 0; f < F; ++f) {
    double v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = __ldg(us + (f * M + m) * g.plane);
    double mx = -inf, mn = inf;
    if (DIM == 2) {
#pragma unroll
      for (int qy = 0; qy < 3; ++qy) {
        double t[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = fma(lp(2, gnode(qy)), v[6 + a], fma(gnode(qy), v[3 + a], v[a]));
#pragma unroll
        for (int qx = 0; qx < 3; ++qx) {
          const double val = fma(lp(2, gnode(qx)), t[2], fma(gnode(qx), t[1], t[0]));
          mx = fmax(mx, val);
          mn = fmin(mn, val);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double val = fma(lp(2, gnode(q)), v[2], fma(gnode(q), v[1], v[0]));
        mx = fmax(mx, val);
        mn = fmin(mn, val);
      }
    }
    double s = active ? v[0] : 0.0;
    if (!active) {
      mx = -inf;
      mn = inf;
    }
    block_reduce3(s, mx, mn, sh);
    if (threadIdx.x == 0) {
      double* p = partials + ((mesh * nblk + blockIdx.x) * F + f) * 3;
      p[0] = s;
      p[1] = mx;
      p[2] = mn;
    }
  }
}

// Device address of the scratch array on the current device, looked up once
// and kept for the life of the process (a device reset would invalidate it;
// the header rules that use out).
static cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace oecdg

using namespace oecdg;

extern "C" cdg_status cdg_oe_damp_noalloc(const cdg_mesh_desc* desc, const double* d_uh, double tau, double* d_usig,
                                          void* stream) {
  if (!desc || !d_uh || !d_usig || d_uh == d_usig) return CDG_EINVAL;
  const cdg_mesh_desc& d = *desc;
  if (d.dim != 1 && d.dim != 2) return CDG_EINVAL;
  if (d.nx < 2 || (d.dim == 2 && d.ny < 2)) return CDG_EINVAL;
  if (invalid_sides(d)) return CDG_EINVAL;
  if (uniform_side_bc(d) < 0) return CDG_EUNSUPPORTED;  // per-side conditions and walls: context path only
  if (d.system != CDG_ADVECTION && d.system != CDG_EULER) return d.system == CDG_BURGERS ? CDG_EUNSUPPORTED : CDG_EINVAL;
  if (d.k != 2 || (d.dim == 2 && d.basis != CDG_BASIS_Q)) return CDG_EUNSUPPORTED;
  if (!(d.bx > d.ax) || (d.dim == 2 && !(d.by > d.ay))) return CDG_EINVAL;
  if (d.system == CDG_EULER && !(d.gamma > 1.0)) return CDG_EINVAL;
  if (!(tau >= 0.0)) return CDG_EINVAL;
  const int F = d.system == CDG_EULER ? d.dim + 2 : 1;
  const long long ny = d.dim == 2 ? d.ny : 1;
  const long long cells = (long long)d.nx * ny;
  const long long nblk = (cells + NA_BLOCK - 1) / NA_BLOCK;
  if (NA_HDR + 2 * nblk * F * 3 > NA_DOUBLES) return CDG_EINVAL;  // beyond the scratch limit

  double* s = nullptr;
  if (noalloc_scratch(&s) != cudaSuccess) return CDG_ECUDA;
  double* dt = s;
  double* sigma = s + 2;
  double* avg = s + 10;
  int* status = (int*)(s + 24);
  double* partials = s + NA_HDR;
  cudaStream_t st = (cudaStream_t)stream;

  Geo g;
  g.nx = d.nx;
  g.ny = (int)ny;
  geo_sides(d, g);  // uniform periodic or transmissive: no padding, plane = cells
  g.hx = (d.bx - d.ax) / d.nx;
  g.hy = d.dim == 2 ? (d.by - d.ay) / d.ny : 1.0;
  g.gamma = d.gamma;
  g.adv_x = d.adv_x;
  g.adv_y = d.adv_y;
  g.cfl = d.cfl;
  finish_geo(g);
  const int sys = d.system == CDG_EULER ? SYS_EULER : SYS_ADV;
  const int bc = uniform_side_bc(d) == CDG_PERIODIC ? BC_PERIODIC : BC_TRANSMISSIVE;

  // everything a previous call left behind is rewritten or cleared here
  if (launch_set2(dt, tau, 1.0, st) != cudaSuccess) return CDG_ECUDA;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return CDG_ECUDA;
  const dim3 grid((unsigned)nblk, 2);
  if (d.dim == 2) {
    if (F == 4) k_sigma_partials_na<4, 2><<<grid, NA_BLOCK, 0, st>>>(g, d_uh, partials, nblk);
    else k_sigma_partials_na<1, 2><<<grid, NA_BLOCK, 0, st>>>(g, d_uh, partials, nblk);
  } else {
    if (F == 3) k_sigma_partials_na<3, 1><<<grid, NA_BLOCK, 0, st>>>(g, d_uh, partials, nblk);
    else k_sigma_partials_na<1, 1><<<grid, NA_BLOCK, 0, st>>>(g, d_uh, partials, nblk);
  }
  if (cudaGetLastError() != cudaSuccess) return CDG_ECUDA;
  if (launch_sigma(partials, nblk, F, plain_norm(cells), sigma, avg, st) != cudaSuccess) return CDG_ECUDA;
  cudaError_t e = d.dim == 2 ? launch_oe2d(sys, bc, g, d_uh, d_usig, dt, sigma, nullptr, status, st)
                             : launch_oe1d(sys, bc, 2, g, d_uh, d_usig, dt, sigma, nullptr, status, st);
  return e == cudaSuccess ? CDG_OK : CDG_ECUDA;
}
