// oecdg_2d.cu -- 2D Q^2 kernels of the OECDG forward step (arXiv:2503.12473):
// launch wrappers around the per-cell code of oecdg_2d_body.cuh.
#include "oecdg_2d_body.cuh"
#include "oecdg_kernels.h"
#include "oecdg_persist.cuh"

namespace oecdg {

#ifndef OECDG_TY
#define OECDG_TY 4
#endif
#ifndef OECDG_STAGE_MINB
#define OECDG_STAGE_MINB 1
#endif
#ifndef OECDG_OE_MINB
#define OECDG_OE_MINB 1
#endif
constexpr int TX = 32, TY = OECDG_TY, NT = TX * TY;  // cell tile of one block

// MODE_RHS: out = L(uin) with tau_max = dt[1].
// MODE_STAGE: out = ca un + cb (uin + tau L(uin)) with (tau, tau_max) = dt[0..1],
//   plus per-block partials of the sigma reduction of the output:
//   partials[(mesh * nblk + blk) * F * 3 + f * 3 + {0,1,2}] = (sum of cell
//   averages, max and min of the values at the cell's 3x3 Gauss points).
template <int SYS, int BC, int MODE>
__global__ void __launch_bounds__(NT, OECDG_STAGE_MINB) k_stage2d(Geo g, const double* __restrict__ uin,
                                                const double* __restrict__ un, double* __restrict__ out,
                                                const double* __restrict__ dt, double ca, double cb,
                                                double* __restrict__ partials) {
  constexpr int F = Fields<SYS>::F;
  const int mesh = blockIdx.x & 1, bx = blockIdx.x >> 1, tx = gridDim.x >> 1;
  const long long nblk = (long long)tx * gridDim.y;
  const long long blk = (long long)blockIdx.y * tx + bx;
  stage_cell2d<SYS, BC, MODE>(g, uin, un, out, dt, ca, cb, partials + (mesh * nblk + blk) * F * 3, mesh,
                              bx * TX + (threadIdx.x % TX), blockIdx.y * TY + (threadIdx.x / TX));
}

// Fixed-order reduction of the block partials: avg and sigma per mesh and
// field (Section 2.2): avg = mean of the cell averages over the stored cells,
// sigma = max(max - avg, avg - min) over the cell Gauss points.  grid = (F, 2),
// 256 threads each (block_sigma): the same summation order, bit for bit, as the
// one warp per (mesh, field) of the persistent kernels' sigma phase.
__global__ void k_sigma(const double* __restrict__ partials, long long nblk, int F, SigmaNorm sn,
                        double* __restrict__ sigma, double* __restrict__ avg) {
  block_sigma<LD_NC>(partials, nblk, F, blockIdx.y, blockIdx.x, sn, avg, sigma);
}

// ---------------------------------------------------------------- OE step --

// Damping coefficients delta_K^m (m = 0, 1, 2) of one cell and the exact OE
// step (Eq. (OEstep2D)).  For each field and each half-face e of K (k+1 = 3
// Gauss points): the derivatives d^alpha (u^C - u^D), |alpha| <= 2, from K's own
// interior trace and the overlapping cell (which is smooth across e);
//   int_e |u^C - u^D|,  int_e (D_x^2 + D_y^2)^{1/2},  int_e (D_xx^2 + D_xy^2 + D_yy^2)^{1/2}.
// delta^m = sum_e beta_e (2m+1) h_e^{m-1} / ((2k-1) m! sigma |e|) int_e ..., max
// over fields (Remark on systems); delta = 0 where sigma = 0.  Mode (a,b) then
// decays by exp(-tau sum_{m <= min(a+b, 2)} delta^m), the average is kept.
// Damping coefficients and the exact OE step of every cell (oe_cell2d).
template <int SYS, int BC, bool WRITE_DELTA, bool ISO>
__global__ void __launch_bounds__(NT, OECDG_OE_MINB) k_oe2d(Geo g, const double* __restrict__ uh, double* __restrict__ usig,
                                             const double* __restrict__ dt, const double* __restrict__ sigma,
                                             double* __restrict__ delta_out, int* __restrict__ status) {
  __shared__ double isg[Fields<SYS>::F];
  __shared__ double osh[2 * TY * TX * OSER_N];  // the rows' shared y-face series
  oe_inv_sigma<Fields<SYS>::F>(sigma, blockIdx.x & 1, isg);
  oe_cell2d<SYS, BC, WRITE_DELTA, 0, ISO, LD_NC, TY>(g, uh, usig, dt, sigma, delta_out, status, blockIdx.x & 1,
                                                     (blockIdx.x >> 1) * TX + (threadIdx.x % TX),
                                                     blockIdx.y * TY + (threadIdx.x / TX), nullptr, isg, osh,
                                                     threadIdx.x / TX);
}

// ------------------------------------------------------------- time step --

// Per-block maximum wave speeds over the cell averages of both meshes.
// partial[blk * 2 + {0,1}] = (max |u| + c, max |v| + c) (advection: |a_x|, |a_y|).
template <int SYS>
__global__ void k_wave2d(Geo g, const double* __restrict__ u, double* __restrict__ partial, int* __restrict__ status) {
  constexpr int F = Fields<SYS>::F;
  __shared__ double sh[32];
  const long long n = 2 * g.plane;
  double mx = 0.0, my = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    const double* us = u + (long long)mesh * F * 9 * g.plane + cell;
    if (SYS == SYS_EULER) {
      double bx, by;
      if (euler2_wave(g.gamma, us[0], us[9 * g.plane], us[18 * g.plane], us[27 * g.plane], bx, by)) {
        mx = fmax(mx, bx);
        my = fmax(my, by);
      } else {
        atomicOr(status, ST_NONPHYSICAL);
      }
    } else {
      mx = fabs(g.adv_x);
      my = fabs(g.adv_y);
    }
  }
  mx = block_reduce_max(mx, sh);
  __syncthreads();
  my = block_reduce_max(my, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 2] = mx;
    partial[blockIdx.x * 2 + 1] = my;
  }
}

// One block: the maxima of the block partials (exact in any order), then
// finish_dt (tau_max, the clipped tau, the time) by thread 0.
__global__ void k_dt_final(const double* __restrict__ partial, int nblk, double hx, double hy, int dim, double cfl,
                           double T_end, double* __restrict__ dt, double* __restrict__ time) {
  __shared__ double sh[32];
  double bx = 0.0, by = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    bx = fmax(bx, partial[2 * b]);
    by = fmax(by, partial[2 * b + 1]);
  }
  bx = block_reduce_max(bx, sh);
  __syncthreads();
  by = block_reduce_max(by, sh);
  if (threadIdx.x == 0) finish_dt(bx, by, hx, hy, dim, cfl, T_end, dt, time);
}

__global__ void k_set2(double* __restrict__ p, double a, double b) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    p[0] = a;
    p[1] = b;
  }
}

// ------------------------------------------------------ initial projection --

// Composite-Gauss sampling points, layout [mesh][j][i][sy][sx][qy][qx] (x, y).
__global__ void k_points2d(Geo g, double ax, double ay, double* __restrict__ xy) {
  const long long n = 2 * g.plane * 36;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % 36);
    const long long c = t / 36;
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    const int j = (int)(cell / g.nx), i = (int)(cell - (long long)j * g.nx);
    const int qx = r % 3, qy = (r / 3) % 3, sx = (r / 9) % 2, sy = r / 18;
    const double xc = ax + (i + 0.5 + 0.5 * mesh) * g.hx, yc = ay + (j + 0.5 + 0.5 * mesh) * g.hy;
    xy[2 * t] = xc + 0.5 * g.hx * xs_self(sx, qx);
    xy[2 * t + 1] = yc + 0.5 * g.hy * xs_self(sy, qy);
  }
}

// u_ab = (2a+1)(2b+1)/4 * sum over the 4 sub-cells and their 3x3 points of
// (w_qx/2)(w_qy/2) u0 P_a(xi) P_b(eta).
template <int F>
__global__ void k_project2d(Geo g, const double* __restrict__ vals, double* __restrict__ u) {
  const long long n = 2 * g.plane;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    double acc[F][9];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int m = 0; m < 9; ++m) acc[f][m] = 0.0;
    const double* v = vals + c * 36 * F;
#pragma unroll
    for (int r = 0; r < 36; ++r) {
      const int qx = r % 3, qy = (r / 3) % 3, sx = (r / 9) % 2, sy = r / 18;
      const double xi = xs_self(sx, qx), eta = xs_self(sy, qy);
      const double w = 0.25 * gwt(qx) * gwt(qy);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const double x = w * v[r * F + f];
#pragma unroll
        for (int m = 0; m < 9; ++m) acc[f][m] = fma(x, lp(m % 3, xi) * lp(m / 3, eta), acc[f][m]);
      }
    }
    double* o = u + (long long)mesh * F * 9 * g.plane + cell;
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int m = 0; m < 9; ++m) o[(f * 9 + m) * g.plane] = acc[f][m] * ((2 * (m % 3) + 1) * (2 * (m / 3) + 1) / 4.0);
  }
}

// ----------------------------------------------------------------- launch --

// The two meshes' blocks of a tile are adjacent in launch order (mesh =
// blockIdx.x & 1), so the cells a block reads from the other mesh were just
// read by its partner block and are still in L2: each state is read from DRAM
// about once per launch instead of once per mesh.
static inline dim3 tile_grid(const Geo& g) { return dim3(2 * ((g.nx + TX - 1) / TX), (g.ny + TY - 1) / TY, 1); }

long long partial_blocks_2d(const Geo& g) { return (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY); }

template <int SYS, int BC>
static cudaError_t stage2d_t(const Geo& g, int mode, const double* uin, const double* un, double* out, const double* dt,
                             double ca, double cb, double* partials, cudaStream_t st) {
  if (mode == MODE_RHS)
    k_stage2d<SYS, BC, MODE_RHS><<<tile_grid(g), NT, 0, st>>>(g, uin, un, out, dt, ca, cb, partials);
  else
    k_stage2d<SYS, BC, MODE_STAGE><<<tile_grid(g), NT, 0, st>>>(g, uin, un, out, dt, ca, cb, partials);
  return cudaGetLastError();
}

cudaError_t launch_stage2d(int sys, int bc, const Geo& g, int rhs_only, const double* uin, const double* un,
                           double* out, const double* dt, double ca, double cb, double* partials, cudaStream_t st) {
  const int mode = rhs_only ? MODE_RHS : MODE_STAGE;
  if (sys == SYS_EULER)
    return bc == BC_PERIODIC ? stage2d_t<SYS_EULER, BC_PERIODIC>(g, mode, uin, un, out, dt, ca, cb, partials, st)
                             : stage2d_t<SYS_EULER, BC_TRANSMISSIVE>(g, mode, uin, un, out, dt, ca, cb, partials, st);
  return bc == BC_PERIODIC ? stage2d_t<SYS_ADV, BC_PERIODIC>(g, mode, uin, un, out, dt, ca, cb, partials, st)
                           : stage2d_t<SYS_ADV, BC_TRANSMISSIVE>(g, mode, uin, un, out, dt, ca, cb, partials, st);
}

cudaError_t launch_sigma(const double* partials, long long nblk, int F, const SigmaNorm& sn, double* sigma,
                         double* avg, cudaStream_t st) {
  k_sigma<<<dim3(F, 2), 256, 0, st>>>(partials, nblk, F, sn, sigma, avg);
  return cudaGetLastError();
}

template <int SYS, int BC>
static cudaError_t oe2d_t(const Geo& g, const double* uh, double* usig, const double* dt, const double* sigma,
                          double* delta, int* status, cudaStream_t st) {
  // square cells: the isotropic variant of the OE body (same result up to rounding)
  const bool iso = g.hx == g.hy;
  if (delta && iso)
    k_oe2d<SYS, BC, true, true><<<tile_grid(g), NT, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
  else if (delta)
    k_oe2d<SYS, BC, true, false><<<tile_grid(g), NT, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
  else if (iso)
    k_oe2d<SYS, BC, false, true><<<tile_grid(g), NT, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
  else
    k_oe2d<SYS, BC, false, false><<<tile_grid(g), NT, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
  return cudaGetLastError();
}

cudaError_t launch_oe2d(int sys, int bc, const Geo& g, const double* uh, double* usig, const double* dt,
                        const double* sigma, double* delta, int* status, cudaStream_t st) {
  if (sys == SYS_EULER)
    return bc == BC_PERIODIC ? oe2d_t<SYS_EULER, BC_PERIODIC>(g, uh, usig, dt, sigma, delta, status, st)
                             : oe2d_t<SYS_EULER, BC_TRANSMISSIVE>(g, uh, usig, dt, sigma, delta, status, st);
  return bc == BC_PERIODIC ? oe2d_t<SYS_ADV, BC_PERIODIC>(g, uh, usig, dt, sigma, delta, status, st)
                           : oe2d_t<SYS_ADV, BC_TRANSMISSIVE>(g, uh, usig, dt, sigma, delta, status, st);
}

int wave_blocks_2d(const Geo& g) {
  const long long n = 2 * g.plane;
  long long b = (n + 255) / 256;
  return (int)(b < 1184 ? b : 1184);
}

cudaError_t launch_dt2d(int sys, const Geo& g, const double* u, double* partial, int nblk, double T_end,
                        double* dt, double* time, int* status, cudaStream_t st) {
  if (sys == SYS_EULER) k_wave2d<SYS_EULER><<<nblk, 256, 0, st>>>(g, u, partial, status);
  else k_wave2d<SYS_ADV><<<nblk, 256, 0, st>>>(g, u, partial, status);
  k_dt_final<<<1, 256, 0, st>>>(partial, nblk, g.hx, g.hy, 2, g.cfl, T_end, dt, time);
  return cudaGetLastError();
}

cudaError_t launch_dt_final(const double* partial, int nblk, double hx, double hy, int dim, double cfl, double T_end,
                            double* dt, double* time, cudaStream_t st) {
  k_dt_final<<<1, 256, 0, st>>>(partial, nblk, hx, hy, dim, cfl, T_end, dt, time);
  return cudaGetLastError();
}

cudaError_t launch_set2(double* p, double a, double b, cudaStream_t st) {
  k_set2<<<1, 32, 0, st>>>(p, a, b);
  return cudaGetLastError();
}

cudaError_t launch_points2d(const Geo& g, double ax, double ay, double* xy, cudaStream_t st) {
  k_points2d<<<1184, 256, 0, st>>>(g, ax, ay, xy);
  return cudaGetLastError();
}

cudaError_t launch_project2d(int sys, const Geo& g, const double* vals, double* u, cudaStream_t st) {
  if (sys == SYS_EULER) k_project2d<4><<<1184, 128, 0, st>>>(g, vals, u);
  else k_project2d<1><<<1184, 128, 0, st>>>(g, vals, u);
  return cudaGetLastError();
}

}  // namespace oecdg
