// oecdg_common.cuh -- device constants and helpers of the OECDG CUDA path
// (arXiv:2503.12473).  Degree k = 2: 3-point Gauss-Legendre rule, unnormalised
// Legendre polynomials P_0 = 1, P_1 = x, P_2 = (3x^2 - 1)/2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace oecdg {

enum { SYS_ADV = 0, SYS_BURGERS = 1, SYS_EULER = 2 };
// Boundary handling of a kernel: BC_PERIODIC / BC_TRANSMISSIVE on every side
// (compile-time), or BC_GENERAL: each side's condition read from Geo::bcs at
// run time (periodic in pairs, transmissive, or a reflective wall).
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_GENERAL = 2 };
enum { SIDE_PERIODIC = 0, SIDE_TRANSMISSIVE = 1, SIDE_REFLECTIVE = 2 };
enum { BASIS_Q = 0, BASIS_P = 1 };

// status bits written by kernels
enum { ST_NONPHYSICAL = 1 };

// sigma_K of one (mesh, field) (Section 2.2): ||u_h - avg(u_h)||_inf over the
// domain, from the maximum mx and the minimum mn of the point values and the
// domain average a, = max(mx - a, a - mn).  The OE coefficients divide by it
// and vanish where it is 0, which in exact arithmetic is a constant field.  A
// field that is constant up to rounding (the uniform density of a blast-wave
// start: every point value within an ulp or two of 1) instead has a sigma of a
// few ulps, whose value depends on how the average was rounded, and jumps of
// the same size: their ratio would damp every field of every cell as hard as a
// shock.  So a sigma at or below 2^-40 of the field's magnitude
// max(|mx|, |mn|) (4096 ulps) counts as 0.
constexpr double SIGMA_FLOOR = 0x1p-40;

__host__ __device__ __forceinline__ double sigma_from_range(double mx, double mn, double a) {
  const double s = fmax(mx - a, a - mn);
  return s <= SIGMA_FLOOR * fmax(fabs(mx), fabs(mn)) ? 0.0 : s;
}

// 3-point Gauss-Legendre rule on [-1, 1]: nodes -sqrt(3/5), 0, sqrt(3/5),
// weights 5/9, 8/9, 5/9.
constexpr double GQ = 0.77459666924148337704;  // sqrt(3/5)

__host__ __device__ constexpr double gnode(int q) { return q == 0 ? -GQ : (q == 1 ? 0.0 : GQ); }
__host__ __device__ constexpr double gwt(int q) { return q == 1 ? (8.0 / 9.0) : (5.0 / 9.0); }

// Legendre P_n and derivatives (n <= 2)
__host__ __device__ constexpr double lp(int n, double x) { return n == 0 ? 1.0 : (n == 1 ? x : 1.5 * x * x - 0.5); }
__host__ __device__ constexpr double dlp(int n, double x) { return n == 0 ? 0.0 : (n == 1 ? 1.0 : 3.0 * x); }
__host__ __device__ constexpr double ddlp(int n) { return n == 2 ? 3.0 : 0.0; }

// Points of sub-cell s (s = 0: [-1, 0], s = 1: [0, 1]) in the cell's own
// reference coordinate, and the same physical points in the overlapping cell of
// the other mesh (its centre sits on this cell's face: xi' = xi + 1 - 2s).
__host__ __device__ constexpr double xs_self(int s, int q) { return s - 0.5 + 0.5 * gnode(q); }
__host__ __device__ constexpr double xs_other(int s, int q) { return 0.5 - s + 0.5 * gnode(q); }

template <int BC>
__device__ __forceinline__ int wrap_index(int i, int n) {
  if (BC == BC_PERIODIC) return i < 0 ? i + n : (i >= n ? i - n : i);
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// FP64 reciprocal and square root of the hot loops.  The seed is the PTX
// approximation computed from the upper 32 bits of the input
// (rcp.approx.ftz.f64, rsqrt.approx.ftz.f64; their residuals e below measure
// at most 2^-19.9 and 2^-19.0 on GB300); one higher-order Newton-Raphson step
// (the iterations for division and square root in J.-M. Muller et al.,
// Handbook of Floating-Point Arithmetic, Birkhauser, 2nd ed. 2018) then
// multiplies it by the Taylor series, in the seed's residual e, of
//   1/x      = y / (1 - e),          e = 1 - x y,
//   sqrt(x)  = s / (1 - e)^(1/2),    s = x y,  e = 1 - s y,
// cut after e^2.  The remainders, e^3 resp. 5e^3/16, stay below 2^-58
// relative, so the results are within about 1 ulp (3 resp. 5 FP64
// instructions after the seed).
//   rcp_pos: within 1 ulp for every normal x of EITHER sign whose reciprocal
//     is normal, 2^-1022 <= |x| <= 2^1022 (the seed and the correction are odd
//     in x, so rcp_pos(-x) = -rcp_pos(x) exactly).  The Euler flux calls it on
//     point densities, which can be negative in discontinuous runs (the paper
//     uses no limiter for them); |x| < 2^-1022 (zero or subnormal) or infinite
//     x give NaN where IEEE division gives +-inf or 0, and |x| > 2^1022 gives 0
//     where it gives a subnormal: a point density that small leaves the flux
//     undefined either way.
//   sqrt_pos: within 1 ulp for normal x > 0; callers add SQ_FLOOR into the
//     sum of squares they pass, which makes a zero sum cost nothing extra and
//     moves a nonzero one by at most 1e-300.
constexpr double SQ_FLOOR = 1e-300;

__device__ __forceinline__ double rcp_pos(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);  // y (1 + e + e^2)
}

__device__ __forceinline__ double sqrt_pos(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double s = x * y;
  const double e = fma(-s, y, 1.0);
  return fma(s * e, fma(0.375, e, 0.5), s);  // s (1 + e/2 + 3e^2/8)
}

// Geometry and physics constants passed by value to every kernel.
//   nx, ny:   primal cells per direction;
//   nxs, nys: stored cells per row / rows of BOTH meshes' planes (the padded
//             layout): nx, ny, plus one where a reflective wall on the low side
//             gives the dual mesh the cell centred on that wall (stored in the
//             slot after its last cell; the primal mesh leaves the slot unused);
//   plane:    nxs * nys;
//   bcs:      per side (x-low, x-high, y-low, y-high): SIDE_PERIODIC,
//             SIDE_TRANSMISSIVE or SIDE_REFLECTIVE (read by BC_GENERAL kernels);
//   i1x ...:  constants of the cell size that the per-cell code of the 2D OE
//             kernels needs, set once on the host by finish_geo, so that no
//             thread divides (an IEEE quotient has the same bits on either
//             side): 1/hx, 1/hy, 2/hx, 2/hy, 1/(12 hx), 1/(12 hy), 5 hx/24,
//             5 hy/24.  (The stage kernels keep their own quotients: taken from
//             here they left the times unchanged or slower, with more of the
//             tiled kernel's register spills reaching DRAM.)
struct Geo {
  int nx, ny;
  long long plane;
  double hx, hy;
  double gamma;
  double adv_x, adv_y;
  double cfl;
  int nxs, nys;
  int bcs[4];
  double i1x, i1y, i2x, i2y, i12x, i12y, h24x5, h24y5;
};

// The cell-size constants of Geo, from hx and hy (the same expressions the
// per-cell code would evaluate).
inline void finish_geo(Geo& g) {
  g.i1x = 1.0 / g.hx;
  g.i1y = 1.0 / g.hy;
  g.i2x = 2.0 / g.hx;
  g.i2y = 2.0 / g.hy;
  g.i12x = 1.0 / (12.0 * g.hx);
  g.i12y = 1.0 / (12.0 * g.hy);
  g.h24x5 = 5.0 * g.hx / 24.0;
  g.h24y5 = 5.0 * g.hy / 24.0;
}

// 1/sigma of the F fields of `mesh` into shared isg[F] by the block's first
// threads (the same IEEE quotient the cell code would take), then a barrier:
// every thread of the block must call it.  The load goes to L2 (ld.global.cg),
// so a persistent kernel may call it on sigma written earlier in the launch.
template <int F>
__device__ __forceinline__ void oe_inv_sigma(const double* sigma, int mesh, double* isg) {
  if (threadIdx.x < F) {
    const double sg = __ldcg(sigma + mesh * F + threadIdx.x);
    isg[threadIdx.x] = sg != 0.0 ? 1.0 / sg : 0.0;
  }
  __syncthreads();
}

// Stored cells of mesh `mesh` per direction (the dual mesh has the wall slots).
__host__ __device__ __forceinline__ int cells_x(const Geo& g, int mesh) { return mesh == 0 ? g.nx : g.nxs; }
__host__ __device__ __forceinline__ int cells_y(const Geo& g, int mesh) { return mesh == 0 ? g.ny : g.nys; }

// Unwrapped index of cell i of mesh `mesh` in direction dir: primal cell iu
// spans [iu h, (iu+1) h], dual cell iu is centred on vertex iu + 1; the dual
// slot after the last cell holds the cell centred on vertex 0 (iu = -1).
__host__ __device__ __forceinline__ int unwrapped(const Geo& g, int dir, int mesh, int i) {
  return (mesh == 1 && i == (dir == 0 ? g.nx : g.ny)) ? -1 : i;
}

// Stored index of the cell of mesh `mesh` with unwrapped index iu in direction
// dir, under the per-side conditions; *mirror = true for the mirror image of a
// stored cell across a reflective wall (primal -1 - iu / 2n - 1 - iu, dual
// vertex v -> -v / 2n - v).  Only one cell beyond a side is ever asked for.
__device__ __forceinline__ int side_index(const Geo& g, int dir, int mesh, int iu, bool& mirror) {
  const int n = dir == 0 ? g.nx : g.ny;
  const int lo = g.bcs[2 * dir], hi = g.bcs[2 * dir + 1];
  mirror = false;
  if (iu >= 0 && iu < n) return iu;
  if (lo == SIDE_PERIODIC) return iu < 0 ? iu + n : iu - n;
  if (iu < 0) {
    if (lo == SIDE_TRANSMISSIVE) return 0;
    if (mesh == 1 && iu == -1) return n;  // the wall-centred dual cell
    mirror = true;
    iu = mesh == 0 ? -1 - iu : -iu - 2;
  } else {
    if (hi == SIDE_TRANSMISSIVE) return n - 1;
    mirror = true;
    iu = mesh == 0 ? 2 * n - 1 - iu : 2 * n - iu - 2;
  }
  return iu < 0 ? 0 : (iu >= n ? n - 1 : iu);
}

// Sign bit to apply to coefficient (field f, mode degrees (a, b)) of a mirror
// image: the mirror across a wall normal to x negates the odd-in-x modes and
// the x-momentum (Euler: field 1), likewise for y (field 2 in 2D).
__device__ __forceinline__ unsigned long long mirror_sign(bool mx, bool my, bool euler, int f, int a, int b) {
  const int neg = (mx ? ((a & 1) ^ (euler && f == 1)) : 0) ^ (my ? ((b & 1) ^ (euler && f == 2)) : 0);
  return neg ? 0x8000000000000000ULL : 0ULL;
}
__device__ __forceinline__ double apply_sign(double v, unsigned long long sgn) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)sgn);
}

// Weight of a cell in the domain average (sigma, avg): halved for each
// reflective wall a dual cell is centred on (the mirror-extended domain holds
// it once, every other cell twice).
__host__ __device__ __forceinline__ double cell_weight(const Geo& g, int mesh, int i, int j, int dim) {
  if (mesh == 0) return 1.0;
  double w = 1.0;
  if ((g.bcs[0] == SIDE_REFLECTIVE && i == g.nx) || (g.bcs[1] == SIDE_REFLECTIVE && i == g.nx - 1)) w *= 0.5;
  if (dim == 2 && ((g.bcs[2] == SIDE_REFLECTIVE && j == g.ny) || (g.bcs[3] == SIDE_REFLECTIVE && j == g.ny - 1)))
    w *= 0.5;
  return w;
}

// 2D Euler flux components at a conserved state (rho, mx, my, E).  Every
// multiply-add is an explicit fma, E + p included (written as one, not left to
// the compiler): its own contraction may differ between the kernels that
// inline these (single-mesh, batched, persistent, recording), whose results
// must agree bit for bit.
struct Euler2 {
  __device__ static __forceinline__ void both(const double* w, double g, double* f1, double* f2) {
    const double r = rcp_pos(w[0]);
    const double vx = w[1] * r, vy = w[2] * r;
    const double e = fma(-0.5, fma(w[1], vx, w[2] * vy), w[3]);  // E - kinetic energy
    const double p = (g - 1.0) * e;
    const double H = fma(g - 1.0, e, w[3]);  // E + p, one rounding
    f1[0] = w[1];
    f1[1] = fma(w[1], vx, p);
    f1[2] = w[2] * vx;
    f1[3] = H * vx;
    f2[0] = w[2];
    f2[1] = f1[2];
    f2[2] = fma(w[2], vy, p);
    f2[3] = H * vy;
  }
  __device__ static __forceinline__ void fx(const double* w, double g, double* f1) {
    const double r = rcp_pos(w[0]);
    const double vx = w[1] * r, vy = w[2] * r;
    const double e = fma(-0.5, fma(w[1], vx, w[2] * vy), w[3]);
    const double p = (g - 1.0) * e;
    f1[0] = w[1];
    f1[1] = fma(w[1], vx, p);
    f1[2] = w[2] * vx;
    f1[3] = fma(g - 1.0, e, w[3]) * vx;
  }
  __device__ static __forceinline__ void fy(const double* w, double g, double* f2) {
    const double r = rcp_pos(w[0]);
    const double vx = w[1] * r, vy = w[2] * r;
    const double e = fma(-0.5, fma(w[1], vx, w[2] * vy), w[3]);
    const double p = (g - 1.0) * e;
    f2[0] = w[2];
    f2[1] = w[1] * vy;
    f2[2] = fma(w[2], vy, p);
    f2[3] = fma(g - 1.0, e, w[3]) * vy;
  }
};

// The 2D Euler wave speeds |u| + c and |v| + c at a cell average (rho, m1,
// m2, E) for the time step, with the seeded reciprocal and square root (the
// OE kernel's beta takes the same formula); false for a non-physical state.
__device__ __forceinline__ bool euler2_wave(double gamma, double rho, double m1, double m2, double E, double& bx,
                                            double& by) {
  const double r = rcp_pos(rho);  // NaN for rho <= 0 or subnormal: rejected below
  const double vx = m1 * r, vy = m2 * r;
  const double p = (gamma - 1.0) * fma(-0.5, fma(m1, vx, m2 * vy), E);
  if (!(rho > 0.0 && p > 0.0)) return false;
  const double c = sqrt_pos(fma(gamma * p, r, SQ_FLOOR));
  bx = fabs(vx) + c;
  by = fabs(vy) + c;
  return true;
}

// Block-level reductions (sum, max, min) over blockDim.x threads (a multiple
// of 32, at most 1024).  `sh` holds 3 * 32 doubles.  Result valid in thread 0.
__device__ __forceinline__ void block_reduce3(double& s, double& mx, double& mn, double* sh) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(full, s, o);
    mx = fmax(mx, __shfl_down_sync(full, mx, o));
    mn = fmin(mn, __shfl_down_sync(full, mn, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
    sh[warp] = s;
    sh[32 + warp] = mx;
    sh[64 + warp] = mn;
  }
  __syncthreads();
  if (warp == 0) {
    s = lane < nw ? sh[lane] : 0.0;
    mx = lane < nw ? sh[32 + lane] : -1.0 / 0.0;
    mn = lane < nw ? sh[64 + lane] : 1.0 / 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(full, s, o);
      mx = fmax(mx, __shfl_down_sync(full, mx, o));
      mn = fmin(mn, __shfl_down_sync(full, mn, o));
    }
  }
}

__device__ __forceinline__ double block_reduce_max(double v, double* sh) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(full, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(full, v, o));
  }
  return v;
}

}  // namespace oecdg
