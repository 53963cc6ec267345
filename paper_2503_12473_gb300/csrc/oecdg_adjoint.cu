// oecdg_adjoint.cu -- hand-written adjoint (vector-Jacobian product) of one
// OECDG time step on a periodic 2D Q^2 mesh pair (arXiv:2503.12473 forward
// scheme; the adjoint itself is not in the paper).
//
// Forward step (Eq. (eq:RKCDG), SSP-RK3, OE after every stage):
//   tau = tau_max = C_CFL / (beta_x/h_x + beta_y/h_y)      (max wave speed of u^n)
//   u_h^l = c_l u^n + (1-c_l)(u_s^{l-1} + tau L(u_s^{l-1}; tau_max)),  u_s^l = F_tau(u_h^l)
// The adjoint recomputes the stages, then runs backwards through them:
//   OE step:  lambda_h = dF/du_h^T lambda_s, through the direct scaling, the
//             damping coefficients delta (half-face traces of u^C - u^D, the
//             cell-average wave speed beta, the global sigma with its max/min
//             Gauss point and its average) and tau;
//   stage:    lambda_n += c_l lambda_h, lambda_in = (1-c_l)(lambda_h + tau dL/du^T lambda_h),
//             plus the scalar adjoints of tau and tau_max;
//   time step: tau and tau_max through the cell with the largest wave speed.
// Subgradients at non-differentiable points: |x|' = sign(x) (0 at 0), the
// derivative of sqrt of a zero sum is 0, max / argmax ties go to the lowest
// index (field, cell, point).
// Every cell writes its contributions to the four overlapping cells of the
// other mesh into its own slots; a gather pass adds them in a fixed order, so
// the result is deterministic.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>

#include "../../include/oecdg.h"
#include "oecdg_2d_body.cuh"
#include "oecdg_kernels.h"

namespace oecdg {

constexpr int AT = 128;  // threads per block of the per-cell adjoint kernels
#ifndef OECDG_ADJ_ROLLED
#define OECDG_ADJ_ROLLED 1
#endif

// w_bar += J1(w)^T fb1 + J2(w)^T fb2 for the 2D Euler flux at the conserved
// state w = (rho, m, n, E) (m = rho u, n = rho v).
__device__ __forceinline__ void euler2_vjp(const double* w, const double* fb1, const double* fb2, double g,
                                           double* wb) {
  const double r = rcp_pos(w[0]);
  const double u = w[1] * r, v = w[2] * r;
  const double g1 = g - 1.0;
  const double p = g1 * (w[3] - 0.5 * (w[1] * u + w[2] * v));
  const double H = w[3] + p;
  const double pr = 0.5 * g1 * (u * u + v * v), pm = -g1 * u, pn = -g1 * v, pE = g1;
  const double Hr = H * r;
  wb[0] += fb1[1] * (pr - u * u) - (fb1[2] + fb2[1]) * u * v + fb1[3] * u * (pr - Hr) + fb2[2] * (pr - v * v) +
           fb2[3] * v * (pr - Hr);
  wb[1] += fb1[0] + fb1[1] * (2.0 * u + pm) + (fb1[2] + fb2[1]) * v + fb1[3] * (Hr + u * pm) + fb2[2] * pm +
           fb2[3] * v * pm;
  wb[2] += fb1[1] * pn + (fb1[2] + fb2[1]) * u + fb1[3] * u * pn + fb2[0] + fb2[2] * (2.0 * v + pn) +
           fb2[3] * (Hr + v * pn);
  wb[3] += (fb1[1] + fb2[2]) * pE + (fb1[3] * u + fb2[3] * v) * (1.0 + pE);
}

template <int SYS>
__device__ __forceinline__ void flux_vjp(const Geo& g, const double* w, const double* fb1, const double* fb2,
                                         double* wb) {
  if (SYS == SYS_EULER) euler2_vjp(w, fb1, fb2, g.gamma, wb);
  else wb[0] += g.adv_x * fb1[0] + g.adv_y * fb2[0];
}

// Per-block sum of one value per thread (fixed order), written by thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(full, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(full, v, o);
  }
  return v;
}

// slot s = sx + 2 sy of cell K: contributions of K to its overlapping cell (sx, sy)
__device__ __forceinline__ long long slot_off(long long numel, int s) { return (long long)s * numel; }

// ------------------------------------------------------------- RHS adjoint --

// Adjoint of one stage combination u_h = ca u^n + cb (u_in + tau L(u_in)) for
// the cells of one mesh (blockIdx.z), given lam_h:
//   lam_in[K] = cb lam_h[K] - (cb tau / tau_max) lam_h[K]   (own cell; the
//               overlapping-cell terms go to the slots and are gathered later)
//   slots     = dL/du_O^T (cb tau lam_h[K]) for the 4 overlapping cells O
//   part_tm   = block partial of <cb tau lam_h, dL/dtau_max>
//   part_t    = block partial of <cb lam_h, L(u_in)>, with L(u_in) taken from
//               the recorded forward states: (u_h - ca u^n - cb u_in) / (cb tau)
// The column structure mirrors cell_rhs2d in reverse.
template <int SYS>
__global__ void __launch_bounds__(AT) k_rhs_vjp2d(Geo g, const double* __restrict__ uin, const double* __restrict__ un,
                                                  const double* __restrict__ uh, const double* __restrict__ lamh,
                                                  double* __restrict__ lamin, double* __restrict__ slots,
                                                  const double* __restrict__ dt, double ca, double cb,
                                                  double* __restrict__ part_tm, double* __restrict__ part_t) {
  constexpr int F = Fields<SYS>::F;
  __shared__ double sh[32];
  const int mesh = blockIdx.z;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = blockIdx.y * (AT / 32) + (threadIdx.x >> 5);
  const bool active = i < g.nx && j < g.ny;
  const int ic = active ? i : 0, jc = active ? j : 0;
  const long long P = g.plane;
  const long long numel = 2LL * F * 9 * P;
  const double tau = dt[0], tm = dt[1];
  const double inv_tm = 1.0 / tm;
  const double s = cb * tau;  // lam_tilde = s lam_h
  const double kd = 0.5 * g.hy * inv_tm;
  const double* uo = uin + (long long)(1 - mesh) * F * 9 * P;
  const long long self = (long long)mesh * F * 9 * P + (long long)jc * g.nx + ic;
  const int off = mesh == 0 ? -1 : 0;

  // R_bar[f][b][a] = (2a+1)(2b+1)/16 * s * lam_h, scaled once into this
  // thread's column of shared memory (keeps 9 F doubles out of the registers
  // and the scaling out of the FP64 pipe; each thread reads only its own column)
  const double sact = active ? s : 0.0;
  const double* lself = lamh + self;
  __shared__ double rbs[F * 9][AT];
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int q = 0; q < 9; ++q)
      rbs[f * 9 + q][threadIdx.x] = (2 * (q % 3) + 1) * (2 * (q / 3) + 1) / 16.0 * sact * __ldg(lself + (f * 9 + q) * P);
#define RB(f, b, a) (rbs[(f) * 9 + (b) * 3 + (a)][threadIdx.x])
  double tm_acc = 0.0, t_acc = 0.0;
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const long long id = self + (f * 9 + b * 3 + a) * P;
        const double lh = active ? __ldg(lamh + id) : 0.0;
        const double uself = __ldg(uin + id);
        // own-cell term: -u/tau_max and its tau_max derivative
        tm_acc += s * lh * uself * inv_tm * inv_tm;
        // L(u_in) from the recorded stage
        const double Lrec = (__ldg(uh + id) - (ca != 0.0 ? ca * __ldg(un + id) : 0.0) - cb * uself) / s;
        t_acc += cb * lh * Lrec;
        if (active) lamin[id] = cb * lh - s * lh * inv_tm;
      }

  const int oj0 = wrap_index<BC_PERIODIC>(jc + off, g.ny), oj1 = wrap_index<BC_PERIODIC>(jc + 1 + off, g.ny);
#if OECDG_ADJ_ROLLED
  // the four sub-cells one after the other (not unrolled: keeps the live
  // registers of one sub-cell only)
#pragma unroll 1
  for (int s4 = 0; s4 < 4; ++s4) {
    const int sx = s4 & 1, sy = s4 >> 1;
    const int oi = wrap_index<BC_PERIODIC>(ic + sx + off, g.nx);
    {
#else
  // the sub-cells one after the other: sx not unrolled (keeps the live
  // registers of one sub-cell only), sy unrolled (its quadrature constants fold)
#pragma unroll 1
  for (int sx = 0; sx < 2; ++sx) {
    const int oi = wrap_index<BC_PERIODIC>(ic + sx + off, g.nx);
#pragma unroll
    for (int sy = 0; sy < 2; ++sy) {
#endif
      // contributions to the overlapping cell O(sx, sy)
      double Wb[F][9];
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int m = 0; m < 9; ++m) Wb[f][m] = 0.0;
      const double* c = uo + (long long)(sy ? oj1 : oj0) * g.nx + oi;
      // ---- x-face column (xi = 2 sx - 1): R += (-s P_a(s)) (4/hx) Bf
      {
        double Bfb[F][3];
        const double sc = 4.0 / g.hx;
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int b = 0; b < 3; ++b)
            Bfb[f][b] = sx ? -sc * (RB(f, b, 0) + RB(f, b, 1) + RB(f, b, 2))
                           : sc * (RB(f, b, 0) - RB(f, b, 1) + RB(f, b, 2));
        double T[F][3], Tb[F][3];
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            T[f][b] = fma(-0.5, __ldg(c + (f * 9 + b * 3 + 2) * P), __ldg(c + (f * 9 + b * 3) * P));
            Tb[f][b] = 0.0;
          }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const double eo = xs_other(sy, q), es = xs_self(sy, q);
          double V[F], f1b[F], f2b[F], Vb[F];
#pragma unroll
          for (int f = 0; f < F; ++f) {
            V[f] = fma(lp(2, eo), T[f][2], fma(eo, T[f][1], T[f][0]));
            f1b[f] = gwt(q) * (Bfb[f][0] + es * Bfb[f][1] + lp(2, es) * Bfb[f][2]);
            f2b[f] = 0.0;
            Vb[f] = 0.0;
          }
          flux_vjp<SYS>(g, V, f1b, f2b, Vb);
#pragma unroll
          for (int f = 0; f < F; ++f) {
            Tb[f][0] += Vb[f];
            Tb[f][1] += eo * Vb[f];
            Tb[f][2] += lp(2, eo) * Vb[f];
          }
        }
        // T = u_0b - u_2b / 2
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            Wb[f][b * 3] += Tb[f][b];
            Wb[f][b * 3 + 2] -= 0.5 * Tb[f][b];
          }
      }
      // ---- the three volume columns of this half, points of sub-cell (sx, sy)
#pragma unroll
      for (int qx = 0; qx < 3; ++qx) {
        const double xo = xs_other(sx, qx), xsf = xs_self(sx, qx);
        const double wa = gwt(qx) * 2.0 / g.hy, wb = gwt(qx) * 2.0 / g.hx;
        double Ab[F][3], Bb[F][3];
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const double r0 = RB(f, b, 0), r1 = RB(f, b, 1), r2 = RB(f, b, 2);
            Ab[f][b] = wa * (r0 + xsf * r1 + lp(2, xsf) * r2);
            Bb[f][b] = wb * (r1 + dlp(2, xsf) * r2);
          }
        double T[F][3], Tb[F][3];
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const double* cb3 = c + (f * 9 + b * 3) * P;
            T[f][b] = fma(lp(2, xo), __ldg(cb3 + 2 * P), fma(xo, __ldg(cb3 + P), __ldg(cb3)));
            Tb[f][b] = 0.0;
          }
#pragma unroll
        for (int qy = 0; qy < 3; ++qy) {
          const double eo = xs_other(sy, qy), es = xs_self(sy, qy);
          const double w = gwt(qy);
          double V[F], f1b[F], f2b[F], Vb[F];
#pragma unroll
          for (int f = 0; f < F; ++f) {
            V[f] = fma(lp(2, eo), T[f][2], fma(eo, T[f][1], T[f][0]));
            const double g0b = w * (Ab[f][0] + es * Ab[f][1] + lp(2, es) * Ab[f][2]);
            f2b[f] = w * (Ab[f][1] + dlp(2, es) * Ab[f][2]);
            f1b[f] = w * (Bb[f][0] + es * Bb[f][1] + lp(2, es) * Bb[f][2]);
            Vb[f] = kd * g0b;
            tm_acc -= g0b * kd * V[f] * inv_tm;
          }
          flux_vjp<SYS>(g, V, f1b, f2b, Vb);
#pragma unroll
          for (int f = 0; f < F; ++f) {
            Tb[f][0] += Vb[f];
            Tb[f][1] += eo * Vb[f];
            Tb[f][2] += lp(2, eo) * Vb[f];
          }
        }
        // y-face point of this column: A_b += -2 s P_b(s) f2, s = 2 sy - 1, eta' = 0
        {
          double V[F], f1b[F], f2b[F], Vb[F];
#pragma unroll
          for (int f = 0; f < F; ++f) {
            V[f] = fma(-0.5, T[f][2], T[f][0]);
            f1b[f] = 0.0;
            f2b[f] = sy ? -2.0 * (Ab[f][0] + Ab[f][1] + Ab[f][2]) : 2.0 * (Ab[f][0] - Ab[f][1] + Ab[f][2]);
            Vb[f] = 0.0;
          }
          flux_vjp<SYS>(g, V, f1b, f2b, Vb);
#pragma unroll
          for (int f = 0; f < F; ++f) {
            Tb[f][0] += Vb[f];
            Tb[f][2] -= 0.5 * Vb[f];
          }
        }
        // T_b = sum_a u_ab P_a(xo)
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            Wb[f][b * 3] += Tb[f][b];
            Wb[f][b * 3 + 1] += xo * Tb[f][b];
            Wb[f][b * 3 + 2] += lp(2, xo) * Tb[f][b];
          }
      }
      if (active) {
        double* sl = slots + slot_off(numel, sx + 2 * sy) + self;
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int m = 0; m < 9; ++m) sl[(f * 9 + m) * P] = Wb[f][m];
      }
    }
  }
#undef RB
  if (!active) {
    tm_acc = 0.0;
    t_acc = 0.0;
  }
  const long long nb = (long long)gridDim.x * gridDim.y;
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  tm_acc = block_sum(tm_acc, sh);
  __syncthreads();
  t_acc = block_sum(t_acc, sh);
  if (threadIdx.x == 0) {
    part_tm[blk] = tm_acc;
    part_t[blk] = t_acc;
  }
  (void)nb;
}

// lam[O] += contributions of the four overlapping cells K of the other mesh:
// O dual (i,j) <- primal (i+a, j+b) slot (1-a, 1-b); O primal (i,j) <- dual
// (i-1+a, j-1+b) slot (1-a, 1-b).  Fixed order a, b.
template <int F>
__global__ void k_gather2d(Geo g, const double* __restrict__ slots, double* __restrict__ lam) {
  const long long P = g.plane;
  const long long numel = 2LL * F * 9 * P;
  const long long n = 2 * P;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / P);
    const long long cell = c - mesh * P;
    const int j = (int)(cell / g.nx), i = (int)(cell - (long long)j * g.nx);
    const int off = mesh == 0 ? -1 : 0;
    const int other = 1 - mesh;
    double acc[F * 9];
#pragma unroll
    for (int q = 0; q < F * 9; ++q) acc[q] = 0.0;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int ki = wrap_index<BC_PERIODIC>(i + a + off, g.nx), kj = wrap_index<BC_PERIODIC>(j + b + off, g.ny);
        const double* sl = slots + slot_off(numel, (1 - a) + 2 * (1 - b)) + (long long)other * F * 9 * P +
                           (long long)kj * g.nx + ki;
#pragma unroll
        for (int q = 0; q < F * 9; ++q) acc[q] += sl[q * P];
      }
    double* o = lam + (long long)mesh * F * 9 * P + cell;
#pragma unroll
    for (int q = 0; q < F * 9; ++q) o[q * P] += acc[q];
  }
}

// sum of `n` block partials in a fixed order, added to *out
__global__ void k_acc_partials(const double* __restrict__ part, long long n, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long b = threadIdx.x; b < n; b += blockDim.x) s += part[b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] += s;
}

// ------------------------------------------------------------ sigma stats --

// (value, index) reductions: larger value wins, ties go to the smaller index
__device__ __forceinline__ void argmax_merge(double& v, double& k, double v2, double k2) {
  if (v2 > v || (v2 == v && k2 < k)) {
    v = v2;
    k = k2;
  }
}
__device__ __forceinline__ void argmin_merge(double& v, double& k, double v2, double k2) {
  if (v2 < v || (v2 == v && k2 < k)) {
    v = v2;
    k = k2;
  }
}

// Per block (one mesh, blockIdx.y) and field: sum of cell averages, max and
// min over the cells' 3x3 Gauss points with their indices (cell * 9 + point).
// part[(mesh * nblk + blk) * F + f][5] = (sum, max, argmax, min, argmin)
template <int F>
__global__ void __launch_bounds__(256) k_sigma_stats2d(Geo g, const double* __restrict__ u, double* __restrict__ part) {
  __shared__ double sh[5][32];
  const int mesh = blockIdx.y;
  const long long nblk = gridDim.x;
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = cell < g.plane;
  const double* us = u + (long long)mesh * F * 9 * g.plane + (active ? cell : 0);
  const unsigned full = 0xffffffffu;
  for (int f = 0; f < F; ++f) {
    double v[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) v[m] = us[(f * 9 + m) * g.plane];
    double s = active ? v[0] : 0.0;
    double mx = -DINF, kmx = 1e300, mn = DINF, kmn = 1e300;
    if (active) {
#pragma unroll
      for (int qy = 0; qy < 3; ++qy) {
        double t[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = fma(lp(2, gnode(qy)), v[6 + a], fma(gnode(qy), v[3 + a], v[a]));
#pragma unroll
        for (int qx = 0; qx < 3; ++qx) {
          const double val = fma(lp(2, gnode(qx)), t[2], fma(gnode(qx), t[1], t[0]));
          const double k = (double)(cell * 9 + qy * 3 + qx);
          argmax_merge(mx, kmx, val, k);
          argmin_merge(mn, kmn, val, k);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(full, s, o);
      argmax_merge(mx, kmx, __shfl_down_sync(full, mx, o), __shfl_down_sync(full, kmx, o));
      argmin_merge(mn, kmn, __shfl_down_sync(full, mn, o), __shfl_down_sync(full, kmn, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
      sh[0][warp] = s;
      sh[1][warp] = mx;
      sh[2][warp] = kmx;
      sh[3][warp] = mn;
      sh[4][warp] = kmn;
    }
    __syncthreads();
    if (warp == 0) {
      s = lane < nw ? sh[0][lane] : 0.0;
      mx = lane < nw ? sh[1][lane] : -DINF;
      kmx = lane < nw ? sh[2][lane] : 1e300;
      mn = lane < nw ? sh[3][lane] : DINF;
      kmn = lane < nw ? sh[4][lane] : 1e300;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(full, s, o);
        argmax_merge(mx, kmx, __shfl_down_sync(full, mx, o), __shfl_down_sync(full, kmx, o));
        argmin_merge(mn, kmn, __shfl_down_sync(full, mn, o), __shfl_down_sync(full, kmn, o));
      }
      if (lane == 0) {
        double* p = part + ((mesh * nblk + blockIdx.x) * F + f) * 5;
        p[0] = s;
        p[1] = mx;
        p[2] = kmx;
        p[3] = mn;
        p[4] = kmn;
      }
    }
  }
}

// stats[mesh * F + f][6] = (avg, max, argmax, min, argmin, sigma); grid (F, 2), one warp
__global__ void k_sigma_stats_final(const double* __restrict__ part, long long nblk, int F, long long ncell,
                                    double* __restrict__ stats) {
  const int f = blockIdx.x, mesh = blockIdx.y;
  if (threadIdx.x != 0) return;
  double s = 0.0, mx = -DINF, kmx = 1e300, mn = DINF, kmn = 1e300;
  for (long long b = 0; b < nblk; ++b) {
    const double* p = part + ((mesh * nblk + b) * F + f) * 5;
    s += p[0];
    argmax_merge(mx, kmx, p[1], p[2]);
    argmin_merge(mn, kmn, p[3], p[4]);
  }
  const double a = s / (double)ncell;
  double* o = stats + (mesh * F + f) * 6;
  o[0] = a;
  o[1] = mx;
  o[2] = kmx;
  o[3] = mn;
  o[4] = kmn;
  o[5] = sigma_from_range(mx, mn, a);
}

// ------------------------------------------------------------- OE adjoint --

// Cell average wave speeds and their gradients w.r.t. the mode-0 fields
template <int SYS>
__device__ __forceinline__ void beta_and_grad(const Geo& g, const double* w, double& bx, double& by, double* gbx,
                                              double* gby) {
  if (SYS == SYS_EULER) {
    const double rho = w[0], r = 1.0 / rho;
    const double vx = w[1] * r, vy = w[2] * r;
    const double g1 = g.gamma - 1.0;
    const double p = g1 * (w[3] - 0.5 * (w[1] * vx + w[2] * vy));
    if (!(rho > 0.0 && p > 0.0)) {
      bx = by = 0.0;
      for (int k = 0; k < 4; ++k) gbx[k] = gby[k] = 0.0;
      return;
    }
    const double c = sqrt(g.gamma * p * r);
    bx = fabs(vx) + c;
    by = fabs(vy) + c;
    // dc = gamma / (2 c rho) (dp - p/rho drho)
    const double kc = g.gamma * r / (2.0 * c);
    const double pr = 0.5 * g1 * (vx * vx + vy * vy), pm = -g1 * vx, pn = -g1 * vy, pE = g1;
    const double dc[4] = {kc * (pr - p * r), kc * pm, kc * pn, kc * pE};
    const double sx = vx > 0.0 ? 1.0 : (vx < 0.0 ? -1.0 : 0.0);
    const double sy = vy > 0.0 ? 1.0 : (vy < 0.0 ? -1.0 : 0.0);
    gbx[0] = dc[0] - sx * vx * r;
    gbx[1] = dc[1] + sx * r;
    gbx[2] = dc[2];
    gbx[3] = dc[3];
    gby[0] = dc[0] - sy * vy * r;
    gby[1] = dc[1];
    gby[2] = dc[2] + sy * r;
    gby[3] = dc[3];
  } else {
    bx = fabs(g.adv_x);
    by = fabs(g.adv_y);
    gbx[0] = gby[0] = 0.0;
  }
}

// Forward OE step that also records (delta^m, field of the max, its face
// sums) per cell for the adjoint.
template <int SYS, bool ISO>
__global__ void __launch_bounds__(AT) k_oe_rec2d(Geo g, const double* __restrict__ uh, double* __restrict__ usig,
                                                 const double* __restrict__ dt, const double* __restrict__ sigma,
                                                 int* __restrict__ status, double* __restrict__ rec) {
  __shared__ double isg[Fields<SYS>::F];
  __shared__ double osh[2 * (AT / 32) * 32 * OSER_N];  // the rows' shared y-face series
  oe_inv_sigma<Fields<SYS>::F>(sigma, blockIdx.z, isg);
  oe_cell2d<SYS, BC_PERIODIC, false, 1, ISO, LD_NC, AT / 32>(g, uh, usig, dt, sigma, nullptr, status, blockIdx.z,
                                                            blockIdx.x * 32 + (threadIdx.x & 31),
                                                            blockIdx.y * (AT / 32) + (threadIdx.x >> 5), rec, isg, osh,
                                                            threadIdx.x >> 5);
}

// Reverse of one derivative order M of the face sums of one field: given the
// adjoints Sbx, Sby of S[x][M], S[y][M], add the adjoints of the cell's own
// modes (ub[9]) and of the 4 overlapping cells' modes (wb[sx + 2 sy][9]).
// Only the series order M needs is formed: M = 0 the value, M = 1 the value
// and first normal derivative, M = 2 all three.
template <int M>
__device__ __forceinline__ void oe_order_vjp(const Geo& g, const double* u, const double* __restrict__ uo_f,
                                             const int* oi, const int* oj, double Sbx, double Sby, double* ub,
                                             double (&wb)[4][9]) {
  const long long P = g.plane;
  const double dx1 = g.i2x, dy1 = g.i2y;  // 2/hx, 2/hy
#pragma unroll
  for (int n = 0; n < 2; ++n) {
    const double Sb = n == 0 ? Sbx : Sby;
    const double dn1 = n == 0 ? dx1 : dy1, dt1 = n == 0 ? dy1 : dx1;
    const double dn2 = dn1 * dn1, dt2 = dt1 * dt1;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const double s = 2.0 * side - 1.0;
      double c0[3], c1[3], c2[3];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const double u0 = n == 0 ? u[t * 3] : u[t], u1 = n == 0 ? u[t * 3 + 1] : u[3 + t];
        const double u2 = n == 0 ? u[t * 3 + 2] : u[6 + t];
        c0[t] = u0 + s * u1 + u2;
        c1[t] = fma(3.0 * s, u2, u1);
        c2[t] = 3.0 * u2;
      }
      double c0b[3] = {0, 0, 0}, c1b[3] = {0, 0, 0}, c2b[3] = {0, 0, 0};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const double dl = 1.0 - 2.0 * h;
        const int ci = n == 0 ? oi[side] : oi[h], cj = n == 0 ? oj[h] : oj[side];
        const int slot = (n == 0 ? side : h) + 2 * (n == 0 ? h : side);
        const double* co = uo_f + (long long)cj * g.nx + ci;
        double w0[3], w1[3], w2[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          w0[t] = co[(n == 0 ? t * 3 : t) * P];
          w1[t] = co[(n == 0 ? t * 3 + 1 : 3 + t) * P];
          w2[t] = co[(n == 0 ? t * 3 + 2 : 6 + t) * P];
        }
        double e0[3], e1[3] = {0, 0, 0}, e2[3] = {0, 0, 0};
        {
          const double o0[3] = {fma(-0.5, w2[0], w0[0]), fma(-0.5, w2[1], w0[1]), fma(-0.5, w2[2], w0[2])};
          e0[2] = c0[2] - o0[2];
          e0[1] = c0[1] - fma(3.0 * dl, o0[2], o0[1]);
          e0[0] = c0[0] - fma(1.5, o0[2], fma(dl, o0[1], o0[0]));
        }
        if (M >= 1) {
          e1[2] = c1[2] - w1[2];
          e1[1] = c1[1] - fma(3.0 * dl, w1[2], w1[1]);
          e1[0] = c1[0] - fma(1.5, w1[2], fma(dl, w1[1], w1[0]));
        }
        if (M == 2) {
          const double o2[3] = {3.0 * w2[0], 3.0 * w2[1], 3.0 * w2[2]};
          e2[2] = c2[2] - o2[2];
          e2[1] = c2[1] - fma(3.0 * dl, o2[2], o2[1]);
          e2[0] = c2[0] - fma(1.5, o2[2], fma(dl, o2[1], o2[0]));
        }
        double e0b[3] = {0, 0, 0}, e1b[3] = {0, 0, 0}, e2b[3] = {0, 0, 0};
        if (M == 0) {
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const double ts = xs_self(h, q), p2 = lp(2, ts);
            const double v = fma(p2, e0[2], fma(ts, e0[1], e0[0]));
            const double vb = gwt(q) * Sb * (v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0));
            e0b[0] += vb;
            e0b[1] += ts * vb;
            e0b[2] += p2 * vb;
          }
        } else if (M == 1) {
          const double a0 = dn1 * e1[0], a1 = dn1 * e1[1], a2 = dn1 * e1[2];
          const double t0 = dt1 * e0[1], t1 = 3.0 * dt1 * e0[2];
          double a0b = 0, a1b = 0, a2b = 0, t0b = 0, t1b = 0;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const double ts = xs_self(h, q), p2 = lp(2, ts);
            const double gn = fma(p2, a2, fma(ts, a1, a0));
            const double gt = fma(ts, t1, t0);
            // the forward kernel's floored norm (SQ_FLOOR): r1 > 0, and the
            // gradient at a zero sum comes out as 0 through gn = gt = 0
            const double r1 = sqrt_pos(fma(gn, gn, fma(gt, gt, SQ_FLOOR)));
            const double k1 = gwt(q) * Sb * rcp_pos(r1);
            const double gnb = k1 * gn, gtb = k1 * gt;
            a0b += gnb;
            a1b += ts * gnb;
            a2b += p2 * gnb;
            t0b += gtb;
            t1b += ts * gtb;
          }
          e0b[1] += dt1 * t0b;
          e0b[2] += 3.0 * dt1 * t1b;
          e1b[0] = dn1 * a0b;
          e1b[1] = dn1 * a1b;
          e1b[2] = dn1 * a2b;
        } else {
          const double a1 = dn1 * e1[1], a2 = dn1 * e1[2];
          const double b0 = dn2 * e2[0], b1 = dn2 * e2[1], b2 = dn2 * e2[2];
          const double m0 = dt1 * a1, m1 = 3.0 * dt1 * a2;
          const double tt = 3.0 * dt2 * e0[2];
          double b0b = 0, b1b = 0, b2b = 0, m0b = 0, m1b = 0, ttb = 0;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const double ts = xs_self(h, q), p2 = lp(2, ts);
            const double hn = fma(p2, b2, fma(ts, b1, b0));
            const double hm = fma(ts, m1, m0);
            const double r2 = sqrt_pos(fma(hn, hn, fma(hm, hm, fma(tt, tt, SQ_FLOOR))));
            const double k2 = gwt(q) * Sb * rcp_pos(r2);
            const double hnb = k2 * hn, hmb = k2 * hm;
            ttb += k2 * tt;
            b0b += hnb;
            b1b += ts * hnb;
            b2b += p2 * hnb;
            m0b += hmb;
            m1b += ts * hmb;
          }
          e0b[2] += 3.0 * dt2 * ttb;
          e1b[1] = dn1 * dt1 * m0b;
          e1b[2] = dn1 * 3.0 * dt1 * m1b;
          e2b[0] = dn2 * b0b;
          e2b[1] = dn2 * b1b;
          e2b[2] = dn2 * b2b;
        }
        // e = c - shift(o): c_bar += e_bar; o_bar = -shift^T e_bar
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          c0b[t] += e0b[t];
          c1b[t] += e1b[t];
          c2b[t] += e2b[t];
        }
        const double o0b[3] = {-e0b[0], -(dl * e0b[0] + e0b[1]), -(1.5 * e0b[0] + 3.0 * dl * e0b[1] + e0b[2])};
        const double o1b[3] = {-e1b[0], -(dl * e1b[0] + e1b[1]), -(1.5 * e1b[0] + 3.0 * dl * e1b[1] + e1b[2])};
        const double o2b[3] = {-e2b[0], -(dl * e2b[0] + e2b[1]), -(1.5 * e2b[0] + 3.0 * dl * e2b[1] + e2b[2])};
        // o0 = w0 - w2/2, o1 = w1, o2 = 3 w2
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          wb[slot][n == 0 ? t * 3 : t] += o0b[t];
          wb[slot][n == 0 ? t * 3 + 1 : 3 + t] += o1b[t];
          wb[slot][n == 0 ? t * 3 + 2 : 6 + t] += -0.5 * o0b[t] + 3.0 * o2b[t];
        }
      }
      // c0 = u0 + s u1 + u2, c1 = u1 + 3 s u2, c2 = 3 u2
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        ub[n == 0 ? t * 3 : t] += c0b[t];
        ub[n == 0 ? t * 3 + 1 : 3 + t] += s * c0b[t] + c1b[t];
        ub[n == 0 ? t * 3 + 2 : 6 + t] += c0b[t] + 3.0 * s * c1b[t] + 3.0 * c2b[t];
      }
    }
  }
}

// Adjoint of the OE step of one cell from its record: lam_h[K] (own modes)
// and the slots of the 4 overlapping cells; block partials of tau_bar and
// sigma_bar[f].  stats: (avg, max, argmax, min, argmin, sigma) per mesh and
// field.
template <int SYS>
__global__ void __launch_bounds__(AT) k_oe_vjp2d(Geo g, const double* __restrict__ uh, const double* __restrict__ lams,
                                                 double* __restrict__ lamh, double* __restrict__ slots,
                                                 const double* __restrict__ dt, const double* __restrict__ stats,
                                                 const double* __restrict__ rec, double* __restrict__ part_t,
                                                 double* __restrict__ part_sig) {
  constexpr int F = Fields<SYS>::F;
  __shared__ double sh[32];
  const int mesh = blockIdx.z;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = blockIdx.y * (AT / 32) + (threadIdx.x >> 5);
  const bool active = i < g.nx && j < g.ny;
  const int ic = active ? i : 0, jc = active ? j : 0;
  const long long P = g.plane;
  const long long numel = 2LL * F * 9 * P;
  const long long self = (long long)mesh * F * 9 * P + (long long)jc * g.nx + ic;
  const double* uo = uh + (long long)(1 - mesh) * F * 9 * P;
  const int off = mesh == 0 ? -1 : 0;
  int oi[2], oj[2];
  oi[0] = wrap_index<BC_PERIODIC>(ic + off, g.nx);
  oi[1] = wrap_index<BC_PERIODIC>(ic + 1 + off, g.nx);
  oj[0] = wrap_index<BC_PERIODIC>(jc + off, g.ny);
  oj[1] = wrap_index<BC_PERIODIC>(jc + 1 + off, g.ny);
  const double tau = dt[0];

  double w0[F];
#pragma unroll
  for (int f = 0; f < F; ++f) w0[f] = uh[self + f * 9 * P];
  double bx, by, gbx[4], gby[4];
  beta_and_grad<SYS>(g, w0, bx, by, gbx, gby);
  const double cx[3] = {g.i12x, 0.25, g.h24x5};  // 1/(12 hx), 1/4, 5 hx/24
  const double cy[3] = {g.i12y, 0.25, g.h24y5};

  // the forward's delta^m, the field of the max and its face sums
  const double* r = rec + ((long long)mesh * P + (long long)jc * g.nx + ic) * 12;
  double d[3], Sxm[3], Sym[3];
  int arg[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    d[m] = r[4 * m];
    arg[m] = (int)r[4 * m + 1];
    Sxm[m] = r[4 * m + 2];
    Sym[m] = r[4 * m + 3];
  }
  const double r1 = d[0] + d[1], r2 = r1 + d[2];
  const double e1 = exp(-tau * r1), e2 = exp(-tau * r2);
  // direct term and e_bar
  double e1b = 0.0, e2b = 0.0;
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      const int deg = (m % 3) + (m / 3);
      const long long id = self + (f * 9 + m) * P;
      const double ls = active ? lams[id] : 0.0;
      const double uv = uh[id];
      if (deg == 1) e1b += ls * uv;
      if (deg >= 2) e2b += ls * uv;
      if (active) lamh[id] = deg == 0 ? ls : (deg == 1 ? ls * e1 : ls * e2);
    }
  const double r1b = -tau * e1 * e1b, r2b = -tau * e2 * e2b;
  double t_acc = -(r1 * e1 * e1b + r2 * e2 * e2b);
  const double db[3] = {r1b + r2b, r1b + r2b, r2b};
  // delta^m = delta^m(arg[m]) = (bx cx Sx + by cy Sy) / sigma: one reverse pass
  // per order m on the field that gives its max (the field is data, so the
  // lanes of a warp follow the same path whatever field each one has)
  double bxb = 0.0, byb = 0.0;
  double sigb[F];
#pragma unroll
  for (int f = 0; f < F; ++f) sigb[f] = 0.0;
  if (active) {
#pragma unroll
    for (int s4 = 0; s4 < 4; ++s4) {
      double* sl = slots + slot_off(numel, s4) + self;
#pragma unroll
      for (int q = 0; q < F * 9; ++q) sl[q * P] = 0.0;
    }
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int f = arg[m];
    if (f < 0 || !active) continue;
    const double sg = stats[(mesh * F + f) * 6 + 5];
    const double k = db[m] / sg;
    bxb += k * cx[m] * Sxm[m];
    byb += k * cy[m] * Sym[m];
#pragma unroll
    for (int ff = 0; ff < F; ++ff)
      if (ff == f) sigb[ff] -= db[m] * d[m] / sg;
    double u[9], ub[9], wbl[4][9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      u[q] = uh[self + (f * 9 + q) * P];
      ub[q] = 0.0;
    }
#pragma unroll
    for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
      for (int q = 0; q < 9; ++q) wbl[s4][q] = 0.0;
    const double* uof = uo + (long long)f * 9 * P;
    if (m == 0) oe_order_vjp<0>(g, u, uof, oi, oj, k * bx * cx[0], k * by * cy[0], ub, wbl);
    else if (m == 1) oe_order_vjp<1>(g, u, uof, oi, oj, k * bx * cx[1], k * by * cy[1], ub, wbl);
    else oe_order_vjp<2>(g, u, uof, oi, oj, k * bx * cx[2], k * by * cy[2], ub, wbl);
#pragma unroll
    for (int q = 0; q < 9; ++q) lamh[self + (f * 9 + q) * P] += ub[q];
#pragma unroll
    for (int s4 = 0; s4 < 4; ++s4) {
      double* sl = slots + slot_off(numel, s4) + self + (long long)f * 9 * P;
#pragma unroll
      for (int q = 0; q < 9; ++q) sl[q * P] += wbl[s4][q];
    }
  }
  // beta at the cell average (mode 0)
  if (active && SYS == SYS_EULER) {
#pragma unroll
    for (int f = 0; f < F; ++f) lamh[self + f * 9 * P] += bxb * gbx[f] + byb * gby[f];
  }
  if (!active) t_acc = 0.0;
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  t_acc = block_sum(t_acc, sh);
  if (threadIdx.x == 0) part_t[blk] = t_acc;
  const long long nb = (long long)gridDim.x * gridDim.y;
  const long long lblk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
  for (int f = 0; f < F; ++f) {
    __syncthreads();
    const double v = block_sum(active ? sigb[f] : 0.0, sh);
    if (threadIdx.x == 0) part_sig[(mesh * F + f) * nb + lblk] = v;
  }
}

// sigma_bar (per mesh and field, summed) -> the avg (mode 0 of every cell of
// that mesh, weight -+1/N) and the extremal Gauss point's cell.
// sigma = max - avg  (if max - avg >= avg - min), else avg - min.
template <int F>
__global__ void k_sigma_adj_avg(Geo g, const double* __restrict__ stats, const double* __restrict__ sigb,
                                double* __restrict__ lam) {
  const long long n = 2 * g.plane;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      const double* st = stats + (mesh * F + f) * 6;
      const double sb = sigb[mesh * F + f];
      if (st[5] == 0.0) continue;
      const double sa = (st[1] - st[0] >= st[0] - st[3]) ? -1.0 : 1.0;
      lam[(long long)mesh * F * 9 * g.plane + (long long)(f * 9) * g.plane + cell] += sa * sb / (double)g.plane;
    }
  }
}

template <int F>
__global__ void k_sigma_adj_point(Geo g, const double* __restrict__ stats, const double* __restrict__ sigb,
                                  double* __restrict__ lam) {
  const int mesh = blockIdx.x / F, f = blockIdx.x % F;
  if (threadIdx.x != 0) return;
  // one thread per (mesh, field), serialised over the fields of a mesh so two
  // fields with the same extremal cell add in a fixed order
  if (f != 0) return;
  for (int ff = 0; ff < F; ++ff) {
    const double* st = stats + (mesh * F + ff) * 6;
    const double sb = sigb[mesh * F + ff];
    if (st[5] == 0.0) continue;
    const bool use_max = st[1] - st[0] >= st[0] - st[3];
    const double kd = use_max ? st[2] : st[4];
    if (!(kd >= 0.0 && kd < 9.0 * (double)g.plane)) continue;  // no finite extremum
    const long long k = (long long)kd;
    const double sgn = use_max ? 1.0 : -1.0;
    const long long cell = k / 9;
    const int pt = (int)(k % 9), qy = pt / 3, qx = pt % 3;
    double* o = lam + (long long)mesh * F * 9 * g.plane + (long long)(ff * 9) * g.plane + cell;
    for (int m = 0; m < 9; ++m) o[m * g.plane] += sgn * sb * lp(m % 3, gnode(qx)) * lp(m / 3, gnode(qy));
  }
}

// ----------------------------------------------------------- tau adjoint --

// per block (grid-stride over both meshes' cells): max of |u|+c and |v|+c with
// the cell index (mesh * plane + cell): part[blk][4] = (bx, kx, by, ky)
template <int SYS>
__global__ void k_wave_stats2d(Geo g, const double* __restrict__ u, double* __restrict__ part) {
  constexpr int F = Fields<SYS>::F;
  __shared__ double sh[4][32];
  const unsigned full = 0xffffffffu;
  const long long n = 2 * g.plane;
  double bx = -1.0, kx = 1e300, by = -1.0, ky = 1e300;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    double w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int f = 0; f < F; ++f) w[f] = u[(long long)mesh * F * 9 * g.plane + (long long)(f * 9) * g.plane + cell];
    double sx, sy, gx[4], gy[4];
    beta_and_grad<SYS>(g, w, sx, sy, gx, gy);
    argmax_merge(bx, kx, sx, (double)c);
    argmax_merge(by, ky, sy, (double)c);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    argmax_merge(bx, kx, __shfl_down_sync(full, bx, o), __shfl_down_sync(full, kx, o));
    argmax_merge(by, ky, __shfl_down_sync(full, by, o), __shfl_down_sync(full, ky, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    sh[0][warp] = bx;
    sh[1][warp] = kx;
    sh[2][warp] = by;
    sh[3][warp] = ky;
  }
  __syncthreads();
  if (warp == 0) {
    bx = lane < nw ? sh[0][lane] : -1.0;
    kx = lane < nw ? sh[1][lane] : 1e300;
    by = lane < nw ? sh[2][lane] : -1.0;
    ky = lane < nw ? sh[3][lane] : 1e300;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      argmax_merge(bx, kx, __shfl_down_sync(full, bx, o), __shfl_down_sync(full, kx, o));
      argmax_merge(by, ky, __shfl_down_sync(full, by, o), __shfl_down_sync(full, ky, o));
    }
    if (lane == 0) {
      part[blockIdx.x * 4] = bx;
      part[blockIdx.x * 4 + 1] = kx;
      part[blockIdx.x * 4 + 2] = by;
      part[blockIdx.x * 4 + 3] = ky;
    }
  }
}

// tau = tau_max = C_CFL / (bx/hx + by/hy): lam[argmax cell, mode 0] += (tb + tmb) dtau/dbeta dbeta/dw
template <int SYS>
__global__ void k_tau_adj(Geo g, const double* __restrict__ part, int nblk, const double* __restrict__ scal,
                          const double* __restrict__ u, double* __restrict__ lam) {
  constexpr int F = Fields<SYS>::F;
  if (threadIdx.x != 0 || blockIdx.x != 0 || SYS != SYS_EULER) return;
  double bx = -1.0, kx = 1e300, by = -1.0, ky = 1e300;
  for (int b = 0; b < nblk; ++b) {
    argmax_merge(bx, kx, part[4 * b], part[4 * b + 1]);
    argmax_merge(by, ky, part[4 * b + 2], part[4 * b + 3]);
  }
  const double rate = bx / g.hx + by / g.hy;
  if (!(rate > 0.0)) return;
  const double tbar = scal[0] + scal[1];
  const double dtdr = -g.cfl / (rate * rate);
  for (int dir = 0; dir < 2; ++dir) {
    const double kd = dir == 0 ? kx : ky;
    if (!(kd >= 0.0 && kd < 2.0 * (double)g.plane)) continue;  // no finite maximum
    const long long c = (long long)kd;
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    double w[4] = {0, 0, 0, 0};
    for (int f = 0; f < F; ++f) w[f] = u[(long long)mesh * F * 9 * g.plane + (long long)(f * 9) * g.plane + cell];
    double sx, sy, gx[4], gy[4];
    beta_and_grad<SYS>(g, w, sx, sy, gx, gy);
    const double k = tbar * dtdr / (dir == 0 ? g.hx : g.hy);
    for (int f = 0; f < F; ++f)
      lam[(long long)mesh * F * 9 * g.plane + (long long)(f * 9) * g.plane + cell] += k * (dir == 0 ? gx[f] : gy[f]);
  }
}

__global__ void k_axpby(long long n, const double* __restrict__ x, double a, double* __restrict__ y, double b) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] = a * x[q] + b * y[q];
}

__global__ void k_zero(double* __restrict__ p, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) p[q] = 0.0;
}

}  // namespace oecdg

// ------------------------------------------------------------------ driver --

#include "oecdg_ctx.h"

using namespace oecdg;

struct AdjScratch {
  double* H[3];     // u_h of the three stages (forward recompute)
  double* S[2];     // u_sigma of stages 1 and 2
  double* LH;       // lambda_h
  double* LI;       // lambda of a stage input
  double* LN;       // lambda^n accumulator
  double* slots;    // 4 x state
  double* part_t;   // [2 nb]
  double* part_tm;  // [2 nb]
  double* part_sig; // [2 F nb]
  double* sstat_part;  // [2 nb256 F 5]
  double* stats;    // [2 F 6]
  double* sigb;     // [2 F]
  double* scal;     // [tau_bar, tau_max_bar]
  double* wpart;    // [WBLK 4]
  double* time;     // scratch time slot of the recompute
  double* rec[3];   // OE records of the three stages: [2 plane][12]
  long long nb, nb256;
};

static const int ADJ_WBLK = 296;

void adj_release(cdg_ctx* c) {
  if (!c || !c->adj) return;
  AdjScratch* a = c->adj;
  cudaFree(a->H[0]);  // one pool
  free(a);
  c->adj = nullptr;
}

static cdg_status adj_fail(cdg_ctx* c, cdg_status s, const char* msg) {
  if (c) snprintf(c->err, sizeof c->err, "%s", msg);
  return s;
}

static cdg_status adj_alloc(cdg_ctx* c) {
  if (c->adj) return CDG_OK;
  AdjScratch* a = (AdjScratch*)calloc(1, sizeof(AdjScratch));
  if (!a) return CDG_ENOMEM;
  const Geo& g = c->g;
  const int F = c->F;
  a->nb = (long long)((g.nx + 31) / 32) * ((g.ny + AT / 32 - 1) / (AT / 32));
  a->nb256 = (g.plane + 255) / 256;
  const size_t n = c->numel;
  size_t tot = 12 * n + 2 * a->nb * 2 + (size_t)2 * F * a->nb + (size_t)2 * a->nb256 * F * 5 + 2 * F * 6 + 2 * F + 2 +
               ADJ_WBLK * 4 + 2 + 3 * (size_t)24 * g.plane;
  double* p = nullptr;
  if (cudaMalloc((void**)&p, tot * sizeof(double)) != cudaSuccess) {
    (void)cudaGetLastError();  // clear the failed allocation: later launch checks must not see it
    free(a);
    return CDG_ENOMEM;
  }
  a->H[0] = p; p += n;
  a->H[1] = p; p += n;
  a->H[2] = p; p += n;
  a->S[0] = p; p += n;
  a->S[1] = p; p += n;
  a->LH = p; p += n;
  a->LI = p; p += n;
  a->LN = p; p += n;
  a->slots = p; p += 4 * n;
  a->part_t = p; p += 2 * a->nb;
  a->part_tm = p; p += 2 * a->nb;
  a->part_sig = p; p += (size_t)2 * F * a->nb;
  a->sstat_part = p; p += (size_t)2 * a->nb256 * F * 5;
  a->stats = p; p += 2 * F * 6;
  a->sigb = p; p += 2 * F;
  a->scal = p; p += 2;
  a->wpart = p; p += ADJ_WBLK * 4;
  a->time = p; p += 2;
  for (int l = 0; l < 3; ++l) {
    a->rec[l] = p;
    p += (size_t)24 * g.plane;
  }
  c->adj = a;
  return CDG_OK;
}

template <int SYS>
static cudaError_t adj_oe(cdg_ctx* c, const double* uh, const double* lams, double* lamh, const double* rec) {
  constexpr int F = Fields<SYS>::F;
  AdjScratch* a = c->adj;
  const Geo& g = c->g;
  cudaStream_t st = c->stream;
  const dim3 grid((g.nx + 31) / 32, (g.ny + AT / 32 - 1) / (AT / 32), 2);
  k_sigma_stats2d<F><<<dim3((unsigned)a->nb256, 2), 256, 0, st>>>(g, uh, a->sstat_part);
  k_sigma_stats_final<<<dim3(F, 2), 32, 0, st>>>(a->sstat_part, a->nb256, F, g.plane, a->stats);
  k_oe_vjp2d<SYS><<<grid, AT, 0, st>>>(g, uh, lams, lamh, a->slots, c->dt, a->stats, rec, a->part_t, a->part_sig);
  k_acc_partials<<<1, 1024, 0, st>>>(a->part_t, 2 * a->nb, a->scal);
  k_zero<<<1, 32, 0, st>>>(a->sigb, 2 * F);
  for (int q = 0; q < 2 * F; ++q) k_acc_partials<<<1, 1024, 0, st>>>(a->part_sig + q * a->nb, a->nb, a->sigb + q);
  k_gather2d<F><<<1184, 256, 0, st>>>(g, a->slots, lamh);
  k_sigma_adj_avg<F><<<1184, 256, 0, st>>>(g, a->stats, a->sigb, lamh);
  k_sigma_adj_point<F><<<2 * F, 32, 0, st>>>(g, a->stats, a->sigb, lamh);
  c->launches += 8 + 2 * F;
  return cudaGetLastError();
}

template <int SYS>
static cudaError_t adj_stage(cdg_ctx* c, const double* uin, const double* un, const double* uh, const double* lamh,
                             double* lamin, double ca, double cb) {
  constexpr int F = Fields<SYS>::F;
  AdjScratch* a = c->adj;
  const Geo& g = c->g;
  cudaStream_t st = c->stream;
  const dim3 grid((g.nx + 31) / 32, (g.ny + AT / 32 - 1) / (AT / 32), 2);
  k_rhs_vjp2d<SYS><<<grid, AT, 0, st>>>(g, uin, un, uh, lamh, lamin, a->slots, c->dt, ca, cb, a->part_tm, a->part_t);
  k_acc_partials<<<1, 1024, 0, st>>>(a->part_tm, 2 * a->nb, a->scal + 1);
  k_acc_partials<<<1, 1024, 0, st>>>(a->part_t, 2 * a->nb, a->scal);
  k_gather2d<F><<<1184, 256, 0, st>>>(g, a->slots, lamin);
  c->launches += 4;
  return cudaGetLastError();
}

// Forward step that records what the adjoint needs: u_h of the three stages
// (H[0..2]) and u_sigma of the first two (S[0..1]); u is advanced in place
// when u_next != nullptr (S[2] := u^{n+1}).  tau, tau_max land in dt.
template <int SYS>
static cudaError_t adj_forward(cdg_ctx* c, const double* un, double* const* H, double* const* S, double* u_next,
                               double* dt, double* const* R) {
  constexpr int F = Fields<SYS>::F;
  AdjScratch* a = c->adj;
  const Geo& g = c->g;
  cudaStream_t st = c->stream;
  const int sys = SYS;
  const bool oe = c->d.oe != 0;
  cudaError_t e;
  if ((e = launch_set2(a->time, 0.0, 0.0, st)) != cudaSuccess) return e;
  if ((e = launch_dt2d(sys, g, un, c->wave_partial, c->wave_blk, 0.0, dt, a->time, c->status, st)) != cudaSuccess)
    return e;
  const double C[3] = {0.0, 0.75, 1.0 / 3.0};
  const double* uin[3] = {un, oe ? S[0] : H[0], oe ? S[1] : H[1]};
  for (int l = 0; l < 3; ++l) {
    if ((e = launch_stage2d(sys, BC_PERIODIC, g, 0, uin[l], un, H[l], dt, C[l], 1.0 - C[l], c->partials, st)) !=
        cudaSuccess)
      return e;
    // the last stage's OE output is u^{n+1}; without u_next it is still run
    // (into the stage buffer H[2]'s partner slot) for its record
    double* dst = l < 2 ? S[l] : (u_next ? u_next : a->LI);
    if (oe) {
      if ((e = launch_sigma(c->partials, c->nblk, F, plain_norm(g.plane), c->sigma, c->avg, st)) != cudaSuccess) return e;
      const dim3 grid((g.nx + 31) / 32, (g.ny + AT / 32 - 1) / (AT / 32), 2);
      // the variant the forward step uses (square cells: isotropic), so the
      // recorded states equal cdg_step's
      if (g.hx == g.hy) k_oe_rec2d<SYS, true><<<grid, AT, 0, st>>>(g, H[l], dst, dt, c->sigma, c->status, R[l]);
      else k_oe_rec2d<SYS, false><<<grid, AT, 0, st>>>(g, H[l], dst, dt, c->sigma, c->status, R[l]);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else if ((e = cudaMemcpyAsync(dst, H[l], c->numel * sizeof(double), cudaMemcpyDeviceToDevice, st)) !=
               cudaSuccess) {
      return e;
    }
  }
  c->launches += 3 + 3 + 2 * 3;
  return cudaSuccess;
}

// Backward through one recorded step: lam = (du^{n+1}/du^n)^T lam_next.
template <int SYS>
static cudaError_t adj_backward(cdg_ctx* c, const double* un, const double* const* H, const double* const* S,
                                const double* const* R, const double* lam_next, double* lam, double* gtau) {
  AdjScratch* a = c->adj;
  const Geo& g = c->g;
  cudaStream_t st = c->stream;
  const long long n = (long long)c->numel;
  const bool oe = c->d.oe != 0;
  const double C[3] = {0.0, 0.75, 1.0 / 3.0};
  const double* uin[3] = {un, oe ? S[0] : H[0], oe ? S[1] : H[1]};
  cudaError_t e;
  k_zero<<<1, 32, 0, st>>>(a->scal, 2);
  const double* lam_s = lam_next;
  for (int l = 2; l >= 0; --l) {
    if (oe) {
      if ((e = adj_oe<SYS>(c, H[l], lam_s, a->LH, R[l])) != cudaSuccess) return e;
    } else {
      k_axpby<<<1184, 256, 0, st>>>(n, lam_s, 1.0, a->LH, 0.0);
    }
    if ((e = adj_stage<SYS>(c, uin[l], un, H[l], a->LH, a->LI, C[l], 1.0 - C[l])) != cudaSuccess) return e;
    // lambda^n += c_l lambda_h (+ lambda_in for the first stage, whose input is u^n)
    if (l == 2) k_axpby<<<1184, 256, 0, st>>>(n, a->LH, C[l], a->LN, 0.0);
    else if (l == 1) k_axpby<<<1184, 256, 0, st>>>(n, a->LH, C[l], a->LN, 1.0);
    else k_axpby<<<1184, 256, 0, st>>>(n, a->LI, 1.0, a->LN, 1.0);
    lam_s = a->LI;
    c->launches += 2;
  }
  // ---- tau = tau_max through the largest wave speed of u^n
  k_wave_stats2d<SYS><<<ADJ_WBLK, 256, 0, st>>>(g, un, a->wpart);
  k_tau_adj<SYS><<<1, 32, 0, st>>>(g, a->wpart, ADJ_WBLK, a->scal, un, a->LN);
  c->launches += 3;
  if ((e = cudaMemcpyAsync(lam, a->LN, n * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if (gtau && (e = cudaMemcpyAsync(gtau, a->scal, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  return cudaGetLastError();
}

static cdg_status adj_check(cdg_ctx* ctx) {
  if (ctx->d.dim != 2 || ctx->gen2 || uniform_side_bc(ctx->d) != CDG_PERIODIC || ctx->d.rk != CDG_RK_SSP3)
    return adj_fail(ctx, CDG_EUNSUPPORTED, "adjoint: 2D periodic Q^2 SSP-RK3 only");
  cdg_status s = adj_alloc(ctx);
  if (s != CDG_OK) return adj_fail(ctx, s, "adjoint: allocation failed");
  return CDG_OK;
}

static cdg_status adj_cuda(cdg_ctx* ctx, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return CDG_OK;
  snprintf(ctx->err, sizeof ctx->err, "%s: %s", where, cudaGetErrorString(e));
  return CDG_ECUDA;
}

// record layout: [u^n][H0][S0][H1][S1][H2][tau, tau_max][OE records of 3 stages: 3 x 2 plane x 12]
static size_t rec_oe_numel(const cdg_ctx* ctx) { return (size_t)24 * ctx->g.plane; }

extern "C" cdg_status cdg_record_numel(const cdg_ctx* ctx, size_t* numel) {
  if (!ctx || !numel) return CDG_EINVAL;
  *numel = 6 * ctx->numel + 2 + 3 * rec_oe_numel(ctx);
  return CDG_OK;
}

extern "C" cdg_status cdg_step_record(cdg_ctx* ctx, double* d_u, double* d_rec) {
  if (!ctx || !d_u || !d_rec) return adj_fail(ctx, CDG_EINVAL, "step_record: null pointer");
  cdg_status s = adj_check(ctx);
  if (s != CDG_OK) return s;
  const size_t n = ctx->numel;
  double* U = d_rec;
  double* H[3] = {d_rec + n, d_rec + 3 * n, d_rec + 5 * n};
  double* S[2] = {d_rec + 2 * n, d_rec + 4 * n};
  double* dt = d_rec + 6 * n;
  double* R[3] = {dt + 2, dt + 2 + rec_oe_numel(ctx), dt + 2 + 2 * rec_oe_numel(ctx)};
  cudaError_t e = cudaMemcpyAsync(U, d_u, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = ctx->d.system == CDG_EULER ? adj_forward<SYS_EULER>(ctx, U, H, S, d_u, dt, R)
                                   : adj_forward<SYS_ADV>(ctx, U, H, S, d_u, dt, R);
  return adj_cuda(ctx, e, "step_record");
}

extern "C" cdg_status cdg_step_adjoint_recorded(cdg_ctx* ctx, const double* d_rec, const double* d_lam_next,
                                                double* d_lam, double* d_gtau) {
  if (!ctx || !d_rec || !d_lam_next || !d_lam) return adj_fail(ctx, CDG_EINVAL, "step_adjoint_recorded: null pointer");
  cdg_status s = adj_check(ctx);
  if (s != CDG_OK) return s;
  const size_t n = ctx->numel;
  const double* U = d_rec;
  const double* H[3] = {d_rec + n, d_rec + 3 * n, d_rec + 5 * n};
  const double* S[2] = {d_rec + 2 * n, d_rec + 4 * n};
  const double* R0 = d_rec + 6 * n + 2;
  const double* R[3] = {R0, R0 + rec_oe_numel(ctx), R0 + 2 * rec_oe_numel(ctx)};
  cudaError_t e = cudaMemcpyAsync(ctx->dt, d_rec + 6 * n, 2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = ctx->d.system == CDG_EULER ? adj_backward<SYS_EULER>(ctx, U, H, S, R, d_lam_next, d_lam, d_gtau)
                                   : adj_backward<SYS_ADV>(ctx, U, H, S, R, d_lam_next, d_lam, d_gtau);
  return adj_cuda(ctx, e, "step_adjoint_recorded");
}

extern "C" cdg_status cdg_step_adjoint(cdg_ctx* ctx, const double* d_un, const double* d_lam_next, double* d_lam,
                                       double* d_gtau) {
  if (!ctx || !d_un || !d_lam_next || !d_lam) return adj_fail(ctx, CDG_EINVAL, "step_adjoint: null pointer");
  if (d_lam == d_un) return adj_fail(ctx, CDG_EINVAL, "step_adjoint: d_lam aliases d_un");
  cdg_status s = adj_check(ctx);
  if (s != CDG_OK) return s;
  AdjScratch* a = ctx->adj;
  double* H[3] = {a->H[0], a->H[1], a->H[2]};
  double* S[2] = {a->S[0], a->S[1]};
  const double* Hc[3] = {a->H[0], a->H[1], a->H[2]};
  const double* Sc[2] = {a->S[0], a->S[1]};
  double* R[3] = {a->rec[0], a->rec[1], a->rec[2]};
  const double* Rc[3] = {a->rec[0], a->rec[1], a->rec[2]};
  cudaError_t e = ctx->d.system == CDG_EULER ? adj_forward<SYS_EULER>(ctx, d_un, H, S, nullptr, ctx->dt, R)
                                             : adj_forward<SYS_ADV>(ctx, d_un, H, S, nullptr, ctx->dt, R);
  if (e == cudaSuccess)
    e = ctx->d.system == CDG_EULER ? adj_backward<SYS_EULER>(ctx, d_un, Hc, Sc, Rc, d_lam_next, d_lam, d_gtau)
                                   : adj_backward<SYS_ADV>(ctx, d_un, Hc, Sc, Rc, d_lam_next, d_lam, d_gtau);
  return adj_cuda(ctx, e, "step_adjoint");
}
