// oecdg_1d.cu -- 1D P^K kernels (K = 1, 2, 3) of the OECDG forward step
// (arXiv:2503.12473): Eq. (eq:1D_H) and the 1D form of the damping
// coefficients (Remark in Section 2.2), for linear advection, Burgers
// (f = u^2/2) and the 1D Euler equations.  One thread per cell of one mesh
// (blockIdx.y = mesh); primal cell i overlaps dual cells i-1 (left half) and i
// (right half), dual cell i overlaps primal cells i and i+1; in the overlapping
// cell the point xi of half s sits at xi' = xi + 1 - 2 s.
#include <type_traits>

#include "oecdg_common.cuh"
#include "oecdg_kernels.h"
#include "oecdg_persist.cuh"
#include "oecdg_poly.cuh"

namespace oecdg {

// Cells (threads) per block.  GB300 executes 2 FP64 thread-operations per
// clock per SM, so a 1D mesh of a few thousand cells is bound by how many SMs
// its blocks reach: small blocks spread it over more of them (64 measured
// best on a 4000-cell mesh, by 5%).
#ifndef OECDG_NT1
#define OECDG_NT1 64
#endif
constexpr int NT1 = OECDG_NT1;
constexpr double DINF1 = __builtin_huge_val();

template <int SYS>
struct Fields1 {
  static constexpr int F = SYS == SYS_EULER ? 3 : 1;
};

template <int SYS>
__device__ __forceinline__ void flux1(const Geo& g, const double* w, double* f) {
  if (SYS == SYS_EULER) {
    const double r = rcp_pos(w[0]);  // seeded reciprocal, within 1 ulp (oecdg_common.cuh)
    const double v = w[1] * r;
    // multiply-adds written out as fma: every kernel that inlines this rounds
    // alike (the compiler's own contraction may differ between them)
    const double e = fma(-0.5 * w[1], v, w[2]);  // E - kinetic energy
    const double p = (g.gamma - 1.0) * e;
    f[0] = w[1];
    f[1] = fma(w[1], v, p);
    f[2] = fma(g.gamma - 1.0, e, w[2]) * v;  // (E + p) v, E + p as one fma
  } else if (SYS == SYS_BURGERS) {
    f[0] = 0.5 * w[0] * w[0];
  } else {
    f[0] = g.adv_x * w[0];
  }
}

// Wave speed |f'(w)| (Euler: |v| + c, with the seeded reciprocal and square
// root as in the 2D kernels); -1 for a non-physical Euler state.
template <int SYS>
__device__ __forceinline__ double speed1(const Geo& g, const double* w) {
  if (SYS == SYS_EULER) {
    const double r = rcp_pos(w[0]);  // NaN for rho <= 0 or subnormal: flagged below
    const double v = w[1] * r;
    const double p = (g.gamma - 1.0) * fma(-0.5 * w[1], v, w[2]);
    if (!(w[0] > 0.0 && p > 0.0)) return -1.0;
    return fabs(v) + sqrt_pos(fma(g.gamma * p, r, SQ_FLOOR));
  } else if (SYS == SYS_BURGERS) {
    return fabs(w[0]);
  }
  return fabs(g.adv_x);
}

// L_a = (2a+1) [ sum_{s,q} (w_q/4)(w/tau_max) P_a(xi) + (1/h) sum (w_q/2) f(w) P_a'(xi)
//               - (1/h)(f_R - (-1)^a f_L) ] - u_a / tau_max
// in two parts.  rhs1d_half: the sums over the K+1 Gauss points of half sx of
// cell i (the overlapping cell there is smooth) and the flux at that half's
// face (sx = 0: the left end, sx = 1: the right end), from zero.  The cell's
// sums are half 0's plus half 1's, one addition per coefficient, so a cell
// computed by one thread and a cell split over two lanes (one half each) get
// the same bits.
template <int SYS, int BC, int K, int LD = LD_NC>
__device__ __forceinline__ void rhs1d_half(const Geo& g, const double* __restrict__ u, int mesh, int i, int sx,
                                           double (&Ad)[Fields1<SYS>::F][K + 1], double (&Bd)[Fields1<SYS>::F][K + 1],
                                           double (&fS)[Fields1<SYS>::F]) {
  constexpr int F = Fields1<SYS>::F, M = K + 1, N = K + 1;
  const long long P = g.plane;
  const double* uo = u + (long long)(1 - mesh) * F * M * P;
  const int off = mesh == 0 ? -1 : 0;
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int a = 0; a < M; ++a) Ad[f][a] = Bd[f][a] = 0.0;
  bool mir = false;
  const int oi = BC == BC_GENERAL ? side_index(g, 0, 1 - mesh, unwrapped(g, 0, mesh, i) + sx + off, mir)
                                  : wrap_index<BC>(i + sx + off, g.nx);
  const double* c = uo + oi;
  double w[F][M];
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int a = 0; a < M; ++a) {
      w[f][a] = ldv<LD>(c + (f * M + a) * P);
      if (BC == BC_GENERAL && mir) w[f][a] = apply_sign(w[f][a], mirror_sign(true, false, SYS == SYS_EULER, f, a, 0));
    }
#pragma unroll
  for (int q = 0; q < N; ++q) {
    // the half's point constants (sx is a run-time value in the split kernels:
    // each constant is folded for both halves and chosen by a select, so no
    // FP64 work is added and both kernels use the same values)
    double po[M], pa[M], pb[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      po[a] = sx ? lpd(a, 0, xo1(N, 1, q)) : lpd(a, 0, xo1(N, 0, q));
      pa[a] = sx ? gw1(N, q) * lpd(a, 0, xs1(N, 1, q)) : gw1(N, q) * lpd(a, 0, xs1(N, 0, q));
      pb[a] = sx ? gw1(N, q) * lpd(a, 1, xs1(N, 1, q)) : gw1(N, q) * lpd(a, 1, xs1(N, 0, q));
    }
    double V[F], fl[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      double v = w[f][0];
#pragma unroll
      for (int a = 1; a < M; ++a) v = fma(po[a], w[f][a], v);
      V[f] = v;
    }
    flux1<SYS>(g, V, fl);
#pragma unroll
    for (int f = 0; f < F; ++f) {
#pragma unroll
      for (int a = 0; a < M; ++a) {
        Ad[f][a] = fma(pa[a], V[f], Ad[f][a]);
        if (a > 0) Bd[f][a] = fma(pb[a], fl[f], Bd[f][a]);
      }
    }
  }
  // face of this half: the overlapping cell's centre (xi' = 0)
  double V[F];
#pragma unroll
  for (int f = 0; f < F; ++f) {
    double v = w[f][0];
#pragma unroll
    for (int a = 2; a < M; a += 2) v = fma(lpd(a, 0, 0.0), w[f][a], v);
    V[f] = v;
  }
  flux1<SYS>(g, V, fS);
}

// L from the cell's sums (Ad, Bd: both halves added) and its face fluxes.
template <int SYS, int K, int LD = LD_NC>
__device__ __forceinline__ void rhs1d_finish(const Geo& g, const double* __restrict__ us, double inv_tm,
                                             const double (&Ad)[Fields1<SYS>::F][K + 1],
                                             const double (&Bd)[Fields1<SYS>::F][K + 1], const double* fL,
                                             const double* fR, double (&L)[Fields1<SYS>::F][K + 1]) {
  constexpr int F = Fields1<SYS>::F, M = K + 1;
  const long long P = g.plane;
  const double ih = g.i1x;  // 1/h from the host
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int a = 0; a < M; ++a) {
      // an explicit add: f_R can be a product (the Euler energy flux) that the
      // compiler would fuse into the subtraction in some kernels and not in
      // others (where it arrives by shuffle)
      const double face = (a & 1) ? __dadd_rn(fR[f], fL[f]) : __dsub_rn(fR[f], fL[f]);
      const double br = fma(0.25 * inv_tm, Ad[f][a], ih * fma(0.5, Bd[f][a], -face));
      L[f][a] = fma((double)(2 * a + 1), br, -inv_tm * ldv<LD>(us + (f * M + a) * P));
    }
}

// The whole cell by one thread: both halves, added.
template <int SYS, int BC, int K, int LD = LD_NC>
__device__ __forceinline__ void cell_rhs1d(const Geo& g, const double* __restrict__ u, int mesh, int i, double inv_tm,
                                           double (&L)[Fields1<SYS>::F][K + 1]) {
  constexpr int F = Fields1<SYS>::F, M = K + 1;
  double A0[F][M], B0[F][M], A1[F][M], B1[F][M], fL[F], fR[F];
  rhs1d_half<SYS, BC, K, LD>(g, u, mesh, i, 0, A0, B0, fL);
  rhs1d_half<SYS, BC, K, LD>(g, u, mesh, i, 1, A1, B1, fR);
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int a = 0; a < M; ++a) {
      A0[f][a] += A1[f][a];
      B0[f][a] += B1[f][a];
    }
  rhs1d_finish<SYS, K, LD>(g, u + (long long)mesh * F * M * g.plane + i, inv_tm, A0, B0, fL, fR, L);
}

enum { MODE1_RHS = 0, MODE1_STAGE = 1 };

// MODE1_RHS:   out = L(uin).
// MODE1_STAGE: out = sum_m cb.c[m] cb.u[m] + cb.ct tau L(uin)  (one Shu-Osher
//              stage), plus per-block sigma partials of out: sum of the cell
//              averages and max / min over the cell's K+1 Gauss points.
template <int SYS, int BC, int K, int MODE, int LD = LD_NC>
__device__ __forceinline__ void stage_cell1d(const Geo& g, const double* __restrict__ uin, const StageComb& cb,
                                             double* __restrict__ out, const double* __restrict__ dt,
                                             double* __restrict__ pblk, int mesh, int i) {
  constexpr int F = Fields1<SYS>::F, M = K + 1, N = K + 1;
  const bool active = i < cells_x(g, mesh);
  const int ic = active ? i : 0;
  const double tau = ldv<LD>(dt), tm = ldv<LD>(dt + 1);
  const double inv_tm = 1.0 / tm;
  double L[F][M];
  cell_rhs1d<SYS, BC, K, LD>(g, uin, mesh, ic, inv_tm, L);
  const long long P = g.plane;
  const long long base = (long long)mesh * F * M * P + ic;
  if (MODE == MODE1_RHS) {
    if (active)
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int a = 0; a < M; ++a) out[base + (f * M + a) * P] = L[f][a];
    return;
  } else {
    __shared__ double sh[96];
    const double tl = cb.ct * tau;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      double v[M];
#pragma unroll
      for (int a = 0; a < M; ++a) {
        const long long id = base + (f * M + a) * P;
        double s = tl * L[f][a];
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (m < cb.n) s = fma(cb.c[m], ldv<LD>(cb.u[m] + id), s);
        v[a] = s;
        if (active) out[id] = s;
      }
      double mx = -DINF1, mn = DINF1;
#pragma unroll
      for (int q = 0; q < N; ++q) {
        double val = v[0];
#pragma unroll
        for (int a = 1; a < M; ++a) val = fma(lpd(a, 0, gn1(N, q)), v[a], val);
        mx = fmax(mx, val);
        mn = fmin(mn, val);
      }
      double s = active ? v[0] : 0.0;
      if (BC == BC_GENERAL) s *= cell_weight(g, mesh, ic, 0, 1);  // a wall-centred dual cell counts half
      if (!active) {
        mx = -DINF1;
        mn = DINF1;
      }
      block_reduce3(s, mx, mn, sh);
      if (threadIdx.x == 0) {
        double* p = pblk + f * 3;
        p[0] = s;
        p[1] = mx;
        p[2] = mn;
      }
    }
  }
}

template <int SYS, int BC, int K, int MODE>
__global__ void __launch_bounds__(NT1) k_stage1d(Geo g, const double* __restrict__ uin, StageComb cb,
                                                 double* __restrict__ out, const double* __restrict__ dt,
                                                 double* __restrict__ partials) {
  constexpr int F = Fields1<SYS>::F;
  const int mesh = blockIdx.y;
  stage_cell1d<SYS, BC, K, MODE>(g, uin, cb, out, dt, partials + (mesh * (long long)gridDim.x + blockIdx.x) * F * 3,
                                 mesh, blockIdx.x * NT1 + threadIdx.x);
}

// The same stage with two lanes per cell (lanes 2c and 2c + 1 of a block of
// 2 NT1 threads take cell blockIdx.x * NT1 + c): lane sx sums half sx and the
// flux at its face, the pair swaps its sums by shuffle and adds them in the
// one-thread order, and both lanes finish the cell alike; lane sx stores the
// modes a with a % 2 == sx.  A 1D mesh of a few thousand cells gives each SM's
// FP64 pipe one warp or less, so the time of a phase is that of its longest
// warp: half the quadrature per lane shortens it.  The sigma partials of
// lane 0 are laid out as the one-thread block's threads (cell c in thread c)
// before the block reduction, so the partials, and hence sigma, are bit for
// bit those of the one-thread kernel.
template <int SYS, int BC, int K, int MODE, int LD = LD_NC>
__device__ __forceinline__ void stage_cell1d_2l(const Geo& g, const double* __restrict__ uin, const StageComb& cb,
                                                double* __restrict__ out, const double* __restrict__ dt,
                                                double* __restrict__ pblk, int mesh, int i, int sx) {
  constexpr int F = Fields1<SYS>::F, M = K + 1, N = K + 1;
  const unsigned full = 0xffffffffu;
  const bool active = i < cells_x(g, mesh);
  const int ic = active ? i : 0;
  const double tau = ldv<LD>(dt), tm = ldv<LD>(dt + 1);
  const double inv_tm = 1.0 / tm;
  double A[F][M], B[F][M], fS[F], fO[F];
  rhs1d_half<SYS, BC, K, LD>(g, uin, mesh, ic, sx, A, B, fS);
#pragma unroll
  for (int f = 0; f < F; ++f) {
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const double oa = __shfl_xor_sync(full, A[f][a], 1), ob = __shfl_xor_sync(full, B[f][a], 1);
      A[f][a] = sx ? oa + A[f][a] : A[f][a] + oa;  // half 0 + half 1
      B[f][a] = sx ? ob + B[f][a] : B[f][a] + ob;
    }
    fO[f] = __shfl_xor_sync(full, fS[f], 1);
  }
  double fL[F], fR[F];
#pragma unroll
  for (int f = 0; f < F; ++f) {
    fL[f] = sx ? fO[f] : fS[f];
    fR[f] = sx ? fS[f] : fO[f];
  }
  const long long P = g.plane;
  const long long base = (long long)mesh * F * M * P + ic;
  double L[F][M];
  rhs1d_finish<SYS, K, LD>(g, uin + base, inv_tm, A, B, fL, fR, L);
  if (MODE == MODE1_RHS) {
    if (active)
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int a = 0; a < M; ++a)
          if ((a & 1) == sx) out[base + (f * M + a) * P] = L[f][a];
    return;
  } else {
    __shared__ double sh[96];
    __shared__ double cell[3][NT1];  // one field's (sum, max, min) per cell
    const double tl = cb.ct * tau;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      double v[M];
#pragma unroll
      for (int a = 0; a < M; ++a) {
        const long long id = base + (f * M + a) * P;
        double s = tl * L[f][a];
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (m < cb.n) s = fma(cb.c[m], ldv<LD>(cb.u[m] + id), s);
        v[a] = s;
        if (active && (a & 1) == sx) out[id] = s;
      }
      double mx = -DINF1, mn = DINF1;
#pragma unroll
      for (int q = 0; q < N; ++q) {
        double val = v[0];
#pragma unroll
        for (int a = 1; a < M; ++a) val = fma(lpd(a, 0, gn1(N, q)), v[a], val);
        mx = fmax(mx, val);
        mn = fmin(mn, val);
      }
      double s = active ? v[0] : 0.0;
      if (BC == BC_GENERAL) s *= cell_weight(g, mesh, ic, 0, 1);  // a wall-centred dual cell counts half
      if (!active) {
        mx = -DINF1;
        mn = DINF1;
      }
      if (sx == 0) {
        const int c = threadIdx.x >> 1;
        cell[0][c] = s;
        cell[1][c] = mx;
        cell[2][c] = mn;
      }
      __syncthreads();
      const int t = threadIdx.x;
      s = t < NT1 ? cell[0][t] : 0.0;
      mx = t < NT1 ? cell[1][t] : -DINF1;
      mn = t < NT1 ? cell[2][t] : DINF1;
      block_reduce3(s, mx, mn, sh);  // its barriers also free cell[] for the next field
      if (threadIdx.x == 0) {
        double* p = pblk + f * 3;
        p[0] = s;
        p[1] = mx;
        p[2] = mn;
      }
    }
  }
}

template <int SYS, int BC, int K, int MODE>
__global__ void __launch_bounds__(2 * NT1) k_stage1d_2l(Geo g, const double* __restrict__ uin, StageComb cb,
                                                        double* __restrict__ out, const double* __restrict__ dt,
                                                        double* __restrict__ partials) {
  constexpr int F = Fields1<SYS>::F;
  const int mesh = blockIdx.y;
  stage_cell1d_2l<SYS, BC, K, MODE>(g, uin, cb, out, dt,
                                    partials + (mesh * (long long)gridDim.x + blockIdx.x) * F * 3, mesh,
                                    blockIdx.x * NT1 + (threadIdx.x >> 1), threadIdx.x & 1);
}

// delta^m = (2m+1) h^{m-1} / ((2K-1) m!) beta (|d^m (u^C-u^D)|_R + |...|_L) / sigma
// for m = 0..K, max over fields; then the exact damping of mode a by
// exp(-tau sum_{m <= a} delta^m).  The face points are the cell ends xi = +-1,
// which are the centres (xi' = 0) of the two overlapping cells.
template <int SYS, int BC, int K, bool WRITE_DELTA, int LD = LD_NC>
__device__ __forceinline__ void oe_cell1d(const Geo& g, const double* __restrict__ uh, double* __restrict__ usig,
                                          const double* __restrict__ dt, const double* __restrict__ sigma,
                                          double* __restrict__ delta_out, int* __restrict__ status, int mesh, int i,
                                          const double* __restrict__ isg = nullptr) {
  constexpr int F = Fields1<SYS>::F, M = K + 1;
  if (i >= cells_x(g, mesh)) return;
  const long long P = g.plane;
  const double* us = uh + (long long)mesh * F * M * P + i;
  const double* uo = uh + (long long)(1 - mesh) * F * M * P;
  const int off = mesh == 0 ? -1 : 0;
  bool mL = false, mR = false;
  const int iu = BC == BC_GENERAL ? unwrapped(g, 0, mesh, i) : i;
  const int oL = BC == BC_GENERAL ? side_index(g, 0, 1 - mesh, iu + off, mL) : wrap_index<BC>(i + off, g.nx);
  const int oR = BC == BC_GENERAL ? side_index(g, 0, 1 - mesh, iu + 1 + off, mR) : wrap_index<BC>(i + 1 + off, g.nx);
  double wa[F];
#pragma unroll
  for (int f = 0; f < F; ++f) wa[f] = ldv<LD>(us + (f * M) * P);
  double beta = speed1<SYS>(g, wa);
  if (beta < 0.0) {
    atomicOr(status, ST_NONPHYSICAL);
    beta = 0.0;
  }
  const double h = g.hx, d1 = g.i2x;  // 2/h from the host
  double km[M];  // (2m+1) h^{m-1} / ((2K-1) m!) (2/h)^m
  {
    double hp = g.i1x, dp = 1.0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      km[m] = (2 * m + 1) * hp * dp * (1.0 / ((2 * K - 1) * fact(m)));
      hp *= h;
      dp *= d1;
    }
  }
  double dl[M];
#pragma unroll
  for (int m = 0; m < M; ++m) dl[m] = 0.0;
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const double sg = ldv<LD>(sigma + mesh * F + f);
    double u[M], l[M], r[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      u[a] = ldv<LD>(us + (f * M + a) * P);
      l[a] = ldv<LD>(uo + (f * M + a) * P + oL);
      r[a] = ldv<LD>(uo + (f * M + a) * P + oR);
      if (BC == BC_GENERAL) {  // mirror images beyond a wall
        l[a] = apply_sign(l[a], mirror_sign(mL, false, SYS == SYS_EULER, f, a, 0));
        r[a] = apply_sign(r[a], mirror_sign(mR, false, SYS == SYS_EULER, f, a, 0));
      }
    }
    if (sg != 0.0) {
      const double is = isg ? beta * isg[f] : beta / sg;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        // reference-coordinate m-th derivatives: own trace at xi = +-1, other at 0
        double jr = 0.0, jl = 0.0;
#pragma unroll
        for (int a = m; a < M; ++a) {
          const double o = lpd(a, m, 0.0);
          jr = fma(lpd(a, m, 1.0), u[a], jr);
          jr = fma(-o, r[a], jr);
          jl = fma(lpd(a, m, -1.0), u[a], jl);
          jl = fma(-o, l[a], jl);
        }
        dl[m] = fmax(dl[m], km[m] * (fabs(jr) + fabs(jl)) * is);
      }
    }
  }
  if (WRITE_DELTA) {
    double* dp = delta_out + ((long long)mesh * g.nxs + i) * M;
#pragma unroll
    for (int m = 0; m < M; ++m) dp[m] = dl[m];
  }
  if (usig != nullptr) {
    const double tau = ldv<LD>(dt);
    double e[M];
    double rate = dl[0];
#pragma unroll
    for (int a = 1; a < M; ++a) {
      rate += dl[a];
      e[a] = exp(-tau * rate);
    }
    double* os = usig + (long long)mesh * F * M * P + i;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      os[(f * M) * P] = ldv<LD>(us + (f * M) * P);
#pragma unroll
      for (int a = 1; a < M; ++a) os[(f * M + a) * P] = ldv<LD>(us + (f * M + a) * P) * e[a];
    }
  }
}

template <int SYS, int BC, int K, bool WRITE_DELTA>
__global__ void __launch_bounds__(NT1) k_oe1d(Geo g, const double* __restrict__ uh, double* __restrict__ usig,
                                              const double* __restrict__ dt, const double* __restrict__ sigma,
                                              double* __restrict__ delta_out, int* __restrict__ status) {
  __shared__ double isg[Fields1<SYS>::F];  // 1/sigma of this mesh's fields, once per block
  oe_inv_sigma<Fields1<SYS>::F>(sigma, blockIdx.y, isg);
  oe_cell1d<SYS, BC, K, WRITE_DELTA>(g, uh, usig, dt, sigma, delta_out, status, blockIdx.y,
                                     blockIdx.x * NT1 + threadIdx.x, isg);
}

// The OE step with two lanes per cell (the layout of k_stage1d_2l): lane sx
// forms the jumps at its cell end (sx = 0: the left end, against the left
// overlapping cell; 1: the right end), the pair swaps them, and both lanes
// take delta^m exactly as oe_cell1d does; lane sx evaluates the decay factors
// of, and stores, the modes a with a % 2 == sx.  Bit for bit oe_cell1d's
// result.
template <int SYS, int BC, int K, bool WRITE_DELTA>
__device__ __forceinline__ void oe_cell1d_2l(const Geo& g, const double* __restrict__ uh, double* __restrict__ usig,
                                             const double* __restrict__ dt, const double* __restrict__ sigma,
                                             double* __restrict__ delta_out, int* __restrict__ status, int mesh,
                                             int i, int sx, const double* __restrict__ isg) {
  constexpr int F = Fields1<SYS>::F, M = K + 1;
  const unsigned full = 0xffffffffu;
  const bool active = i < cells_x(g, mesh);  // no early return: the pair shuffles
  const int ic = active ? i : 0;
  const long long P = g.plane;
  const double* us = uh + (long long)mesh * F * M * P + ic;
  const double* uo = uh + (long long)(1 - mesh) * F * M * P;
  const int off = mesh == 0 ? -1 : 0;
  bool mir = false;
  const int iu = BC == BC_GENERAL ? unwrapped(g, 0, mesh, ic) : ic;
  const int on = BC == BC_GENERAL ? side_index(g, 0, 1 - mesh, iu + sx + off, mir)
                                  : wrap_index<BC>(ic + sx + off, g.nx);
  double wa[F];
#pragma unroll
  for (int f = 0; f < F; ++f) wa[f] = __ldg(us + (f * M) * P);
  double beta = speed1<SYS>(g, wa);
  if (beta < 0.0) {
    if (active && sx == 0) atomicOr(status, ST_NONPHYSICAL);
    beta = 0.0;
  }
  const double h = g.hx, d1 = g.i2x;
  double km[M];
  {
    double hp = g.i1x, dp = 1.0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      km[m] = (2 * m + 1) * hp * dp * (1.0 / ((2 * K - 1) * fact(m)));
      hp *= h;
      dp *= d1;
    }
  }
  double dl[M];
#pragma unroll
  for (int m = 0; m < M; ++m) dl[m] = 0.0;
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const double sg = sigma[mesh * F + f];  // global or shared
    double u[M], nb[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      u[a] = __ldg(us + (f * M + a) * P);
      nb[a] = __ldg(uo + (f * M + a) * P + on);
      if (BC == BC_GENERAL) nb[a] = apply_sign(nb[a], mirror_sign(mir, false, SYS == SYS_EULER, f, a, 0));
    }
    const double is = beta * isg[f];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      // this lane's end: own trace at xi = -1 (sx = 0) or +1, the other cell at 0
      double j = 0.0;
#pragma unroll
      for (int a = m; a < M; ++a) {
        const double o = lpd(a, m, 0.0);
        j = fma(sx ? lpd(a, m, 1.0) : lpd(a, m, -1.0), u[a], j);
        j = fma(-o, nb[a], j);
      }
      const double jo = __shfl_xor_sync(full, j, 1);
      const double jr = sx ? j : jo, jl = sx ? jo : j;
      if (sg != 0.0) dl[m] = fmax(dl[m], km[m] * (fabs(jr) + fabs(jl)) * is);
    }
  }
  if (!active) return;
  if (WRITE_DELTA && sx == 0) {
    double* dp = delta_out + ((long long)mesh * g.nxs + ic) * M;
#pragma unroll
    for (int m = 0; m < M; ++m) dp[m] = dl[m];
  }
  if (usig != nullptr) {
    const double tau = __ldg(dt);
    double e[M];
    double rate = dl[0];
    e[0] = 1.0;
#pragma unroll
    for (int a = 1; a < M; ++a) {
      rate += dl[a];
      e[a] = (a & 1) == sx ? exp(-tau * rate) : 0.0;
    }
    double* os = usig + (long long)mesh * F * M * P + ic;
#pragma unroll
    for (int f = 0; f < F; ++f) {
#pragma unroll
      for (int a = 0; a < M; ++a)
        if ((a & 1) == sx) os[(f * M + a) * P] = a == 0 ? __ldg(us + (f * M) * P) : __ldg(us + (f * M + a) * P) * e[a];
    }
  }
}

template <int SYS, int BC, int K, bool WRITE_DELTA>
__global__ void __launch_bounds__(2 * NT1) k_oe1d_2l(Geo g, const double* __restrict__ uh, double* __restrict__ usig,
                                                     const double* __restrict__ dt, const double* __restrict__ sigma,
                                                     double* __restrict__ delta_out, int* __restrict__ status) {
  __shared__ double isg[Fields1<SYS>::F];  // 1/sigma of this mesh's fields, once per block
  oe_inv_sigma<Fields1<SYS>::F>(sigma, blockIdx.y, isg);
  oe_cell1d_2l<SYS, BC, K, WRITE_DELTA>(g, uh, usig, dt, sigma, delta_out, status, blockIdx.y,
                                        blockIdx.x * NT1 + (threadIdx.x >> 1), threadIdx.x & 1, isg);
}

// The OE step of a step's stage with sigma taken in the same launch: warp f
// of every block folds the stage kernel's block partials for (its mesh, field
// f) in warp_sigma's fixed order (the order of k_sigma, so sigma is the same
// bits), into shared memory; block 0 of each mesh also stores sigma and avg
// for the context.  One launch instead of two per stage: a 1D stage is a few
// microseconds of work, and a launch costs about as much.
template <int SYS, int BC, int K, bool WRITE_DELTA>
__global__ void __launch_bounds__(2 * NT1) k_oe1d_2l_sig(Geo g, const double* __restrict__ uh,
                                                         double* __restrict__ usig, const double* __restrict__ dt,
                                                         const double* __restrict__ partials, long long nblk,
                                                         SigmaNorm sn, double* __restrict__ sigma,
                                                         double* __restrict__ avg, double* __restrict__ delta_out,
                                                         int* __restrict__ status) {
  constexpr int F = Fields1<SYS>::F;
  __shared__ double s_sig[2 * F], s_avg[2 * F], isg[F];
  const int mesh = blockIdx.y, w = threadIdx.x >> 5;
  if (w < F) warp_sigma<LD_NC>(partials, nblk, F, mesh, w, sn, s_avg, s_sig);
  __syncthreads();
  if (threadIdx.x < F) {
    const double sg = s_sig[mesh * F + threadIdx.x];
    isg[threadIdx.x] = sg != 0.0 ? 1.0 / sg : 0.0;
    if (blockIdx.x == 0) {
      sigma[mesh * F + threadIdx.x] = sg;
      avg[mesh * F + threadIdx.x] = s_avg[mesh * F + threadIdx.x];
    }
  }
  __syncthreads();
  oe_cell1d_2l<SYS, BC, K, WRITE_DELTA>(g, uh, usig, dt, s_sig, delta_out, status, mesh,
                                        blockIdx.x * NT1 + (threadIdx.x >> 1), threadIdx.x & 1, isg);
}

template <int SYS, int K>
__global__ void k_wave1d(Geo g, const double* __restrict__ u, double* __restrict__ partial,
                         unsigned long long* __restrict__ ticket, double T_end, double* __restrict__ dt,
                         double* __restrict__ time, int* __restrict__ status) {
  constexpr int F = Fields1<SYS>::F, M = K + 1;
  __shared__ double sh[32];
  const long long n = 2 * g.plane;
  double mx = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    if (cell >= cells_x(g, mesh)) continue;  // the primal mesh's unused slot
    const double* us = u + (long long)mesh * F * M * g.plane + cell;
    double w[F];
#pragma unroll
    for (int f = 0; f < F; ++f) w[f] = us[(f * M) * g.plane];
    const double s = speed1<SYS>(g, w);
    if (s >= 0.0) mx = fmax(mx, s);
    else atomicOr(status, ST_NONPHYSICAL);
  }
  mx = block_reduce_max(mx, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 2] = mx;
    partial[blockIdx.x * 2 + 1] = 0.0;
  }
  // the last block to finish (ticket: a monotone counter, zero when the
  // context was made) folds the partials (the maximum is exact in any order)
  // and sets tau, tau_max and the time: one launch for the time step
  if (last_block(ticket)) {
    double bx = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) bx = fmax(bx, __ldcg(partial + 2 * b));
    __syncthreads();  // sh is reused
    bx = block_reduce_max(bx, sh);
    if (threadIdx.x == 0) finish_dt(bx, 0.0, g.hx, g.hy, 1, g.cfl, T_end, dt, time);
  }
}

// Sampling points of the initial projection: K+1 Gauss points on each half of
// every cell of both meshes, layout [mesh][i][s][q].
template <int K>
__global__ void k_points1d(Geo g, double ax, double bx, double* __restrict__ x) {
  constexpr int N = K + 1, R = 2 * N;
  const long long n = 2 * g.plane * R;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % R);
    const long long c = t / R;
    const int mesh = (int)(c / g.plane);
    const long long i = c - mesh * g.plane;
    // the unused primal slot takes the dual cell's points (ignored)
    const int cm = i < cells_x(g, mesh) ? mesh : 1;
    const double xc = ax + (unwrapped(g, 0, cm, (int)i) + 0.5 + 0.5 * cm) * g.hx;
    double xp = xc + 0.5 * g.hx * xs1(N, r / N, r % N);
    if (g.bcs[0] == SIDE_REFLECTIVE && xp < ax) xp = 2.0 * ax - xp;  // folded back across a wall
    if (g.bcs[1] == SIDE_REFLECTIVE && xp > bx) xp = 2.0 * bx - xp;
    x[t] = xp;
  }
}

// L2 projection onto P^K from values at the points of k_points1d:
// u_a = (2a+1)/2 sum_{s,q} (w_q / 2) u0(x_sq) P_a(xi_sq).
template <int F, int K>
__global__ void k_project1d(Geo g, const double* __restrict__ vals, double* __restrict__ u) {
  constexpr int M = K + 1, N = K + 1, R = 2 * N;
  const long long n = 2 * g.plane;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    double acc[F][M];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int a = 0; a < M; ++a) acc[f][a] = 0.0;
    const double* v = vals + c * R * F;
    // the outer half of a wall-centred dual cell was sampled at its mirror
    // image inside: the normal momentum (Euler, field 1) changes sign there
    const bool wl = mesh == 1 && g.bcs[0] == SIDE_REFLECTIVE && cell == g.nx;
    const bool wr = mesh == 1 && g.bcs[1] == SIDE_REFLECTIVE && cell == g.nx - 1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double xi = xs1(N, r / N, r % N), w = 0.5 * gw1(N, r % N);
      const bool folded = (wl && r / N == 0) || (wr && r / N == 1);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const double x = (folded && F == 3 && f == 1) ? -w * v[r * F + f] : w * v[r * F + f];
#pragma unroll
        for (int a = 0; a < M; ++a) acc[f][a] = fma(x, lpd(a, 0, xi), acc[f][a]);
      }
    }
    const bool used = cell < cells_x(g, mesh);  // the primal mesh's unused slot is set to 0
    double* o = u + (long long)mesh * F * M * g.plane + cell;
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int a = 0; a < M; ++a) o[(f * M + a) * g.plane] = used ? acc[f][a] * ((2 * a + 1) / 2.0) : 0.0;
  }
}

// ------------------------------------------------------- persistent step --

// Maximum wave speed over the cell averages of both meshes of `u`, grid-stride
// (the same speeds as k_wave1d), into wpart[blockIdx.x]; the last block to
// finish takes the maximum over all blocks and sets (tau, tau_max, time)
// exactly as k_dt_final does.
template <int SYS, int K>
__device__ __forceinline__ void persist_wave1d(const Geo& g, const Persist1& a, const double* u, double* sh) {
  constexpr int F = Fields1<SYS>::F, M = K + 1;
  const long long ncell = 2 * g.plane;
  double mx = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    if (c - mesh * g.plane >= cells_x(g, mesh)) continue;  // the primal mesh's unused slot
    const double* uc = u + (long long)mesh * F * M * g.plane + (c - mesh * g.plane);
    double w[F];
#pragma unroll
    for (int f = 0; f < F; ++f) w[f] = ldv<LD_CA>(uc + (f * M) * g.plane);
    const double sp = speed1<SYS>(g, w);
    if (sp >= 0.0) mx = fmax(mx, sp);
    else atomicOr(a.status, ST_NONPHYSICAL);
  }
  mx = block_reduce_max(mx, sh);
  if (threadIdx.x == 0) a.wpart[blockIdx.x] = mx;
  if (last_block(a.bar + 1)) {
    // all threads of the last block fold the partials (the maximum is exact:
    // any order gives k_dt_final's value)
    double bx = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) bx = fmax(bx, ldv<LD_CA>(a.wpart + b));
    __syncthreads();  // sh is reused
    bx = block_reduce_max(bx, sh);
    if (threadIdx.x == 0) finish_dt(bx, 0.0, g.hx, g.hy, 1, g.cfl, a.T_end, a.dt, a.time);
  }
}

// nsteps steps in one cooperative launch.  Phases, each ended by a grid
// barrier with a bounded wait: [stage tiles, then sigma by the last block to
// finish them] -> [OE tiles (or a copy without OE); after the last stage of a
// step, the next step's wave speeds and tau, by the last block] per stage, plus
// one wave-speed phase before the first step: 2 barriers per stage.  Stage
// tile b is mesh b & 1, stage block b >> 1 of the per-phase layout, so the
// sigma partials land where the per-phase kernel puts them; the wave speeds
// come from u_h's cell averages, which the OE step leaves unchanged.
template <int SYS, int BC, int K>
__global__ void __launch_bounds__(NT1) k_persist1d(Geo g, Persist1 a) {
  constexpr int F = Fields1<SYS>::F, M = K + 1;
  __shared__ double sh[32];
  __shared__ double isg[F];  // 1/sigma of the OE phase's current tile (its mesh)
  const long long ntiles = 2 * a.nblk;
  persist_wave1d<SYS, K>(g, a, a.uin[0], sh);
  if (!grid_sync(a.bar, a.expected, a.status, a.limit_ns)) return;
  for (int s = 0; s < a.nsteps; ++s) {
    for (int l = 0; l < a.nst; ++l) {
      for (long long b = blockIdx.x; b < ntiles; b += gridDim.x) {
        const int mesh = (int)(b & 1);
        const long long blk = b >> 1;
        stage_cell1d<SYS, BC, K, MODE1_STAGE, LD_CA>(g, a.uin[l], a.cb[l], a.ua, a.dt,
                                                     a.partials + (mesh * a.nblk + blk) * F * 3, mesh,
                                                     (int)(blk * NT1) + threadIdx.x);
      }
      if (a.oe && last_block(a.bar + 1)) {
        for (int it = threadIdx.x >> 5; it < 2 * F; it += blockDim.x >> 5)
          warp_sigma<LD_CA>(a.partials, a.nblk, F, it / F, it % F, a.sn, a.avg, a.sigma);
      }
      if (!grid_sync(a.bar, a.expected, a.status, a.limit_ns)) return;
      if (a.oe) {
        for (long long b = blockIdx.x; b < ntiles; b += gridDim.x) {
          __syncthreads();  // the previous tile's readers of isg are done
          oe_inv_sigma<F>(a.sigma, (int)(b & 1), isg);
          oe_cell1d<SYS, BC, K, false, LD_CA>(g, a.ua, a.dst[l], a.dt, a.sigma, nullptr, a.status, (int)(b & 1),
                                              (int)((b >> 1) * NT1) + threadIdx.x, isg);
        }
      } else {
        const long long n = 2LL * F * M * g.plane;
        for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
             q += (long long)gridDim.x * blockDim.x)
          a.dst[l][q] = ldv<LD_CA>(a.ua + q);
      }
      const bool last = l == a.nst - 1 && s + 1 == a.nsteps;
      if (last) return;  // the kernel's end orders everything for the host
      if (l == a.nst - 1) persist_wave1d<SYS, K>(g, a, a.ua, sh);
      if (!grid_sync(a.bar, a.expected, a.status, a.limit_ns)) return;
    }
  }
}

// ----------------------------------------------------------------- launch --

template <int V>
using IC = std::integral_constant<int, V>;

// fn(IC<SYS>, IC<BC>, IC<K>) for the runtime (sys, bc, k); k in {1, 2, 3}
template <class Fn>
static void by_sys_bc_k(int sys, int bc, int k, Fn&& fn) {
  auto kk = [&](auto S, auto B) {
    if (k == 1) fn(S, B, IC<1>{});
    else if (k == 2) fn(S, B, IC<2>{});
    else fn(S, B, IC<3>{});
  };
  auto bb = [&](auto S) {
    if (bc == BC_PERIODIC) kk(S, IC<BC_PERIODIC>{});
    else if (bc == BC_TRANSMISSIVE) kk(S, IC<BC_TRANSMISSIVE>{});
    else kk(S, IC<BC_GENERAL>{});
  };
  if (sys == SYS_EULER) bb(IC<SYS_EULER>{});
  else if (sys == SYS_BURGERS) bb(IC<SYS_BURGERS>{});
  else bb(IC<SYS_ADV>{});
}

long long partial_blocks_1d(const Geo& g) { return (g.nxs + NT1 - 1) / NT1; }

cudaError_t launch_stage1d(int sys, int bc, int k, const Geo& g, int rhs_only, const double* uin,
                           const StageComb& cb, double* out, const double* dt, double* partials, cudaStream_t st) {
  const dim3 grid((g.nxs + NT1 - 1) / NT1, 2);  // NT1 cells per block, two lanes each
  by_sys_bc_k(sys, bc, k, [&](auto S, auto B, auto Kc) {
    constexpr int S_ = decltype(S)::value, B_ = decltype(B)::value, K_ = decltype(Kc)::value;
    if (rhs_only) k_stage1d_2l<S_, B_, K_, MODE1_RHS><<<grid, 2 * NT1, 0, st>>>(g, uin, cb, out, dt, partials);
    else k_stage1d_2l<S_, B_, K_, MODE1_STAGE><<<grid, 2 * NT1, 0, st>>>(g, uin, cb, out, dt, partials);
  });
  return cudaGetLastError();
}

cudaError_t launch_oe1d(int sys, int bc, int k, const Geo& g, const double* uh, double* usig, const double* dt,
                        const double* sigma, double* delta, int* status, cudaStream_t st) {
  const dim3 grid((g.nxs + NT1 - 1) / NT1, 2);
  by_sys_bc_k(sys, bc, k, [&](auto S, auto B, auto Kc) {
    constexpr int S_ = decltype(S)::value, B_ = decltype(B)::value, K_ = decltype(Kc)::value;
    if (delta) k_oe1d_2l<S_, B_, K_, true><<<grid, 2 * NT1, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
    else k_oe1d_2l<S_, B_, K_, false><<<grid, 2 * NT1, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
  });
  return cudaGetLastError();
}

cudaError_t launch_oe1d_sig(int sys, int bc, int k, const Geo& g, const double* uh, double* usig, const double* dt,
                            const double* partials, long long nblk, const SigmaNorm& sn, double* sigma, double* avg,
                            double* delta, int* status, cudaStream_t st) {
  const dim3 grid((g.nxs + NT1 - 1) / NT1, 2);
  by_sys_bc_k(sys, bc, k, [&](auto S, auto B, auto Kc) {
    constexpr int S_ = decltype(S)::value, B_ = decltype(B)::value, K_ = decltype(Kc)::value;
    if (delta)
      k_oe1d_2l_sig<S_, B_, K_, true><<<grid, 2 * NT1, 0, st>>>(g, uh, usig, dt, partials, nblk, sn, sigma, avg, delta,
                                                               status);
    else
      k_oe1d_2l_sig<S_, B_, K_, false><<<grid, 2 * NT1, 0, st>>>(g, uh, usig, dt, partials, nblk, sn, sigma, avg,
                                                                delta, status);
  });
  return cudaGetLastError();
}

int wave_blocks_1d(const Geo& g) {
  long long b = (2 * g.plane + 255) / 256;
  return (int)(b < 1184 ? b : 1184);
}

cudaError_t launch_dt1d(int sys, int k, const Geo& g, const double* u, double* partial, int nblk, double T_end,
                        double* dt, double* time, int* status, cudaStream_t st) {
  // partial holds nblk pairs and, after them, the ticket counter of the last block
  unsigned long long* ticket = (unsigned long long*)(partial + 2 * (long long)nblk);
  by_sys_bc_k(sys, BC_PERIODIC, k, [&](auto S, auto, auto Kc) {
    k_wave1d<decltype(S)::value, decltype(Kc)::value><<<nblk, 256, 0, st>>>(g, u, partial, ticket, T_end, dt, time,
                                                                              status);
  });
  return cudaGetLastError();
}

// One block per SM: a 1D step is latency-bound and the FP64 pipe of an SM is
// shared by its blocks, so the persistent grid spreads its blocks over the
// SMs (each block reserves more than half of an SM's shared memory, which the
// kernel does not use, so that no two blocks share an SM) and loops over the
// tiles when there are more tiles than SMs.
constexpr size_t PERSIST1_SMEM = 120 * 1024;

cudaError_t persist_grid_1d(int sys, int bc, int k, const Geo& g, int nsm, long long* grid) {
  cudaError_t e = cudaSuccess;
  int occ = 0;
  by_sys_bc_k(sys, bc, k, [&](auto S, auto B, auto Kc) {
    auto kern = k_persist1d<decltype(S)::value, decltype(B)::value, decltype(Kc)::value>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PERSIST1_SMEM);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT1, PERSIST1_SMEM);
  });
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  long long gsz = (long long)occ * nsm;
  const long long tiles = 2 * partial_blocks_1d(g);
  *grid = gsz < tiles ? gsz : tiles;
  return cudaSuccess;
}

cudaError_t launch_persist1d(int sys, int bc, int k, const Geo& g, const Persist1& a, long long grid,
                             cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned long long), st);  // barrier, tickets
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NT1);
  cfg.dynamicSmemBytes = PERSIST1_SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  by_sys_bc_k(sys, bc, k, [&](auto S, auto B, auto Kc) {
    e = cudaLaunchKernelEx(&cfg, k_persist1d<decltype(S)::value, decltype(B)::value, decltype(Kc)::value>, g, a);
  });
  return e;
}

cudaError_t launch_points1d(int k, const Geo& g, double ax, double bx, double* x, cudaStream_t st) {
  if (k == 1) k_points1d<1><<<256, 256, 0, st>>>(g, ax, bx, x);
  else if (k == 2) k_points1d<2><<<256, 256, 0, st>>>(g, ax, bx, x);
  else k_points1d<3><<<256, 256, 0, st>>>(g, ax, bx, x);
  return cudaGetLastError();
}

cudaError_t launch_project1d(int sys, int k, const Geo& g, const double* vals, double* u, cudaStream_t st) {
  by_sys_bc_k(sys, BC_PERIODIC, k, [&](auto S, auto, auto Kc) {
    constexpr int F = Fields1<decltype(S)::value>::F;
    k_project1d<F, decltype(Kc)::value><<<256, 128, 0, st>>>(g, vals, u);
  });
  return cudaGetLastError();
}

}  // namespace oecdg
