// oecdg_2d.cu -- 2D Q^2 kernels of the OECDG forward step (arXiv:2503.12473).
//
// One thread per cell of one mesh (blockIdx.z = mesh); primal and dual cells run
// the same code: cell K's four sub-cells (quarters) and its eight half-faces all
// lie in the four overlapping cells of the other mesh,
//   primal (i,j): dual (i-1+sx, j-1+sy);   dual (i,j): primal (i+sx, j+sy),
// and in the overlapping cell the point of K's reference coordinate xi sits at
// xi' = xi + 1 - 2 sx (the overlapping cell's centre lies on K's face).
#include "oecdg_common.cuh"
#include "oecdg_kernels.h"

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
constexpr double DINF = __builtin_huge_val();

template <int SYS>
struct Fields {
  static constexpr int F = SYS == SYS_EULER ? 4 : 1;
};

// flux of one point: both components
template <int SYS>
__device__ __forceinline__ void flux_both(const Geo& g, const double* V, double* f1, double* f2) {
  if (SYS == SYS_EULER) {
    Euler2::both(V, g.gamma, f1, f2);
  } else {
    f1[0] = g.adv_x * V[0];
    f2[0] = g.adv_y * V[0];
  }
}
template <int SYS>
__device__ __forceinline__ void flux_x(const Geo& g, const double* V, double* f1) {
  if (SYS == SYS_EULER) Euler2::fx(V, g.gamma, f1);
  else f1[0] = g.adv_x * V[0];
}
template <int SYS>
__device__ __forceinline__ void flux_y(const Geo& g, const double* V, double* f2) {
  if (SYS == SYS_EULER) Euler2::fy(V, g.gamma, f2);
  else f2[0] = g.adv_y * V[0];
}

// CDG right-hand side of one cell, Eq. (eq:2D_H) restricted to the test
// functions of cell (i, j) of `mesh`:
//   L_ab = (2a+1)(2b+1)/(hx hy) * [ (1/tau_max) int_K (w - u_K) phi_ab
//          + int_K f(w) . grad phi_ab - sum_e int_e f(w) . n phi_ab ],
// w = the other mesh's solution.  Volume integrals by the 3x3 Gauss rule of
// each quarter sub-cell, face integrals by the 3-point rule of each half-face.
// Sum factorisation by x-columns: for each column of points (fixed xi) the
// overlapping cell is contracted in x, evaluated along the column, the fluxes
// are formed and projected in y into A (dissipation + f2 terms) and B (f1
// term); the column is then projected in x into the accumulators R.  The
// half-faces normal to x are two more columns (xi = -1, +1), the half-faces
// normal to y two more points of every column (eta = -1, +1).
// R holds 16 hx hy / ((2a+1)(2b+1)) times the bracket, indexed [f][b][a].
template <int SYS, int BC>
__device__ __forceinline__ void cell_rhs2d(const Geo& g, const double* __restrict__ u, int mesh, int i, int j,
                                           double inv_tm, double (&L)[Fields<SYS>::F][9]) {
  constexpr int F = Fields<SYS>::F;
  const long long P = g.plane;
  const double* uo = u + (long long)(1 - mesh) * F * 9 * P;
  const double* us = u + (long long)mesh * F * 9 * P;
  const int off = mesh == 0 ? -1 : 0;
  const double kd = 0.5 * g.hy * inv_tm;  // dissipation scale inside A
  double R[F][3][3];
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) R[f][b][a] = 0.0;

  const int oj0 = wrap_index<BC>(j + off, g.ny), oj1 = wrap_index<BC>(j + 1 + off, g.ny);
#pragma unroll
  for (int sx = 0; sx < 2; ++sx) {
    const int oi = wrap_index<BC>(i + sx + off, g.nx);
    const double* c0 = uo + (long long)oj0 * g.nx + oi;
    const double* c1 = uo + (long long)oj1 * g.nx + oi;
    // ---- half-faces normal to x: xi = 2 sx - 1 (in the overlapping cell xi' = 0)
    {
      double Bf[F][3];
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int b = 0; b < 3; ++b) Bf[f][b] = 0.0;
#pragma unroll
      for (int sy = 0; sy < 2; ++sy) {
        const double* c = sy ? c1 : c0;
        double T[F][3];
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int b = 0; b < 3; ++b)
            T[f][b] = fma(-0.5, __ldg(c + (f * 9 + b * 3 + 2) * P), __ldg(c + (f * 9 + b * 3) * P));
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const double eo = xs_other(sy, q), es = xs_self(sy, q);
          double V[F], f1[F];
#pragma unroll
          for (int f = 0; f < F; ++f) V[f] = fma(lp(2, eo), T[f][2], fma(eo, T[f][1], T[f][0]));
          flux_x<SYS>(g, V, f1);
#pragma unroll
          for (int f = 0; f < F; ++f) {
            Bf[f][0] = fma(gwt(q), f1[f], Bf[f][0]);
            Bf[f][1] = fma(gwt(q) * es, f1[f], Bf[f][1]);
            Bf[f][2] = fma(gwt(q) * lp(2, es), f1[f], Bf[f][2]);
          }
        }
      }
      // R += (-s) P_a(s) (4/hx) Bf, s = 2 sx - 1
      const double sc = 4.0 / g.hx;
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const double v = sc * Bf[f][b];
          if (sx) {
            R[f][b][0] -= v;
            R[f][b][1] -= v;
            R[f][b][2] -= v;
          } else {
            R[f][b][0] += v;
            R[f][b][1] -= v;
            R[f][b][2] += v;
          }
        }
    }
    // ---- the three volume columns of this half
#pragma unroll
    for (int qx = 0; qx < 3; ++qx) {
      const double xo = xs_other(sx, qx), xsf = xs_self(sx, qx);
      double A[F][3], B[F][3];
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int b = 0; b < 3; ++b) A[f][b] = B[f][b] = 0.0;
#pragma unroll
      for (int sy = 0; sy < 2; ++sy) {
        const double* c = sy ? c1 : c0;
        double T[F][3];
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const double* cb = c + (f * 9 + b * 3) * P;
            T[f][b] = fma(lp(2, xo), __ldg(cb + 2 * P), fma(xo, __ldg(cb + P), __ldg(cb)));
          }
#pragma unroll
        for (int qy = 0; qy < 3; ++qy) {
          const double eo = xs_other(sy, qy), es = xs_self(sy, qy);
          const double w = gwt(qy);
          double V[F], f1[F], f2[F];
#pragma unroll
          for (int f = 0; f < F; ++f) V[f] = fma(lp(2, eo), T[f][2], fma(eo, T[f][1], T[f][0]));
          flux_both<SYS>(g, V, f1, f2);
#pragma unroll
          for (int f = 0; f < F; ++f) {
            const double g0 = kd * V[f];
            A[f][0] = fma(w, g0, A[f][0]);
            A[f][1] = fma(w * es, g0, fma(w, f2[f], A[f][1]));
            A[f][2] = fma(w * lp(2, es), g0, fma(w * dlp(2, es), f2[f], A[f][2]));
            B[f][0] = fma(w, f1[f], B[f][0]);
            B[f][1] = fma(w * es, f1[f], B[f][1]);
            B[f][2] = fma(w * lp(2, es), f1[f], B[f][2]);
          }
        }
        // the half-face normal to y crossed by this column: eta = 2 sy - 1, eta' = 0
        {
          double V[F], f2[F];
#pragma unroll
          for (int f = 0; f < F; ++f) V[f] = fma(-0.5, T[f][2], T[f][0]);
          flux_y<SYS>(g, V, f2);
#pragma unroll
          for (int f = 0; f < F; ++f) {
            // A_b += -2 s P_b(s) f2, s = 2 sy - 1
            if (sy) {
              A[f][0] = fma(-2.0, f2[f], A[f][0]);
              A[f][1] = fma(-2.0, f2[f], A[f][1]);
              A[f][2] = fma(-2.0, f2[f], A[f][2]);
            } else {
              A[f][0] = fma(2.0, f2[f], A[f][0]);
              A[f][1] = fma(-2.0, f2[f], A[f][1]);
              A[f][2] = fma(2.0, f2[f], A[f][2]);
            }
          }
        }
      }
      // R += w_qx [ P_a(xi) (2/hy) A + P'_a(xi) (2/hx) B ]
      const double wa = gwt(qx) * 2.0 / g.hy, wb = gwt(qx) * 2.0 / g.hx;
      const double wa1 = wa * xsf, wa2 = wa * lp(2, xsf), wb2 = wb * dlp(2, xsf);
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          R[f][b][0] = fma(wa, A[f][b], R[f][b][0]);
          R[f][b][1] = fma(wa1, A[f][b], fma(wb, B[f][b], R[f][b][1]));
          R[f][b][2] = fma(wa2, A[f][b], fma(wb2, B[f][b], R[f][b][2]));
        }
    }
  }
  // L_ab = (2a+1)(2b+1)/16 R_ab - u_ab / tau_max  (the -(1/tau_max) int u_K phi term
  // is exact through the diagonal mass matrix)
  const double* cs = us + (long long)j * g.nx + i;
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a)
        L[f][b * 3 + a] = fma((2 * a + 1) * (2 * b + 1) / 16.0, R[f][b][a],
                              -inv_tm * __ldg(cs + (f * 9 + b * 3 + a) * P));
}

// MODE_RHS: out = L(uin) with tau_max = dt[1].
// MODE_STAGE: out = ca un + cb (uin + tau L(uin)) with (tau, tau_max) = dt[0..1],
//   plus per-block partials of the sigma reduction of the output:
//   partials[(mesh * nblk + blk) * F * 3 + f * 3 + {0,1,2}] = (sum of cell
//   averages, max and min of the values at the cell's 3x3 Gauss points).
enum { MODE_RHS = 0, MODE_STAGE = 1 };

template <int SYS, int BC, int MODE>
__global__ void __launch_bounds__(NT, OECDG_STAGE_MINB) k_stage2d(Geo g, const double* __restrict__ uin,
                                                const double* __restrict__ un, double* __restrict__ out,
                                                const double* __restrict__ dt, double ca, double cb,
                                                double* __restrict__ partials) {
  constexpr int F = Fields<SYS>::F;
  const int mesh = blockIdx.z;
  const int i = blockIdx.x * TX + (threadIdx.x % TX);
  const int j = blockIdx.y * TY + (threadIdx.x / TX);
  const bool active = i < g.nx && j < g.ny;
  const int ic = active ? i : 0, jc = active ? j : 0;
  const double tau = dt[0], tm = dt[1];
  const double inv_tm = 1.0 / tm;
  double L[F][9];
  cell_rhs2d<SYS, BC>(g, uin, mesh, ic, jc, inv_tm, L);
  const long long P = g.plane;
  const long long base = (long long)mesh * F * 9 * P + (long long)jc * g.nx + ic;
  if (MODE == MODE_RHS) {
    if (active)
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int m = 0; m < 9; ++m) out[base + (f * 9 + m) * P] = L[f][m];
    return;
  } else {
    __shared__ double sh[96];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      double v[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        const long long id = base + (f * 9 + m) * P;
        double s = fma(tau, L[f][m], __ldg(uin + id));
        if (ca != 0.0) s = fma(ca, __ldg(un + id), cb * s);
        v[m] = s;
        if (active) out[id] = s;
      }
      // values at the cell's own 3x3 Gauss points: x-contraction then y
      double mx = -DINF, mn = DINF;
#pragma unroll
      for (int qy = 0; qy < 3; ++qy) {
        double t[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
          t[a] = fma(lp(2, gnode(qy)), v[6 + a], fma(gnode(qy), v[3 + a], v[a]));
#pragma unroll
        for (int qx = 0; qx < 3; ++qx) {
          const double val = fma(lp(2, gnode(qx)), t[2], fma(gnode(qx), t[1], t[0]));
          mx = fmax(mx, val);
          mn = fmin(mn, val);
        }
      }
      double s = active ? v[0] : 0.0;
      if (!active) {
        mx = -DINF;
        mn = DINF;
      }
      block_reduce3(s, mx, mn, sh);
      if (threadIdx.x == 0) {
        const long long nblk = (long long)gridDim.x * gridDim.y;
        const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
        double* p = partials + ((mesh * nblk + blk) * F + f) * 3;
        p[0] = s;
        p[1] = mx;
        p[2] = mn;
      }
    }
  }
}

// Fixed-order reduction of the block partials: avg and sigma per mesh and
// field (Section 2.2): avg = mean of the cell averages over the stored cells,
// sigma = max(max - avg, avg - min) over the cell Gauss points.
// grid = (F, 2), block = 1024.
__global__ void k_sigma(const double* __restrict__ partials, long long nblk, int F, long long ncell,
                        double* __restrict__ sigma, double* __restrict__ avg) {
  const int f = blockIdx.x, mesh = blockIdx.y;
  __shared__ double sh[96];
  double s = 0.0, mx = -DINF, mn = DINF;
  for (long long b = threadIdx.x; b < nblk; b += blockDim.x) {
    const double* p = partials + ((mesh * nblk + b) * F + f) * 3;
    s += p[0];
    mx = fmax(mx, p[1]);
    mn = fmin(mn, p[2]);
  }
  block_reduce3(s, mx, mn, sh);
  if (threadIdx.x == 0) {
    const double a = s / (double)ncell;
    avg[mesh * F + f] = a;
    sigma[mesh * F + f] = fmax(mx - a, a - mn);
  }
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
template <int SYS, int BC, bool WRITE_DELTA>
__global__ void __launch_bounds__(NT, OECDG_OE_MINB) k_oe2d(Geo g, const double* __restrict__ uh, double* __restrict__ usig,
                                             const double* __restrict__ dt, const double* __restrict__ sigma,
                                             double* __restrict__ delta_out, int* __restrict__ status) {
  constexpr int F = Fields<SYS>::F;
  const int mesh = blockIdx.z;
  const int i = blockIdx.x * TX + (threadIdx.x % TX);
  const int j = blockIdx.y * TY + (threadIdx.x / TX);
  if (i >= g.nx || j >= g.ny) return;
  const long long P = g.plane;
  const double* us = uh + (long long)mesh * F * 9 * P + (long long)j * g.nx + i;
  const double* uo = uh + (long long)(1 - mesh) * F * 9 * P;
  const int off = mesh == 0 ? -1 : 0;
  const int oi0 = wrap_index<BC>(i + off, g.nx), oi1 = wrap_index<BC>(i + 1 + off, g.nx);
  const int oj0 = wrap_index<BC>(j + off, g.ny), oj1 = wrap_index<BC>(j + 1 + off, g.ny);

  // wave speeds beta_{e,K} at the cell average
  double bx, by;
  if (SYS == SYS_EULER) {
    const double rho = __ldg(us), mx = __ldg(us + 9 * P), my = __ldg(us + 18 * P), E = __ldg(us + 27 * P);
    const double r = 1.0 / rho;
    const double vx = mx * r, vy = my * r;
    const double p = (g.gamma - 1.0) * (E - 0.5 * (mx * vx + my * vy));
    double c = 0.0;
    if (rho > 0.0 && p > 0.0) {
      c = sqrt(g.gamma * p * r);
    } else {
      atomicOr(status, ST_NONPHYSICAL);
    }
    bx = fabs(vx) + c;
    by = fabs(vy) + c;
    if (!(rho > 0.0 && p > 0.0)) bx = by = 0.0;
  } else {
    bx = fabs(g.adv_x);
    by = fabs(g.adv_y);
  }
  // (2m+1) h^{m-1} / ((2k-1) m!) / 4  (1/4: the half-face rule over |e|)
  const double cx0 = 1.0 / (12.0 * g.hx), cx1 = 0.25, cx2 = 5.0 * g.hx / 24.0;
  const double cy0 = 1.0 / (12.0 * g.hy), cy1 = 0.25, cy2 = 5.0 * g.hy / 24.0;
  const double dx1 = 2.0 / g.hx, dy1 = 2.0 / g.hy;  // reference -> physical derivative

  double d0 = 0.0, d1 = 0.0, d2 = 0.0;  // max over fields
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const double sg = __ldg(sigma + mesh * F + f);
    const double* cs = us + f * 9 * P;
    double u[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) u[m] = __ldg(cs + m * P);
    double Sx0 = 0.0, Sx1 = 0.0, Sx2 = 0.0, Sy0 = 0.0, Sy1 = 0.0, Sy2 = 0.0;
    // Faces normal to direction n (0: x, 1: y), at reference coordinate s of K.
    // Along the face, K's trace and its normal derivatives of order 0, 1, 2 are
    // Legendre series c0, c1, c2 in the tangential coordinate t; the overlapping
    // cell's are o0, o1, o2 in its own tangential coordinate t' = t + dl,
    // dl = 1 - 2 h (h = the half), re-expanded in t with
    //   P_1(t + dl) = P_1(t) + dl,  P_2(t + dl) = P_2(t) + 3 dl P_1(t) + 3/2.
    // The difference series (u_K - w) is then scaled to physical derivatives
    // and evaluated at the half-face's Gauss points.
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      const double dn1 = n == 0 ? dx1 : dy1, dt1 = n == 0 ? dy1 : dx1;  // normal / tangential scales
      const double dn2 = dn1 * dn1, dt2 = dt1 * dt1;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const double s = 2.0 * side - 1.0;
        double c0[3], c1[3], c2[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          // coefficient (normal degree a, tangential degree t)
          const double u0 = n == 0 ? u[t * 3] : u[t], u1 = n == 0 ? u[t * 3 + 1] : u[3 + t];
          const double u2 = n == 0 ? u[t * 3 + 2] : u[6 + t];
          c0[t] = u0 + s * u1 + u2;
          c1[t] = fma(3.0 * s, u2, u1);
          c2[t] = 3.0 * u2;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const double dl = 1.0 - 2.0 * h;
          const int oi = n == 0 ? (side ? oi1 : oi0) : (h ? oi1 : oi0);
          const int oj = n == 0 ? (h ? oj1 : oj0) : (side ? oj1 : oj0);
          const double* co = uo + f * 9 * P + (long long)oj * g.nx + oi;
          double w0[3], w1[3], w2[3];
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            w0[t] = __ldg(co + (n == 0 ? t * 3 : t) * P);
            w1[t] = __ldg(co + (n == 0 ? t * 3 + 1 : 3 + t) * P);
            w2[t] = __ldg(co + (n == 0 ? t * 3 + 2 : 6 + t) * P);
          }
          // overlapping trace at its centre line (normal coordinate 0)
          const double o0[3] = {fma(-0.5, w2[0], w0[0]), fma(-0.5, w2[1], w0[1]), fma(-0.5, w2[2], w0[2])};
          const double* o1 = w1;
          const double o2[3] = {3.0 * w2[0], 3.0 * w2[1], 3.0 * w2[2]};
          // difference series in K's tangential coordinate
          double e0[3], e1[3], e2[3];
          e0[2] = c0[2] - o0[2];
          e0[1] = c0[1] - fma(3.0 * dl, o0[2], o0[1]);
          e0[0] = c0[0] - fma(1.5, o0[2], fma(dl, o0[1], o0[0]));
          e1[2] = c1[2] - o1[2];
          e1[1] = c1[1] - fma(3.0 * dl, o1[2], o1[1]);
          e1[0] = c1[0] - fma(1.5, o1[2], fma(dl, o1[1], o1[0]));
          e2[2] = c2[2] - o2[2];
          e2[1] = c2[1] - fma(3.0 * dl, o2[2], o2[1]);
          e2[0] = c2[0] - fma(1.5, o2[2], fma(dl, o2[1], o2[0]));
          // physical scalings: normal derivative series (order 1, 2), tangential
          // derivative of the value and of the normal derivative, second
          // tangential derivative (a constant on the half-face)
          const double a0 = dn1 * e1[0], a1 = dn1 * e1[1], a2 = dn1 * e1[2];
          const double b0 = dn2 * e2[0], b1 = dn2 * e2[1], b2 = dn2 * e2[2];
          const double t0 = dt1 * e0[1], t1 = 3.0 * dt1 * e0[2];
          const double m0 = dt1 * a1, m1 = 3.0 * dt1 * a2;
          const double tt = 3.0 * dt2 * e0[2];
          const double tt2 = tt * tt;
          double S0 = 0.0, S1 = 0.0, S2 = 0.0;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const double ts = xs_self(h, q);
            const double p2 = lp(2, ts);
            const double v = fma(p2, e0[2], fma(ts, e0[1], e0[0]));   // u_K - w
            const double gn = fma(p2, a2, fma(ts, a1, a0));           // normal derivative
            const double gt = fma(ts, t1, t0);                        // tangential derivative
            const double hn = fma(p2, b2, fma(ts, b1, b0));           // second normal
            const double hm = fma(ts, m1, m0);                        // mixed
            S0 = fma(gwt(q), fabs(v), S0);
            S1 = fma(gwt(q), sqrt(fma(gn, gn, gt * gt)), S1);
            S2 = fma(gwt(q), sqrt(fma(hn, hn, fma(hm, hm, tt2))), S2);
          }
          if (n == 0) {
            Sx0 += S0;
            Sx1 += S1;
            Sx2 += S2;
          } else {
            Sy0 += S0;
            Sy1 += S1;
            Sy2 += S2;
          }
        }
      }
    }
    if (sg != 0.0) {
      const double is = 1.0 / sg;
      d0 = fmax(d0, (bx * cx0 * Sx0 + by * cy0 * Sy0) * is);
      d1 = fmax(d1, (bx * cx1 * Sx1 + by * cy1 * Sy1) * is);
      d2 = fmax(d2, (bx * cx2 * Sx2 + by * cy2 * Sy2) * is);
    }
  }
  if (WRITE_DELTA) {
    double* dp = delta_out + (((long long)mesh * g.ny + j) * g.nx + i) * 3;
    dp[0] = d0;
    dp[1] = d1;
    dp[2] = d2;
  }
  if (usig != nullptr) {
    const double tau = dt[0];
    const double r1 = d0 + d1, r2 = r1 + d2;
    const double e1 = exp(-tau * r1), e2 = exp(-tau * r2);
    double* os = usig + (long long)mesh * F * 9 * P + (long long)j * g.nx + i;
#pragma unroll
    for (int f = 0; f < F; ++f) {
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        const int deg = (m % 3) + (m / 3);
        const double v = __ldg(us + (f * 9 + m) * P);
        os[(f * 9 + m) * P] = deg == 0 ? v : (deg == 1 ? v * e1 : v * e2);
      }
    }
  }
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
      const double rho = us[0], m1 = us[9 * g.plane], m2 = us[18 * g.plane], E = us[27 * g.plane];
      const double vx = m1 / rho, vy = m2 / rho;
      const double p = (g.gamma - 1.0) * (E - 0.5 * (m1 * vx + m2 * vy));
      if (rho > 0.0 && p > 0.0) {
        const double cs = sqrt(g.gamma * p / rho);
        mx = fmax(mx, fabs(vx) + cs);
        my = fmax(my, fabs(vy) + cs);
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

// One thread: tau_max = C_CFL / (beta_x/h_x + beta_y/h_y) (1D: C_CFL h / beta),
// tau = tau_max clipped at T_end (a step that would leave a sliver shorter
// than 1e-12 T_end is stretched to T_end); time[0] is advanced by tau.
__global__ void k_dt_final(const double* __restrict__ partial, int nblk, double hx, double hy, int dim, double cfl,
                           double T_end, double* __restrict__ dt, double* __restrict__ time) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double bx = 0.0, by = 0.0;
  for (int b = 0; b < nblk; ++b) {
    bx = fmax(bx, partial[2 * b]);
    by = fmax(by, partial[2 * b + 1]);
  }
  const double rate = bx / hx + (dim == 2 ? by / hy : 0.0);
  const double tm = rate > 0.0 ? cfl / rate : 0.0;
  const double t = time[0];
  double tau = tm;
  if (T_end > 0.0) {
    if (t >= T_end) tau = 0.0;
    else if (T_end - (t + tm) < 1e-12 * T_end) tau = T_end - t;
  }
  dt[0] = tau;
  dt[1] = tm > 0.0 ? tm : 1.0;
  time[0] = (T_end > 0.0 && tau == T_end - t) ? T_end : t + tau;
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

static inline dim3 tile_grid(const Geo& g) { return dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, 2); }

long long partial_blocks_2d(const Geo& g) {
  const dim3 gr = tile_grid(g);
  return (long long)gr.x * gr.y;
}

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

cudaError_t launch_sigma(const double* partials, long long nblk, int F, long long ncell, double* sigma, double* avg,
                         cudaStream_t st) {
  k_sigma<<<dim3(F, 2), 1024, 0, st>>>(partials, nblk, F, ncell, sigma, avg);
  return cudaGetLastError();
}

template <int SYS, int BC>
static cudaError_t oe2d_t(const Geo& g, const double* uh, double* usig, const double* dt, const double* sigma,
                          double* delta, int* status, cudaStream_t st) {
  if (delta)
    k_oe2d<SYS, BC, true><<<tile_grid(g), NT, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
  else
    k_oe2d<SYS, BC, false><<<tile_grid(g), NT, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
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
  k_dt_final<<<1, 32, 0, st>>>(partial, nblk, g.hx, g.hy, 2, g.cfl, T_end, dt, time);
  return cudaGetLastError();
}

cudaError_t launch_dt_final(const double* partial, int nblk, double hx, double hy, int dim, double cfl, double T_end,
                            double* dt, double* time, cudaStream_t st) {
  k_dt_final<<<1, 32, 0, st>>>(partial, nblk, hx, hy, dim, cfl, T_end, dt, time);
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
