// oecdg_2dk.cu -- degree-generic 2D kernels of the OECDG forward step
// (arXiv:2503.12473): the tensor space Q^k and the total-degree space P^k for
// k = 1, 2, 3 (Section 2.1), linear advection, Burgers (f1 = f2 = u^2/2) and
// the 2D Euler equations.  The CDG operator is Eq. (eq:2D_H); the damping
// coefficients delta_K^m, m = 0..k, and the exact OE step are those of
// Section 2.2 (Eq. (OEstep2D)).  One thread per cell, 32 x 4 cells per block,
// blockIdx.z = mesh.  The tiled Q^2 kernels of oecdg_2d.cu remain the fast
// path for the Q^2 configurations; this file serves every other one.
//
// Geometry as in the Q^2 kernels: primal cell (i, j) overlaps dual cells
// (i - 1 + sx, j - 1 + sy), dual cell (i, j) overlaps primal cells (i + sx,
// j + sy); sub-cell (sx, sy) of K lies in that overlapping cell, whose centre
// sits on K's faces, so a point xi of half s of K is xi' = xi + 1 - 2 s there.
// The overlapping cell of sub-cell (sx, sy) also holds the x-face half sy on
// side sx and the y-face half sx on side sy.
#include <type_traits>

#include "oecdg_common.cuh"
#include "oecdg_kernels.h"
#include "oecdg_poly.cuh"

namespace oecdg {

constexpr int NTK = 128;  // 32 x 4 cells
constexpr double DINFK = __builtin_huge_val();

// Mode lists.  Q^k: index b (k+1) + a.  P^k: by total degree s = a + b, then
// by decreasing a (index of (a, b) = s (s+1) / 2 + b).
__host__ __device__ constexpr int pk_a(int m, int s) { return m < s + 1 ? s - m : pk_a(m - s - 1, s + 1); }
__host__ __device__ constexpr int pk_b(int m, int s) { return m < s + 1 ? m : pk_b(m - s - 1, s + 1); }

template <int K, int B>
struct Modes2 {
  static constexpr int M = B == BASIS_Q ? (K + 1) * (K + 1) : (K + 1) * (K + 2) / 2;
  __host__ __device__ static constexpr int a(int m) { return B == BASIS_Q ? m % (K + 1) : pk_a(m, 0); }
  __host__ __device__ static constexpr int b(int m) { return B == BASIS_Q ? m / (K + 1) : pk_b(m, 0); }
  // phi_m and its reference derivatives (dx, dy) at (x, y)
  __host__ __device__ static constexpr double phi(int m, int dx, int dy, double x, double y) {
    return lpd(a(m), dx, x) * lpd(b(m), dy, y);
  }
};

template <int SYS>
struct Fields2 {
  static constexpr int F = SYS == SYS_EULER ? 4 : 1;
};

template <int SYS>
__device__ __forceinline__ void flux2(const Geo& g, const double* w, double* f1, double* f2) {
  if (SYS == SYS_EULER) {
    Euler2::both(w, g.gamma, f1, f2);
  } else if (SYS == SYS_BURGERS) {
    f1[0] = f2[0] = 0.5 * w[0] * w[0];
  } else {
    f1[0] = g.adv_x * w[0];
    f2[0] = g.adv_y * w[0];
  }
}

// Normal wave speeds (beta_x, beta_y) at a state: Euler |v_n| + c, advection
// |a_n|, Burgers |u|.  Returns false for a non-physical Euler state.
template <int SYS>
__device__ __forceinline__ bool speeds2(const Geo& g, const double* w, double& bx, double& by) {
  if (SYS == SYS_EULER) {
    const double r = 1.0 / w[0];
    const double vx = w[1] * r, vy = w[2] * r;
    const double p = (g.gamma - 1.0) * fma(-0.5, fma(w[1], vx, w[2] * vy), w[3]);
    if (!(w[0] > 0.0 && p > 0.0)) {
      bx = by = 0.0;
      return false;
    }
    const double c = sqrt(g.gamma * p * r);
    bx = fabs(vx) + c;
    by = fabs(vy) + c;
  } else if (SYS == SYS_BURGERS) {
    bx = by = fabs(w[0]);
  } else {
    bx = fabs(g.adv_x);
    by = fabs(g.adv_y);
  }
  return true;
}

// Gauss nodes and weights of the N-point rules (N = 2, 3, 4) for runtime
// point loops: [N - 2][q].
__constant__ double GNK[3][4] = {{gn1(2, 0), gn1(2, 1), 0.0, 0.0},
                                 {gn1(3, 0), gn1(3, 1), gn1(3, 2), 0.0},
                                 {gn1(4, 0), gn1(4, 1), gn1(4, 2), gn1(4, 3)}};
__constant__ double GWK[3][4] = {{gw1(2, 0), gw1(2, 1), 0.0, 0.0},
                                 {gw1(3, 0), gw1(3, 1), gw1(3, 2), 0.0},
                                 {gw1(4, 0), gw1(4, 1), gw1(4, 2), gw1(4, 3)}};

// P_a^(d)(x), a = 0..K, at a runtime point
template <int K, int D>
__device__ __forceinline__ void leg_row(double x, double (&p)[K + 1]) {
#pragma unroll
  for (int a = 0; a <= K; ++a) p[a] = lpd(a, D, x);
}

// Every field of the expansion c (stride P per mode, F * M coefficients) at
// reference point (x, y).
template <int F, int K, int B>
__device__ __forceinline__ void eval_fields(const double* __restrict__ c, long long P, double x, double y,
                                            double (&V)[F]) {
  using MD = Modes2<K, B>;
  double px[K + 1], py[K + 1];
  leg_row<K, 0>(x, px);
  leg_row<K, 0>(y, py);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < MD::M; ++m) v = fma(px[MD::a(m)] * py[MD::b(m)], __ldg(c + (f * MD::M + m) * P), v);
    V[f] = v;
  }
}

// L_m = (2a+1)(2b+1)/4 R_m - u_m / tau_max with, in reference coordinates of
// K (weights of the half rules: w_q / 2),
//   R_m = sum_{sub-cells, points} W (w phi_m / tau_max + f1 (2/hx) phi_m,xi + f2 (2/hy) phi_m,eta)
//         - (2/hx) sum_{x-faces} (w_q/2) s f1 phi_m - (2/hy) sum_{y-faces} (w_q/2) s f2 phi_m,
// s = -1 / +1 the face side.  (The u_K part of the dissipation term is exact:
// int_K u_K phi_m = u_m ||phi_m||^2.)
// Sum factorisation by rows of points: for each row qy of a sub-cell the
// overlapping cell is contracted in y once (T), each point then costs K+1
// terms per field, and the x sums of the row (X: value and d/dx terms, Y: d/dy
// term) are projected in y once.  Face rows likewise: the overlapping cell at
// its centre line (Z), the face sums per tangential degree (G), one projection.
template <int SYS, int BC, int K, int B>
__device__ __forceinline__ void cell_rhs2k(const Geo& g, const double* __restrict__ u, int mesh, int i, int j,
                                           double inv_tm, double (&L)[Fields2<SYS>::F][Modes2<K, B>::M]) {
  using MD = Modes2<K, B>;
  constexpr int F = Fields2<SYS>::F, M = MD::M, N = K + 1;
  const long long P = g.plane;
  const double* uo = u + (long long)(1 - mesh) * F * M * P;
  const int off = mesh == 0 ? -1 : 0;
  const double sx2 = 2.0 / g.hx, sy2 = 2.0 / g.hy;
  const int iu = BC == BC_GENERAL ? unwrapped(g, 0, mesh, i) : i, ju = BC == BC_GENERAL ? unwrapped(g, 1, mesh, j) : j;
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int m = 0; m < M; ++m) L[f][m] = 0.0;
#pragma unroll 1
  for (int sub = 0; sub < 4; ++sub) {
    const int sx = sub & 1, sy = sub >> 1;
    bool mx = false, my = false;  // the overlapping cell is a mirror image across a wall
    const int oi = BC == BC_GENERAL ? side_index(g, 0, 1 - mesh, iu + sx + off, mx) : wrap_index<BC>(i + sx + off, g.nx);
    const int oj = BC == BC_GENERAL ? side_index(g, 1, 1 - mesh, ju + sy + off, my) : wrap_index<BC>(j + sy + off, g.ny);
    const double* c = uo + (long long)oj * g.nxs + oi;
    // ---- volume and dissipation terms on sub-cell (sx, sy), row by row
#pragma unroll 1
    for (int qy = 0; qy < N; ++qy) {
      const double gy = GNK[N - 2][qy], wy = GWK[N - 2][qy];
      double T[F][K + 1];  // overlapping cell contracted in y at this row
      {
        double pyo[K + 1];
        leg_row<K, 0>(0.5 - sy + 0.5 * gy, pyo);
#pragma unroll
        for (int f = 0; f < F; ++f) {
#pragma unroll
          for (int a = 0; a <= K; ++a) T[f][a] = 0.0;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            double cv = __ldg(c + (f * M + m) * P);
            if (BC == BC_GENERAL) cv = apply_sign(cv, mirror_sign(mx, my, SYS == SYS_EULER, f, MD::a(m), MD::b(m)));
            T[f][MD::a(m)] = fma(pyo[MD::b(m)], cv, T[f][MD::a(m)]);
          }
        }
      }
      double X[F][K + 1], Y[F][K + 1];
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int a = 0; a <= K; ++a) X[f][a] = Y[f][a] = 0.0;
#pragma unroll 1
      for (int qx = 0; qx < N; ++qx) {
        const double gx = GNK[N - 2][qx];
        const double W = 0.25 * GWK[N - 2][qx] * wy;
        double pxo[K + 1], px[K + 1], dpx[K + 1];
        leg_row<K, 0>(0.5 - sx + 0.5 * gx, pxo);
        leg_row<K, 0>(sx - 0.5 + 0.5 * gx, px);
        leg_row<K, 1>(sx - 0.5 + 0.5 * gx, dpx);
        double V[F], f1[F], f2[F];
#pragma unroll
        for (int f = 0; f < F; ++f) {
          double v = 0.0;
#pragma unroll
          for (int a = 0; a <= K; ++a) v = fma(pxo[a], T[f][a], v);
          V[f] = v;
        }
        flux2<SYS>(g, V, f1, f2);
#pragma unroll
        for (int f = 0; f < F; ++f) {
          const double av = W * inv_tm * V[f], a1 = W * sx2 * f1[f], a2 = W * sy2 * f2[f];
#pragma unroll
          for (int a = 0; a <= K; ++a) {
            X[f][a] = fma(px[a], av, a > 0 ? fma(dpx[a], a1, X[f][a]) : X[f][a]);
            Y[f][a] = fma(px[a], a2, Y[f][a]);
          }
        }
      }
      double py[K + 1], dpy[K + 1];
      leg_row<K, 0>(sy - 0.5 + 0.5 * gy, py);
      leg_row<K, 1>(sy - 0.5 + 0.5 * gy, dpy);
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int m = 0; m < M; ++m) {
          double r = fma(py[MD::b(m)], X[f][MD::a(m)], L[f][m]);
          if (MD::b(m) > 0) r = fma(dpy[MD::b(m)], Y[f][MD::a(m)], r);
          L[f][m] = r;
        }
    }
    // ---- x-face on side sx, half sy (K's xi = 2 sx - 1, overlapping xi' = 0)
    //      y-face on side sy, half sx (K's eta = 2 sy - 1, overlapping eta' = 0)
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const int h = dir == 0 ? sy : sx;
      const double sgn = dir == 0 ? 2.0 * sx - 1.0 : 2.0 * sy - 1.0;
      double Z[F][K + 1];  // overlapping cell on its centre line, by tangential degree
      {
        double p0[K + 1];
        leg_row<K, 0>(0.0, p0);
#pragma unroll
        for (int f = 0; f < F; ++f) {
#pragma unroll
          for (int a = 0; a <= K; ++a) Z[f][a] = 0.0;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const int an = dir == 0 ? MD::a(m) : MD::b(m), at = dir == 0 ? MD::b(m) : MD::a(m);
            double cv = __ldg(c + (f * M + m) * P);
            if (BC == BC_GENERAL) cv = apply_sign(cv, mirror_sign(mx, my, SYS == SYS_EULER, f, MD::a(m), MD::b(m)));
            Z[f][at] = fma(p0[an], cv, Z[f][at]);
          }
        }
      }
      double Gs[F][K + 1];  // sum over the points of the face weight x P_at(t)
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int a = 0; a <= K; ++a) Gs[f][a] = 0.0;
      const double sc = -0.5 * sgn * (dir == 0 ? sx2 : sy2);
#pragma unroll 1
      for (int q = 0; q < N; ++q) {
        const double gq = GNK[N - 2][q], wq = GWK[N - 2][q];
        double pto[K + 1], pt[K + 1];
        leg_row<K, 0>(0.5 - h + 0.5 * gq, pto);
        leg_row<K, 0>(h - 0.5 + 0.5 * gq, pt);
        double V[F], f1[F], f2[F];
#pragma unroll
        for (int f = 0; f < F; ++f) {
          double v = 0.0;
#pragma unroll
          for (int a = 0; a <= K; ++a) v = fma(pto[a], Z[f][a], v);
          V[f] = v;
        }
        flux2<SYS>(g, V, f1, f2);
#pragma unroll
        for (int f = 0; f < F; ++f) {
          const double cf = sc * wq * (dir == 0 ? f1[f] : f2[f]);
#pragma unroll
          for (int a = 0; a <= K; ++a) Gs[f][a] = fma(pt[a], cf, Gs[f][a]);
        }
      }
      double pn[K + 1];
      leg_row<K, 0>(sgn, pn);
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int an = dir == 0 ? MD::a(m) : MD::b(m), at = dir == 0 ? MD::b(m) : MD::a(m);
          L[f][m] = fma(pn[an], Gs[f][at], L[f][m]);
        }
    }
  }
  const double* us = u + (long long)mesh * F * M * P + (long long)j * g.nxs + i;
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const double nrm = 0.25 * (2 * MD::a(m) + 1) * (2 * MD::b(m) + 1);
      L[f][m] = fma(nrm, L[f][m], -inv_tm * __ldg(us + (f * M + m) * P));
    }
}

enum { MODEK_RHS = 0, MODEK_STAGE = 1 };

__device__ __forceinline__ void cell_of_thread(const Geo& g, int& i, int& j) {
  i = blockIdx.x * 32 + (threadIdx.x & 31);
  j = blockIdx.y * (NTK / 32) + (threadIdx.x >> 5);
}

// MODEK_RHS:   out = L(uin).
// MODEK_STAGE: out = sum_m cb.c[m] cb.u[m] + cb.ct tau L(uin), plus per-block
//              sigma partials of out (sum of cell averages; max / min over the
//              (k+1)^2 Gauss points of each cell), [mesh][block][F][3].
template <int SYS, int BC, int K, int B, int MODE>
__global__ void __launch_bounds__(NTK) k_stage2k(Geo g, const double* __restrict__ uin, StageComb cb,
                                                 double* __restrict__ out, const double* __restrict__ dt,
                                                 double* __restrict__ partials) {
  using MD = Modes2<K, B>;
  constexpr int F = Fields2<SYS>::F, M = MD::M, N = K + 1;
  const int mesh = blockIdx.z;
  int i, j;
  cell_of_thread(g, i, j);
  const bool active = i < cells_x(g, mesh) && j < cells_y(g, mesh);
  const int ic = active ? i : 0, jc = active ? j : 0;
  const double tau = dt[0], tm = dt[1];
  double L[F][M];
  cell_rhs2k<SYS, BC, K, B>(g, uin, mesh, ic, jc, 1.0 / tm, L);
  const long long P = g.plane;
  const long long base = (long long)mesh * F * M * P + (long long)jc * g.nxs + ic;
  if (MODE == MODEK_RHS) {
    if (active)
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int m = 0; m < M; ++m) out[base + (f * M + m) * P] = L[f][m];
    return;
  } else {
    __shared__ double sh[96];
    const double tl = cb.ct * tau;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      double v[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const long long id = base + (f * M + m) * P;
        double s = tl * L[f][m];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (r < cb.n) s = fma(cb.c[r], __ldg(cb.u[r] + id), s);
        v[m] = s;
        if (active) out[id] = s;
      }
      double mx = -DINFK, mn = DINFK;
#pragma unroll 1
      for (int q = 0; q < N * N; ++q) {
        double px[K + 1], py[K + 1];
        leg_row<K, 0>(GNK[N - 2][q % N], px);
        leg_row<K, 0>(GNK[N - 2][q / N], py);
        double val = 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m) val = fma(px[MD::a(m)] * py[MD::b(m)], v[m], val);
        mx = fmax(mx, val);
        mn = fmin(mn, val);
      }
      double s = active ? v[0] : 0.0;
      if (BC == BC_GENERAL) s *= cell_weight(g, mesh, ic, jc, 2);  // wall-centred dual cells count half
      if (!active) {
        mx = -DINFK;
        mn = DINFK;
      }
      block_reduce3(s, mx, mn, sh);
      if (threadIdx.x == 0) {
        const long long nblk = (long long)gridDim.x * gridDim.y;
        double* p = partials + ((mesh * nblk + (long long)blockIdx.y * gridDim.x + blockIdx.x) * F + f) * 3;
        p[0] = s;
        p[1] = mx;
        p[2] = mn;
      }
    }
  }
}

// delta_K^m, m = 0..K (Section 2.2): for every face e of K (x-faces: h_e = hx,
// beta_x; y-faces: h_e = hy, beta_y), over its 2 halves with K+1 Gauss points
// each, the integral of (sum_{|alpha| = m} (d^alpha (u_K - w))^2)^(1/2) with
// K's interior trace and the overlapping cell's solution w, weighted by
// beta_e (2m+1) h_e^(m-1) / ((2K-1) m! sigma |e|); max over fields.  Then the
// exact OE step: mode (a, b) decays by exp(-tau sum_{m <= min(a+b, K)} delta^m).
// On a face normal to direction n the multi-index is (normal order an,
// tangential order m - an); K's trace sits at normal coordinate s = +-1, the
// overlapping cell's at its centre line (normal coordinate 0).
template <int SYS, int BC, int K, int B, bool WRITE_DELTA>
__global__ void __launch_bounds__(NTK) k_oe2k(Geo g, const double* __restrict__ uh, double* __restrict__ usig,
                                              const double* __restrict__ dt, const double* __restrict__ sigma,
                                              double* __restrict__ delta_out, int* __restrict__ status) {
  using MD = Modes2<K, B>;
  constexpr int F = Fields2<SYS>::F, M = MD::M, N = K + 1;
  const int mesh = blockIdx.z;
  __shared__ double isg[F];  // 1/sigma of this mesh's fields, once per block
  oe_inv_sigma<F>(sigma, mesh, isg);
  int i, j;
  cell_of_thread(g, i, j);
  if (i >= cells_x(g, mesh) || j >= cells_y(g, mesh)) return;
  const long long P = g.plane;
  const double* us = uh + (long long)mesh * F * M * P + (long long)j * g.nxs + i;
  const double* uo = uh + (long long)(1 - mesh) * F * M * P;
  const int off = mesh == 0 ? -1 : 0;
  const int iu = BC == BC_GENERAL ? unwrapped(g, 0, mesh, i) : i, ju = BC == BC_GENERAL ? unwrapped(g, 1, mesh, j) : j;
  double wa[F];
#pragma unroll
  for (int f = 0; f < F; ++f) wa[f] = __ldg(us + (f * M) * P);
  double bx, by;
  if (!speeds2<SYS>(g, wa, bx, by)) atomicOr(status, ST_NONPHYSICAL);
  double dl[K + 1];
#pragma unroll
  for (int m = 0; m <= K; ++m) dl[m] = 0.0;
#pragma unroll 1
  for (int f = 0; f < F; ++f) {
    const double sg = __ldg(sigma + mesh * F + f);
    double cu[M];
#pragma unroll
    for (int m = 0; m < M; ++m) cu[m] = __ldg(us + (long long)(f * M + m) * P);
    double S[2][K + 1];
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int m = 0; m <= K; ++m) S[n][m] = 0.0;
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      const double sn = n == 0 ? g.i2x : g.i2y, st = n == 0 ? g.i2y : g.i2x;  // 2/h normal, tangential
#pragma unroll 1
      for (int side = 0; side < 2; ++side) {
        const double s = 2.0 * side - 1.0;
        // K's trace series on the face: Tu[an][at] = coefficient of P_at(t) in
        // the an-th normal derivative (reference) at normal coordinate s
        double Tu[K + 1][K + 1];
        {
          double pn[K + 1][K + 1];  // pn[d][a] = P_a^(d)(s)
#pragma unroll
          for (int d = 0; d <= K; ++d)
#pragma unroll
            for (int a = 0; a <= K; ++a) pn[d][a] = lpd(a, d, s);
#pragma unroll
          for (int d = 0; d <= K; ++d)
#pragma unroll
            for (int a = 0; a <= K; ++a) Tu[d][a] = 0.0;
#pragma unroll
          for (int mm = 0; mm < M; ++mm) {
            const int a_n = n == 0 ? MD::a(mm) : MD::b(mm), a_t = n == 0 ? MD::b(mm) : MD::a(mm);
#pragma unroll
            for (int d = 0; d <= a_n; ++d) Tu[d][a_t] = fma(pn[d][a_n], cu[mm], Tu[d][a_t]);
          }
        }
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          bool mx = false, my = false;  // a mirror image across a wall
          const int oi = BC == BC_GENERAL ? side_index(g, 0, 1 - mesh, iu + (n == 0 ? side : h) + off, mx)
                                          : wrap_index<BC>(i + (n == 0 ? side : h) + off, g.nx);
          const int oj = BC == BC_GENERAL ? side_index(g, 1, 1 - mesh, ju + (n == 0 ? h : side) + off, my)
                                          : wrap_index<BC>(j + (n == 0 ? h : side) + off, g.ny);
          const double* co = uo + (long long)(f * M) * P + (long long)oj * g.nxs + oi;
          // the overlapping cell's series on its centre line (normal coordinate 0)
          double Tw[K + 1][K + 1];
#pragma unroll
          for (int d = 0; d <= K; ++d)
#pragma unroll
            for (int a = 0; a <= K; ++a) Tw[d][a] = 0.0;
#pragma unroll
          for (int mm = 0; mm < M; ++mm) {
            const int a_n = n == 0 ? MD::a(mm) : MD::b(mm), a_t = n == 0 ? MD::b(mm) : MD::a(mm);
            double cw = __ldg(co + (long long)mm * P);
            if (BC == BC_GENERAL) cw = apply_sign(cw, mirror_sign(mx, my, SYS == SYS_EULER, f, MD::a(mm), MD::b(mm)));
#pragma unroll
            for (int d = 0; d <= a_n; ++d)
              if (lpd(a_n, d, 0.0) != 0.0) Tw[d][a_t] = fma(lpd(a_n, d, 0.0), cw, Tw[d][a_t]);
          }
          // difference series in K's tangential coordinate t (t' = t + dl):
          // E[an] = Tu[an] - Tw[an] re-expanded about t
          const double dl = 1.0 - 2.0 * h;
          double E[K + 1][K + 1];
#pragma unroll
          for (int d = 0; d <= K; ++d)
#pragma unroll
            for (int a = 0; a <= K; ++a) {
              double e = Tu[d][a];
#pragma unroll
              for (int a2 = a; a2 <= K; ++a2)
                if (!(B == BASIS_P && a2 + d > K)) e = fma(-lshift(a2, a, dl), Tw[d][a2], e);
              E[d][a] = e;
            }
#pragma unroll 1
          for (int q = 0; q < N; ++q) {
            const double gq = GNK[N - 2][q], wq = GWK[N - 2][q];
            const double t = h - 0.5 + 0.5 * gq;
#pragma unroll
            for (int m = 0; m <= K; ++m) {
              double ss = SQ_FLOOR;
#pragma unroll
              for (int an = 0; an <= m; ++an) {
                const int at = m - an;
                double v = 0.0;
#pragma unroll
                for (int a = at; a <= K; ++a) {
                  if (B == BASIS_P && a + an > K) continue;  // no such mode in P^K
                  v = fma(E[an][a], lpd(a, at, t), v);
                }
                double sc = 1.0;
#pragma unroll
                for (int r = 0; r < an; ++r) sc *= sn;
#pragma unroll
                for (int r = 0; r < at; ++r) sc *= st;
                const double dv = v * sc;
                ss = fma(dv, dv, ss);
              }
              S[n][m] = fma(wq, sqrt_pos(ss), S[n][m]);
            }
          }
        }
      }
    }
    if (sg != 0.0) {
      const double is = isg[f];
      double hx = g.i1x, hy = g.i1y;  // h^(m-1)
#pragma unroll
      for (int m = 0; m <= K; ++m) {
        const double c = 0.25 * (2 * m + 1) / ((2 * K - 1) * fact(m));
        dl[m] = fmax(dl[m], fma(bx * c * hx, S[0][m], (by * c * hy) * S[1][m]) * is);
        hx *= g.hx;
        hy *= g.hy;
      }
    }
  }
  if (WRITE_DELTA) {
    double* dp = delta_out + (((long long)mesh * g.nys + j) * g.nxs + i) * (K + 1);
#pragma unroll
    for (int m = 0; m <= K; ++m) dp[m] = dl[m];
  }
  if (usig != nullptr) {
    const double tau = dt[0];
    double e[2 * K + 1];  // decay factor by total degree (degrees above K: as K)
    double rate = dl[0];
    e[0] = 1.0;
#pragma unroll
    for (int d = 1; d <= 2 * K; ++d) {
      if (d <= K) {
        rate += dl[d];
        e[d] = exp(-tau * rate);
      } else {
        e[d] = e[K];
      }
    }
    double* os = usig + (long long)mesh * F * M * P + (long long)j * g.nxs + i;
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const double v = __ldg(us + (f * M + m) * P);
        os[(f * M + m) * P] = v * e[MD::a(m) + MD::b(m)];
      }
  }
}

// Maximum normal wave speeds over the cell averages of both meshes: per block
// (max beta_x, max beta_y).
template <int SYS, int M>
__global__ void k_wave2k(Geo g, const double* __restrict__ u, double* __restrict__ partial, int* __restrict__ status) {
  constexpr int F = Fields2<SYS>::F;
  __shared__ double sh[32];
  const long long n = 2 * g.plane;
  double mx = 0.0, my = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    const int cj = (int)(cell / g.nxs), ci = (int)(cell - (long long)cj * g.nxs);
    if (ci >= cells_x(g, mesh) || cj >= cells_y(g, mesh)) continue;  // the primal mesh's unused slots
    const double* us = u + (long long)mesh * F * M * g.plane + cell;
    double w[F];
#pragma unroll
    for (int f = 0; f < F; ++f) w[f] = us[(long long)(f * M) * g.plane];
    double bx, by;
    if (speeds2<SYS>(g, w, bx, by)) {
      mx = fmax(mx, bx);
      my = fmax(my, by);
    } else {
      atomicOr(status, ST_NONPHYSICAL);
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

// Sampling points of the initial projection: (k+1)^2 Gauss points on each of
// the 4 sub-cells of every stored cell of both meshes (the padded layout: an
// unused primal slot takes the dual cell's points), layout
// [mesh][j][i][sy][sx][qy][qx] of (x, y); points beyond a reflective wall
// (the outer half of a wall-centred dual cell) folded back to their mirror
// images inside [ax, bx] x [ay, by].
template <int K>
__global__ void k_points2k(Geo g, double ax, double ay, double bx, double by, double* __restrict__ xy) {
  constexpr int N = K + 1, R = 4 * N * N;
  const long long n = 2 * g.plane * R;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % R);
    const long long c = t / R;
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    const int j = (int)(cell / g.nxs), i = (int)(cell - (long long)j * g.nxs);
    const int cm = (i < cells_x(g, mesh) && j < cells_y(g, mesh)) ? mesh : 1;
    const int qx = r % N, qy = (r / N) % N, sx = (r / (N * N)) % 2, sy = r / (2 * N * N);
    const double xc = ax + (unwrapped(g, 0, cm, i) + 0.5 + 0.5 * cm) * g.hx;
    const double yc = ay + (unwrapped(g, 1, cm, j) + 0.5 + 0.5 * cm) * g.hy;
    double x = xc + 0.5 * g.hx * xs1(N, sx, qx), y = yc + 0.5 * g.hy * xs1(N, sy, qy);
    if (g.bcs[0] == SIDE_REFLECTIVE && x < ax) x = 2.0 * ax - x;
    if (g.bcs[1] == SIDE_REFLECTIVE && x > bx) x = 2.0 * bx - x;
    if (g.bcs[2] == SIDE_REFLECTIVE && y < ay) y = 2.0 * ay - y;
    if (g.bcs[3] == SIDE_REFLECTIVE && y > by) y = 2.0 * by - y;
    xy[2 * t] = x;
    xy[2 * t + 1] = y;
  }
}

// L2 projection: u_m = (2a+1)(2b+1)/4 sum over the sub-cells and their points
// of (w_qx/2)(w_qy/2) u0 phi_m(xi, eta).
template <int F, int K, int B>
__global__ void k_project2k(Geo g, const double* __restrict__ vals, double* __restrict__ u) {
  using MD = Modes2<K, B>;
  constexpr int M = MD::M, N = K + 1, R = 4 * N * N;
  const long long n = 2 * g.plane;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    double acc[F][M];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int m = 0; m < M; ++m) acc[f][m] = 0.0;
    const double* v = vals + c * R * F;
    const int cj = (int)(cell / g.nxs), ci = (int)(cell - (long long)cj * g.nxs);
    // sub-cells beyond a wall were sampled at their mirror images: the normal
    // momentum (Euler: field 1 for x, 2 for y) changes sign there
    const bool wxl = mesh == 1 && g.bcs[0] == SIDE_REFLECTIVE && ci == g.nx;
    const bool wxh = mesh == 1 && g.bcs[1] == SIDE_REFLECTIVE && ci == g.nx - 1;
    const bool wyl = mesh == 1 && g.bcs[2] == SIDE_REFLECTIVE && cj == g.ny;
    const bool wyh = mesh == 1 && g.bcs[3] == SIDE_REFLECTIVE && cj == g.ny - 1;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      const int qx = r % N, qy = (r / N) % N, sx = (r / (N * N)) % 2, sy = r / (2 * N * N);
      double px[K + 1], py[K + 1];
      leg_row<K, 0>(sx - 0.5 + 0.5 * GNK[N - 2][qx], px);
      leg_row<K, 0>(sy - 0.5 + 0.5 * GNK[N - 2][qy], py);
      const double w = 0.25 * GWK[N - 2][qx] * GWK[N - 2][qy];
      const bool fx = (wxl && sx == 0) || (wxh && sx == 1), fy = (wyl && sy == 0) || (wyh && sy == 1);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const bool neg = F == 4 && ((fx && f == 1) || (fy && f == 2));
        const double x = neg ? -w * v[r * F + f] : w * v[r * F + f];
#pragma unroll
        for (int m = 0; m < M; ++m) acc[f][m] = fma(x, px[MD::a(m)] * py[MD::b(m)], acc[f][m]);
      }
    }
    const bool used = ci < cells_x(g, mesh) && cj < cells_y(g, mesh);  // unused primal slots: 0
    double* o = u + (long long)mesh * F * M * g.plane + cell;
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int m = 0; m < M; ++m)
        o[(long long)(f * M + m) * g.plane] =
            used ? acc[f][m] * ((2 * MD::a(m) + 1) * (2 * MD::b(m) + 1) / 4.0) : 0.0;
  }
}

// ----------------------------------------------------------------- launch --

template <int V>
using ICk = std::integral_constant<int, V>;

// fn(IC<SYS>, IC<BC>, IC<K>, IC<B>) for the runtime (sys, bc, k, basis)
template <class Fn>
static void by_sys_bc_k_b(int sys, int bc, int k, int basis, Fn&& fn) {
  auto kb = [&](auto S, auto Bc) {
    if (basis == BASIS_Q) {
      if (k == 1) fn(S, Bc, ICk<1>{}, ICk<BASIS_Q>{});
      else if (k == 2) fn(S, Bc, ICk<2>{}, ICk<BASIS_Q>{});
      else fn(S, Bc, ICk<3>{}, ICk<BASIS_Q>{});
    } else {
      if (k == 1) fn(S, Bc, ICk<1>{}, ICk<BASIS_P>{});
      else if (k == 2) fn(S, Bc, ICk<2>{}, ICk<BASIS_P>{});
      else fn(S, Bc, ICk<3>{}, ICk<BASIS_P>{});
    }
  };
  auto bb = [&](auto S) {
    if (bc == BC_PERIODIC) kb(S, ICk<BC_PERIODIC>{});
    else if (bc == BC_TRANSMISSIVE) kb(S, ICk<BC_TRANSMISSIVE>{});
    else kb(S, ICk<BC_GENERAL>{});
  };
  if (sys == SYS_EULER) bb(ICk<SYS_EULER>{});
  else if (sys == SYS_BURGERS) bb(ICk<SYS_BURGERS>{});
  else bb(ICk<SYS_ADV>{});
}

static dim3 grid2k(const Geo& g) { return dim3((g.nxs + 31) / 32, (g.nys + NTK / 32 - 1) / (NTK / 32), 2); }

long long partial_blocks_2k(const Geo& g) {
  const dim3 gr = grid2k(g);
  return (long long)gr.x * gr.y;
}

int modes_2k(int k, int basis) { return basis == BASIS_Q ? (k + 1) * (k + 1) : (k + 1) * (k + 2) / 2; }

cudaError_t launch_stage2k(int sys, int bc, int k, int basis, const Geo& g, int rhs_only, const double* uin,
                           const StageComb& cb, double* out, const double* dt, double* partials, cudaStream_t st) {
  by_sys_bc_k_b(sys, bc, k, basis, [&](auto S, auto Bc, auto Kc, auto Bs) {
    constexpr int S_ = decltype(S)::value, B_ = decltype(Bc)::value, K_ = decltype(Kc)::value;
    constexpr int Q_ = decltype(Bs)::value;
    if (rhs_only) k_stage2k<S_, B_, K_, Q_, MODEK_RHS><<<grid2k(g), NTK, 0, st>>>(g, uin, cb, out, dt, partials);
    else k_stage2k<S_, B_, K_, Q_, MODEK_STAGE><<<grid2k(g), NTK, 0, st>>>(g, uin, cb, out, dt, partials);
  });
  return cudaGetLastError();
}

cudaError_t launch_oe2k(int sys, int bc, int k, int basis, const Geo& g, const double* uh, double* usig,
                        const double* dt, const double* sigma, double* delta, int* status, cudaStream_t st) {
  by_sys_bc_k_b(sys, bc, k, basis, [&](auto S, auto Bc, auto Kc, auto Bs) {
    constexpr int S_ = decltype(S)::value, B_ = decltype(Bc)::value, K_ = decltype(Kc)::value;
    constexpr int Q_ = decltype(Bs)::value;
    if (delta) k_oe2k<S_, B_, K_, Q_, true><<<grid2k(g), NTK, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
    else k_oe2k<S_, B_, K_, Q_, false><<<grid2k(g), NTK, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
  });
  return cudaGetLastError();
}

cudaError_t launch_dt2k(int sys, int k, int basis, const Geo& g, const double* u, double* partial, int nblk,
                        double T_end, double* dt, double* time, int* status, cudaStream_t st) {
  by_sys_bc_k_b(sys, BC_PERIODIC, k, basis, [&](auto S, auto, auto Kc, auto Bs) {
    constexpr int M = Modes2<decltype(Kc)::value, decltype(Bs)::value>::M;
    k_wave2k<decltype(S)::value, M><<<nblk, 256, 0, st>>>(g, u, partial, status);
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_dt_final(partial, nblk, g.hx, g.hy, 2, g.cfl, T_end, dt, time, st);
}

cudaError_t launch_points2k(int k, const Geo& g, double ax, double ay, double bx, double by, double* xy,
                            cudaStream_t st) {
  if (k == 1) k_points2k<1><<<1184, 256, 0, st>>>(g, ax, ay, bx, by, xy);
  else if (k == 2) k_points2k<2><<<1184, 256, 0, st>>>(g, ax, ay, bx, by, xy);
  else k_points2k<3><<<1184, 256, 0, st>>>(g, ax, ay, bx, by, xy);
  return cudaGetLastError();
}

cudaError_t launch_project2k(int sys, int k, int basis, const Geo& g, const double* vals, double* u,
                             cudaStream_t st) {
  by_sys_bc_k_b(sys, BC_PERIODIC, k, basis, [&](auto S, auto, auto Kc, auto Bs) {
    constexpr int F = Fields2<decltype(S)::value>::F;
    k_project2k<F, decltype(Kc)::value, decltype(Bs)::value><<<1184, 128, 0, st>>>(g, vals, u);
  });
  return cudaGetLastError();
}

}  // namespace oecdg
