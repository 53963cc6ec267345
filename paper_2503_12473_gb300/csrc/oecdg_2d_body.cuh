// oecdg_2d_body.cuh -- per-cell device code of the 2D Q^2 OECDG kernels
// (arXiv:2503.12473), shared by the single-mesh kernels (oecdg_2d.cu) and the
// batched kernels (oecdg_batch.cu).
//
// One thread per cell of one mesh; primal and dual cells run the same code:
// cell K's four sub-cells (quarters) and its eight half-faces all lie in the
// four overlapping cells of the other mesh,
//   primal (i,j): dual (i-1+sx, j-1+sy);   dual (i,j): primal (i+sx, j+sy),
// and in the overlapping cell the point of K's reference coordinate xi sits at
// xi' = xi + 1 - 2 sx (the overlapping cell's centre lies on K's face).
#pragma once

#include <climits>

#include "oecdg_common.cuh"
#include "oecdg_persist.cuh"

namespace oecdg {

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
template <int F>
struct RhsAcc {
  double r[F][3][3];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) r[f][b][a] = 0.0;
  }
  __device__ __forceinline__ double& at(int f, int b, int a) { return r[f][b][a]; }
};

template <int SYS, int BC, int LD, class Acc>
__device__ __forceinline__ void cell_rhs2d(const Geo& g, const double* __restrict__ u, int mesh, int i, int j,
                                           const double* stc, Acc& R) {
  constexpr int F = Fields<SYS>::F;
  const long long P = g.plane;
  const double* uo = u + (long long)(1 - mesh) * F * 9 * P;
  const int off = mesh == 0 ? -1 : 0;
  // stc: the caller's shared step constants, stc[0] = 1/tau_max, written by
  // thread 32 before this function's barrier (read only after it)
  // the dissipation weights w_qy kd P_b(eta) (b = 0, 1, 2) of every point row,
  // uniform over the block: computed once into shared memory, so the points
  // take them by broadcast instead of scaling every field value by kd
  __shared__ double wk[2][3][3];
  __syncthreads();  // stc
  if (threadIdx.x < 18) {
    const double kd = 0.5 * g.hy * stc[0];  // dissipation scale inside A
    const int sy = threadIdx.x / 9, qy = (threadIdx.x / 3) % 3, c = threadIdx.x % 3;
    const double es = xs_self(sy, qy);
    wk[sy][qy][c] = gwt(qy) * (c == 0 ? 1.0 : (c == 1 ? es : lp(2, es))) * kd;
  }
  __syncthreads();
  R.zero();

  const int oj0 = wrap_index<BC>(j + off, g.ny), oj1 = wrap_index<BC>(j + 1 + off, g.ny);
// OECDG_STAGE_ROLL_SX=1 keeps the two halves apart (spill loads 1.6 -> 1.0 KB
// per thread) but makes their quadrature constants run-time values: 2.5%
// slower at 1024^2, so the halves stay unrolled by default.
#if OECDG_STAGE_ROLL_SX
#pragma unroll 1
#else
#pragma unroll
#endif
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
            T[f][b] = fma(-0.5, ldv<LD>(c + (f * 9 + b * 3 + 2) * P), ldv<LD>(c + (f * 9 + b * 3) * P));
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
      // R += (-s) P_a(s) (4/hx) Bf, s = 2 sx - 1 (explicit fma: one rounding
      // per update, the same in every kernel that inlines this)
      const double sc = 4.0 / g.hx, sp = sx ? -sc : sc;
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          R.at(f, b, 0) = fma(sp, Bf[f][b], R.at(f, b, 0));
          R.at(f, b, 1) = fma(-sc, Bf[f][b], R.at(f, b, 1));
          R.at(f, b, 2) = fma(sp, Bf[f][b], R.at(f, b, 2));
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
            T[f][b] = fma(lp(2, xo), ldv<LD>(cb + 2 * P), fma(xo, ldv<LD>(cb + P), ldv<LD>(cb)));
          }
#pragma unroll
        for (int qy = 0; qy < 3; ++qy) {
          const double eo = xs_other(sy, qy), es = xs_self(sy, qy);
          const double w = gwt(qy);
          double V[F], f1[F], f2[F];
#pragma unroll
          for (int f = 0; f < F; ++f) V[f] = fma(lp(2, eo), T[f][2], fma(eo, T[f][1], T[f][0]));
          flux_both<SYS>(g, V, f1, f2);
          const double k0 = wk[sy][qy][0], k1 = wk[sy][qy][1], k2 = wk[sy][qy][2];
#pragma unroll
          for (int f = 0; f < F; ++f) {
            A[f][0] = fma(k0, V[f], A[f][0]);
            A[f][1] = fma(k1, V[f], fma(w, f2[f], A[f][1]));
            A[f][2] = fma(k2, V[f], fma(w * dlp(2, es), f2[f], A[f][2]));
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
      // (taking these per-block constants from shared memory instead moved
      // register spills out to DRAM and lengthened the kernel)
      const double wa = gwt(qx) * 2.0 / g.hy, wb = gwt(qx) * 2.0 / g.hx;
      const double wa1 = wa * xsf, wa2 = wa * lp(2, xsf), wb2 = wb * dlp(2, xsf);
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          R.at(f, b, 0) = fma(wa, A[f][b], R.at(f, b, 0));
          R.at(f, b, 1) = fma(wa1, A[f][b], fma(wb, B[f][b], R.at(f, b, 1)));
          R.at(f, b, 2) = fma(wa2, A[f][b], fma(wb2, B[f][b], R.at(f, b, 2)));
        }
    }
  }
  // The caller forms L_ab = (2a+1)(2b+1)/16 R_ab - u_ab / tau_max: the
  // -(1/tau_max) int u_K phi term is exact through the diagonal mass matrix.
}

// Order-preserving map of a double to a signed 64-bit key and back: the
// sigma extrema are taken on the integer pipes, which leaves the FP64 pipe
// (the kernel's bound) to the arithmetic.  For every non-NaN x, y:
// x < y <=> key(x) < key(y) (-0 sorts just below +0).
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dunkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// block reduction of (sum, key max, key min): result valid in thread 0
__device__ __forceinline__ void block_reduce_sum_keys(double& s, long long& kx, long long& kn, double* sh) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(full, s, o);
    kx = max(kx, __shfl_down_sync(full, kx, o));
    kn = min(kn, __shfl_down_sync(full, kn, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  long long* shk = (long long*)(sh + 32);
  __syncthreads();
  if (lane == 0) {
    sh[warp] = s;
    shk[warp] = kx;
    shk[32 + warp] = kn;
  }
  __syncthreads();
  if (warp == 0) {
    s = lane < nw ? sh[lane] : 0.0;
    kx = lane < nw ? shk[lane] : LLONG_MIN;
    kn = lane < nw ? shk[32 + lane] : LLONG_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(full, s, o);
      kx = max(kx, __shfl_down_sync(full, kx, o));
      kn = min(kn, __shfl_down_sync(full, kn, o));
    }
  }
}

enum { MODE_RHS = 0, MODE_STAGE = 1 };

// The work of one thread of a stage block: cell (i, j) of `mesh` (inactive
// threads of a ragged tile compute a clamped cell, store nothing and give
// neutral partials).  `pblk` = this block's partials [F][3].
template <int SYS, int BC, int MODE, int LD = LD_NC>
__device__ __forceinline__ void stage_cell2d(const Geo& g, const double* __restrict__ uin,
                                             const double* __restrict__ un, double* __restrict__ out,
                                             const double* __restrict__ dt, double ca, double cb,
                                             double* __restrict__ pblk, int mesh, int i, int j) {
  constexpr int F = Fields<SYS>::F;
  const bool active = i < g.nx && j < g.ny;
  const int ic = active ? i : 0, jc = active ? j : 0;
  // the step's constants, once per block: 1/tau_max and the combination's
  // cb alpha, cb tau and cb tau c_ab (below); the barrier in cell_rhs2d
  // publishes them
  __shared__ double stc[12];
  if (threadIdx.x == 32) {
    const double tau = ldv<LD>(dt), tm = ldv<LD>(dt + 1);
    stc[0] = 1.0 / tm;
    // u_out = ca u^n + cb (u_in + tau L(u_in)) with L = c_ab R - u_in / tau_max
    //       = ca u^n + cb alpha u_in + cb tau c_ab R,   alpha = 1 - tau / tau_max:
    // alpha = 0 unless the step is clipped at the end time, and then the cell's
    // own coefficients drop out (the two u_in terms cancel exactly).
    const double alpha = tau == tm ? 0.0 : (tm - tau) / tm;
    stc[1] = cb * alpha;
    stc[2] = cb * tau;
#pragma unroll
    for (int m = 0; m < 9; ++m) stc[3 + m] = stc[2] * ((2 * (m % 3) + 1) * (2 * (m / 3) + 1) / 16.0);  // cb tau c_ab
  }
  RhsAcc<F> R;
  cell_rhs2d<SYS, BC, LD>(g, uin, mesh, ic, jc, stc, R);
  const double inv_tm = stc[0];
  const long long P = g.plane;
  const long long base = (long long)mesh * F * 9 * P + (long long)jc * g.nx + ic;
  if (MODE == MODE_RHS) {
    if (active)
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int m = 0; m < 9; ++m)
          out[base + (f * 9 + m) * P] = fma((2 * (m % 3) + 1) * (2 * (m / 3) + 1) / 16.0, R.at(f, m / 3, m % 3),
                                            -inv_tm * ldv<LD>(uin + base + (f * 9 + m) * P));
    return;
  } else {
    const double cba = stc[1];
    __shared__ double sh[96];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      double v[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        const long long id = base + (f * 9 + m) * P;
        double s = stc[3 + m] * R.at(f, m / 3, m % 3);  // (cb tau c_ab) R
        if (cba != 0.0) s = fma(cba, ldv<LD>(uin + id), s);
        if (ca != 0.0) s = fma(ca, ldv<LD>(un + id), s);
        v[m] = s;
        if (active) out[id] = s;
      }
      // values at the cell's own 3x3 Gauss points, y-contraction then x; their
      // extrema as integer keys.  The 3-point nodes are 0 and +-g, so along
      // each direction c0 + c1 P_1 + c2 P_2 takes c0 - c2/2 at 0 and
      // (c0 + P_2(g) c2) +- g c1 at +-g: 4 FMA for the 3 points, not 6.
      long long kx = LLONG_MIN, kn = LLONG_MAX;
      constexpr double G = gnode(2), P2G = lp(2, gnode(2));
      double t[3][3];  // [node of eta: -g, 0, +g][a]
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double e = fma(P2G, v[6 + a], v[a]);
        t[0][a] = fma(-G, v[3 + a], e);
        t[1][a] = fma(-0.5, v[6 + a], v[a]);
        t[2][a] = fma(G, v[3 + a], e);
      }
#pragma unroll
      for (int qy = 0; qy < 3; ++qy) {
        const double e = fma(P2G, t[qy][2], t[qy][0]);
        const long long k0 = dkey(fma(-G, t[qy][1], e)), k1 = dkey(fma(-0.5, t[qy][2], t[qy][0]));
        const long long k2 = dkey(fma(G, t[qy][1], e));
        kx = max(kx, max(k0, max(k1, k2)));
        kn = min(kn, min(k0, min(k1, k2)));
      }
      double s = active ? v[0] : 0.0;
      if (!active) {
        kx = LLONG_MIN;
        kn = LLONG_MAX;
      }
      block_reduce_sum_keys(s, kx, kn, sh);
      if (threadIdx.x == 0) {
        double* p = pblk + f * 3;
        p[0] = s;
        p[1] = dunkey(kx);
        p[2] = dunkey(kn);
      }
    }
  }
}

// REC = 1 also records, per cell and order m, (delta^m, the field that gives
// the max, that field's x- and y-face sums) for the adjoint: rec[cell][3][4].
// isg (optional): 1/sigma of this mesh's fields (0 where sigma = 0), taken
// once per block by the caller (oe_inv_sigma) instead of once per cell.
// ISO = true requires hx == hy: every m-th derivative then carries the same
// factor (2/h)^m, so the traces stay in reference units and the factor is
// applied once, in the constants of delta^m (the recorded sums are physical).
// The overlapping cell's part of one half-face's difference series: its
// trace at its centre line (normal coordinate 0) re-expanded in K's
// tangential coordinate (shift dl): for each series X (value o0, first normal
// derivative o1, second / 3 o2), X_2, the P_1 coefficient fma(3 dl, X_2, X_1)
// and the P_0 coefficient fma(3/2, X_2, fma(dl, X_1, X_0)), plus o2's raw
// first two coefficients.  It depends on the overlapping cell and dl only, so
// the two cells on either side of a face (cells j and j + 1 for a face normal
// to y) can share it.
struct OSer {
  double o02, E01, E00, o12, E11, E10, o22, E21, E20, o20, o21;
};
constexpr int OSER_N = 11;

template <int LD, bool ISO>
__device__ __forceinline__ OSer oe_oseries(const double* co, long long P, int n, double dl) {
  double w0[3], w1[3], w2[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    w0[t] = ldv<LD>(co + (n == 0 ? t * 3 : t) * P);
    w1[t] = ldv<LD>(co + (n == 0 ? t * 3 + 1 : 3 + t) * P);
    w2[t] = ldv<LD>(co + (n == 0 ? t * 3 + 2 : 6 + t) * P);
  }
  const double o0[3] = {fma(-0.5, w2[0], w0[0]), fma(-0.5, w2[1], w0[1]), fma(-0.5, w2[2], w0[2])};
  OSer s;
  s.o02 = o0[2];
  s.E01 = fma(3.0 * dl, o0[2], o0[1]);
  s.E00 = fma(1.5, o0[2], fma(dl, o0[1], o0[0]));
  s.o12 = w1[2];
  s.E11 = fma(3.0 * dl, w1[2], w1[1]);
  s.E10 = fma(1.5, w1[2], fma(dl, w1[1], w1[0]));
  s.o22 = w2[2];
  s.E21 = fma(3.0 * dl, w2[2], w2[1]);
  s.E20 = ISO ? 0.0 : fma(1.5, w2[2], fma(dl, w2[1], w2[0]));
  s.o20 = w2[0];
  s.o21 = w2[1];
  return s;
}

__device__ __forceinline__ void oser_store(double* p, const OSer& s) {
  p[0] = s.o02; p[1] = s.E01; p[2] = s.E00; p[3] = s.o12; p[4] = s.E11; p[5] = s.E10;
  p[6] = s.o22; p[7] = s.E21; p[8] = s.E20; p[9] = s.o20; p[10] = s.o21;
}
__device__ __forceinline__ OSer oser_load(const double* p) {
  OSer s;
  s.o02 = p[0]; s.E01 = p[1]; s.E00 = p[2]; s.o12 = p[3]; s.E11 = p[4]; s.E10 = p[5];
  s.o22 = p[6]; s.E21 = p[7]; s.E20 = p[8]; s.o20 = p[9]; s.o21 = p[10];
  return s;
}

// ROWS > 0: the block is ROWS rows of 32 cells (row ty = warp ty, cell i of
// lane i % 32), and the rows share the faces between them: for each field,
// every cell first takes the overlapping-cell series of its upper y-face
// (both halves) into osh[2][ROWS][32][OSER_N] (shared), and after a barrier a
// cell above row 0 reads its lower face's series from the row below instead
// of loading and forming it.  The arithmetic is the same, so the results are
// the same bits as with ROWS = 0.  Every thread of the block must call it (no
// early return: a cell outside the mesh computes a clamped cell and stores
// nothing).
template <int SYS, int BC, bool WRITE_DELTA, int REC = 0, bool ISO = false, int LD = LD_NC, int ROWS = 0>
__device__ __forceinline__ void oe_cell2d(const Geo& g, const double* __restrict__ uh, double* __restrict__ usig,
                                          const double* __restrict__ dt, const double* __restrict__ sigma,
                                          double* __restrict__ delta_out, int* __restrict__ status, int mesh, int i,
                                          int j, double* __restrict__ rec = nullptr,
                                          const double* __restrict__ isg = nullptr, double* osh = nullptr,
                                          int ty = 0) {
  constexpr int F = Fields<SYS>::F;
  const bool active = i < g.nx && j < g.ny;
  if (ROWS == 0 && !active) return;
  if (!active) i = j = 0;
  const int lane = threadIdx.x & 31;
  const long long P = g.plane;
  const double* us = uh + (long long)mesh * F * 9 * P + (long long)j * g.nx + i;
  const double* uo = uh + (long long)(1 - mesh) * F * 9 * P;
  const int off = mesh == 0 ? -1 : 0;
  const int oi0 = wrap_index<BC>(i + off, g.nx), oi1 = wrap_index<BC>(i + 1 + off, g.nx);
  const int oj0 = wrap_index<BC>(j + off, g.ny), oj1 = wrap_index<BC>(j + 1 + off, g.ny);

  // wave speeds beta_{e,K} at the cell average
  double bx, by;
  if (SYS == SYS_EULER) {
    const double rho = ldv<LD>(us), mx = ldv<LD>(us + 9 * P), my = ldv<LD>(us + 18 * P), E = ldv<LD>(us + 27 * P);
    const double r = rcp_pos(rho);  // NaN for rho <= 0 or subnormal: flagged below
    const double vx = mx * r, vy = my * r;
    const double p = (g.gamma - 1.0) * fma(-0.5, fma(mx, vx, my * vy), E);
    double c = 0.0;
    if (rho > 0.0 && p > 0.0) {
      c = sqrt_pos(fma(g.gamma * p, r, SQ_FLOOR));
    } else if (active) {
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
  const double dx1 = g.i2x, dy1 = g.i2y;  // reference -> physical derivative: 2/hx, 2/hy
  // ISO: the face sums of orders 1 and 2 are in reference units; their
  // physical factors dx1 and dx1^2 join the constants
  const double iso1 = ISO ? dx1 : 1.0, iso2 = ISO ? dx1 * dx1 : 1.0;
  const double cx0 = g.i12x, cx1 = 0.25 * iso1, cx2 = g.h24x5 * iso2;  // 1/(12 hx), 5 hx/24
  const double cy0 = g.i12y, cy1 = 0.25 * iso1, cy2 = g.h24y5 * iso2;

  double d0 = 0.0, d1 = 0.0, d2 = 0.0;  // max over fields
  int rf[3] = {-1, -1, -1};             // REC: field of the max, and its face sums
  double rs[3][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const double sg = ldv<LD>(sigma + mesh * F + f);
    const double* cs = us + f * 9 * P;
    double u[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) u[m] = ldv<LD>(cs + m * P);
    if (ROWS > 0) {  // this cell's upper y-face, both halves, for itself and the row above
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const double* co = uo + f * 9 * P + (long long)oj1 * g.nx + (h ? oi1 : oi0);
        oser_store(osh + ((h * ROWS + ty) * 32 + lane) * OSER_N, oe_oseries<LD, ISO>(co, P, 1, 1.0 - 2.0 * h));
      }
      __syncthreads();
    }
    double Sx0 = 0.0, Sx1 = 0.0, Sx2 = 0.0, Sy0 = 0.0, Sy1 = 0.0, Sy2 = 0.0;
    // Faces normal to direction n (0: x, 1: y), at reference coordinate s of K.
    // Along the face, K's trace and its normal derivatives of order 0, 1, 2 are
    // Legendre series c0, c1, 3 c2 in the tangential coordinate t; the
    // overlapping cell's are o0, o1, 3 o2 in its own tangential coordinate t' = t + dl,
    // dl = 1 - 2 h (h = the half), re-expanded in t with
    //   P_1(t + dl) = P_1(t) + dl,  P_2(t + dl) = P_2(t) + 3 dl P_1(t) + 3/2.
    // The difference series (u_K - w) is then scaled to physical derivatives
    // and evaluated at the half-face's Gauss points; the weighted point values
    // accumulate straight into the direction's face sums (12 points each).
    // Two coefficients are formed already multiplied by 3, where the factor
    // is needed (3 e0_2 for the tangential derivative, ISO: 3 e2_0 for the
    // second normal derivative), from 3 x K's coefficient taken once per
    // direction: one FMA per half-face instead of a subtraction and a product.
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      const double dn1 = n == 0 ? dx1 : dy1, dt1 = n == 0 ? dy1 : dx1;  // normal / tangential scales
      const double dn2 = dn1 * dn1, dt2 = dt1 * dt1;
      double& A0 = n == 0 ? Sx0 : Sy0;
      double& A1 = n == 0 ? Sx1 : Sy1;
      double& A2 = n == 0 ? Sx2 : Sy2;
      // K's coefficients (normal degree a = 0, 1, 2; tangential degree t)
      double k02[3], k1[3], k2[3];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const double u0 = n == 0 ? u[t * 3] : u[t];
        k1[t] = n == 0 ? u[t * 3 + 1] : u[3 + t];
        k2[t] = n == 0 ? u[t * 3 + 2] : u[6 + t];
        k02[t] = u0 + k2[t];  // P_0 + P_2 at either side (P_2(+-1) = 1)
      }
      const double k02x3 = 3.0 * k02[2];
      const double k2x3 = 3.0 * k2[0];  // ISO: 3 c2_0
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const double s = 2.0 * side - 1.0;
        double c0[2], c1[3];
#pragma unroll
        for (int t = 0; t < 2; ++t) c0[t] = k02[t] + s * k1[t];
        const double c0x3 = fma(3.0 * s, k1[2], k02x3);  // 3 c0_2
#pragma unroll
        for (int t = 0; t < 3; ++t) c1[t] = fma(3.0 * s, k2[t], k1[t]);
        const double* c2 = k2;  // the second normal derivative is 3 c2; the 3 is applied below
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const double dl = 1.0 - 2.0 * h;
          // the overlapping cell's series: shared with the row below / above
          // where ROWS > 0, else formed here
          OSer o;
          if (ROWS > 0 && n == 1 && side == 1) {
            o = oser_load(osh + ((h * ROWS + ty) * 32 + lane) * OSER_N);
          } else if (ROWS > 0 && n == 1 && side == 0 && ty > 0) {
            o = oser_load(osh + ((h * ROWS + ty - 1) * 32 + lane) * OSER_N);
          } else {
            const int oi = n == 0 ? (side ? oi1 : oi0) : (h ? oi1 : oi0);
            const int oj = n == 0 ? (h ? oj1 : oj0) : (side ? oj1 : oj0);
            o = oe_oseries<LD, ISO>(uo + f * 9 * P + (long long)oj * g.nx + oi, P, n, dl);
          }
          // difference series in K's tangential coordinate (e0_2 as 3 e0_2)
          double e0[2], e1[3], e2[3];
          const double e02x3 = fma(-3.0, o.o02, c0x3);
          e0[1] = c0[1] - o.E01;
          e0[0] = c0[0] - o.E00;
          e1[2] = c1[2] - o.o12;
          e1[1] = c1[1] - o.E11;
          e1[0] = c1[0] - o.E10;
          e2[2] = c2[2] - o.o22;
          e2[1] = c2[1] - o.E21;
          // physical scalings: normal derivative series (order 1, 2), tangential
          // derivative of the value and of the normal derivative, second
          // tangential derivative (a constant on the half-face)
          double a0, a1, a2, b0, b1, b2, t0, t1, m0, m1, tt;
          // (ISO: the factors 3 of the second normal and the mixed derivative
          // go into the points' constant coefficients, see hn and hm below)
          if constexpr (ISO) {
            a0 = e1[0], a1 = e1[1], a2 = e1[2];
            b0 = fma(-4.5, o.o22, fma(-3.0 * dl, o.o21, fma(-3.0, o.o20, k2x3)));  // 3 e2_0
            b1 = e2[1], b2 = e2[2];
            t0 = e0[1], t1 = e02x3;
            m0 = a1, m1 = a2;
            tt = t1;
          } else {
            const double dn2x3 = 3.0 * dn2;
            e2[0] = c2[0] - o.E20;
            a0 = dn1 * e1[0], a1 = dn1 * e1[1], a2 = dn1 * e1[2];
            b0 = dn2x3 * e2[0], b1 = dn2x3 * e2[1], b2 = dn2x3 * e2[2];
            t0 = dt1 * e0[1], t1 = dt1 * e02x3;
            m0 = dt1 * a1, m1 = 3.0 * dt1 * a2;
            tt = dt2 * e02x3;
          }
          const double tt2 = fma(tt, tt, SQ_FLOOR);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const double ts = xs_self(h, q);
            const double p2 = lp(2, ts);
            const double v = fma(p2 / 3.0, e02x3, fma(ts, e0[1], e0[0]));  // u_K - w
            const double gn = fma(p2, a2, fma(ts, a1, a0));                 // normal derivative
            const double gt = fma(ts, t1, t0);                              // tangential derivative
            const double hn = ISO ? fma(3.0 * p2, b2, fma(3.0 * ts, b1, b0))  // second normal
                                  : fma(p2, b2, fma(ts, b1, b0));
            const double hm = ISO ? fma(3.0 * ts, m1, m0) : fma(ts, m1, m0);  // mixed
            A0 = fma(gwt(q), fabs(v), A0);
            A1 = fma(gwt(q), sqrt_pos(fma(gn, gn, fma(gt, gt, SQ_FLOOR))), A1);
            A2 = fma(gwt(q), sqrt_pos(fma(hn, hn, fma(hm, hm, tt2))), A2);
          }
        }
      }
    }
    if (sg != 0.0) {
      // explicit fma: the recording and the plain instantiation must round alike
      const double is = isg ? isg[f] : 1.0 / sg;
      const double v0 = fma(bx * cx0, Sx0, (by * cy0) * Sy0) * is;
      const double v1 = fma(bx * cx1, Sx1, (by * cy1) * Sy1) * is;
      const double v2 = fma(bx * cx2, Sx2, (by * cy2) * Sy2) * is;
      if (REC) {
        if (v0 > d0) { d0 = v0; rf[0] = f; rs[0][0] = Sx0; rs[0][1] = Sy0; }
        if (v1 > d1) { d1 = v1; rf[1] = f; rs[1][0] = Sx1; rs[1][1] = Sy1; }
        if (v2 > d2) { d2 = v2; rf[2] = f; rs[2][0] = Sx2; rs[2][1] = Sy2; }
      } else {
        d0 = fmax(d0, v0);
        d1 = fmax(d1, v1);
        d2 = fmax(d2, v2);
      }
    }
    if (ROWS > 0) __syncthreads();  // osh is rewritten for the next field
  }
  if (!active) return;
  if (REC) {
    double* r = rec + ((long long)mesh * P + (long long)j * g.nx + i) * 12;
    const double dd[3] = {d0, d1, d2};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      r[4 * m] = dd[m];
      r[4 * m + 1] = (double)rf[m];
      const double sc = m == 0 ? 1.0 : (m == 1 ? iso1 : iso2);  // physical sums
      r[4 * m + 2] = ISO ? rs[m][0] * sc : rs[m][0];
      r[4 * m + 3] = ISO ? rs[m][1] * sc : rs[m][1];
    }
  }
  if (WRITE_DELTA) {
    double* dp = delta_out + (((long long)mesh * g.ny + j) * g.nx + i) * 3;
    dp[0] = d0;
    dp[1] = d1;
    dp[2] = d2;
  }
  if (usig != nullptr) {
    const double tau = ldv<LD>(dt);
    const double r1 = d0 + d1, r2 = r1 + d2;
    const double e1 = exp(-tau * r1), e2 = exp(-tau * r2);
    double* os = usig + (long long)mesh * F * 9 * P + (long long)j * g.nx + i;
#pragma unroll
    for (int f = 0; f < F; ++f) {
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        const int deg = (m % 3) + (m / 3);
        const double v = ldv<LD>(us + (f * 9 + m) * P);
        os[(f * 9 + m) * P] = deg == 0 ? v : (deg == 1 ? v * e1 : v * e2);
      }
    }
  }
}

}  // namespace oecdg
