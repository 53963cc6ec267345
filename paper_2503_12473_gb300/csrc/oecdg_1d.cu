// oecdg_1d.cu -- 1D P^2 kernels of the OECDG forward step (arXiv:2503.12473),
// Eq. (eq:1D_H) and the 1D form of the damping coefficients (Remark in
// Section 2.2).  One thread per cell of one mesh (blockIdx.y = mesh); primal
// cell i overlaps dual cells i-1 (left half) and i (right half), dual cell i
// overlaps primal cells i and i+1; in the overlapping cell the point xi of
// half s sits at xi' = xi + 1 - 2 s.
#include "oecdg_common.cuh"
#include "oecdg_kernels.h"

namespace oecdg {

constexpr int NT1 = 128;
constexpr double DINF1 = __builtin_huge_val();

template <int SYS>
struct Fields1 {
  static constexpr int F = SYS == SYS_EULER ? 3 : 1;
};

template <int SYS>
__device__ __forceinline__ void flux1(const Geo& g, const double* w, double* f) {
  if (SYS == SYS_EULER) {
    const double r = __drcp_rn(w[0]);
    const double v = w[1] * r;
    const double p = (g.gamma - 1.0) * (w[2] - 0.5 * w[1] * v);
    f[0] = w[1];
    f[1] = fma(w[1], v, p);
    f[2] = (w[2] + p) * v;
  } else {
    f[0] = g.adv_x * w[0];
  }
}

// L_a = (2a+1) [ sum_{s,q} (w_q/4)(w/tau_max) P_a(xi) + (1/h) sum (w_q/2) f(w) P_a'(xi)
//               - (1/h)(f_R - (-1)^a f_L) ] - u_a / tau_max
template <int SYS, int BC>
__device__ __forceinline__ void cell_rhs1d(const Geo& g, const double* __restrict__ u, int mesh, int i, double inv_tm,
                                           double (&L)[Fields1<SYS>::F][3]) {
  constexpr int F = Fields1<SYS>::F;
  const long long P = g.plane;
  const double* uo = u + (long long)(1 - mesh) * F * 3 * P;
  const double* us = u + (long long)mesh * F * 3 * P + i;
  const int off = mesh == 0 ? -1 : 0;
  double Ad[F][3], Bd[F][3];  // dissipation and flux-gradient sums
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int a = 0; a < 3; ++a) Ad[f][a] = Bd[f][a] = 0.0;
  double fL[F], fR[F];
#pragma unroll
  for (int sx = 0; sx < 2; ++sx) {
    const double* c = uo + wrap_index<BC>(i + sx + off, g.nx);
    double w0[F], w1[F], w2[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      w0[f] = __ldg(c + (f * 3) * P);
      w1[f] = __ldg(c + (f * 3 + 1) * P);
      w2[f] = __ldg(c + (f * 3 + 2) * P);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double xo = xs_other(sx, q), xsf = xs_self(sx, q);
      double V[F], fl[F];
#pragma unroll
      for (int f = 0; f < F; ++f) V[f] = fma(lp(2, xo), w2[f], fma(xo, w1[f], w0[f]));
      flux1<SYS>(g, V, fl);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        Ad[f][0] = fma(gwt(q), V[f], Ad[f][0]);
        Ad[f][1] = fma(gwt(q) * xsf, V[f], Ad[f][1]);
        Ad[f][2] = fma(gwt(q) * lp(2, xsf), V[f], Ad[f][2]);
        Bd[f][1] = fma(gwt(q), fl[f], Bd[f][1]);
        Bd[f][2] = fma(gwt(q) * dlp(2, xsf), fl[f], Bd[f][2]);
      }
    }
    // face of this half: the overlapping cell's centre (xi' = 0)
    double V[F];
#pragma unroll
    for (int f = 0; f < F; ++f) V[f] = fma(-0.5, w2[f], w0[f]);
    if (sx) flux1<SYS>(g, V, fR);
    else flux1<SYS>(g, V, fL);
  }
  const double ih = 1.0 / g.hx;
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double face = fR[f] - ((a & 1) ? -fL[f] : fL[f]);
      const double br = 0.25 * inv_tm * Ad[f][a] + ih * (0.5 * Bd[f][a] - face);
      L[f][a] = fma((double)(2 * a + 1), br, -inv_tm * __ldg(us + (f * 3 + a) * P));
    }
}

enum { MODE1_RHS = 0, MODE1_STAGE = 1 };

template <int SYS, int BC, int MODE>
__global__ void __launch_bounds__(NT1) k_stage1d(Geo g, const double* __restrict__ uin, const double* __restrict__ un,
                                                 double* __restrict__ out, const double* __restrict__ dt, double ca,
                                                 double cb, double* __restrict__ partials) {
  constexpr int F = Fields1<SYS>::F;
  const int mesh = blockIdx.y;
  const int i = blockIdx.x * NT1 + threadIdx.x;
  const bool active = i < g.nx;
  const int ic = active ? i : 0;
  const double tau = dt[0], tm = dt[1];
  const double inv_tm = 1.0 / tm;
  double L[F][3];
  cell_rhs1d<SYS, BC>(g, uin, mesh, ic, inv_tm, L);
  const long long P = g.plane;
  const long long base = (long long)mesh * F * 3 * P + ic;
  if (MODE == MODE1_RHS) {
    if (active)
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int a = 0; a < 3; ++a) out[base + (f * 3 + a) * P] = L[f][a];
    return;
  } else {
    __shared__ double sh[96];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      double v[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const long long id = base + (f * 3 + a) * P;
        double s = fma(tau, L[f][a], __ldg(uin + id));
        if (ca != 0.0) s = fma(ca, __ldg(un + id), cb * s);
        v[a] = s;
        if (active) out[id] = s;
      }
      double mx = -DINF1, mn = DINF1;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double val = fma(lp(2, gnode(q)), v[2], fma(gnode(q), v[1], v[0]));
        mx = fmax(mx, val);
        mn = fmin(mn, val);
      }
      double s = active ? v[0] : 0.0;
      if (!active) {
        mx = -DINF1;
        mn = DINF1;
      }
      block_reduce3(s, mx, mn, sh);
      if (threadIdx.x == 0) {
        const long long nblk = gridDim.x;
        double* p = partials + ((mesh * nblk + blockIdx.x) * F + f) * 3;
        p[0] = s;
        p[1] = mx;
        p[2] = mn;
      }
    }
  }
}

// delta^m = (2m+1) h^{m-1} / ((2k-1) m!) beta (|d^m (u^C-u^D)|_R + |...|_L) / sigma,
// max over fields; then the exact damping of the modes of degree 1 and 2.
template <int SYS, int BC, bool WRITE_DELTA>
__global__ void __launch_bounds__(NT1) k_oe1d(Geo g, const double* __restrict__ uh, double* __restrict__ usig,
                                              const double* __restrict__ dt, const double* __restrict__ sigma,
                                              double* __restrict__ delta_out, int* __restrict__ status) {
  constexpr int F = Fields1<SYS>::F;
  const int mesh = blockIdx.y;
  const int i = blockIdx.x * NT1 + threadIdx.x;
  if (i >= g.nx) return;
  const long long P = g.plane;
  const double* us = uh + (long long)mesh * F * 3 * P + i;
  const double* uo = uh + (long long)(1 - mesh) * F * 3 * P;
  const int off = mesh == 0 ? -1 : 0;
  const int oL = wrap_index<BC>(i + off, g.nx), oR = wrap_index<BC>(i + 1 + off, g.nx);
  double beta;
  if (SYS == SYS_EULER) {
    const double rho = __ldg(us), m = __ldg(us + 3 * P), E = __ldg(us + 6 * P);
    const double v = m / rho;
    const double p = (g.gamma - 1.0) * (E - 0.5 * m * v);
    if (rho > 0.0 && p > 0.0) {
      beta = fabs(v) + sqrt(g.gamma * p / rho);
    } else {
      atomicOr(status, ST_NONPHYSICAL);
      beta = 0.0;
    }
  } else {
    beta = fabs(g.adv_x);
  }
  const double h = g.hx, d1 = 2.0 / h, d2 = d1 * d1;
  // (2m+1) h^{m-1} / ((2k-1) m!), k = 2
  const double k0 = 1.0 / (3.0 * h), k1 = 1.0, k2 = 5.0 * h / 6.0;
  double dl0 = 0.0, dl1 = 0.0, dl2 = 0.0;
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const double sg = __ldg(sigma + mesh * F + f);
    const double u0 = __ldg(us + (f * 3) * P), u1 = __ldg(us + (f * 3 + 1) * P), u2 = __ldg(us + (f * 3 + 2) * P);
    const double* cl = uo + (f * 3) * P + oL;
    const double* cr = uo + (f * 3) * P + oR;
    const double l0 = __ldg(cl), l1 = __ldg(cl + P), l2 = __ldg(cl + 2 * P);
    const double r0 = __ldg(cr), r1 = __ldg(cr + P), r2 = __ldg(cr + 2 * P);
    // right face xi = 1 (overlapping cell oR at its centre), left face xi = -1 (oL)
    const double jr0 = fabs((u0 + u1 + u2) - fma(-0.5, r2, r0));
    const double jl0 = fabs((u0 - u1 + u2) - fma(-0.5, l2, l0));
    const double jr1 = fabs(d1 * (fma(3.0, u2, u1) - r1));
    const double jl1 = fabs(d1 * (fma(-3.0, u2, u1) - l1));
    const double jr2 = fabs(d2 * 3.0 * (u2 - r2));
    const double jl2 = fabs(d2 * 3.0 * (u2 - l2));
    if (sg != 0.0) {
      const double is = beta / sg;
      dl0 = fmax(dl0, k0 * (jr0 + jl0) * is);
      dl1 = fmax(dl1, k1 * (jr1 + jl1) * is);
      dl2 = fmax(dl2, k2 * (jr2 + jl2) * is);
    }
  }
  if (WRITE_DELTA) {
    double* dp = delta_out + ((long long)mesh * g.nx + i) * 3;
    dp[0] = dl0;
    dp[1] = dl1;
    dp[2] = dl2;
  }
  if (usig != nullptr) {
    const double tau = dt[0];
    const double e1 = exp(-tau * (dl0 + dl1)), e2 = exp(-tau * (dl0 + dl1 + dl2));
    double* os = usig + (long long)mesh * F * 3 * P + i;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      os[(f * 3) * P] = __ldg(us + (f * 3) * P);
      os[(f * 3 + 1) * P] = __ldg(us + (f * 3 + 1) * P) * e1;
      os[(f * 3 + 2) * P] = __ldg(us + (f * 3 + 2) * P) * e2;
    }
  }
}

template <int SYS>
__global__ void k_wave1d(Geo g, const double* __restrict__ u, double* __restrict__ partial, int* __restrict__ status) {
  constexpr int F = Fields1<SYS>::F;
  __shared__ double sh[32];
  const long long n = 2 * g.plane;
  double mx = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    const double* us = u + (long long)mesh * F * 3 * g.plane + cell;
    if (SYS == SYS_EULER) {
      const double rho = us[0], m = us[3 * g.plane], E = us[6 * g.plane];
      const double v = m / rho;
      const double p = (g.gamma - 1.0) * (E - 0.5 * m * v);
      if (rho > 0.0 && p > 0.0) mx = fmax(mx, fabs(v) + sqrt(g.gamma * p / rho));
      else atomicOr(status, ST_NONPHYSICAL);
    } else {
      mx = fabs(g.adv_x);
    }
  }
  mx = block_reduce_max(mx, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 2] = mx;
    partial[blockIdx.x * 2 + 1] = 0.0;
  }
}

__global__ void k_points1d(Geo g, double ax, double* __restrict__ x) {
  const long long n = 2 * g.plane * 6;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % 6);
    const long long c = t / 6;
    const int mesh = (int)(c / g.plane);
    const long long i = c - mesh * g.plane;
    const double xc = ax + (i + 0.5 + 0.5 * mesh) * g.hx;
    x[t] = xc + 0.5 * g.hx * xs_self(r / 3, r % 3);
  }
}

template <int F>
__global__ void k_project1d(Geo g, const double* __restrict__ vals, double* __restrict__ u) {
  const long long n = 2 * g.plane;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    double acc[F][3];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f][0] = acc[f][1] = acc[f][2] = 0.0;
    const double* v = vals + c * 6 * F;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      const double xi = xs_self(r / 3, r % 3), w = 0.5 * gwt(r % 3);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const double x = w * v[r * F + f];
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[f][a] = fma(x, lp(a, xi), acc[f][a]);
      }
    }
    double* o = u + (long long)mesh * F * 3 * g.plane + cell;
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int a = 0; a < 3; ++a) o[(f * 3 + a) * g.plane] = acc[f][a] * ((2 * a + 1) / 2.0);
  }
}

// ----------------------------------------------------------------- launch --

long long partial_blocks_1d(const Geo& g) { return (g.nx + NT1 - 1) / NT1; }

template <int SYS, int BC>
static cudaError_t stage1d_t(const Geo& g, int rhs_only, const double* uin, const double* un, double* out,
                             const double* dt, double ca, double cb, double* partials, cudaStream_t st) {
  const dim3 grid((g.nx + NT1 - 1) / NT1, 2);
  if (rhs_only) k_stage1d<SYS, BC, MODE1_RHS><<<grid, NT1, 0, st>>>(g, uin, un, out, dt, ca, cb, partials);
  else k_stage1d<SYS, BC, MODE1_STAGE><<<grid, NT1, 0, st>>>(g, uin, un, out, dt, ca, cb, partials);
  return cudaGetLastError();
}

cudaError_t launch_stage1d(int sys, int bc, const Geo& g, int rhs_only, const double* uin, const double* un,
                           double* out, const double* dt, double ca, double cb, double* partials, cudaStream_t st) {
  if (sys == SYS_EULER)
    return bc == BC_PERIODIC ? stage1d_t<SYS_EULER, BC_PERIODIC>(g, rhs_only, uin, un, out, dt, ca, cb, partials, st)
                             : stage1d_t<SYS_EULER, BC_TRANSMISSIVE>(g, rhs_only, uin, un, out, dt, ca, cb, partials, st);
  return bc == BC_PERIODIC ? stage1d_t<SYS_ADV, BC_PERIODIC>(g, rhs_only, uin, un, out, dt, ca, cb, partials, st)
                           : stage1d_t<SYS_ADV, BC_TRANSMISSIVE>(g, rhs_only, uin, un, out, dt, ca, cb, partials, st);
}

template <int SYS, int BC>
static cudaError_t oe1d_t(const Geo& g, const double* uh, double* usig, const double* dt, const double* sigma,
                          double* delta, int* status, cudaStream_t st) {
  const dim3 grid((g.nx + NT1 - 1) / NT1, 2);
  if (delta) k_oe1d<SYS, BC, true><<<grid, NT1, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
  else k_oe1d<SYS, BC, false><<<grid, NT1, 0, st>>>(g, uh, usig, dt, sigma, delta, status);
  return cudaGetLastError();
}

cudaError_t launch_oe1d(int sys, int bc, const Geo& g, const double* uh, double* usig, const double* dt,
                        const double* sigma, double* delta, int* status, cudaStream_t st) {
  if (sys == SYS_EULER)
    return bc == BC_PERIODIC ? oe1d_t<SYS_EULER, BC_PERIODIC>(g, uh, usig, dt, sigma, delta, status, st)
                             : oe1d_t<SYS_EULER, BC_TRANSMISSIVE>(g, uh, usig, dt, sigma, delta, status, st);
  return bc == BC_PERIODIC ? oe1d_t<SYS_ADV, BC_PERIODIC>(g, uh, usig, dt, sigma, delta, status, st)
                           : oe1d_t<SYS_ADV, BC_TRANSMISSIVE>(g, uh, usig, dt, sigma, delta, status, st);
}

int wave_blocks_1d(const Geo& g) {
  long long b = (2 * g.plane + 255) / 256;
  return (int)(b < 1184 ? b : 1184);
}

cudaError_t launch_dt1d(int sys, const Geo& g, const double* u, double* partial, int nblk, double T_end, double* dt,
                        double* time, int* status, cudaStream_t st) {
  if (sys == SYS_EULER) k_wave1d<SYS_EULER><<<nblk, 256, 0, st>>>(g, u, partial, status);
  else k_wave1d<SYS_ADV><<<nblk, 256, 0, st>>>(g, u, partial, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_dt_final(partial, nblk, g.hx, g.hy, 1, g.cfl, T_end, dt, time, st);
}

cudaError_t launch_points1d(const Geo& g, double ax, double* x, cudaStream_t st) {
  k_points1d<<<256, 256, 0, st>>>(g, ax, x);
  return cudaGetLastError();
}

cudaError_t launch_project1d(int sys, const Geo& g, const double* vals, double* u, cudaStream_t st) {
  if (sys == SYS_EULER) k_project1d<3><<<256, 128, 0, st>>>(g, vals, u);
  else k_project1d<1><<<256, 128, 0, st>>>(g, vals, u);
  return cudaGetLastError();
}

}  // namespace oecdg
