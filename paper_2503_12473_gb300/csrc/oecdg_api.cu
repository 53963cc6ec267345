// oecdg_api.cu -- the C-ABI of include/oecdg.h: context, argument checks and
// the stage pipeline of Eq. (eq:RKCDG):
//   per step:  wave-speed reduction -> (tau, tau_max) on the device
//   per stage: k_stage (CDG RHS + RK combine + sigma partials) -> k_sigma ->
//              k_oe (damping coefficients + exact OE step)
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/oecdg.h"
#include "oecdg_common.cuh"
#include "oecdg_ctx.h"
#include "oecdg_kernels.h"
#include "oecdg_persist.cuh"

using namespace oecdg;

enum { PROF_STAGE = 0, PROF_OE = 1 };

static void prof_mark(cdg_ctx* c, int cls, int stop) {
  if (!c->prof_on || c->capturing) return;
  const int n = c->prof_n[cls];
  if (n >= c->prof_cap) return;
  cudaEventRecord(c->prof_ev[cls][2 * n + stop], c->stream);
  if (stop) c->prof_n[cls] = n + 1;
}

static void prof_release(cdg_ctx* c) {
  for (int k = 0; k < 2; ++k) {
    if (!c->prof_ev[k]) continue;
    for (int q = 0; q < 2 * c->prof_cap; ++q) cudaEventDestroy(c->prof_ev[k][q]);
    free(c->prof_ev[k]);
    c->prof_ev[k] = nullptr;
  }
  c->prof_cap = 0;
  c->prof_on = 0;
}

static int basis_of(const cdg_ctx* c) { return c->d.basis == CDG_BASIS_Q ? BASIS_Q : BASIS_P; }

static cdg_status fail(cdg_ctx* c, cdg_status s, const char* msg) {
  if (c) snprintf(c->err, sizeof c->err, "%s", msg);
  return s;
}

static cdg_status cuda_fail(cdg_ctx* c, cudaError_t e, const char* where) {
  if (c) snprintf(c->err, sizeof c->err, "%s: %s", where, cudaGetErrorString(e));
  return CDG_ECUDA;
}

#define CK(expr, where)                          \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

extern "C" {

cdg_status cdg_init_mesh(const cdg_mesh_desc* desc, void* stream, cdg_ctx** out) {
  if (out) *out = nullptr;
  if (!desc || !out) return CDG_EINVAL;
  const cdg_mesh_desc& d = *desc;
  if (d.dim != 1 && d.dim != 2) return CDG_EINVAL;
  if (d.nx < 2 || (d.dim == 2 && d.ny < 2)) return CDG_EINVAL;
  if (invalid_sides(d)) return CDG_EINVAL;
  if (d.system != CDG_ADVECTION && d.system != CDG_BURGERS && d.system != CDG_EULER) return CDG_EINVAL;
  if (d.rk < CDG_RK_EULER1 || d.rk > CDG_RK_RK4) return CDG_EINVAL;
  if (d.basis != CDG_BASIS_Q && d.basis != CDG_BASIS_P) return CDG_EINVAL;
  if (d.k < 1 || d.k > 3) return CDG_EUNSUPPORTED;
  if (!(d.bx > d.ax) || (d.dim == 2 && !(d.by > d.ay)) || !(d.cfl > 0.0)) return CDG_EINVAL;
  if (d.system == CDG_EULER && !(d.gamma > 1.0)) return CDG_EINVAL;
  const long long ny = d.dim == 2 ? d.ny : 1;
  if ((long long)d.nx * ny > (1LL << 31)) return CDG_EINVAL;

  cdg_ctx* c = (cdg_ctx*)calloc(1, sizeof(cdg_ctx));
  if (!c) return CDG_ENOMEM;
  c->d = d;
  c->d.ny = (int)ny;
  c->stream = (cudaStream_t)stream;
  c->F = d.system == CDG_EULER ? d.dim + 2 : 1;
  // the tiled kernels serve Q^2 with forward Euler / SSP-RK2 / SSP-RK3 for
  // advection and Euler with the same periodic or transmissive condition on
  // every side; every other 2D configuration runs the generic ones
  const int ubc = uniform_side_bc(d);
  c->gen2 = d.dim == 2 &&
            (d.k != 2 || d.basis != CDG_BASIS_Q || d.system == CDG_BURGERS || d.rk == CDG_RK_RK4 || ubc < 0);
  c->M = d.dim == 2 ? modes_2k(d.k, d.basis == CDG_BASIS_Q ? BASIS_Q : BASIS_P) : d.k + 1;
  c->sys = d.system == CDG_EULER ? SYS_EULER : d.system == CDG_BURGERS ? SYS_BURGERS : SYS_ADV;
  c->bc = ubc < 0 ? BC_GENERAL : (ubc == CDG_PERIODIC ? BC_PERIODIC : BC_TRANSMISSIVE);
  Geo& g = c->g;
  g.nx = d.nx;
  g.ny = (int)ny;
  geo_sides(d, g);
  g.hx = (d.bx - d.ax) / d.nx;
  g.hy = d.dim == 2 ? (d.by - d.ay) / d.ny : 1.0;
  g.gamma = d.gamma;
  g.adv_x = d.adv_x;
  g.adv_y = d.adv_y;
  g.cfl = d.cfl;
  finish_geo(g);
  c->numel = (size_t)2 * c->F * c->M * g.plane;
  c->nblk = d.dim == 2 ? (c->gen2 ? partial_blocks_2k(g) : partial_blocks_2d(g)) : partial_blocks_1d(g);
  c->wave_blk = d.dim == 2 ? wave_blocks_2d(g) : wave_blocks_1d(g);

  cudaError_t e = cudaSuccess;
  void* p = nullptr;
#define ALLOC(field, bytes)                         \
  do {                                              \
    e = cudaMalloc(&p, (bytes));                    \
    if (e != cudaSuccess) goto nomem;               \
    c->field = (decltype(c->field))p;               \
  } while (0)
  ALLOC(buf_a, c->numel * sizeof(double));
  ALLOC(buf_b, c->numel * sizeof(double));
  if (d.rk == CDG_RK_RK4) {
    ALLOC(buf_c, c->numel * sizeof(double));
    ALLOC(buf_d, c->numel * sizeof(double));
  }
  ALLOC(partials, (size_t)2 * c->nblk * c->F * 3 * sizeof(double));
  ALLOC(wave_partial, ((size_t)c->wave_blk * 2 + 1) * sizeof(double));  // + the 1D time step's ticket
  ALLOC(dt, 2 * sizeof(double));
  ALLOC(rhs_dt, 2 * sizeof(double));
  ALLOC(time, 2 * sizeof(double));
  ALLOC(sigma, (size_t)2 * c->F * sizeof(double));
  ALLOC(avg, (size_t)2 * c->F * sizeof(double));
  ALLOC(status, sizeof(int));
#undef ALLOC
  c->wait_s = 5.0;
  e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->time, 0, sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->dt, 0, 2 * sizeof(double), c->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->wave_partial + 2 * (size_t)c->wave_blk, 0, sizeof(double), c->stream);
  // the scratch states start at 0, so that the primal mesh's unused slots of
  // the padded layout (walls) stay 0 through every stage and copy
  if (e == cudaSuccess) e = cudaMemsetAsync(c->buf_a, 0, c->numel * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->buf_b, 0, c->numel * sizeof(double), c->stream);
  if (e == cudaSuccess && c->buf_c) e = cudaMemsetAsync(c->buf_c, 0, c->numel * sizeof(double), c->stream);
  if (e == cudaSuccess && c->buf_d) e = cudaMemsetAsync(c->buf_d, 0, c->numel * sizeof(double), c->stream);
  c->sn = sigma_norm(d, g);
  if (e != cudaSuccess) {
    cdg_free(c);
    return CDG_ECUDA;
  }
  *out = c;
  return CDG_OK;
nomem:
  (void)cudaGetLastError();  // clear the failed allocation: later launch checks must not see it
  cdg_free(c);
  return CDG_ENOMEM;
}

cdg_status cdg_free(cdg_ctx* c) {
  if (!c) return CDG_OK;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->buf_a);
  cudaFree(c->buf_b);
  cudaFree(c->buf_c);
  cudaFree(c->buf_d);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  cudaFree(c->partials);
  cudaFree(c->wave_partial);
  cudaFree(c->dt);
  cudaFree(c->rhs_dt);
  cudaFree(c->time);
  cudaFree(c->sigma);
  cudaFree(c->avg);
  cudaFree(c->status);
  cudaFree(c->p_wpart);
  cudaFree(c->p_bar);
  prof_release(c);
  adj_release(c);
  free(c);
  return CDG_OK;
}

const char* cdg_last_error(const cdg_ctx* c) { return c ? c->err : ""; }

cdg_status cdg_state_numel(const cdg_ctx* c, size_t* n) {
  if (!c || !n) return CDG_EINVAL;
  *n = c->numel;
  return CDG_OK;
}

cdg_status cdg_launch_count(const cdg_ctx* c, long long* n) {
  if (!c || !n) return CDG_EINVAL;
  *n = c->launches;
  return CDG_OK;
}

cdg_status cdg_quad_points(cdg_ctx* ctx, double* d_xy, size_t* npts) {
  if (!ctx || !npts) return CDG_EINVAL;
  const size_t q = ctx->d.k + 1;
  const size_t per = ctx->d.dim == 2 ? 4 * q * q : 2 * q;
  *npts = (size_t)2 * ctx->g.plane * per;  // the padded layout's cells
  if (!d_xy) return CDG_OK;
  if (ctx->gen2)
    CK(launch_points2k(ctx->d.k, ctx->g, ctx->d.ax, ctx->d.ay, ctx->d.bx, ctx->d.by, d_xy, ctx->stream), "quad_points");
  else if (ctx->d.dim == 2) CK(launch_points2d(ctx->g, ctx->d.ax, ctx->d.ay, d_xy, ctx->stream), "quad_points");
  else CK(launch_points1d(ctx->d.k, ctx->g, ctx->d.ax, ctx->d.bx, d_xy, ctx->stream), "quad_points");
  ctx->launches += 1;
  return CDG_OK;
}

cdg_status cdg_project_ic(cdg_ctx* ctx, const double* d_vals, double* d_u) {
  if (!ctx || !d_vals || !d_u) return fail(ctx, CDG_EINVAL, "project_ic: null pointer");
  if (ctx->gen2) CK(launch_project2k(ctx->sys, ctx->d.k, basis_of(ctx), ctx->g, d_vals, d_u, ctx->stream), "project_ic");
  else if (ctx->d.dim == 2) CK(launch_project2d(ctx->sys, ctx->g, d_vals, d_u, ctx->stream), "project_ic");
  else CK(launch_project1d(ctx->sys, ctx->d.k, ctx->g, d_vals, d_u, ctx->stream), "project_ic");
  ctx->launches += 1;
  return CDG_OK;
}

// One stage kernel: out = sum_m cb.c[m] cb.u[m] + cb.ct tau L(uin) (rhs_only:
// out = L(uin)).  The 2D kernel takes the two-state form
// ca un + cb (uin + tau L(uin)); other forms are refused there.
static cudaError_t run_stage(cdg_ctx* ctx, int rhs_only, const double* uin, const StageComb& cb, double* out,
                             const double* dt) {
  cudaError_t e;
  if (ctx->gen2) {
    ctx->launches += 1;
    prof_mark(ctx, PROF_STAGE, 0);
    e = launch_stage2k(ctx->sys, ctx->bc, ctx->d.k, basis_of(ctx), ctx->g, rhs_only, uin, cb, out, dt, ctx->partials,
                       ctx->stream);
  } else if (ctx->d.dim == 2) {
    const double* un = nullptr;
    double ca = 0.0, cw = 1.0;
    if (cb.n == 2 && cb.u[1] == uin && cb.c[1] == cb.ct) {
      un = cb.u[0];
      ca = cb.c[0];
      cw = cb.ct;
    } else if (!(cb.n == 1 && cb.u[0] == uin && cb.c[0] == 1.0 && cb.ct == 1.0)) {
      return cudaErrorNotSupported;
    }
    ctx->launches += 1;
    prof_mark(ctx, PROF_STAGE, 0);
    e = launch_stage2d(ctx->sys, ctx->bc, ctx->g, rhs_only, uin, un, out, dt, ca, cw, ctx->partials, ctx->stream);
  } else {
    ctx->launches += 1;
    prof_mark(ctx, PROF_STAGE, 0);
    e = launch_stage1d(ctx->sys, ctx->bc, ctx->d.k, ctx->g, rhs_only, uin, cb, out, dt, ctx->partials, ctx->stream);
  }
  prof_mark(ctx, PROF_STAGE, 1);
  return e;
}

static StageComb comb1(const double* u0, double c0, double ct) {
  StageComb cb{};
  cb.u[0] = u0;
  cb.c[0] = c0;
  cb.n = 1;
  cb.ct = ct;
  return cb;
}

static StageComb comb2(const double* u0, double c0, const double* u1, double c1, double ct) {
  StageComb cb = comb1(u0, c0, ct);
  cb.u[1] = u1;
  cb.c[1] = c1;
  cb.n = 2;
  return cb;
}

// sigma from the partials of the last stage kernel, then the OE kernel (1D:
// both in one launch)
static cudaError_t run_oe(cdg_ctx* ctx, const double* uh, double* usig, double* delta) {
  if (ctx->d.dim == 1) {
    ctx->launches += 1;
    prof_mark(ctx, PROF_OE, 0);
    cudaError_t e = launch_oe1d_sig(ctx->sys, ctx->bc, ctx->d.k, ctx->g, uh, usig, ctx->dt, ctx->partials, ctx->nblk,
                                    ctx->sn, ctx->sigma, ctx->avg, delta, ctx->status, ctx->stream);
    prof_mark(ctx, PROF_OE, 1);
    return e;
  }
  cudaError_t e = launch_sigma(ctx->partials, ctx->nblk, ctx->F, ctx->sn, ctx->sigma, ctx->avg, ctx->stream);
  if (e != cudaSuccess) return e;
  ctx->launches += 2;
  prof_mark(ctx, PROF_OE, 0);
  if (ctx->gen2)
    e = launch_oe2k(ctx->sys, ctx->bc, ctx->d.k, basis_of(ctx), ctx->g, uh, usig, ctx->dt, ctx->sigma, delta,
                    ctx->status, ctx->stream);
  else if (ctx->d.dim == 2)
    e = launch_oe2d(ctx->sys, ctx->bc, ctx->g, uh, usig, ctx->dt, ctx->sigma, delta, ctx->status, ctx->stream);
  else
    e = launch_oe1d(ctx->sys, ctx->bc, ctx->d.k, ctx->g, uh, usig, ctx->dt, ctx->sigma, delta, ctx->status,
                    ctx->stream);
  prof_mark(ctx, PROF_OE, 1);
  return e;
}

cdg_status cdg_rhs(cdg_ctx* ctx, const double* d_u, double tau_max, double* d_L) {
  if (!ctx || !d_u || !d_L) return fail(ctx, CDG_EINVAL, "rhs: null pointer");
  if (d_u == d_L) return fail(ctx, CDG_EINVAL, "rhs: d_L aliases d_u");
  if (!(tau_max > 0.0)) return fail(ctx, CDG_EINVAL, "rhs: tau_max must be > 0");
  CK(launch_set2(ctx->rhs_dt, 0.0, tau_max, ctx->stream), "rhs");
  ctx->launches += 1;
  CK(run_stage(ctx, 1, d_u, comb1(d_u, 1.0, 1.0), d_L, ctx->rhs_dt), "rhs");
  return CDG_OK;
}

static cudaError_t launch_dt(cdg_ctx* ctx, const double* d_u, double T_end) {
  ctx->launches += ctx->d.dim == 1 ? 1 : 2;  // 1D: the last block sets tau
  if (ctx->gen2)
    return launch_dt2k(ctx->sys, ctx->d.k, basis_of(ctx), ctx->g, d_u, ctx->wave_partial, ctx->wave_blk, T_end,
                       ctx->dt, ctx->time, ctx->status, ctx->stream);
  if (ctx->d.dim == 2)
    return launch_dt2d(ctx->sys, ctx->g, d_u, ctx->wave_partial, ctx->wave_blk, T_end, ctx->dt, ctx->time, ctx->status,
                       ctx->stream);
  return launch_dt1d(ctx->sys, ctx->d.k, ctx->g, d_u, ctx->wave_partial, ctx->wave_blk, T_end, ctx->dt, ctx->time, ctx->status,
                     ctx->stream);
}

cdg_status cdg_compute_dt(cdg_ctx* ctx, const double* d_u, double t, double T_end) {
  if (!ctx || !d_u) return fail(ctx, CDG_EINVAL, "compute_dt: null pointer");
  CK(launch_set2(ctx->time, t, 0.0, ctx->stream), "compute_dt");
  ctx->launches += 1;
  CK(launch_dt(ctx, d_u, T_end), "compute_dt");
  return CDG_OK;
}

cdg_status cdg_set_dt(cdg_ctx* ctx, double tau, double tau_max) {
  if (!ctx) return CDG_EINVAL;
  if (!(tau >= 0.0) || !(tau_max > 0.0)) return fail(ctx, CDG_EINVAL, "set_dt: need tau >= 0, tau_max > 0");
  CK(launch_set2(ctx->dt, tau, tau_max, ctx->stream), "set_dt");
  ctx->launches += 1;
  return CDG_OK;
}

cdg_status cdg_get_dt(cdg_ctx* ctx, double* tau, double* tau_max) {
  if (!ctx || !tau || !tau_max) return CDG_EINVAL;
  double h[2];
  CK(cudaMemcpyAsync(h, ctx->dt, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "get_dt");
  CK(cudaStreamSynchronize(ctx->stream), "get_dt");
  *tau = h[0];
  *tau_max = h[1];
  return CDG_OK;
}

cdg_status cdg_get_time(cdg_ctx* ctx, double* t) {
  if (!ctx || !t) return CDG_EINVAL;
  CK(cudaMemcpyAsync(t, ctx->time, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "get_time");
  CK(cudaStreamSynchronize(ctx->stream), "get_time");
  return CDG_OK;
}

static int n_stages(int rk) { return rk == CDG_RK_RK4 ? 4 : rk; }

// Shu-Osher form of the context's RK method (Eq. (eq:RKCDG) with SSP-RK2/3;
// classical RK4 for the 1D convergence study of Table 2).  U[0] = u^n, U[l] =
// the OE-damped stage l; stage l evaluates L at U[l].
static StageComb rk_comb(int rk, int l, const double* const* U) {
  if (rk == CDG_RK_SSP2) return l == 0 ? comb1(U[0], 1.0, 1.0) : comb2(U[0], 0.5, U[1], 0.5, 0.5);
  if (rk == CDG_RK_SSP3) {
    // c_l un + (1 - c_l)(...), c = (0, 3/4, 1/3), the weights written as 1 - c_l
    // so that every SSP-RK3 driver (single, batched, adjoint) rounds alike
    if (l == 0) return comb1(U[0], 1.0, 1.0);
    const double c = l == 1 ? 0.75 : 1.0 / 3.0;
    return comb2(U[0], c, U[l], 1.0 - c, 1.0 - c);
  }
  if (rk == CDG_RK_RK4) {
    if (l < 3) return comb1(U[0], 1.0, l == 2 ? 1.0 : 0.5);
    StageComb cb = comb2(U[0], -1.0 / 3.0, U[1], 1.0 / 3.0, 1.0 / 6.0);
    cb.u[2] = U[2];
    cb.c[2] = 2.0 / 3.0;
    cb.u[3] = U[3];
    cb.c[3] = 1.0 / 3.0;
    cb.n = 4;
    return cb;
  }
  return comb1(U[0], 1.0, 1.0);
}

cdg_status cdg_rk_stage(cdg_ctx* ctx, int l, const double* d_un, const double* d_ul, double* d_out) {
  if (!ctx || !d_ul || !d_out) return fail(ctx, CDG_EINVAL, "rk_stage: null pointer");
  const int rk = ctx->d.rk, nst = n_stages(rk);
  if (l < 0 || l >= nst) return fail(ctx, CDG_EINVAL, "rk_stage: stage index out of range");
  if (rk == CDG_RK_RK4 && l == 3) return fail(ctx, CDG_EINVAL, "rk_stage: RK4's last stage needs cdg_rk_combine");
  if (l > 0 && !d_un) return fail(ctx, CDG_EINVAL, "rk_stage: d_un is null");
  if (d_out == d_ul || (l > 0 && d_out == d_un)) return fail(ctx, CDG_EINVAL, "rk_stage: output aliases an input");
  const double* U[4] = {l == 0 ? d_ul : d_un, d_ul, d_ul, d_ul};
  CK(run_stage(ctx, 0, d_ul, rk_comb(rk, l, U), d_out, ctx->dt), "rk_stage");
  return CDG_OK;
}

cdg_status cdg_rk_combine(cdg_ctx* ctx, const double* d_ul, int n, const double* const* d_terms, const double* coef,
                          double ct, double* d_out) {
  if (!ctx || !d_ul || !d_out || !d_terms || !coef) return fail(ctx, CDG_EINVAL, "rk_combine: null pointer");
  if (n < 1 || n > 4) return fail(ctx, CDG_EINVAL, "rk_combine: n must be 1..4");
  if (d_out == d_ul) return fail(ctx, CDG_EINVAL, "rk_combine: output aliases d_ul");
  StageComb cb{};
  for (int m = 0; m < n; ++m) {
    if (!d_terms[m]) return fail(ctx, CDG_EINVAL, "rk_combine: null term");
    if (d_terms[m] == d_out) return fail(ctx, CDG_EINVAL, "rk_combine: output aliases a term");
    cb.u[m] = d_terms[m];
    cb.c[m] = coef[m];
  }
  cb.n = n;
  cb.ct = ct;
  cudaError_t e = run_stage(ctx, 0, d_ul, cb, d_out, ctx->dt);
  if (e == cudaErrorNotSupported)
    return fail(ctx, CDG_EUNSUPPORTED, "rk_combine: the tiled Q^2 stage kernel takes only the two-state form");
  CK(e, "rk_combine");
  return CDG_OK;
}

cdg_status cdg_oe_damp(cdg_ctx* ctx, const double* d_uh, double* d_usig) {
  if (!ctx || !d_uh || !d_usig) return fail(ctx, CDG_EINVAL, "oe_damp: null pointer");
  if (d_uh == d_usig) return fail(ctx, CDG_EINVAL, "oe_damp: d_usig aliases d_uh");
  // sigma partials of d_uh: a stage with tau = 0 copies d_uh into scratch and
  // leaves the partials of d_uh behind (this standalone entry point is not on
  // the cdg_step path, where the partials come from the stage that made u_h)
  CK(launch_set2(ctx->rhs_dt, 0.0, 1.0, ctx->stream), "oe_damp");
  ctx->launches += 1;
  CK(run_stage(ctx, 0, d_uh, comb1(d_uh, 1.0, 1.0), ctx->buf_a == d_uh ? ctx->buf_b : ctx->buf_a, ctx->rhs_dt),
     "oe_damp");
  if (ctx->d.k == 0) return CDG_OK;
  CK(run_oe(ctx, d_uh, d_usig, nullptr), "oe_damp");
  return CDG_OK;
}

cdg_status cdg_oe_coefficients(cdg_ctx* ctx, const double* d_uh, double* d_delta, double* d_sigma) {
  if (!ctx || !d_uh) return fail(ctx, CDG_EINVAL, "oe_coefficients: null pointer");
  CK(launch_set2(ctx->rhs_dt, 0.0, 1.0, ctx->stream), "oe_coefficients");
  ctx->launches += 1;
  CK(run_stage(ctx, 0, d_uh, comb1(d_uh, 1.0, 1.0), ctx->buf_a == d_uh ? ctx->buf_b : ctx->buf_a, ctx->rhs_dt),
     "oe_coefficients");
  if (d_delta) CK(run_oe(ctx, d_uh, nullptr, d_delta), "oe_coefficients");
  else {
    CK(launch_sigma(ctx->partials, ctx->nblk, ctx->F, ctx->sn, ctx->sigma, ctx->avg, ctx->stream),
       "oe_coefficients");
    ctx->launches += 1;
  }
  if (d_sigma)
    CK(cudaMemcpyAsync(d_sigma, ctx->sigma, (size_t)2 * ctx->F * sizeof(double), cudaMemcpyDeviceToDevice,
                       ctx->stream),
       "oe_coefficients");
  return CDG_OK;
}

// The kernels of one time step on d_u (no host synchronisation): wave speed
// and tau, then every stage of the context's RK method with the OE step.
static cudaError_t enqueue_step(cdg_ctx* ctx, double* d_u, double T_end) {
  const int rk = ctx->d.rk, nst = n_stages(rk);
  // U[l]: the damped stage values.  u_h of every stage -> buf_a; u_sigma ->
  // buf_b (RK4: stages 1..3 -> buf_b, buf_c, buf_d), the last one back into d_u.
  const double* U[4] = {d_u, ctx->buf_b, rk == CDG_RK_RK4 ? ctx->buf_c : ctx->buf_b,
                        rk == CDG_RK_RK4 ? ctx->buf_d : ctx->buf_b};
  cudaError_t e = launch_dt(ctx, d_u, T_end);
  if (e != cudaSuccess) return e;
  for (int l = 0; l < nst; ++l) {
    if ((e = run_stage(ctx, 0, U[l], rk_comb(rk, l, U), ctx->buf_a, ctx->dt)) != cudaSuccess) return e;
    double* dst = (l == nst - 1) ? d_u : (double*)U[l + 1];
    if (ctx->d.oe) e = run_oe(ctx, ctx->buf_a, dst, nullptr);
    else e = cudaMemcpyAsync(dst, ctx->buf_a, ctx->numel * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cdg_status cdg_step_async(cdg_ctx* ctx, double* d_u, double t, double T_end, int nsteps) {
  if (!ctx || !d_u) return fail(ctx, CDG_EINVAL, "step: null pointer");
  if (nsteps < 0) return fail(ctx, CDG_EINVAL, "step: nsteps < 0");
  if (d_u == ctx->buf_a || d_u == ctx->buf_b || d_u == ctx->buf_c || d_u == ctx->buf_d)
    return fail(ctx, CDG_EINVAL, "step: d_u is a context buffer");
  CK(launch_set2(ctx->time, t, 0.0, ctx->stream), "step");
  ctx->launches += 1;
  for (int s = 0; s < nsteps; ++s) CK(enqueue_step(ctx, d_u, T_end), "step");
  return CDG_OK;
}

cdg_status cdg_step_graph(cdg_ctx* ctx, double* d_u, double t, double T_end, int nsteps) {
  if (!ctx || !d_u) return fail(ctx, CDG_EINVAL, "step_graph: null pointer");
  if (nsteps < 0) return fail(ctx, CDG_EINVAL, "step_graph: nsteps < 0");
  if (!ctx->stream) return fail(ctx, CDG_EINVAL, "step_graph: the context needs its own stream");
  if (d_u == ctx->buf_a || d_u == ctx->buf_b || d_u == ctx->buf_c || d_u == ctx->buf_d)
    return fail(ctx, CDG_EINVAL, "step_graph: d_u is a context buffer");
  if (!ctx->graph_exec || ctx->graph_u != d_u || ctx->graph_tend != T_end) {
    if (ctx->graph_exec) {
      CK(cudaStreamSynchronize(ctx->stream), "step_graph");
      cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const long long l0 = ctx->launches;
    ctx->capturing = 1;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    cudaError_t e2 = e == cudaSuccess ? enqueue_step(ctx, d_u, T_end) : e;
    if (e == cudaSuccess) e = cudaStreamEndCapture(ctx->stream, &graph);
    ctx->capturing = 0;
    const long long per_step = ctx->launches - l0;  // the kernels of one captured step
    ctx->launches = l0;
    if (e2 != cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->graph_exec = nullptr;
      return cuda_fail(ctx, e, "step_graph: capture");
    }
    ctx->graph_u = d_u;
    ctx->graph_tend = T_end;
    ctx->graph_launches = per_step;
  }
  CK(launch_set2(ctx->time, t, 0.0, ctx->stream), "step_graph");
  ctx->launches += 1;
  for (int s = 0; s < nsteps; ++s) CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream), "step_graph: launch");
  ctx->launches += ctx->graph_launches * nsteps;
  return CDG_OK;
}

cdg_status cdg_check_status(cdg_ctx* ctx) {
  if (!ctx) return CDG_EINVAL;
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "check_status");
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "check_status");
  CK(cudaStreamSynchronize(ctx->stream), "check_status");
  if (h & ST_TIMEOUT) return fail(ctx, CDG_ETIMEOUT, "a grid barrier of the persistent step ran out of time");
  if (h & ST_NONPHYSICAL) return fail(ctx, CDG_ENONPHYSICAL, "non-physical cell average (rho <= 0 or p <= 0)");
  return CDG_OK;
}

cdg_status cdg_set_wait(cdg_ctx* ctx, double limit_s, int withheld) {
  if (!ctx) return CDG_EINVAL;
  if (!(limit_s > 0.0) || limit_s > 3600.0 || withheld < 0) return fail(ctx, CDG_EINVAL, "set_wait: bad arguments");
  ctx->wait_s = limit_s;
  ctx->withhold = withheld;
  return CDG_OK;
}

cdg_status cdg_step_persistent(cdg_ctx* ctx, double* d_u, double t, double T_end, int nsteps) {
  if (!ctx || !d_u) return fail(ctx, CDG_EINVAL, "step_persistent: null pointer");
  if (nsteps < 0) return fail(ctx, CDG_EINVAL, "step_persistent: nsteps < 0");
  if (ctx->d.dim != 1) return fail(ctx, CDG_EUNSUPPORTED, "step_persistent: 1D meshes only");
  if (d_u == ctx->buf_a || d_u == ctx->buf_b || d_u == ctx->buf_c || d_u == ctx->buf_d)
    return fail(ctx, CDG_EINVAL, "step_persistent: d_u is a context buffer");
  if (!ctx->p_bar) {
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev), "step_persistent");
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "step_persistent");
    CK(persist_grid_1d(ctx->sys, ctx->bc, ctx->d.k, ctx->g, nsm, &ctx->p_grid), "step_persistent");
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)ctx->p_grid * sizeof(double)) != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(ctx, CDG_ENOMEM, "step_persistent: scratch");
    }
    ctx->p_wpart = (double*)p;
    if (cudaMalloc(&p, 2 * sizeof(unsigned long long)) != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(ctx, CDG_ENOMEM, "step_persistent: scratch");
    }
    ctx->p_bar = (unsigned long long*)p;
  }
  CK(launch_set2(ctx->time, t, 0.0, ctx->stream), "step_persistent");
  ctx->launches += 1;
  if (nsteps == 0) return CDG_OK;
  const int rk = ctx->d.rk, nst = n_stages(rk);
  const double* U[4] = {d_u, ctx->buf_b, rk == CDG_RK_RK4 ? ctx->buf_c : ctx->buf_b,
                        rk == CDG_RK_RK4 ? ctx->buf_d : ctx->buf_b};
  Persist1 a = {};
  for (int l = 0; l < nst; ++l) {
    a.cb[l] = rk_comb(rk, l, U);
    a.uin[l] = U[l];
    a.dst[l] = l == nst - 1 ? d_u : (double*)U[l + 1];
  }
  a.ua = ctx->buf_a;
  a.dt = ctx->dt;
  a.time = ctx->time;
  a.sigma = ctx->sigma;
  a.avg = ctx->avg;
  a.partials = ctx->partials;
  a.wpart = ctx->p_wpart;
  a.status = ctx->status;
  a.nst = nst;
  a.oe = ctx->d.oe;
  a.nsteps = nsteps;
  a.T_end = T_end;
  a.nblk = ctx->nblk;
  a.sn = ctx->sn;
  a.bar = ctx->p_bar;
  a.expected = (unsigned long long)ctx->p_grid + (unsigned long long)ctx->withhold;
  a.limit_ns = (unsigned long long)(ctx->wait_s * 1e9);
  CK(launch_persist1d(ctx->sys, ctx->bc, ctx->d.k, ctx->g, a, ctx->p_grid, ctx->stream), "step_persistent");
  ctx->launches += 1;
  return CDG_OK;
}

cdg_status cdg_profile_begin(cdg_ctx* ctx, int max_launches) {
  if (!ctx || max_launches < 1) return CDG_EINVAL;
  prof_release(ctx);
  for (int k = 0; k < 2; ++k) {
    ctx->prof_ev[k] = (cudaEvent_t*)calloc((size_t)2 * max_launches, sizeof(cudaEvent_t));
    if (!ctx->prof_ev[k]) {
      prof_release(ctx);
      return CDG_ENOMEM;
    }
  }
  ctx->prof_cap = max_launches;
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < 2 * max_launches; ++q) {
      cudaError_t e = cudaEventCreate(&ctx->prof_ev[k][q]);
      if (e != cudaSuccess) {
        prof_release(ctx);
        return cuda_fail(ctx, e, "profile_begin");
      }
    }
  ctx->prof_n[0] = ctx->prof_n[1] = 0;
  ctx->prof_on = 1;
  return CDG_OK;
}

cdg_status cdg_profile_end(cdg_ctx* ctx, double* ms_stage, long long* n_stage, double* ms_oe, long long* n_oe) {
  if (!ctx || !ctx->prof_on) return CDG_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream), "profile_end");
  double tot[2] = {0.0, 0.0};
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < ctx->prof_n[k]; ++q) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ctx->prof_ev[k][2 * q], ctx->prof_ev[k][2 * q + 1]), "profile_end");
      tot[k] += ms;
    }
  if (ms_stage) *ms_stage = tot[0];
  if (n_stage) *n_stage = ctx->prof_n[0];
  if (ms_oe) *ms_oe = tot[1];
  if (n_oe) *n_oe = ctx->prof_n[1];
  prof_release(ctx);
  return CDG_OK;
}

}  // extern "C"

template <int OP>
__global__ void k_math_eval(const double* __restrict__ x, size_t n, double* __restrict__ y) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = OP == CDG_MATH_RCP ? rcp_pos(x[t]) : sqrt_pos(x[t]);
}

extern "C" {

cdg_status cdg_math_eval(int op, const double* d_x, size_t n, double* d_y, void* stream) {
  if (op != CDG_MATH_RCP && op != CDG_MATH_SQRT) return CDG_EINVAL;
  if (n == 0) return CDG_OK;
  if (!d_x || !d_y) return CDG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = (n + 255) / 256;
  const unsigned blocks = (unsigned)(need < 152 * 16 ? need : 152 * 16);
  if (op == CDG_MATH_RCP) k_math_eval<CDG_MATH_RCP><<<blocks, 256, 0, st>>>(d_x, n, d_y);
  else k_math_eval<CDG_MATH_SQRT><<<blocks, 256, 0, st>>>(d_x, n, d_y);
  return cudaGetLastError() == cudaSuccess ? CDG_OK : CDG_ECUDA;
}

cdg_status cdg_step(cdg_ctx* ctx, double* d_u, double t, double T_end, int nsteps) {
  cdg_status s = cdg_step_async(ctx, d_u, t, T_end, nsteps);
  if (s != CDG_OK) return s;
  return cdg_check_status(ctx);
}

}  // extern "C"
