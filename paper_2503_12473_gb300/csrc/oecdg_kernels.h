// oecdg_kernels.h -- internal launch functions of the OECDG CUDA path.
#pragma once
#include <cuda_runtime.h>
#include "../../include/oecdg.h"
#include "oecdg_common.cuh"
#include "oecdg_persist.cuh"

namespace oecdg {

// 2D Q^2
long long partial_blocks_2d(const Geo& g);
int wave_blocks_2d(const Geo& g);
cudaError_t launch_stage2d(int sys, int bc, const Geo& g, int rhs_only, const double* uin, const double* un,
                           double* out, const double* dt, double ca, double cb, double* partials, cudaStream_t st);
cudaError_t launch_oe2d(int sys, int bc, const Geo& g, const double* uh, double* usig, const double* dt,
                        const double* sigma, double* delta, int* status, cudaStream_t st);
cudaError_t launch_dt2d(int sys, const Geo& g, const double* u, double* partial, int nblk, double T_end, double* dt,
                        double* time, int* status, cudaStream_t st);
cudaError_t launch_points2d(const Geo& g, double ax, double ay, double* xy, cudaStream_t st);
cudaError_t launch_project2d(int sys, const Geo& g, const double* vals, double* u, cudaStream_t st);

// One Shu-Osher stage: out = sum_{m < n} c[m] u[m] + ct tau L(u_l).
struct StageComb {
  const double* u[4];
  double c[4];
  int n;
  double ct;
};

// 1D P^k, k in {1, 2, 3}
long long partial_blocks_1d(const Geo& g);
int wave_blocks_1d(const Geo& g);
cudaError_t launch_stage1d(int sys, int bc, int k, const Geo& g, int rhs_only, const double* uin,
                           const StageComb& cb, double* out, const double* dt, double* partials, cudaStream_t st);
cudaError_t launch_oe1d(int sys, int bc, int k, const Geo& g, const double* uh, double* usig, const double* dt,
                        const double* sigma, double* delta, int* status, cudaStream_t st);
// sigma from the stage partials and the OE step in one launch (1D)
cudaError_t launch_oe1d_sig(int sys, int bc, int k, const Geo& g, const double* uh, double* usig, const double* dt,
                            const double* partials, long long nblk, const SigmaNorm& sn, double* sigma, double* avg,
                            double* delta, int* status, cudaStream_t st);
cudaError_t launch_dt1d(int sys, int k, const Geo& g, const double* u, double* partial, int nblk, double T_end,
                        double* dt, double* time, int* status, cudaStream_t st);
cudaError_t launch_points1d(int k, const Geo& g, double ax, double bx, double* x, cudaStream_t st);
cudaError_t launch_project1d(int sys, int k, const Geo& g, const double* vals, double* u, cudaStream_t st);

// Persistent 1D step: nsteps steps of Eq. (eq:RKCDG) in one cooperative launch
// (oecdg_1d.cu).  Stage l evaluates L at uin[l], combines cb[l] into ua, and
// the OE step (or a copy without OE) writes dst[l].
struct Persist1 {
  StageComb cb[4];
  const double* uin[4];
  double* dst[4];
  double* ua;
  double *dt, *time, *sigma, *avg, *partials, *wpart;
  int* status;
  int nst, oe, nsteps;
  double T_end;
  long long nblk;               // stage blocks per mesh (partials layout)
  SigmaNorm sn;                 // sigma normalisation
  unsigned long long* bar;      // [barrier arrivals, last-block tickets], zeroed before the launch
  unsigned long long expected;  // arrivals per barrier (the grid, plus withheld ones in a test)
  unsigned long long limit_ns;  // bounded wait of every barrier
};
// blocks of the persistent grid: as many as fit on the device, at most the tiles
cudaError_t persist_grid_1d(int sys, int bc, int k, const Geo& g, int nsm, long long* grid);
cudaError_t launch_persist1d(int sys, int bc, int k, const Geo& g, const Persist1& a, long long grid,
                             cudaStream_t st);

// 2D Q^k / P^k, k in {1, 2, 3}: every configuration outside the tiled Q^2 path
long long partial_blocks_2k(const Geo& g);
int modes_2k(int k, int basis);
cudaError_t launch_stage2k(int sys, int bc, int k, int basis, const Geo& g, int rhs_only, const double* uin,
                           const StageComb& cb, double* out, const double* dt, double* partials, cudaStream_t st);
cudaError_t launch_oe2k(int sys, int bc, int k, int basis, const Geo& g, const double* uh, double* usig,
                        const double* dt, const double* sigma, double* delta, int* status, cudaStream_t st);
cudaError_t launch_dt2k(int sys, int k, int basis, const Geo& g, const double* u, double* partial, int nblk,
                        double T_end, double* dt, double* time, int* status, cudaStream_t st);
cudaError_t launch_points2k(int k, const Geo& g, double ax, double ay, double bx, double by, double* xy,
                            cudaStream_t st);
cudaError_t launch_project2k(int sys, int k, int basis, const Geo& g, const double* vals, double* u,
                             cudaStream_t st);

// shared
cudaError_t launch_sigma(const double* partials, long long nblk, int F, const SigmaNorm& sn, double* sigma,
                         double* avg, cudaStream_t st);

// Side conditions of a description: 0 if valid (per direction periodic on both
// sides or on neither; reflective walls for Euler only), else 1.
inline int invalid_sides(const cdg_mesh_desc& d) {
  for (int dir = 0; dir < d.dim; ++dir) {
    const int lo = d.bc[2 * dir], hi = d.bc[2 * dir + 1];
    if (lo < CDG_PERIODIC || lo > CDG_REFLECTIVE || hi < CDG_PERIODIC || hi > CDG_REFLECTIVE) return 1;
    if ((lo == CDG_PERIODIC) != (hi == CDG_PERIODIC)) return 1;
    if ((lo == CDG_REFLECTIVE || hi == CDG_REFLECTIVE) && d.system != CDG_EULER) return 1;
  }
  return 0;
}

// The condition shared by every side that matters (x only in 1D) when it is
// periodic or transmissive, else -1 (mixed sides or a wall).
inline int uniform_side_bc(const cdg_mesh_desc& d) {
  const int b = d.bc[0];
  if (b != CDG_PERIODIC && b != CDG_TRANSMISSIVE) return -1;
  for (int s = 1; s < 2 * d.dim; ++s)
    if (d.bc[s] != b) return -1;
  return b;
}

// Padded layout, per-side conditions and plane of a description, into g.
inline void geo_sides(const cdg_mesh_desc& d, Geo& g) {
  const int ny = d.dim == 2 ? d.ny : 1;
  g.nxs = d.nx + (d.bc[0] == CDG_REFLECTIVE ? 1 : 0);
  g.nys = d.dim == 2 ? ny + (d.bc[2] == CDG_REFLECTIVE ? 1 : 0) : 1;
  for (int s = 0; s < 4; ++s) g.bcs[s] = (d.dim == 2 || s < 2) ? d.bc[s] : SIDE_PERIODIC;
  g.plane = (long long)g.nxs * g.nys;
}

// Sigma normalisation of a description (the dual mesh's wall-centred cells
// count half; the normal momentum beside a wall averages to 0).
inline SigmaNorm sigma_norm(const cdg_mesh_desc& d, const Geo& g) {
  SigmaNorm sn;
  const int xl = d.bc[0] == CDG_REFLECTIVE, xh = d.bc[1] == CDG_REFLECTIVE;
  const int yl = d.dim == 2 && d.bc[2] == CDG_REFLECTIVE, yh = d.dim == 2 && d.bc[3] == CDG_REFLECTIVE;
  sn.ncell[0] = (double)g.nx * (d.dim == 2 ? g.ny : 1);
  sn.ncell[1] = (g.nxs - 0.5 * (xl + xh)) * (d.dim == 2 ? (g.nys - 0.5 * (yl + yh)) : 1.0);
  sn.odd = 0;
  if (d.system == CDG_EULER) {
    if (xl || xh) sn.odd |= 1 << 1;
    if (yl || yh) sn.odd |= 1 << 2;
  }
  return sn;
}
cudaError_t launch_set2(double* p, double a, double b, cudaStream_t st);
cudaError_t launch_dt_final(const double* partial, int nblk, double hx, double hy, int dim, double cfl, double T_end,
                            double* dt, double* time, cudaStream_t st);

}  // namespace oecdg
