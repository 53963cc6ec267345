// oecdg_kernels.h -- internal launch functions of the OECDG CUDA path.
#pragma once
#include <cuda_runtime.h>
#include "oecdg_common.cuh"

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
cudaError_t launch_dt1d(int sys, int k, const Geo& g, const double* u, double* partial, int nblk, double T_end,
                        double* dt, double* time, int* status, cudaStream_t st);
cudaError_t launch_points1d(int k, const Geo& g, double ax, double* x, cudaStream_t st);
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
cudaError_t launch_points2k(int k, const Geo& g, double ax, double ay, double* xy, cudaStream_t st);
cudaError_t launch_project2k(int sys, int k, int basis, const Geo& g, const double* vals, double* u,
                             cudaStream_t st);

// shared
cudaError_t launch_sigma(const double* partials, long long nblk, int F, long long ncell, double* sigma, double* avg,
                         cudaStream_t st);
cudaError_t launch_set2(double* p, double a, double b, cudaStream_t st);
cudaError_t launch_dt_final(const double* partial, int nblk, double hx, double hy, int dim, double cfl, double T_end,
                            double* dt, double* time, cudaStream_t st);

}  // namespace oecdg
