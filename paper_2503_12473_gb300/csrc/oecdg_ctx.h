// oecdg_ctx.h -- the context behind the C-ABI handle cdg_ctx (internal).
#pragma once
#include <cuda_runtime.h>

#include "../../include/oecdg.h"
#include "oecdg_common.cuh"
#include "oecdg_persist.cuh"

using oecdg::Geo;

struct AdjScratch;

struct cdg_ctx {
  cdg_mesh_desc d;
  Geo g;
  cudaStream_t stream;
  int F, M;
  size_t numel;
  long long nblk;        // stage-kernel blocks per mesh (sigma partials)
  int wave_blk;          // blocks of the wave-speed reduction
  double* buf_a;         // scratch state (u_h)
  double* buf_b;         // scratch state (u_sigma)
  double* buf_c;         // RK4 only: u^(2)
  double* buf_d;         // RK4 only: u^(3)
  int sys;               // SYS_ADV / SYS_BURGERS / SYS_EULER
  int bc;                // BC_PERIODIC / BC_TRANSMISSIVE
  int gen2;              // 2D configuration served by the degree-generic kernels
  oecdg::SigmaNorm sn;   // sigma normalisation (walls: weighted counts, odd fields)
  double* partials;      // [2][nblk][F][3]
  double* wave_partial;  // [wave_blk][2]
  double* dt;            // [tau, tau_max]
  double* rhs_dt;        // [0, tau_max] for cdg_rhs
  double* time;          // [t, unused]
  double* sigma;         // [2][F]
  double* avg;           // [2][F]
  int* status;           // status bits
  long long launches;
  // cdg_step_graph: one captured step, valid for (graph_u, graph_tend)
  cudaGraphExec_t graph_exec;
  double* graph_u;
  double graph_tend;
  long long graph_launches;  // kernels in one captured step
  int capturing;             // no profiling events while capturing
  // optional per-kernel timing (cdg_profile_begin / cdg_profile_end)
  int prof_on;
  int prof_cap;
  int prof_n[2];
  cudaEvent_t* prof_ev[2];  // [class][2 * cap]: start, stop
  struct AdjScratch* adj;   // adjoint buffers, allocated by the first cdg_step_adjoint
  // persistent step (cdg_step_persistent): allocated by its first call
  double* p_wpart;          // one wave-speed partial per persistent block
  unsigned long long* p_bar;  // grid-barrier arrival counter
  long long p_grid;         // blocks of the persistent grid
  double wait_s;            // bounded wait of every grid barrier (cdg_set_wait)
  int withhold;             // test hook: arrivals that never come
  char err[256];
};


// release the adjoint scratch of a context (oecdg_adjoint.cu)
void adj_release(cdg_ctx* c);
