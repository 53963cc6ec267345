// oecdg_batch.cu -- many independent 2D Q^2 OECDG problems of uneven mesh
// sizes advanced together (arXiv:2503.12473 applied to a batch of meshes).
//
// Every phase of a step is ONE launch over all instances: the blocks of the
// stage and OE kernels are laid out instance after instance (2 meshes x tiles
// of 32 x R cells each), and a block finds its instance by binary search over
// the instances' first-block offsets.  Reductions (sigma, wave speed) and the
// time step are kept per instance, so each instance evolves exactly as it
// would alone (bitwise, for the same tile height R = 4 as the single-mesh
// kernels).  A step is 11 launches whatever the number of instances, and
// cdg_batch_step can capture the launches of nsteps steps in a CUDA graph.
// The tile height R (2, 4 or 8 rows) is picked by cdg_batch_autotune.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/oecdg.h"
#include "oecdg_2d_body.cuh"
#include "oecdg_kernels.h"

namespace oecdg {

struct BatchInst {
  Geo g;
  double* u;      // caller's state (u^n, and u^{n+1} after the last stage)
  double* a;      // scratch u_h
  double* b;      // scratch u_sigma
  double* part;   // sigma partials [2][tiles][F][3]
  double* wpart;  // wave-speed partials [WB][2]
  double* dt;     // [tau, tau_max]
  double* time;   // [t, unused]
  double* sigma;  // [2][F]
  double* avg;    // [2][F]
  long long blk0; // first block of this instance
  int tx, ty;     // tiles per direction (per mesh)
};

constexpr int WB = 32;  // wave-speed blocks per instance

__device__ __forceinline__ int find_instance(const BatchInst* __restrict__ I, int n, long long blk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (I[mid].blk0 <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int SYS, int BC, int R>
__global__ void __launch_bounds__(32 * R) k_bstage(const BatchInst* __restrict__ I, int n, int l, double ca,
                                                   double cb) {
  constexpr int F = Fields<SYS>::F;
  const long long blk = blockIdx.x;
  const int q = find_instance(I, n, blk);
  const BatchInst& in = I[q];
  const int tiles = in.tx * in.ty;
  const int local = (int)(blk - in.blk0);
  const int mesh = local / tiles, t = local - mesh * tiles;
  const int i = (t % in.tx) * 32 + (threadIdx.x & 31);
  const int j = (t / in.tx) * R + (threadIdx.x >> 5);
  stage_cell2d<SYS, BC, MODE_STAGE>(in.g, l == 0 ? in.u : in.b, in.u, in.a, in.dt, ca, cb,
                                    in.part + ((long long)mesh * tiles + t) * F * 3, mesh, i, j);
}

template <int SYS, int BC, int R>
__global__ void __launch_bounds__(32 * R) k_boe(const BatchInst* __restrict__ I, int n, int last,
                                                int* __restrict__ status) {
  const long long blk = blockIdx.x;
  const int q = find_instance(I, n, blk);
  const BatchInst& in = I[q];
  const int tiles = in.tx * in.ty;
  const int local = (int)(blk - in.blk0);
  const int mesh = local / tiles, t = local - mesh * tiles;
  const int i = (t % in.tx) * 32 + (threadIdx.x & 31);
  const int j = (t / in.tx) * R + (threadIdx.x >> 5);
  // square cells: the isotropic variant, as the single-mesh launch chooses it
  if (in.g.hx == in.g.hy)
    oe_cell2d<SYS, BC, false, 0, true>(in.g, in.a, last ? in.u : in.b, in.dt, in.sigma, nullptr, status, mesh, i, j);
  else
    oe_cell2d<SYS, BC, false>(in.g, in.a, last ? in.u : in.b, in.dt, in.sigma, nullptr, status, mesh, i, j);
}

// avg and sigma per instance, mesh and field: grid (F, 2, n), fixed order
__global__ void k_bsigma(const BatchInst* __restrict__ I, int F) {
  const int f = blockIdx.x, mesh = blockIdx.y;
  const BatchInst& in = I[blockIdx.z];
  const long long nblk = (long long)in.tx * in.ty;
  __shared__ double sh[96];
  double s = 0.0, mx = -DINF, mn = DINF;
  for (long long b = threadIdx.x; b < nblk; b += blockDim.x) {
    const double* p = in.part + ((mesh * nblk + b) * F + f) * 3;
    s += p[0];
    mx = fmax(mx, p[1]);
    mn = fmin(mn, p[2]);
  }
  block_reduce3(s, mx, mn, sh);
  if (threadIdx.x == 0) {
    const double a = s / (double)in.g.plane;
    in.avg[mesh * F + f] = a;
    in.sigma[mesh * F + f] = fmax(mx - a, a - mn);
  }
}

// per-instance maximum wave speeds over both meshes' cell averages: grid (WB, n)
template <int SYS>
__global__ void k_bwave(const BatchInst* __restrict__ I, int* __restrict__ status) {
  constexpr int F = Fields<SYS>::F;
  const BatchInst& in = I[blockIdx.y];
  const Geo& g = in.g;
  __shared__ double sh[32];
  const long long nc = 2 * g.plane;
  double mx = 0.0, my = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x) {
    const int mesh = (int)(c / g.plane);
    const long long cell = c - mesh * g.plane;
    const double* us = in.u + (long long)mesh * F * 9 * g.plane + cell;
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
    in.wpart[blockIdx.x * 2] = mx;
    in.wpart[blockIdx.x * 2 + 1] = my;
  }
}

// tau_max = C_CFL / (beta_x/h_x + beta_y/h_y) per instance (no end time)
__global__ void k_bdt(const BatchInst* __restrict__ I, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const BatchInst& in = I[q];
  double bx = 0.0, by = 0.0;
  for (int b = 0; b < WB; ++b) {
    bx = fmax(bx, in.wpart[2 * b]);
    by = fmax(by, in.wpart[2 * b + 1]);
  }
  const double rate = bx / in.g.hx + by / in.g.hy;
  const double tm = rate > 0.0 ? in.g.cfl / rate : 0.0;
  in.dt[0] = tm;
  in.dt[1] = tm > 0.0 ? tm : 1.0;
  in.time[0] += tm;
}

__global__ void k_bset_time(const BatchInst* __restrict__ I, int n, double t) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) I[q].time[0] = t;
}

}  // namespace oecdg

using namespace oecdg;

struct cdg_batch {
  int n;
  int F;
  int sys, bc;
  int rows;                // tile height R in use
  cudaStream_t stream;
  int own_stream;
  BatchInst* h_inst;       // host copy of the instance table
  BatchInst* d_inst;       // device instance table
  long long total_blocks;  // stage / OE grid size for `rows`
  double* pool;            // one allocation: scratch states + partials + small slots
  int* status;
  double** h_ptrs;         // the caller's state pointers last uploaded
  cudaGraphExec_t graph;
  int graph_steps;
  long long launches;
  char err[256];
};

static cdg_status bfail(cdg_batch* b, cdg_status s, const char* msg) {
  if (b) snprintf(b->err, sizeof b->err, "%s", msg);
  return s;
}

// tile table for tile height R; uploads the instance table
static cudaError_t batch_layout(cdg_batch* B, int R) {
  long long blk = 0;
  for (int q = 0; q < B->n; ++q) {
    BatchInst& in = B->h_inst[q];
    in.tx = (in.g.nx + 31) / 32;
    in.ty = (in.g.ny + R - 1) / R;
    in.blk0 = blk;
    blk += 2LL * in.tx * in.ty;
  }
  B->total_blocks = blk;
  B->rows = R;
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
    B->graph_steps = 0;
  }
  return cudaMemcpy(B->d_inst, B->h_inst, sizeof(BatchInst) * B->n, cudaMemcpyHostToDevice);
}

template <int SYS, int BC>
static cudaError_t launch_bstage_t(cdg_batch* B, int l, double ca, double cb) {
  const unsigned grid = (unsigned)B->total_blocks;
  switch (B->rows) {
    case 2: k_bstage<SYS, BC, 2><<<grid, 64, 0, B->stream>>>(B->d_inst, B->n, l, ca, cb); break;
    case 8: k_bstage<SYS, BC, 8><<<grid, 256, 0, B->stream>>>(B->d_inst, B->n, l, ca, cb); break;
    default: k_bstage<SYS, BC, 4><<<grid, 128, 0, B->stream>>>(B->d_inst, B->n, l, ca, cb); break;
  }
  return cudaGetLastError();
}

template <int SYS, int BC>
static cudaError_t launch_boe_t(cdg_batch* B, int last) {
  const unsigned grid = (unsigned)B->total_blocks;
  switch (B->rows) {
    case 2: k_boe<SYS, BC, 2><<<grid, 64, 0, B->stream>>>(B->d_inst, B->n, last, B->status); break;
    case 8: k_boe<SYS, BC, 8><<<grid, 256, 0, B->stream>>>(B->d_inst, B->n, last, B->status); break;
    default: k_boe<SYS, BC, 4><<<grid, 128, 0, B->stream>>>(B->d_inst, B->n, last, B->status); break;
  }
  return cudaGetLastError();
}

static cudaError_t launch_bstage(cdg_batch* B, int l, double ca, double cb) {
  B->launches += 1;
  if (B->bc == BC_PERIODIC) return launch_bstage_t<SYS_EULER, BC_PERIODIC>(B, l, ca, cb);
  return launch_bstage_t<SYS_EULER, BC_TRANSMISSIVE>(B, l, ca, cb);
}

static cudaError_t launch_boe(cdg_batch* B, int last) {
  B->launches += 1;
  if (B->bc == BC_PERIODIC) return launch_boe_t<SYS_EULER, BC_PERIODIC>(B, last);
  return launch_boe_t<SYS_EULER, BC_TRANSMISSIVE>(B, last);
}

static const double BSSP3_C[3] = {0.0, 0.75, 1.0 / 3.0};

// one SSP-RK3 step of every instance: 11 launches
static cudaError_t batch_one_step(cdg_batch* B) {
  k_bwave<SYS_EULER><<<dim3(WB, B->n), 256, 0, B->stream>>>(B->d_inst, B->status);
  k_bdt<<<(B->n + 127) / 128, 128, 0, B->stream>>>(B->d_inst, B->n);
  B->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int l = 0; l < 3; ++l) {
    const double ca = BSSP3_C[l];
    if ((e = launch_bstage(B, l, ca, 1.0 - ca)) != cudaSuccess) return e;
    k_bsigma<<<dim3(B->F, 2, B->n), 1024, 0, B->stream>>>(B->d_inst, B->F);
    B->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_boe(B, l == 2)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

extern "C" {

cdg_status cdg_init_batch(const cdg_mesh_desc* descs, int n, void* stream, cdg_batch** out) {
  if (out) *out = nullptr;
  if (!descs || !out || n < 1) return CDG_EINVAL;
  for (int q = 0; q < n; ++q) {
    const cdg_mesh_desc& d = descs[q];
    if (d.dim != 2 || d.nx < 2 || d.ny < 2) return CDG_EINVAL;
    if (d.system != CDG_EULER || d.k != 2 || d.basis != CDG_BASIS_Q || d.rk != CDG_RK_SSP3 || d.oe != 1)
      return CDG_EUNSUPPORTED;
    if (d.bc != descs[0].bc || (d.bc != CDG_PERIODIC && d.bc != CDG_TRANSMISSIVE)) return CDG_EINVAL;
    if (!(d.bx > d.ax) || !(d.by > d.ay) || !(d.cfl > 0.0) || !(d.gamma > 1.0)) return CDG_EINVAL;
  }
  cdg_batch* B = (cdg_batch*)calloc(1, sizeof(cdg_batch));
  if (!B) return CDG_ENOMEM;
  B->n = n;
  B->F = 4;
  B->sys = SYS_EULER;
  B->bc = descs[0].bc == CDG_PERIODIC ? BC_PERIODIC : BC_TRANSMISSIVE;
  B->h_inst = (BatchInst*)calloc(n, sizeof(BatchInst));
  B->h_ptrs = (double**)calloc(n, sizeof(double*));
  if (!B->h_inst || !B->h_ptrs) {
    cdg_batch_free(B);
    return CDG_ENOMEM;
  }
  if (stream) {
    B->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cdg_batch_free(B);
      return CDG_ECUDA;
    }
    B->own_stream = 1;
  }
  // pool: per instance 2 scratch states, partials for the smallest tile height
  // (the most tiles), wave partials and the small slots
  size_t total = 0;
  for (int q = 0; q < n; ++q) {
    const cdg_mesh_desc& d = descs[q];
    const size_t plane = (size_t)d.nx * d.ny;
    const size_t tiles = (size_t)((d.nx + 31) / 32) * ((d.ny + 1) / 2);
    total += 2 * (size_t)2 * 4 * 9 * plane + 2 * tiles * 4 * 3 + WB * 2 + 2 + 2 + 8 + 8;
  }
  if (cudaMalloc((void**)&B->pool, total * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&B->d_inst, sizeof(BatchInst) * n) != cudaSuccess ||
      cudaMalloc((void**)&B->status, sizeof(int)) != cudaSuccess) {
    (void)cudaGetLastError();  // clear the failed allocation: later launch checks must not see it
    cdg_batch_free(B);
    return CDG_ENOMEM;
  }
  double* p = B->pool;
  for (int q = 0; q < n; ++q) {
    const cdg_mesh_desc& d = descs[q];
    BatchInst& in = B->h_inst[q];
    Geo& g = in.g;
    g.nx = d.nx;
    g.ny = d.ny;
    g.plane = (long long)d.nx * d.ny;
    g.hx = (d.bx - d.ax) / d.nx;
    g.hy = (d.by - d.ay) / d.ny;
    g.gamma = d.gamma;
    g.adv_x = d.adv_x;
    g.adv_y = d.adv_y;
    g.cfl = d.cfl;
    const size_t st = (size_t)2 * 4 * 9 * g.plane;
    const size_t tiles = (size_t)((d.nx + 31) / 32) * ((d.ny + 1) / 2);
    in.a = p; p += st;
    in.b = p; p += st;
    in.part = p; p += 2 * tiles * 4 * 3;
    in.wpart = p; p += WB * 2;
    in.dt = p; p += 2;
    in.time = p; p += 2;
    in.sigma = p; p += 8;
    in.avg = p; p += 8;
    in.u = nullptr;
  }
  if (batch_layout(B, 4) != cudaSuccess || cudaMemsetAsync(B->status, 0, sizeof(int), B->stream) != cudaSuccess) {
    cdg_batch_free(B);
    return CDG_ECUDA;
  }
  k_bset_time<<<(n + 127) / 128, 128, 0, B->stream>>>(B->d_inst, n, 0.0);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(B->stream) != cudaSuccess) {
    cdg_batch_free(B);
    return CDG_ECUDA;
  }
  *out = B;
  return CDG_OK;
}

cdg_status cdg_batch_free(cdg_batch* B) {
  if (!B) return CDG_OK;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  cudaFree(B->pool);
  cudaFree(B->d_inst);
  cudaFree(B->status);
  if (B->own_stream) cudaStreamDestroy(B->stream);
  free(B->h_inst);
  free(B->h_ptrs);
  free(B);
  return CDG_OK;
}

const char* cdg_batch_last_error(const cdg_batch* B) { return B ? B->err : ""; }

// point the instance table at the caller's states (re-uploads only on change)
static cdg_status batch_bind(cdg_batch* B, double* const* d_us) {
  int changed = 0;
  for (int q = 0; q < B->n; ++q) {
    if (!d_us[q]) return bfail(B, CDG_EINVAL, "batch: null state pointer");
    if (B->h_ptrs[q] != d_us[q]) changed = 1;
  }
  if (!changed) return CDG_OK;
  for (int q = 0; q < B->n; ++q) {
    B->h_ptrs[q] = d_us[q];
    B->h_inst[q].u = d_us[q];
  }
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
    B->graph_steps = 0;
  }
  if (cudaStreamSynchronize(B->stream) != cudaSuccess ||
      cudaMemcpy(B->d_inst, B->h_inst, sizeof(BatchInst) * B->n, cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(B, CDG_ECUDA, "batch: uploading the instance table failed");
  return CDG_OK;
}

cdg_status cdg_batch_step(cdg_batch* B, double* const* d_us, int nsteps, int use_graph) {
  if (!B || !d_us || nsteps < 0) return bfail(B, CDG_EINVAL, "batch_step: bad arguments");
  cdg_status s = batch_bind(B, d_us);
  if (s != CDG_OK) return s;
  if (nsteps == 0) return CDG_OK;
  if (!use_graph) {
    for (int k = 0; k < nsteps; ++k)
      if (batch_one_step(B) != cudaSuccess) return bfail(B, CDG_ECUDA, "batch_step: launch failed");
    return CDG_OK;
  }
  if (!B->graph || B->graph_steps != nsteps) {
    if (B->graph) {
      cudaGraphExecDestroy(B->graph);
      B->graph = nullptr;
    }
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return bfail(B, CDG_ECUDA, "batch_step: stream capture failed to begin");
    cudaError_t e = cudaSuccess;
    const long long before = B->launches;  // captured launches are counted when the graph runs
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = batch_one_step(B);
    B->launches = before;
    cudaError_t e2 = cudaStreamEndCapture(B->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) return bfail(B, CDG_ECUDA, "batch_step: capture failed");
    e = cudaGraphInstantiate(&B->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(B, CDG_ECUDA, "batch_step: graph instantiation failed");
    B->graph_steps = nsteps;
  }
  if (cudaGraphLaunch(B->graph, B->stream) != cudaSuccess) return bfail(B, CDG_ECUDA, "batch_step: graph launch failed");
  B->launches += 11LL * nsteps;
  return CDG_OK;
}

cdg_status cdg_batch_check_status(cdg_batch* B) {
  if (!B) return CDG_EINVAL;
  int h = 0;
  if (cudaMemcpyAsync(&h, B->status, sizeof(int), cudaMemcpyDeviceToHost, B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->status, 0, sizeof(int), B->stream) != cudaSuccess ||
      cudaStreamSynchronize(B->stream) != cudaSuccess)
    return bfail(B, CDG_ECUDA, "batch_check_status: CUDA error");
  if (h & ST_NONPHYSICAL) return bfail(B, CDG_ENONPHYSICAL, "non-physical cell average in the batch");
  return CDG_OK;
}

cdg_status cdg_batch_get_time(cdg_batch* B, double* t) {
  if (!B || !t) return CDG_EINVAL;
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return CDG_ECUDA;
  for (int q = 0; q < B->n; ++q)
    if (cudaMemcpy(t + q, B->h_inst[q].time, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return CDG_ECUDA;
  return CDG_OK;
}

cdg_status cdg_batch_launch_count(const cdg_batch* B, long long* count) {
  if (!B || !count) return CDG_EINVAL;
  *count = B->launches;
  return CDG_OK;
}

cdg_status cdg_batch_set_rows(cdg_batch* B, int rows) {
  if (!B || (rows != 2 && rows != 4 && rows != 8)) return CDG_EINVAL;
  if (cudaStreamSynchronize(B->stream) != cudaSuccess || batch_layout(B, rows) != cudaSuccess) return CDG_ECUDA;
  return CDG_OK;
}

cdg_status cdg_batch_rows(const cdg_batch* B, int* rows) {
  if (!B || !rows) return CDG_EINVAL;
  *rows = B->rows;
  return CDG_OK;
}

// signature of a batch for the autotune cache: sizes, boundary and count
static void batch_signature(const cdg_batch* B, char* sig, size_t len) {
  unsigned long long h = 1469598103934665603ULL;
  for (int q = 0; q < B->n; ++q) {
    h = (h ^ (unsigned long long)B->h_inst[q].g.nx) * 1099511628211ULL;
    h = (h ^ (unsigned long long)B->h_inst[q].g.ny) * 1099511628211ULL;
  }
  snprintf(sig, len, "euler_q2_bc%d_n%d_%016llx", B->bc, B->n, h);
}

static int cache_lookup(const char* path, const char* sig) {
  FILE* f = fopen(path, "r");
  if (!f) return 0;
  char buf[1 << 16];
  size_t m = fread(buf, 1, sizeof buf - 1, f);
  fclose(f);
  buf[m] = 0;
  char key[160];
  snprintf(key, sizeof key, "\"%s\": ", sig);
  const char* p = strstr(buf, key);
  if (!p) return 0;
  int r = atoi(p + strlen(key));
  return (r == 2 || r == 4 || r == 8) ? r : 0;
}

static void cache_store(const char* path, const char* sig, int rows) {
  char buf[1 << 16];
  buf[0] = 0;
  FILE* f = fopen(path, "r");
  size_t m = 0;
  if (f) {
    m = fread(buf, 1, sizeof buf - 1, f);
    fclose(f);
  }
  buf[m] = 0;
  // keep previous entries: strip the closing brace of an existing object
  char* end = strrchr(buf, '}');
  f = fopen(path, "w");
  if (!f) return;
  if (end && strchr(buf, '{')) {
    *end = 0;
    char* last = end;
    while (last > buf && (last[-1] == ' ' || last[-1] == '\n')) --last;
    *last = 0;
    const int empty = last > buf && last[-1] == '{';
    fprintf(f, "%s%s\n  \"%s\": %d\n}\n", buf, empty ? "" : ",", sig, rows);
  } else {
    fprintf(f, "{\n  \"%s\": %d\n}\n", sig, rows);
  }
  fclose(f);
}

cdg_status cdg_batch_autotune(cdg_batch* B, double* const* d_us, const char* cache_path, int* rows_out) {
  if (!B || !d_us) return CDG_EINVAL;
  cdg_status s = batch_bind(B, d_us);
  if (s != CDG_OK) return s;
  char sig[128];
  batch_signature(B, sig, sizeof sig);
  int best = cache_path ? cache_lookup(cache_path, sig) : 0;
  if (!best) {
    // time one stage + sigma + OE of every candidate (reads the states, writes
    // only the scratch buffers), best of 3
    const int cand[3] = {2, 4, 8};
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CDG_ECUDA;
    k_bwave<SYS_EULER><<<dim3(WB, B->n), 256, 0, B->stream>>>(B->d_inst, B->status);
    k_bdt<<<(B->n + 127) / 128, 128, 0, B->stream>>>(B->d_inst, B->n);
    k_bset_time<<<(B->n + 127) / 128, 128, 0, B->stream>>>(B->d_inst, B->n, 0.0);
    for (int c = 0; c < 3; ++c) {
      if (batch_layout(B, cand[c]) != cudaSuccess) return CDG_ECUDA;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, B->stream);
        launch_bstage(B, 0, 0.0, 1.0);
        k_bsigma<<<dim3(B->F, 2, B->n), 1024, 0, B->stream>>>(B->d_inst, B->F);
        launch_boe(B, 0);
        cudaEventRecord(e1, B->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return CDG_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best_ms) {
          best_ms = ms;
          best = cand[c];
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cache_path) cache_store(cache_path, sig, best);
  }
  if (batch_layout(B, best) != cudaSuccess) return CDG_ECUDA;
  if (rows_out) *rows_out = best;
  return CDG_OK;
}

}  // extern "C"
