// oecdg_persist.cuh -- pieces shared by the persistent (cooperative) kernels:
// a grid-wide barrier with a bounded wait, coherent loads for data written
// earlier in the same launch, and the fixed-order sigma reduction that every
// path (per-phase launches and persistent kernels) runs, so that their
// results agree bit for bit.
#pragma once

#include <cuda_runtime.h>

#include "oecdg_common.cuh"

namespace oecdg {

// Status bit of a grid barrier that gave up waiting (CDG_ETIMEOUT on the host).
enum { ST_TIMEOUT = 2 };

// Load policy of the per-cell bodies.  LD_NC: the read-only (non-coherent)
// path, valid when nothing the kernel reads is written during the launch (one
// launch per phase).  LD_CA: plain (coherent, L1-cached) loads, for persistent
// kernels, whose phases read what earlier phases of the same launch wrote: the
// grid barrier's fences order those writes before the reads (the read-only
// path is outside that guarantee).  LD_CG: cached in L2 only.
enum { LD_NC = 0, LD_CA = 1, LD_CG = 2 };

template <int LD>
__device__ __forceinline__ double ldv(const double* p) {
  if (LD == LD_NC) return __ldg(p);
  if (LD == LD_CG) return __ldcg(p);
  return *p;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch.  `count` is a 64-bit arrival
// counter, zero at launch; the k-th barrier completes when it reaches
// k * expected (expected = gridDim.x, or more to make the wait run out on
// purpose in a test).  Thread 0 of each block publishes the block's writes
// (__syncthreads, then a device-scope fence before its arrival: release),
// spins with a short sleep until the barrier completes, until another block
// has given up (the status word has ST_TIMEOUT), or until limit_ns of its own
// wait have passed, when it sets ST_TIMEOUT; then a device-scope fence
// (acquire) and __syncthreads order the block's later loads after every
// block's writes.  Returns false after a timeout: the caller then leaves the
// kernel, so every block ends within about one limit.
__device__ __forceinline__ bool grid_sync(unsigned long long* count, unsigned long long expected, int* status,
                                          unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long arrive = atomicAdd(count, 1ULL);
    const unsigned long long target = (arrive / expected + 1) * expected;
    const unsigned long long t0 = global_ns();
    int good = 1;
    while (*(volatile unsigned long long*)count < target) {
      if (*(volatile int*)status & ST_TIMEOUT) {
        good = 0;
        break;
      }
      if (global_ns() - t0 > limit_ns) {
        atomicOr(status, ST_TIMEOUT);
        good = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// True in exactly one block per call: the last of gridDim.x blocks to finish
// the phase that precedes the call (a monotone ticket counter, zero at
// launch).  That block then sees every other block's writes of the phase
// (release fence before each ticket, acquire fence after the last one).
__device__ __forceinline__ bool last_block(unsigned long long* tickets) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long t = atomicAdd(tickets, 1ULL);
    last = (t + 1) % gridDim.x == 0;
    if (last) __threadfence();
  }
  __syncthreads();
  return last != 0;
}

// Normalisation of the sigma reduction: the (weighted) cell count of each mesh
// and the fields (bit f) whose domain average is 0 by mirror symmetry (the
// normal momentum beside a reflective wall).  Without walls: ncell = the
// cells of a mesh, odd = 0.
struct SigmaNorm {
  double ncell[2];
  int odd;
};

// avg and sigma of one (mesh, field) from the block partials [2][nblk][F][3]
// (sum of weighted cell averages, max, min), by one full warp in a fixed
// order: lane l folds partials l + 32 r + 256 q into accumulator r (r = 0..7,
// eight independent chains, so that the loads overlap), the accumulators are
// folded r = 0..7, then a shuffle tree.  avg = sum / ncell (0 for an odd
// field), sigma = max(max - avg, avg - min) (Section 2.2, sigma_K; 0 at the
// rounding level of the field, sigma_from_range).
template <int LD>
__device__ __forceinline__ void warp_sigma(const double* part, long long nblk, int F, int mesh, int f,
                                           const SigmaNorm& sn, double* avg, double* sigma) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  constexpr int CH = 8;
  double sr[CH], xr[CH], nr[CH];
#pragma unroll
  for (int r = 0; r < CH; ++r) {
    sr[r] = 0.0;
    xr[r] = -__builtin_huge_val();
    nr[r] = __builtin_huge_val();
  }
  for (long long b0 = lane; b0 < nblk; b0 += 32 * CH) {
#pragma unroll
    for (int r = 0; r < CH; ++r) {
      const long long b = b0 + 32 * r;
      if (b < nblk) {
        const double* p = part + ((mesh * nblk + b) * F + f) * 3;
        sr[r] += ldv<LD>(p);
        xr[r] = fmax(xr[r], ldv<LD>(p + 1));
        nr[r] = fmin(nr[r], ldv<LD>(p + 2));
      }
    }
  }
  double s = sr[0], mx = xr[0], mn = nr[0];
#pragma unroll
  for (int r = 1; r < CH; ++r) {
    s += sr[r];
    mx = fmax(mx, xr[r]);
    mn = fmin(mn, nr[r]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(full, s, o);
    mx = fmax(mx, __shfl_down_sync(full, mx, o));
    mn = fmin(mn, __shfl_down_sync(full, mn, o));
  }
  if (lane == 0) {
    const double a = ((sn.odd >> f) & 1) ? 0.0 : s / sn.ncell[mesh];
    avg[mesh * F + f] = a;
    sigma[mesh * F + f] = sigma_from_range(mx, mn, a);
  }
}

// The same reduction as warp_sigma, bit for bit, by the 8 warps of one block
// of 256 threads: warp r runs accumulator chain r (partials lane + 32 r + 256 q,
// q = 0, 1, ..., in that order), then warp 0 folds the chains r = 0..7 of its
// lane and runs the same shuffle tree.  For the per-phase launch, where the
// single warp's 8 chains of L2 round trips would dominate the kernel.
template <int LD>
__device__ __forceinline__ void block_sigma(const double* part, long long nblk, int F, int mesh, int f,
                                            const SigmaNorm& sn, double* avg, double* sigma) {
  constexpr int CH = 8;
  __shared__ double sh[3][CH][32];
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
  double sr = 0.0, xr = -__builtin_huge_val(), nr = __builtin_huge_val();
  for (long long b = lane + 32 * r; b < nblk; b += 32 * CH) {
    const double* p = part + ((mesh * nblk + b) * F + f) * 3;
    sr += ldv<LD>(p);
    xr = fmax(xr, ldv<LD>(p + 1));
    nr = fmin(nr, ldv<LD>(p + 2));
  }
  sh[0][r][lane] = sr;
  sh[1][r][lane] = xr;
  sh[2][r][lane] = nr;
  __syncthreads();
  if (r != 0) return;
  const unsigned full = 0xffffffffu;
  double s = sh[0][0][lane], mx = sh[1][0][lane], mn = sh[2][0][lane];
#pragma unroll
  for (int q = 1; q < CH; ++q) {
    s += sh[0][q][lane];
    mx = fmax(mx, sh[1][q][lane]);
    mn = fmin(mn, sh[2][q][lane]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(full, s, o);
    mx = fmax(mx, __shfl_down_sync(full, mx, o));
    mn = fmin(mn, __shfl_down_sync(full, mn, o));
  }
  if (lane == 0) {
    const double a = ((sn.odd >> f) & 1) ? 0.0 : s / sn.ncell[mesh];
    avg[mesh * F + f] = a;
    sigma[mesh * F + f] = sigma_from_range(mx, mn, a);
  }
}

// The plain normalisation: every cell of a mesh counts once, no odd field.
__host__ __device__ __forceinline__ SigmaNorm plain_norm(long long ncell) {
  SigmaNorm sn;
  sn.ncell[0] = sn.ncell[1] = (double)ncell;
  sn.odd = 0;
  return sn;
}

// tau_max = C_CFL / (beta_x/h_x + beta_y/h_y) (1D: C_CFL h / beta) from the
// maxima bx, by; tau = tau_max clipped at T_end > 0 (a step that would leave a
// sliver shorter than 1e-12 T_end is stretched to T_end); time[0] advances.
__device__ __forceinline__ void finish_dt(double bx, double by, double hx, double hy, int dim, double cfl,
                                          double T_end, double* dt, double* time) {
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

}  // namespace oecdg
