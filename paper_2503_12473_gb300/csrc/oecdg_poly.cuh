// oecdg_poly.cuh -- Gauss-Legendre rules with 2, 3 and 4 points and the
// unnormalised Legendre polynomials P_0..P_3 with their derivatives, as
// constexpr functions of (rule size, point index) so that fully unrolled loops
// over points and modes fold them into constants.  Used by the degree-generic
// kernels (1D P^k, 2D Q^k / P^k, k = 1, 2, 3).
#pragma once

#include "oecdg_common.cuh"

namespace oecdg {

// N-point Gauss-Legendre rules on [-1, 1] (N = K + 1), nodes in increasing order:
//  2 points: +-1/sqrt(3), weights 1;
//  3 points: 0, +-sqrt(3/5), weights 8/9, 5/9;
//  4 points: +-sqrt(3/7 -+ (2/7) sqrt(6/5)), weights (18 +- sqrt(30)) / 36.
__host__ __device__ constexpr double gn1(int N, int q) {
  return N == 2 ? (q == 0 ? -0.57735026918962576451 : 0.57735026918962576451)
       : N == 3 ? gnode(q)
       : (q == 0 ? -0.86113631159405257522
          : q == 1 ? -0.33998104358485626480 : q == 2 ? 0.33998104358485626480 : 0.86113631159405257522);
}
__host__ __device__ constexpr double gw1(int N, int q) {
  return N == 2 ? 1.0
       : N == 3 ? gwt(q)
       : ((q == 0 || q == 3) ? 0.34785484513745385737 : 0.65214515486254614263);
}

// d-th derivative of the unnormalised Legendre polynomial P_n (n <= 3)
__host__ __device__ constexpr double lpd(int n, int d, double x) {
  return d == 0 ? (n == 0 ? 1.0 : n == 1 ? x : n == 2 ? 1.5 * x * x - 0.5 : (2.5 * x * x - 1.5) * x)
       : d == 1 ? (n == 0 ? 0.0 : n == 1 ? 1.0 : n == 2 ? 3.0 * x : 7.5 * x * x - 1.5)
       : d == 2 ? (n < 2 ? 0.0 : n == 2 ? 3.0 : 15.0 * x)
       : d == 3 ? (n == 3 ? 15.0 : 0.0)
       : 0.0;
}
// Coefficient of P_to(t) in P_from(t + d) for d = +1 or -1 (re-expansion of a
// Legendre series under a shift by a whole reference half-width):
//   P_1(t+d) = P_1 + d,  P_2(t+d) = P_2 + 3d P_1 + 3/2,
//   P_3(t+d) = P_3 + 5d P_2 + 15/2 P_1 + 7/2 d.
__host__ __device__ constexpr double lshift(int from, int to, double d) {
  return from == to ? 1.0
       : from == 1 ? (to == 0 ? d : 0.0)
       : from == 2 ? (to == 1 ? 3.0 * d : to == 0 ? 1.5 : 0.0)
       : from == 3 ? (to == 2 ? 5.0 * d : to == 1 ? 7.5 : to == 0 ? 3.5 * d : 0.0)
       : 0.0;
}
__host__ __device__ constexpr double fact(int m) { return m <= 1 ? 1.0 : m * fact(m - 1); }

// Points of half (sub-cell) s in the cell's own reference coordinate and the
// same physical points in the overlapping cell of the other mesh (N-point rule).
__host__ __device__ constexpr double xs1(int N, int s, int q) { return s - 0.5 + 0.5 * gn1(N, q); }
__host__ __device__ constexpr double xo1(int N, int s, int q) { return 0.5 - s + 0.5 * gn1(N, q); }

}  // namespace oecdg
