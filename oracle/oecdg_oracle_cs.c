/*
 * oecdg_oracle_cs.c -- the oracle of oecdg_oracle.c compiled with complex
 * state values, for complex-step differentiation of the scheme.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as oecdg_oracle.c).
 *
 * With the state u + i h v (h tiny, v a direction) every function of the
 * oracle returns f(u) + i h J(u) v up to rounding, with no subtractive
 * cancellation, so Im(f) / h is the Jacobian-vector product of the oracle's
 * own arithmetic (Squire and Trapp, SIAM Review 40 (1998); Martins, Sturdza
 * and Alonso, ACM TOMS 29 (2003)).  The non-smooth operations take the branch
 * of the real part: |x| is x or -x by the sign of Re x, max / min and
 * comparisons use real parts; sqrt and exp are the complex functions.
 * Columns J e_q for every basis direction e_q give the oracle's Jacobian of a
 * step, and J^T lambda its adjoint.
 *
 * Exports the state-dependent functions of oecdg_oracle.c with double complex
 * state arrays (interleaved re, im); projection, sampling points and
 * evaluation helpers are left out.
 */
#define ORC_COMPLEX_STEP 1
#include "oecdg_oracle.c"

/* Jacobian of nsteps steps of the scheme (tau = tau_max from the state at the
 * start of every step, no end time, as orc_advance) at the real state u:
 * column q is Im(step(u + i h e_q)) / h.  J is n x n row-major with
 * J[r * n + q] = d step(u)_r / d u_q, n the state size.  The columns are
 * independent and computed in parallel (one thread per column, the oracle's
 * own loops then run on that thread).  Returns ORC_ENONPHYSICAL if any run
 * met a non-physical cell average. */
int orc_step_jacobian(const orc_problem* p, const double* u, int nsteps, double h, double* J) {
  const long n = (long)state_len(p);
  int bad = 0;
#ifdef _OPENMP
  omp_set_max_active_levels(1);
#endif
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
  for (long q = 0; q < n; ++q) {
    real* z = (real*)malloc((size_t)n * sizeof(real));
    for (long r = 0; r < n; ++r) z[r] = u[r];
    z[q] += h * I;
    double t = 0.0;
    int done = 0;
    if (orc_advance(p, z, &t, 0.0, nsteps, &done) != ORC_OK) bad = 1;
    for (long r = 0; r < n; ++r) J[(size_t)r * n + q] = cimag(z[r]) / h;
    free(z);
  }
  return bad ? ORC_ENONPHYSICAL : ORC_OK;
}
