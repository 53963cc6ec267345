/*
 * oecdg_oracle.c -- plain, slow FP64 CPU oracle of the OECDG scheme
 * (Peng, Wu, Yuan, "Oscillation-eliminating central DG schemes for hyperbolic
 * conservation laws", arXiv:2503.12473).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA path.  It is
 * called from the test-suite, from the package's smoke() entry and from the
 * benchmark's CPU-baseline leg; nothing in the product path may link or call it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Every quantity is computed the literal way the paper defines it:
 *   - the CDG operator H (Section 2.1, Eq. (equcdg) / 1D Eq. (eq:1D_H) /
 *     2D Eq. (eq:2D_H)) by Gauss quadrature on the sub-cells cut by the
 *     overlapping mesh and on the half-faces, locating the overlapping cell of
 *     every quadrature point from its physical coordinates and evaluating both
 *     Legendre expansions directly at that point;
 *   - the damping coefficients delta_K^m, sigma_K and beta_{e,K} (Section 2.2,
 *     the definitions that follow Eq. (OEstep2D), and the two Remarks on 1D and
 *     on systems);
 *   - the exact solution of the damping ODE (OEstep2D) in the orthogonal
 *     Legendre basis (the coefficients decay exponentially, Section 3.3);
 *   - the fully discrete RK scheme (Eq. (eq:RKCDG)) with the Shu-Osher forms of
 *     forward Euler, SSP-RK2, SSP-RK3 and classical RK4 (Section 4).
 *
 * Readings of points the paper leaves open (the CUDA path implements the same
 * readings independently):
 *   - the dual mesh is the primal mesh shifted by (+hx/2, +hy/2), with the same
 *     number of cells; transmissive boundaries: a ghost cell outside the stored
 *     range is a copy of the nearest stored cell (all modes), per direction;
 *   - reflective walls (Euler): the restriction of the mirror-extended problem.
 *     Beyond a wall the solution is the mirror image of the inside (normal
 *     momentum negated); the dual mesh gains the cell centred on a low-side wall
 *     (stored in the slot after the last cell, so that both meshes keep the
 *     same padded layout); sigma and avg are those of the mirror-extended
 *     domain (wall-centred dual cells count half, a normal momentum has
 *     average 0);
 *   - quadrature: (k+1)-point Gauss-Legendre per direction on every sub-cell and
 *     half-face; Legendre polynomials unnormalised (P_n(1) = 1);
 *   - tau_max is the CFL value at the start of the step (maximum wave speed over
 *     the cell averages of both meshes), tau = tau_max except a final clipped step;
 *   - sigma: max over the (k+1)^d cell Gauss points, avg over stored cells;
 *   - h_{e,K} = the cell width normal to e; Sum_{|alpha|=m} is the plain
 *     multi-index sum; beta_{e,K} at K's cell average;
 *   - Q^k cells: P^{m-1} is the total-degree projection, so mode (a,b) decays at
 *     rate Sum_{m=0}^{min(a+b,k)} delta^m;
 *   - the OE time is the full step tau after every stage; OE is off for k = 0.
 *
 * Every function whose result has no independent pin in tests/ says
 * "parity unpinned" in its comment.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -shared -fPIC
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* State-dependent values have type `real`: double here.  The same source,
 * compiled with ORC_COMPLEX_STEP defined (oecdg_oracle_cs.c), makes `real`
 * double complex for complex-step differentiation: f(u + i h v) carries
 * h J v in its imaginary part.  |x|, comparisons and max/min then act on real
 * parts (the branch the value takes), sqrt and exp are the complex ones. */
#ifdef ORC_COMPLEX_STEP
#include <complex.h>
typedef double complex real;
#define RE(x) creal(x)
#define R_ABS(x) (creal(x) < 0.0 ? -(x) : (x))
#define R_SQRT(x) csqrt(x)
#define R_EXP(x) cexp(x)
#else
typedef double real;
#define RE(x) (x)
#define R_ABS(x) fabs(x)
#define R_SQRT(x) sqrt(x)
#define R_EXP(x) exp(x)
#endif

#define ORC_MAXK 3
#define ORC_MAXQ (ORC_MAXK + 1)
#define ORC_MAXF 4
#define ORC_MAXM ((ORC_MAXK + 1) * (ORC_MAXK + 1))

enum { ORC_ADVECTION = 0, ORC_BURGERS = 1, ORC_EULER = 2 };
enum { ORC_BASIS_Q = 0, ORC_BASIS_P = 1 };
enum { ORC_PERIODIC = 0, ORC_TRANSMISSIVE = 1, ORC_REFLECTIVE = 2 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENONPHYSICAL = 4 };

/* Problem description (mirrored by a ctypes.Structure in oracle/oracle.py). */
typedef struct {
  int dim;     /* 1 or 2 */
  int nx, ny;  /* primal cells per direction (ny = 1 when dim = 1) */
  int k;       /* polynomial degree, 0..3 */
  int basis;   /* ORC_BASIS_Q (tensor Q^k) or ORC_BASIS_P (total degree P^k) */
  int system;  /* ORC_ADVECTION, ORC_BURGERS, ORC_EULER */
  int bc[4];   /* per side: x-low, x-high, y-low, y-high (1D: x only); ORC_PERIODIC
                  (on both sides of a direction), ORC_TRANSMISSIVE or ORC_REFLECTIVE */
  int oe;      /* 1: apply the OE step after every stage */
  int rk;      /* 1 forward Euler, 2 SSP-RK2, 3 SSP-RK3, 4 classical RK4 */
  double ax, bx, ay, by; /* domain [ax,bx] x [ay,by] */
  double gamma;          /* ratio of specific heats (Euler) */
  double adv_x, adv_y;   /* advection velocity */
  double cfl;            /* C_CFL */
} orc_problem;

/* ---------------------------------------------------------------- basics -- */

static int nfields(const orc_problem* p) {
  return p->system == ORC_EULER ? p->dim + 2 : 1;
}

/* Mode list: (a, b) degrees in x and y.  Q^k: index b*(k+1)+a.  P^k: ordered
 * by total degree s = a+b, then by decreasing a.  1D: (a, 0), a = 0..k. */
static int modes(const orc_problem* p, int* ma, int* mb) {
  int k = p->k, n = 0;
  if (p->dim == 1) {
    for (int a = 0; a <= k; ++a) { ma[n] = a; mb[n] = 0; ++n; }
  } else if (p->basis == ORC_BASIS_Q) {
    for (int b = 0; b <= k; ++b)
      for (int a = 0; a <= k; ++a) { ma[n] = a; mb[n] = b; ++n; }
  } else {
    for (int s = 0; s <= k; ++s)
      for (int a = s; a >= 0; --a) { ma[n] = a; mb[n] = s - a; ++n; }
  }
  return n;
}

static int nmodes(const orc_problem* p) {
  int ma[ORC_MAXM], mb[ORC_MAXM];
  return modes(p, ma, mb);
}

static double hx_of(const orc_problem* p) { return (p->bx - p->ax) / p->nx; }
static double hy_of(const orc_problem* p) { return p->dim == 2 ? (p->by - p->ay) / p->ny : 1.0; }

/* 1 if side s (0: x-low, 1: x-high, 2: y-low, 3: y-high) is a reflective wall. */
static int refl(const orc_problem* p, int s) { return (p->dim == 2 || s < 2) && p->bc[s] == ORC_REFLECTIVE; }

/* Stored cells per direction of the padded layout (both meshes): nx, plus the
 * slot of the dual cell centred on a reflective low-side wall. */
static int nxs(const orc_problem* p) { return p->nx + refl(p, 0); }
static int nys(const orc_problem* p) { return p->dim == 2 ? p->ny + refl(p, 2) : 1; }
/* cells of mesh `mesh` per direction (the primal mesh leaves the slot unused) */
static int ncx(const orc_problem* p, int mesh) { return mesh == 0 ? p->nx : nxs(p); }
static int ncy(const orc_problem* p, int mesh) { return mesh == 0 ? (p->dim == 2 ? p->ny : 1) : nys(p); }

/* Index of coefficient (mesh, field, mode, j, i) in the state array. */
static size_t sidx(const orc_problem* p, int mesh, int f, int m, int j, int i) {
  int F = nfields(p), M = nmodes(p);
  return ((((size_t)mesh * F + f) * M + m) * nys(p) + j) * (size_t)nxs(p) + i;
}

/* Doubles in a state array (2 meshes x fields x modes x the padded cells). */
static size_t state_len(const orc_problem* p) { return (size_t)2 * nfields(p) * nmodes(p) * nys(p) * nxs(p); }

/* d-th derivative of the Legendre polynomial P_n at x (unnormalised, P_n(1)=1).
 * Three-term recurrence for the values and P^{(d)}_{n+1} = P^{(d)}_{n-1} +
 * (2n+1) P^{(d-1)}_n for the derivatives. */
double orc_legendre(int n, int d, double x) {
  double t[ORC_MAXK + 3][ORC_MAXK + 3];
  int N = n + 1;
  memset(t, 0, sizeof t);
  t[0][0] = 1.0;
  if (N > 1) t[0][1] = x;
  for (int q = 1; q + 1 < N; ++q) t[0][q + 1] = ((2.0 * q + 1.0) * x * t[0][q] - q * t[0][q - 1]) / (q + 1.0);
  for (int e = 1; e <= d; ++e) {
    t[e][0] = 0.0;
    if (N > 1) t[e][1] = (e == 1) ? 1.0 : 0.0;
    for (int q = 1; q + 1 < N; ++q) t[e][q + 1] = t[e][q - 1] + (2.0 * q + 1.0) * t[e - 1][q];
  }
  return t[d][n];
}

/* n-point Gauss-Legendre rule on [-1,1]: Newton iteration on P_n started from
 * the asymptotic root guesses; weights 2 / ((1 - x^2) P_n'(x)^2). */
void orc_gauss(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double dz = orc_legendre(n, 0, z) / orc_legendre(n, 1, z);
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    double d1 = orc_legendre(n, 1, z);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * d1 * d1);
  }
}

/* Centre of cell (i, j) of mesh `mesh` (0 primal, 1 dual).  The dual mesh is
 * the primal mesh shifted by (+hx/2, +hy/2) (Section 2.1): dual cell i spans
 * [x_i, x_{i+1}] between primal centres, i.e. it is centred on primal vertex i+1. */
static void cell_centre(const orc_problem* p, int mesh, int i, int j, double* xc, double* yc) {
  double hx = hx_of(p), hy = hy_of(p);
  /* the slot after the last dual cell holds the cell centred on the low wall */
  int iu = (mesh == 1 && i == p->nx) ? -1 : i, ju = (mesh == 1 && j == p->ny) ? -1 : j;
  *xc = p->ax + (iu + 0.5 + 0.5 * mesh) * hx;
  *yc = p->dim == 2 ? p->ay + (ju + 0.5 + 0.5 * mesh) * hy : 0.0;
}

/* Map an unwrapped cell index of direction `dir` (cell iu of the primal mesh
 * spans [iu h, (iu+1) h], dual cell iu is centred on vertex iu + 1) to a stored
 * one; *mirror = 1 when the cell is the mirror image of the stored cell across
 * a reflective wall.
 *   periodic: wrap;
 *   transmissive: the ghost cell outside the stored range is a copy of the
 *     nearest stored cell, every mode copied (corners by composition).  The
 *     paper does not say how the dual mesh is closed at an outflow boundary.
 *     Pinned where an outflow boundary is fixed by the physics: while the flow
 *     beside the boundary is uniform in the normal direction, a run equals the
 *     run on an enlarged domain cell for cell (tests/test_oracle_transmissive.py);
 *     the zeroth-order extrapolation beyond that is a convention;
 *   reflective: the dual cell centred on a low wall (vertex 0) is a stored cell
 *     (slot n); cells beyond a wall are mirror images: primal -1 - iu across the
 *     low wall and 2n - 1 - iu across the high one, dual (vertex v -> -v, 2n - v).
 *     Pinned: a reflective run equals the mirror-extended periodic run
 *     (tests/test_oracle_reflective.py). */
static int store_index(const orc_problem* p, int dir, int mesh, int iu, int* mirror) {
  int n = dir == 0 ? p->nx : p->ny;
  int lo = p->bc[2 * dir], hi = p->bc[2 * dir + 1];
  *mirror = 0;
  if (iu >= 0 && iu < n) return iu;
  if (lo == ORC_PERIODIC) return ((iu % n) + n) % n;
  if (iu < 0) {
    if (lo == ORC_TRANSMISSIVE) return 0;
    if (mesh == 1 && iu == -1) return n; /* the wall-centred dual cell */
    *mirror = 1;
    iu = mesh == 0 ? -1 - iu : -iu - 2;
  } else {
    if (hi == ORC_TRANSMISSIVE) return n - 1;
    *mirror = 1;
    iu = mesh == 0 ? 2 * n - 1 - iu : 2 * n - iu - 2;
  }
  return iu < 0 ? 0 : (iu >= n ? n - 1 : iu); /* one cell deep is all the scheme reads */
}

/* Locate the cell of mesh `mesh` containing the physical point (x, y) and give
 * the stored index, the point's reference coordinates in that cell and whether
 * the cell is a mirror image in x / y (the coordinate is then mirrored too). */
static void locate(const orc_problem* p, int mesh, double x, double y, int* si, int* sj, double* xi,
                   double* eta, int* mirx, int* miry) {
  double hx = hx_of(p), hy = hy_of(p);
  int iu = (int)floor((x - p->ax) / hx - 0.5 * mesh);
  double xc = p->ax + (iu + 0.5 + 0.5 * mesh) * hx;
  *xi = (x - xc) / (0.5 * hx);
  *si = store_index(p, 0, mesh, iu, mirx);
  if (*mirx) *xi = -*xi;
  if (p->dim == 2) {
    int ju = (int)floor((y - p->ay) / hy - 0.5 * mesh);
    double yc = p->ay + (ju + 0.5 + 0.5 * mesh) * hy;
    *eta = (y - yc) / (0.5 * hy);
    *sj = store_index(p, 1, mesh, ju, miry);
    if (*miry) *eta = -*eta;
  } else {
    *eta = 0.0;
    *sj = 0;
    *miry = 0;
  }
}

/* Basis function (a, b) with derivative orders (dx, dy) in reference
 * coordinates, converted to physical derivatives. */
static double basis(const orc_problem* p, int a, int b, int dx, int dy, double xi, double eta) {
  double v = orc_legendre(a, dx, xi) * pow(2.0 / hx_of(p), dx);
  if (p->dim == 2) v *= orc_legendre(b, dy, eta) * pow(2.0 / hy_of(p), dy);
  else if (dy > 0) v = 0.0;
  return v;
}

/* Value (dx = dy = 0) or physical derivative of every field of stored cell
 * (i, j) of mesh `mesh` at reference point (xi, eta). */
static void cell_eval(const orc_problem* p, const real* u, int mesh, int i, int j, double xi, double eta,
                      int dx, int dy, real* out) {
  int ma[ORC_MAXM], mb[ORC_MAXM];
  int M = modes(p, ma, mb), F = nfields(p);
  for (int f = 0; f < F; ++f) {
    real s = 0.0;
    for (int m = 0; m < M; ++m) s += u[sidx(p, mesh, f, m, j, i)] * basis(p, ma[m], mb[m], dx, dy, xi, eta);
    out[f] = s;
  }
}

/* cell_eval of a located cell: for a mirror image across a wall normal to x
 * (resp. y), the x-momentum (resp. y-momentum) changes sign and so does every
 * odd-order x- (resp. y-) derivative: g(x) = S u(2 x_w - x). */
static void located_eval(const orc_problem* p, const real* u, int mesh, int si, int sj, double xi, double eta,
                         int mirx, int miry, int dx, int dy, real* out) {
  cell_eval(p, u, mesh, si, sj, xi, eta, dx, dy, out);
  if (!mirx && !miry) return;
  int F = nfields(p);
  for (int f = 0; f < F; ++f) {
    int neg = 0;
    if (mirx) neg ^= (dx & 1) ^ (p->system == ORC_EULER && f == 1);
    if (miry) neg ^= (dy & 1) ^ (p->system == ORC_EULER && f == 2);
    if (neg) out[f] = -out[f];
  }
}

/* Value of the mesh-`mesh` solution at a physical point. */
static void point_eval(const orc_problem* p, const real* u, int mesh, double x, double y, real* out) {
  int si, sj, mx, my;
  double xi, eta;
  locate(p, mesh, x, y, &si, &sj, &xi, &eta, &mx, &my);
  located_eval(p, u, mesh, si, sj, xi, eta, mx, my, 0, 0, out);
}

/* ----------------------------------------------------------------- flux --- */

/* Physical flux components f1(w), f2(w) of the conservation law. Euler:
 * Section 4, 1D and 2D Euler subsections; advection u_t + a.grad u = 0;
 * Burgers f = u^2/2 (1D). */
static void flux(const orc_problem* p, const real* w, real* f1, real* f2) {
  if (p->system == ORC_ADVECTION) {
    f1[0] = p->adv_x * w[0];
    f2[0] = p->adv_y * w[0];
  } else if (p->system == ORC_BURGERS) {
    f1[0] = 0.5 * w[0] * w[0];
    f2[0] = 0.5 * w[0] * w[0];
  } else if (p->dim == 1) {
    real rho = w[0], m = w[1], E = w[2];
    real v = m / rho;
    real pr = (p->gamma - 1.0) * (E - 0.5 * rho * v * v);
    f1[0] = m;
    f1[1] = m * v + pr;
    f1[2] = (E + pr) * v;
    f2[0] = f2[1] = f2[2] = 0.0;
  } else {
    real rho = w[0], mx = w[1], my = w[2], E = w[3];
    real vx = mx / rho, vy = my / rho;
    real pr = (p->gamma - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy));
    f1[0] = mx;
    f1[1] = mx * vx + pr;
    f1[2] = my * vx;
    f1[3] = (E + pr) * vx;
    f2[0] = my;
    f2[1] = mx * vy;
    f2[2] = my * vy + pr;
    f2[3] = (E + pr) * vy;
  }
}

/* Spectral radius of n . df/du at state w (the local wave speed beta_{e,K},
 * Section 2.2 and the Remark on systems).  Returns -1 on a non-physical Euler
 * state (rho <= 0 or p <= 0). */
static real wave_speed(const orc_problem* p, const real* w, double nx, double ny) {
  if (p->system == ORC_ADVECTION) return fabs(p->adv_x * nx + p->adv_y * ny);
  if (p->system == ORC_BURGERS) return R_ABS(w[0] * (nx + ny));
  real rho = w[0];
  real vx = w[1] / rho, vy = p->dim == 2 ? w[2] / rho : 0.0;
  real E = w[p->dim + 1];
  real pr = (p->gamma - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy));
  if (!(RE(rho) > 0.0) || !(RE(pr) > 0.0)) return -1.0;
  real c = R_SQRT(p->gamma * pr / rho);
  return R_ABS(vx * nx + vy * ny) + c;
}

/* ------------------------------------------------------- CDG operator H --- */

/* L = M^{-1} R, where R_phi = H(u, phi) restricted to one mesh's test function
 * phi (Eq. (equcdg)):
 *   R = (1/tau_max) int_K (w - u_K) phi + int_K f(w) . grad phi
 *       - sum_e int_e f(w) . n_e phi^-,
 * with w the overlapping mesh's solution.  Volume integrals: (k+1)^d Gauss
 * points on each of the 2^d sub-cells of K cut by the overlapping mesh; face
 * integrals: (k+1) Gauss points on each of the 2 half-faces of every face (1D:
 * point faces).  Both are exact for a linear flux. */
static void cell_rhs(const orc_problem* p, const real* u, real inv_tmax, int mesh, int i, int j,
                     real* L /* [F][M] */) {
  int ma[ORC_MAXM], mb[ORC_MAXM];
  int M = modes(p, ma, mb), F = nfields(p), k = p->k, nq = k + 1, d = p->dim;
  int other = 1 - mesh;
  double hx = hx_of(p), hy = hy_of(p);
  double gx[ORC_MAXQ], gw[ORC_MAXQ];
  orc_gauss(nq, gx, gw);
  double xc, yc;
  cell_centre(p, mesh, i, j, &xc, &yc);
  real R[ORC_MAXF][ORC_MAXM];
  memset(R, 0, sizeof R);
  real w[ORC_MAXF], uk[ORC_MAXF], f1[ORC_MAXF], f2[ORC_MAXF];

  /* volume and dissipation terms on the sub-cells */
  int nsy = d == 2 ? 2 : 1, nqy = d == 2 ? nq : 1;
  for (int sy = 0; sy < nsy; ++sy)
    for (int sx = 0; sx < 2; ++sx)
      for (int qy = 0; qy < nqy; ++qy)
        for (int qx = 0; qx < nq; ++qx) {
          /* sub-cell s spans [-1+s, s] in reference coordinates */
          double xi = sx - 0.5 + 0.5 * gx[qx];
          double eta = d == 2 ? sy - 0.5 + 0.5 * gx[qy] : 0.0;
          double W = 0.5 * gw[qx] * 0.5 * hx;
          if (d == 2) W *= 0.5 * gw[qy] * 0.5 * hy;
          double x = xc + 0.5 * hx * xi, y = yc + 0.5 * hy * eta;
          point_eval(p, u, other, x, y, w);
          cell_eval(p, u, mesh, i, j, xi, eta, 0, 0, uk);
          flux(p, w, f1, f2);
          for (int m = 0; m < M; ++m) {
            double ph = basis(p, ma[m], mb[m], 0, 0, xi, eta);
            double phx = basis(p, ma[m], mb[m], 1, 0, xi, eta);
            double phy = d == 2 ? basis(p, ma[m], mb[m], 0, 1, xi, eta) : 0.0;
            for (int f = 0; f < F; ++f)
              R[f][m] += W * (inv_tmax * (w[f] - uk[f]) * ph + f1[f] * phx + (d == 2 ? f2[f] * phy : 0.0));
          }
        }

  /* face terms: - sum_e int_e f(w) . n_e phi^- */
  for (int face = 0; face < 2 * d; ++face) {
    int dir = face / 2;            /* 0: x-normal, 1: y-normal */
    double side = (face % 2) ? 1.0 : -1.0;
    for (int s = 0; s < (d == 2 ? 2 : 1); ++s)
      for (int q = 0; q < (d == 2 ? nq : 1); ++q) {
        double t = d == 2 ? s - 0.5 + 0.5 * gx[q] : 0.0; /* tangential reference coordinate */
        double xi = dir == 0 ? side : t, eta = dir == 0 ? t : side;
        double W = d == 2 ? 0.5 * gw[q] * 0.5 * (dir == 0 ? hy : hx) : 1.0;
        double x = xc + 0.5 * hx * xi, y = yc + 0.5 * hy * eta;
        point_eval(p, u, other, x, y, w);
        flux(p, w, f1, f2);
        for (int m = 0; m < M; ++m) {
          double ph = basis(p, ma[m], mb[m], 0, 0, xi, d == 2 ? eta : 0.0);
          for (int f = 0; f < F; ++f) {
            real fn = dir == 0 ? side * f1[f] : side * f2[f];
            R[f][m] -= W * fn * ph;
          }
        }
      }
  }

  /* M^{-1}: the Legendre basis is orthogonal, ||phi_ab||^2 = |K| / ((2a+1)(2b+1)) */
  for (int m = 0; m < M; ++m) {
    double nrm = hx / (2.0 * ma[m] + 1.0);
    if (d == 2) nrm *= hy / (2.0 * mb[m] + 1.0);
    for (int f = 0; f < F; ++f) L[f * M + m] = R[f][m] / nrm;
  }
}

/* Semi-discrete right-hand side dU/dt = L(U) on both meshes. */
void orc_rhs(const orc_problem* p, const real* u, real tau_max, real* L) {
  int F = nfields(p), M = nmodes(p);
  real inv = 1.0 / tau_max;
  for (int mesh = 0; mesh < 2; ++mesh) {
    int cy = ncy(p, mesh), cx = ncx(p, mesh);
#pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < cy; ++j)
      for (int i = 0; i < cx; ++i) {
        real Lc[ORC_MAXF * ORC_MAXM];
        cell_rhs(p, u, inv, mesh, i, j, Lc);
        for (int f = 0; f < F; ++f)
          for (int m = 0; m < M; ++m) L[sidx(p, mesh, f, m, j, i)] = Lc[f * M + m];
      }
  }
}

#ifndef ORC_COMPLEX_STEP
/* Bilinear form H(u, phi) for a test function given by its modal coefficients
 * (both meshes): H(u, phi) = sum_K sum_modes R_K(u) phi_K. */
double orc_bilinear(const orc_problem* p, const double* u, const double* phi, double tau_max) {
  int F = nfields(p), M = nmodes(p);
  int ma[ORC_MAXM], mb[ORC_MAXM];
  modes(p, ma, mb);
  size_t n = state_len(p);
  double* L = (double*)malloc(n * sizeof(double));
  orc_rhs(p, u, tau_max, L);
  double hx = hx_of(p), hy = hy_of(p), s = 0.0;
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int f = 0; f < F; ++f)
      for (int m = 0; m < M; ++m) {
        double nrm = hx / (2.0 * ma[m] + 1.0) * (p->dim == 2 ? hy / (2.0 * mb[m] + 1.0) : 1.0);
        for (int j = 0; j < ncy(p, mesh); ++j)
          for (int i = 0; i < ncx(p, mesh); ++i) {
            size_t id = sidx(p, mesh, f, m, j, i);
            s += nrm * L[id] * phi[id];
          }
      }
  free(L);
  return s;
}
#endif

/* --------------------------------------------------------- OE procedure --- */

/* Weight of a cell of mesh `mesh` in the domain average: 1, halved for each
 * reflective wall the cell is centred on (dual cells only: the mirror-extended
 * domain holds such a cell once, every other cell twice). */
static double cell_weight(const orc_problem* p, int mesh, int i, int j) {
  if (mesh == 0) return 1.0;
  double w = 1.0;
  if ((refl(p, 0) && i == p->nx) || (refl(p, 1) && i == p->nx - 1)) w *= 0.5;
  if (p->dim == 2 && ((refl(p, 2) && j == p->ny) || (refl(p, 3) && j == p->ny - 1))) w *= 0.5;
  return w;
}

/* 1 if field f changes sign in the mirror image across a reflective wall (the
 * normal momentum): its average over the mirror-extended domain is 0. */
static int odd_field(const orc_problem* p, int f) {
  if (p->system != ORC_EULER) return 0;
  return (f == 1 && (refl(p, 0) || refl(p, 1))) || (p->dim == 2 && f == 2 && (refl(p, 2) || refl(p, 3)));
}

/* Global scales of one mesh, per field (Section 2.2, definition of sigma_K):
 *   avg(u) = (1/|Omega|) int_Omega u   (cell Gauss rule, stored cells only),
 *   sigma  = || u - avg(u) ||_{L^inf}, the max taken over the (k+1)^d Gauss
 *            points of every stored cell (parity unpinned: a convention).
 * With reflective walls Omega is the mirror-extended domain: wall-centred dual
 * cells count half in the average, a normal momentum has average 0 (its mirror
 * image is its negative), and the max of |u - avg| over the mirror images
 * equals that over the stored cells.
 * Reading of "sigma_K = 0" in floating point: a field that is constant in exact
 * arithmetic (a uniform density) carries rounding noise of an ulp or two in its
 * point values and in the rounded average, so its computed sigma is a few ulps
 * and the jumps it is divided into are of the same size; the ratio would damp
 * as hard as a shock.  A sigma at or below 2^-40 max|u| (max over the same
 * points, 4096 ulps of the field's magnitude) is therefore taken as 0. */
#define ORC_SIGMA_FLOOR 0x1p-40
static void mesh_sigma(const orc_problem* p, const real* u, int mesh, real* avg, real* sig) {
  int F = nfields(p), nq = p->k + 1, d = p->dim;
  double gx[ORC_MAXQ], gw[ORC_MAXQ];
  orc_gauss(nq, gx, gw);
  double hx = hx_of(p), hy = hy_of(p);
  int nqy = d == 2 ? nq : 1;
  int cy = ncy(p, mesh), cx = ncx(p, mesh);
  /* fixed summation order: each row of cells in sequence, then the rows in
   * sequence (the rows may be summed by different threads) */
  real* rows = (real*)calloc((size_t)cy * (F + 1), sizeof(real));
#pragma omp parallel for schedule(static)
  for (int j = 0; j < cy; ++j) {
    real v[ORC_MAXF];
    real* r = rows + (size_t)j * (F + 1);
    for (int i = 0; i < cx; ++i) {
      double wc = cell_weight(p, mesh, i, j);
      for (int qy = 0; qy < nqy; ++qy)
        for (int qx = 0; qx < nq; ++qx) {
          double W = 0.5 * gw[qx] * hx * (d == 2 ? 0.5 * gw[qy] * hy : 1.0);
          if (wc != 1.0) W *= wc;
          cell_eval(p, u, mesh, i, j, gx[qx], d == 2 ? gx[qy] : 0.0, 0, 0, v);
          for (int f = 0; f < F; ++f) r[f] += W * v[f];
          r[F] += W;
        }
    }
  }
  real vol = 0.0;
  real tot[ORC_MAXF] = {0};
  for (int j = 0; j < cy; ++j) {
    for (int f = 0; f < F; ++f) tot[f] += rows[(size_t)j * (F + 1) + f];
    vol += rows[(size_t)j * (F + 1) + F];
  }
  free(rows);
  for (int f = 0; f < F; ++f) {
    avg[f] = odd_field(p, f) ? 0.0 : tot[f] / vol;
    sig[f] = 0.0;
  }
  /* the max of |u - avg| and of |u| over all points (order-independent) */
  double mag[ORC_MAXF] = {0};
#pragma omp parallel
  {
    real loc[ORC_MAXF] = {0};
    double lmag[ORC_MAXF] = {0};
    real v[ORC_MAXF];
#pragma omp for schedule(static)
    for (int j = 0; j < cy; ++j)
      for (int i = 0; i < cx; ++i)
        for (int qy = 0; qy < nqy; ++qy)
          for (int qx = 0; qx < nq; ++qx) {
            cell_eval(p, u, mesh, i, j, gx[qx], d == 2 ? gx[qy] : 0.0, 0, 0, v);
            for (int f = 0; f < F; ++f) {
              real e = R_ABS(v[f] - avg[f]);
              if (RE(e) > RE(loc[f])) loc[f] = e;
              if (fabs(RE(v[f])) > lmag[f]) lmag[f] = fabs(RE(v[f]));
            }
          }
#pragma omp critical
    for (int f = 0; f < F; ++f) {
      if (RE(loc[f]) > RE(sig[f])) sig[f] = loc[f];
      if (lmag[f] > mag[f]) mag[f] = lmag[f];
    }
  }
  for (int f = 0; f < F; ++f)
    if (RE(sig[f]) <= ORC_SIGMA_FLOOR * mag[f]) sig[f] = 0.0;
}

static double factorial(int m) {
  double r = 1.0;
  for (int i = 2; i <= m; ++i) r *= i;
  return r;
}

/* Damping coefficients delta_K^m, m = 0..k, of stored cell (i, j) of mesh
 * `mesh` (Section 2.2):
 *   delta_K^m = sum_{e in dK} beta_{e,K} (2m+1) h_{e,K}^{m-1} / ((2k-1) m! sigma_K |e|)
 *               * int_e ( sum_{|alpha|=m} (d^alpha (u^C - u^D))^2 )^{1/2} ds,
 * delta = 0 where sigma_K = 0; for systems the max over the components of the
 * per-component value, for each m (Remark on systems).  u_K is K's own interior
 * trace on e, the overlapping solution is evaluated at the physical point;
 * every face is integrated as 2 half-faces with (k+1) Gauss points (1D: the
 * face is a point and the integral / |e| is the point value).
 * beta_{e,K} is the normal wave speed at K's cell average.
 * Returns 0, or ORC_ENONPHYSICAL if the cell average is not a physical state. */
static int cell_delta(const orc_problem* p, const real* u, int mesh, int i, int j, const real* sig,
                      real* delta /* [k+1] */) {
  int F = nfields(p), k = p->k, nq = k + 1, d = p->dim;
  int other = 1 - mesh;
  double gx[ORC_MAXQ], gw[ORC_MAXQ];
  orc_gauss(nq, gx, gw);
  double hx = hx_of(p), hy = hy_of(p);
  double xc, yc;
  cell_centre(p, mesh, i, j, &xc, &yc);
  real avg[ORC_MAXF];
  for (int f = 0; f < F; ++f) avg[f] = u[sidx(p, mesh, f, 0, j, i)]; /* mode 0 = cell average */
  real per_field[ORC_MAXF][ORC_MAXQ];
  memset(per_field, 0, sizeof per_field);
  int status = ORC_OK;

  for (int face = 0; face < 2 * d; ++face) {
    int dir = face / 2;
    double side = (face % 2) ? 1.0 : -1.0;
    double nxv = dir == 0 ? side : 0.0, nyv = dir == 1 ? side : 0.0;
    real beta = wave_speed(p, avg, nxv, nyv);
    if (RE(beta) < 0.0) { status = ORC_ENONPHYSICAL; beta = 0.0; }
    double he = dir == 0 ? hx : hy;                  /* h_{e,K}: cell width normal to e */
    double elen = d == 2 ? (dir == 0 ? hy : hx) : 1.0; /* |e| */
    for (int m = 0; m <= k; ++m) {
      real integ[ORC_MAXF] = {0};
      for (int s = 0; s < (d == 2 ? 2 : 1); ++s)
        for (int q = 0; q < (d == 2 ? nq : 1); ++q) {
          double t = d == 2 ? s - 0.5 + 0.5 * gx[q] : 0.0;
          double xi = dir == 0 ? side : t, eta = dir == 0 ? t : side;
          double W = d == 2 ? 0.5 * gw[q] * 0.5 * elen : 1.0;
          double x = xc + 0.5 * hx * xi, y = yc + 0.5 * hy * eta;
          int si, sj, mx, my;
          double oxi, oeta;
          locate(p, other, x, y, &si, &sj, &oxi, &oeta, &mx, &my);
          real sq[ORC_MAXF] = {0};
          for (int ax = 0; ax <= m; ++ax) {
            int ay = m - ax;
            if (d == 1 && ay > 0) continue;
            real a1[ORC_MAXF], a2[ORC_MAXF];
            cell_eval(p, u, mesh, i, j, xi, d == 2 ? eta : 0.0, ax, ay, a1);
            located_eval(p, u, other, si, sj, oxi, oeta, mx, my, ax, ay, a2);
            for (int f = 0; f < F; ++f) {
              real df = mesh == 0 ? a1[f] - a2[f] : a2[f] - a1[f]; /* u^C - u^D */
              sq[f] += df * df;
            }
          }
          for (int f = 0; f < F; ++f) integ[f] += W * R_SQRT(sq[f]);
        }
      real coef = beta * (2.0 * m + 1.0) * pow(he, m - 1.0) / ((2.0 * k - 1.0) * factorial(m) * elen);
      for (int f = 0; f < F; ++f)
        if (RE(sig[f]) != 0.0) per_field[f][m] += coef * integ[f] / sig[f];
    }
  }
  for (int m = 0; m <= k; ++m) {
    real mx = 0.0;
    for (int f = 0; f < F; ++f)
      if (RE(per_field[f][m]) > RE(mx)) mx = per_field[f][m];
    delta[m] = mx;
  }
  return status;
}

/* sigma and avg of both meshes (out arrays [2][F]) and delta of every cell
 * ([2][ny][nx][k+1] in the padded layout of the state).  Returns ORC_ENONPHYSICAL if any cell average is not a
 * physical state. */
int orc_oe_coefficients(const orc_problem* p, const real* u, real* delta, real* sigma, real* avg) {
  int F = nfields(p), K1 = p->k + 1;
  int status = ORC_OK;
  for (int mesh = 0; mesh < 2; ++mesh) {
    real a[ORC_MAXF], s[ORC_MAXF];
    mesh_sigma(p, u, mesh, a, s);
    for (int f = 0; f < F; ++f) {
      if (sigma) sigma[mesh * F + f] = s[f];
      if (avg) avg[mesh * F + f] = a[f];
    }
    int bad = 0;
    int cy = ncy(p, mesh), cx = ncx(p, mesh);
#pragma omp parallel for collapse(2) schedule(static) reduction(| : bad)
    for (int j = 0; j < cy; ++j)
      for (int i = 0; i < cx; ++i) {
        real dl[ORC_MAXQ];
        if (cell_delta(p, u, mesh, i, j, s, dl) != ORC_OK) bad = 1;
        for (int m = 0; m < K1; ++m) delta[(((size_t)mesh * nys(p) + j) * nxs(p) + i) * K1 + m] = dl[m];
      }
    if (bad) status = ORC_ENONPHYSICAL;
  }
  return status;
}

/* Decay factor of a mode of total degree deg >= 1 over the OE step of length
 * tau (Eq. (OEstep2D) solved exactly): exp(-tau sum_{m=0}^{min(deg,k)} delta^m). */
static real oe_factor(const orc_problem* p, const real* dl, int deg, real tau) {
  real rate = 0.0;
  for (int q = 0; q <= p->k && q <= deg; ++q) rate += dl[q];
  return R_EXP(-tau * rate);
}

/* Sampled evaluation for checks on meshes too large for a whole-mesh oracle
 * run: the same per-cell functions as orc_rhs / orc_oe_coefficients /
 * orc_oe_apply, applied to a list of cells only.  cells: n triples
 * (mesh, i, j) of stored cells (j = 0 in 1D).
 *   orc_rhs_cells: L of the listed cells, out [n][F][M].
 *   orc_oe_cells:  sigma and avg of both meshes (whole meshes, as in
 *                  orc_oe_coefficients; out [2][F] each, either may be NULL),
 *                  delta of the listed cells (out [n][k+1]) and, if usig is not
 *                  NULL, their coefficients after the OE step of length tau
 *                  (out [n][F][M]).  Returns ORC_ENONPHYSICAL if a listed
 *                  cell's average is not a physical state. */
void orc_rhs_cells(const orc_problem* p, const real* u, real tau_max, int n, const int* cells, real* L) {
  int F = nfields(p), M = nmodes(p);
  real inv = 1.0 / tau_max;
#pragma omp parallel for schedule(static)
  for (int c = 0; c < n; ++c) cell_rhs(p, u, inv, cells[3 * c], cells[3 * c + 1], cells[3 * c + 2], L + (size_t)c * F * M);
}

int orc_oe_cells(const orc_problem* p, const real* u, real tau, int n, const int* cells, real* delta,
                 real* sigma, real* avg, real* usig) {
  int F = nfields(p), K1 = p->k + 1;
  int ma[ORC_MAXM], mb[ORC_MAXM];
  int M = modes(p, ma, mb);
  real s[2][ORC_MAXF], a[2][ORC_MAXF];
  for (int mesh = 0; mesh < 2; ++mesh) {
    mesh_sigma(p, u, mesh, a[mesh], s[mesh]);
    for (int f = 0; f < F; ++f) {
      if (sigma) sigma[mesh * F + f] = s[mesh][f];
      if (avg) avg[mesh * F + f] = a[mesh][f];
    }
  }
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int c = 0; c < n; ++c) {
    int mesh = cells[3 * c], i = cells[3 * c + 1], j = cells[3 * c + 2];
    real dl[ORC_MAXQ];
    if (cell_delta(p, u, mesh, i, j, s[mesh], dl) != ORC_OK) bad = 1;
    for (int m = 0; m < K1; ++m) delta[(size_t)c * K1 + m] = dl[m];
    if (usig) {
      for (int m = 0; m < M; ++m) {
        real fac = m > 0 ? oe_factor(p, dl, ma[m] + mb[m], tau) : 1.0;
        for (int f = 0; f < F; ++f) usig[((size_t)c * F + f) * M + m] = u[sidx(p, mesh, f, m, j, i)] * fac;
      }
    }
  }
  return bad ? ORC_ENONPHYSICAL : ORC_OK;
}

/* Exact solution of the damping ODE (OEstep2D) at t_hat = tau.  In the
 * orthogonal Legendre basis, u - P^{m-1} u keeps exactly the modes of total
 * degree >= max(m, 1) (P^{-1} := P^0), so mode (a, b) obeys
 *   d/dt u_ab = -( sum_{m=0}^{min(a+b, k)} delta^m ) u_ab   for a + b >= 1,
 * and the cell average is untouched. */
void orc_oe_apply(const orc_problem* p, const real* delta, real tau, real* u) {
  int ma[ORC_MAXM], mb[ORC_MAXM];
  int M = modes(p, ma, mb), F = nfields(p), K1 = p->k + 1;
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int j = 0; j < ncy(p, mesh); ++j)
      for (int i = 0; i < ncx(p, mesh); ++i) {
        const real* dl = delta + (((size_t)mesh * nys(p) + j) * nxs(p) + i) * K1;
        for (int m = 1; m < M; ++m) {
          real fac = oe_factor(p, dl, ma[m] + mb[m], tau);
          for (int f = 0; f < F; ++f) u[sidx(p, mesh, f, m, j, i)] *= fac;
        }
      }
}

/* The OE step F_tau applied in place to both meshes.  k = 0 has no modes to
 * damp and (2k-1) < 0, so the step is the identity there. */
int orc_oe(const orc_problem* p, real* u, real tau) {
  if (p->k == 0) return ORC_OK;
  size_t nd = (size_t)2 * nys(p) * nxs(p) * (p->k + 1);
  real* delta = (real*)calloc(nd, sizeof(real));
  int st = orc_oe_coefficients(p, u, delta, NULL, NULL);
  orc_oe_apply(p, delta, tau, u);
  free(delta);
  return st;
}

/* ------------------------------------------------------------ time step --- */

/* tau_max from the CFL condition at the start of a step (Section 2.1 and
 * Section 4): 1D  C_CFL h / beta;  2D  C_CFL / (beta_x/h_x + beta_y/h_y), with
 * beta the maximum wave speed over the cell averages of both meshes.
 * Returns ORC_ENONPHYSICAL on a non-physical cell average. */
int orc_tau_max(const orc_problem* p, const real* u, real* tau_max) {
  int F = nfields(p);
  real bxm = 0.0, bym = 0.0;
  int st = ORC_OK;
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int j = 0; j < ncy(p, mesh); ++j)
      for (int i = 0; i < ncx(p, mesh); ++i) {
        real w[ORC_MAXF];
        for (int f = 0; f < F; ++f) w[f] = u[sidx(p, mesh, f, 0, j, i)];
        real sx = wave_speed(p, w, 1.0, 0.0);
        real sy = p->dim == 2 ? wave_speed(p, w, 0.0, 1.0) : 0.0;
        if (RE(sx) < 0.0 || RE(sy) < 0.0) { st = ORC_ENONPHYSICAL; continue; }
        if (RE(sx) > RE(bxm)) bxm = sx;
        if (RE(sy) > RE(bym)) bym = sy;
      }
  double hx = hx_of(p), hy = hy_of(p);
  real rate = bxm / hx + (p->dim == 2 ? bym / hy : 0.0);
  *tau_max = RE(rate) > 0.0 ? p->cfl / rate : 0.0;
  return st;
}

/* One stage combination of the Shu-Osher form: out = sum_m c_m U_m + tau d L(U_last). */
static void axpy_stage(size_t n, real* out, const real* a, double ca, const real* b, double cb,
                       const real* L, real cl) {
  for (size_t q = 0; q < n; ++q) out[q] = ca * a[q] + cb * b[q] + cl * L[q];
}

/* One full time step of Eq. (eq:RKCDG) in place: the stages of the chosen RK
 * method, each followed by the OE step F_tau (if enabled). */
int orc_step_tau(const orc_problem* p, real* u, real tau, real tau_max) {
  size_t n = state_len(p);
  real* L = (real*)calloc(n, sizeof(real)); /* the primal mesh's padding slots stay 0 */
  real* u1 = (real*)malloc(n * sizeof(real));
  real* u2 = (real*)malloc(n * sizeof(real));
  real* u3 = (real*)malloc(n * sizeof(real));
  int st = ORC_OK, s;
#define OE(x)                          \
  do {                                 \
    if (p->oe) {                       \
      s = orc_oe(p, (x), tau);         \
      if (s != ORC_OK) st = s;         \
    }                                  \
  } while (0)
  if (p->rk == 1) {
    orc_rhs(p, u, tau_max, L);
    axpy_stage(n, u1, u, 1.0, u, 0.0, L, tau);
    OE(u1);
    memcpy(u, u1, n * sizeof(real));
  } else if (p->rk == 2) {
    orc_rhs(p, u, tau_max, L);
    axpy_stage(n, u1, u, 1.0, u, 0.0, L, tau);
    OE(u1);
    orc_rhs(p, u1, tau_max, L);
    axpy_stage(n, u2, u, 0.5, u1, 0.5, L, 0.5 * tau);
    OE(u2);
    memcpy(u, u2, n * sizeof(real));
  } else if (p->rk == 3) {
    orc_rhs(p, u, tau_max, L);
    axpy_stage(n, u1, u, 1.0, u, 0.0, L, tau);
    OE(u1);
    orc_rhs(p, u1, tau_max, L);
    axpy_stage(n, u2, u, 0.75, u1, 0.25, L, 0.25 * tau);
    OE(u2);
    orc_rhs(p, u2, tau_max, L);
    axpy_stage(n, u3, u, 1.0 / 3.0, u2, 2.0 / 3.0, L, 2.0 / 3.0 * tau);
    OE(u3);
    memcpy(u, u3, n * sizeof(real));
  } else {
    /* classical RK4 in Shu-Osher form */
    real* u4 = (real*)malloc(n * sizeof(real));
    orc_rhs(p, u, tau_max, L);
    axpy_stage(n, u1, u, 1.0, u, 0.0, L, 0.5 * tau);
    OE(u1);
    orc_rhs(p, u1, tau_max, L);
    axpy_stage(n, u2, u, 1.0, u, 0.0, L, 0.5 * tau);
    OE(u2);
    orc_rhs(p, u2, tau_max, L);
    axpy_stage(n, u3, u, 1.0, u, 0.0, L, tau);
    OE(u3);
    orc_rhs(p, u3, tau_max, L);
    for (size_t q = 0; q < n; ++q)
      u4[q] = -u[q] / 3.0 + u1[q] / 3.0 + 2.0 * u2[q] / 3.0 + u3[q] / 3.0 + tau / 6.0 * L[q];
    OE(u4);
    memcpy(u, u4, n * sizeof(real));
    free(u4);
  }
#undef OE
  free(L);
  free(u1);
  free(u2);
  free(u3);
  return st;
}

/* Advance from time *t by up to nsteps steps, stopping at T_end (T_end <= 0: no
 * end time).  tau_max is recomputed at the start of every step; tau = tau_max,
 * except that the step that reaches T_end is clipped to T_end - t (and a step
 * that would leave a sliver shorter than 1e-12 T_end is stretched to T_end).
 * Returns the status; *t is advanced and *steps_done counts the steps taken. */
int orc_advance(const orc_problem* p, real* u, double* t, double T_end, int nsteps, int* steps_done) {
  int st = ORC_OK;
  int done = 0;
  for (int s = 0; s < nsteps; ++s) {
    if (T_end > 0.0 && *t >= T_end) break;
    real tm;
    int q = orc_tau_max(p, u, &tm);
    if (q != ORC_OK) { st = q; break; }
    real tau = tm;
    if (T_end > 0.0 && (T_end - (*t + RE(tm)) < 1e-12 * T_end)) tau = T_end - *t;
    q = orc_step_tau(p, u, tau, tm);
    if (q != ORC_OK) st = q;
    *t = (T_end > 0.0 && RE(tau) == T_end - *t) ? T_end : *t + RE(tau);
    ++done;
  }
  if (steps_done) *steps_done = done;
  return st;
}

#ifndef ORC_COMPLEX_STEP
/* ------------------------------------------------- initial projection --- */

/* A sampling point outside a reflective wall (the outer half of a
 * wall-centred dual cell) is folded back to its mirror image inside; *mx, *my
 * say whether it was (the initial data there is the mirror image of the data
 * inside: the normal momentum changes sign). */
static void fold_point(const orc_problem* p, double* x, double* y, int* mx, int* my) {
  *mx = *my = 0;
  if (refl(p, 0) && *x < p->ax) { *x = 2.0 * p->ax - *x; *mx = 1; }
  if (refl(p, 1) && *x > p->bx) { *x = 2.0 * p->bx - *x; *mx = 1; }
  if (p->dim == 2) {
    if (refl(p, 2) && *y < p->ay) { *y = 2.0 * p->ay - *y; *my = 1; }
    if (refl(p, 3) && *y > p->by) { *y = 2.0 * p->by - *y; *my = 1; }
  }
}

/* Physical sampling point (qx, qy) of sub-cell (sx, sy) of cell (i, j). */
static void sample_point(const orc_problem* p, int mesh, int i, int j, int sx, int sy, int qx, int qy,
                         const double* gx, double* x, double* y) {
  double xc, yc;
  cell_centre(p, mesh, i, j, &xc, &yc);
  double xi = sx - 0.5 + 0.5 * gx[qx];
  double eta = sy - 0.5 + 0.5 * gx[qy];
  *x = xc + 0.5 * hx_of(p) * xi;
  *y = p->dim == 2 ? yc + 0.5 * hy_of(p) * eta : 0.0;
}

/* Composite Gauss points for sampling the initial data: on every stored cell
 * of both meshes (the padded layout: the primal mesh's unused slots get the
 * points of the matching dual cell, whose values are ignored), (k+1)^d Gauss
 * points on each of its 2^d sub-cells, points beyond a reflective wall folded
 * back inside.  Layout: [mesh][j][i][sy][sx][qy][qx] with (x, y) pairs (1D: x
 * only, layout [mesh][i][sx][qx]).  Returns the number of points. */
size_t orc_quad_points(const orc_problem* p, double* xy) {
  int nq = p->k + 1, d = p->dim;
  double gx[ORC_MAXQ], gw[ORC_MAXQ];
  orc_gauss(nq, gx, gw);
  size_t n = 0;
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int j = 0; j < nys(p); ++j)
      for (int i = 0; i < nxs(p); ++i) {
        int cm = (i < ncx(p, mesh) && j < ncy(p, mesh)) ? mesh : 1; /* padding: any valid cell */
        for (int sy = 0; sy < (d == 2 ? 2 : 1); ++sy)
          for (int sx = 0; sx < 2; ++sx)
            for (int qy = 0; qy < (d == 2 ? nq : 1); ++qy)
              for (int qx = 0; qx < nq; ++qx) {
                if (xy) {
                  double x, y;
                  int mx, my;
                  sample_point(p, cm, i, j, sx, sy, qx, qy, gx, &x, &y);
                  fold_point(p, &x, &y, &mx, &my);
                  xy[n * d] = x;
                  if (d == 2) xy[n * d + 1] = y;
                }
                ++n;
              }
      }
  return n;
}

/* L^2 projection of sampled initial data onto both meshes (the
 * projection-based initialisation of Section 3.3), with the composite Gauss rule
 * of orc_quad_points: u_ab = (int_K u0 phi_ab) / ||phi_ab||^2.
 * vals layout: [point][F]. */
void orc_project(const orc_problem* p, const double* vals, double* u) {
  int ma[ORC_MAXM], mb[ORC_MAXM];
  int M = modes(p, ma, mb), F = nfields(p), nq = p->k + 1, d = p->dim;
  double gx[ORC_MAXQ], gw[ORC_MAXQ];
  orc_gauss(nq, gx, gw);
  int per_cell = (d == 2 ? 4 : 2) * (d == 2 ? nq * nq : nq);
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int j = 0; j < ncy(p, mesh); ++j)
      for (int i = 0; i < ncx(p, mesh); ++i) {
        size_t base = (((size_t)mesh * nys(p) + j) * nxs(p) + i) * per_cell;
        double acc[ORC_MAXF][ORC_MAXM];
        memset(acc, 0, sizeof acc);
        size_t n = 0;
        for (int sy = 0; sy < (d == 2 ? 2 : 1); ++sy)
          for (int sx = 0; sx < 2; ++sx)
            for (int qy = 0; qy < (d == 2 ? nq : 1); ++qy)
              for (int qx = 0; qx < nq; ++qx) {
                double xi = sx - 0.5 + 0.5 * gx[qx];
                double eta = sy - 0.5 + 0.5 * gx[qy];
                /* reference-square weights: the sub-cell has half the width */
                double W = 0.5 * gw[qx] * (d == 2 ? 0.5 * gw[qy] : 1.0);
                /* a point folded back across a wall carries the mirror image */
                double x, y;
                int mx, my;
                sample_point(p, mesh, i, j, sx, sy, qx, qy, gx, &x, &y);
                fold_point(p, &x, &y, &mx, &my);
                for (int m = 0; m < M; ++m) {
                  double ph = orc_legendre(ma[m], 0, xi) * (d == 2 ? orc_legendre(mb[m], 0, eta) : 1.0);
                  for (int f = 0; f < F; ++f) {
                    double v = vals[(base + n) * F + f];
                    if (p->system == ORC_EULER && ((mx && f == 1) || (my && f == 2))) v = -v;
                    acc[f][m] += W * v * ph;
                  }
                }
                ++n;
              }
        for (int m = 0; m < M; ++m) {
          /* ||phi||^2 on the reference cell [-1,1]^d */
          double nrm = 2.0 / (2.0 * ma[m] + 1.0) * (d == 2 ? 2.0 / (2.0 * mb[m] + 1.0) : 1.0);
          for (int f = 0; f < F; ++f) u[sidx(p, mesh, f, m, j, i)] = acc[f][m] / nrm;
        }
      }
}

/* ------------------------------------------------------------ utilities --- */

/* Evaluate the solution of mesh `mesh` (field values) at nq reference points
 * (xi[q], eta[q]) of every stored cell: out[j][i][q][F]. */
void orc_eval_cells(const orc_problem* p, const double* u, int mesh, int nq, const double* xi,
                    const double* eta, double* out) {
  int F = nfields(p);
  for (int j = 0; j < ncy(p, mesh); ++j)
    for (int i = 0; i < ncx(p, mesh); ++i)
      for (int q = 0; q < nq; ++q)
        cell_eval(p, u, mesh, i, j, xi[q], p->dim == 2 ? eta[q] : 0.0, 0, 0,
                  out + ((((size_t)j * nxs(p) + i) * nq + q) * F));
}

/* 0 if the problem description is valid, ORC_EINVAL otherwise: periodic on
 * both sides of a direction or on neither, reflective walls for the Euler
 * equations only (a wall reflects a velocity). */
int orc_check(const orc_problem* p) {
  for (int dir = 0; dir < p->dim; ++dir) {
    int lo = p->bc[2 * dir], hi = p->bc[2 * dir + 1];
    if (lo < 0 || lo > 2 || hi < 0 || hi > 2) return ORC_EINVAL;
    if ((lo == ORC_PERIODIC) != (hi == ORC_PERIODIC)) return ORC_EINVAL;
    if ((lo == ORC_REFLECTIVE || hi == ORC_REFLECTIVE) && p->system != ORC_EULER) return ORC_EINVAL;
  }
  return ORC_OK;
}

/* Evaluate the mesh-`mesh` solution at arbitrary physical points (located). */
void orc_eval_points(const orc_problem* p, const double* u, int mesh, size_t n, const double* xy, double* out) {
  int F = nfields(p), d = p->dim;
  for (size_t q = 0; q < n; ++q) point_eval(p, u, mesh, xy[q * d], d == 2 ? xy[q * d + 1] : 0.0, out + q * F);
}

#endif /* ORC_COMPLEX_STEP */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
