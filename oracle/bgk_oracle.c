/*
 * FP64 CPU oracle for one time step of the meshfree ALE / weighted-least-squares
 * scheme for the BGK equation (Mariappan, Willems, Boregowda, Tiwari, Klar,
 * arXiv 2408.02350).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA library never
 * links it, and the two share no code: this file includes nothing but libc (and,
 * in the second build made with -fopenmp to time the oracle on all host cores,
 * the OpenMP runtime; that build splits the loops over points among threads and
 * computes every point exactly as the plain build does).
 *
 * Plain, slow loops in IEEE double, written to be checked against the paper by
 * eye.  Built with -ffp-contract=off so that no multiply-add is fused.
 *
 * Layouts (all row-major, C order):
 *   x       [n][dim]               point positions
 *   kind    [n]                    0 interior, >0 wall id
 *   normal  [n][dim]               inward unit normal of a wall point
 *   cnt/col [n], [n][cap]          neighbour lists, ascending index per row
 *   f       [n][ncomp][NV]         ncomp = 2 in 2D (Chu g1, g2), 1 in 3D
 *   velocity index k = kx + nv*(ky + nv*kz)
 *
 * Readings of the paper taken where it is garbled or silent:
 *   - Maxwellian exponent carries a minus sign; the Chu G1 prefactor is
 *     rho/(2 pi R T) (Eqs. maxwellian, Maxw_G1).
 *   - In the upwind flux the second and third projected coefficients are beta
 *     and gamma, "sign(b |c.t|)" means sign(b)|c.t|, and the 3D third bracket
 *     uses c.b (Sec. 3.4.2).  The projected coefficients are the rows n, t, b
 *     of the frame matrix applied to (alpha, beta, gamma).
 *   - Nondimensional units R = 1, L = 1, rho0 = 1, T0 = 1, so
 *     tau = sqrt(2/pi) Kn / (rho sqrt(T)) (Eqs. tau, lambda).
 *   - Velocity nodes v_j = -vmax + j dv, j = 0..nv-1, dv = 2 vmax/(nv-1),
 *     quadrature weight dv per axis (Sec. 3.3); nv counts the nodes (N_v + 1).
 *   - Walls: diffuse reflection.  Velocities with (v - u_w).n <= 0 (n inward,
 *     u_w the wall velocity) are reconstructed from interior neighbours by a
 *     linear WLS fit (a constant fit where fewer than dim+1 interior neighbours
 *     exist); velocities with (v - u_w).n > 0 get rho_w M(v; 1, u_w, T_w), rho_w
 *     from zero net mass flux through the wall.
 *   - A rigid body's boundary points move with the body (Sec. 3.4.1); interior
 *     points are kept outside a guard sphere around its centre.
 *   - Sub-step order: neighbours and stencils, transport, moments, relaxation,
 *     boundary, point motion.  The transport uses U^n, the moments of the
 *     previous transported state (moments of f^0 at the first step).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t dim;       /* 2: Chu-reduced g1, g2 ; 3: full f */
  int32_t nv;        /* velocity nodes per axis */
  double vmax;
  double kn;         /* Knudsen number */
  int32_t tau_mode;  /* 0 local tau(rho,T); 1 constant sqrt(2/pi) Kn; 2 no collisions */
  int32_t ale;       /* 1: points move with U (Lagrangian form), transport with v - U */
  int32_t periodic;  /* 1: periodic unit box, minimum-image separations, no walls */
  int32_t lid_wall;  /* wall id that carries the lid velocity */
  int32_t max_nbrs;  /* neighbour-list capacity per point */
  int32_t pad_;
  double dt, h, alpha, wall_T, guard;
  double lid_u[3];
  /* Rigid body moving through the gas (Sec. 3.4.1: boundary points move with the
   * boundary).  body_wall > 0 is the wall id of its boundary points; they move with
   * the constant velocity body_u, which is also their wall velocity.  body_c is the
   * current centre of the body (advanced with the points by or_move and or_run);
   * interior points are kept at distance >= body_r + guard from it. */
  int32_t body_wall;
  /* order of the Taylor expansion behind the interior derivative stencils (Sec. 3.4.1):
   * 0 or 1 linear (the paper's scheme), 2 quadratic (its higher-order variant) */
  int32_t wls_order;
  double body_u[3];
  double body_c[3];
  double body_r;
  /* time discretisation: 0 or 1 the paper's first-order splitting (Sec. 3.2: explicit
   * transport, implicit relaxation); 2 a second-order variant the paper leaves to future
   * work: Strang splitting R(dt/2) T(dt) R(dt/2) with the exact relaxation solve and the
   * transport advanced by two explicit stages (SSP-RK2, Heun); fixed points only */
  int32_t time_order;
  /* velocity grid: 0 the paper's nv nodes with both ends at -vmax and vmax (Sec. 3.3),
   * 1 the midpoint grid, nv cells of width 2 vmax / nv with a node at each centre */
  int32_t vgrid;
} or_params;

enum { OR_OK = 0, OR_E_OVERFLOW = 1, OR_E_SINGULAR = 2, OR_E_INVAL = 3, OR_E_NOMEM = 4 };

static int ncomp_of(int dim) { return dim == 2 ? 2 : 1; }
static int64_t nvel_of(int dim, int nv) { return dim == 2 ? (int64_t)nv * nv : (int64_t)nv * nv * nv; }

/* ---- velocity grid (Sec. 3.3) ---- */

/* node spacing of the endpoint grid (vgrid 0) or the midpoint grid (vgrid 1) */
double or_dv_g(int32_t nv, double vmax, int32_t vgrid) {
  return vgrid == 1 ? 2.0 * vmax / (double)nv : 2.0 * vmax / (double)(nv - 1);
}
double or_dv(int32_t nv, double vmax) { return or_dv_g(nv, vmax, 0); }

/* Endpoint grid v_j = -vmax + j dv, midpoint grid v_j = -vmax + (j + 1/2) dv, both
 * written in the centred form (j - (nv-1)/2) dv, which is the same number in exact
 * arithmetic and makes the grid exactly symmetric in floating point (v_{nv-1-j} =
 * -v_j), so that a grazing velocity has v.n = 0 exactly on axis-aligned and diagonal
 * walls. */
void or_velocity_nodes_g(int32_t nv, double vmax, int32_t vgrid, double* v) {
  double dv = or_dv_g(nv, vmax, vgrid);
  for (int j = 0; j < nv; ++j) v[j] = ((double)j - 0.5 * (double)(nv - 1)) * dv;
}
void or_velocity_nodes(int32_t nv, double vmax, double* v) { or_velocity_nodes_g(nv, vmax, 0, v); }

/* vel[k][a] for the tensor-product grid, kx fastest. */
void or_velocity_grid_g(int32_t dim, int32_t nv, double vmax, int32_t vgrid, double* vel) {
  double* nodes = (double*)malloc(sizeof(double) * nv);
  or_velocity_nodes_g(nv, vmax, vgrid, nodes);
  int64_t NV = nvel_of(dim, nv);
  for (int64_t k = 0; k < NV; ++k) {
    int64_t r = k;
    for (int a = 0; a < dim; ++a) {
      vel[k * dim + a] = nodes[r % nv];
      r /= nv;
    }
  }
  free(nodes);
}
void or_velocity_grid(int32_t dim, int32_t nv, double vmax, double* vel) { or_velocity_grid_g(dim, nv, vmax, 0, vel); }

static double quad_weight(const or_params* p) {
  double dv = or_dv_g(p->nv, p->vmax, p->vgrid);
  return p->dim == 2 ? dv * dv : dv * dv * dv;
}

/* ---- kinetic model (Sec. 2) ---- */

/* Relaxation time, Eqs. (tau) and (lambda) in SI units. */
double or_tau_si(double kb, double R, double diam, double rho, double T) {
  const double pi = 3.14159265358979323846;
  double lambda = kb / (sqrt(2.0) * pi * rho * R * diam * diam);
  double cbar = sqrt(8.0 * R * T / pi);
  return 4.0 * lambda / (pi * cbar);
}

/* Mean free path, Eq. (lambda). */
double or_lambda_si(double kb, double R, double diam, double rho) {
  const double pi = 3.14159265358979323846;
  return kb / (sqrt(2.0) * pi * rho * R * diam * diam);
}

/* Nondimensional relaxation time: Eqs. (tau), (lambda) with R = L = rho0 = T0 = 1. */
double or_tau(const or_params* p, double rho, double T) {
  const double pi = 3.14159265358979323846;
  if (p->tau_mode == 1) return sqrt(2.0 / pi) * p->kn;
  return sqrt(2.0 / pi) * p->kn / (rho * sqrt(T));
}

/* Maxwellian at every node, Eq. (maxwellian) in 3D, Eqs. (Maxw_G1), (Maxw_G2) in 2D.
 * out[ncomp][NV]. */
void or_maxwellian(const or_params* p, double rho, const double* U, double T, double* out) {
  const double pi = 3.14159265358979323846;
  int dim = p->dim;
  int64_t NV = nvel_of(dim, p->nv);
  double* vel = (double*)malloc(sizeof(double) * NV * dim);
  or_velocity_grid_g(dim, p->nv, p->vmax, p->vgrid, vel);
  for (int64_t k = 0; k < NV; ++k) {
    double c2 = 0.0;
    for (int a = 0; a < dim; ++a) {
      double c = vel[k * dim + a] - U[a];
      c2 = c2 + c * c;
    }
    if (dim == 3) {
      out[k] = rho / pow(2.0 * pi * T, 1.5) * exp(-c2 / (2.0 * T));
    } else {
      double g1 = rho / (2.0 * pi * T) * exp(-c2 / (2.0 * T));
      out[k] = g1;
      out[NV + k] = T * g1;
    }
  }
  free(vel);
}

/* Moments of one point's distribution, Eqs. (moments), (internal_energy), (macroeq),
 * two-pass centred form.  fi[ncomp][NV] -> rho, U[dim], T. */
void or_moments_point(const or_params* p, const double* fi, double* rho, double* U, double* T) {
  int dim = p->dim;
  int64_t NV = nvel_of(dim, p->nv);
  double wv = quad_weight(p);
  double* vel = (double*)malloc(sizeof(double) * NV * dim);
  or_velocity_grid_g(dim, p->nv, p->vmax, p->vgrid, vel);
  double r = 0.0, mom[3] = {0.0, 0.0, 0.0};
  for (int64_t k = 0; k < NV; ++k) {
    r += fi[k] * wv;
    for (int a = 0; a < dim; ++a) mom[a] += vel[k * dim + a] * fi[k] * wv;
  }
  for (int a = 0; a < dim; ++a) U[a] = mom[a] / r;
  double e = 0.0;
  for (int64_t k = 0; k < NV; ++k) {
    double c2 = 0.0;
    for (int a = 0; a < dim; ++a) {
      double c = vel[k * dim + a] - U[a];
      c2 = c2 + c * c;
    }
    e += c2 * fi[k] * wv;
    if (dim == 2) e += fi[NV + k] * wv; /* + integral of g2, Eq. (macroeq) */
  }
  *rho = r;
  *T = e / (3.0 * r);
  free(vel);
}

/* ---- neighbour search (Sec. 3.5.1, Sec. 4.2) ---- */

static double sep(double xi, double xj, int periodic) {
  double d = xj - xi;
  if (periodic) {
    if (d > 0.5) d -= 1.0;
    else if (d < -0.5) d += 1.0;
  }
  return d;
}

/* Squared distance as dx*dx + dy*dy (+ dz*dz), left to right, no fused multiply-add. */
static double dist2(int dim, const double* xi, const double* xj, int periodic) {
  double d2 = 0.0;
  for (int a = 0; a < dim; ++a) {
    double d = sep(xi[a], xj[a], periodic);
    d2 = d2 + d * d;
  }
  return d2;
}

/* Definition: N(i) = { j != i : |x_j - x_i|^2 <= h^2 }, ascending j.  O(n^2).
 * Returns nnz, or -1 when a row exceeds cap (cnt then holds the true counts). */
int64_t or_neighbours_brute(int32_t dim, int64_t n, const double* x, double h, int32_t periodic,
                            int32_t cap, int32_t* cnt, int32_t* col) {
  double h2 = h * h;
  int64_t nnz = 0;
  int overflow = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      if (dist2(dim, x + i * dim, x + j * dim, periodic) <= h2) {
        if (c < cap) col[i * cap + c] = (int32_t)j;
        ++c;
      }
    }
    if (c > cap) overflow = 1;
    cnt[i] = c;
    nnz += c;
  }
  return overflow ? -1 : nnz;
}

/* Voxel (cell) search, as the paper's program does it: cells of side >= h,
 * each point scans its own and the adjacent cells, then the row is sorted.
 * Same contract as or_neighbours_brute. */
int64_t or_neighbours_cells(int32_t dim, int64_t n, const double* x, double h, int32_t periodic,
                            int32_t cap, int32_t* cnt, int32_t* col) {
  double h2 = h * h;
  int nc = (int)floor(1.0 / (h * (1.0 + 1e-9)));
  if (nc < 1) nc = 1;
  int64_t ncell = 1;
  for (int a = 0; a < dim; ++a) ncell *= nc;
  int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * n);
  int64_t* start = (int64_t*)calloc(ncell + 1, sizeof(int64_t));
  int64_t* fill = (int64_t*)calloc(ncell, sizeof(int64_t));
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0, stride = 1;
    for (int a = 0; a < dim; ++a) {
      int ca = (int)floor(x[i * dim + a] * nc);
      if (ca < 0) ca = 0;
      if (ca > nc - 1) ca = nc - 1;
      c += ca * stride;
      stride *= nc;
    }
    cell[i] = (int32_t)c;
    start[c + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  for (int64_t i = 0; i < n; ++i) order[start[cell[i]] + fill[cell[i]]++] = (int32_t)i;

  int64_t nnz = 0;
  int overflow = 0;
  for (int64_t i = 0; i < n; ++i) {
    int ci[3] = {0, 0, 0};
    int64_t r = cell[i];
    for (int a = 0; a < dim; ++a) { ci[a] = (int)(r % nc); r /= nc; }
    /* per-axis list of distinct cells to scan */
    int lst[3][3], len[3];
    for (int a = 0; a < 3; ++a) { len[a] = 1; lst[a][0] = 0; }
    for (int a = 0; a < dim; ++a) {
      len[a] = 0;
      if (periodic && nc < 3) {
        for (int c = 0; c < nc; ++c) lst[a][len[a]++] = c;
      } else {
        for (int o = -1; o <= 1; ++o) {
          int c = ci[a] + o;
          if (periodic) c = (c + nc) % nc;
          else if (c < 0 || c >= nc) continue;
          lst[a][len[a]++] = c;
        }
      }
    }
    int32_t m = 0;
    for (int u = 0; u < len[2]; ++u)
      for (int t = 0; t < len[1]; ++t)
        for (int s = 0; s < len[0]; ++s) {
          int64_t c = lst[0][s];
          if (dim >= 2) c += (int64_t)lst[1][t] * nc;
          if (dim >= 3) c += (int64_t)lst[2][u] * nc * nc;
          for (int64_t q = start[c]; q < start[c + 1]; ++q) {
            int32_t j = order[q];
            if (j == i) continue;
            if (dist2(dim, x + i * dim, x + (int64_t)j * dim, periodic) <= h2) cand[m++] = j;
          }
        }
    /* insertion sort, ascending index */
    for (int32_t a = 1; a < m; ++a) {
      int32_t v = cand[a], b = a - 1;
      while (b >= 0 && cand[b] > v) { cand[b + 1] = cand[b]; --b; }
      cand[b + 1] = v;
    }
    for (int32_t a = 0; a < m && a < cap; ++a) col[i * cap + a] = cand[a];
    if (m > cap) overflow = 1;
    cnt[i] = m;
    nnz += m;
  }
  free(cell); free(start); free(fill); free(order); free(cand);
  return overflow ? -1 : nnz;
}

/* ---- weighted least squares (Sec. 3.4.1) ---- */

/* Inverse of a small symmetric matrix (m <= 9) by Gauss-Jordan elimination with
 * partial pivoting.  Returns 0, or OR_E_SINGULAR when a pivot is not above tol * max|A|. */
static int gj_inverse(int m, const double* A, double* Ainv) {
  double a[9][18];
  double amax = 0.0;
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c) {
      a[r][c] = A[r * m + c];
      a[r][m + c] = (r == c) ? 1.0 : 0.0;
      if (fabs(a[r][c]) > amax) amax = fabs(a[r][c]);
    }
  if (!(amax > 0.0)) return OR_E_SINGULAR;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r) if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (!(fabs(a[piv][c]) > 1e-12 * amax)) return OR_E_SINGULAR;
    if (piv != c)
      for (int k = 0; k < 2 * m; ++k) { double t = a[c][k]; a[c][k] = a[piv][k]; a[piv][k] = t; }
    double d = a[c][c];
    for (int k = 0; k < 2 * m; ++k) a[c][k] /= d;
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      double fct = a[r][c];
      for (int k = 0; k < 2 * m; ++k) a[r][k] -= fct * a[c][k];
    }
  }
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c) Ainv[r * m + c] = a[r][m + c];
  return OR_OK;
}

/* Truncated Gaussian weight, Eq. (weight); callers pass only r <= h. */
static double weight(const or_params* p, double r2) { return exp(-p->alpha * r2 / (p->h * p->h)); }

/* Local frame of the pair (i, j) from the angles of Sec. 3.4.2:
 * 2D  n = (cos phi, sin phi), t = (-sin phi, cos phi), phi = atan2(dy, dx);
 * 3D  rows n, t, b of the matrix A, phi = atan2(dy, dx), theta = arccos(dz / r). */
void or_frame(int32_t dim, const double* dr, double* frame /* [dim][dim], rows n, t(, b) */) {
  if (dim == 2) {
    double phi = atan2(dr[1], dr[0]);
    frame[0] = cos(phi); frame[1] = sin(phi);
    frame[2] = -sin(phi); frame[3] = cos(phi);
  } else {
    double r = sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
    double phi = atan2(dr[1], dr[0]);
    double theta = acos(dr[2] / r);
    frame[0] = sin(theta) * cos(phi); frame[1] = sin(theta) * sin(phi); frame[2] = cos(theta);
    frame[3] = cos(theta) * cos(phi); frame[4] = cos(theta) * sin(phi); frame[5] = -sin(theta);
    frame[6] = -sin(phi);             frame[7] = cos(phi);              frame[8] = 0.0;
  }
}

/* Basis of the second-order Taylor fit at x_i for neighbour x_j: (dr, then the
 * products dr_a dr_b for a <= b, halved on the diagonal), dim + dim (dim + 1) / 2 entries. */
static void quad_basis(int dim, const double* xi, const double* xj, int periodic, double* b) {
  double dr[3];
  for (int a = 0; a < dim; ++a) dr[a] = sep(xi[a], xj[a], periodic);
  int k = 0;
  for (int a = 0; a < dim; ++a) b[k++] = dr[a];
  for (int a = 0; a < dim; ++a)
    for (int c = a; c < dim; ++c) b[k++] = a == c ? 0.5 * dr[a] * dr[a] : dr[a] * dr[c];
}

/* Stencils of every point.
 * Interior i: S = (M^T W M)^-1 (Eq. solution), gradient coefficients
 *   coef_j = w_j S dr_j, i.e. (alpha_ij, beta_ij, gamma_ij) of Eqs. (x_derivative)-(z_derivative);
 *   frame_j (rows n, t, b) and the projected coefficients abar_j = frame_j coef_j.
 * With wls_order = 2 the interior fit also carries the second derivatives (the
 * higher-order Taylor expansion of Sec. 3.4.1) and coef_j are the gradient rows of its
 * solution; frames and projected coefficients follow as above.
 * Wall b: linear WLS reconstruction over interior neighbours, p_j = (1, dr_j):
 *   recon_j = e_0^T (sum_k w_k p_k p_k^T)^-1 w_j p_j, so that f_b = sum_j recon_j f_j;
 *   with fewer than dim+1 interior neighbours (3D corners) the constant fit
 *   recon_j = w_j / sum_k w_k.
 * Slots of a row that do not apply are zero.  Returns OR_OK or OR_E_SINGULAR. */
int or_stencils(const or_params* p, int64_t n, const double* x, const int32_t* kind,
                const int32_t* cnt, const int32_t* col, double* coef, double* abar, double* frame,
                double* recon) {
  int dim = p->dim, cap = p->max_nbrs;
  int status = OR_OK;
  memset(coef, 0, sizeof(double) * n * cap * dim);
  memset(abar, 0, sizeof(double) * n * cap * dim);
  memset(frame, 0, sizeof(double) * n * cap * dim * dim);
  memset(recon, 0, sizeof(double) * n * cap);
  /* every point's stencil is independent (the OpenMP build splits the points over threads;
   * the arithmetic of each point is the same in either build) */
#pragma omp parallel for schedule(dynamic, 64) reduction(max : status)
  for (int64_t i = 0; i < n; ++i) {
    const double* xi = x + i * dim;
    if (kind[i] == 0 && p->wls_order == 2) {
      /* second-order Taylor expansion f_j - f_i = grad f . dr + 1/2 dr^T H dr: unknowns
       * q = (grad f, the dim (dim + 1) / 2 entries of H), basis b_j = (dr, dr_a dr_b /
       * (1 + [a == b])), coef_j = the gradient rows of (sum_k w_k b_k b_k^T)^-1 w_j b_j */
      const int mq = dim + dim * (dim + 1) / 2;
      double A[81] = {0}, S[81];
      for (int s = 0; s < cnt[i]; ++s) {
        const double* xj = x + (int64_t)col[i * cap + s] * dim;
        double b[9];
        quad_basis(dim, xi, xj, p->periodic, b);
        double w = weight(p, dist2(dim, xi, xj, p->periodic));
        for (int a = 0; a < mq; ++a)
          for (int c = 0; c < mq; ++c) A[a * mq + c] += w * b[a] * b[c];
      }
      if (cnt[i] < mq || gj_inverse(mq, A, S) != OR_OK) { status = OR_E_SINGULAR; continue; }
      for (int s = 0; s < cnt[i]; ++s) {
        int64_t slot = i * cap + s;
        const double* xj = x + (int64_t)col[slot] * dim;
        double dr[3], fr[9], b[9];
        for (int a = 0; a < dim; ++a) dr[a] = sep(xi[a], xj[a], p->periodic);
        quad_basis(dim, xi, xj, p->periodic, b);
        double w = weight(p, dist2(dim, xi, xj, p->periodic));
        for (int a = 0; a < dim; ++a) {
          double acc = 0.0;
          for (int c = 0; c < mq; ++c) acc += S[a * mq + c] * b[c];
          coef[slot * dim + a] = w * acc;
        }
        or_frame(dim, dr, fr);
        for (int d = 0; d < dim; ++d) {
          double acc = 0.0;
          for (int a = 0; a < dim; ++a) acc += fr[d * dim + a] * coef[slot * dim + a];
          abar[slot * dim + d] = acc;
        }
        for (int q = 0; q < dim * dim; ++q) frame[slot * dim * dim + q] = fr[q];
      }
    } else if (kind[i] == 0) {
      double A[9] = {0}, S[9];
      for (int s = 0; s < cnt[i]; ++s) {
        const double* xj = x + (int64_t)col[i * cap + s] * dim;
        double dr[3];
        for (int a = 0; a < dim; ++a) dr[a] = sep(xi[a], xj[a], p->periodic);
        double w = weight(p, dist2(dim, xi, xj, p->periodic));
        for (int a = 0; a < dim; ++a)
          for (int b = 0; b < dim; ++b) A[a * dim + b] += w * dr[a] * dr[b];
      }
      if (cnt[i] < dim || gj_inverse(dim, A, S) != OR_OK) { status = OR_E_SINGULAR; continue; }
      for (int s = 0; s < cnt[i]; ++s) {
        int64_t slot = i * cap + s;
        const double* xj = x + (int64_t)col[slot] * dim;
        double dr[3], fr[9];
        for (int a = 0; a < dim; ++a) dr[a] = sep(xi[a], xj[a], p->periodic);
        double w = weight(p, dist2(dim, xi, xj, p->periodic));
        for (int a = 0; a < dim; ++a) {
          double acc = 0.0;
          for (int b = 0; b < dim; ++b) acc += S[a * dim + b] * dr[b];
          coef[slot * dim + a] = w * acc;
        }
        or_frame(dim, dr, fr);
        for (int d = 0; d < dim; ++d) {
          double acc = 0.0;
          for (int a = 0; a < dim; ++a) acc += fr[d * dim + a] * coef[slot * dim + a];
          abar[slot * dim + d] = acc;
        }
        for (int q = 0; q < dim * dim; ++q) frame[slot * dim * dim + q] = fr[q];
      }
    } else {
      int m = dim + 1, ninner = 0;
      double B[16] = {0}, Binv[16];
      for (int s = 0; s < cnt[i]; ++s) {
        int32_t j = col[i * cap + s];
        if (kind[j] != 0) continue;
        const double* xj = x + (int64_t)j * dim;
        double pj[4];
        pj[0] = 1.0;
        for (int a = 0; a < dim; ++a) pj[1 + a] = sep(xi[a], xj[a], p->periodic);
        double w = weight(p, dist2(dim, xi, xj, p->periodic));
        for (int a = 0; a < m; ++a)
          for (int b = 0; b < m; ++b) B[a * m + b] += w * pj[a] * pj[b];
        ++ninner;
      }
      if (ninner == 0) { status = OR_E_SINGULAR; continue; }
      if (ninner < m) {
        /* too few interior neighbours for a linear fit: weighted mean (constant fit) */
        double wsum = 0.0;
        for (int s = 0; s < cnt[i]; ++s) {
          int32_t j = col[i * cap + s];
          if (kind[j] != 0) continue;
          wsum += weight(p, dist2(dim, xi, x + (int64_t)j * dim, p->periodic));
        }
        for (int s = 0; s < cnt[i]; ++s) {
          int32_t j = col[i * cap + s];
          if (kind[j] != 0) continue;
          recon[i * cap + s] = weight(p, dist2(dim, xi, x + (int64_t)j * dim, p->periodic)) / wsum;
        }
        continue;
      }
      if (gj_inverse(m, B, Binv) != OR_OK) { status = OR_E_SINGULAR; continue; }
      for (int s = 0; s < cnt[i]; ++s) {
        int32_t j = col[i * cap + s];
        if (kind[j] != 0) continue;
        const double* xj = x + (int64_t)j * dim;
        double pj[4];
        pj[0] = 1.0;
        for (int a = 0; a < dim; ++a) pj[1 + a] = sep(xi[a], xj[a], p->periodic);
        double w = weight(p, dist2(dim, xi, xj, p->periodic));
        double acc = 0.0;
        for (int b = 0; b < m; ++b) acc += Binv[b] * pj[b];
        recon[i * cap + s] = w * acc;
      }
    }
  }
  return status;
}

/* ---- point management (Sec. 3.5.2: removing and adding points) ---- */

/* Linear WLS reconstruction at the position y from the points k in src[0..m): p_k =
 * (1, x_k - y), w_k = exp(-alpha |x_k - y|^2 / h^2) (no cutoff), r_k = e_0^T (sum w p p^T)^-1
 * w_k p_k, so that f(y) = sum_k r_k f_k reproduces linear fields; the constant fit
 * w_k / sum w where m < dim + 1 or the system is singular. */
static void recon_at(const or_params* p, const double* y, const double* x, const int32_t* src, int m, double* r) {
  const int dim = p->dim, mm = dim + 1;
  double B[16] = {0}, Binv[16];
  for (int s = 0; s < m; ++s) {
    const double* xk = x + (int64_t)src[s] * dim;
    double pk[4];
    pk[0] = 1.0;
    for (int a = 0; a < dim; ++a) pk[1 + a] = sep(y[a], xk[a], p->periodic);
    double w = exp(-p->alpha * dist2(dim, y, xk, p->periodic) / (p->h * p->h));
    for (int u = 0; u < mm; ++u)
      for (int v = 0; v < mm; ++v) B[u * mm + v] += w * pk[u] * pk[v];
  }
  if (m < mm || gj_inverse(mm, B, Binv) != OR_OK) {
    double wsum = 0.0;
    for (int s = 0; s < m; ++s) {
      const double* xk = x + (int64_t)src[s] * dim;
      r[s] = exp(-p->alpha * dist2(dim, y, xk, p->periodic) / (p->h * p->h));
      wsum += r[s];
    }
    for (int s = 0; s < m; ++s) r[s] /= wsum;
    return;
  }
  for (int s = 0; s < m; ++s) {
    const double* xk = x + (int64_t)src[s] * dim;
    double pk[4];
    pk[0] = 1.0;
    for (int a = 0; a < dim; ++a) pk[1 + a] = sep(y[a], xk[a], p->periodic);
    double w = exp(-p->alpha * dist2(dim, y, xk, p->periodic) / (p->h * p->h));
    double acc = 0.0;
    for (int b = 0; b < mm; ++b) acc += Binv[b] * pk[b];
    r[s] = w * acc;
  }
}

/*
 * One pass of point management on the neighbour lists cnt/col of x (radius h).
 * Readings (the paper names the operations, not their thresholds):
 *  - remove next to a wall: an interior point closer than rmin to a wall point
 *    (any wall id, the body's included) is removed; the wall point stays on the
 *    boundary;
 *  - remove a pair: interior points i and j that stay after that, are each
 *    other's nearest such neighbour (ties to the smaller index) and are closer
 *    than rmin are replaced by one point at their midpoint (the survivor keeps
 *    i's slot, i < j);
 *  - add: an interior point i that takes part in no merge and has fewer than
 *    min_nbrs neighbours gets a new interior point at x_i - (h/2) c/|c|, c the
 *    sum of the separations to its neighbours (away from them, into the hole),
 *    if that position lies in [guard, 1 - guard]^dim (wrapped in a periodic box),
 *    outside the body's guard sphere (distance >= body_r + guard from body_c)
 *    and no point of N(i) + {i} is closer than rmin to it;
 *  - f at a new position y is the linear WLS reconstruction at y from
 *    N(i) + {i} (all point kinds), the least-squares update of the paper.
 * Output: the surviving points in index order (survivor slots take the
 * midpoint), then the added points in the order of the points that made them;
 * at most cap_out points (later additions are dropped).  origin[k] is the old
 * index of output point k, -1 for an added point.  counts[0] = merged pairs,
 * counts[1] = added points, counts[2] = points removed next to a wall.  Returns
 * the new point count.
 */
int64_t or_manage(const or_params* p, int64_t n, const double* x, const int32_t* kind, const double* normal,
                  const double* f, const int32_t* cnt, const int32_t* col, double rmin, int32_t min_nbrs,
                  int64_t cap_out, double* x_out, int32_t* kind_out, double* normal_out, double* f_out,
                  int64_t* origin, int64_t* counts) {
  const int dim = p->dim, cap = p->max_nbrs;
  const int64_t NV = nvel_of(dim, p->nv), row = (int64_t)ncomp_of(dim) * NV;
  const double rmin2 = rmin * rmin;
  int64_t* nn = (int64_t*)malloc(sizeof(int64_t) * n);
  /* 0 keep, 1 merge survivor, 2 merged away, 3 adds, 4 removed next to a wall */
  int32_t* role = (int32_t*)calloc(n, sizeof(int32_t));
  double* ynew = (double*)malloc(sizeof(double) * n * dim);
  int32_t* src = (int32_t*)malloc(sizeof(int32_t) * (cap + 1));
  double* r = (double*)malloc(sizeof(double) * (cap + 1));
  if (!nn || !role || !ynew || !src || !r) { free(nn); free(role); free(ynew); free(src); free(r); return -1; }
  /* interior points too close to a wall point */
  int64_t wall_removed = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (kind[i] != 0) continue;
    for (int s = 0; s < cnt[i]; ++s) {
      int32_t j = col[i * cap + s];
      if (kind[j] != 0 && dist2(dim, x + i * dim, x + (int64_t)j * dim, p->periodic) < rmin2) {
        role[i] = 4;
        ++wall_removed;
        break;
      }
    }
  }
  /* nearest interior neighbour among the points that stay */
  for (int64_t i = 0; i < n; ++i) {
    nn[i] = -1;
    if (kind[i] != 0 || role[i] == 4) continue;
    double best = 0.0;
    for (int s = 0; s < cnt[i]; ++s) {
      int32_t j = col[i * cap + s];
      if (kind[j] != 0 || role[j] == 4) continue;
      double d2 = dist2(dim, x + i * dim, x + (int64_t)j * dim, p->periodic);
      if (nn[i] < 0 || d2 < best) { nn[i] = j; best = d2; }
    }
    if (nn[i] >= 0 && !(best < rmin2)) nn[i] = -1;
  }
  /* mutual nearest pairs closer than rmin */
  int64_t merges = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t j = nn[i];
    if (j > i && nn[j] == i) { role[i] = 1; role[j] = 2; ++merges; }
  }
  /* additions into holes */
  for (int64_t i = 0; i < n; ++i) {
    if (kind[i] != 0 || role[i] != 0 || cnt[i] >= min_nbrs || cnt[i] == 0) continue;
    const double* xi = x + i * dim;
    double c[3] = {0.0, 0.0, 0.0}, c2 = 0.0;
    for (int s = 0; s < cnt[i]; ++s) {
      const double* xj = x + (int64_t)col[i * cap + s] * dim;
      for (int a = 0; a < dim; ++a) c[a] = c[a] + sep(xi[a], xj[a], p->periodic);
    }
    for (int a = 0; a < dim; ++a) c2 = c2 + c[a] * c[a];
    if (!(c2 > 0.0)) continue;
    const double cl = sqrt(c2), step = 0.5 * p->h;
    double* y = ynew + i * dim;
    int ok = 1;
    for (int a = 0; a < dim; ++a) {
      double ya = xi[a] - step * (c[a] / cl);
      if (p->periodic) {
        if (ya >= 1.0) ya -= 1.0;
        else if (ya < 0.0) ya += 1.0;
      } else if (ya < p->guard || ya > 1.0 - p->guard) {
        ok = 0;
      }
      y[a] = ya;
    }
    if (!ok) continue;
    if (p->body_wall > 0) {
      const double rg = p->body_r + p->guard;
      if (dist2(dim, y, p->body_c, 0) < rg * rg) continue;
    }
    if (dist2(dim, y, xi, p->periodic) < rmin2) continue;
    for (int s = 0; s < cnt[i] && ok; ++s)
      if (dist2(dim, y, x + (int64_t)col[i * cap + s] * dim, p->periodic) < rmin2) ok = 0;
    if (ok) role[i] = 3;
  }
  /* output: survivors, then additions */
  int64_t k = 0;
  for (int64_t i = 0; i < n && k < cap_out; ++i) {
    if (role[i] == 2 || role[i] == 4) continue;
    for (int a = 0; a < dim; ++a) normal_out[k * dim + a] = normal[i * dim + a];
    kind_out[k] = kind[i];
    origin[k] = i;
    if (role[i] == 1) {
      const int64_t j = nn[i];
      double* y = x_out + k * dim;
      for (int a = 0; a < dim; ++a) {
        double ya = x[i * dim + a] + 0.5 * sep(x[i * dim + a], x[j * dim + a], p->periodic);
        if (p->periodic) {
          if (ya >= 1.0) ya -= 1.0;
          else if (ya < 0.0) ya += 1.0;
        }
        y[a] = ya;
      }
      int m = 0;
      src[m++] = (int32_t)i;
      for (int s = 0; s < cnt[i]; ++s) src[m++] = col[i * cap + s];
      recon_at(p, y, x, src, m, r);
      for (int64_t q = 0; q < row; ++q) {
        double acc = 0.0;
        for (int s = 0; s < m; ++s) acc += r[s] * f[(int64_t)src[s] * row + q];
        f_out[k * row + q] = acc;
      }
    } else {
      for (int a = 0; a < dim; ++a) x_out[k * dim + a] = x[i * dim + a];
      memcpy(f_out + k * row, f + i * row, sizeof(double) * row);
    }
    ++k;
  }
  int64_t adds = 0;
  for (int64_t i = 0; i < n && k < cap_out; ++i) {
    if (role[i] != 3) continue;
    const double* y = ynew + i * dim;
    for (int a = 0; a < dim; ++a) { x_out[k * dim + a] = y[a]; normal_out[k * dim + a] = 0.0; }
    kind_out[k] = 0;
    origin[k] = -1;
    int m = 0;
    src[m++] = (int32_t)i;
    for (int s = 0; s < cnt[i]; ++s) src[m++] = col[i * cap + s];
    recon_at(p, y, x, src, m, r);
    for (int64_t q = 0; q < row; ++q) {
      double acc = 0.0;
      for (int s = 0; s < m; ++s) acc += r[s] * f[(int64_t)src[s] * row + q];
      f_out[k * row + q] = acc;
    }
    ++k;
    ++adds;
  }
  counts[0] = merges;
  counts[1] = adds;
  counts[2] = wall_removed;
  free(nn); free(role); free(ynew); free(src); free(r);
  return k;
}

/* Threads the loops over points use: 1 in the plain build, the OpenMP thread count in
 * the build with -fopenmp (used only to time the oracle on all host cores). */
int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---- explicit transport with the positive upwind flux (Eq. explicit, Sec. 3.4.2) ---- */

static double sgn(double a) { return a > 0.0 ? 1.0 : (a < 0.0 ? -1.0 : 0.0); }

/* Upwind coefficient of neighbour slot s for convective velocity c (Sec. 3.4.2):
 * abar_n [(c.n) - sign(abar_n)|c.n|] + abar_t [(c.t) - sign(abar_t)|c.t|] + abar_b [(c.b) - sign(abar_b)|c.b|],
 * i.e. sum_d (abar_d c_d - |abar_d||c_d|) with every direction treated alike.  The printed
 * normal term abar_n [(c.n) - |c.n|] is this form for abar_n > 0, which the linear fit
 * guarantees (abar_n = w r n^T S n with S positive definite); the second-order fit can give
 * abar_n < 0, where only the sign-aware form keeps every term non-positive. */
static double upwind_coef(int dim, const double* ab, const double* fr, const double* c) {
  double cn = 0.0, ct = 0.0, cb = 0.0;
  for (int a = 0; a < dim; ++a) {
    cn += c[a] * fr[a];
    ct += c[a] * fr[dim + a];
    if (dim == 3) cb += c[a] * fr[2 * dim + a];
  }
  double K = ab[0] * (cn - sgn(ab[0]) * fabs(cn)) + ab[1] * (ct - sgn(ab[1]) * fabs(ct));
  if (dim == 3) K += ab[2] * (cb - sgn(ab[2]) * fabs(cb));
  return K;
}

/* ft_i = f_i - dt Q(f)_i at one interior point i, Q = sum_j K_ij(v - U_i) (f_j - f_i);
 * U enters only with ale = 1.  vel is the velocity grid [NV][dim]. */
static void transport_point(const or_params* p, int64_t i, const int32_t* cnt, const int32_t* col,
                            const double* abar, const double* frame, const double* U, const double* f,
                            const double* vel, double* fti) {
  int dim = p->dim, cap = p->max_nbrs, nc = ncomp_of(dim);
  int64_t NV = nvel_of(dim, p->nv), row = nc * NV;
  const double* fi = f + i * row;
  for (int64_t k = 0; k < NV; ++k) {
    double c[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < dim; ++a) c[a] = vel[k * dim + a] - (p->ale ? U[i * dim + a] : 0.0);
    double Q[2] = {0.0, 0.0};
    for (int s = 0; s < cnt[i]; ++s) {
      int64_t slot = i * cap + s;
      const double* fj = f + (int64_t)col[slot] * row;
      double K = upwind_coef(dim, abar + slot * dim, frame + slot * dim * dim, c);
      for (int q = 0; q < nc; ++q) Q[q] += K * (fj[q * NV + k] - fi[q * NV + k]);
    }
    for (int q = 0; q < nc; ++q) fti[q * NV + k] = fi[q * NV + k] - p->dt * Q[q];
  }
}

/* Transport at every interior point; wall rows are copied. */
void or_transport(const or_params* p, int64_t n, const int32_t* kind, const int32_t* cnt,
                  const int32_t* col, const double* abar, const double* frame, const double* U,
                  const double* f, double* ft) {
  int dim = p->dim;
  int64_t NV = nvel_of(dim, p->nv), row = ncomp_of(dim) * NV;
  double* vel = (double*)malloc(sizeof(double) * NV * dim);
  or_velocity_grid_g(dim, p->nv, p->vmax, p->vgrid, vel);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    if (kind[i] != 0) { memcpy(ft + i * row, f + i * row, sizeof(double) * row); continue; }
    transport_point(p, i, cnt, col, abar, frame, U, f, vel, ft + i * row);
  }
  free(vel);
}

/* ---- moments and implicit relaxation (Sec. 3.2.1, 3.2.2) ---- */

void or_moments(const or_params* p, int64_t n, const double* f, double* rho, double* U, double* T) {
  int dim = p->dim;
  int64_t row = ncomp_of(dim) * nvel_of(dim, p->nv);
  for (int64_t i = 0; i < n; ++i) or_moments_point(p, f + i * row, rho + i, U + i * dim, T + i);
}

/* f^{n+1} = (tau ft + dt M^{n+1}) / (tau + dt) at one point, M^{n+1} from the moments
 * of ft (Eqs. fullmoment1a, moment1a, moment1b); the moments go to rho, U[dim], T. */
static void relax_point(const or_params* p, const double* fti, double* fi, double* M, double* rho,
                        double* U, double* T) {
  int64_t row = ncomp_of(p->dim) * nvel_of(p->dim, p->nv);
  or_moments_point(p, fti, rho, U, T);
  if (p->tau_mode == 2) { memcpy(fi, fti, sizeof(double) * row); return; }
  double tau = or_tau(p, *rho, *T);
  or_maxwellian(p, *rho, U, *T, M);
  for (int64_t q = 0; q < row; ++q) fi[q] = (tau * fti[q] + p->dt * M[q]) / (tau + p->dt);
}

/* Relaxation at every interior point; writes the moments of ft to rho, U, T. */
void or_relax(const or_params* p, int64_t n, const int32_t* kind, const double* ft, double* f,
              double* rho, double* U, double* T) {
  int dim = p->dim;
  int64_t row = ncomp_of(dim) * nvel_of(dim, p->nv);
#pragma omp parallel
  {
    double* M = (double*)malloc(sizeof(double) * row);  /* scratch of one thread */
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
      if (kind[i] != 0) continue;
      relax_point(p, ft + i * row, f + i * row, M, rho + i, U + i * dim, T + i);
    }
    free(M);
  }
}

/* Transport and relaxation of the listed interior points only (for spot checks of
 * large clouds): out[nidx][ncomp][NV] = f^{n+1}, mom_out[nidx][dim+2] = (rho, U, T). */
void or_transport_relax_points(const or_params* p, int64_t nidx, const int64_t* idx, const int32_t* cnt,
                               const int32_t* col, const double* abar, const double* frame,
                               const double* U, const double* f, double* out, double* mom_out) {
  int dim = p->dim;
  int64_t NV = nvel_of(dim, p->nv), row = ncomp_of(dim) * NV;
  double* vel = (double*)malloc(sizeof(double) * NV * dim);
  double* ft = (double*)malloc(sizeof(double) * row);
  double* M = (double*)malloc(sizeof(double) * row);
  or_velocity_grid_g(dim, p->nv, p->vmax, p->vgrid, vel);
  for (int64_t q = 0; q < nidx; ++q) {
    double* mo = mom_out + q * (dim + 2);
    transport_point(p, idx[q], cnt, col, abar, frame, U, f, vel, ft);
    relax_point(p, ft, out + q * row, M, mo, mo + 1, mo + 1 + dim);
  }
  free(vel); free(ft); free(M);
}

/* ---- second-order time discretisation (time_order = 2) ---- */

/* Exact solution of the relaxation df/dt = (M - f)/tau over a time h at one point.  The
 * relaxation keeps rho, U and T (and so M and tau), hence f(h) = M + (f - M) e^{-h/tau}
 * with M and tau from the moments of f.  The moments of f go to rho, U[dim], T. */
static void relax_exact_point(const or_params* p, double* fi, double h, double* M, double* rho, double* U,
                              double* T) {
  int64_t row = ncomp_of(p->dim) * nvel_of(p->dim, p->nv);
  or_moments_point(p, fi, rho, U, T);
  if (p->tau_mode == 2) return;
  double tau = or_tau(p, *rho, *T);
  double e = exp(-h / tau);
  or_maxwellian(p, *rho, U, *T, M);
  for (int64_t q = 0; q < row; ++q) fi[q] = M[q] + (fi[q] - M[q]) * e;
}

/* The exact relaxation over h at every interior point, in place. */
void or_relax_exact(const or_params* p, int64_t n, const int32_t* kind, double* f, double h) {
  int dim = p->dim;
  int64_t row = ncomp_of(dim) * nvel_of(dim, p->nv);
  double* M = (double*)malloc(sizeof(double) * row);
  double rho, U[3], T;
  for (int64_t i = 0; i < n; ++i)
    if (kind[i] == 0) relax_exact_point(p, f + i * row, h, M, &rho, U, &T);
  free(M);
}

/* ---- diffuse-reflection walls (Sec. 5.1, 5.2; Table 3) ---- */

/* At every wall point, with c_n = (v - u_w).n the normal velocity relative to the
 * wall: c_n <= 0 reconstructed, f_b = sum_j recon_j f_j; c_n > 0: rho_w M(v; 1, u_w, T_w)
 * with rho_w = sum_{c_n<=0} |c_n| g_b / sum_{c_n>0} c_n M(v; 1, u_w, T_w)  (g = first
 * component), so that no mass crosses the (moving) wall.  u_w is the lid velocity on
 * kind == lid_wall, the body velocity on kind == body_wall, zero elsewhere (the lid
 * moves tangentially, so there c_n = v.n).  Then the wall point's moments are taken
 * from f_b.  Returns OR_OK or OR_E_SINGULAR (no flux). */
int or_boundary(const or_params* p, int64_t n, const int32_t* kind, const double* normal,
                const int32_t* cnt, const int32_t* col, const double* recon, double* f,
                double* rho, double* U, double* T) {
  int dim = p->dim, cap = p->max_nbrs, nc = ncomp_of(dim);
  int64_t NV = nvel_of(dim, p->nv), row = nc * NV;
  int status = OR_OK;
  double* vel = (double*)malloc(sizeof(double) * NV * dim);
  or_velocity_grid_g(dim, p->nv, p->vmax, p->vgrid, vel);
  /* wall points are independent: each reads interior rows only and writes its own row */
#pragma omp parallel reduction(max : status)
  {
  double* Mw = (double*)malloc(sizeof(double) * row);  /* scratch of one thread */
#pragma omp for schedule(dynamic, 4)
  for (int64_t b = 0; b < n; ++b) {
    if (kind[b] == 0) continue;
    double* fb = f + b * row;
    const double* nb = normal + b * dim;
    double uw[3] = {0.0, 0.0, 0.0};
    if (kind[b] == p->lid_wall)
      for (int a = 0; a < dim; ++a) uw[a] = p->lid_u[a];
    if (p->body_wall > 0 && kind[b] == p->body_wall)
      for (int a = 0; a < dim; ++a) uw[a] = p->body_u[a];
    or_maxwellian(p, 1.0, uw, p->wall_T, Mw);
    double out_flux = 0.0, in_norm = 0.0;
    for (int64_t k = 0; k < NV; ++k) {
      double vn = 0.0;
      for (int a = 0; a < dim; ++a) vn += (vel[k * dim + a] - uw[a]) * nb[a];
      if (vn <= 0.0) {
        for (int q = 0; q < nc; ++q) {
          double acc = 0.0;
          for (int s = 0; s < cnt[b]; ++s) {
            int64_t slot = b * cap + s;
            if (kind[col[slot]] != 0) continue;
            acc += recon[slot] * f[(int64_t)col[slot] * row + q * NV + k];
          }
          fb[q * NV + k] = acc;
        }
        out_flux += -vn * fb[k];
      } else {
        in_norm += vn * Mw[k];
      }
    }
    if (!(in_norm > 0.0)) { status = OR_E_SINGULAR; continue; }
    double rho_w = out_flux / in_norm;
    for (int64_t k = 0; k < NV; ++k) {
      double vn = 0.0;
      for (int a = 0; a < dim; ++a) vn += (vel[k * dim + a] - uw[a]) * nb[a];
      if (vn > 0.0)
        for (int q = 0; q < nc; ++q) fb[q * NV + k] = rho_w * Mw[q * NV + k];
    }
    or_moments_point(p, fb, rho + b, U + b * dim, T + b);
  }
  free(Mw);
  }
  free(vel);
  return status;
}

/* ---- point motion (Eq. originalALE1, ALE1): x^{n+1} = x^n + dt U^{n+1} ---- */

/* Interior points: x += dt U.  Cavity: each coordinate is clamped to [guard, 1 - guard];
 * periodic box: wrapped into [0, 1).  With a body, its centre advances first,
 * c' = c + dt body_u, its boundary points move with it (x += dt body_u), and an
 * interior point that ends closer than rg = body_r + guard to c' is put back on that
 * sphere along the ray from c' (at c' + rg e_x if it sits on c' itself).  Returns the
 * number of clamps (one per clamped coordinate, one per point put back); p->body_c
 * becomes c'. */
int64_t or_move(or_params* p, int64_t n, const int32_t* kind, const double* U, double* x) {
  int dim = p->dim;
  int64_t clamps = 0;
  const int body = p->body_wall > 0;
  double cn[3] = {0.0, 0.0, 0.0};
  const double rg = p->body_r + p->guard, rg2 = rg * rg;
  if (body)
    for (int a = 0; a < dim; ++a) cn[a] = p->body_c[a] + p->dt * p->body_u[a];
  for (int64_t i = 0; i < n; ++i) {
    if (body && kind[i] == p->body_wall) {
      for (int a = 0; a < dim; ++a) x[i * dim + a] = x[i * dim + a] + p->dt * p->body_u[a];
      continue;
    }
    if (kind[i] != 0) continue;
    double y[3];
    for (int a = 0; a < dim; ++a) {
      double ya = x[i * dim + a] + p->dt * U[i * dim + a];
      if (p->periodic) {
        if (ya >= 1.0) ya -= 1.0;
        else if (ya < 0.0) ya += 1.0;
      } else if (ya < p->guard) { ya = p->guard; ++clamps; }
      else if (ya > 1.0 - p->guard) { ya = 1.0 - p->guard; ++clamps; }
      y[a] = ya;
    }
    if (body) {
      double d[3], r2 = 0.0;
      for (int a = 0; a < dim; ++a) {
        d[a] = y[a] - cn[a];
        r2 = r2 + d[a] * d[a];
      }
      if (r2 < rg2) {
        if (r2 > 0.0) {
          const double s = rg / sqrt(r2);
          for (int a = 0; a < dim; ++a) y[a] = cn[a] + d[a] * s;
        } else {
          for (int a = 0; a < dim; ++a) y[a] = cn[a] + (a == 0 ? rg : 0.0);
        }
        ++clamps;
      }
    }
    for (int a = 0; a < dim; ++a) x[i * dim + a] = y[a];
  }
  if (body)
    for (int a = 0; a < dim; ++a) p->body_c[a] = cn[a];
  return clamps;
}

/* ---- initial state (Sec. 2.1): f^0 = Maxwellian(rho0, U0, T0) everywhere ---- */

void or_init_maxwellian(const or_params* p, int64_t n, double rho0, const double* U0, double T0,
                        double* f, double* rho, double* U, double* T) {
  int dim = p->dim;
  int64_t row = ncomp_of(dim) * nvel_of(dim, p->nv);
  or_maxwellian(p, rho0, U0, T0, f);
  for (int64_t i = 1; i < n; ++i) memcpy(f + i * row, f, sizeof(double) * row);
  or_moments(p, n, f, rho, U, T);
}


/* ---- discrete adjoint of one step (fixed points, ale = 0) ----
 *
 * Not in the paper: the vector-Jacobian product of the step map
 * f^{n+1} = Phi(f^n; u_lid, Kn) written out from the forward sub-steps above,
 * for gradients of an objective J(f^1..f^N).  Given f^n and lam1 = dJ/df^{n+1}
 * it returns lam0 = (dPhi/df^n)^T lam1 and adds to dtheta[0..2] the derivative
 * with respect to the lid velocity and to dtheta[3] the one with respect to Kn.
 * Transport is linear for fixed points (K does not depend on f); relaxation is
 * differentiated through rho, U, T, tau and M; walls through the reconstruction
 * weights and rho_w = F / N (F the arriving normal mass flux, N the
 * normalisation of the wall Maxwellian, which depends on u_lid). */
int or_adjoint_step(const or_params* p, int64_t n, const int32_t* kind, const double* normal,
                    const int32_t* cnt, const int32_t* col, const double* abar, const double* frame,
                    const double* recon, const double* f, const double* lam1, double* lam0, double* dtheta) {
  int dim = p->dim, cap = p->max_nbrs, nc = ncomp_of(dim);
  int64_t NV = nvel_of(dim, p->nv), row = nc * NV;
  double wv = quad_weight(p);
  double Dm = dim == 2 ? 2.0 : 3.0; /* exponent of 2 pi T in the Maxwellian prefactor */
  double* vel = (double*)malloc(sizeof(double) * NV * dim);
  double* ft = (double*)malloc(sizeof(double) * n * row);
  double* y = (double*)malloc(sizeof(double) * n * row);
  double* lamy = (double*)calloc(n * row, sizeof(double));
  double* lamft = (double*)calloc(n * row, sizeof(double));
  double* Mw = (double*)malloc(sizeof(double) * row);
  double* M = (double*)malloc(sizeof(double) * row);
  double rho_, U_[3], T_;
  or_velocity_grid_g(dim, p->nv, p->vmax, p->vgrid, vel);

  /* forward recomputation of the step's intermediates */
  double zero3[3] = {0.0, 0.0, 0.0};
  (void)zero3;
  or_transport(p, n, kind, cnt, col, abar, frame, zero3, f, ft);
  memcpy(y, ft, sizeof(double) * n * row);
  for (int64_t i = 0; i < n; ++i) {
    if (kind[i] != 0) continue;
    relax_point(p, ft + i * row, y + i * row, M, &rho_, U_, &T_);
  }

  /* walls, backward: lamy (interior rows) = lam1 + contributions of the wall values */
  for (int64_t i = 0; i < n; ++i)
    if (kind[i] == 0) memcpy(lamy + i * row, lam1 + i * row, sizeof(double) * row);
  for (int64_t b = 0; b < n && !p->periodic; ++b) {
    if (kind[b] == 0) continue;
    const double* nb = normal + b * dim;
    double uw[3] = {0.0, 0.0, 0.0};
    int lid = kind[b] == p->lid_wall;
    if (lid) for (int a = 0; a < dim; ++a) uw[a] = p->lid_u[a];
    or_maxwellian(p, 1.0, uw, p->wall_T, Mw);
    /* F, N and rho_w of the forward wall step */
    double F = 0.0, N = 0.0, dN[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < NV; ++k) {
      double vn = 0.0;
      for (int a = 0; a < dim; ++a) vn += vel[k * dim + a] * nb[a];
      if (vn <= 0.0) {
        double g = 0.0;
        for (int s = 0; s < cnt[b]; ++s) {
          int64_t slot = b * cap + s;
          if (kind[col[slot]] != 0) continue;
          g += recon[slot] * y[(int64_t)col[slot] * row + k];
        }
        F += -vn * g;
      } else {
        N += vn * Mw[k];
        for (int a = 0; a < dim; ++a) dN[a] += vn * Mw[k] * (vel[k * dim + a] - uw[a]) / p->wall_T;
      }
    }
    double rho_w = F / N;
    /* mu = dJ/drho_w, and the lid-velocity derivative of the leaving values */
    const double* lb = lam1 + b * row;
    double mu = 0.0, du[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < NV; ++k) {
      double vn = 0.0;
      for (int a = 0; a < dim; ++a) vn += vel[k * dim + a] * nb[a];
      if (vn <= 0.0) continue;
      for (int q = 0; q < nc; ++q) {
        mu += lb[q * NV + k] * Mw[q * NV + k];
        for (int a = 0; a < dim; ++a)
          du[a] += lb[q * NV + k] * rho_w * Mw[q * NV + k] * (vel[k * dim + a] - uw[a]) / p->wall_T;
      }
    }
    if (lid)
      for (int a = 0; a < dim; ++a) dtheta[a] += du[a] - mu * rho_w / N * dN[a];
    /* arriving values f_b = sum_j r_bj y_j, and rho_w depends on them through F */
    for (int64_t k = 0; k < NV; ++k) {
      double vn = 0.0;
      for (int a = 0; a < dim; ++a) vn += (vel[k * dim + a] - uw[a]) * nb[a];
      if (vn > 0.0) continue;
      double l0 = lb[k] + mu * (-vn) / N;
      for (int s = 0; s < cnt[b]; ++s) {
        int64_t slot = b * cap + s;
        int32_t j = col[slot];
        if (kind[j] != 0) continue;
        lamy[(int64_t)j * row + k] += recon[slot] * l0;
        if (nc == 2) lamy[(int64_t)j * row + NV + k] += recon[slot] * lb[NV + k];
      }
    }
  }

  /* relaxation, backward, at interior points */
  for (int64_t i = 0; i < n; ++i) {
    if (kind[i] != 0) continue;
    const double* fti = ft + i * row;
    const double* ly = lamy + i * row;
    double* lf = lamft + i * row;
    double rho, U[3] = {0.0, 0.0, 0.0}, T;
    or_moments_point(p, fti, &rho, U, &T);
    double R = rho / wv;
    if (p->tau_mode == 2) { memcpy(lf, ly, sizeof(double) * row); continue; }
    double tau = or_tau(p, rho, T);
    double a = tau / (tau + p->dt), b = p->dt / (tau + p->dt);
    double dadtau = p->dt / ((tau + p->dt) * (tau + p->dt));
    or_maxwellian(p, rho, U, T, M);
    /* L = sum lam_y (a ft + b M): derivatives with respect to rho, U, T, Kn */
    double Af = 0.0, AM = 0.0, g_rho = 0.0, g_U[3] = {0.0, 0.0, 0.0}, g_T = 0.0;
    for (int64_t k = 0; k < NV; ++k) {
      double c2 = 0.0;
      for (int d = 0; d < dim; ++d) { double c = vel[k * dim + d] - U[d]; c2 += c * c; }
      double m0 = M[k];
      for (int q = 0; q < nc; ++q) { Af += ly[q * NV + k] * fti[q * NV + k]; AM += ly[q * NV + k] * M[q * NV + k]; }
      double lm = ly[k] + (nc == 2 ? T * ly[NV + k] : 0.0); /* M_1 = T M_0 */
      g_rho += b * lm * m0 / rho;
      for (int d = 0; d < dim; ++d) g_U[d] += b * lm * m0 * (vel[k * dim + d] - U[d]) / T;
      g_T += b * lm * m0 * (c2 / (2.0 * T * T) - Dm / (2.0 * T));
      if (nc == 2) g_T += b * ly[NV + k] * m0;
    }
    double dLda = Af - AM;
    if (p->tau_mode == 0) {
      g_rho += dLda * dadtau * (-tau / rho);
      g_T += dLda * dadtau * (-tau / (2.0 * T));
    }
    dtheta[3] += dLda * dadtau * tau / p->kn;
    /* chain to ft through rho = wv R, U = M/R, T = (E - R|U|^2)/(3R) */
    for (int64_t k = 0; k < NV; ++k) {
      double c2 = 0.0, gu = 0.0;
      for (int d = 0; d < dim; ++d) {
        double c = vel[k * dim + d] - U[d];
        c2 += c * c;
        gu += g_U[d] * c / R;
      }
      lf[k] = a * ly[k] + g_rho * wv + gu + g_T * (c2 - 3.0 * T) / (3.0 * R);
      if (nc == 2) lf[NV + k] = a * ly[NV + k] + g_T / (3.0 * R);
    }
  }

  /* transport, backward: ft_i = f_i (1 + dt sum_j K_ij) - dt sum_j K_ij f_j, scattered */
  memset(lam0, 0, sizeof(double) * n * row);
  for (int64_t i = 0; i < n; ++i) {
    if (kind[i] != 0) continue;
    for (int64_t k = 0; k < NV; ++k) {
      double c[3] = {0.0, 0.0, 0.0};
      for (int a = 0; a < dim; ++a) c[a] = vel[k * dim + a];
      for (int s = 0; s < cnt[i]; ++s) {
        int64_t slot = i * cap + s;
        int64_t j = col[slot];
        double K = upwind_coef(dim, abar + slot * dim, frame + slot * dim * dim, c);
        for (int q = 0; q < nc; ++q) {
          double l = lamft[i * row + q * NV + k];
          lam0[i * row + q * NV + k] += p->dt * K * l;
          lam0[j * row + q * NV + k] -= p->dt * K * l;
        }
      }
      for (int q = 0; q < nc; ++q) lam0[i * row + q * NV + k] += lamft[i * row + q * NV + k];
    }
  }
  free(vel); free(ft); free(y); free(lamy); free(lamft); free(Mw); free(M);
  return OR_OK;
}

/* Objective of one state: the x-momentum flux through the lid plane averaged over the
 * lid points, J = (1/|lid|) sum_{b in lid} sum_k v_x v_n g_b(v_k) dv^dim (v_n the last
 * velocity component, normal to the lid); lam += scale dJ/df when lam is not NULL. */
double or_objective(const or_params* p, int64_t n, const int32_t* kind, const double* f, double* lam, double scale) {
  int dim = p->dim;
  int64_t NV = nvel_of(dim, p->nv), row = ncomp_of(dim) * NV;
  double wv = quad_weight(p);
  double* vel = (double*)malloc(sizeof(double) * NV * dim);
  or_velocity_grid_g(dim, p->nv, p->vmax, p->vgrid, vel);
  int64_t nlid = 0;
  for (int64_t b = 0; b < n; ++b) nlid += kind[b] == p->lid_wall;
  double J = 0.0;
  for (int64_t b = 0; b < n && nlid > 0; ++b) {
    if (kind[b] != p->lid_wall) continue;
    for (int64_t k = 0; k < NV; ++k) {
      double w = vel[k * dim] * vel[k * dim + dim - 1] * wv / (double)nlid;
      J += w * f[b * row + k];
      if (lam) lam[b * row + k] += scale * w;
    }
  }
  free(vel);
  return J;
}

/* ---- full time steps ---- */

/* nsteps steps in place on (x, f, rho, U, T).  rho/U/T hold the moments of the
 * last transported state (interior) or of f_b (walls) and supply U^n on entry.
 * Neighbours and stencils are rebuilt every step with ale = 1, once otherwise.
 * With a body, p->body_c advances with the motion.
 * Returns OR_OK or an error code; *clamps accumulates wall-guard clamps. */
int or_run(or_params* p, int64_t n, double* x, const int32_t* kind, const double* normal,
           double* f, double* rho, double* U, double* T, int32_t nsteps, int64_t* clamps) {
  int dim = p->dim, cap = p->max_nbrs;
  int64_t row = ncomp_of(dim) * nvel_of(dim, p->nv);
  int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * n);
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * n * cap);
  double* coef = (double*)malloc(sizeof(double) * n * cap * dim);
  double* abar = (double*)malloc(sizeof(double) * n * cap * dim);
  double* frame = (double*)malloc(sizeof(double) * n * cap * dim * dim);
  double* recon = (double*)malloc(sizeof(double) * n * cap);
  double* ft = (double*)malloc(sizeof(double) * n * row);
  const int second = p->time_order == 2;
  double* f2 = second ? (double*)malloc(sizeof(double) * n * row) : NULL;
  double* mom2 = second ? (double*)malloc(sizeof(double) * n * (dim + 2)) : NULL;
  int status = OR_OK;
  if (!cnt || !col || !coef || !abar || !frame || !recon || !ft || (second && (!f2 || !mom2))) {
    status = OR_E_NOMEM;
    goto done;
  }
  if (second && p->ale) { status = OR_E_INVAL; goto done; }
  for (int32_t s = 0; s < nsteps; ++s) {
    if (s == 0 || p->ale) {
      if (or_neighbours_cells(dim, n, x, p->h, p->periodic, cap, cnt, col) < 0) { status = OR_E_OVERFLOW; goto done; }
      if ((status = or_stencils(p, n, x, kind, cnt, col, coef, abar, frame, recon)) != OR_OK) goto done;
    }
    if (second) {
      /* f^{n+1} = R(dt/2) T(dt) R(dt/2) f^n; T by two explicit stages with the walls applied
       * to each stage, f^T = (f + T1(T1 f))/2 with T1 the first-order transport */
      or_relax_exact(p, n, kind, f, 0.5 * p->dt);
      or_transport(p, n, kind, cnt, col, abar, frame, U, f, ft);
      if (!p->periodic)
        if ((status = or_boundary(p, n, kind, normal, cnt, col, recon, ft, mom2, mom2 + n, mom2 + n * (1 + dim))) !=
            OR_OK)
          goto done;
      or_transport(p, n, kind, cnt, col, abar, frame, U, ft, f2);
      double* M = (double*)malloc(sizeof(double) * row);
      for (int64_t i = 0; i < n; ++i) {
        if (kind[i] != 0) continue;
        double* fi = f + i * row;
        for (int64_t q = 0; q < row; ++q) fi[q] = 0.5 * (fi[q] + f2[i * row + q]);
        relax_exact_point(p, fi, 0.5 * p->dt, M, rho + i, U + i * dim, T + i);
      }
      free(M);
    } else {
      or_transport(p, n, kind, cnt, col, abar, frame, U, f, ft);
      or_relax(p, n, kind, ft, f, rho, U, T);
    }
    if (!p->periodic)
      if ((status = or_boundary(p, n, kind, normal, cnt, col, recon, f, rho, U, T)) != OR_OK) goto done;
    if (p->ale) {
      int64_t c = or_move(p, n, kind, U, x);
      if (clamps) *clamps += c;
    }
  }
done:
  free(cnt); free(col); free(coef); free(abar); free(frame); free(recon); free(ft); free(f2); free(mom2);
  return status;
}
