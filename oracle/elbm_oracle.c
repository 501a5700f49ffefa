/*
 * elbm_oracle.c -- plain FP64 CPU oracle of the entropic lattice Boltzmann
 * method with the relaxation-rate formula (Zhao & Yong).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the product path.  It shares no code
 * with the CUDA library.  It is written to be read against the paper: every
 * function follows one passage, in the paper's order and notation, with no
 * blocking, fusion or reordering.  Compile with -ffp-contract=off.
 *
 * Which passage each function follows:
 *   orc_equilibrium      entropic equilibrium minimising Eq. (3) under the
 *                        mass/momentum constraints stated after Eq. (3); the
 *                        paper cites the analytic D2Q9 form (its ref. AKO2003)
 *                        in the double-shear-layer experiment; the tensor
 *                        product form below is that form for D1Q3/D2Q9/D3Q27
 *   orc_entropy          Eq. (3)
 *   orc_delta_h          H(f*(alpha)) - H(f) of Eqs. (4) and (7)
 *   orc_alpha_max        the alpha_max definition preceding Fig. 1
 *   alpha_formula        Eq. (8), the acceptance test after it, Eq. (9)
 *   alpha_root           bisection on Eq. (4) with the stop rule
 *                        -1e-13 <= H(f*(alpha)) - H(f) <= 0 quoted for the
 *                        double shear layer
 *   alpha_secant         the modified secant iteration of the conclusion
 *   orc_collide_node     Eq. (1) = Eq. (5a) at one node
 *   orc_step             Eq. (5a) at every node, then Eq. (5b) (periodic)
 *   orc_enstrophy        1/2 <|curl u|^2> by central differences (the
 *                        diagnostic of the Taylor-Green histories; not in the
 *                        paper), pinned to closed forms for single-mode flows
 */
#include "elbm_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_QMAX 27
#define ROOT_TOL 1e-13      /* stop rule of the bisection comparison */
#define ROOT_MAX_ITERS 64   /* iteration cap (reading: the paper sets none) */

/* ------------------------------------------------------------------------ */
/* Lattices: rest velocity first, then +/- pairs.  Weights are products of  */
/* the D1Q3 weights {2/3, 1/6, 1/6}; c_s^2 = 1/3, dt = 1.                   */
/* ------------------------------------------------------------------------ */
static const int C_D1Q3[3][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}};
static const double W_D1Q3[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};

static const int C_D2Q9[9][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
static const double W_D2Q9[9] = {
    4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const int C_D3Q27[27][3] = {
    {0, 0, 0},                                                /* rest   */
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},        /* faces  */
    {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},        /* edges  */
    {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},
    {1, 1, 1},   {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},       /* corners */
    {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
static const double W_D3Q27[27] = {
    8.0 / 27.0,
    2.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0,
    1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,
    1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,
    1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0,
    1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0};

typedef struct {
  int d, q;
  const int (*c)[3];
  const double *w;
} lat_t;

static int get_lattice(int lattice, lat_t *L) {
  switch (lattice) {
    case ORC_D1Q3: L->d = 1; L->q = 3; L->c = C_D1Q3; L->w = W_D1Q3; return 0;
    case ORC_D2Q9: L->d = 2; L->q = 9; L->c = C_D2Q9; L->w = W_D2Q9; return 0;
    case ORC_D3Q27: L->d = 3; L->q = 27; L->c = C_D3Q27; L->w = W_D3Q27; return 0;
    default: return -1;
  }
}

int orc_lattice(int lattice, int *c_out, double *w_out) {
  lat_t L;
  if (get_lattice(lattice, &L)) return -1;
  for (int i = 0; i < L.q; i++) {
    for (int a = 0; a < 3; a++) c_out[3 * i + a] = L.c[i][a];
    w_out[i] = L.w[i];
  }
  return L.q;
}

int orc_lattice_dim(int lattice) {
  lat_t L;
  return get_lattice(lattice, &L) ? -1 : L.d;
}

int orc_lattice_q(int lattice) {
  lat_t L;
  return get_lattice(lattice, &L) ? -1 : L.q;
}

/* ------------------------------------------------------------------------ */
/* Entropic equilibrium.  The minimiser of H = sum f ln(f/W) under          */
/* sum f = rho, sum c f = rho u is f^eq_i = W_i exp(a + b.c_i).  On the      */
/* tensor-product lattices it factorises per axis:                          */
/*   f^eq_i = rho W_i prod_a (2 - s_a) r_a^{c_ia},                          */
/*   s_a = sqrt(1 + 3 u_a^2),  r_a = (2 u_a + s_a) / (1 - u_a).             */
/* ------------------------------------------------------------------------ */
int orc_equilibrium(int lattice, double rho, const double *u, double *feq) {
  lat_t L;
  if (get_lattice(lattice, &L)) return -1;
  if (!(rho > 0.0)) return -1;
  double s[3], r[3];
  for (int a = 0; a < L.d; a++) {
    if (!(fabs(u[a]) < 1.0)) return -1;
    s[a] = sqrt(1.0 + 3.0 * u[a] * u[a]);
    r[a] = (2.0 * u[a] + s[a]) / (1.0 - u[a]);
  }
  for (int i = 0; i < L.q; i++) {
    double p = rho * L.w[i];
    for (int a = 0; a < L.d; a++) {
      p *= (2.0 - s[a]);
      if (L.c[i][a] == 1) p *= r[a];
      if (L.c[i][a] == -1) p /= r[a];
    }
    feq[i] = p;
  }
  return 0;
}

/* Eq. (3): H(f) = sum_i f_i ln(f_i / W_i), with 0 ln 0 = 0. */
double orc_entropy(int lattice, const double *f) {
  lat_t L;
  if (get_lattice(lattice, &L)) return NAN;
  double h = 0.0;
  for (int i = 0; i < L.q; i++)
    if (f[i] > 0.0) h += f[i] * log(f[i] / L.w[i]);
  return h;
}

/* ------------------------------------------------------------------------ */
/* Entropy change along the ray f*(alpha) = f + alpha (f^eq - f), Eq. (4).  */
/* With f*_i = f_i (1 + alpha x_i), x_i = f^eq_i / f_i - 1, and              */
/* ln(f_i/W_i) = ln(f^eq_i/W_i) - ln(1 + x_i):                               */
/*   H(f*) - H(f) = sum f_i (1 + alpha x_i) ln(1 + alpha x_i)                */
/*                - alpha sum f_i x_i ln(1 + x_i)                            */
/*                + alpha sum (f^eq_i - f_i) ln(f^eq_i / W_i).               */
/* The last sum is 0 (ln(f^eq/W) is a combination of the collision           */
/* invariants 1, c and f^eq - f carries no mass or momentum), and so is      */
/* alpha sum f_i x_i = alpha sum (f^eq_i - f_i).  Removing both zero terms   */
/* from the sum (they only add rounding noise) leaves                        */
/*   Delta H(alpha) = sum f_i [phi(alpha x_i) - alpha x_i ln(1 + x_i)],      */
/*   phi(y) = (1 + y) ln(1 + y) - y.                                         */
/* At alpha = alpha_max one f*_i is 0: phi(-1) = 1 (0 ln 0 := 0).            */
/* ------------------------------------------------------------------------ */
static double phi(double y) {
  if (y <= -1.0) return 1.0;
  if (fabs(y) < 0.1) {
    /* phi(y) = sum_{k>=2} (-1)^k y^k / (k (k-1)), summed until negligible */
    double term = y * y, sum = 0.0;
    for (int k = 2; k < 40; k++) {
      double t = term / (double)(k * (k - 1));
      sum += (k % 2 == 0) ? t : -t;
      if (fabs(t) < 1e-18 * fabs(sum)) break;
      term *= y;
    }
    return sum;
  }
  return (1.0 + y) * log1p(y) - y;
}

double orc_delta_h(int q, const double *f, const double *x, double alpha) {
  double sum = 0.0;
  for (int i = 0; i < q; i++) {
    double y = alpha * x[i];
    sum += f[i] * (phi(y) - y * log1p(x[i]));
  }
  return sum;
}

/* Bound on |computed - exact| Delta H(alpha) at the given alpha:
 *   summation and log rounding:  64 eps sum f (|phi(y)| + |y ln(1+x)|);
 *   rounding of x_i from rho, u and f^eq (|dx_i| <= 4 q eps (1 + |x_i|)),
 *   through d/dx_i of the bracket, alpha (ln(1+alpha x) - ln(1+x) - x/(1+x));
 *   one rounding of alpha itself, 4 eps alpha |d Delta H / d alpha|,
 *   d Delta H / d alpha = sum f x (ln(1 + alpha x) - ln(1 + x)).
 * A node violates the H-inequality Eq. (7) when Delta H exceeds this. */
double orc_delta_h_bound(int q, const double *f, const double *x,
                         double alpha) {
  double mag = 0.0, prop = 0.0, slope = 0.0;
  for (int i = 0; i < q; i++) {
    double y = alpha * x[i];
    double ly = (1.0 + y > 1e-300) ? log1p(y) : log(1e-300);
    double lx = log1p(x[i]);
    mag += f[i] * (fabs(phi(y)) + fabs(y * lx));
    prop += f[i] * (1.0 + fabs(x[i])) * alpha *
            fabs(ly - lx - x[i] / (1.0 + x[i]));
    slope += f[i] * x[i] * (ly - lx);
  }
  return DBL_EPSILON *
         (64.0 * mag + 4.0 * q * prop + 4.0 * alpha * fabs(slope));
}

double orc_delta_h_literal(int lattice, const double *f, const double *feq,
                           double alpha) {
  lat_t L;
  if (get_lattice(lattice, &L)) return NAN;
  double fs[ORC_QMAX];
  for (int i = 0; i < L.q; i++) {
    fs[i] = f[i] + alpha * (feq[i] - f[i]);
    if (fs[i] < 0.0) fs[i] = 0.0; /* only at alpha = alpha_max, by rounding */
  }
  return orc_entropy(lattice, fs) - orc_entropy(lattice, f);
}

/* alpha_max = min_{i: f^eq_i < f_i} f_i / (f_i - f^eq_i). */
double orc_alpha_max(int q, const double *f, const double *feq) {
  double am = INFINITY;
  for (int i = 0; i < q; i++) {
    if (feq[i] < f[i]) {
      double a = f[i] / (f[i] - feq[i]);
      if (a < am) am = a;
    }
  }
  return am;
}

/* ------------------------------------------------------------------------ */
/* Choices of alpha.  All three start from alpha_* = min(2, alpha_max),      */
/* Eq. (8), and D_* = Delta H(alpha_*).                                      */
/* ------------------------------------------------------------------------ */

/* Eq. (8) + acceptance test + Eq. (9). */
static double alpha_formula(int q, const double *f, const double *x,
                            double alpha_star, int *flags) {
  double d_star = orc_delta_h(q, f, x, alpha_star);
  if (d_star <= 0.0) {
    *flags |= ORC_F_ACCEPT_STAR;
    if (alpha_star == 2.0) *flags |= ORC_F_ACCEPT_TWO;
    return alpha_star;
  }
  /* H(f*(alpha_*)) - H(f^eq) = D_* - Delta H(1), since f*(1) = f^eq. */
  double d_one = orc_delta_h(q, f, x, 1.0);
  *flags |= ORC_F_FORMULA;
  /* d_star - d_one = H(f*(alpha_*)) - H(f^eq) > 0 in exact arithmetic; a
   * non-positive value means f equals f^eq to rounding: take alpha = 1
   * (f* = f^eq). */
  if (!(d_star - d_one > 0.0)) return 1.0;
  return alpha_star + d_star / (d_star - d_one) * (1.0 - alpha_star);
}

/* Bisection for the root of Eq. (4) on [1, alpha_max], where Delta H is
 * convex and increasing; stop when -1e-13 <= Delta H <= 0. */
static double alpha_root(int q, const double *f, const double *x,
                         double alpha_max, int *flags, int *iters) {
  double lo = 1.0, hi = alpha_max;
  if (orc_delta_h(q, f, x, hi) <= 0.0) {
    /* no root inside the admissible range (reading: take alpha_max) */
    *flags |= ORC_F_NO_ROOT;
    return hi;
  }
  for (int k = 0; k < ROOT_MAX_ITERS; k++) {
    double mid = 0.5 * (lo + hi);
    double d = orc_delta_h(q, f, x, mid);
    (*iters)++;
    if (d >= -ROOT_TOL && d <= 0.0) return mid;
    if (d > 0.0)
      hi = mid;
    else
      lo = mid;
    if (hi - lo < 1e-15 * hi) return lo;
  }
  *flags |= ORC_F_ROOT_CAP;
  return lo;
}

/* Modified secant iteration from the conclusion, alpha^(0) = 1, so the
 * first iterate is Eq. (9).  Stops after n_iter iterates or when the
 * bisection stop rule holds. */
static double alpha_secant(int q, const double *f, const double *x,
                           double alpha_star, int n_iter, int *flags,
                           int *iters) {
  double d_star = orc_delta_h(q, f, x, alpha_star);
  if (d_star <= 0.0) {
    *flags |= ORC_F_ACCEPT_STAR;
    if (alpha_star == 2.0) *flags |= ORC_F_ACCEPT_TWO;
    return alpha_star;
  }
  *flags |= ORC_F_FORMULA;
  double a = 1.0;
  double d_a = orc_delta_h(q, f, x, a);
  if (!(d_star - d_a > 0.0)) return 1.0; /* f == f^eq to rounding */
  /* The iterates keep Delta H <= 0 in exact arithmetic; an iterate whose
   * computed Delta H is positive (rounding) ends the iteration at the
   * previous iterate. */
  for (int k = 0; k < n_iter; k++) {
    double a_next = alpha_star + d_star / (d_star - d_a) * (a - alpha_star);
    double d_next = orc_delta_h(q, f, x, a_next);
    (*iters)++;
    if (d_next > 0.0) break;
    a = a_next;
    d_a = d_next;
    if (d_a >= -ROOT_TOL) break;
  }
  return a;
}

/* ------------------------------------------------------------------------ */
/* One node: Eq. (1), f~_i = f_i + alpha beta (f^eq_i - f_i).                */
/* ------------------------------------------------------------------------ */
int orc_collide_node(int lattice, const double *f, double beta, int mode,
                     int secant_iters, double *f_tilde, double *alpha,
                     int *flags, int *iters) {
  lat_t L;
  if (get_lattice(lattice, &L)) return -1;
  const int q = L.q;
  *flags = 0;
  *iters = 0;

  double rho = 0.0, u[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < q; i++) {
    if (!(f[i] > 0.0)) return -1;
    rho += f[i];
  }
  for (int a = 0; a < L.d; a++) {
    double m = 0.0;
    for (int i = 0; i < q; i++) m += L.c[i][a] * f[i];
    u[a] = m / rho;
  }
  double feq[ORC_QMAX], x[ORC_QMAX];
  if (orc_equilibrium(lattice, rho, u, feq)) return -1;
  for (int i = 0; i < q; i++) x[i] = feq[i] / f[i] - 1.0;

  double amax = orc_alpha_max(q, f, feq);
  double a;
  if (isinf(amax)) {
    /* f^eq == f: "alpha can be any number"; reading: alpha = 2 */
    *flags |= ORC_F_DEGENERATE;
    a = 2.0;
  } else {
    double astar = amax < 2.0 ? amax : 2.0; /* Eq. (8) */
    if (mode == ORC_ROOT)
      a = alpha_root(q, f, x, amax, flags, iters);
    else if (mode == ORC_SECANT)
      a = alpha_secant(q, f, x, astar, secant_iters, flags, iters);
    else
      a = alpha_formula(q, f, x, astar, flags);
    if (orc_delta_h(q, f, x, a) > orc_delta_h_bound(q, f, x, a))
      *flags |= ORC_F_VIOLATION;
  }
  *alpha = a;
  for (int i = 0; i < q; i++) f_tilde[i] = f[i] + a * beta * (feq[i] - f[i]);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole-lattice step: collide every node, push f~_i to x + c_i (periodic). */
/* Diagnostics are summed per (y, z) row, then rows are summed in order, so  */
/* the result does not depend on the number of threads.                     */
/* ------------------------------------------------------------------------ */
typedef struct {
  double mass, mom[3], ke, h, amin, amax, asum;
  long long deg, acc, form, two, viol, iters, cap, noroot;
  int err;
} row_acc;

static int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

int orc_step(int lattice, int nx, int ny, int nz, double beta, int mode,
             int secant_iters, const double *f_in, double *f_out,
             double *alpha_map, orc_stats *stats, int threads) {
  lat_t L;
  if (get_lattice(lattice, &L)) return -1;
  if (nx < 1 || ny < 1 || nz < 1) return -1;
  const int q = L.q;
  const long long n = (long long)nx * ny * nz;
  const int rows = ny * nz;
  row_acc *acc = (row_acc *)calloc((size_t)rows, sizeof(row_acc));
  if (!acc) return -1;
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(threads)
#endif
  for (int row = 0; row < rows; row++) {
    int y = row % ny, z = row / ny;
    row_acc *A = &acc[row];
    A->amin = INFINITY;
    A->amax = -INFINITY;
    for (int xx = 0; xx < nx; xx++) {
      long long node = ((long long)z * ny + y) * nx + xx;
      double f[ORC_QMAX], ft[ORC_QMAX], alpha;
      int flags, iters;
      for (int i = 0; i < q; i++) f[i] = f_in[i * n + node];
      if (orc_collide_node(lattice, f, beta, mode, secant_iters, ft, &alpha,
                           &flags, &iters)) {
        A->err = 1;
        continue;
      }
      /* diagnostics of the pre-collision state f^n */
      double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
      for (int i = 0; i < q; i++) {
        rho += f[i];
        for (int a = 0; a < 3; a++) m[a] += L.c[i][a] * f[i];
      }
      A->mass += rho;
      for (int a = 0; a < 3; a++) A->mom[a] += m[a];
      A->ke += 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
      A->h += orc_entropy(lattice, f);
      if (alpha < A->amin) A->amin = alpha;
      if (alpha > A->amax) A->amax = alpha;
      A->asum += alpha;
      A->deg += (flags & ORC_F_DEGENERATE) != 0;
      A->acc += (flags & ORC_F_ACCEPT_STAR) != 0;
      A->form += (flags & ORC_F_FORMULA) != 0;
      A->two += (flags & ORC_F_ACCEPT_TWO) != 0;
      A->viol += (flags & ORC_F_VIOLATION) != 0;
      A->cap += (flags & ORC_F_ROOT_CAP) != 0;
      A->noroot += (flags & ORC_F_NO_ROOT) != 0;
      A->iters += iters;
      if (alpha_map) alpha_map[node] = alpha;
      /* Eq. (5b): push to the neighbour x + c_i */
      for (int i = 0; i < q; i++) {
        int xd = wrap(xx + L.c[i][0], nx);
        int yd = wrap(y + L.c[i][1], ny);
        int zd = wrap(z + L.c[i][2], nz);
        f_out[i * n + ((long long)zd * ny + yd) * nx + xd] = ft[i];
      }
    }
  }
  int err = 0;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->alpha_min = INFINITY;
    stats->alpha_max = -INFINITY;
  }
  for (int row = 0; row < rows; row++) {
    row_acc *A = &acc[row];
    err |= A->err;
    if (!stats) continue;
    stats->mass += A->mass;
    for (int a = 0; a < 3; a++) stats->momentum[a] += A->mom[a];
    stats->kinetic_energy += A->ke;
    stats->h_total += A->h;
    if (A->amin < stats->alpha_min) stats->alpha_min = A->amin;
    if (A->amax > stats->alpha_max) stats->alpha_max = A->amax;
    stats->alpha_sum += A->asum;
    stats->n_degenerate += A->deg;
    stats->n_accept_star += A->acc;
    stats->n_formula += A->form;
    stats->n_accept_two += A->two;
    stats->n_violations += A->viol;
    stats->n_root_iters += A->iters;
    stats->n_root_cap += A->cap;
    stats->n_no_root += A->noroot;
  }
  if (stats) stats->n_nodes = n;
  free(acc);
  return err ? -1 : 0;
}

int orc_init_equilibrium(int lattice, int nx, int ny, int nz,
                         const double *rho, const double *u, double *f) {
  lat_t L;
  if (get_lattice(lattice, &L)) return -1;
  const long long n = (long long)nx * ny * nz;
  for (long long node = 0; node < n; node++) {
    double uu[3] = {0.0, 0.0, 0.0}, feq[ORC_QMAX];
    for (int a = 0; a < L.d; a++) uu[a] = u[a * n + node];
    if (orc_equilibrium(lattice, rho[node], uu, feq)) return -1;
    for (int i = 0; i < L.q; i++) f[i * n + node] = feq[i];
  }
  return 0;
}

int orc_moments(int lattice, int nx, int ny, int nz, const double *f,
                double *rho_out, double *u_out) {
  lat_t L;
  if (get_lattice(lattice, &L)) return -1;
  const long long n = (long long)nx * ny * nz;
  for (long long node = 0; node < n; node++) {
    double rho = 0.0;
    for (int i = 0; i < L.q; i++) rho += f[i * n + node];
    rho_out[node] = rho;
    for (int a = 0; a < L.d; a++) {
      double m = 0.0;
      for (int i = 0; i < L.q; i++) m += L.c[i][a] * f[i * n + node];
      u_out[a * n + node] = m / rho;
    }
  }
  return 0;
}

/* Enstrophy 1/2 <|omega|^2>, omega = curl u by second-order central
 * differences on the periodic lattice (2D: omega_z only). */
double orc_enstrophy(int lattice, int nx, int ny, int nz, const double *f) {
  lat_t L;
  if (get_lattice(lattice, &L)) return NAN;
  const long long n = (long long)nx * ny * nz;
  double *rho = (double *)malloc(sizeof(double) * n);
  double *u = (double *)calloc((size_t)(3 * n), sizeof(double));
  if (!rho || !u) {
    free(rho);
    free(u);
    return NAN;
  }
  orc_moments(lattice, nx, ny, nz, f, rho, u);
#define U(a, xx, yy, zz) \
  u[(a) * n + ((long long)wrap(zz, nz) * ny + wrap(yy, ny)) * nx + wrap(xx, nx)]
  double sum = 0.0;
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        double dwdy = 0.5 * (U(2, x, y + 1, z) - U(2, x, y - 1, z));
        double dvdz = 0.5 * (U(1, x, y, z + 1) - U(1, x, y, z - 1));
        double dudz = 0.5 * (U(0, x, y, z + 1) - U(0, x, y, z - 1));
        double dwdx = 0.5 * (U(2, x + 1, y, z) - U(2, x - 1, y, z));
        double dvdx = 0.5 * (U(1, x + 1, y, z) - U(1, x - 1, y, z));
        double dudy = 0.5 * (U(0, x, y + 1, z) - U(0, x, y - 1, z));
        double wx = (L.d == 3) ? dwdy - dvdz : 0.0;
        double wy = (L.d == 3) ? dudz - dwdx : 0.0;
        double wz = dvdx - dudy;
        sum += wx * wx + wy * wy + wz * wz;
      }
#undef U
  free(rho);
  free(u);
  return 0.5 * sum / (double)n;
}
