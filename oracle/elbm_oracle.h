/*
 * elbm_oracle.h -- plain FP64 CPU oracle of the entropic lattice Boltzmann
 * method (ELBM) with the relaxation-rate formula of Zhao & Yong,
 * "Relaxation-rate formula for the entropic lattice Boltzmann method".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it, and the two share
 * no code, tables or headers.
 *
 * Conventions (all of them readings of the paper, listed in the design notes):
 *   - lattice units: time step dt = 1, sound speed c_s^2 = 1/3;
 *   - velocity sets D1Q3, D2Q9, D3Q27 in the ordering "rest first, then
 *     +/- pairs" (index 2k-1 and 2k are opposite velocities);
 *   - populations are stored SoA as f[i][z][y][x], x fastest;
 *   - periodic boundaries on every axis;
 *   - a "step" maps the pre-collision state f^n to f^{n+1} by Eq. (1):
 *     collide at every node (Eq. 5a), then push to x + c_i (Eq. 5b).
 */
#ifndef ELBM_ORACLE_H
#define ELBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_D2Q9 = 0, ORC_D3Q27 = 1, ORC_D1Q3 = 2 };
enum { ORC_FORMULA = 0, ORC_ROOT = 1, ORC_SECANT = 2 };

/* Flags set per node by orc_collide_node (bit mask). */
enum {
  ORC_F_DEGENERATE = 1,   /* f^eq == f: alpha = 2 by reading            */
  ORC_F_ACCEPT_STAR = 2,  /* H(f*(alpha_*)) <= H(f): alpha = alpha_*     */
  ORC_F_FORMULA = 4,      /* Eq. (9) chord used                          */
  ORC_F_ACCEPT_TWO = 8,   /* alpha_* == 2 and H(f*(2)) <= H(f) (Fig. 5)  */
  ORC_F_VIOLATION = 16,   /* Delta H(alpha) above its rounding bound     */
  ORC_F_ROOT_CAP = 32,    /* bisection stopped on the iteration cap      */
  ORC_F_NO_ROOT = 64      /* Delta H(alpha_max) <= 0: alpha = alpha_max  */
};

/* Per-step diagnostics, accumulated over the pre-collision state f^n and
 * over the collisions performed by the step. */
typedef struct {
  double mass;            /* sum_x rho                                    */
  double momentum[3];     /* sum_x rho u                                  */
  double kinetic_energy;  /* 1/2 sum_x rho |u|^2                          */
  double h_total;         /* sum_x H(f(x)), Eq. (3)                       */
  double alpha_min, alpha_max, alpha_sum;
  long long n_nodes, n_degenerate, n_accept_star, n_formula, n_accept_two,
      n_violations, n_root_iters, n_root_cap, n_no_root;
} orc_stats;

/* Lattice tables.  c_out: q*3 ints (unused axes 0), w_out: q doubles.
 * Returns q, or -1 for an unknown lattice id. */
int orc_lattice(int lattice, int *c_out, double *w_out);
int orc_lattice_dim(int lattice);
int orc_lattice_q(int lattice);

/* Entropic equilibrium (minimiser of Eq. (3) under mass/momentum
 * constraints), closed product form.  u has 3 entries (unused axes 0).
 * Returns 0, or -1 when |u_a| >= 1 or rho <= 0. */
int orc_equilibrium(int lattice, double rho, const double *u, double *feq);

/* H(f) = sum_i f_i ln(f_i / W_i), Eq. (3).  0 ln 0 := 0. */
double orc_entropy(int lattice, const double *f);

/* Delta H(alpha) = H(f + alpha (f^eq - f)) - H(f), moment-consistent form
 * sum_i f_i [(1 + alpha x_i) ln(1 + alpha x_i) - alpha x_i ln(1 + x_i)],
 * x_i = f^eq_i / f_i - 1.  Requires f_i > 0. */
double orc_delta_h(int q, const double *f, const double *x, double alpha);
/* Rounding bound of the sum above (violation threshold tau_v). */
double orc_delta_h_bound(int q, const double *f, const double *x, double alpha);
/* The literal difference H(f*(alpha)) - H(f), for cross-checks. */
double orc_delta_h_literal(int lattice, const double *f, const double *feq,
                           double alpha);

/* alpha_max = min over {i : f^eq_i < f_i} of f_i / (f_i - f^eq_i).
 * Returns +inf when the set is empty (f^eq == f). */
double orc_alpha_max(int q, const double *f, const double *feq);

/* Collide one node.  f: q pre-collision populations (all > 0).
 * beta from Eq. (2).  mode: ORC_FORMULA / ORC_ROOT / ORC_SECANT;
 * secant_iters: number of modified-secant iterations (SECANT only).
 * Outputs: f_tilde (q values, may alias nothing), *alpha, *flags, *iters.
 * Returns 0 on success, -1 on invalid state (f_i <= 0, |u| >= 1). */
int orc_collide_node(int lattice, const double *f, double beta, int mode,
                     int secant_iters, double *f_tilde, double *alpha,
                     int *flags, int *iters);

/* One Eq. (1) time step on a periodic nx*ny*nz lattice (nz=1 / ny=1 for
 * lower dimensions).  f_in, f_out: SoA [q][nz][ny][nx], distinct buffers.
 * alpha_map (optional, nx*ny*nz) receives the alpha used at every node.
 * stats (optional) receives the diagnostics of this step.
 * threads: OpenMP threads (<= 0: library default).  Returns 0 or -1. */
int orc_step(int lattice, int nx, int ny, int nz, double beta, int mode,
             int secant_iters, const double *f_in, double *f_out,
             double *alpha_map, orc_stats *stats, int threads);

/* f <- f^eq(rho(x), u(x)) at every node.  rho: [nz][ny][nx],
 * u: [d][nz][ny][nx] with d = lattice dimension. */
int orc_init_equilibrium(int lattice, int nx, int ny, int nz,
                         const double *rho, const double *u, double *f);

/* Density and velocity of every node.  u_out: [d][nz][ny][nx]. */
int orc_moments(int lattice, int nx, int ny, int nz, const double *f,
                double *rho_out, double *u_out);

/* Enstrophy 1/2 <|omega|^2> with central differences of u (periodic). */
double orc_enstrophy(int lattice, int nx, int ny, int nz, const double *f);

#ifdef __cplusplus
}
#endif
#endif
