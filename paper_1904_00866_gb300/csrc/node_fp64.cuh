// FP64 per-node arithmetic of the ELBM collision (Eqs. (1)-(9)).
//
// Used for FP64 storage, for the ROOT and SECANT alpha modes, for FP32
// nodes far from equilibrium, and for the FP64 entropy check of diagnostic
// steps.  Notation: x_i = f^eq_i / f_i - 1, so f*(alpha)_i = f_i (1 + alpha x_i).
//
// Entropy change along the ray f*(alpha) = f + alpha (f^eq - f) (Eq. (4)):
//   Delta H(alpha) = sum_i f_i [phi(alpha x_i) - alpha x_i ln(1 + x_i)],
//   phi(y) = (1 + y) ln(1 + y) - y.
// This equals H(f*(alpha)) - H(f) exactly: the dropped terms
// alpha sum (f^eq - f) ln(f^eq / W) and alpha sum f x vanish because
// ln(f^eq / W) is a combination of the collision invariants and f^eq - f
// carries no mass or momentum.  Removing them removes their rounding noise.
#pragma once
#include <math.h>

#include "lattice.cuh"

namespace elbm {

constexpr double kRootTol = 1e-13;   // bisection stop rule of the paper
constexpr int kRootMaxIters = 64;    // cap (the paper states none)

// Per-node outcome flags.
enum : unsigned {
  NF_DEGENERATE = 1u,
  NF_ACCEPT_STAR = 2u,
  NF_FORMULA = 4u,
  NF_ACCEPT_TWO = 8u,
  NF_BAND = 16u,
  NF_FAR = 32u,
  NF_ROOT_CAP = 64u,
  NF_NO_ROOT = 128u,
  NF_BAD_NEG = 256u,
  NF_BAD_NONFINITE = 512u,
  NF_TIMEOUT = 1024u,    // a bounded pipeline wait ran out (kernel left)
  NF_REFINE = 2048u      // FP32 decision not certified: second stage due
};

enum { MODE_FORMULA = 0, MODE_ROOT = 1, MODE_SECANT = 2 };

// phi(y) = (1 + y) ln(1 + y) - y for y >= -1 (phi(-1) = 1, 0 ln 0 := 0).
// |y| < 0.1: y^2 sum_{k=2}^{17} (-1)^k y^(k-2) / (k (k-1)) (Horner, literal
// coefficients); the first omitted term is below 1e-18 of the sum.
__device__ __forceinline__ double phi64(double y) {
  if (y <= -1.0) return 1.0;
  if (fabs(y) < 0.1) {
    double s = -1.0 / 272.0;                // k = 17
    s = fma(s, y, 1.0 / 240.0);             // 16
    s = fma(s, y, -1.0 / 210.0);            // 15
    s = fma(s, y, 1.0 / 182.0);             // 14
    s = fma(s, y, -1.0 / 156.0);            // 13
    s = fma(s, y, 1.0 / 132.0);             // 12
    s = fma(s, y, -1.0 / 110.0);            // 11
    s = fma(s, y, 1.0 / 90.0);              // 10
    s = fma(s, y, -1.0 / 72.0);             // 9
    s = fma(s, y, 1.0 / 56.0);              // 8
    s = fma(s, y, -1.0 / 42.0);             // 7
    s = fma(s, y, 1.0 / 30.0);              // 6
    s = fma(s, y, -1.0 / 20.0);             // 5
    s = fma(s, y, 1.0 / 12.0);              // 4
    s = fma(s, y, -1.0 / 6.0);              // 3
    s = fma(s, y, 1.0 / 2.0);               // 2
    return y * y * s;
  }
  return (1.0 + y) * log1p(y) - y;
}

template <class L>
struct Node64 {
  double f[L::Q];   // pre-collision populations
  double x[L::Q];   // f^eq_i / f_i - 1
  double rho;
  double j[3];      // momentum sum_i c_i f_i
  double amax;      // alpha_max (+inf when f^eq == f)
};

// Moments, equilibrium, x_i and alpha_max of a node whose f[] is filled.
// The entropic equilibrium is f^eq_i = rho W_i prod_a psi_a(c_ia) with the
// per-axis factors psi(0) = 1 - s, psi(+-1) = 1 +- 3u + 2s,
// s = 3u^2 / (1 + sqrt(1 + 3u^2)); this is the D1Q3 minimiser of Eq. (3)
// (psi(0) = 2 - sqrt(1+3u^2), psi(+1)/psi(0) = (2u + sqrt(1+3u^2))/(1-u)),
// written without cancellation.  Returns NF_BAD_* flags (0 when valid).
template <class L>
__device__ __forceinline__ unsigned node64_prepare(Node64<L>& s) {
  unsigned bad = 0;
  double rho = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    rho += s.f[i];
    if (!(s.f[i] > 0.0)) bad |= NF_BAD_NEG;
  }
  double u[3] = {0.0, 0.0, 0.0}, dp[3], dm[3], d0[3];
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    double m = 0.0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      if (L::c(i, a) == 1) m += s.f[i];
      if (L::c(i, a) == -1) m -= s.f[i];
    }
    s.j[a] = m;
    u[a] = m / rho;
    if (!(fabs(u[a]) < 1.0)) bad |= NF_BAD_NONFINITE;
    double sg = 3.0 * u[a] * u[a] / (1.0 + sqrt(1.0 + 3.0 * u[a] * u[a]));
    dp[a] = 3.0 * u[a] + 2.0 * sg;
    dm[a] = -3.0 * u[a] + 2.0 * sg;
    d0[a] = -sg;
  }
  if (L::D < 3) s.j[2] = 0.0;
  if (L::D < 2) s.j[1] = 0.0;
  if (!(rho > 0.0) || !isfinite(rho)) bad |= NF_BAD_NONFINITE;
  s.rho = rho;
  double amax = INFINITY;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    double P = rho * L::w(i);
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
      const int ca = L::c(i, a);
      P *= 1.0 + (ca == 1 ? dp[a] : (ca == -1 ? dm[a] : d0[a]));
    }
    const double x = (P - s.f[i]) / s.f[i];
    s.x[i] = x;
    if (x < 0.0) amax = fmin(amax, -1.0 / x);
  }
  s.amax = amax;
  return bad;
}

// Delta H(alpha) = sum_i f_i phi(alpha x_i) - alpha * B, B = sum f_i x_i L_i.
template <class L>
__device__ __forceinline__ double dH64_phi_sum(const Node64<L>& s,
                                               double alpha) {
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) sum += s.f[i] * phi64(alpha * s.x[i]);
  return sum;
}

// Eq. (8) + acceptance test + Eq. (9).
template <class L>
__device__ __forceinline__ double alpha_formula64(const Node64<L>& s,
                                                  unsigned& flags) {
  const double astar = fmin(2.0, s.amax);
  double B = 0.0, D1 = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const double Li = log1p(s.x[i]);
    B += s.f[i] * s.x[i] * Li;
    D1 += s.f[i] * (Li - s.x[i]);   // phi(x) - x ln(1+x) = ln(1+x) - x
  }
  const double Dstar = dH64_phi_sum(s, astar) - astar * B;
  if (Dstar <= 0.0) {
    flags |= NF_ACCEPT_STAR;
    if (astar == 2.0) flags |= NF_ACCEPT_TWO;
    return astar;
  }
  flags |= NF_FORMULA;
  // H(f*(alpha_*)) - H(f^eq) = Delta H(alpha_*) - Delta H(1) > 0 in exact
  // arithmetic; a non-positive value means f equals f^eq to rounding, where
  // alpha = 1 (f* = f^eq) is taken.
  if (!(Dstar - D1 > 0.0)) return 1.0;
  return astar + Dstar / (Dstar - D1) * (1.0 - astar);
}

// Bisection on [1, alpha_max] for Eq. (4), stop rule -1e-13 <= dH <= 0.
template <class L>
__device__ __forceinline__ double alpha_root64(const Node64<L>& s,
                                               unsigned& flags, int& iters) {
  double B = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) B += s.f[i] * s.x[i] * log1p(s.x[i]);
  double lo = 1.0, hi = s.amax;
  if (dH64_phi_sum(s, hi) - hi * B <= 0.0) {
    flags |= NF_NO_ROOT;
    return hi;
  }
  for (int k = 0; k < kRootMaxIters; ++k) {
    const double mid = 0.5 * (lo + hi);
    const double d = dH64_phi_sum(s, mid) - mid * B;
    ++iters;
    if (d >= -kRootTol && d <= 0.0) return mid;
    if (d > 0.0)
      hi = mid;
    else
      lo = mid;
    if (hi - lo < 1e-15 * hi) return lo;
  }
  flags |= NF_ROOT_CAP;
  return lo;
}

// Modified secant iteration, alpha^(0) = 1 (first iterate = Eq. (9)).
template <class L>
__device__ __forceinline__ double alpha_secant64(const Node64<L>& s,
                                                 int n_iter, unsigned& flags,
                                                 int& iters) {
  const double astar = fmin(2.0, s.amax);
  double B = 0.0, D1 = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const double Li = log1p(s.x[i]);
    B += s.f[i] * s.x[i] * Li;
    D1 += s.f[i] * (Li - s.x[i]);
  }
  const double Dstar = dH64_phi_sum(s, astar) - astar * B;
  if (Dstar <= 0.0) {
    flags |= NF_ACCEPT_STAR;
    if (astar == 2.0) flags |= NF_ACCEPT_TWO;
    return astar;
  }
  flags |= NF_FORMULA;
  if (!(Dstar - D1 > 0.0)) return 1.0;   // f == f^eq to rounding
  // Every iterate keeps Delta H <= 0 in exact arithmetic; an iterate whose
  // computed Delta H is positive (rounding) ends the iteration at the
  // previous one.
  double a = 1.0, da = D1;
  for (int k = 0; k < n_iter; ++k) {
    const double an = astar + Dstar / (Dstar - da) * (a - astar);
    const double dn = dH64_phi_sum(s, an) - an * B;
    ++iters;
    if (dn > 0.0) break;
    a = an;
    da = dn;
    if (da >= -kRootTol) break;
  }
  return a;
}

template <class L, int MODE>
__device__ __forceinline__ double node64_alpha(const Node64<L>& s,
                                               int secant_iters,
                                               unsigned& flags, int& iters) {
  if (isinf(s.amax)) {   // f^eq == f: alpha is arbitrary; take 2
    flags |= NF_DEGENERATE;
    return 2.0;
  }
  if (MODE == MODE_ROOT) return alpha_root64(s, flags, iters);
  if (MODE == MODE_SECANT) return alpha_secant64(s, secant_iters, flags, iters);
  return alpha_formula64(s, flags);
}

// Whether a node's branch (acceptance of alpha_* or Eq. (9)) differs from
// the FP64 check's.  Nodes whose evaluation found f^eq = f to its working
// precision (NF_DEGENERATE: n = 0, so f*(alpha) = f for every alpha) have no
// branch to compare: the FP64 evaluation of the same node decides by its
// own rounding noise there.
__device__ __forceinline__ bool decision_mismatch(unsigned flags,
                                                  bool accept_ref) {
  return (flags & NF_DEGENERATE) == 0u &&
         ((flags & NF_ACCEPT_STAR) != 0) != accept_ref;
}

// FP64 check of one node at the alpha actually used: Delta H(alpha) against
// its rounding bound (the Eq. (7) violation test), the entropy H(f) of
// Eq. (3), and the FP64 FORMULA alpha for comparison.
struct Check64 {
  double h;          // H(f)
  bool violation;
  double alpha_ref;  // FP64 FORMULA alpha
  bool accept_ref;   // FP64 FORMULA accepts alpha_*
};

template <class L>
__device__ __forceinline__ Check64 node64_check(const Node64<L>& s,
                                                double alpha) {
  Check64 r;
  double h = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) h += s.f[i] * log(s.f[i] / L::w(i));
  r.h = h;
  if (isinf(s.amax)) {
    r.violation = false;
    r.alpha_ref = 2.0;
    r.accept_ref = true;
    return r;
  }
  // Delta H(alpha) and the bound
  //   eps (64 sum f (|phi(y)| + |y L|)
  //        + 4 Q sum f (1 + |x|) alpha |ln(1+y) - L - x/(1+x)|
  //        + 4 alpha |sum f x (ln(1+y) - L)|)
  double d = 0.0, mag = 0.0, prop = 0.0, slope = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const double x = s.x[i];
    const double y = alpha * x;
    const double Li = log1p(x);
    const double ly = (1.0 + y > 1e-300) ? log1p(y) : log(1e-300);
    const double p = phi64(y);
    d += s.f[i] * (p - y * Li);
    mag += s.f[i] * (fabs(p) + fabs(y * Li));
    prop += s.f[i] * (1.0 + fabs(x)) * alpha * fabs(ly - Li - x / (1.0 + x));
    slope += s.f[i] * x * (ly - Li);
  }
  const double eps = 2.220446049250313e-16;
  const double bound =
      eps * (64.0 * mag + 4.0 * L::Q * prop + 4.0 * alpha * fabs(slope));
  r.violation = d > bound;
  unsigned fl = 0;
  r.alpha_ref = alpha_formula64(s, fl);
  r.accept_ref = (fl & NF_ACCEPT_STAR) != 0;
  return r;
}

}  // namespace elbm
