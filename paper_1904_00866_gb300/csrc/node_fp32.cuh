// FP32 per-node FORMULA arithmetic with a certified entropy decision.
//
// Populations arrive as delta_i = f_i - W_i rho0 (FP32, exact), so the
// non-equilibrium part n_i = f^eq_i - f_i is formed without the O(1)
// cancellation of f^eq_i - f_i:
//   f^eq_i - W_i rho0 = W_i (drho + rho (P_i - 1)),  drho = sum_i delta_i,
//   P_i - 1 = prod_a (1 + d_a(c_ia)) - 1,  d(0) = -s, d(+-1) = +-3u + 2s,
//   s = 3u^2 / (1 + sqrt(1 + 3u^2))          (entropic equilibrium, Eq. (3)).
// Mass and momentum sums are exact to ~1e-11: each delta_i is split into a
// multiple of 2^-20 (summed exactly) and a remainder below 2^-21.
//
// The entropy changes needed by Eqs. (8)-(9) come from the moments
// M_k = sum_i f_i x_i^k = sum_i n_i x_i^(k-1), x_i = n_i / f_i:
//   Delta H(alpha) = sum_{k>=2} (-1)^k (alpha^k - k alpha) / (k (k-1)) M_k,
// the Taylor series of sum f [phi(alpha x) - alpha x ln(1 + x)] (the linear
// term alpha sum f x is exactly zero).  At alpha = 2 the k = 2 coefficient
// vanishes, so Delta H(2) carries no O(x^2) cancellation.  The series is
// truncated after k = 4, or k = 8 when max|x_i| > 1/100; nodes with
// max|x_i| > 1/8 (or invalid states) are solved in FP64.
//
// Every quantity has an a-priori bound on its FP32 error (unit roundoff
// u = 2^-24):  E_x bounds |x_i - x_i exact| (equilibrium products, velocity
// division, the x division); e2 / e1 bound the errors of Delta H(2) /
// Delta H(1) from E_x (first and second order), the series rounding and the
// truncation.  Decision, each branch exact for the stored state:
//   Delta H(2) + e2 <= 0            -> alpha = 2 (acceptance after Eq. (8));
//   Delta H(2) - e2 > 0 and Delta H(1) + e1 < 0
//                                   -> alpha = Eq. (9) chord evaluated on the
//                                      upper bounds and rounded down (the
//                                      chord root decreases in both values,
//                                      so it stays at or below the exact
//                                      Eq. (9) value, which is at or below
//                                      the root of Eq. (4)); in the exact
//                                      mode only when the bounds fix the
//                                      chord to within 2^-16;
//   otherwise (a sign within the FP32 error, or n zero in FP32)
//                                   -> second stage: n_i recomputed in
//                                      double-float arithmetic and the same
//                                      decision retaken with its much smaller
//                                      error (flag NF_BAND); a node still
//                                      undecided goes to the FP64 fixup.
// So every node takes the branch the exact arithmetic takes, except where
// Delta H(2) lies within the FP64 evaluation's own rounding.

// Opposite-velocity populations are processed in pairs with packed f32x2
// arithmetic (see npairs below); every lane operation rounds like its
// scalar form, so only the order of the moment sums differs from a scalar
// loop, which the summation error term of the bounds covers.
#pragma once
#include <math.h>

#include "df32.cuh"
#include "lattice.cuh"
#include "node_fp64.cuh"

namespace elbm {

// Populations 2k-1 and 2k (k = 1..P, P = (Q - 1) / 2) have opposite
// velocities.  Their values travel together as the two lanes of a float2,
// so the per-population arithmetic issues as packed f32x2 instructions: one
// issue slot for two IEEE operations, each lane rounded exactly like the
// scalar operation.  Lane x holds population 2k-1 (velocity c), lane y
// population 2k (velocity -c); population 0 (rest) stays scalar.
template <class L>
__host__ __device__ constexpr int npairs() {
  return (L::Q - 1) / 2;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  return __fadd2_rn(a, b);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  return __fmul2_rn(a, b);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
// a - b rounded once (the product with -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
// lane signs (s, -s) of a velocity component s of lane x
__device__ __forceinline__ float2 lane_sign(int s) {
  return make_float2((float)s, (float)-s);
}

// Per-node result of the FP32 FORMULA evaluation.
template <class L>
struct N32 {
  float n0;                    // f^eq_0 - f_0 (not yet projected)
  float2 n2[npairs<L>()];      // the same for the pairs
  float alpha;
  unsigned flags;
  float drho, rho;
  float j[3];
};

__host__ __device__ constexpr int cidx(int c) { return c + 1; }

// Largest velocity component the FP32 paths take.  Their error bounds use
// 1 - Dd, Dd = 3U + 3U^2 >= |d_a|, as a lower bound of every equilibrium
// factor 1 + d_a; that bound is positive only for U < 0.264, so nodes with
// a larger component go to the FP64 fixup.
constexpr float kUMax32 = 0.25f;

// Largest uncertainty of an Eq. (9) chord the exact decision mode accepts
// from an evaluation's bounds (2^-16); a wider one goes to the next stage.
constexpr float kChordWidth = 1.52587890625e-05f;

// 1 / y and 1 / sqrt(y) by the SFU (rcp.approx.ftz.f32, relative error
// below 2^-23; rsqrt.approx.ftz.f32, relative error below 2^-22; subnormal
// arguments flush to zero, so callers pass normal values).  __fdividef is
// used within its documented 2 ulp for divisors of normal magnitude.  None
// of them needs the IEEE division's or square root's special-case path,
// nor the subnormal scaling of the non-flushing forms (conversion-class
// instructions, which GB300 issues on its FP64 pipe).
__device__ __forceinline__ float rcp_approx(float y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float y) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}
__device__ __forceinline__ float2 rcp_approx2(float2 y) {
  return make_float2(rcp_approx(y.x), rcp_approx(y.y));
}

// Index 0..3 of the distinct weight of population i (number of nonzero
// velocity components).
template <class L>
__host__ __device__ constexpr int wclass(int i) {
  return L::nonzero(i);
}

// Mass and momentum sums m0 = sum_i v_i, m_a = sum_i c_ia v_i of a set
// given as the rest value v0 and the pairs vv[k] (each lane accumulates
// its own population's terms; 40 packed and 5 scalar operations for
// D3Q27, 10 and 4 for D2Q9).
template <class L>
__device__ __forceinline__ void moments2(float v0,
                                         const float2 (&vv)[npairs<L>()],
                                         float& m0, float& mx, float& my,
                                         float& mz) {
  constexpr int P = npairs<L>();
  float2 s = vv[0];
  float2 acc[3] = {f2(0.0f), f2(0.0f), f2(0.0f)};
  bool started[3] = {false, false, false};
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int i = 2 * k + 1;
    if (k > 0) s = add2(s, vv[k]);
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
      const int c = L::c(i, a);
      if (c == 0) continue;
      acc[a] = started[a] ? fma2(lane_sign(c), vv[k], acc[a])
                          : mul2(lane_sign(c), vv[k]);
      started[a] = true;
    }
  }
  m0 = v0 + (s.x + s.y);
  mx = acc[0].x + acc[0].y;
  my = acc[1].x + acc[1].y;
  mz = L::D == 3 ? acc[2].x + acc[2].y : 0.0f;
}

// Delta H(2) and Delta H(1) from the moments M[k] = sum_i f_i x_i^k
// (k = 2..8) by the series sum_k c_k(alpha) M_k,
// c_k(alpha) = (-1)^k (alpha^k - k alpha) / (k (k-1)), truncated after k = 4
// (k8 false) or k = 8, with bounds e2 / e1 on their errors given a bound Ex
// on the absolute error of every x_i: first- and second-order propagation
// of Ex, rounding of the sums over i and of the series, and the tail.
struct DH32 {
  float D2, D1, e2, e1;
};

template <int Q>
__device__ __forceinline__ DH32 series_dh32(const float (&M)[9], bool k8,
                                            float xabs, float Ex, float rho) {
  constexpr float uu = 5.9604645e-8f;   // 2^-24
  constexpr float kUp = 1.00000095367431640625f;   // 1 + 2^-20
  const float gq = (float)(Q + 9) * uu * 1.01f;
  // c(2): k=3..8: -1/3, 2/3, -11/10, 26/15, -19/7, 30/7
  // c(1): k=2..8: -1/2, 1/3, -1/4, 1/5, -1/6, 1/7, -1/8
  DH32 h;
  h.D2 = fmaf(-1.0f / 3.0f, M[3], (2.0f / 3.0f) * M[4]);
  h.D1 = fmaf(-0.5f, M[2], fmaf(1.0f / 3.0f, M[3], -0.25f * M[4]));
  float tr2, tr1, rnd;
  const float r2 = 2.0f * xabs;
  if (k8) {
    h.D2 = fmaf(-1.1f, M[5],
                fmaf(26.0f / 15.0f, M[6],
                     fmaf(-19.0f / 7.0f, M[7], fmaf(30.0f / 7.0f, M[8], h.D2))));
    h.D1 = fmaf(0.2f, M[5],
                fmaf(-1.0f / 6.0f, M[6],
                     fmaf(1.0f / 7.0f, M[7], fmaf(-0.125f, M[8], h.D1))));
    const float r2_7 = r2 * r2 * r2 * r2 * r2 * r2 * r2;
    const float x7 = xabs * xabs * xabs * xabs * xabs * xabs * xabs;
    // tails sum_{k>=9}: |c_k(2)| <= 2^k / (k (k-1)), |c_k(1)| = 1 / k,
    // |M_k| <= xabs^(k-2) M_2; upper bounds of positive quotients are the
    // 2-ulp approximate division raised by 2^-20
    tr2 = __fdividef(r2_7, 18.0f * (1.0f - r2)) * kUp;
    tr1 = __fdividef(x7, 9.0f * (1.0f - xabs)) * kUp;
    rnd = fabsf(M[5]) * 1.1f + fabsf(M[6]) * 1.74f + fabsf(M[7]) * 2.72f +
          fabsf(M[8]) * 4.29f;
  } else {
    // tails sum_{k>=5}
    const float r2_3 = r2 * r2 * r2;
    tr2 = __fdividef(r2_3 * 0.2f, 1.0f - r2) * kUp;
    tr1 = __fdividef(xabs * xabs * xabs, 5.0f * (1.0f - xabs)) * kUp;
    rnd = 0.0f;
  }
  const float M2 = M[2];
  // First-order propagation of the x errors: with x_i^c = x_i + dx_i
  // (|dx_i| <= Ex) and n_i^c = f_i (dx_i - x_i e_i) + n_i (e_i the
  // quotient's relative rounding, below 3u), the computed term
  // n^c (x^c)^(k-1) is off by k f x^(k-1) dx - f x^k e, so Delta H(2) is off
  // by at most sum_k |c_k(2)| k f |x|^(k-1) Ex + 3u sum_k |c_k(2)| f |x|^k
  // <= M2 Ex (1 + 2.67 xabs + 5.5 xabs^2 + ...) + 2u xabs M2, and
  // 1 + 4 xabs covers the bracket for xabs <= 1/8 (1.445 there).
  h.e2 = M2 * (1.01f * (1.0f + 4.0f * xabs) * Ex + 2.0f * uu * xabs +
               gq * xabs * (0.34f + xabs * (0.7f + xabs * (1.2f + 1.8f * xabs))) +
               tr2) +
         4.0f * uu * (fabsf(M[3]) * (1.0f / 3.0f) + fabsf(M[4]) * (2.0f / 3.0f) +
                      rnd) +
         2.0f * rho * (xabs + Ex) * Ex * Ex;
  // S1b >= sqrt(rho M2) >= sum f |x|  (Cauchy-Schwarz); 1e-15 bounds the
  // root of any rm <= 1e-30 (no subnormal reaches the reciprocal root)
  const float rm = rho * M2;
  const float S1b = rm > 1e-30f ? rm * rsqrt_approx(rm) * kUp : 1e-15f;
  h.e1 = __fdividef(1.01f * Ex * S1b, 1.0f - xabs) * kUp +
         M2 * (gq * (0.5f + xabs) + tr1) + 4.0f * uu * (0.5f * M2 + fabsf(M[3])) +
         2.0f * rho * Ex * Ex;
  return h;
}

// The FP32 decision between the acceptance of alpha = 2 (after Eq. (8)) and
// the chord of Eq. (9), each taken only when certified by the bounds.  A
// chord whose value the bounds leave uncertain by more than wmax (the
// chord on the lower bounds minus the chord on the upper bounds) is left
// undecided too, so that the exact mode's alpha stays within wmax of the
// Eq. (9) value of the exact state (pass INFINITY to accept any width).
enum { kAcceptTwo = 0, kChord = 1, kUndecided = 2 };
__device__ __forceinline__ int decide32(const DH32& h, float& alpha,
                                        float wmax) {
  const float D2hi = __fadd_ru(h.D2, h.e2);
  if (D2hi <= 0.0f) {
    alpha = 2.0f;
    return kAcceptTwo;
  }
  const float D1hi = __fadd_ru(h.D1, h.e1);
  const float D2lo = __fsub_rd(h.D2, h.e2);
  if (!(D2lo > 0.0f) || !(D1hi < 0.0f)) return kUndecided;
  // alpha = 2 + D2hi / (D2hi - D1hi) (1 - 2), rounded down: the chord root
  // decreases in both values, so it stays at or below the exact Eq. (9)
  // value.  t = D2hi / (D2hi - D1hi) rounded up: the approximate quotient
  // (error <= 2 ulp) is raised by 4 ulp
  const float den = __fsub_rd(D2hi, D1hi);
  const float tt = __fmul_ru(__fdividef(D2hi, den), 1.0f + 2.384185791e-7f);
  alpha = __fsub_rd(2.0f, tt);
  if (wmax < INFINITY) {
    // the chord on the lower bounds, t rounded down: the exact Eq. (9)
    // value lies in [alpha, 2 - tlo]
    const float tlo =
        __fmul_rd(__fdividef(D2lo, __fsub_ru(D2lo, __fsub_rd(h.D1, h.e1))),
                  1.0f - 2.384185791e-7f);
    if (!(tt - tlo <= wmax)) return kUndecided;
  }
  return kChord;
}

// The certified alpha of an undecided node: the Eq. (9) chord evaluated on
// the upper bounds and rounded down when Delta H(1) + e1 < 0 (the chord
// root decreases in both values, so it stays at or below the exact Eq. (9)
// value, itself at or below the root of Eq. (4)), else 1 (f* = f^eq, for
// which H(f*) <= H(f) holds exactly).
__device__ __forceinline__ float certified_alpha32(const DH32& h) {
  const float D2hi = __fadd_ru(h.D2, h.e2);
  const float D1hi = __fadd_ru(h.D1, h.e1);
  if (!(D1hi < 0.0f) || !(D2hi > 0.0f)) return 1.0f;
  const float den = __fsub_rd(D2hi, D1hi);
  const float tt = __fmul_ru(__fdividef(D2hi, den), 1.0f + 2.384185791e-7f);
  return __fsub_rd(2.0f, tt);
}

// Mass and momentum sums of the deviations, exact as double-floats.  Each
// delta = hi + mid + lo with hi on the 2^-20 grid, mid on the 2^-40 grid and
// |lo| <= 2^-41 (all three splits exact); with sum_i |delta_i| < 4 the hi
// and mid sums are exact in FP32 (at most 27 terms on their grids) and the
// lo sum is off by less than 2^-58.  m[0] = sum delta, m[1 + a] = sum c_a
// delta.
template <class L>
__device__ __forceinline__ void exact_moments(float d0,
                                              const float2 (&dd)[npairs<L>()],
                                              DF<float> (&m)[4]) {
  constexpr int P = npairs<L>();
  constexpr float C20 = 12.0f;                  // 1.5 * 2^3, ulp 2^-20
  constexpr float C40 = 1.1444091796875e-05f;   // 1.5 * 2^-17, ulp 2^-40
  float2 h[P], md[P], lw[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    h[k] = sub_(add_(dd[k], f2(C20)), f2(C20));
    const float2 r1 = sub_(dd[k], h[k]);
    md[k] = sub_(add_(r1, f2(C40)), f2(C40));
    lw[k] = sub_(r1, md[k]);
  }
  const float h0 = sub_(add_(d0, C20), C20);
  const float r0 = sub_(d0, h0);
  const float md0 = sub_(add_(r0, C40), C40);
  const float lw0 = sub_(r0, md0);
  float H[4], M[4], W[4];
  moments2<L>(h0, h, H[0], H[1], H[2], H[3]);
  moments2<L>(md0, md, M[0], M[1], M[2], M[3]);
  moments2<L>(lw0, lw, W[0], W[1], W[2], W[3]);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const DF<float> t = two_sum(H[a], M[a]);
    m[a] = fast_two_sum(t.hi, add_(t.lo, W[a]));
  }
}

// Second stage for a node whose FP32 decision is not certified (run by the
// fixup kernel, out of the stream-collide kernels' register budget): n_i is
// recomputed in double-float arithmetic from the exact moments, so x_i is
// known to 6.1 u |x_i| + G (1 + Dd)^3 2^-37 instead of the FP32 path's
// equilibrium rounding, and the decision is retaken with the bounds of that
// accuracy (series always to k = 8).  A node this leaves undecided is
// flagged NF_FAR | NF_REFINE; the DFS variant then evaluates the leading
// terms of Delta H(2) in double-float too (its resolution is set by the
// double-float n, ~1e-12 of W_i rho, instead of the FP32 series' ~75 u),
// and a node still undecided (NF_FAR) goes to the FP64 fixup.  Writes
// r.n0 / r.n2 (the more accurate n, used by the relaxation), r.alpha,
// r.flags (NF_BAND set: the second stage decided) and the moments r.drho,
// r.rho, r.j.
template <class L, bool SHIFTED, bool DFS = false>
__device__ __forceinline__ void node32_refine(
    float d0, const float2 (&dd)[npairs<L>()], float rho0, float corr_rho,
    const float* __restrict__ corr, float a_extra, N32<L>& r) {
  constexpr int P = npairs<L>();
  constexpr float uu = 5.9604645e-8f;  // 2^-24
  // DFS: the leading terms -M3/3 + 2 M4/3 of Delta H(2) in double-float as
  // well (x_i = n_i / f_i as a double-float quotient), for the nodes the
  // FP32 series on the double-float n leaves undecided
  DF<float> m3d = {0.0f, 0.0f}, m4d = {0.0f, 0.0f};
  // exact_moments needs sum |delta_i| < 4
  {
    float2 sa = make_float2(fabsf(dd[0].x), fabsf(dd[0].y));
#pragma unroll
    for (int k = 1; k < P; ++k)
      sa = add2(sa, make_float2(fabsf(dd[k].x), fabsf(dd[k].y)));
    if (!(fabsf(d0) + (sa.x + sa.y) < 3.99f)) {
      r.flags = NF_FAR;
      return;
    }
  }
  DF<float> m[4];
  exact_moments<L>(d0, dd, m);
  DF<float> rho = df_add(m[0], rho0);
  if (!SHIFTED) rho = df_add(rho, corr_rho);
  if (!(rho.hi > 0.0f)) {
    r.flags = NF_FAR;
    return;
  }
  const float rinv = rcp_approx(rho.hi);
  r.drho = add_(m[0].hi, m[0].lo) + (SHIFTED ? 0.0f : corr_rho);
  r.rho = rho.hi;
  r.j[0] = add_(m[1].hi, m[1].lo);
  r.j[1] = add_(m[2].hi, m[2].lo);
  r.j[2] = add_(m[3].hi, m[3].lo);

  // per-axis factors psi[a][c + 1] = 1 + d_a(c) of the entropic equilibrium
  DF<float> psi[3][3];
  float U = 0.0f;
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    // u = j / rho: FP32 quotient plus the corrected residual
    const DF<float> j = m[a + 1];
    const float q = mul_(j.hi, rinv);
    const DF<float> qp = two_prod(q, rho.hi);
    const float res = sub_(add_(sub_(sub_(j.hi, qp.hi), qp.lo), j.lo),
                           mul_(q, rho.lo));
    const DF<float> u = fast_two_sum(q, mul_(res, rinv));
    U = fmaxf(U, fabsf(u.hi));
    // s = sqrt(1 + 3u^2) - 1: one Newton step on s^2 + 2s - 3u^2 = 0 from
    // the FP32 value (relative error 9.5 u, squared by the step)
    const float y = fmaf(3.0f * u.hi, u.hi, 1.0f);
    const float s0 = 3.0f * u.hi * u.hi * rcp_approx(1.0f + y * rsqrt_approx(y));
    const DF<float> sq = two_prod(s0, s0);
    const DF<float> t = two_sum(sq.hi, add_(s0, s0));
    const DF<float> u3 = df_mul(u, 3.0f);
    const DF<float> u23 = df_mul(u3, u);
    const float g =
        add_(sub_(t.hi, u23.hi), sub_(add_(t.lo, sq.lo), u23.lo));
    const DF<float> sv =
        fast_two_sum(s0, mul_(neg_(g), rcp_approx(fma_(2.0f, s0, 2.0f))));
    const DF<float> s2 = {add_(sv.hi, sv.hi), add_(sv.lo, sv.lo)};
    psi[a][2] = df_add(df_add(u3, s2), 1.0f);           // 1 + 3u + 2s
    psi[a][0] = df_add(df_add(df_neg(u3), s2), 1.0f);   // 1 - 3u + 2s
    psi[a][1] = df_add(df_neg(sv), 1.0f);               // 1 - s
  }
  if (!(U < kUMax32)) {
    r.flags = NF_FAR;
    return;
  }
  // n_i = W_i (rho P_i - rho0) [+ corr_i] - delta_i, P_i = prod_a psi_a;
  // W_i as double-float constants per weight class (compile-time tables)
  constexpr float whi[4] = {df_hi(L::w(0)), df_hi(L::w(1)),
                            df_hi(L::w(L::D == 3 ? 7 : 5)),
                            df_hi(L::w(L::D == 3 ? 19 : 5))};
  constexpr float wlo[4] = {df_lo(L::w(0)), df_lo(L::w(1)),
                            df_lo(L::w(L::D == 3 ? 7 : 5)),
                            df_lo(L::w(L::D == 3 ? 19 : 5))};
  auto wdf = [&](int i) {
    return DF<float>{whi[wclass<L>(i)], wlo[wclass<L>(i)]};
  };
  float w0[4];
#pragma unroll
  for (int k = 0; k <= L::D; ++k)
    w0[k] = (k == 0 ? L::wf(0) : L::wf(k == 1 ? 1 : (k == 2 ? 7 : 19))) * rho0;
  float M[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float xabs;
  {
    DF<float> Pr = df_mul(psi[0][1], psi[1][1]);
    if (L::D == 3) Pr = df_mul(Pr, psi[2][1]);
    DF<float> t = df_mul(df_add(df_mul(rho, Pr), -rho0), wdf(0));
    if (!SHIFTED) t = df_add(t, corr[0]);
    t = df_add(t, -d0);
    const float ni = add_(t.hi, t.lo);
    r.n0 = ni;
    const float x = ni * rcp_approx(w0[0] + d0);
    xabs = fabsf(x);
    float pw = ni * x;   // n x^(k-1) = f x^k
#pragma unroll
    for (int k = 2; k <= 8; ++k) {
      M[k] = pw;
      pw *= x;
    }
    if (DFS) {
      const DF<float> fd = df_add(df_mul(wdf(0), rho0), d0);   // f_0
      const DF<float> xd = df_div(t, fd);
      const DF<float> n2 = df_mul(df_mul(t, xd), xd);          // f x^3
      m3d = n2;
      m4d = df_mul(n2, xd);                                    // f x^4
    }
  }
  auto pair = [&](int a, int c) { return df_pair(psi[a][c + 1], psi[a][1 - c]); };
  DF<float2> pxy[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) pxy[a][b] = df_mul(pair(0, a - 1), pair(1, b - 1));
  float2 mk[9];
#pragma unroll
  for (int k = 2; k <= 8; ++k) mk[k] = f2(0.0f);
  const DF<float2> rho2 = df_bcast(rho);
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int i = 2 * k + 1;
    DF<float2> Pp = pxy[cidx(L::c(i, 0))][cidx(L::c(i, 1))];
    if (L::D == 3) Pp = df_mul(Pp, pair(2, L::c(i, 2)));
    DF<float2> t = df_add(df_mul(rho2, Pp), f2(-rho0));
    t = df_mul(t, df_bcast(wdf(i)));
    if (!SHIFTED) t = df_add(t, make_float2(corr[i], corr[i + 1]));
    t = df_add(t, neg_(dd[k]));
    const float2 ni = add_(t.hi, t.lo);
    r.n2[k] = ni;
    const int kc = wclass<L>(i);
    const float2 x = mul2(ni, rcp_approx2(add2(f2(w0[kc]), dd[k])));
    xabs = fmaxf(xabs, fmaxf(fabsf(x.x), fabsf(x.y)));
    float2 pw = mul2(ni, x);
#pragma unroll
    for (int e = 2; e <= 8; ++e) {
      mk[e] = add2(mk[e], pw);
      pw = mul2(pw, x);
    }
    if (DFS) {
      const DF<float2> fd =
          df_add(df_mul(df_bcast(wdf(i)), f2(rho0)), dd[k]);   // f_i
      const DF<float2> xd = df_div(t, fd);
      const DF<float2> n2 = df_mul(df_mul(t, xd), xd);
      const DF<float2> n3 = df_mul(n2, xd);
      const DF<float> a3 = df_add(DF<float>{n2.hi.x, n2.lo.x},
                                  DF<float>{n2.hi.y, n2.lo.y});
      const DF<float> a4 = df_add(DF<float>{n3.hi.x, n3.lo.x},
                                  DF<float>{n3.hi.y, n3.lo.y});
      m3d = df_add(m3d, a3);
      m4d = df_add(m4d, a4);
    }
  }
#pragma unroll
  for (int k = 2; k <= 8; ++k) M[k] += mk[k].x + mk[k].y;
  if (!(xabs <= 0.125f)) {
    r.flags = NF_FAR;
    return;
  }
  if (xabs == 0.0f) {
    // n == 0 to double-float accuracy: alpha = 1 (f* = f^eq) keeps
    // H(f*) <= H(f) exactly; the relaxation leaves f unchanged either way
    r.flags = NF_DEGENERATE | NF_BAND;
    r.alpha = 1.0f;
    return;
  }
  // Error of x_i: the rounding of n_i to FP32, of f_i and of the quotient
  // (6.1 u |x_i|) plus the double-float error of n_i divided by
  // f_i >= W_i rho / G.  With e = u^2 and |u_a| <= U < 1/4: u within
  // 23 e U (corrected quotient), s within 40 e s <= 60 e U^2 (one Newton
  // step from a 9.5 u value), d = +-3u + 2s within 93 e U + 144 e U^2 (with
  // its sum's rounding), 1 + d within c e, c = 8 + 117 U + 168 U^2; the
  // D-fold product P within (1 + Dd)^D (3c + 16) e, rho P - rho0 (rho within
  // 3 e rho), the product with W_i and the difference with delta_i add
  // 36 e (1 + Dd)^D + 25 e rho0 / rho in units of W_i rho and 8 e |delta_i|;
  // |delta_i| <= f_i + W_i rho0.  The bound below doubles that sum.
  constexpr float kUp = 1.00000095367431640625f;   // 1 + 2^-20
  constexpr float e2u = 3.5527136788005009e-15f;   // u^2 = 2^-48
  const float Dd = fmaf(3.0f * U, U, 3.0f * U);
  const float omd = 1.0f - Dd;
  const float omdD = L::D == 3 ? omd * omd * omd : omd * omd;
  const float G = __fdividef(1.0f + xabs, omdD) * kUp;
  const float opdD = L::D == 3 ? (1.0f + Dd) * (1.0f + Dd) * (1.0f + Dd)
                               : (1.0f + Dd) * (1.0f + Dd);
  const float cpsi = fmaf(U, fmaf(168.0f, U, 117.0f), 8.0f);
  const float r0r = rho0 * rinv * 1.01f;           // rho0 / rho, rounded up
  const float En = 2.0f * e2u *
                   (G * (opdD * fmaf(3.0f, cpsi, 52.0f) + 33.0f * r0r) + 8.0f);
  const float Ex = 1.01f * (6.1f * uu * xabs + En + G * a_extra);
  DH32 h = series_dh32<L::Q>(M, true, xabs, Ex, rho.hi);
  if (DFS) {
    // Delta H(2) = [-M3 / 3 + 2 M4 / 3] (double-float) + sum_{k=5..8} c_k M_k
    // (FP32) + tail.  Errors: x_i within Exd = En + G a_extra + 2^-42 |x_i|
    // (the double-float n, f_i and quotient), propagated through the
    // leading terms as M2 (1 + 3 xabs) Exd; their double-float rounding
    // (2,000 u^2 xabs M2 covers 27 terms of a few operations each); the
    // FP32 terms k = 5..8 from x within Ex (100 u xabs^3 M2 with their
    // rounding); the tail beyond k = 8; the final FP32 sum.
    constexpr float c3h = df_hi(-1.0 / 3.0), c3l = df_lo(-1.0 / 3.0);
    constexpr float c4h = df_hi(2.0 / 3.0), c4l = df_lo(2.0 / 3.0);
    const DF<float> lead = df_add(df_mul(m3d, DF<float>{c3h, c3l}),
                                  df_mul(m4d, DF<float>{c4h, c4l}));
    const float tail =
        fmaf(-1.1f, M[5],
             fmaf(26.0f / 15.0f, M[6], fmaf(-19.0f / 7.0f, M[7],
                                           (30.0f / 7.0f) * M[8])));
    const float D2 = lead.hi + (lead.lo + tail);
    const float Exd = 1.01f * (En + G * a_extra + 2.3e-13f * xabs);
    const float r2 = 2.0f * xabs;
    const float r2_7 = r2 * r2 * r2 * r2 * r2 * r2 * r2;
    const float tr2 = __fdividef(r2_7, 18.0f * (1.0f - r2)) * kUp;
    const float x3 = xabs * xabs * xabs;
    h.D2 = D2;
    h.e2 = 1.1f * (M[2] * ((1.0f + 3.0f * xabs) * Exd + 2.0e3f * e2u * xabs +
                           100.0f * uu * x3 + tr2) +
                   2.0f * uu * (fabsf(lead.hi) + fabsf(tail)) +
                   2.0f * rho.hi * (xabs + Exd) * Exd * Exd);
  }
  float alpha = 1.0f;
  const int k = decide32(h, alpha, kChordWidth);
  if (k == kUndecided) {
    // the double-float leading terms (DFS) may still decide it
    r.flags = DFS ? NF_FAR : (NF_FAR | NF_REFINE);
    return;
  }
  r.alpha = alpha;
  r.flags = NF_BAND | (k == kAcceptTwo ? (NF_ACCEPT_TWO | NF_ACCEPT_STAR)
                                       : NF_FORMULA);
}

// d0, dd: FP32 deviations delta_i of the rest population and the pairs
// (registers).  corr_rho / corr: used only for plain FP32 storage
// (delta_i = v_i - s_i, s_i = fl(W_i rho0)), where corr_rho = sum_i s_i -
// rho0 and corr_i = W_i rho0 - s_i.
template <class L, bool SHIFTED>
__device__ __forceinline__ void node32_formula(
    float d0, const float2 (&dd)[npairs<L>()], float rho0, float corr_rho,
    const float* __restrict__ corr, float a_extra, N32<L>& r,
    bool exact = false) {
  constexpr int Q = L::Q;
  constexpr int P = npairs<L>();
  constexpr float uu = 5.9604645e-8f;  // 2^-24
  r.flags = 0;
  r.alpha = 2.0f;

  // ---- exact mass and momentum: delta = hi + lo, hi on a 2^-20 grid ------
  const float hi0 = (d0 + 12.0f) - 12.0f;
  float2 hi[P], lo[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    hi[k] = add2(add2(dd[k], f2(12.0f)), f2(-12.0f));
    lo[k] = sub2(dd[k], hi[k]);
  }
  float h0, hx, hy, hz, l0, lx, ly, lz;
  moments2<L>(hi0, hi, h0, hx, hy, hz);
  moments2<L>(d0 - hi0, lo, l0, lx, ly, lz);
  float drho = h0 + l0;
  if (!SHIFTED) drho += corr_rho;
  const float j[3] = {hx + lx, hy + ly, hz + lz};
  const float rho = rho0 + drho;
  r.drho = drho;
  r.rho = rho;
  r.j[0] = j[0];
  r.j[1] = j[1];
  r.j[2] = j[2];
  if (!(rho > 0.0f) || !isfinite(rho)) {
    r.flags = NF_FAR;          // the FP64 fixup classifies the state
    return;
  }
  const float inv_rho = rcp_approx(rho);

  // ---- per-axis equilibrium factors -------------------------------------
  float dp[3], dm[3], dz[3];
  float U = 0.0f;
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    const float u = j[a] * inv_rho;
    U = fmaxf(U, fabsf(u));
    // s = 3u^2 / (1 + sqrt(1 + 3u^2)), relative error <= 9.5 u (numerator
    // 2 u, 1 + 3u^2 2 u, its root via rsqrt_approx 6 u, 1 + root 4.5 u, the
    // reciprocal 2 u, the product u)
    const float y = fmaf(3.0f * u, u, 1.0f);
    const float s = 3.0f * u * u * rcp_approx(1.0f + y * rsqrt_approx(y));
    dp[a] = fmaf(3.0f, u, 2.0f * s);
    dm[a] = fmaf(-3.0f, u, 2.0f * s);
    dz[a] = -s;
  }
  if (!(U < kUMax32)) {
    r.flags = NF_FAR;
    return;
  }
  // factor pairs: lane x takes d(c), lane y takes d(-c)
  auto fac = [&](int a, int c) {
    return c == 1 ? make_float2(dp[a], dm[a])
                  : (c == -1 ? make_float2(dm[a], dp[a]) : f2(dz[a]));
  };
  // two-axis products (1 + a)(1 + b) - 1 for lane-x velocities (cx, cy);
  // entries no pair uses are never evaluated
  float2 pxy[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float2 da = fac(0, a - 1), db = fac(1, b - 1);
      pxy[a][b] = fma2(da, db, add2(da, db));
    }

  // ---- n_i, x_i and the moments M_2..M_4 ---------------------------------
  // A population f_i <= 0 gives |x_i| >= 1 (f^eq_i > 0), so invalid states
  // leave through the far branch, where the FP64 fixup flags them.
  // per weight class: W rho, W drho, W rho0
  float wr[4], wd[4], w0[4];
#pragma unroll
  for (int k = 0; k <= L::D; ++k) {
    const float wk = k == 0 ? L::wf(0) : L::wf(k == 1 ? 1 : (k == 2 ? 7 : 19));
    wr[k] = wk * rho;
    wd[k] = wk * drho;
    w0[k] = wk * rho0;
  }
  float M2, M3, M4, xabs, gmax;
  {   // rest population
    float pm1 = pxy[1][1].x;
    if (L::D == 3) pm1 = fmaf(pm1, dz[2], pm1 + dz[2]);
    float deq = fmaf(wr[0], pm1, wd[0]);
    if (!SHIFTED) deq += corr[0];
    const float ni = deq - d0;
    r.n0 = ni;
    const float rf = rcp_approx(w0[0] + d0);
    const float x = ni * rf;
    xabs = fabsf(x);
    gmax = wr[0] * rf;                         // W rho / f
    M2 = ni * x;                               // f x^2
    M3 = M2 * x;                               // f x^3
    M4 = M3 * x;                               // f x^4
  }
  float2 m2 = f2(0.0f), m3 = f2(0.0f), m4 = f2(0.0f);
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int i = 2 * k + 1;
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    float2 pm1 = pxy[cidx(cx)][cidx(cy)];
    if (L::D == 3) {
      const float2 a2 = fac(2, cz);
      pm1 = fma2(pm1, a2, add2(pm1, a2));
    }
    const int kc = wclass<L>(i);
    float2 deq = fma2(f2(wr[kc]), pm1, f2(wd[kc]));  // W (drho + rho (P - 1))
    if (!SHIFTED) deq = add2(deq, make_float2(corr[i], corr[i + 1]));
    const float2 ni = sub2(deq, dd[k]);
    r.n2[k] = ni;
    const float2 rf = rcp_approx2(add2(f2(w0[kc]), dd[k]));
    const float2 x = mul2(ni, rf);
    xabs = fmaxf(xabs, fmaxf(fabsf(x.x), fabsf(x.y)));
    const float2 gw = mul2(f2(wr[kc]), rf);
    gmax = fmaxf(gmax, fmaxf(gw.x, gw.y));
    const float2 q1 = mul2(ni, x);
    const float2 q2 = mul2(q1, x);
    if (k == 0) {
      m2 = q1;
      m3 = q2;
      m4 = mul2(q2, x);
    } else {
      m2 = add2(m2, q1);
      m3 = add2(m3, q2);
      m4 = fma2(q2, x, m4);
    }
  }
  M2 += m2.x + m2.y;
  M3 += m3.x + m3.y;
  M4 += m4.x + m4.y;
  if (!(xabs <= 0.125f)) {   // far from equilibrium, invalid, or NaN
    r.flags = NF_FAR;
    return;
  }
  if (xabs == 0.0f) {
    // f^eq == f in FP32 only: the exact state may still differ from its
    // equilibrium below FP32 resolution; the second stage decides.  The
    // provisional alpha = 1 (f* = f^eq) keeps H(f*) <= H(f) exactly; the
    // relaxation leaves f unchanged either way (n = 0).
    r.flags = NF_REFINE | NF_DEGENERATE;
    r.alpha = 1.0f;
    return;
  }
  // longer series for nodes further from equilibrium
  const bool k8 = xabs > 0.01f;
  float M[9] = {0.f, 0.f, M2, M3, M4, 0.f, 0.f, 0.f, 0.f};
  if (k8) {
    {
      const float x = r.n0 * rcp_approx(w0[0] + d0);
      const float x2 = x * x;
      float p = r.n0 * x2 * x2;   // n x^4 = f x^5
      M[5] = p;
      p *= x;
      M[6] = p;
      p *= x;
      M[7] = p;
      p *= x;
      M[8] = p;
    }
    float2 m5 = f2(0.0f), m6 = f2(0.0f), m7 = f2(0.0f), m8 = f2(0.0f);
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int kc = wclass<L>(2 * k + 1);
      const float2 x = mul2(r.n2[k], rcp_approx2(add2(f2(w0[kc]), dd[k])));
      const float2 x2 = mul2(x, x);
      float2 p = mul2(mul2(r.n2[k], x2), x2);
      m5 = add2(m5, p);
      p = mul2(p, x);
      m6 = add2(m6, p);
      p = mul2(p, x);
      m7 = add2(m7, p);
      p = mul2(p, x);
      m8 = add2(m8, p);
    }
    M[5] += m5.x + m5.y;
    M[6] += m6.x + m6.y;
    M[7] += m7.x + m7.y;
    M[8] += m8.x + m8.y;
  }

  // ---- error bounds -------------------------------------------------------
  const float Dd = fmaf(3.0f * U, U, 3.0f * U);      // max |d_a|
  const float Eu = 4.0f * uu * U + 2e-11f * inv_rho;
  // |d(d)/du| <= 3 + 6U; rounding of d = fma(+-3, u, 2s): u (3U + 3U^2),
  // of 2s: 19 u s <= 28.5 u U^2
  const float Ed = (3.0f + 6.0f * U) * Eu + 6.0f * uu * U * (1.0f + 5.5f * U);
  const float opd2 = (1.0f + Dd) * (1.0f + Dd);
  const float EP = (3.0f * Ed + 18.0f * uu * Dd) * opd2;
  const float omd = 1.0f - Dd;
  const float omdD = L::D == 3 ? omd * omd * omd : omd * omd;
  // upper bound of a positive quotient: the 2-ulp approximate division
  // raised by 2^-20 (covers its error and the product's rounding)
  constexpr float kUp = 1.00000095367431640625f;   // 1 + 2^-20
  // G >= max_i W_i rho / f_i: the a-priori bound (1 + xabs) / (1 - Dd)^D,
  // or the node's own maximum gmax of W_i rho fl(1 / fl(W_i rho0 + delta_i))
  // when smaller.  gmax kUp covers the reciprocal's and the products'
  // rounding; the sum fl(W_i rho0 + delta_i) is within u (W_i rho0 + f_i)
  // of f_i, which the division by 1 - u - u gmax kUp rho0 / rho covers
  // (the denominator stays above 1/2 whenever the result is used).
  const float Gb = __fdividef(1.0f + xabs, omdD) * kUp;
  const float gk = gmax * kUp;
  const float den =
      1.0f - uu - uu * gk * (rho0 * inv_rho * 1.01f);
  const float G =
      den > 0.5f ? fminf(Gb, __fdividef(gk, den) * kUp) : Gb;
  const float Ex =
      1.05f * (G * (EP + 3.0f * uu * (fabsf(drho) * inv_rho + 3.0f * Dd) +
                    2e-11f * inv_rho + a_extra) +
               6.0f * uu * xabs);
  const DH32 h = series_dh32<Q>(M, k8, xabs, Ex, rho);
  float alpha = 2.0f;
  const int k = decide32(h, alpha, exact ? kChordWidth : INFINITY);
  if (k == kUndecided) {
    // The sign of Delta H(2) or of Delta H(1) is within the FP32 error.
    // Without a second stage (exact false) the node takes the certified
    // alpha -- the Eq. (9) chord on the upper bounds, rounded down, when
    // Delta H(1) + e1 < 0, else 1 (f* = f^eq) -- for which
    // H(f*(alpha)) <= H(f) holds too.  With it, the node is written
    // provisionally with the nominal FP32 decision (alpha = 2 when
    // Delta H(2) <= 0, else the chord of the nominal values), which the
    // second stage (node32_refine) usually confirms, so that few
    // populations need rewriting.
    r.flags = NF_REFINE | NF_BAND;
    r.alpha = exact ? (h.D2 <= 0.0f
                           ? 2.0f
                           : (h.D1 < 0.0f
                                  ? 2.0f - __fdividef(h.D2, h.D2 - h.D1)
                                  : 1.0f))
                    : certified_alpha32(h);
    return;
  }
  r.alpha = alpha;
  r.flags = k == kAcceptTwo ? (NF_ACCEPT_TWO | NF_ACCEPT_STAR) : NF_FORMULA;
}

// Conservation projection of n (applied to the relaxation only): removes
// the mass/momentum that rounding left in n,
//   n_i <- n_i - W_i (r0 + 3 c_i . r),  r0 = sum n_i,  r = sum c_i n_i,
// using sum W = 1 and sum W c c = I / 3.  Emits W_i t_i through
// emit0(W_0 t_0) for the rest population and emit2(k, (W t) of pair k).
template <class L, class Emit0, class Emit2>
__device__ __forceinline__ void projection(const N32<L>& r, Emit0 emit0,
                                           Emit2 emit2) {
  float r0, rx, ry, rz;
  moments2<L>(r.n0, r.n2, r0, rx, ry, rz);
  // t for lane-x velocity c in lane x and for -c in lane y
  const float2 R0 = f2(r0), RX = f2(rx), RY = f2(ry), RZ = f2(rz);
  float2 tx[3], txy[3][3];
  tx[1] = R0;
  tx[2] = fma2(lane_sign(3), RX, R0);
  tx[0] = fma2(lane_sign(-3), RX, R0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    txy[a][1] = tx[a];
    txy[a][2] = fma2(lane_sign(3), RY, tx[a]);
    txy[a][0] = fma2(lane_sign(-3), RY, tx[a]);
  }
  emit0(L::wf(0) * r0);
#pragma unroll
  for (int k = 0; k < npairs<L>(); ++k) {
    const int i = 2 * k + 1;
    const int cz = L::c(i, 2);
    float2 t = txy[cidx(L::c(i, 0))][cidx(L::c(i, 1))];
    if (cz != 0) t = fma2(lane_sign(3 * cz), RZ, t);
    emit2(k, mul2(f2(L::wf(i)), t));
  }
}

}  // namespace elbm
