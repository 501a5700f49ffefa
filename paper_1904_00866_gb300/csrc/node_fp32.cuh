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
// truncation.  Decision ladder, each rung H-safe for the stored state:
//   Delta H(2) + e2 <= 0   -> alpha = 2 (acceptance after Eq. (8));
//   else Delta H(1) + e1 < 0 -> alpha = Eq. (9) chord evaluated on the upper
//                              bounds and rounded down (the chord root
//                              decreases in both values, so it stays at or
//                              below the exact Eq. (9) value, which is at or
//                              below the root of Eq. (4));
//   else (node within FP32 noise of equilibrium) -> alpha = 1, for which
//                              H(f*) = H(f^eq) <= H(f) holds exactly.
// A node whose n evaluates to exactly zero in FP32 (the degenerate case of
// the paper seen at FP32 resolution) also takes alpha = 1.
// When |Delta H(2)| <= e2 the decision is flagged NF_BAND.
//
// Opposite-velocity populations are processed in pairs with packed f32x2
// arithmetic (see npairs below); every lane operation rounds like its
// scalar form, so only the order of the moment sums differs from a scalar
// loop, which the summation error term of the bounds covers.
#pragma once
#include <math.h>

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

// 1 / y by the SFU (rcp.approx.ftz.f32, relative error below 2^-23).
__device__ __forceinline__ float rcp_approx(float y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
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

// d0, dd: FP32 deviations delta_i of the rest population and the pairs
// (registers).  corr_rho / corr: used only for plain FP32 storage
// (delta_i = v_i - s_i, s_i = fl(W_i rho0)), where corr_rho = sum_i s_i -
// rho0 and corr_i = W_i rho0 - s_i.
template <class L, bool SHIFTED>
__device__ __forceinline__ void node32_formula(
    float d0, const float2 (&dd)[npairs<L>()], float rho0, float corr_rho,
    const float* __restrict__ corr, float a_extra, N32<L>& r) {
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
    const float s = 3.0f * u * u / (1.0f + sqrtf(fmaf(3.0f * u, u, 1.0f)));
    dp[a] = fmaf(3.0f, u, 2.0f * s);
    dm[a] = fmaf(-3.0f, u, 2.0f * s);
    dz[a] = -s;
  }
  if (!(U < 0.5f)) {
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
  float M2, M3, M4, xabs;
  {   // rest population
    float pm1 = pxy[1][1].x;
    if (L::D == 3) pm1 = fmaf(pm1, dz[2], pm1 + dz[2]);
    float deq = fmaf(wr[0], pm1, wd[0]);
    if (!SHIFTED) deq += corr[0];
    const float ni = deq - d0;
    r.n0 = ni;
    const float x = ni * rcp_approx(w0[0] + d0);
    xabs = fabsf(x);
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
    const float2 x = mul2(ni, rcp_approx2(add2(f2(w0[kc]), dd[k])));
    xabs = fmaxf(xabs, fmaxf(fabsf(x.x), fabsf(x.y)));
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
    // equilibrium below FP32 resolution, where alpha = 2 can raise H by a
    // rounding-level amount.  alpha = 1 (f* = f^eq) keeps H(f*) <= H(f)
    // exactly; the relaxation writes f unchanged either way (n = 0).
    r.flags = NF_DEGENERATE;
    r.alpha = 1.0f;
    return;
  }
  // longer series for nodes further from equilibrium
  const bool k8 = xabs > 0.01f;
  float M5 = 0.f, M6 = 0.f, M7 = 0.f, M8 = 0.f;
  if (k8) {
    {
      const float x = r.n0 * rcp_approx(w0[0] + d0);
      const float x2 = x * x;
      float p = r.n0 * x2 * x2;   // n x^4 = f x^5
      M5 = p;
      p *= x;
      M6 = p;
      p *= x;
      M7 = p;
      p *= x;
      M8 = p;
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
    M5 += m5.x + m5.y;
    M6 += m6.x + m6.y;
    M7 += m7.x + m7.y;
    M8 += m8.x + m8.y;
  }

  // ---- error bounds -------------------------------------------------------
  const float Dd = fmaf(3.0f * U, U, 3.0f * U);      // max |d_a|
  const float Eu = 4.0f * uu * U + 2e-11f * inv_rho;
  const float Ed = (3.0f + 6.0f * U) * Eu + 6.0f * uu * U * (1.0f + 2.5f * U);
  const float opd2 = (1.0f + Dd) * (1.0f + Dd);
  const float EP = (3.0f * Ed + 18.0f * uu * Dd) * opd2;
  const float omd = 1.0f - Dd;
  const float omdD = L::D == 3 ? omd * omd * omd : omd * omd;
  const float G = (1.0f + xabs) / omdD;
  const float Ex =
      1.05f * (G * (EP + 3.0f * uu * (fabsf(drho) * inv_rho + 3.0f * Dd) +
                    2e-11f * inv_rho + a_extra) +
               6.0f * uu * xabs);
  const float gq = (float)(Q + 9) * uu * 1.01f;

  // c_k(alpha) = (-1)^k (alpha^k - k alpha) / (k (k-1))
  // c(2): k=3..8: -1/3, 2/3, -11/10, 26/15, -19/7, 30/7
  // c(1): k=2..8: -1/2, 1/3, -1/4, 1/5, -1/6, 1/7, -1/8
  float D2 = fmaf(-1.0f / 3.0f, M3, (2.0f / 3.0f) * M4);
  float D1 = fmaf(-0.5f, M2, fmaf(1.0f / 3.0f, M3, -0.25f * M4));
  float tr2, tr1, rnd;
  const float r2 = 2.0f * xabs;
  if (k8) {
    D2 = fmaf(-1.1f, M5, fmaf(26.0f / 15.0f, M6, fmaf(-19.0f / 7.0f, M7,
                                                  fmaf(30.0f / 7.0f, M8, D2))));
    D1 = fmaf(0.2f, M5, fmaf(-1.0f / 6.0f, M6,
                             fmaf(1.0f / 7.0f, M7, fmaf(-0.125f, M8, D1))));
    const float r2_7 = r2 * r2 * r2 * r2 * r2 * r2 * r2;
    const float x7 = xabs * xabs * xabs * xabs * xabs * xabs * xabs;
    // tails sum_{k>=9}: |c_k(2)| <= 2^k / (k (k-1)), |c_k(1)| = 1 / k,
    // |M_k| <= xabs^(k-2) M_2
    tr2 = r2_7 / (18.0f * (1.0f - r2));
    tr1 = x7 / (9.0f * (1.0f - xabs));
    rnd = fabsf(M5) * 1.1f + fabsf(M6) * 1.74f + fabsf(M7) * 2.72f +
          fabsf(M8) * 4.29f;
  } else {
    // tails sum_{k>=5}
    const float r2_3 = r2 * r2 * r2;
    tr2 = r2_3 * 0.2f / (1.0f - r2);
    tr1 = xabs * xabs * xabs / (5.0f * (1.0f - xabs));
    rnd = 0.0f;
  }
  const float e2 =
      M2 * (2.02f * Ex +
            gq * xabs * (0.34f + xabs * (0.7f + xabs * (1.2f + 1.8f * xabs))) +
            tr2) +
      4.0f * uu * (fabsf(M3) * (1.0f / 3.0f) + fabsf(M4) * (2.0f / 3.0f) + rnd) +
      2.0f * rho * (xabs + Ex) * Ex * Ex;
  const float S1b = sqrtf(rho * M2);   // >= sum f |x|  (Cauchy-Schwarz)
  const float e1 = 1.01f * Ex * S1b / (1.0f - xabs) +
                   M2 * (gq * (0.5f + xabs) + tr1) +
                   4.0f * uu * (0.5f * M2 + fabsf(M3)) + 2.0f * rho * Ex * Ex;

  const float D2hi = __fadd_ru(D2, e2);
  if (D2hi <= 0.0f) {
    r.flags = NF_ACCEPT_TWO | NF_ACCEPT_STAR;
    r.alpha = 2.0f;
    return;
  }
  const float D1hi = __fadd_ru(D1, e1);
  if (!(D1hi < 0.0f)) {
    // Within FP32 noise of equilibrium: neither sign is certified, but
    // alpha = 1 (f* = f^eq) satisfies H(f*) <= H(f) exactly.  Here n is at
    // the level of the FP32 error of the equilibrium, so the relaxation
    // rate it implies is immaterial.
    r.flags = NF_FORMULA | NF_BAND;
    r.alpha = 1.0f;
    return;
  }
  const bool band = __fsub_rd(D2, e2) <= 0.0f;
  // alpha = 2 + D2hi / (D2hi - D1hi) (1 - 2), rounded down
  // t = D2hi / (D2hi - D1hi) rounded up: the approximate quotient (error
  // <= 2 ulp) is raised by 4 ulp
  const float den = __fsub_rd(D2hi, D1hi);
  const float tt = __fmul_ru(__fdividef(D2hi, den), 1.0f + 2.384185791e-7f);
  r.alpha = __fsub_rd(2.0f, tt);
  r.flags = NF_FORMULA | (band ? NF_BAND : 0u);
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
