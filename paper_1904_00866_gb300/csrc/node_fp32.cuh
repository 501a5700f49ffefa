// FP32 per-node FORMULA arithmetic with a certified entropy decision.
//
// Populations arrive as delta_i = f_i - W_i rho0 (FP32, exact), so the
// non-equilibrium part n_i = f^eq_i - f_i is formed without the O(1)
// cancellation of f^eq_i - f_i:
//   f^eq_i - W_i rho0 = W_i (drho + rho (P_i - 1)),  drho = sum_i delta_i,
//   P_i - 1 = prod_a (1 + d_a(c_ia)) - 1,  d(0) = -s, d(+-1) = +-3u + 2s,
//   s = 3u^2 / (1 + sqrt(1 + 3u^2))          (entropic equilibrium, Eq. (3)).
//
// The entropy changes needed by Eqs. (8)-(9) come from the moments
// M_k = sum_i f_i x_i^k = sum_i n_i x_i^(k-1), x_i = n_i / f_i:
//   Delta H(alpha) = sum_{k>=2} (-1)^k (alpha^k - k alpha) / (k (k-1)) M_k,
// the Taylor series of sum f [phi(alpha x) - alpha x ln(1 + x)] (the linear
// term alpha sum f x is exactly zero).  At alpha = 2 the k = 2 coefficient
// vanishes, so Delta H(2) carries no O(x^2) cancellation.  Truncated after
// k = 6; |x_i| <= 1/8 is required (other nodes go to FP64).
//
// Every quantity below has an a-priori bound on its FP32 error (unit
// roundoff u = 2^-24):  E_x bounds |x_i - x_i exact| from the moment sums,
// the equilibrium products and the division; e2 / e1 bound the errors of
// Delta H(2) / Delta H(1) from E_x (first and second order), the series
// rounding and the truncation.  Decision ladder, each rung H-safe for the
// stored state:
//   Delta H(2) + e2 <= 0                -> alpha = 2 (acceptance, Eq. (8));
//   else Delta H(1) + e1 < 0            -> alpha = Eq. (9) chord evaluated on
//                                          the upper bounds, rounded down
//                                          (chord root decreases in both
//                                          values, so it stays below the
//                                          exact Eq. (9) value <= root);
//   else (node within FP32 noise of equilibrium) -> alpha = 1, for which
//                                          H(f*) = H(f^eq) <= H(f) exactly.
// When |Delta H(2)| <= e2 the decision is flagged NF_BAND.
#pragma once
#include <math.h>

#include "lattice.cuh"
#include "node_fp64.cuh"

namespace elbm {

template <int N>
__device__ __forceinline__ float tree_sum(float (&t)[N]) {
#pragma unroll
  for (int w = 1; w < N; w *= 2) {
#pragma unroll
    for (int i = 0; i + w < N; i += 2 * w) t[i] += t[i + w];
  }
  return t[0];
}

__host__ __device__ constexpr int ceil_log2(int n) {
  return n <= 1 ? 0 : 1 + ceil_log2((n + 1) / 2);
}

template <class L>
__host__ __device__ constexpr int n_nonzero(int a) {
  int k = 0;
  for (int i = 0; i < L::Q; ++i) k += L::c(i, a) != 0;
  return k;
}

struct Node32Result {
  float alpha;
  unsigned flags;
  float drho;   // rho - rho0
  float rho;
  float j[3];   // momentum
};

// delta: FP32 deviations (f_i = W_i rho0 + delta_i); n: out, f^eq_i - f_i.
// corr_rho / corr: zero for shifted storage; for plain FP32 storage, where
// delta_i = v_i - s_i with s_i = fl(W_i rho0), corr_rho = sum_i s_i - rho0
// and corr_i = W_i rho0 - s_i.
// Returns with NF_FAR set when the node must be redone in FP64.
template <class L>
__device__ __forceinline__ Node32Result node32_formula(
    const float (&dl)[L::Q], float (&n)[L::Q], float rho0, float corr_rho,
    const float* __restrict__ corr) {
  constexpr int Q = L::Q;
  constexpr float uu = 5.9604645e-8f;  // 2^-24
  Node32Result r;
  r.flags = 0;

  // ---- mass and momentum (pairwise sums, height H) --------------------
  float t[Q];
  float A = 0.0f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    t[i] = dl[i];
    A += fabsf(dl[i]);
  }
  const float drho = tree_sum(t) + corr_rho;
  float j[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    constexpr int NZ = n_nonzero<L>(0);
    float tj[NZ];
    int k = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (L::c(i, a) == 1) tj[k++] = dl[i];
      if (L::c(i, a) == -1) tj[k++] = -dl[i];
    }
    j[a] = tree_sum(tj);
  }
  const float rho = rho0 + drho;
  r.drho = drho;
  r.rho = rho;
  r.j[0] = j[0];
  r.j[1] = j[1];
  r.j[2] = j[2];
  if (!(rho > 0.0f) || !isfinite(rho)) {
    r.flags = NF_BAD_NONFINITE;
    r.alpha = 2.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) n[i] = 0.0f;
    return r;
  }
  const float inv_rho = 1.0f / rho;

  // ---- per-axis equilibrium factors -------------------------------------
  float dp[3], dm[3], d0[3];
  float U = 0.0f;
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    const float u = j[a] * inv_rho;
    U = fmaxf(U, fabsf(u));
    const float s = 3.0f * u * u / (1.0f + sqrtf(fmaf(3.0f * u, u, 1.0f)));
    dp[a] = fmaf(3.0f, u, 2.0f * s);
    dm[a] = fmaf(-3.0f, u, 2.0f * s);
    d0[a] = -s;
  }
  if (!(U < 0.5f)) {   // far outside the FP32 series regime
    r.flags = (U < 1.0f) ? NF_FAR : NF_BAD_NONFINITE;
    r.alpha = 2.0f;
    return r;
  }

  // ---- n_i, x_i and the moments M_2..M_6 ---------------------------------
  float M2 = 0.f, M3 = 0.f, M4 = 0.f, M5 = 0.f, M6 = 0.f, S1 = 0.f;
  float xabs = 0.0f;
  bool nonpos = false;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const float a0 = cx == 1 ? dp[0] : (cx == -1 ? dm[0] : d0[0]);
    const float a1 = cy == 1 ? dp[1] : (cy == -1 ? dm[1] : d0[1]);
    float pm1 = fmaf(a0, a1, a0 + a1);            // (1+a0)(1+a1) - 1
    if (L::D == 3) {
      const float a2 = cz == 1 ? dp[2] : (cz == -1 ? dm[2] : d0[2]);
      pm1 = fmaf(pm1, a2, pm1 + a2);
    }
    const float wf = (float)L::w(i);
    float deq = wf * fmaf(rho, pm1, drho);
    if (corr) deq += corr[i];
    const float ni = deq - dl[i];
    n[i] = ni;
    const float fi = fmaf(wf, rho0, dl[i]);
    nonpos |= !(fi > 0.0f);
    const float x = __fdividef(ni, fi);
    xabs = fmaxf(xabs, fabsf(x));
    S1 += fabsf(ni);
    float p = ni * x;
    M2 += p;
    p *= x;
    M3 += p;
    p *= x;
    M4 += p;
    p *= x;
    M5 += p;
    p *= x;
    M6 += p;
  }
  if (nonpos) {
    r.flags = NF_BAD_NEG;
    r.alpha = 2.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) n[i] = 0.0f;
    return r;
  }
  if (!(xabs <= 0.125f)) {   // includes NaN
    r.flags = isfinite(xabs) ? NF_FAR : NF_BAD_NONFINITE;
    r.alpha = 2.0f;
    return r;
  }
  if (xabs == 0.0f) {        // f^eq == f in FP32
    r.flags = NF_DEGENERATE;
    r.alpha = 2.0f;
    return r;
  }

  // ---- error bounds --------------------------------------------------------
  constexpr int H = ceil_log2(Q) > ceil_log2(n_nonzero<L>(0))
                        ? ceil_log2(Q)
                        : ceil_log2(n_nonzero<L>(0));
  const float a = A * inv_rho;                       // sum |delta| / rho
  const float Dd = fmaf(3.0f * U, U, 3.0f * U);      // max |d_a|
  const float gh = (float)H * uu * 1.01f;
  const float Eu = gh * a * (1.0f + U) + 4.0f * uu * U;
  const float Ed = (3.0f + 6.0f * U) * Eu + 6.0f * uu * U * (1.0f + 2.5f * U);
  const float opd2 = (1.0f + Dd) * (1.0f + Dd);
  const float EP = (3.0f * Ed + 18.0f * uu * Dd) * opd2;
  float omd = 1.0f - Dd;
  float omdD = omd * omd;
  if (L::D == 3) omdD *= omd;
  const float G = (1.0f + xabs) / omdD;
  const float Ex =
      1.05f * (G * (gh * a * (2.0f + 3.0f * Dd) + EP +
                    3.0f * uu * (fabsf(drho) * inv_rho + 3.0f * Dd) +
                    2.0f * uu * a) +
               8.0f * uu * xabs);
  const float gq = (float)(Q + 6) * uu * 1.01f;

  // Delta H(2) and Delta H(1) from the series, c_k(alpha) = (-1)^k
  // (alpha^k - k alpha) / (k (k-1)):  c(2) = {0, -1/3, 2/3, -11/10, 26/15},
  // c(1) = {-1/2, 1/3, -1/4, 1/5, -1/6}.
  const float D2 = fmaf(-1.0f / 3.0f, M3,
                        fmaf(2.0f / 3.0f, M4,
                             fmaf(-1.1f, M5, (26.0f / 15.0f) * M6)));
  const float D1 =
      fmaf(-0.5f, M2,
           fmaf(1.0f / 3.0f, M3,
                fmaf(-0.25f, M4, fmaf(0.2f, M5, (-1.0f / 6.0f) * M6))));
  const float r2 = 2.0f * xabs;
  const float r2_5 = r2 * r2 * r2 * r2 * r2;
  const float x5 = xabs * xabs * xabs * xabs * xabs;
  const float e2 =
      M2 * (2.02f * Ex +
            gq * xabs * (0.34f + xabs * (0.7f + xabs * (1.2f + 1.8f * xabs))) +
            4.0f * r2_5 / (42.0f * (1.0f - r2))) +
      4.0f * uu *
          (fabsf(M3) * (1.0f / 3.0f) + fabsf(M4) * (2.0f / 3.0f) +
           fabsf(M5) * 1.1f + fabsf(M6) * 1.74f) +
      2.0f * rho * (xabs + Ex) * Ex * Ex;
  const float e1 = Ex * S1 / (1.0f - xabs) +
                   M2 * (gq * (0.5f + xabs) + x5 / (7.0f * (1.0f - xabs))) +
                   4.0f * uu * (0.5f * M2 + fabsf(M3)) + 2.0f * rho * Ex * Ex;

  const float D2hi = __fadd_ru(D2, e2);
  if (D2hi <= 0.0f) {
    r.flags = NF_ACCEPT_TWO | NF_ACCEPT_STAR;
    r.alpha = 2.0f;
    return r;
  }
  const bool band = __fsub_rd(D2, e2) <= 0.0f;
  const float D1hi = __fadd_ru(D1, e1);
  if (D1hi < 0.0f) {
    // alpha = 2 + D2hi / (D2hi - D1hi) (1 - 2), rounded down
    const float den = __fsub_rd(D2hi, D1hi);
    const float tt = __fdiv_ru(D2hi, den);
    r.alpha = __fsub_rd(2.0f, tt);
    r.flags = NF_FORMULA | (band ? NF_BAND : 0u);
  } else {
    r.alpha = 1.0f;
    r.flags = NF_FORMULA | NF_BAND;
  }
  return r;
}

}  // namespace elbm
