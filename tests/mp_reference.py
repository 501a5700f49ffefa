"""High-precision (mpmath) reference computations used to pin the oracle.

Nothing here reuses the oracle's formulas: the equilibrium is found by a
Newton solve for the Lagrange multipliers of the constrained entropy
minimum (no closed form), entropy differences are taken literally as
H(f*) - H(f) at 60 significant digits, and the root of Eq. (4) comes from
a 200-step bisection at that precision.
"""
import mpmath as mp

mp.mp.dps = 60


def mpf_vec(v):
    return [mp.mpf(float(a)) for a in v]


def moments(c, f):
    d = len(c[0])
    rho = mp.fsum(f)
    j = [mp.fsum(ci[a] * fi for ci, fi in zip(c, f)) for a in range(d)]
    return rho, j


def equilibrium(c, w, rho, j):
    """Minimiser of sum f ln(f/W) with sum f = rho, sum c f = j: stationarity
    gives f_i = W_i exp(l0 + l . c_i); solve the constraints for (l0, l) by
    Newton's method."""
    d = len(c[0])
    lam = [mp.log(rho)] + [mp.mpf(0)] * d
    for _ in range(200):
        f = [wi * mp.exp(lam[0] + mp.fsum(lam[1 + a] * ci[a]
                                          for a in range(d)))
             for ci, wi in zip(c, w)]
        basis = [[mp.mpf(1)] + [mp.mpf(ci[a]) for a in range(d)] for ci in c]
        g = [mp.fsum(f[i] * basis[i][k] for i in range(len(c)))
             for k in range(d + 1)]
        target = [rho] + list(j)
        r = [g[k] - target[k] for k in range(d + 1)]
        J = mp.matrix(d + 1, d + 1)
        for k in range(d + 1):
            for m in range(d + 1):
                J[k, m] = mp.fsum(f[i] * basis[i][k] * basis[i][m]
                                  for i in range(len(c)))
        step = mp.lu_solve(J, mp.matrix(r))
        lam = [lam[k] - step[k] for k in range(d + 1)]
        if max(abs(s) for s in step) < mp.mpf(10) ** (-50):
            break
    return [wi * mp.exp(lam[0] + mp.fsum(lam[1 + a] * ci[a] for a in range(d)))
            for ci, wi in zip(c, w)]


def entropy(w, f):
    return mp.fsum(fi * mp.log(fi / wi) for fi, wi in zip(f, w) if fi > 0)


class Node:
    """One population vector, with its exact-to-60-digits equilibrium."""

    def __init__(self, c, w, f):
        self.c = [[int(v) for v in ci] for ci in c]
        self.w = mpf_vec(w)
        self.f = mpf_vec(f)
        rho, j = moments(self.c, self.f)
        self.feq = equilibrium(self.c, self.w, rho, j)
        self.h0 = entropy(self.w, self.f)

    def fstar(self, alpha):
        alpha = mp.mpf(alpha)
        out = []
        for fi, ei in zip(self.f, self.feq):
            v = fi + alpha * (ei - fi)
            out.append(v if v > 0 else mp.mpf(0))
        return out

    def delta_h(self, alpha):
        """H(f*(alpha)) - H(f), literally."""
        return entropy(self.w, self.fstar(alpha)) - self.h0

    def alpha_max(self):
        cands = [fi / (fi - ei) for fi, ei in zip(self.f, self.feq) if ei < fi]
        return min(cands) if cands else mp.inf

    def root(self):
        """Non-trivial root alpha_bar of Eq. (4) on [1, alpha_max], or None
        when Delta H(alpha_max) <= 0."""
        lo, hi = mp.mpf(1), self.alpha_max()
        if self.delta_h(hi) <= 0:
            return None
        for _ in range(200):
            mid = (lo + hi) / 2
            if self.delta_h(mid) > 0:
                hi = mid
            else:
                lo = mid
        return (lo + hi) / 2

    def slope(self, alpha):
        """d Delta H / d alpha = sum (f^eq - f) ln(f*_i / W_i)."""
        fs = self.fstar(alpha)
        return mp.fsum((ei - fi) * mp.log(si / wi)
                       for fi, ei, si, wi in zip(self.f, self.feq, fs, self.w))
