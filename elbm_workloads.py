"""Seeded synthetic inputs for the ELBM hot path: initial density/velocity
fields and request mixes.

This module holds no arithmetic of the method (no equilibrium, no entropy,
no relaxation): it only builds the analytic initial conditions and the random
workload mixes that both the CUDA path and the CPU oracle consume.  Fields are
float64 numpy arrays in the library's layout: rho is (nz, ny, nx) and u is
(d, nz, ny, nx), x fastest.

Workloads (all periodic, lattice units):
  * 2D Taylor-Green vortex: u_x = -u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky),
    k = 2 pi / n, density either uniform or consistent with the analytic
    pressure p = p0 - rho0 u0^2 / 4 (cos 2kx + cos 2ky).
  * 3D Taylor-Green vortex: u = u0 sin x cos y cos z, v = -u0 cos x sin y cos z,
    w = 0 on [0, 2 pi)^3, p = p0 + rho0 u0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2).
  * Double shear layer of the paper's second experiment on [0, 1]^2 (nodes at
    i/n): u_x = U tanh(lambda (y - 1/4)) for y <= 1/2, U tanh(lambda (3/4 - y))
    above; u_y = delta sin(2 pi (x + 1/4)); rho = 1.
  * Random-phase low-mode flows (|k| <= kmax), divergence-free, rescaled to a
    given max |u|: 2D from a stream function, 3D as the curl of a vector
    potential; in 1D a random low-mode density and velocity profile.
  * Shock tube of the paper's first experiment: a density step at rest on
    the nodes 0..nodes, with zero-gradient ends realised by even reflection
    into a periodic row of 2 (nodes + 1) nodes, or with periodic ends.
"""
import math

import numpy as np

CS2 = 1.0 / 3.0  # lattice sound speed squared, used for pressure -> density


def _grid(n_axes):
    return np.meshgrid(*[np.arange(n, dtype=np.float64) for n in n_axes],
                       indexing="ij")


def taylor_green_2d(n, u0=0.05, rho0=1.0, pressure=True, ny=None):
    """2D TGV on an n x ny lattice.  Returns rho (1, ny, n), u (2, 1, ny, n)."""
    ny = n if ny is None else ny
    y, x = _grid((ny, n))
    kx, ky = 2 * math.pi / n, 2 * math.pi / ny
    ux = -u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = u0 * np.sin(kx * x) * np.cos(ky * y)
    if pressure:
        rho = rho0 - rho0 * u0 ** 2 / (4 * CS2) * (np.cos(2 * kx * x)
                                                   + np.cos(2 * ky * y))
    else:
        rho = np.full_like(x, rho0)
    return rho[None], np.stack([ux, uy])[:, None]


def taylor_green_3d(n, u0=0.05, rho0=1.0, pressure=True, ny=None, nz=None):
    """3D TGV on [0, 2 pi)^3 mapped to n x ny x nz nodes.
    Returns rho (nz, ny, n), u (3, nz, ny, n).  Built from 1D factors by
    broadcasting (the fields are products of functions of one axis)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    X = (2 * math.pi * np.arange(n, dtype=np.float64) / n)[None, None, :]
    Y = (2 * math.pi * np.arange(ny, dtype=np.float64) / ny)[None, :, None]
    Z = (2 * math.pi * np.arange(nz, dtype=np.float64) / nz)[:, None, None]
    u = np.empty((3, nz, ny, n))
    u[0] = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    u[2] = 0.0
    if pressure:
        p = rho0 * u0 ** 2 / 16 * (np.cos(2 * X) + np.cos(2 * Y)) * (
            np.cos(2 * Z) + 2)
        rho = rho0 + p / CS2
    else:
        rho = np.full((nz, ny, n), rho0)
    return np.ascontiguousarray(np.broadcast_to(rho, (nz, ny, n))), u


def shear_layer(n, U=0.04, lam=80.0, delta=2e-3, ny=None):
    """Doubly periodic double shear layer.  Returns rho (1, ny, n),
    u (2, 1, ny, n)."""
    ny = n if ny is None else ny
    j, i = _grid((ny, n))
    x, y = i / n, j / ny
    ux = np.where(y <= 0.5, U * np.tanh(lam * (y - 0.25)),
                  U * np.tanh(lam * (0.75 - y)))
    uy = delta * np.sin(2 * math.pi * (x + 0.25))
    return np.ones_like(x)[None], np.stack([ux, uy])[:, None]


def uniform_flow(shape, u, rho0=1.0):
    """Uniform state.  shape = (nz, ny, nx); u has d entries."""
    rho = np.full(shape, rho0)
    uu = np.stack([np.full(shape, float(c)) for c in u])
    return rho, uu


def shock_tube(nodes=800, rho_left=1.5, rho_right=0.75, split=400,
               ends="zero_gradient"):
    """Density step at rest on x = 0..nodes (rho_left for x <= split).

    ends="zero_gradient": the row is mirrored onto x = nodes + 1 .. 2 nodes + 1
    so that the periodic row of 2 (nodes + 1) nodes has zero-gradient ends
    at x = 0 and x = nodes.  ends="periodic": the nodes + 1 nodes wrap
    around, so a second step (rho_right | rho_left) sits at the wrap.
    Returns rho (1, 1, n), u (1, 1, 1, n)."""
    if ends == "periodic":
        n = nodes + 1
        rho = np.where(np.arange(n) <= split, rho_left, rho_right)
    elif ends == "zero_gradient":
        n = 2 * (nodes + 1)
        x = np.arange(n)
        rho = np.where((x <= split) | (x >= n - 1 - split), rho_left,
                       rho_right)
    else:
        raise ValueError("ends must be 'zero_gradient' or 'periodic'")
    return rho.astype(np.float64).reshape(1, 1, n), np.zeros((1, 1, 1, n))


def random_phase_1d(n, seed, kmax=4, umax=0.05, drho=0.05):
    """Random low-mode periodic row: rho = 1 + drho s(x) and u = umax v(x),
    s and v sums of modes 1..kmax with random phases, scaled to max |s| =
    max |v| = 1.  Returns rho (1, 1, n), u (1, 1, 1, n)."""
    rng = np.random.default_rng(seed)
    t = 2 * math.pi * np.arange(n) / n
    out = []
    for _ in range(2):
        a = rng.standard_normal(kmax)
        ph = rng.uniform(0, 2 * math.pi, kmax)
        v = sum(a[k] * np.cos((k + 1) * t + ph[k]) for k in range(kmax))
        out.append(v / np.abs(v).max())
    rho = 1.0 + drho * out[0]
    return rho.reshape(1, 1, n), (umax * out[1]).reshape(1, 1, 1, n)


def random_phase_2d(n, seed, kmax=4, umax=0.05, ny=None):
    """Divergence-free random low-mode 2D flow, max |u| = umax, rho = 1."""
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    y, x = _grid((ny, n))
    X, Y = 2 * math.pi * x / n, 2 * math.pi * y / ny
    ux = np.zeros_like(X)
    uy = np.zeros_like(X)
    for kx in range(-kmax, kmax + 1):
        for ky in range(0, kmax + 1):
            if kx * kx + ky * ky == 0 or kx * kx + ky * ky > kmax * kmax:
                continue
            if ky == 0 and kx < 0:
                continue
            a, ph = rng.standard_normal(), rng.uniform(0, 2 * math.pi)
            # stream function psi = a cos(kx X + ky Y + ph)
            s = np.sin(kx * X + ky * Y + ph)
            ux += -a * ky * s   # d psi / dy
            uy += a * kx * s    # -d psi / dx
    m = np.sqrt(ux ** 2 + uy ** 2).max()
    ux *= umax / m
    uy *= umax / m
    return np.ones_like(X)[None], np.stack([ux, uy])[:, None]


def random_phase_3d(n, seed, kmax=4, umax=0.05, ny=None, nz=None):
    """Divergence-free random low-mode 3D flow (curl of a random vector
    potential), max |u| = umax, rho = 1."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    z, y, x = _grid((nz, ny, n))
    X = 2 * math.pi * x / n
    Y = 2 * math.pi * y / ny
    Z = 2 * math.pi * z / nz
    u = np.zeros((3,) + X.shape)
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            for kz in range(0, kmax + 1):
                k2 = kx * kx + ky * ky + kz * kz
                if k2 == 0 or k2 > kmax * kmax:
                    continue
                a = rng.standard_normal(3)
                ph = rng.uniform(0, 2 * math.pi)
                s = np.sin(kx * X + ky * Y + kz * Z + ph)
                k = np.array([kx, ky, kz], dtype=np.float64)
                # A = a cos(k.x + ph)  =>  curl A = -(k x a) sin(k.x + ph)
                kxa = np.cross(k, a)
                for d in range(3):
                    u[d] += -kxa[d] * s
    m = np.sqrt((u ** 2).sum(0)).max()
    u *= umax / m
    return np.ones_like(X), u


def batch_specs(seed=20190401, count=64):
    """Mixed lattice set of the batched workload: half D2Q9 with edge
    n ~ U{64..1024}, half D3Q27 with n ~ U{32..192}, nu log-uniform in
    [1e-5, 1e-2], random-phase low-mode flow with max |u| = 0.05."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(count):
        lat = "D2Q9" if k % 2 == 0 else "D3Q27"
        n = int(rng.integers(64, 1025)) if lat == "D2Q9" else int(
            rng.integers(32, 193))
        nu = float(10 ** rng.uniform(-5, -2))
        specs.append({"lattice": lat, "n": n, "nu": nu,
                      "seed": int(rng.integers(0, 2 ** 31))})
    return specs


def request_stream(seed=20190402, count=2000, rate=50.0, min_steps=100,
                   max_steps=10000):
    """Poisson stream of requests: exponential gaps (mean 1/rate s), lattice
    type, size and nu as in batch_specs, steps log-uniform integers."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        lat = "D2Q9" if rng.uniform() < 0.5 else "D3Q27"
        n = int(rng.integers(64, 1025)) if lat == "D2Q9" else int(
            rng.integers(32, 193))
        nu = float(10 ** rng.uniform(-5, -2))
        steps = int(round(10 ** rng.uniform(math.log10(min_steps),
                                            math.log10(max_steps))))
        reqs.append({"id": k, "arrival": t, "lattice": lat, "n": n, "nu": nu,
                     "steps": steps, "seed": int(rng.integers(0, 2 ** 31))})
    return reqs


def abc_flow_3d(n, seed, umax=0.05, kmax=4):
    """Random-phase low-mode 3D flow built from separable terms (an
    Arnold-Beltrami-Childress flow with random amplitudes, phases and mode
    numbers 1..kmax per term): divergence-free, max |u| rescaled to umax,
    rho = 1.  Fast for large lattices (only 1D trigonometric factors)."""
    rng = np.random.default_rng(seed)
    A, B, C = rng.uniform(0.5, 1.5, size=3)
    ka, kb, kc = rng.integers(1, kmax + 1, size=3)
    pa, pb, pc = rng.uniform(0, 2 * math.pi, size=3)
    t = 2 * math.pi * np.arange(n, dtype=np.float64) / n
    X, Y, Z = t[None, None, :], t[None, :, None], t[:, None, None]
    u = np.empty((3, n, n, n))
    # u = A sin(k z) + C cos(k y), v = B sin(k x) + A cos(k z),
    # w = C sin(k y) + B cos(k x): each term depends on the other two axes
    u[0] = A * np.sin(ka * Z + pa) + C * np.cos(kc * Y + pc)
    u[1] = B * np.sin(kb * X + pb) + A * np.cos(ka * Z + pa)
    u[2] = C * np.sin(kc * Y + pc) + B * np.cos(kb * X + pb)
    m = np.sqrt((u ** 2).sum(0)).max()
    u *= umax / m
    return np.ones((n, n, n)), u


def shear_waves_2d(n, seed, umax=0.05, kmax=4):
    """Random-phase low-mode 2D flow from separable shear waves,
    u_x = a sin(k1 y + p1) + c cos(k3 y + p3), u_y = b sin(k2 x + p2)
    (divergence-free), max |u| rescaled to umax, rho = 1."""
    rng = np.random.default_rng(seed)
    a, b, c = rng.uniform(0.5, 1.5, size=3)
    k1, k2, k3 = rng.integers(1, kmax + 1, size=3)
    p1, p2, p3 = rng.uniform(0, 2 * math.pi, size=3)
    t = 2 * math.pi * np.arange(n, dtype=np.float64) / n
    X, Y = t[None, :], t[:, None]
    u = np.empty((2, 1, n, n))
    u[0, 0] = a * np.sin(k1 * Y + p1) + c * np.cos(k3 * Y + p3) + 0.0 * X
    u[1, 0] = b * np.sin(k2 * X + p2) + 0.0 * Y
    m = np.sqrt((u ** 2).sum(0)).max()
    u *= umax / m
    return np.ones((1, n, n)), u


def fields_for(lattice, n, seed, umax=0.05):
    """Initial fields for one batched / served lattice: random-phase
    low-mode divergence-free flow, max |u| = umax, rho = 1."""
    if lattice == "D2Q9":
        return shear_waves_2d(n, seed, umax=umax)
    return abc_flow_3d(n, seed, umax=umax)


def random_multipliers(rng, q, amp):
    """q positive multipliers 1 + amp * U(-1, 1) (amp < 1), for perturbing a
    population vector away from equilibrium in pin tests."""
    return 1.0 + amp * rng.uniform(-1.0, 1.0, size=q)
