"""Pins of the oracle's enstrophy against closed forms.

The enstrophy of a velocity field is 1/2 <|omega|^2>, omega = curl u, here by
second-order central differences on the periodic lattice (the definition the
Taylor-Green history comparisons use).  For a velocity field built from
single Fourier modes the central difference of sin(k x) is exactly
cos(k x) sin(k), so the discrete enstrophy has a closed form.  The oracle is
fed f = f^eq(rho, u) (its own equilibrium, whose moments return u to
rounding) and must reproduce these values to rounding.

The flows are chosen so that a plausible mistake fails a test: a wrong sign
in any of the six curl terms, a missing factor 1/2 of the central
difference or of the enstrophy, a one-sided difference, or a mean over the
wrong count.  Non-square lattices keep the axes apart.
"""
import math

import numpy as np
import pytest

import oracle

TOL = 1e-12


def _lattice_at(lat, u, rho=None):
    d, nz, ny, nx = u.shape
    o = oracle.Lattice(lat, nx, ny, nz, nu=1e-3)
    if rho is None:
        rho = np.ones((nz, ny, nx))
    o.init_fields(rho, u)
    return o


def _axes(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


@pytest.mark.parametrize("nx,ny", [(64, 64), (24, 40), (7, 5)])
def test_taylor_green_2d_enstrophy_closed_form(nx, ny):
    # u = -u0 cos(kx x) sin(ky y), v = u0 sin(kx x) cos(ky y):
    # omega = u0 (sin kx + sin ky) cos(kx x) cos(ky y) with central
    # differences, so 1/2 <omega^2> = u0^2 (sin kx + sin ky)^2 / 8.
    u0 = 0.05
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    x, y, _ = _axes(nx, ny, 1)
    u = np.stack([-u0 * np.cos(kx * x) * np.sin(ky * y),
                  u0 * np.sin(kx * x) * np.cos(ky * y)])
    # a nonuniform density (the pressure-consistent one) leaves u unchanged
    rho = 1.0 - 0.25 * 3 * u0 ** 2 * (np.cos(2 * kx * x) + np.cos(2 * ky * y))
    o = _lattice_at("D2Q9", u, rho)
    want = u0 ** 2 * (math.sin(kx) + math.sin(ky)) ** 2 / 8
    got = o.enstrophy()
    assert abs(got - want) <= TOL * want, (got, want)
    if nx == ny:   # the square case reduces to u0^2 sin^2(2 pi / n) / 2
        assert abs(got - u0 ** 2 * math.sin(kx) ** 2 / 2) <= TOL * want


@pytest.mark.parametrize("nx,ny,nz", [(16, 16, 16), (12, 10, 8)])
def test_taylor_green_3d_enstrophy_closed_form(nx, ny, nz):
    # u = u0 sin X cos Y cos Z, v = -u0 cos X sin Y cos Z, w = 0:
    # omega_x = -u0 sz cX sY sZ, omega_y = -u0 sz sX cY sZ,
    # omega_z = u0 (sx + sy) sX sY cZ  (s_a = sin k_a, central differences),
    # so 1/2 <|omega|^2> = u0^2 (2 sz^2 + (sx + sy)^2) / 16.
    u0 = 0.05
    k = [2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz]
    x, y, z = _axes(nx, ny, nz)
    X, Y, Z = k[0] * x, k[1] * y, k[2] * z
    u = np.stack([u0 * np.sin(X) * np.cos(Y) * np.cos(Z),
                  -u0 * np.cos(X) * np.sin(Y) * np.cos(Z),
                  np.zeros_like(X)])
    o = _lattice_at("D3Q27", u)
    sx, sy, sz = (math.sin(v) for v in k)
    want = u0 ** 2 * (2 * sz ** 2 + (sx + sy) ** 2) / 16
    got = o.enstrophy()
    assert abs(got - want) <= TOL * want, (got, want)
    if nx == ny == nz:
        assert abs(got - 3 * u0 ** 2 * sx ** 2 / 8) <= TOL * want


# One tilted shear wave per vorticity component: both velocity components
# that enter omega_a vary with the same phase theta, so the two terms of
# omega_a interfere and a sign error in either changes the value.
#   omega_x = dw/dy - dv/dz,  omega_y = du/dz - dw/dx,  omega_z = dv/dx - du/dy
# With (p, q) the two velocity components along theta = k_b b + k_c c and
# amplitudes (A, B), omega_a = cos(theta) * (difference of A s and B s), and
# 1/2 <omega_a^2> = (that difference)^2 / 4.
CASES = {
    # component: (velocity axes carrying A and B, the phase's axes, closed
    # form of omega_a / cos(theta) from (A, B, s))
    "x": ((1, 2), (1, 2), lambda A, B, s: B * s[1] - A * s[2]),
    "y": ((0, 2), (0, 2), lambda A, B, s: A * s[2] - B * s[0]),
    "z": ((0, 1), (0, 1), lambda A, B, s: B * s[0] - A * s[1]),
}


@pytest.mark.parametrize("comp", ["x", "y", "z"])
@pytest.mark.parametrize("A,B", [(0.03, 0.02), (-0.04, 0.01)])
def test_curl_component_signs(comp, A, B):
    nx, ny, nz = 12, 10, 8
    (va, vb), (pa, pb), form = CASES[comp]
    k = [2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz]
    coords = _axes(nx, ny, nz)
    theta = k[pa] * coords[pa] + k[pb] * coords[pb]
    u = np.zeros((3, nz, ny, nx))
    u[va] = A * np.sin(theta)
    u[vb] = B * np.sin(theta)
    o = _lattice_at("D3Q27", u)
    s = [math.sin(v) for v in k]
    want = form(A, B, s) ** 2 / 4
    got = o.enstrophy()
    assert abs(got - want) <= TOL * max(want, 1e-30), (got, want)
    # the same wave with one sign of the pair flipped gives the other
    # combination, so the two terms really interfere
    flipped = form(A, -B, s) ** 2 / 4
    assert abs(flipped - want) > 1e-3 * want


def test_uniform_flow_has_zero_enstrophy():
    u = np.zeros((3, 6, 5, 7))
    u[0], u[1], u[2] = 0.03, -0.02, 0.01
    assert _lattice_at("D3Q27", u).enstrophy() == 0.0
