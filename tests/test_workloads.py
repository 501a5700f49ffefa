"""The seeded synthetic inputs (elbm_workloads) have the properties the
benchmark and the tests rely on: divergence-free low-mode flows with the
stated maximum speed, the Taylor-Green and shear-layer definitions, the
batched mix and the Poisson request stream with their stated ranges, and
determinism in the seed."""
import math

import numpy as np

import elbm_workloads as W


def _div_spectral(u):
    """Spectral divergence of a periodic field u[d][...] (axes z, y, x)."""
    d = u.shape[0]
    shape = u.shape[1:]
    div = np.zeros(shape, dtype=complex)
    for a in range(d):
        axis = len(shape) - 1 - a            # component a varies along axis
        k = np.fft.fftfreq(shape[axis]) * shape[axis]
        kshape = [1] * len(shape)
        kshape[axis] = -1
        div += 1j * k.reshape(kshape) * np.fft.fftn(u[a])
    return np.abs(np.fft.ifftn(div)).max()


def test_random_phase_flows_are_divergence_free_with_max_speed():
    rho, u = W.random_phase_2d(48, seed=3, umax=0.07)
    assert rho.shape == (1, 48, 48) and np.all(rho == 1.0)
    uu = u[:, 0]
    assert abs(np.sqrt((uu ** 2).sum(0)).max() - 0.07) < 1e-15
    assert _div_spectral(uu) < 1e-13
    rho, u = W.random_phase_3d(24, seed=4, umax=0.05, ny=20, nz=16)
    assert rho.shape == (16, 20, 24) and u.shape == (3, 16, 20, 24)
    assert abs(np.sqrt((u ** 2).sum(0)).max() - 0.05) < 1e-15
    assert _div_spectral(u) < 1e-13
    rho, u = W.abc_flow_3d(20, seed=5)
    assert _div_spectral(u) < 1e-13


def test_random_phase_flows_are_deterministic_in_the_seed():
    a = W.random_phase_3d(16, seed=9)[1]
    b = W.random_phase_3d(16, seed=9)[1]
    c = W.random_phase_3d(16, seed=10)[1]
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_taylor_green_fields():
    n, u0 = 32, 0.05
    rho, u = W.taylor_green_3d(n, u0)
    t = 2 * math.pi * np.arange(n) / n
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    assert np.allclose(u[0], u0 * np.sin(x) * np.cos(y) * np.cos(z),
                       atol=1e-16)
    assert np.allclose(u[1], -u0 * np.cos(x) * np.sin(y) * np.cos(z),
                       atol=1e-16)
    assert np.all(u[2] == 0.0)
    p = u0 ** 2 / 16 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2)
    assert np.allclose(rho, 1.0 + 3.0 * p, atol=1e-16)
    assert _div_spectral(u) < 1e-15


def test_shear_layer_fields():
    n = 64
    rho, u = W.shear_layer(n)
    j = np.arange(n) / n
    assert np.all(rho == 1.0)
    ux = u[0, 0]
    assert np.allclose(ux[:, 0], np.where(j <= 0.5,
                                          0.04 * np.tanh(80 * (j - 0.25)),
                                          0.04 * np.tanh(80 * (0.75 - j))))
    i = np.arange(n) / n
    assert np.allclose(u[1, 0][0], 2e-3 * np.sin(2 * math.pi * (i + 0.25)))


def test_batch_specs_ranges():
    specs = W.batch_specs()
    assert len(specs) == 64
    assert sum(s["lattice"] == "D2Q9" for s in specs) == 32
    for s in specs:
        lo, hi = (64, 1024) if s["lattice"] == "D2Q9" else (32, 192)
        assert lo <= s["n"] <= hi
        assert 1e-5 <= s["nu"] <= 1e-2
    assert specs == W.batch_specs()


def test_request_stream_is_poisson_at_the_stated_rate():
    reqs = W.request_stream()
    assert len(reqs) == 2000
    t = np.array([r["arrival"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps >= 0)
    # mean gap 1/50 s within 4 standard errors of the exponential mean
    assert abs(gaps.mean() - 0.02) < 4 * 0.02 / math.sqrt(len(gaps))
    # exponential: standard deviation equals the mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    steps = np.array([r["steps"] for r in reqs])
    assert steps.min() >= 100 and steps.max() <= 10000
    assert 0.4 < np.mean([r["lattice"] == "D2Q9" for r in reqs]) < 0.6


def test_shock_tube_is_an_even_reflection_of_the_step():
    rho, u = W.shock_tube(800, 1.5, 0.75, 400)
    n = rho.size
    assert n == 1602 and rho.shape == (1, 1, n) and u.shape == (1, 1, 1, n)
    r = rho.ravel()
    assert np.all(r[:401] == 1.5) and np.all(r[401:801] == 0.75)
    # mirror image about the midpoint between x = 800 and x = 801: the
    # periodic row has zero-gradient ends at x = 0 and x = 800
    assert np.array_equal(r[801:], r[800::-1])
    assert np.all(u == 0.0)
    rho, u = W.shock_tube(800, 1.5, 0.75, 400, ends="periodic")
    r = rho.ravel()
    assert r.size == 801 and np.all(r[:401] == 1.5) and np.all(r[401:] == 0.75)


def test_random_phase_1d_ranges_and_seed():
    rho, u = W.random_phase_1d(97, seed=2, umax=0.1, drho=0.05)
    assert rho.shape == (1, 1, 97) and u.shape == (1, 1, 1, 97)
    assert abs(np.abs(rho - 1).max() - 0.05) < 1e-15
    assert abs(np.abs(u).max() - 0.1) < 1e-15
    assert np.array_equal(u, W.random_phase_1d(97, seed=2, umax=0.1)[1])
