"""Pins of the oracle's damped leapfrog step, sources and initial conditions.

Fixed against: the damped Eq. 1 discretised at space order 2 on a unit grid
(sign of the damping and the r0 denominator as in Listing 2),
a dense-matrix brute force with sources, the exact discrete plane-wave
solution, the closed form of the one-node domain (a damped scalar recurrence),
discrete energy conservation (and decay with damping), reciprocity, linearity
and the zero initial conditions of Eq. 1.
"""
import os

import numpy as np
import pytest

from pinlib import dense_forward, symbol, vandermonde_weights


def _eq1_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "eq1_k2_damped.txt")
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                term, level, dx, dy, dz, sign, scale, factor, p = line.split()
                rows.append((term, int(level), (int(dx), int(dy), int(dz)), int(sign) * float(scale),
                             factor, int(p)))
    return rows


def _eq1_update(u, u_prev, m, damp, dt):
    """Solve the fixture's discrete residual of Eq. 1 (damped, k = 2, h = 1)
    for u^{n+1} at the points whose neighbours all lie inside the arrays:
    residual = A u^{n+1} + B = 0 with A the u^{n+1} coefficient and B every
    other term applied to u^n and u^{n-1}. Also returns A dt^3, which must be
    Listing 2's r0 = dt m + dt^2 damp / 2."""
    nx, ny, nz = u.shape
    core = (slice(1, nx - 1), slice(1, ny - 1), slice(1, nz - 1))
    fields = {0: u, -1: u_prev}
    factors = {"1": np.ones_like(m[core]), "m": m[core], "eta": damp[core]}
    a = np.zeros_like(m[core])
    b = np.zeros_like(m[core])
    for term, level, (dx, dy, dz), coef, factor, p in _eq1_rows():
        c = coef * factors[factor] * dt ** p
        if level == 1:
            assert (dx, dy, dz) == (0, 0, 0)
            a += c
            continue
        sh = (slice(1 + dx, nx - 1 + dx), slice(1 + dy, ny - 1 + dy), slice(1 + dz, nz - 1 + dz))
        b += c * fields[level][sh]
    return -b / a, a * dt ** 3, core


def test_step_solves_damped_eq1_k2(oracle_mod):
    """The oracle's step equals u^{n+1} solved from the damped Eq. 1 residual
    (space order 2, unit grid) written out in the golden fixture, and the
    u^{n+1} coefficient times dt^3 is Listing 2's denominator r0."""
    rng = np.random.default_rng(0)
    shape = (7, 8, 9)
    u = rng.standard_normal(shape)
    u_prev = rng.standard_normal(shape)
    m = rng.uniform(0.2, 1.5, shape)
    damp = rng.uniform(0.0, 0.8, shape)
    dt = 0.37
    want, r0, core = _eq1_update(u, u_prev, m, damp, dt)
    np.testing.assert_allclose(r0, dt * m[core] + 0.5 * dt ** 2 * damp[core], rtol=1e-15)
    got = oracle_mod.step(u, u_prev, m, damp, 2, 1.0, dt)
    np.testing.assert_allclose(got[core], want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k,shape", [(2, (5, 6, 7)), (4, (6, 7, 5)), (8, (7, 5, 6)),
                                     (16, (5, 6, 5))])
def test_forward_matches_dense_brute_force(oracle_mod, k, shape):
    rng = np.random.default_rng(k)
    m = rng.uniform(0.5, 2.0, shape)
    eta = rng.uniform(0.0, 0.3, shape)
    h, dt, nt = 1.3, 0.05, 12
    sources = [(1, 2, 3), (shape[0] - 1, 0, shape[2] - 2)]
    wav = rng.standard_normal((2, nt - 2))  # shorter than nt: zero afterwards
    want_u, want_up = dense_forward(m, eta, vandermonde_weights(k), h, dt, nt, sources, wav)
    got_u, got_up = oracle_mod.forward(m, eta, k, h, dt, nt, sources, wav)
    scale = np.max(np.abs(want_u))
    np.testing.assert_allclose(got_u, want_u, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(got_up, want_up, rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("k", [2, 4, 8])
def test_exact_discrete_plane_wave(oracle_mod, k):
    """With eta = 0, q = 0, periodic boundaries and constant m, the scheme's
    exact solution is u^n = cos(kappa.x - omega n dt) with
    sin^2(omega dt / 2) = v^2 dt^2 / (4 h^2) sum_a sigma(kappa_a h)."""
    shape = (16, 16, 16)
    h, v = 10.0, 1500.0
    dt = 0.9 * oracle_mod.dt_max(k, h, v)
    modes = (1, 2, 3)
    theta = [2 * np.pi * modes[a] / shape[a] for a in range(3)]
    s = sum(symbol(vandermonde_weights(k), t) for t in theta)
    omega = 2.0 / dt * np.arcsin(np.sqrt(v * v * dt * dt / (4 * h * h) * s))
    g = np.indices(shape).astype(np.float64)
    phase = sum(theta[a] * g[a] for a in range(3))
    m = np.full(shape, 1.0 / v ** 2)
    nt = 1000
    u, up = oracle_mod.forward(m, None, k, h, dt, nt, u0=np.cos(phase),
                               u_prev0=np.cos(phase + omega * dt), periodic=True)
    np.testing.assert_allclose(u, np.cos(phase - omega * nt * dt), rtol=0, atol=1e-11)
    np.testing.assert_allclose(up, np.cos(phase - omega * (nt - 1) * dt), rtol=0, atol=1e-11)


@pytest.mark.parametrize("k", [2, 8, 16])
def test_energy_conserved_without_damping(oracle_mod, k):
    rng = np.random.default_rng(7)
    shape = (14, 12, 10)
    h = 10.0
    m = 1.0 / rng.uniform(1500, 4500, shape) ** 2
    dt = 0.9 * oracle_mod.dt_max(k, h, 4500.0)
    u0 = rng.standard_normal(shape)
    u1 = u0 + 0.01 * rng.standard_normal(shape)
    e0 = oracle_mod.energy(u1, u0, m, k, h, dt, periodic=True)
    assert e0 > 0
    u, up = u1, u0
    for _ in range(5):
        u, up = oracle_mod.forward(m, None, k, h, dt, 40, u0=u, u_prev0=up, periodic=True)
        e = oracle_mod.energy(u, up, m, k, h, dt, periodic=True)
        assert e == pytest.approx(e0, rel=1e-12)


def test_energy_decays_with_damping(oracle_mod):
    rng = np.random.default_rng(8)
    shape = (12, 12, 12)
    k, h = 4, 10.0
    m = np.full(shape, 1.0 / 2000.0 ** 2)
    eta = m * rng.uniform(0, 20.0, shape)
    dt = 0.9 * oracle_mod.dt_max(k, h, 2000.0)
    u0 = rng.standard_normal(shape)
    u, up = u0, u0.copy()
    first = last = oracle_mod.energy(u, up, m, k, h, dt)
    assert first > 0
    for _ in range(20):
        u, up = oracle_mod.forward(m, eta, k, h, dt, 5, u0=u, u_prev0=up)
        e = oracle_mod.energy(u, up, m, k, h, dt)
        assert e <= last * (1 + 1e-13)
        last = e
    assert last < 0.9 * first


def test_reciprocity(oracle_mod):
    """Trace at B from a source at A equals trace at A from a source at B
    (L symmetric, m and eta diagonal), for any m and eta."""
    rng = np.random.default_rng(9)
    shape = (10, 11, 12)
    k, h = 8, 10.0
    m = 1.0 / rng.uniform(1500, 4500, shape) ** 2
    eta = m * rng.uniform(0, 30.0, shape)
    dt = 0.8 * oracle_mod.dt_max(k, h, 4500.0)
    a, b = (2, 3, 4), (7, 8, 6)
    wav = rng.standard_normal((1, 60))
    tr_ab, tr_ba = [], []
    ua = upa = ub = upb = None
    for n in range(1, 61):
        ua, upa = oracle_mod.forward(m, eta, k, h, dt, 1, [a], wav, u0=ua, u_prev0=upa,
                                     step0=n - 1)
        ub, upb = oracle_mod.forward(m, eta, k, h, dt, 1, [b], wav, u0=ub, u_prev0=upb,
                                     step0=n - 1)
        tr_ab.append(ua[b])
        tr_ba.append(ub[a])
    tr_ab, tr_ba = np.array(tr_ab), np.array(tr_ba)
    assert np.max(np.abs(tr_ab)) > 0
    np.testing.assert_allclose(tr_ab, tr_ba, rtol=0, atol=1e-12 * np.max(np.abs(tr_ab)))


def test_linearity_and_zero_initial_state(oracle_mod):
    rng = np.random.default_rng(10)
    shape = (9, 9, 9)
    m = np.full(shape, 0.5)
    eta = rng.uniform(0, 0.2, shape)
    wav = rng.standard_normal((1, 20))
    u1, _ = oracle_mod.forward(m, eta, 4, 1.0, 0.1, 20, [(4, 4, 4)], wav)
    u3, _ = oracle_mod.forward(m, eta, 4, 1.0, 0.1, 20, [(4, 4, 4)], 3.0 * wav)
    np.testing.assert_allclose(u3, 3.0 * u1, rtol=1e-13, atol=1e-300)
    z, zp = oracle_mod.forward(m, eta, 4, 1.0, 0.1, 20)
    assert not z.any() and not zp.any()


def test_forward_chunks_compose(oracle_mod):
    """forward(a) then forward(b) from step a equals forward(a+b)."""
    rng = np.random.default_rng(12)
    shape = (8, 9, 10)
    m = rng.uniform(0.5, 1.0, shape)
    wav = rng.standard_normal((1, 30))
    src = [(3, 4, 5)]
    u, up = oracle_mod.forward(m, None, 4, 1.0, 0.1, 30, src, wav)
    ua, upa = oracle_mod.forward(m, None, 4, 1.0, 0.1, 13, src, wav)
    ub, upb = oracle_mod.forward(m, None, 4, 1.0, 0.1, 17, src, wav, u0=ua, u_prev0=upa,
                                 step0=13)
    np.testing.assert_array_equal(u, ub)
    np.testing.assert_array_equal(up, upb)


def test_default_damping_invariants(oracle_mod):
    """The default profile (a convention): zero in the interior, zero with no
    layer, non-negative, mirror-symmetric for a symmetric model, largest at the
    corners where it equals m * 3 d_max with d_max = 3 v ln(1e3) / (2 nbl h)."""
    nbl, h = 5, 10.0
    shape = (20, 22, 24)
    m = np.full(shape, 1.0 / 3000.0 ** 2)
    eta = oracle_mod.default_damping(m, nbl, h)
    assert (eta >= 0).all()
    interior = eta[nbl:-nbl, nbl:-nbl, nbl:-nbl]
    assert not interior.any()
    assert eta[nbl - 1, nbl, nbl] > 0
    np.testing.assert_array_equal(eta, eta[::-1, :, :])
    np.testing.assert_array_equal(eta, eta[:, ::-1, :])
    np.testing.assert_array_equal(eta, eta[:, :, ::-1])
    dmax = 3 * 3000.0 * np.log(1e3) / (2 * nbl * h)
    assert eta.max() == pytest.approx(eta[0, 0, 0])
    assert eta[0, 0, 0] == pytest.approx(m[0, 0, 0] * 3 * dmax, rel=1e-14)
    assert not oracle_mod.default_damping(m, 0, h).any()


@pytest.mark.parametrize("k", [2, 4, 8, 16, 24])
@pytest.mark.parametrize("damped", [False, True])
def test_one_node_domain_is_a_scalar_recurrence(oracle_mod, k, damped):
    """On a one-node domain every tap but the centre falls in the zero halo, so
    the damped Eq. 1 at that node is the scalar recurrence
    (m/dt^2 + eta/(2 dt)) u^{n+1} = (2 m/dt^2 + 3 c_0/h^2) u^n - (m/dt^2 - eta/(2 dt)) u^{n-1}.
    Its characteristic roots are rho e^{+-i theta}, so u^n = rho^n (A cos n theta
    + B sin n theta) with A, B fixed by u^0 and u^{-1}: a closed form of the
    scheme's degenerate case (centre weight from exact rational arithmetic)."""
    h, v = 10.0, 2000.0
    m = 1.0 / v ** 2
    dt = 0.8 * oracle_mod.dt_max(k, h, v)
    eta = 0.01 * m / dt if damped else 0.0  # eta dt / (2 m) = 0.005: about 0.5 % decay per step
    c0 = float(vandermonde_weights(k)[0])
    a = m / dt ** 2 + eta / (2 * dt)
    b = 2 * m / dt ** 2 + 3 * c0 / h ** 2
    c = m / dt ** 2 - eta / (2 * dt)
    rho = np.sqrt(c / a)
    theta = np.arccos(b / (2 * a * rho))
    u0, um1 = 0.7, -0.4
    A = u0
    B = (A * np.cos(theta) - rho * um1) / np.sin(theta)
    nt = 400

    def closed(n):
        return rho ** n * (A * np.cos(n * theta) + B * np.sin(n * theta))

    one = (1, 1, 1)
    got, got_prev = oracle_mod.forward(np.full(one, m), np.full(one, eta), k, h, dt, nt,
                                       u0=np.full(one, u0), u_prev0=np.full(one, um1))
    assert abs(got[0, 0, 0] - closed(nt)) <= 1e-11
    assert abs(got_prev[0, 0, 0] - closed(nt - 1)) <= 1e-11
    if damped:  # the envelope decays as rho^n
        assert rho < 1.0 and abs(closed(nt)) <= rho ** nt * np.hypot(A, B) * (1 + 1e-12)
