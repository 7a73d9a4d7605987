"""Pins of the oracle's Laplacian L u = (1/h^2) sum_a sum_j c_|j| u(p + j e_a).

Fixed against: the closed-form symbol on periodic plane waves, symmetry of the
operator, exact differentiation of 3D polynomials of degree <= k+1 away from
the boundary, and the dense Kronecker-product operator built from exactly
solved weights (non-cubic grids, so a swapped axis fails).
"""
import numpy as np
import pytest

from pinlib import dense_laplacian, symbol, vandermonde_weights


@pytest.mark.parametrize("k", [2, 4, 6, 8, 12, 16])
def test_plane_wave_symbol(oracle_mod, k):
    """On a periodic grid, cos(kappa.x + phi) is an eigenfunction with
    eigenvalue -(1/h^2) sum_a sigma(kappa_a h)."""
    shape = (18, 20, 22)
    h = 7.5
    w = vandermonde_weights(k)
    modes = (3, 5, 7)
    g = np.indices(shape).astype(np.float64)
    theta = [2 * np.pi * modes[a] / shape[a] for a in range(3)]
    phase = sum(theta[a] * g[a] for a in range(3)) + 0.37
    u = np.cos(phase)
    lam = -sum(symbol(w, theta[a]) for a in range(3)) / h ** 2
    got = oracle_mod.laplacian(u, k, h, periodic=True)
    np.testing.assert_allclose(got, lam * u, rtol=0, atol=1e-12 * abs(lam))


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("k", [2, 8, 16])
def test_symmetry(oracle_mod, k, periodic):
    rng = np.random.default_rng(11)
    shape = (9, 11, 13)
    v = rng.standard_normal(shape)
    w = rng.standard_normal(shape)
    lv = oracle_mod.laplacian(v, k, 2.0, periodic)
    lw = oracle_mod.laplacian(w, k, 2.0, periodic)
    a, b = np.vdot(v, lw), np.vdot(lv, w)
    assert a == pytest.approx(b, rel=1e-12)


@pytest.mark.parametrize("k", [2, 4, 8])
def test_polynomial_exactness_3d(oracle_mod, k):
    """A random polynomial of total degree k+1 with mixed terms (x^2 y z^3 ...)
    is differentiated exactly at points at least r from the boundary."""
    rng = np.random.default_rng(k)
    r = k // 2
    shape = (2 * r + 5, 2 * r + 6, 2 * r + 7)
    h = 0.25
    deg = k + 1
    exps = [(a, b, c) for a in range(deg + 1) for b in range(deg + 1) for c in range(deg + 1)
            if a + b + c <= deg]
    coef = rng.standard_normal(len(exps))
    g = np.indices(shape).astype(np.float64) * h - 1.0
    x, y, z = g
    u = sum(cf * x ** a * y ** b * z ** c for cf, (a, b, c) in zip(coef, exps))
    lap = np.zeros(shape)
    for cf, (a, b, c) in zip(coef, exps):
        if a >= 2:
            lap += cf * a * (a - 1) * x ** (a - 2) * y ** b * z ** c
        if b >= 2:
            lap += cf * b * (b - 1) * x ** a * y ** (b - 2) * z ** c
        if c >= 2:
            lap += cf * c * (c - 1) * x ** a * y ** b * z ** (c - 2)
    got = oracle_mod.laplacian(u, k, h)
    sl = tuple(slice(r, n - r) for n in shape)
    scale = np.max(np.abs(u)) / h ** 2
    np.testing.assert_allclose(got[sl], lap[sl], rtol=0, atol=1e-10 * scale)


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("k,shape", [(2, (5, 6, 7)), (4, (7, 6, 5)), (8, (6, 8, 7)),
                                     (16, (5, 7, 6))])
def test_matches_dense_kronecker_operator(oracle_mod, k, shape, periodic):
    """Brute force: the operator assembled as Kronecker products of 1D stencil
    matrices (including stencils wider than the grid)."""
    rng = np.random.default_rng(5)
    u = rng.standard_normal(shape)
    h = 3.0
    dense = dense_laplacian(shape, vandermonde_weights(k), h, periodic)
    want = (dense @ u.reshape(-1)).reshape(shape)
    got = oracle_mod.laplacian(u, k, h, periodic)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.max(np.abs(want)))
