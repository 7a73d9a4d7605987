"""Pins of the oracle's finite-difference weights and stability limit.

The oracle computes c_j in closed form; these tests fix it against an exact
rational Vandermonde solve, exactness on polynomials, the weights printed in
Listing 2 (space order 2), and dt_max against the operator's spectrum.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from pinlib import dense_laplacian, vandermonde_weights

ORDERS = list(range(2, 25, 2))


@pytest.mark.parametrize("k", ORDERS)
def test_weights_match_exact_vandermonde(oracle_mod, k):
    exact = vandermonde_weights(k)
    got = oracle_mod.fd_weights(k)
    assert len(got) == k // 2 + 1
    for j, e in enumerate(exact):
        assert got[j] == pytest.approx(float(e), rel=2e-15, abs=0.0), (k, j)


@pytest.mark.parametrize("k", ORDERS)
def test_weights_exact_on_polynomials(oracle_mod, k):
    """The stencil differentiates x^p exactly for p <= k+1, and not for p = k+2.

    Evaluated in exact rational arithmetic on the oracle's (binary) weights, so
    the only error left is the rounding of the weights themselves.
    """
    c = [Fraction(float(v)) for v in oracle_mod.fd_weights(k)]
    exact_c = vandermonde_weights(k)
    r = k // 2
    h = Fraction(1, 8)
    x0 = Fraction(1, 4)
    for p in range(0, k + 3):
        approx = sum(c[abs(j)] * (x0 + j * h) ** p for j in range(-r, r + 1)) / (h * h)
        exact = p * (p - 1) * x0 ** (p - 2) if p >= 2 else Fraction(0)
        scale = sum(abs(cj) * abs(x0 + j * h) ** p for j, cj in
                    ((j, c[abs(j)]) for j in range(-r, r + 1))) / (h * h)
        err = abs(approx - exact)
        if p <= k + 1:
            assert err <= Fraction(1, 10 ** 13) * scale, (k, p, float(err))
        else:
            # leading truncation term h^k * sum_j c_j j^(k+2), from the exact weights
            lead = h ** k * sum(exact_c[abs(j)] * Fraction(j) ** p for j in range(-r, r + 1))
            assert lead != 0
            assert err >= abs(lead) / 2, (k, float(err), float(lead))


def _read_eq1_lap_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "eq1_k2_damped.txt")
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line and line.split()[0] == "lap":
                _, _, dx, dy, dz, sign, scale, _, _ = line.split()
                rows.append(((int(dx), int(dy), int(dz)), int(sign) * float(scale)))
    return rows


def test_weights_k2_match_three_point_laplacian(oracle_mod):
    """Space order 2 (h = 1): the residual's -lap(u) rows give each of the six
    neighbours -1 and the centre +6, i.e. c_1 = 1 and 3*c_0 = -6 (the same 1 and
    -6 that Listing 2, Sec. 2.1, multiplies by dt^3)."""
    rows = _read_eq1_lap_rows()
    nb = [c for off, c in rows if off != (0, 0, 0)]
    centre = [c for off, c in rows if off == (0, 0, 0)]
    assert len(nb) == 6 and len(centre) == 1
    c = oracle_mod.fd_weights(2)
    for v in nb:
        assert -v == c[1]
    assert -centre[0] == 3 * c[0]


@pytest.mark.parametrize("k", [2, 4, 8, 12, 16])
def test_dt_max_is_nyquist_limit(oracle_mod, k):
    """-L's largest eigenvalue on an even periodic grid is 3 sum|c_j| / h^2,
    attained by the Nyquist mode; dt_max = 2 / (v sqrt(lambda_max))."""
    h = 10.0
    v = 4500.0
    n = 2 * (k // 2) + 2  # even, wider than the stencil
    lap = dense_laplacian((n, n, n), vandermonde_weights(k), h, periodic=True) \
        if n ** 3 <= 2000 else None
    c = oracle_mod.fd_weights(k)
    lam_closed = 3 * (abs(c[0]) + 2 * np.sum(np.abs(c[1:]))) / h ** 2
    # Nyquist mode (-1)^(x+y+z) is an eigenvector of the oracle Laplacian
    g = np.indices((n, n, n)).sum(axis=0)
    nyq = (-1.0) ** g
    ln = oracle_mod.laplacian(nyq, k, h, periodic=True)
    np.testing.assert_allclose(-ln, lam_closed * nyq, rtol=1e-12, atol=0)
    if lap is not None:
        lam_dense = np.max(np.linalg.eigvalsh(-lap))
        assert lam_dense == pytest.approx(lam_closed, rel=1e-10)
    dt = oracle_mod.dt_max(k, h, v)
    assert dt == pytest.approx(2.0 / (v * np.sqrt(lam_closed)), rel=1e-14)


@pytest.mark.parametrize("k", [2, 8])
def test_dt_max_separates_stable_from_unstable(oracle_mod, k):
    """Just below dt_max a random start stays bounded; just above it blows up."""
    h, v = 10.0, 1500.0
    n = 12
    m = np.full((n, n, n), 1.0 / v ** 2)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((n, n, n))
    dtm = oracle_mod.dt_max(k, h, v)
    res = {}
    for f in (0.98, 1.02):
        u, up = oracle_mod.forward(m, None, k, h, f * dtm, 400, u0=u0, u_prev0=u0,
                                   periodic=True)
        res[f] = np.max(np.abs(u))
    assert res[0.98] < 50 * np.max(np.abs(u0))
    assert res[1.02] > 1e3 * np.max(np.abs(u0))


def test_weights_reject_bad_orders(oracle_mod):
    for k in (0, 1, 3, 26, -2):
        with pytest.raises(ValueError):
            oracle_mod.fd_weights(k)
