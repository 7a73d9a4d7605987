"""Independent reference constructions used to pin the oracle (test-side only).

Nothing here calls the oracle or the library. Each helper derives a quantity by
a route different from the oracle's: weights by an exact rational Vandermonde
solve (the oracle uses a closed form), the Laplacian as a sum of Kronecker
products of 1D Toeplitz matrices (the oracle loops over stencil offsets), the
plane-wave symbol in closed form.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def vandermonde_weights(space_order: int) -> list[Fraction]:
    """Exact symmetric weights c_0..c_r of the centred 2nd derivative.

    Solves sum_{j=-r..r} c_|j| j^(2p) = 2 * [p == 1] for p = 0..r in exact
    rational arithmetic (Gaussian elimination on Fractions): the conditions
    that the stencil differentiates x^(2p) exactly at 0, which for an even
    stencil is accuracy order 2r.
    """
    r = space_order // 2
    n = r + 1
    # unknowns c_0..c_r; row p: c_0 * [p == 0] + sum_{j>=1} 2 c_j j^(2p)
    a = [[Fraction(0)] * n for _ in range(n)]
    b = [Fraction(0)] * n
    for p in range(n):
        a[p][0] = Fraction(1 if p == 0 else 0)
        for j in range(1, n):
            a[p][j] = Fraction(2 * j ** (2 * p))
        b[p] = Fraction(2 if p == 1 else 0)
    # Gaussian elimination with exact pivoting
    for col in range(n):
        piv = next(i for i in range(col, n) if a[i][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        b[col], b[piv] = b[piv], b[col]
        for i in range(n):
            if i != col and a[i][col] != 0:
                f = a[i][col] / a[col][col]
                a[i] = [x - f * y for x, y in zip(a[i], a[col])]
                b[i] -= f * b[col]
    return [b[i] / a[i][i] for i in range(n)]


def symbol(weights, theta):
    """sigma(theta) = -c_0 - 2 sum_j c_j cos(j theta): minus the 1D stencil's
    eigenvalue on the Fourier mode exp(i j theta), times h^2."""
    c = [float(w) for w in weights]
    theta = np.asarray(theta, dtype=np.float64)
    s = -c[0] * np.ones_like(theta)
    for j in range(1, len(c)):
        s -= 2.0 * c[j] * np.cos(j * theta)
    return s


def second_derivative_matrix(n: int, weights, h: float, periodic: bool) -> np.ndarray:
    """1D Toeplitz (circulant when periodic) matrix of the centred stencil."""
    c = [float(w) for w in weights]
    r = len(c) - 1
    d = np.zeros((n, n))
    for i in range(n):
        for j in range(-r, r + 1):
            k = i + j
            if periodic:
                d[i, k % n] += c[abs(j)]
            elif 0 <= k < n:
                d[i, k] += c[abs(j)]
    return d / (h * h)


def dense_laplacian(shape, weights, h: float, periodic: bool = False) -> np.ndarray:
    """L = Dx (x) I (x) I + I (x) Dy (x) I + I (x) I (x) Dz for C-order [x][y][z]."""
    nx, ny, nz = shape
    ix, iy, iz = np.eye(nx), np.eye(ny), np.eye(nz)
    dx = second_derivative_matrix(nx, weights, h, periodic)
    dy = second_derivative_matrix(ny, weights, h, periodic)
    dz = second_derivative_matrix(nz, weights, h, periodic)
    return (np.kron(np.kron(dx, iy), iz) + np.kron(np.kron(ix, dy), iz)
            + np.kron(np.kron(ix, iy), dz))


def dense_forward(m, eta, weights, h, dt, nt, sources=(), wavelets=None, periodic=False):
    """Brute-force time stepping with the assembled dense operator.

    Each step solves  A u^{n+1} = dt^2 (L u^n + q^n) + M (2 u^n - u^{n-1}) + (dt/2) E u^{n-1}
    with A = M + (dt/2) E as a dense linear system (M, E diagonal matrices of m, eta).
    """
    shape = m.shape
    n = int(np.prod(shape))
    lap = dense_laplacian(shape, weights, h, periodic)
    mm = np.diag(m.reshape(-1).astype(np.float64))
    ee = np.diag((np.zeros(n) if eta is None else eta.reshape(-1)).astype(np.float64))
    a = mm + 0.5 * dt * ee
    u = np.zeros(n)
    up = np.zeros(n)
    flat = [np.ravel_multi_index(s, shape) for s in sources]
    for step in range(nt):
        rhs = dt * dt * (lap @ u) + mm @ (2 * u - up) + 0.5 * dt * (ee @ up)
        for s, p in enumerate(flat):
            w = wavelets[s]
            q = w[step] if step < len(w) else 0.0
            rhs[p] += dt * dt * q
        nxt = np.linalg.solve(a, rhs)
        up, u = u, nxt
    return u.reshape(shape), up.reshape(shape)
