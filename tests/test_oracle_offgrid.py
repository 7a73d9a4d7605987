"""Pins of the oracle's off-grid sources and receivers (trilinear spreading and
sampling between nodes, the next step of the workflow named in Sec. 5).

Fixed against: scipy's linear interpolator (sampling), integer-node sources
combined by linearity and a dense brute force whose operators are assembled
from scipy's interpolator (spreading), exactness on affine fields, and
reciprocity between off-grid points with damping.
"""
import numpy as np
import pytest
from scipy.ndimage import map_coordinates

from pinlib import dense_laplacian, vandermonde_weights


def _scipy_row(point, shape):
    """Sampling operator row of a point, assembled from scipy's order-1
    interpolator applied to every unit field (independent of the oracle)."""
    n = int(np.prod(shape))
    row = np.zeros(n)
    e = np.zeros(n)
    coords = np.asarray(point, dtype=np.float64).reshape(3, 1)
    for i in range(n):
        e[i] = 1.0
        row[i] = map_coordinates(e.reshape(shape), coords, order=1, mode="nearest")[0]
        e[i] = 0.0
    return row


def test_trilinear_weights(oracle_mod):
    rng = np.random.default_rng(0)
    shape = (7, 9, 8)
    a, b = rng.standard_normal(3), rng.standard_normal()
    for _ in range(200):
        p = rng.uniform(0, 1, 3) * (np.array(shape) - 1)
        nodes, w = oracle_mod.trilinear(p, shape)
        assert abs(w.sum() - 1.0) < 1e-15
        assert np.all(w >= 0)
        assert np.all(nodes >= 0) and np.all(nodes < np.array(shape))
        # affine fields are reproduced exactly
        np.testing.assert_allclose(np.dot(w, nodes @ a + b), p @ a + b, rtol=0, atol=1e-12)
    # a node (including the last one on every axis) carries weight 1 on itself
    for p in [(0, 0, 0), (3, 4, 5), (6, 8, 7), (6, 0, 7)]:
        nodes, w = oracle_mod.trilinear(p, shape)
        assert np.isclose(w.max(), 1.0) and np.count_nonzero(w) == 1
        assert tuple(nodes[np.argmax(w)]) == tuple(p)
    for bad in [(-1e-9, 1, 1), (6.0000001, 1, 1), (1, 1, 7.5)]:
        with pytest.raises(ValueError):
            oracle_mod.trilinear(bad, shape)


def test_receivers_sample_like_scipy(oracle_mod):
    """A receiver's last sample equals scipy's linear interpolation of the
    final field at that point."""
    rng = np.random.default_rng(1)
    shape = (12, 10, 11)
    k, h = 4, 10.0
    m = 1.0 / rng.uniform(1500, 3000, shape) ** 2
    dt = 0.8 * oracle_mod.dt_max(k, h, 3000.0)
    recs = [tuple(rng.uniform(0, 1, 3) * (np.array(shape) - 1)) for _ in range(25)]
    recs += [(0.0, 0.0, 0.0), (11.0, 9.0, 10.0), (11.0, 4.5, 0.25)]
    wav = rng.standard_normal((1, 30))
    u, _, tr = oracle_mod.forward_offgrid(m, None, k, h, dt, 30, [(5.3, 4.6, 5.1)], wav, recs)
    want = map_coordinates(u, np.array(recs).T, order=1, mode="nearest")
    assert np.max(np.abs(want)) > 0
    np.testing.assert_allclose(tr[:, -1], want, rtol=0, atol=1e-13 * np.max(np.abs(want)))


def test_offgrid_source_is_weighted_integer_sources(oracle_mod):
    """Spreading: a source between nodes equals the 8 integer-node sources with
    the wavelet scaled by scipy's interpolation weights; a source on a node
    equals the integer-node source."""
    rng = np.random.default_rng(2)
    shape = (9, 10, 8)
    k, h = 8, 10.0
    m = 1.0 / rng.uniform(1500, 3500, shape) ** 2
    eta = m * rng.uniform(0, 20.0, shape)
    dt = 0.8 * oracle_mod.dt_max(k, h, 3500.0)
    wav = rng.standard_normal((1, 25))
    p = (4.3, 2.75, 6.6)
    u_off, _, _ = oracle_mod.forward_offgrid(m, eta, k, h, dt, 25, [p], wav)
    row = _scipy_row(p, shape)
    nodes = [np.unravel_index(i, shape) for i in np.flatnonzero(row)]
    assert len(nodes) == 8
    u_sum = np.zeros(shape)
    for nd in nodes:
        u_i, _ = oracle_mod.forward(m, eta, k, h, dt, 25, [tuple(int(v) for v in nd)], wav)
        u_sum += row[np.ravel_multi_index(nd, shape)] * u_i
    np.testing.assert_allclose(u_off, u_sum, rtol=0, atol=1e-12 * np.max(np.abs(u_sum)))
    u_on, _, _ = oracle_mod.forward_offgrid(m, eta, k, h, dt, 25, [(4.0, 2.0, 6.0)], wav)
    u_int, _ = oracle_mod.forward(m, eta, k, h, dt, 25, [(4, 2, 6)], wav)
    np.testing.assert_array_equal(u_on, u_int)


def test_offgrid_dense_brute_force(oracle_mod):
    """Dense operators: A u^{n+1} = dt^2 (L u^n + s q^n) + M (2u^n - u^{n-1}) +
    (dt/2) E u^{n-1}, traces = R u^{n+1}, with the spreading vector s and the
    sampling rows R assembled from scipy's interpolator."""
    rng = np.random.default_rng(3)
    shape = (6, 7, 6)
    k, h = 4, 10.0
    n = int(np.prod(shape))
    m = 1.0 / rng.uniform(1500, 3000, shape) ** 2
    eta = m * rng.uniform(0, 30.0, shape)
    dt = 0.8 * oracle_mod.dt_max(k, h, 3000.0)
    nt = 20
    src = [(2.4, 3.7, 1.2), (4.9, 0.3, 5.0)]
    recs = [(1.5, 5.5, 4.25), (0.0, 6.0, 2.8), (3.3, 3.3, 3.3)]
    wav = rng.standard_normal((2, nt))
    lap = dense_laplacian(shape, [float(c) for c in vandermonde_weights(k)], h)
    mm, ee = m.reshape(-1), eta.reshape(-1)
    s_vecs = [_scipy_row(p, shape) for p in src]
    r_rows = np.array([_scipy_row(p, shape) for p in recs])
    u, up = np.zeros(n), np.zeros(n)
    want = np.zeros((len(recs), nt))
    for it in range(nt):
        rhs = dt * dt * (lap @ u) + mm * (2 * u - up) + 0.5 * dt * ee * up
        for s, sv in enumerate(s_vecs):
            rhs += dt * dt * wav[s, it] * sv
        nxt = rhs / (mm + 0.5 * dt * ee)
        up, u = u, nxt
        want[:, it] = r_rows @ u
    got_u, _, got_tr = oracle_mod.forward_offgrid(m, eta, k, h, dt, nt, src, wav, recs)
    np.testing.assert_allclose(got_u.reshape(-1), u, rtol=0, atol=1e-12 * np.max(np.abs(u)))
    np.testing.assert_allclose(got_tr, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


def test_offgrid_reciprocity(oracle_mod):
    """Trace at B from a source at A equals the trace at A from a source at B
    for off-grid A and B (spreading is the transpose of sampling), with damping."""
    rng = np.random.default_rng(4)
    shape = (10, 11, 9)
    k, h = 8, 10.0
    m = 1.0 / rng.uniform(1500, 4500, shape) ** 2
    eta = m * rng.uniform(0, 30.0, shape)
    dt = 0.8 * oracle_mod.dt_max(k, h, 4500.0)
    a, b = (2.2, 3.9, 4.45), (7.6, 8.1, 1.5)
    wav = rng.standard_normal((1, 50))
    _, _, tr_ab = oracle_mod.forward_offgrid(m, eta, k, h, dt, 50, [a], wav, [b])
    _, _, tr_ba = oracle_mod.forward_offgrid(m, eta, k, h, dt, 50, [b], wav, [a])
    assert np.max(np.abs(tr_ab)) > 0
    np.testing.assert_allclose(tr_ab, tr_ba, rtol=0, atol=1e-12 * np.max(np.abs(tr_ab)))
