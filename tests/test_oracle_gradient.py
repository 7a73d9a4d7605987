"""Pins of the oracle's adjoint propagation and FWI gradient (the motivating
workloads of Sec. 1 and Sec. 5, not formulated in the paper).

Fixed against: central finite differences of the misfit J(m) along random
model perturbations (the gradient is the exact derivative of the discrete
scheme, so the agreement is limited only by the O(eps^2) truncation), the
dot-product test <F q, d> = <q, F^T d> of the adjoint, and the zero gradient
of a zero residual.
"""
import numpy as np
import pytest

from paper_1912_00695_gb300 import inputs


def _setup(seed, shape=(9, 10, 8), k=4, damping=True):
    rng = np.random.default_rng(seed)
    h = 10.0
    vel = inputs._gaussian_smooth(rng.uniform(1500, 3000, shape), 1.0)
    m = 1.0 / vel ** 2
    eta = m * rng.uniform(0, 25.0, shape) if damping else None
    return rng, m, eta, k, h


@pytest.mark.parametrize("damping", [False, True])
def test_gradient_matches_finite_differences(oracle_mod, damping):
    rng, m, eta, k, h = _setup(1, damping=damping)
    dt = 0.7 * oracle_mod.dt_max(k, h, float(1 / np.sqrt(m.min())))
    nt = 40
    src = [(4.3, 5.2, 3.7)]
    recs = [(1.5, 2.5, 2.0), (7.2, 8.1, 5.5), (2.0, 7.75, 6.0), (6.6, 1.0, 1.25)]
    wav = inputs.ricker(30.0, dt, nt)[None, :].astype(np.float64)
    # observed data: the same shot in a perturbed model (so the residual is not small)
    m_true = m * (1 + 0.05 * inputs._gaussian_smooth(rng.standard_normal(m.shape), 1.5))
    _, obs, _ = oracle_mod.fwi_gradient(m_true, eta, k, h, dt, nt, src, wav, recs, np.zeros((4, nt)))
    g, _, J0 = oracle_mod.fwi_gradient(m, eta, k, h, dt, nt, src, wav, recs, obs)
    assert J0 > 0 and np.max(np.abs(g)) > 0
    for trial in range(3):
        dm = m * inputs._gaussian_smooth(rng.standard_normal(m.shape), 1.0)
        eps = 1e-4
        _, _, jp = oracle_mod.fwi_gradient(m + eps * dm, eta, k, h, dt, nt, src, wav, recs, obs)
        _, _, jm = oracle_mod.fwi_gradient(m - eps * dm, eta, k, h, dt, nt, src, wav, recs, obs)
        fd = (jp - jm) / (2 * eps)
        an = float(np.sum(g * dm))
        assert abs(fd - an) <= 1e-6 * abs(an), (trial, fd, an)


def test_adjoint_dot_product(oracle_mod):
    """<F q, d> = <q, F^T d> for the map from source wavelets to traces."""
    rng, m, eta, k, h = _setup(2)
    dt = 0.7 * oracle_mod.dt_max(k, h, float(1 / np.sqrt(m.min())))
    nt = 35
    src = [(4.3, 5.2, 3.7), (2.0, 2.5, 6.25)]
    recs = [(1.5, 2.5, 2.0), (7.2, 8.1, 5.5), (2.0, 7.75, 6.0)]
    q = rng.standard_normal((2, nt))
    d = rng.standard_normal((3, nt))
    _, fq, _, ftd = oracle_mod.fwi_gradient(m, eta, k, h, dt, nt, src, q, recs, d, adjoint=True)
    lhs = float(np.sum(fq * d))
    rhs = float(np.sum(q * ftd))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300), (lhs, rhs)


def test_zero_residual_zero_gradient(oracle_mod):
    rng, m, eta, k, h = _setup(3)
    dt = 0.7 * oracle_mod.dt_max(k, h, float(1 / np.sqrt(m.min())))
    nt = 20
    src = [(4.0, 5.0, 3.0)]
    recs = [(1.5, 2.5, 2.0)]
    wav = rng.standard_normal((1, nt))
    _, syn, _ = oracle_mod.fwi_gradient(m, eta, k, h, dt, nt, src, wav, recs, np.zeros((1, nt)))
    g, _, J = oracle_mod.fwi_gradient(m, eta, k, h, dt, nt, src, wav, recs, syn)
    assert J == 0.0 and np.all(g == 0.0)
