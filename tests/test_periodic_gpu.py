"""GPU tests of the periodic-boundary test mode (every axis wraps around).

On a 3-torus the discrete scheme has exact solutions and invariants that do
not depend on the oracle: a discrete plane wave cos(k.x - w n dt) is an exact
solution when sin^2(w dt/2) = (v^2 dt^2 / 4h^2) sum_a sigma(k_a h), with
sigma(theta) = -c_0 - 2 sum_j c_j cos(j theta) the symbol of the central
second difference; and with eta = 0 and no source the discrete energy
E = sum m ((u^{n+1} - u^n)/dt)^2 - sum u^{n+1} (L u^n) is conserved (L is
symmetric). The mode is also checked against the FP64 oracle's periodic
stepping, and, where no tap wraps, bit for bit against the zero-boundary
naive kernel (same per-point arithmetic).
"""
from math import factorial

import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import _abi, inputs
from harness import rel_l2

pytestmark = pytest.mark.gpu
H = inputs.H


def _weights(k):
    """Central second-derivative weights of accuracy order k in closed form."""
    r = k // 2
    c = np.zeros(r + 1)
    for j in range(1, r + 1):
        c[j] = 2.0 * (-1) ** (j + 1) * factorial(r) ** 2 / (j * j * factorial(r - j) * factorial(r + j))
    c[0] = -2.0 * c[1:].sum()
    return c


def _smooth_model(shape, seed, vmin=1500.0, vmax=3000.0):
    rng = np.random.default_rng(seed)
    v = inputs.smooth_random_velocity(shape, 0, rng, vmin=vmin, vmax=vmax, sigma=3.0)
    return inputs.slowness2(v).astype(np.float32), rng


@pytest.mark.parametrize("form", ["factored", "expanded"])
@pytest.mark.parametrize("k", [2, 8, 16])
def test_periodic_matches_oracle(oracle_mod, k, form):
    """Random smooth model, damping in scattered cells, six sources (two at
    corners, so their stencils wrap; two beyond the four fused ones)."""
    shape = (37, 29, 44)
    m, rng = _smooth_model(shape, seed=k)
    eta = np.where(rng.uniform(size=shape) < 0.1, m * rng.uniform(0, 20.0, shape), 0).astype(np.float32)
    dt = 0.8 * fd.fd_dt_max(k, H, 3000.0)
    nodes = [(0, 0, 0), (36, 28, 43), (18, 3, 40), (5, 20, 1), (30, 14, 22), (18, 3, 40)]
    wavs = [inputs.ricker(20.0 + 2 * i, dt, 50) for i in range(len(nodes))]
    nt = 60
    with fd.Shot(shape, k, H, dt, 0, form=form, boundary="periodic") as shot:
        shot.set_model(m, eta)
        for n, w in zip(nodes, wavs):
            shot.inject(*n, w)
        shot.forward(nt)
        got, got_prev = shot.wavefield(0), shot.wavefield(1)
    w64 = np.stack([np.asarray(w, np.float32).astype(np.float64) for w in wavs])
    want, want_prev = oracle_mod.forward(m.astype(np.float64), eta.astype(np.float64), k, H, dt, nt, nodes, w64,
                                         periodic=True)
    e0, e1 = rel_l2(got, want), rel_l2(got_prev, want_prev)
    print(f"PARITY periodic_so{k}_{form} {e0:.3e} {e1:.3e}")
    assert e0 <= 1e-5 and e1 <= 1e-5


@pytest.mark.parametrize("k", [4, 8])
def test_periodic_plane_wave_closed_form(k):
    """u^0 = cos(k.x), u^{-1} = cos(k.x + w dt) in a constant medium: after 300
    steps the field is cos(k.x - 300 w dt) with w from the scheme's dispersion
    relation (FP32 rounding only)."""
    shape = (24, 20, 16)
    v = 2000.0
    m = np.full(shape, 1.0 / v ** 2, np.float32)
    dt = 0.9 * fd.fd_dt_max(k, H, v)
    n_wave = (3, 2, 5)
    kvec = [2 * np.pi * n_wave[a] / (shape[a] * H) for a in range(3)]
    c = _weights(k)
    sigma = sum(-c[0] - 2 * sum(c[j] * np.cos(j * kvec[a] * H) for j in range(1, k // 2 + 1)) for a in range(3))
    w = 2.0 / dt * np.arcsin(np.sqrt(v * v * dt * dt / (4 * H * H) * sigma))
    ix = np.meshgrid(*[np.arange(n) * H for n in shape], indexing="ij")
    phase = sum(kvec[a] * ix[a] for a in range(3))
    nt = 300
    with fd.Shot(shape, k, H, dt, 0, boundary="periodic") as shot:
        shot.set_model(m, np.zeros(shape, np.float32))
        shot.load_state(np.cos(phase).astype(np.float32), np.cos(phase + w * dt).astype(np.float32), 0)
        shot.forward(nt)
        got, got_prev = shot.wavefield(0), shot.wavefield(1)
    want, want_prev = np.cos(phase - w * nt * dt), np.cos(phase - w * (nt - 1) * dt)
    e0, e1 = rel_l2(got, want), rel_l2(got_prev, want_prev)
    print(f"PLANE_WAVE periodic_so{k} w*dt={w * dt:.4f} {e0:.3e} {e1:.3e}")
    assert e0 <= 5e-5 and e1 <= 5e-5


@pytest.mark.parametrize("form", ["factored", "expanded"])
def test_periodic_energy_conserved(oracle_mod, form):
    """eta = 0: a source that acts for the first 30 steps only; from then on
    the discrete energy of the FP32 levels stays constant to FP32 rounding."""
    k = 8
    shape = (32, 28, 36)
    m, _ = _smooth_model(shape, seed=11)
    dt = 0.9 * fd.fd_dt_max(k, H, 3000.0)
    energies = []
    with fd.Shot(shape, k, H, dt, 0, form=form, boundary="periodic") as shot:
        shot.set_model(m, np.zeros(shape, np.float32))
        shot.inject(16, 14, 18, inputs.ricker(30.0, dt, 30))
        shot.forward(40)
        for _ in range(4):
            shot.forward(100)
            energies.append(oracle_mod.energy(shot.wavefield(0), shot.wavefield(1), m, k, H, dt, periodic=True))
    e = np.array(energies)
    drift = np.max(np.abs(e - e[0])) / e[0]
    print(f"ENERGY periodic_so{k}_{form} E={e[0]:.6e} max rel drift {drift:.3e}")
    assert e[0] > 0 and drift <= 2e-5


@pytest.mark.parametrize("form", ["factored", "expanded"])
def test_periodic_equals_zero_boundary_before_the_wave_wraps(form):
    """A centred source on a 40^3 torus, 8 steps of space order 4: no tap that
    wraps reads a nonzero value yet, so the periodic kernel and the zero-halo
    naive kernel give the same bits (same per-point arithmetic)."""
    k, shape = 4, (40, 40, 40)
    m, rng = _smooth_model(shape, seed=3)
    eta = (m * rng.uniform(0, 10.0, shape)).astype(np.float32)
    dt = 0.9 * fd.fd_dt_max(k, H, 3000.0)
    out = []
    for boundary, kernel in (("periodic", "auto"), ("zero", "naive")):
        with fd.Shot(shape, k, H, dt, 0, form=form, kernel=kernel, boundary=boundary) as shot:
            shot.set_model(m, eta)
            shot.inject(20, 20, 20, inputs.ricker(40.0, dt, 8))
            shot.forward(8)
            out.append((shot.wavefield(0), shot.wavefield(1)))
    assert np.count_nonzero(out[0][0]) > 1000
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_periodic_rejections():
    shape = (24, 24, 24)
    m, _ = _smooth_model(shape, seed=4)
    dt = 0.9 * fd.fd_dt_max(4, H, 3000.0)
    for kw in (dict(kernel="tma"), dict(kernel="stream"), dict(storage="bf16")):
        with pytest.raises(fd.FdError) as e:
            fd.Shot(shape, 4, H, dt, 0, boundary="periodic", **kw)
        assert e.value.code == fd.FD_ENOTSUP
    o = fd.options()
    o.boundary = 7
    with pytest.raises(fd.FdError) as e:
        _abi.fd_acoustic_create_ex(*shape, 4, H, dt, 0, o)
    assert e.value.code == fd.FD_ENOTSUP
    with pytest.raises(fd.FdError) as e:
        _abi.fd_batch_create(4, H, fd.options(boundary="periodic"))
    assert e.value.code == fd.FD_ENOTSUP
    with fd.Shot(shape, 2, H, dt, 0, boundary="periodic") as shot:
        shot.set_model(m, np.zeros(shape, np.float32))
        with pytest.raises(fd.FdError) as e:
            shot.forward_two_step(2)
        assert e.value.code == fd.FD_ENOTSUP
        with pytest.raises(fd.FdError) as e:
            shot.fwi_gradient([(3.0, 3.0, 3.0)], np.zeros((1, 4), np.float32))
        assert e.value.code == fd.FD_ENOTSUP
        # the auto kernel choice is the naive kernel
        assert shot.config[0] == fd.FD_KERNEL_NAIVE
