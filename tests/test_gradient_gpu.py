"""GPU tests of the FWI gradient (forward pass storing the second time
difference, adjoint pass backward in time with the residuals injected at the
receivers and the gradient accumulated in the step kernel) against the FP64
oracle's exact discrete gradient, for integer-node and off-grid sources."""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2

pytestmark = pytest.mark.gpu
H = inputs.H


def _case(k, seed):
    rng = np.random.default_rng(seed)
    interior = (30, 34, 38)
    nbl = 6
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=4.0)
    spec = inputs.ShotSpec(interior, nbl, k, vel, (0, 0, 0), 25.0, 60)
    hi = np.array(interior, dtype=np.float64) - 1
    recs = np.vstack([rng.uniform(0, 1, (40, 3)) * hi, [[0, 0, 0], hi]])
    # observed data: the oracle's traces in a perturbed model
    pert = 1 + 0.03 * inputs._gaussian_smooth(rng.standard_normal(spec.shape), 3.0)
    return spec, recs, (spec.m.astype(np.float64) * pert)


@pytest.mark.parametrize("obs_kind", ["zero", "perturbed"])
@pytest.mark.parametrize("offgrid", [False, True])
@pytest.mark.parametrize("k", [4, 8])
def test_fwi_gradient_matches_oracle(oracle_mod, k, offgrid, obs_kind):
    """obs_kind "zero": d_obs = 0, the residual is the traces themselves; "perturbed":
    d_obs from a 3 % smooth model perturbation, so the residual is a small
    difference of traces and its FP32 error is amplified by |syn| / |residual|
    (the bounds scale with that ratio)."""
    spec, recs, m_true = _case(k, seed=10 + k)
    dt = dt_for(spec, 0.8)
    eta = eta_for(spec)
    nt = spec.nt
    wav = inputs.ricker(25.0, dt, nt)
    src = (14.3, 17.6, 20.45) if offgrid else (14, 17, 20)
    nbl = spec.nbl
    s_dom = [tuple(c + nbl for c in src)]
    r_dom = recs + nbl
    w64 = np.asarray(wav, dtype=np.float32).astype(np.float64)[None, :]
    if obs_kind == "zero":
        obs = np.zeros((len(recs), nt), np.float32)
    else:
        _, obs, _ = oracle_mod.fwi_gradient(m_true, eta.astype(np.float64), k, H, dt, nt, s_dom, w64, r_dom,
                                            np.zeros((len(recs), nt)))
        obs = obs.astype(np.float32)
    g_want, syn_want, J_want = oracle_mod.fwi_gradient(spec.m.astype(np.float64), eta.astype(np.float64), k, H, dt,
                                                       nt, s_dom, w64, r_dom, obs.astype(np.float64))
    with fd.Shot(spec.interior, k, H, dt, nbl) as shot:
        shot.set_model(spec.m, eta)
        if offgrid:
            shot.inject_at(*src, wav)
        else:
            shot.inject(*src, wav)
        g, syn, J = shot.fwi_gradient(recs, obs)
        # a second call on the same handle gives the same result
        g2, _, J2 = shot.fwi_gradient(recs, obs)
    e_syn, e_g = rel_l2(syn, syn_want), rel_l2(g, g_want)
    e_j = abs(J - J_want) / J_want
    amp = np.linalg.norm(syn_want) / np.linalg.norm(syn_want - obs)  # |syn| / |residual|
    print(f"PARITY fwi_grad_so{k}_{'offgrid' if offgrid else 'node'}_{obs_kind} traces {e_syn:.3e} misfit "
          f"{e_j:.3e} gradient {e_g:.3e} (|syn|/|res| {amp:.1f})")
    assert J_want > 0 and np.max(np.abs(g_want)) > 0
    # traces: the FP32 parity bound; misfit and gradient: that bound carried through
    # the residual (x2 for the square in J), plus the FP32 rounding of the two passes
    assert e_syn <= 1e-5
    assert e_j <= 2 * 1e-5 * amp
    assert e_g <= 1e-5 * amp + 2e-5
    np.testing.assert_array_equal(g, g2)
    assert J == J2


@pytest.mark.parametrize("segment", [1, 7, 13, 60])
def test_checkpointed_gradient_is_bitwise_equal(segment):
    """Checkpointing (states kept every `segment` steps, histories recomputed in
    the adjoint pass) gives the full-history gradient, traces and misfit bit for
    bit, and leaves the handle at the same final state."""
    spec, recs, m_true = _case(8, seed=21)
    dt = dt_for(spec, 0.8)
    wav = inputs.ricker(25.0, dt, spec.nt)
    rng = np.random.default_rng(5)
    obs = (rng.standard_normal((len(recs), spec.nt)) * 1e-4).astype(np.float32)
    out = []
    for seg in (0, segment):
        with fd.Shot(spec.interior, 8, H, dt, spec.nbl) as shot:
            shot.set_model(spec.m)
            shot.inject_at(14.3, 17.6, 20.45, wav)
            g, syn, J = shot.fwi_gradient(recs, obs, segment=seg)
            out.append((g, syn, J, shot.wavefield(0), shot.wavefield(1), shot.step))
    (g0, s0, j0, u0, p0, n0), (g1, s1, j1, u1, p1, n1) = out
    np.testing.assert_array_equal(g1, g0)
    np.testing.assert_array_equal(s1, s0)
    assert j1 == j0 and n1 == n0 == spec.nt
    np.testing.assert_array_equal(u1, u0)
    np.testing.assert_array_equal(p1, p0)


def test_fwi_gradient_errors():
    spec, recs, _ = _case(4, seed=3)
    dt = dt_for(spec, 0.8)
    with fd.Shot(spec.interior, 4, H, dt, spec.nbl) as shot:
        with pytest.raises(fd.FdError) as e:
            shot.fwi_gradient(recs, np.zeros((len(recs), 5), np.float32))
        assert e.value.code == fd.FD_ESTATE
        shot.set_model(spec.m)
        with pytest.raises(fd.FdError) as e:
            shot.fwi_gradient([(40.0, 1, 1)], np.zeros((1, 5), np.float32))
        assert e.value.code == fd.FD_ERANGE
    with fd.Shot(spec.interior, 4, H, dt, spec.nbl, storage="bf16") as shot:
        shot.set_model(spec.m)
        with pytest.raises(fd.FdError) as e:
            shot.fwi_gradient(recs, np.zeros((len(recs), 5), np.float32))
        assert e.value.code == fd.FD_ENOTSUP
