"""The synthetic input recipe pinned to the workloads it stands for: the plain
64^3 shot, the 256^3 + 10 sweep (4 equal horizontal layers 1.5-4.5 km/s along
z, 15 Hz Ricker at (128, 128, 20), 500 steps), the 64 uneven batched shots
(each axis U{96..256}, smooth random velocity in [1.5, 4.5] km/s, 300 steps),
the 384^3 + 20 precision shot and the Poisson serving trace; and the Ricker
wavelet against its closed form."""
import math

import numpy as np

from paper_1912_00695_gb300 import inputs


def test_plain_shot():
    s = inputs.plain_shot()
    assert s.interior == (64, 64, 64) and s.nbl == 10 and s.space_order == 4 and s.nt == 100
    assert s.shape == (84, 84, 84) and s.source == (32, 32, 32) and s.f0 == 10.0
    assert np.all(s.velocity == 1500.0)
    np.testing.assert_allclose(s.m, 1.0 / 1500.0 ** 2, rtol=1e-7)


def test_sweep_shot_layers_and_source():
    s = inputs.sweep_shot(8)
    assert s.interior == (256, 256, 256) and s.nbl == 10 and s.shape == (276, 276, 276)
    assert s.source == (128, 128, 20) and s.f0 == 15.0 and s.nt == 500 and s.points == 276 ** 3
    v = s.velocity
    # layers of 64 interior cells along z (depth), edge-replicated into the absorbing layer
    for i, vel in enumerate((1500.0, 2500.0, 3500.0, 4500.0)):
        z0, z1 = 10 + 64 * i, 10 + 64 * (i + 1)
        assert np.all(v[:, :, z0:z1] == vel)
    assert np.all(v[:, :, :10] == 1500.0) and np.all(v[:, :, -10:] == 4500.0)
    assert np.all(v == v[:1, :1, :])  # horizontal layers: no x or y dependence
    assert s.vmax == 4500.0


def test_batched_shots():
    shots = inputs.batched_shots()
    assert len(shots) == 64
    sizes = np.array([s.interior for s in shots])
    assert sizes.min() >= 96 and sizes.max() <= 256 and len({s.interior for s in shots}) > 60
    for s in shots[:6]:  # velocity fields are the costly part: a sample
        assert s.space_order == 8 and s.nt == 300 and s.nbl == 10 and s.f0 == 10.0
        assert 1500.0 - 1e-6 <= s.velocity.min() and s.velocity.max() <= 4500.0 + 1e-6
        assert all(0 <= c < n for c, n in zip(s.source, s.interior))
    # seeded: the same draws again
    again = inputs.batched_shots(count=3)
    assert [s.interior for s in again] == [s.interior for s in shots[:3]]
    np.testing.assert_array_equal(again[0].velocity, shots[0].velocity)


def test_precision_shot():
    s = inputs.precision_shot()
    assert s.interior == (384, 384, 384) and s.nbl == 20 and s.space_order == 12 and s.nt == 1000
    assert s.shape == (424, 424, 424)
    v = s.velocity
    for i, vel in enumerate((1500.0, 2500.0, 3500.0, 4500.0)):
        assert np.all(v[:, :, 20 + 96 * i:20 + 96 * (i + 1)] == vel)


def test_serving_trace():
    tr = inputs.serving_trace(count=400, rate=20.0, lo=128, hi=256, steps=(200, 1000))
    arr = np.array([s.arrival for s in tr])
    assert np.all(np.diff(arr) > 0)
    # Poisson at 20 per second: mean gap 0.05 s (400 gaps: within 4 standard errors)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 0.05) < 4 * 0.05 / math.sqrt(len(gaps))
    assert all(128 <= s.interior[0] <= 256 and s.interior[0] == s.interior[1] == s.interior[2] for s in tr)
    assert {s.space_order for s in tr} == {8, 16} and {s.storage for s in tr} == {"f32", "bf16"}
    assert all(200 <= s.nt <= 1000 for s in tr)
    v = inputs.velocity_for(tr[0])
    assert v.shape == tr[0].shape and v.min() >= 1500.0 - 1e-6 and v.max() <= 4500.0 + 1e-6


def test_ricker_closed_form():
    f0, dt, nt = 10.0, 1e-3, 400  # the peak t = 1/f0 falls on a sample
    w = inputs.ricker(f0, dt, nt).astype(np.float64)
    n_peak = int(round(1.0 / f0 / dt))
    assert abs(w[n_peak] - 1.0) < 1e-6 and np.argmax(w) == n_peak  # peak 1 at t = 1/f0
    # zero crossings at tau = +-1/(pi f0 sqrt 2)
    tau0 = 1.0 / (math.pi * f0 * math.sqrt(2.0))
    t = np.arange(nt) * dt - 1.0 / f0
    sign = np.sign(w)
    crossings = t[1:][sign[1:] != sign[:-1]]
    assert np.allclose(sorted(np.abs(crossings))[:2], tau0, atol=dt)
    # the closed form at a few samples
    for n in (0, 30, 66, 100, 250):
        a = (math.pi * f0 * (n * dt - 1.0 / f0)) ** 2
        assert abs(w[n] - (1 - 2 * a) * math.exp(-a)) < 1e-6
