"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Tolerance: relative L2 <= 1e-5 over the whole computational domain (the FP32
target), on the same seeded inputs. Grids span several tiles in every axis with
ragged tails; every space order 2..16, both stencil forms, both kernels, user
and default damping, sources near edges and in the layer, more sources than
the fused limit, chunked forwards, and the full 256^3 + 10 workload in the
benchmark's launch configuration (from a random full-field state, so that every
boundary and layer path is exercised in a few steps).
"""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = 1e-5


def report(name, *errs):
    """Print the measured error (visible with pytest -s) and return it."""
    print(f"PARITY {name} " + " ".join(f"{e:.3e}" for e in errs))


def test_plain_config_parity(oracle_mod):
    """64^3 + 10, space order 4, 1.5 km/s, 10 Hz Ricker at the centre, 100 steps."""
    spec = inputs.plain_shot()
    dt = dt_for(spec)
    eta = eta_for(spec)
    want, want_prev = run_oracle(oracle_mod, spec, spec.nt, dt, eta)
    for form in ("factored", "expanded"):
        for kernel in ("stream", "naive"):
            got, got_prev, shot = run_gpu(spec, spec.nt, dt, None, form=form, kernel=kernel)
            assert shot.step == spec.nt
            e0, e1 = rel_l2(got, want), rel_l2(got_prev, want_prev)
            report(f"plain_so4_{form}_{kernel}", e0, e1)
            assert e0 <= TOL and e1 <= TOL, (form, kernel, e0, e1)
            shot.close()


def _ragged_spec(k, seed=0):
    rng = np.random.default_rng(seed + k)
    interior = (37, 45, 51)
    nbl = 6
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=4.0)
    return inputs.ShotSpec(interior, nbl, k, vel, (1, 43, 25), 25.0, 60)


TMA_TILES = [(32, 32), (64, 16), (128, 8), (32, 16), (64, 8)]


@pytest.mark.parametrize("kernel", ["stream", "tma"])
@pytest.mark.parametrize("form", ["factored", "expanded"])
@pytest.mark.parametrize("k", [2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 22, 24])
def test_every_space_order_ragged(oracle_mod, k, form, kernel):
    spec = _ragged_spec(k)
    dt = dt_for(spec)
    eta = eta_for(spec)
    want, want_prev = run_oracle(oracle_mod, spec, spec.nt, dt, eta)
    tile = TMA_TILES[k % 5] if k <= 16 else [(32, 32), (32, 16)][k // 2 % 2]  # 32-wide above 16
    shape = dict(tile_y=8, x_block=16) if kernel == "stream" else \
        dict(zip(("tile_z", "tile_y"), tile), x_block=21)
    got, got_prev, shot = run_gpu(spec, spec.nt, dt, None, form=form, kernel=kernel, **shape)
    report(f"ragged_so{k}_{form}_{kernel}{shot.config}", rel_l2(got, want),
           rel_l2(got_prev, want_prev))
    assert rel_l2(got, want) <= TOL
    assert rel_l2(got_prev, want_prev) <= TOL
    shot.close()


@pytest.mark.parametrize("k", [2, 8, 16, 24])
def test_naive_kernel_ragged(oracle_mod, k):
    spec = _ragged_spec(k, seed=3)
    dt = dt_for(spec)
    eta = eta_for(spec)
    want, _ = run_oracle(oracle_mod, spec, spec.nt, dt, eta)
    got, _, shot = run_gpu(spec, spec.nt, dt, None, kernel="naive")
    assert rel_l2(got, want) <= TOL
    shot.close()


def test_user_damping_everywhere_and_many_sources(oracle_mod):
    """eta nonzero in the interior (no skipped loads), 6 sources (4 fused + 2
    injected separately), two at the same node, one in the layer corner."""
    rng = np.random.default_rng(4)
    spec = _ragged_spec(8, seed=4)
    dt = dt_for(spec)
    eta = (spec.m * rng.uniform(0, 15.0, spec.m.shape)).astype(np.float32)
    srcs = []
    for i, node in enumerate([(0, 0, 0), (36, 44, 50), (18, 22, 25), (5, 40, 3), (18, 22, 25),
                              (30, 1, 49)]):
        srcs.append((node, inputs.ricker(12.0 + i, dt, 40 + 3 * i, amplitude=1.0 + i)))
    want, want_prev = run_oracle(oracle_mod, spec, 50, dt, eta, sources=srcs)
    for form in ("factored", "expanded"):
        for kernel, shape in (("stream", dict(tile_y=4, x_block=32)),
                              ("tma", dict(tile_z=64, tile_y=8, x_block=19)),
                              ("naive", {})):
            got, got_prev, shot = run_gpu(spec, 50, dt, eta, sources=srcs, form=form,
                                          kernel=kernel, **shape)
            assert rel_l2(got, want) <= TOL, (form, kernel)
            assert rel_l2(got_prev, want_prev) <= TOL, (form, kernel)
            shot.close()


def test_chunked_forward_is_bitwise_identical():
    spec = _ragged_spec(6, seed=5)
    dt = dt_for(spec)
    for kernel, shape in (("stream", dict(tile_y=8, x_block=16)),
                          ("tma", dict(tile_z=32, tile_y=16, x_block=30))):
        a, ap, s1 = run_gpu(spec, 100, dt, chunks=[100], kernel=kernel, **shape)
        b, bp, s2 = run_gpu(spec, 100, dt, chunks=[50, 50], kernel=kernel, **shape)
        c, cp, s3 = run_gpu(spec, 100, dt, chunks=[1, 33, 7, 59], kernel=kernel, **shape)
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(ap, bp)
        np.testing.assert_array_equal(a, c)
        for s in (s1, s2, s3):
            s.close()


def test_launch_shape_does_not_change_results():
    """Per-point arithmetic order is independent of the tile shape and x-block,
    so every launch shape of a kernel gives the same bits."""
    spec = _ragged_spec(8, seed=6)
    dt = dt_for(spec)
    ref, _, s0 = run_gpu(spec, 40, dt, kernel="stream", tile_y=8, x_block=16)
    s0.close()
    for ty, xb in ((4, 7), (16, 49), (8, 3), (4, 100)):
        got, _, s = run_gpu(spec, 40, dt, kernel="stream", tile_y=ty, x_block=xb)
        np.testing.assert_array_equal(got, ref, err_msg=f"tile_y={ty} x_block={xb}")
        s.close()
    for form in ("factored", "expanded"):
        ref, _, s0 = run_gpu(spec, 40, dt, form=form, kernel="tma", tile_z=32, tile_y=32,
                             x_block=49)
        s0.close()
        for (tz, ty), xb in zip(TMA_TILES[1:], (5, 17, 32, 100)):
            got, _, s = run_gpu(spec, 40, dt, form=form, kernel="tma", tile_z=tz, tile_y=ty,
                                x_block=xb)
            np.testing.assert_array_equal(got, ref, err_msg=f"{form} tile {tz}x{ty} x_block={xb}")
            s.close()


def test_load_state_resume_matches_oracle(oracle_mod):
    """Random full-field state (every point nonzero, layer included), resumed at
    step 7 so that the wavelet index continues."""
    rng = np.random.default_rng(7)
    spec = _ragged_spec(12, seed=7)
    dt = dt_for(spec)
    eta = eta_for(spec)
    u0 = rng.standard_normal(spec.shape).astype(np.float32)
    u1 = (u0 + 0.05 * rng.standard_normal(spec.shape)).astype(np.float32)
    state = (u0, u1, 7)
    want, want_prev = run_oracle(oracle_mod, spec, 30, dt, eta, state=state)
    for kernel, shape in (("stream", dict(tile_y=16, x_block=16)),
                          ("tma", dict(tile_z=128, tile_y=8, x_block=16))):
        got, got_prev, shot = run_gpu(spec, 30, dt, None, state=state, kernel=kernel, **shape)
        assert shot.step == 37
        assert rel_l2(got, want) <= TOL, kernel
        assert rel_l2(got_prev, want_prev) <= TOL, kernel
        shot.close()


@pytest.mark.parametrize("form", ["factored", "expanded"])
@pytest.mark.parametrize("k", [2, 4, 8, 12, 16, 24])
def test_full_size_sweep_parity(oracle_mod, k, form):
    """The benchmark workload (256^3 + 10-cell layer, 4-layer model) with the
    autotuned launch shape (space order 2, factored: two steps per launch), 6
    steps from a smooth random full-field state."""
    spec = inputs.sweep_shot(k)
    dt = dt_for(spec)
    eta = eta_for(spec)
    rng = np.random.default_rng(k)
    u0 = inputs._gaussian_smooth(rng.standard_normal(spec.shape), 3.0).astype(np.float32)
    u1 = (0.98 * u0).astype(np.float32)
    state = (u0, u1, 0)
    want, want_prev = run_oracle(oracle_mod, spec, 6, dt, eta, state=state)
    got, got_prev, shot = run_gpu(spec, 6, dt, None, state=state, form=form)
    report(f"full276_so{k}_{form}_autotuned{shot.config}", rel_l2(got, want),
           rel_l2(got_prev, want_prev))
    assert rel_l2(got, want) <= TOL
    assert rel_l2(got_prev, want_prev) <= TOL
    shot.close()


@pytest.mark.parametrize("form", ["factored", "expanded"])
def test_full_size_sweep_100_steps(oracle_mod, form):
    """The benchmark shot itself (space order 8: 15 Hz Ricker at (128, 128, 20),
    zero initial state) for 100 steps, the step count of the FP32 parity bound."""
    spec = inputs.sweep_shot(8)
    dt = dt_for(spec)
    eta = eta_for(spec)
    want, want_prev = run_oracle(oracle_mod, spec, 100, dt, eta)
    got, got_prev, shot = run_gpu(spec, 100, dt, None, form=form)
    report(f"full276_so8_{form}_100steps{shot.config}", rel_l2(got, want), rel_l2(got_prev, want_prev))
    assert rel_l2(got, want) <= TOL
    assert rel_l2(got_prev, want_prev) <= TOL
    shot.close()


def test_error_codes():
    spec = inputs.plain_shot()
    dt = dt_for(spec)
    for bad_k in (5, 26):
        with pytest.raises(fd.FdError) as e:
            fd.Shot((8, 8, 8), bad_k, 10.0, 1e-3, 2)
        assert e.value.code == fd.FD_EINVAL
    with pytest.raises(fd.FdError) as e:  # batches stop at space order 16
        fd.Batch(18, 10.0)
    assert e.value.code == fd.FD_EINVAL
    shot = fd.Shot(spec.interior, 4, inputs.H, dt, spec.nbl)
    with pytest.raises(fd.FdError) as e:
        shot.forward(1)
    assert e.value.code == fd.FD_ESTATE
    bad = spec.m.copy()
    bad[3, 3, 3] = -1.0
    with pytest.raises(fd.FdError) as e:
        shot.set_model(bad)
    assert e.value.code == fd.FD_EINVAL
    with pytest.raises(fd.FdError) as e:
        shot.inject(64, 0, 0, np.ones(4, np.float32))
    assert e.value.code == fd.FD_ERANGE
    shot.close()
    fast = fd.Shot(spec.interior, 4, inputs.H, 1.2 * dt / 0.9, spec.nbl)
    with pytest.raises(fd.FdError) as e:
        fast.set_model(spec.m)
    assert e.value.code == fd.FD_EUNSTABLE
    fast.close()


def test_16bit_storage_options_rejected():
    """16-bit storage is the increment form on the TMA kernel, factored only."""
    for kw in (dict(storage="bf16", form="expanded"), dict(storage="f16", kernel="stream"),
               dict(storage="bf16", kernel="naive")):
        with pytest.raises(fd.FdError) as e:
            fd.Shot((16, 16, 16), 4, 10.0, 1e-3, 2, **kw)
        assert e.value.code == fd.FD_ENOTSUP, kw


def test_nonfinite_is_reported():
    spec = _ragged_spec(4, seed=8)
    dt = dt_for(spec)
    huge = np.full(10, 3e38, dtype=np.float32)
    shot = fd.Shot(spec.interior, spec.space_order, inputs.H, dt, spec.nbl)
    shot.set_model(spec.m)
    shot.inject(10, 10, 10, huge)
    shot.forward(30)
    with pytest.raises(fd.FdError) as e:
        shot.wavefield(0)
    assert e.value.code == fd.FD_ENONFINITE
    shot.reset()
    shot.synchronize()  # status cleared by reset
    shot.close()


# ---- 16-bit storage ------------------------------------------------------------
# 16-bit storage keeps u^n and the increment d^n, each rounded once per step to
# at most one half-ulp of the format (bf16: 2^-9, fp16 with a per-level
# power-of-two scale that keeps values in the normal range: 2^-12). The
# increment carries the velocity at full relative precision, so rounding only
# adds a random walk to u: the relative L2 error stays within a small multiple
# of half-ulp * sqrt(n). The tolerances below are about twice the largest
# errors measured over every order and shape of these tests after 60 steps
# (GB300: bf16 6.8e-3 at space order 2, fp16 8.7e-4), inside 4 half-ulp sqrt(60)
# (bf16 6.1e-2, fp16 7.6e-3).
STORAGE_TOL = {"bf16": 1.4e-2, "f16": 1.8e-3}


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("k", [2, 4, 8, 12, 16, 20, 24])
def test_16bit_storage_ragged(oracle_mod, k, storage):
    spec = _ragged_spec(k, seed=11)
    dt = dt_for(spec)
    eta = eta_for(spec)
    want, want_prev = run_oracle(oracle_mod, spec, spec.nt, dt, eta)
    shape = dict(zip(("tile_z", "tile_y"), [(32, 16), (64, 8)][k % 4 // 2]), x_block=13)
    got, got_prev, shot = run_gpu(spec, spec.nt, dt, None, storage=storage, **shape)
    e0, e1 = rel_l2(got, want), rel_l2(got_prev, want_prev)
    report(f"ragged_so{k}_{storage}{shot.config}", e0, e1)
    assert e0 <= STORAGE_TOL[storage] and e1 <= STORAGE_TOL[storage]
    shot.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_16bit_resume_and_chunks(oracle_mod, storage):
    """Loaded state (per-level scales picked from max|u|), chunked forwards."""
    rng = np.random.default_rng(13)
    spec = _ragged_spec(8, seed=13)
    dt = dt_for(spec)
    eta = eta_for(spec)
    u0 = inputs._gaussian_smooth(rng.standard_normal(spec.shape), 2.0).astype(np.float32) * 1e-3
    u1 = (0.99 * u0).astype(np.float32)
    state = (u0, u1, 3)
    want, _ = run_oracle(oracle_mod, spec, 40, dt, eta, state=state)
    got, _, shot = run_gpu(spec, 40, dt, None, state=state, chunks=[7, 33], storage=storage)
    e = rel_l2(got, want)
    report(f"resume_so8_{storage}{shot.config}", e)
    assert e <= STORAGE_TOL[storage]
    shot.close()


def test_precision_error_report(oracle_mod):
    """The precision workload shape (space order 12, 4-layer model, 20-cell
    layer, 1000 steps) on a 96^3 interior where the FP64 oracle finishes in
    seconds: every 100 steps, the L2 error on the 64^3 crop around the source
    relative to the largest crop norm the oracle reaches, and the discrete
    energy E^{n+1/2} error relative to the largest oracle energy (the wave
    leaves through the absorbing layer, so errors relative to the current,
    decaying values would grow even for a constant noise floor), for FP32, BF16
    and FP16 storage. Bounds about twice the measured worst crop errors
    (GB300: FP32 1.6e-6, FP16 2.3e-3, BF16 1.76e-2): FP32 3.5e-6, FP16 5e-3,
    BF16 3.6e-2."""
    spec = inputs.precision_shot(n=96, nbl=20, nt=1000)
    dt = dt_for(spec)
    eta = eta_for(spec)
    m64 = spec.m.astype(np.float64)
    k = spec.space_order
    wav = inputs.ricker(spec.f0, dt, spec.nt)
    src = [tuple(c + spec.nbl for c in spec.source)]
    c = [s + spec.nbl for s in spec.source]
    crop = tuple(slice(max(ci - 32, 0), max(ci - 32, 0) + 64) for ci in c)
    shots = {st: fd.Shot(spec.interior, k, inputs.H, dt, spec.nbl, storage=st)
             for st in ("f32", "bf16", "f16")}
    for shot in shots.values():
        shot.set_model(spec.m, eta)
        shot.inject(*spec.source, wav)
    u = up = None
    rows = []
    for chunk in range(10):
        u, up = oracle_mod.forward(m64, eta.astype(np.float64), k, inputs.H, dt, 100, src,
                                   wav.astype(np.float64)[None, :], u0=u, u_prev0=up,
                                   step0=100 * chunk)
        e_ref = oracle_mod.energy(u, up, m64, k, inputs.H, dt)
        for st, shot in shots.items():
            shot.forward(100)
            g0, g1 = shot.wavefield(0), shot.wavefield(1)
            d_crop = float(np.linalg.norm(g0[crop].astype(np.float64) - u[crop]))
            d_en = abs(oracle_mod.energy(g0, g1, m64, k, inputs.H, dt) - e_ref)
            rows.append((100 * (chunk + 1), st, d_crop, float(np.linalg.norm(u[crop])), d_en, abs(e_ref)))
    for shot in shots.values():
        shot.close()
    peak_crop = max(r[3] for r in rows)
    peak_en = max(r[5] for r in rows)
    worst = {}
    for step, st, d_crop, n_crop, d_en, e in rows:
        ec, ee = d_crop / peak_crop, d_en / peak_en
        worst[st] = max(worst.get(st, 0.0), ec)
        print(f"PRECISION step {step} {st} crop_err_vs_peak {ec:.3e} energy_err_vs_peak {ee:.3e} "
              f"crop_rel_now {d_crop / n_crop:.3e}")
    assert worst["f32"] <= 3.5e-6
    assert worst["f16"] <= 5e-3
    assert worst["bf16"] <= 3.6e-2
