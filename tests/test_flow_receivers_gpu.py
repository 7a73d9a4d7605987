"""GPU tests of receivers and of sources beyond the four fused ones on the FP32
flow schedule: each work item samples its input level at the receivers whose
lower trilinear corner lies in its region and adds the extra sources of its
region after its stores. The traces and both wavefield levels are bit for bit
those of the per-step launches (the TMA kernel's own sampling and the
extra-source kernel), for several space orders, both forms, launch shapes and
x-blocks, receivers on region edges and at the grid's last nodes, sources that
share nodes, chunked calls, a trace cap shorter than the run, and the FP64
oracle within the FP32 bound."""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2, run_oracle

pytestmark = pytest.mark.gpu
H = inputs.H


def _spec(k, seed, interior=(47, 39, 66), nbl=6, nt=36):
    rng = np.random.default_rng(seed)
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=4.0)
    return inputs.ShotSpec(interior, nbl, k, vel, (0, 0, 0), 25.0, nt)


def _receivers(interior, nbl, tz, ty, xb, seed):
    """Random interior points plus points whose lower corner sits on the last
    node before a region edge (x-chunk, y tile, z tile) and at the grid's end."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = interior
    pts = [rng.uniform(0, [nx - 1, ny - 1, nz - 1]) for _ in range(40)]
    for e in range(1, 4):
        # computational node c = interior + nbl: put c = e * tile - 1 + fraction
        cx, cy, cz = e * xb - 1 - nbl, e * ty - 1 - nbl, e * tz - 1 - nbl
        pts.append((min(max(cx + 0.5, 0), nx - 1), min(max(cy + 0.25, 0), ny - 1), min(max(cz + 0.75, 0), nz - 1)))
    pts += [(nx - 1, ny - 1, nz - 1), (0, 0, 0), (nx - 1.0, 0.5, nz - 1.5)]
    return np.array(pts, dtype=np.float64)


def _sources(interior, n=11):
    nx, ny, nz = interior
    s = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx // 2, ny // 2, nz // 2), (3, ny - 2, 9)]
    s += [(nx // 2, ny // 2, nz // 2), (1, 1, 1), (nx - 1, 0, nz // 3), (nx // 3, ny // 4, nz - 1),
          (1, 1, 1), (nx // 5, ny - 1, 17), (11, 13, 15)]
    return s[:n]


def _run(spec, eta, recs, srcs, chunks, flow, nt_max=None, **opts):
    dt = dt_for(spec)
    with fd.Shot(spec.interior, spec.space_order, H, dt, spec.nbl, kernel="tma", **opts) as shot:
        shot.set_model(spec.m, eta)
        for i, s in enumerate(srcs):
            shot.inject(*s, inputs.ricker(18.0 + 2 * i, dt, spec.nt) * (1.0 + 0.1 * i))
        if recs is not None:
            shot.set_receivers(recs, nt_max or spec.nt)
        for n in chunks:
            (shot.forward_flow if flow else shot.forward)(n)
        tr = shot.traces() if recs is not None else None
        return shot.wavefield(0), shot.wavefield(1), tr


CASES = [
    (4, "factored", 32, 16, 1, 9), (4, "expanded", 64, 8, 1, 5),
    (8, "factored", 32, 32, 2, 8), (8, "expanded", 32, 16, 1, 13),
    (12, "factored", 32, 16, 1, 6), (16, "factored", 64, 8, 1, 30), (16, "expanded", 32, 16, 1, 8),
]


@pytest.mark.parametrize("k,form,tz,ty,rows,xb", CASES)
def test_flow_receivers_and_sources_equal_per_step(k, form, tz, ty, rows, xb):
    spec = _spec(k, seed=300 + k + tz)
    eta = eta_for(spec)
    recs = _receivers(spec.interior, spec.nbl, tz, ty, xb, seed=k)
    srcs = _sources(spec.interior)
    opts = dict(form=form, tile_z=tz, tile_y=ty, rows=rows, x_block=xb)
    want = _run(spec, eta, recs, srcs, [spec.nt], False, **opts)
    assert np.abs(want[2]).max() > 0
    for chunks in ([spec.nt], [1, 14, spec.nt - 15]):
        got = _run(spec, eta, recs, srcs, chunks, True, **opts)
        np.testing.assert_array_equal(got[2], want[2])
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])


def test_flow_receivers_only_and_sources_only():
    k, tz, ty, xb = 8, 32, 16, 10
    spec = _spec(k, seed=41)
    eta = eta_for(spec)
    recs = _receivers(spec.interior, spec.nbl, tz, ty, xb, seed=3)
    opts = dict(tile_z=tz, tile_y=ty, x_block=xb)
    few = _sources(spec.interior, n=2)
    want = _run(spec, eta, recs, few, [spec.nt], False, **opts)
    got = _run(spec, eta, recs, few, [7, spec.nt - 7], True, **opts)
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)
    many = _sources(spec.interior, n=9)
    want = _run(spec, eta, None, many, [spec.nt], False, **opts)
    got = _run(spec, eta, None, many, [spec.nt], True, **opts)
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])


def test_flow_trace_cap_shorter_than_run():
    """nt_max below the steps run: samples past the cap are dropped by both."""
    k, tz, ty, xb = 4, 32, 16, 12
    spec = _spec(k, seed=7)
    eta = eta_for(spec)
    recs = _receivers(spec.interior, spec.nbl, tz, ty, xb, seed=5)
    srcs = _sources(spec.interior, n=6)
    opts = dict(tile_z=tz, tile_y=ty, x_block=xb)
    want = _run(spec, eta, recs, srcs, [spec.nt], False, nt_max=13, **opts)
    got = _run(spec, eta, recs, srcs, [5, spec.nt - 5], True, nt_max=13, **opts)
    assert got[2].shape == (len(recs), 13)
    np.testing.assert_array_equal(got[2], want[2])
    np.testing.assert_array_equal(got[0], want[0])


def test_flow_receivers_match_oracle(oracle_mod):
    """The automatic schedule with receivers and six sources against the FP64
    oracle (fields; the traces are point samples of the same fields)."""
    k = 8
    spec = _spec(k, seed=12, interior=(40, 35, 44), nbl=6, nt=30)
    dt = dt_for(spec)
    eta = eta_for(spec)
    nodes = [(20, 9, 1), (0, 0, 0), (39, 34, 43), (12, 21, 30), (5, 5, 5), (30, 2, 40)]
    srcs = [(s, inputs.ricker(20.0 + 3 * i, dt, spec.nt)) for i, s in enumerate(nodes)]
    want, want_prev = run_oracle(oracle_mod, spec, spec.nt, dt, eta, sources=srcs)
    with fd.Shot(spec.interior, k, H, dt, spec.nbl) as shot:
        shot.set_model(spec.m, eta)
        for s, w in srcs:
            shot.inject(*s, w)
        shot.set_receivers(np.array(nodes, dtype=np.float64), spec.nt)
        shot.forward_flow(spec.nt)
        u = shot.wavefield(0)
        e0, e1 = rel_l2(u, want), rel_l2(shot.wavefield(1), want_prev)
        tr = shot.traces()
    print(f"PARITY flow_receivers_so{k} {e0:.3e} {e1:.3e}")
    assert e0 <= 1e-5 and e1 <= 1e-5
    # receivers on nodes (weights 1 and 0): the last sample is the final field at
    # the node, exactly that of the GPU and within the bound that of the oracle
    b = spec.nbl
    assert tr.shape == (len(nodes), spec.nt)
    np.testing.assert_array_equal(tr[:, -1], np.array([u[x + b, y + b, z + b] for x, y, z in nodes]))
    assert rel_l2(tr[:, -1], np.array([want[x + b, y + b, z + b] for x, y, z in nodes])) <= 1e-4
