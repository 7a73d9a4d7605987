"""GPU tests of off-grid sources and receivers (trilinear spreading and
sampling): traces and wavefields against the FP64 oracle on ragged grids for
every storage, on-node positions equal to the integer-node path bit for bit,
chunking invariance of the recorded traces, the nt_max cap, reset/load-state
restarts and the error codes."""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2

pytestmark = pytest.mark.gpu

H = inputs.H
# 16-bit storage: the same bounds as the wavefield parity of the ragged tests
# (4 half-ulp sqrt(steps)); traces are point samples of the same fields
STORAGE_TOL = {"f32": 1e-5, "bf16": 4 * 2.0 ** -9 * 60 ** 0.5, "f16": 4 * 2.0 ** -12 * 60 ** 0.5}


def _spec(k, seed):
    rng = np.random.default_rng(seed + 100 * k)
    interior = (37, 45, 51)
    nbl = 6
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=4.0)
    return inputs.ShotSpec(interior, nbl, k, vel, (0, 0, 0), 25.0, 60), rng


def _receivers(rng, interior, n=60):
    hi = np.array(interior, dtype=np.float64) - 1
    pts = rng.uniform(0, 1, (n, 3)) * hi
    edges = np.array([[0, 0, 0], hi, [hi[0], 0.5, hi[2]], [0, hi[1], 7.25], [3.0, 4.0, 5.0],
                      [hi[0], hi[1], 0.0]])
    return np.vstack([pts, edges])


def _oracle_traces(oracle_mod, spec, dt, eta, srcs, recs, nt):
    nbl = spec.nbl
    wav = np.array([np.asarray(w, dtype=np.float32).astype(np.float64) for _, w in srcs])
    s_dom = [tuple(c + nbl for c in p) for p, _ in srcs]
    r_dom = [tuple(c + nbl for c in p) for p in recs]
    return oracle_mod.forward_offgrid(spec.m.astype(np.float64), eta.astype(np.float64), spec.space_order, H,
                                      dt, nt, s_dom, wav, r_dom)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("k", [4, 8, 16])
def test_offgrid_traces_match_oracle(oracle_mod, k, storage):
    spec, rng = _spec(k, seed=1)
    dt = dt_for(spec)
    eta = eta_for(spec)
    nt = spec.nt
    srcs = [((18.3, 22.7, 9.45), inputs.ricker(25.0, dt, nt)),
            ((2.5, 40.0, 44.125), inputs.ricker(18.0, dt, nt))]
    recs = _receivers(rng, spec.interior)
    u_want, _, tr_want = _oracle_traces(oracle_mod, spec, dt, eta, srcs, recs, nt)
    with fd.Shot(spec.interior, k, H, dt, spec.nbl, storage=storage) as shot:
        shot.set_model(spec.m, eta)
        for p, w in srcs:
            shot.inject_at(*p, w)
        shot.set_receivers(recs, nt)
        shot.forward(nt)
        tr = shot.traces()
        u = shot.wavefield(0)
    assert tr.shape == (len(recs), nt)
    e_tr, e_u = rel_l2(tr, tr_want), rel_l2(u, u_want)
    print(f"PARITY offgrid_so{k}_{storage} traces {e_tr:.3e} field {e_u:.3e}")
    assert e_tr <= STORAGE_TOL[storage] and e_u <= STORAGE_TOL[storage]


def test_on_node_points_equal_integer_path():
    """A source and receivers placed exactly on nodes reproduce fd_inject and
    the wavefield values bit for bit (one corner weight 1, the others 0)."""
    spec, rng = _spec(8, seed=2)
    dt = dt_for(spec)
    wav = inputs.ricker(25.0, dt, spec.nt)
    nodes = [(5, 9, 11), (36, 44, 50), (0, 0, 0), (20, 3, 47)]
    with fd.Shot(spec.interior, 8, H, dt, spec.nbl) as a, fd.Shot(spec.interior, 8, H, dt, spec.nbl) as b:
        for s in (a, b):
            s.set_model(spec.m)
        a.inject(17, 21, 30, wav)
        b.inject_at(17.0, 21.0, 30.0, wav)
        b.set_receivers(np.array(nodes, dtype=np.float64), 40)
        a.forward(40)
        b.forward(40)
        ua = a.wavefield(0)
        np.testing.assert_array_equal(ua, b.wavefield(0))
        tr = b.traces()
        n = spec.nbl
        np.testing.assert_array_equal(tr[:, -1], [ua[x + n, y + n, z + n] for x, y, z in nodes])


def test_traces_chunks_cap_reset_and_resume():
    spec, rng = _spec(4, seed=3)
    dt = dt_for(spec)
    recs = _receivers(rng, spec.interior, n=10)
    wav = inputs.ricker(25.0, dt, spec.nt)

    def run(chunks, nt_max):
        with fd.Shot(spec.interior, 4, H, dt, spec.nbl) as s:
            s.set_model(spec.m)
            s.inject_at(10.2, 11.9, 30.5, wav)
            s.set_receivers(recs, nt_max)
            for c in chunks:
                s.forward(c)
            return s.traces()

    full = run([60], 60)
    np.testing.assert_array_equal(run([13, 1, 46], 60), full)
    capped = run([60], 25)
    assert capped.shape == (len(recs), 25)
    np.testing.assert_array_equal(capped, full[:, :25])
    with fd.Shot(spec.interior, 4, H, dt, spec.nbl) as s:
        s.set_model(spec.m)
        s.inject_at(10.2, 11.9, 30.5, wav)
        s.set_receivers(recs, 60)
        s.forward(30)
        s.reset()  # traces restart at step 0
        s.forward(60)
        np.testing.assert_array_equal(s.traces(), full)
        # a loaded state restarts the traces at the loaded step
        u, up = s.wavefield(0), s.wavefield(1)
        s.load_state(u, up, 60)
        assert s.traces().shape == (len(recs), 0)
        s.forward(5)
        assert s.traces().shape == (len(recs), 5)


def test_receiver_errors():
    spec, _ = _spec(4, seed=4)
    dt = dt_for(spec)
    with fd.Shot(spec.interior, 4, H, dt, spec.nbl) as s:
        s.set_model(spec.m)
        with pytest.raises(fd.FdError) as e:
            fd.fd_read_traces(s.handle, np.zeros(1, np.float32))
        assert e.value.code == fd.FD_ESTATE
        for bad in ([(-0.01, 1, 1)], [(1, 1, 50.5)], [(np.nan, 1, 1)]):
            with pytest.raises(fd.FdError) as e:
                s.set_receivers(bad, 10)
            assert e.value.code == fd.FD_ERANGE
        with pytest.raises(fd.FdError) as e:
            s.inject_at(36.5, 1, 1, np.ones(3, np.float32))
        assert e.value.code == fd.FD_ERANGE
        with pytest.raises(fd.FdError) as e:
            s.set_receivers([(1, 1, 1)], 0)
        assert e.value.code == fd.FD_EINVAL
        s.set_receivers([(1, 1, 1)], 5)
        s.set_receivers(np.zeros((0, 3)), 5)  # removes them
        with pytest.raises(fd.FdError) as e:
            fd.fd_read_traces(s.handle, np.zeros(5, np.float32))
        assert e.value.code == fd.FD_ESTATE
