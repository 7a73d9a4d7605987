"""GPU tests of the slab decomposition (one shot split along x, r ghost planes
per neighbour exchanged every step; the paper's ops_partition, Sec. 3 item
(vii), and Devito's halo exchange, Sec. 5): two and three slabs on one GPU,
driven from one process (SlabGroup: boundary part, device copies of the
halos on a second stream, interior part), equal the undivided shot's
fd_forward bit for bit for every space order and both stencil forms, match
the FP64 oracle, and hold at the benchmark's 276^3 size; two processes
(one slab each, HaloDriver over gloo with host staging) on the same GPU do
the same; the unsupported uses are rejected."""
import os
import socket
import sys

import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import _abi, inputs
from paper_1912_00695_gb300.slabs import SlabGroup, partition
from harness import dt_for, eta_for, rel_l2, run_oracle

pytestmark = pytest.mark.gpu
H = inputs.H
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _spec(k, seed, interior=(43, 29, 45), nbl=6, nt=30):
    rng = np.random.default_rng(seed)
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=4.0)
    return inputs.ShotSpec(interior, nbl, k, vel, (0, 0, 0), 25.0, nt)


# interior nodes: the first plane, slab edges of a 2- and 3-way split, the last plane
SOURCES = [(0, 3, 7), (18, 14, 22), (24, 1, 44), (42, 28, 0)]


def _whole(spec, eta, nt, form):
    dt = dt_for(spec)
    with fd.Shot(spec.interior, spec.space_order, H, dt, spec.nbl, form=form) as shot:
        shot.set_model(spec.m, eta)
        for i, s in enumerate(SOURCES):
            shot.inject(*s, inputs.ricker(20.0 + 2 * i, dt, nt))
        shot.forward(nt)
        return shot.wavefield(0), shot.wavefield(1)


def _slabs(spec, eta, nt, form, parts, chunks=None):
    dt = dt_for(spec)
    with SlabGroup(spec.interior, spec.space_order, H, dt, spec.nbl, parts, form=form) as g:
        g.set_model(spec.m, eta)
        for i, s in enumerate(SOURCES):
            g.inject(*s, inputs.ricker(20.0 + 2 * i, dt, nt))
        for n in (chunks or [nt]):
            g.forward(n)
        assert g.step == nt
        return g.wavefield(0), g.wavefield(1)


@pytest.mark.parametrize("form", ["factored", "expanded"])
@pytest.mark.parametrize("k", [2, 4, 8, 12, 16])
def test_slabs_equal_whole_shot(k, form):
    spec = _spec(k, seed=k)
    eta = eta_for(spec)
    want = _whole(spec, eta, spec.nt, form)
    for parts in (2, 3):
        got = _slabs(spec, eta, spec.nt, form, parts, chunks=[7, spec.nt - 7])
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])


def test_slabs_match_oracle(oracle_mod):
    k = 8
    spec = _spec(k, seed=40)
    dt = dt_for(spec)
    eta = eta_for(spec)
    srcs = [(s, inputs.ricker(20.0 + 2 * i, dt, spec.nt)) for i, s in enumerate(SOURCES)]
    want, want_prev = run_oracle(oracle_mod, spec, spec.nt, dt, eta, sources=srcs)
    got, got_prev = _slabs(spec, eta, spec.nt, "factored", 3)
    e0, e1 = rel_l2(got, want), rel_l2(got_prev, want_prev)
    print(f"PARITY slabs3_so{k} {e0:.3e} {e1:.3e}")
    assert e0 <= 1e-5 and e1 <= 1e-5


def test_slabs_full_size():
    """The 276^3 sweep shot (space order 8) in two slabs, 20 steps: equal to the
    undivided shot bit for bit."""
    spec = inputs.sweep_shot(8, nt=20)
    dt = dt_for(spec)
    eta = fd.fd_default_damping(spec.m, spec.nbl, H)
    wav = inputs.ricker(spec.f0, dt, spec.nt)
    with fd.Shot(spec.interior, 8, H, dt, spec.nbl) as shot:
        shot.set_model(spec.m, eta)
        shot.inject(*spec.source, wav)
        shot.forward(spec.nt)
        want = shot.wavefield(0)
    with SlabGroup(spec.interior, 8, H, dt, spec.nbl, 2) as g:
        g.set_model(spec.m, eta)
        g.inject(*spec.source, wav)
        g.forward(spec.nt)
        got = g.wavefield(0)
    assert np.abs(want).max() > 0
    np.testing.assert_array_equal(got, want)


def test_slab_rejections():
    spec = _spec(8, seed=2)
    dt = dt_for(spec)
    nx, ny, nz = spec.interior
    N = spec.shape[0]
    hd = _abi.fd_slab_create(nx, ny, nz, 8, H, dt, spec.nbl, 0, 20)
    try:
        assert _abi.fd_slab_info(hd) == (0, 20, 0, 4)
        m = np.ascontiguousarray(spec.m[:24])
        with pytest.raises(fd.FdError) as e:
            _abi.fd_set_model(hd, m, None)  # slabs need an explicit eta
        assert e.value.code == fd.FD_EINVAL
        _abi.fd_set_model(hd, m, np.zeros_like(m))
        for call in (lambda: _abi.fd_forward(hd, 1), lambda: _abi.fd_forward_flow(hd, 1),
                     lambda: _abi.fd_set_receivers(hd, [(1.0, 1.0, 1.0)], 4)):
            with pytest.raises(fd.FdError) as e:
                call()
            assert e.value.code == fd.FD_ENOTSUP
    finally:
        _abi.fd_destroy(hd)
    for x0, x1 in ((0, 3), (N - 2, N), (5, N + 1)):  # fewer than k/2 planes, or past the domain
        with pytest.raises(fd.FdError) as e:
            _abi.fd_slab_create(nx, ny, nz, 8, H, dt, spec.nbl, x0, x1)
        assert e.value.code == fd.FD_EINVAL
    with pytest.raises(fd.FdError) as e:
        _abi.fd_slab_create(nx, ny, nz, 8, H, dt, spec.nbl, 0, 20, fd.options(storage="bf16"))
    assert e.value.code == fd.FD_ENOTSUP
    assert partition(N, 3, 4)[0][0] == 0


def _rank_worker(rank, world, port, k, nt, q):
    """One slab per process on GPU 0: HaloDriver over gloo, host-staged halos."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    try:
        import torch
        import torch.distributed as tdist

        import paper_1912_00695_gb300 as fd_
        from paper_1912_00695_gb300 import inputs as inp
        from paper_1912_00695_gb300.slabs import GpuSlab, HaloDriver, HostStage, partition as part
        torch.cuda.set_device(0)
        tdist.init_process_group("gloo", rank=rank, world_size=world)
        spec = _spec(k, seed=77)
        dt = 0.9 * fd_.fd_dt_max(k, H, spec.vmax)
        eta = fd_.fd_default_damping(spec.m, spec.nbl, H)
        ranges = part(spec.shape[0], world, k // 2)
        slab = GpuSlab(spec.interior, k, H, dt, spec.nbl, ranges, rank)
        slab.set_model(spec.m, eta)
        for i, s in enumerate(SOURCES):
            slab.inject(*s, inp.ricker(20.0 + 2 * i, dt, nt))
        HaloDriver(slab, stage=HostStage()).forward(nt)
        torch.cuda.synchronize()
        own = torch.from_numpy(np.ascontiguousarray(slab.own_planes(0)))
        if rank == 0:
            parts = [own] + [torch.empty((b - a,) + spec.shape[1:], dtype=torch.float32) for a, b in ranges[1:]]
            for src in range(1, world):
                tdist.recv(parts[src], src)
            q.put(("ok", np.concatenate([p.numpy() for p in parts])))
        else:
            tdist.send(own, 0)
        tdist.barrier()
        slab.close()
        tdist.destroy_process_group()
    except Exception as e:
        q.put(("error", repr(e)))
        raise


def test_halo_driver_two_processes_one_gpu():
    torch = pytest.importorskip("torch")
    k, nt = 8, 24
    spec = _spec(k, seed=77)
    dt = 0.9 * fd.fd_dt_max(k, H, spec.vmax)
    eta = fd.fd_default_damping(spec.m, spec.nbl, H)
    with fd.Shot(spec.interior, k, H, dt, spec.nbl) as shot:
        shot.set_model(spec.m, eta)
        for i, s in enumerate(SOURCES):
            shot.inject(*s, inputs.ricker(20.0 + 2 * i, dt, nt))
        shot.forward(nt)
        want = shot.wavefield(0)
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_rank_worker, args=(r, 2, port, k, nt, q)) for r in range(2)]
    for p in procs:
        p.start()
    kind, got = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
    assert kind == "ok", got
    np.testing.assert_array_equal(got, want)
