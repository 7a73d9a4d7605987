"""Host-side checks of the slab decomposition (one shot split along x with an
r-plane halo exchange per step; the paper's ops_partition, Sec. 3 item (vii),
and Devito's halo exchange, Sec. 5), without a GPU:

* the partition and the exchange plan (which planes go where);
* the per-rank schedule of HaloDriver over gloo ranks (world size 2 and 3),
  with each rank's slab advanced by the FP64 oracle on its planes plus ghost
  planes: after the exchange of every step the gathered slabs equal the
  undivided oracle run bit for bit (same arithmetic per point), and a
  planted mistake in the exchange (a ghost plane off by one) is caught.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1912_00695_gb300.slabs import (Transfer, exchange_plan, ghost_planes, partition,  # noqa: E402
                                          slab_window)


def test_partition_even_and_ragged():
    assert partition(10, 2, 2) == [(0, 5), (5, 10)]
    assert partition(11, 3, 3) == [(0, 4), (4, 8), (8, 11)]
    for n, p, r in [(276, 2, 8), (276, 3, 8), (57, 4, 6), (9, 1, 12)]:
        rg = partition(n, p, r)
        assert rg[0][0] == 0 and rg[-1][1] == n
        assert all(b - a >= min(r, n) for a, b in rg)
        assert all(a1 == b0 for (_, a1), (b0, _) in zip(rg, rg[1:]))
        sizes = [b - a for a, b in rg]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        partition(10, 4, 3)  # slabs of 2 or 3 planes cannot hold r = 3 ghosts from one neighbour


def test_exchange_plan_and_windows():
    rg = partition(20, 3, 2)
    plan = exchange_plan(rg)
    assert plan == [Transfer(0, 1, "up"), Transfer(1, 0, "down"), Transfer(1, 2, "up"), Transfer(2, 1, "down")]
    assert ghost_planes(rg, 0, 2, 20) == (0, 2)
    assert ghost_planes(rg, 1, 2, 20) == (2, 2)
    assert ghost_planes(rg, 2, 2, 20) == (2, 0)
    assert slab_window(rg, 1, 2, 20) == (rg[1][0] - 2, rg[1][1] + 2)
    with pytest.raises(ValueError):
        exchange_plan([(0, 5), (6, 10)])


class OracleSlab:
    """A HaloDriver stepper backed by the FP64 oracle: the slab's planes plus
    its ghost planes as a local domain; the boundary part computes the whole
    next level of that local domain (only the own planes are kept: their
    stencils reach at most r planes into the ghosts), the interior part
    rotates the levels. views() are torch tensors sharing the numpy memory."""

    def __init__(self, oracle, m, eta, k, h, dt, ranges, index, sources, wavelets, shift=0):
        self.oracle, self.k, self.h, self.dt = oracle, k, h, dt
        self.r = k // 2
        n = m.shape[0]
        self.w0, self.w1 = slab_window(ranges, index, self.r, n)
        self.x0, self.x1 = ranges[index]
        self.glo, self.ghi = ghost_planes(ranges, index, self.r, n)
        self.m = np.ascontiguousarray(m[self.w0:self.w1])
        self.eta = np.ascontiguousarray(eta[self.w0:self.w1])
        keep = [i for i, s in enumerate(sources) if self.x0 <= s[0] < self.x1]
        self.src = [(sources[i][0] - self.w0, sources[i][1], sources[i][2]) for i in keep]
        self.wav = wavelets[keep] if keep else None
        self.u = np.zeros(self.m.shape)
        self.up = np.zeros(self.m.shape)
        self.next = None
        self.n = 0
        self.shift = shift  # planted mistake: send planes shifted by this many planes

    def boundary(self):
        self.next, _ = self.oracle.forward(self.m, self.eta, self.k, self.h, self.dt, 1, self.src,
                                           self.wav, u0=self.u, u_prev0=self.up, step0=self.n)

    def interior(self):
        self.up, self.u = self.u, self.next
        self.n += 1

    def views(self, level):
        import torch
        assert level == 1
        a = torch.from_numpy(self.next)
        r, lo, hi = self.r, self.x0 - self.w0, self.x1 - self.w0
        s = self.shift
        send_lo = a[lo + s:lo + s + r] if self.glo else None
        send_hi = a[hi - r - s:hi - s] if self.ghi else None
        recv_lo = a[0:self.glo] if self.glo else None
        recv_hi = a[hi:hi + self.ghi] if self.ghi else None
        return send_lo, send_hi, recv_lo, recv_hi

    def own(self):
        return self.u[self.x0 - self.w0:self.x1 - self.w0]


def _problem(k):
    from paper_1912_00695_gb300 import inputs
    rng = np.random.default_rng(3 + k)
    interior, nbl = (17, 9, 11), 3
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=2.0)
    m = inputs.slowness2(vel).astype(np.float64)
    eta = (m * rng.uniform(0.0, 20.0, m.shape) * (rng.uniform(size=m.shape) < 0.4))
    sources = [(3, 4, 5), (11, 6, 2), (16, 1, 9)]  # domain nodes in several slabs
    wav = rng.standard_normal((len(sources), 30))
    return m, eta, sources, wav


def _worker(rank, world, port, k, nt, shift, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as tdist

    import oracle
    from paper_1912_00695_gb300.slabs import HaloDriver, partition
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, eta, sources, wav = _problem(k)
        h, dt = 10.0, 5e-4
        ranges = partition(m.shape[0], world, k // 2)
        slab = OracleSlab(oracle, m, eta, k, h, dt, ranges, rank, sources, wav, shift=shift)
        HaloDriver(slab).forward(nt)
        own = torch.from_numpy(np.ascontiguousarray(slab.own()))
        if rank == 0:
            parts = [own] + [torch.empty((b - a,) + m.shape[1:], dtype=torch.float64) for a, b in ranges[1:]]
            for src in range(1, world):
                tdist.recv(parts[src], src)
            q.put(("ok", np.concatenate([p.numpy() for p in parts])))
        else:
            tdist.send(own, 0)
        tdist.barrier()
    except Exception as e:  # report instead of hanging the parent
        q.put(("error", repr(e)))
        raise
    finally:
        tdist.destroy_process_group()


def _run(world, k, nt, shift=0):
    torch = pytest.importorskip("torch")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_worker, args=(r, world, port, k, nt, shift, q)) for r in range(world)]
    for p in procs:
        p.start()
    kind, got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
    assert kind == "ok", got
    return got


@pytest.mark.parametrize("world,k", [(2, 4), (3, 6), (2, 8)])
def test_halo_driver_gloo_equals_undivided_oracle(oracle_mod, world, k):
    nt = 12
    got = _run(world, k, nt)
    m, eta, sources, wav = _problem(k)
    want, _ = oracle_mod.forward(m, eta, k, 10.0, 5e-4, nt, sources, wav)
    assert np.abs(want).max() > 0
    np.testing.assert_array_equal(got, want)


def test_halo_driver_gloo_catches_shifted_ghosts(oracle_mod):
    """A planted mistake in the exchange (the planes sent shifted by one) is caught."""
    k, nt = 4, 12
    got = _run(2, k, nt, shift=1)
    m, eta, sources, wav = _problem(k)
    want, _ = oracle_mod.forward(m, eta, k, 10.0, 5e-4, nt, sources, wav)
    assert np.abs(got - want).max() > 1e-6 * np.abs(want).max()
