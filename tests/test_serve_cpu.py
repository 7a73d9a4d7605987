"""Host-side checks of the serving loop's policy with a fake batch (no GPU):
admission by memory budget, FIFO order, chunks that never overshoot a shot,
slots and memory returned on completion."""
import numpy as np

from paper_1912_00695_gb300.serve import Request, Server


class _Done:
    """A completion handle that is ready at once (the fake batch is synchronous)."""

    def __init__(self, value):
        self.value = value

    def ready(self):
        return True

    def result(self):
        return self.value

    def wait(self):
        pass


class FakeBatch:
    def __init__(self, k, h, storage):
        self.steps = {}
        self.shapes = {}
        self.next = 0
        self.forwards = []

    def add(self, interior, nbl, dt, m):
        s = self.next
        self.next += 1
        self.steps[s] = 0
        self.shapes[s] = interior
        return s

    def inject(self, slot, *args):
        pass

    def forward(self, n):
        self.forwards.append(n)
        for s in self.steps:
            self.steps[s] += n

    def synchronize(self):
        pass

    def read_async(self, slot):
        return _Done(np.full(3, float(self.steps[slot])))

    def mark(self):
        return _Done(None)

    def remove(self, slot):
        del self.steps[slot]

    def close(self):
        pass


def _req(rid, nt, arrival=0.0, k=8, storage="f32", size=1):
    r = Request(rid, arrival, (4, 4, 4), 1, k, storage, 1e-3, None, (0, 0, 0), None, nt)
    r.size = size
    return r


def test_admission_budget_fifo_and_exact_steps():
    reqs = [_req(0, 30, size=2), _req(1, 70, size=2), _req(2, 10, size=3), _req(3, 55, size=1),
            _req(4, 20, k=16, size=1)]
    srv = Server(10.0, budget_bytes=5, chunk=25, batch_factory=FakeBatch,
                 bytes_fn=lambda r: r.size)
    stats = srv.run(reqs, realtime=False)
    assert stats["requests"] == 5
    assert srv.peak_used <= 5 and srv.used == 0 and not srv.active and not srv.reads
    for r in reqs:
        assert r.result[0] == r.nt  # every shot took exactly its steps
        assert r.completed >= r.admitted >= 0
    # FIFO: request 2 (size 3) had to wait for memory, request 3 was not admitted before it
    assert reqs[2].admitted >= reqs[0].admitted
    assert reqs[3].admitted >= reqs[2].admitted
    # two classes (k=8, k=16) got their own batches
    assert set(srv.classes) == {(8, "f32"), (16, "f32")}
    for b in srv.classes.values():
        assert all(0 < n <= 25 for n in b.forwards)


def test_realtime_arrivals_wait():
    reqs = [_req(0, 10, arrival=0.0), _req(1, 10, arrival=0.05)]
    srv = Server(10.0, budget_bytes=10, chunk=5, batch_factory=FakeBatch, bytes_fn=lambda r: 1)
    stats = srv.run(reqs, realtime=True)
    assert stats["requests"] == 2
    assert reqs[1].admitted >= 0.05
    assert stats["p99_s"] >= stats["p50_s"] >= 0
