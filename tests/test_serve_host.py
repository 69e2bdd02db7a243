"""Host logic of the serving loop (paper_2606_31061_b300.serve) on fake pools, no GPU:
admission by HBM budget, first-come-first-served waiting, slot reuse, FIFO frames and
masked steps (only streams with a frame take part)."""
from paper_2606_31061_b300 import serve


class _Ev:
    def query(self):
        return True


class FakePool:
    def __init__(self, dims, ranks, slots, nbytes=100):
        self.dims, self.ranks, self.slots, self.bytes = dims, ranks, slots, nbytes
        self.steps, self.resets = [], []

    def reset_slot(self, slot, sid, init=None):
        self.resets.append((slot, sid))

    def step(self, frames):
        self.steps.append(dict(frames))
        return _Ev()

    def close(self):
        pass


def _server(budget, slots=2):
    made = []

    def factory(d, r, n):
        p = FakePool(d, r, n)
        made.append(p)
        return p
    return serve.Server(budget, slots=slots, rank_step=16, pool_factory=factory), made


def test_rank_rounding_and_feasible_keys():
    assert serve.round_ranks((8, 17, 48), 16) == (16, 32, 48)
    assert serve.feasible_ranks((1080, 1920, 3), (32, 32, 3)) == (32, 9, 3)
    s, _ = _server(10**9)
    # every bond rounds up to a multiple of 16 (20, 30 -> 32), then the clamp applies:
    # r_2 <= I_3 r_3 = 3 x 16
    assert s.key((720, 1280, 3), (20, 10, 3)) == s.key((720, 1280, 3), (30, 16, 16)) == ((720, 1280, 3), (32, 16, 16))
    assert s.key((720, 1280, 3), (20, 60, 3)) == ((720, 1280, 3), (32, 48, 16))


def test_admission_by_budget_and_waiting():
    s, made = _server(250)                      # two pools of 100 bytes fit, a third does not
    a = [s.connect(i, (64, 64), (8, 8)) for i in range(5)]
    assert a == [True, True, True, True, False] and len(made) == 3     # the third was refused
    assert s.used == 200 and list(s.waiting) == [4]
    assert not s.connect(9, (32, 32), (8, 8))   # first come, first served: 9 queues behind 4
    s.disconnect(1)
    assert s.admitted(4) and not s.admitted(9) and list(s.waiting) == [9]
    pool, slot = s.where[4]
    assert (slot, 4) in pool.resets             # the reused slot was reset for the new stream
    s.disconnect(9)                             # leaving the queue
    assert not s.waiting


def test_ticks_are_masked_fifo_and_timed():
    s, made = _server(10**6)
    for i in range(3):
        assert s.connect(i, (64, 64), (8, 8))
    s.submit(0, "f0a", 0.0)
    s.submit(0, "f0b", 0.1)
    s.submit(2, "f2a", 0.05)
    assert s.tick() == 2                         # one frame per stream per step
    pool0, pool1 = made
    assert pool0.steps == [{0: "f0a"}] and pool1.steps == [{0: "f2a"}]
    assert s.poll(now=1.0) == 2
    assert sorted(s.latencies) == [0.95, 1.0]
    assert s.tick() == 1 and pool0.steps[-1] == {0: "f0b"}
    assert s.poll(now=2.0) == 1 and s.completed[0] == 2 and s.backlog() == 0
    assert s.tick() == 0
    p = serve.percentiles([3.0, 1.0, 2.0])
    assert p["p50"] == 2.0 and p["n"] == 3


def test_restart_streams_reseeds_and_clears():
    srv, made = _server(10_000, slots=2)
    assert srv.connect("a", (4, 4), (2, 2)) and srv.connect("b", (4, 4), (2, 2))
    srv.submit("a", "f0", 0.0)
    srv.tick()
    srv.poll(now=1.0)
    assert srv.latencies and srv.steps == 1
    n0 = len(made[0].resets)
    srv.restart_streams()
    assert srv.latencies == [] and srv.steps == 0 and not srv.completed
    assert sorted(made[0].resets[n0:]) == [(0, "a"), (1, "b")]
    assert srv.admitted("a") and srv.admitted("b")
