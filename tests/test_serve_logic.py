"""Host logic of the continuous-batching driver, on CPU with a fake runtime:
FIFO admission as slots free up, rejection after the admission deadline,
latency bookkeeping and overlap accounting."""
import paper_2502_04189_b300.serve as S


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001  # every look at the clock advances 1 ms
        return self.t


class FakeServer:
    """slots slots; a launched request finishes `service` seconds later."""

    def __init__(self, clock, slots=2, service=0.02, budget_cells=10 ** 9):
        self.clock, self.n, self.service = clock, slots, service
        self.busy = {}
        self.budget_cells = budget_cells
        self.used = 0
        self.admit_calls = 0

    def admit(self, **d):
        self.admit_calls += 1
        cells = d["nx"] * d["ny"] * d["nz"]
        free = [s for s in range(self.n) if s not in self.busy]
        if not free:
            return -7, -1, None
        if self.used + cells > self.budget_cells:
            return -3, -1, None
        s = free[0]
        self.busy[s] = [None, cells]
        self.used += cells
        return 0, s, [0] * 7

    def stream(self, slot):
        return None

    def launch(self, slot):
        self.busy[slot][0] = self.clock.t + self.service

    def poll(self):
        return [s for s, (t, _) in self.busy.items() if t is not None and t <= self.clock.t]

    def stats(self, slot):
        return {"converged": 1, "relres": 1e-12}

    def release(self, slot):
        self.used -= self.busy.pop(slot)[1]


def reqs(times, size=8):
    return [S.Request(i, t, dict(nx=size, ny=size, nz=size)) for i, t in enumerate(times)]


def test_all_admitted_when_capacity_suffices():
    clk = FakeClock()
    srv = FakeServer(clk, slots=4, service=0.005)
    out, summ = S.run(srv, reqs([0.01 * i for i in range(20)]), fill=lambda r, v, s: None,
                      view_fn=lambda p, sh: None, clock=clk)
    assert summ["admitted"] == 20 and summ["rejected"] == 0
    assert all(o.latency >= 0.005 for o in out)


def test_overload_rejects_after_deadline_and_overlaps():
    clk = FakeClock()
    srv = FakeServer(clk, slots=2, service=0.05)
    out, summ = S.run(srv, reqs([0.0] * 30), fill=lambda r, v, s: None,
                      view_fn=lambda p, sh: None, clock=clk, deadline=0.1)
    assert summ["max_inflight"] == 2
    assert 0 < summ["admitted"] < 30
    assert summ["rejected"] == 30 - summ["admitted"]
    # FIFO: the admitted requests are the earliest in the queue
    adm = [o.index for o in out if o.admitted]
    assert adm == list(range(len(adm)))
    assert all(o.latency <= 0.1 + 0.05 + 0.02 for o in out if o.admitted)


def test_budget_refusal_waits_then_rejects():
    clk = FakeClock()
    srv = FakeServer(clk, slots=4, service=0.03, budget_cells=600)
    out, summ = S.run(srv, reqs([0.0, 0.0, 0.0, 0.0], size=8), fill=lambda r, v, s: None,
                      view_fn=lambda p, sh: None, clock=clk, deadline=0.05)
    # 512 cells each: only one fits the 600-cell budget at a time
    assert summ["max_inflight"] == 1
    assert summ["admitted"] >= 2 and summ["rejected"] >= 1
