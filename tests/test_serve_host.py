"""Host logic of the request loop, against a fake engine with a virtual clock (CPU)."""
import numpy as np
import pytest

from paper_1507_07294_gb300 import serve as S


class FakeEngine:
    """Counts steps per run and charges virtual time: per time step, the stepped runs'
    cells / `rate` plus three launches of `launch` seconds (shared in a batch)."""

    def __init__(self, bytes_per_cell=236, rate=1e4, launch=1e-3, diverge_at=None):
        self.t = 0.0
        self.diverge_at = diverge_at or {}  # rid -> step count from which the run is NaN
        self.checked = {}
        self.bytes_per_cell = bytes_per_cell
        self.rate = rate
        self.launch = launch
        self.taken = {}
        self.first = {}
        self.open_runs = set()
        self.max_open = 0
        self.batches = []
        self.alone_chunks = [0]

    def clock(self):
        return self.t

    def sleep(self, dt):
        self.t += dt

    def footprint(self, r):
        return r.cells * self.bytes_per_cell

    def open(self, r):
        h = (r.rid, r.steps, r.cells)
        self.taken[h] = 0
        self.open_runs.add(h)
        self.max_open = max(self.max_open, len(self.open_runs))
        return h

    def step_alone(self, h, n):
        assert n >= 1
        if self.taken[h] == 0:
            self.first[h] = n
        else:
            self.alone_chunks.append(n)
        self.taken[h] += n
        self.t += n * (h[2] / self.rate + 3 * self.launch)

    def step_batch(self, hs, n):
        assert len(set(hs)) == len(hs)
        for h in hs:
            assert self.taken[h] >= 1, "a batched run must have taken its first step alone"
            self.taken[h] += n
        self.batches.append((len(hs), n))
        self.t += n * (sum(h[2] for h in hs) / self.rate + 3 * self.launch)

    def _bad(self, h):
        return self.taken[h] >= self.diverge_at.get(h[0], float("inf"))

    def check(self, h):
        self.checked[h] = self._bad(h)

    def diverged(self, h):
        return self.checked.get(h, False)

    def fence(self, hs):
        return list(hs)

    def wait(self, fence):
        for h in fence:
            assert h in self.open_runs

    def finish(self, h):
        self.open_runs.discard(h)
        return not self._bad(h), self.taken[h]


def _server(eng, **kw):
    return S.Server(eng, clock=eng.clock, sleep=eng.sleep, **kw)


def _reqs(n=40, seed=3, steps=(1, 300), gap=0.05):
    return S.request_stream(n, seed=seed, grids=((8, 8, 8), (16, 16, 16), (16, 16, 64)),
                            steps=steps, mean_interarrival=gap)


@pytest.mark.parametrize("batched", [True, False])
def test_every_request_finishes_with_exactly_its_steps(batched):
    eng = FakeEngine()
    reqs = _reqs()
    out = _server(eng, budget_bytes=10**9, max_runs=8, quantum=16, batched=batched).serve(reqs)
    assert sorted(o.rid for o in out) == [r.rid for r in reqs]
    by = {r.rid: r for r in reqs}
    for o in out:
        assert o.result == by[o.rid].steps
        assert o.arrival <= o.admitted <= o.finished
    if batched:
        # the first chunk aligns the rest to whole quanta
        for h, n in eng.first.items():
            assert 1 <= n <= 16 and (h[1] - n) % 16 == 0
        assert all(n == 16 for _, n in eng.batches)
    else:
        assert eng.max_open == 1 and not eng.batches
        assert all(n == 16 for n in eng.alone_chunks[1:])


def test_finished_runs_hold_their_slot_until_read():
    """The pipelined loop reads a run out one quantum after its last steps; until then it
    counts against the slots and the budget, so open runs never exceed max_runs."""
    eng = FakeEngine()
    reqs = _reqs(n=40, gap=0.0001, steps=(1, 40))
    srv = _server(eng, budget_bytes=10**9, max_runs=3, quantum=8)
    out = srv.serve(reqs)
    assert len(out) == 40 and eng.max_open <= 3 and srv.peak_runs <= 3


def test_diverged_runs_are_stopped_early():
    reqs = _reqs(n=20, gap=0.001, steps=(200, 400))
    diverge = {3: 40, 7: 1, 11: 150}
    eng = FakeEngine(diverge_at=diverge)
    srv = _server(eng, budget_bytes=10**9, max_runs=8, quantum=16, check_every=2)
    out = srv.serve(reqs)
    by = {r.rid: r for r in reqs}
    for o in out:
        if o.rid in diverge:
            assert not o.stable
            # found at the first check at or after the divergence; stopped one quantum
            # later at most (the next quantum is already queued when the check is read)
            assert diverge[o.rid] <= o.steps <= diverge[o.rid] + 16 + 2 * 2 * 16
            assert o.steps < by[o.rid].steps
            assert o.result == o.steps
        else:
            assert o.stable and o.steps == by[o.rid].steps == o.result
    assert srv.stopped == 3


def test_budget_and_slots_are_respected():
    eng = FakeEngine()
    reqs = _reqs(n=60, gap=0.001)
    big = 16 * 16 * 64 * eng.bytes_per_cell
    srv = _server(eng, budget_bytes=2 * big, max_runs=5, quantum=8)
    out = srv.serve(reqs)
    assert len(out) == 60
    assert srv.peak_bytes <= 2 * big
    assert srv.peak_runs <= 5 and eng.max_open <= 5
    assert srv.peak_runs >= 2  # runs did share the device


def test_admission_is_first_come_first_served():
    eng = FakeEngine()
    reqs = _reqs(n=50, gap=0.002)
    out = _server(eng, budget_bytes=10**9, max_runs=4, quantum=8).serve(reqs)
    adm = sorted(out, key=lambda o: (o.arrival, o.rid))
    assert all(a.admitted <= b.admitted for a, b in zip(adm, adm[1:]))


def test_request_larger_than_budget_is_refused():
    eng = FakeEngine()
    reqs = _reqs(n=3)
    with pytest.raises(ValueError, match="exceeds the memory budget"):
        _server(eng, budget_bytes=100, quantum=8).serve(reqs)


def test_idle_server_waits_for_arrivals():
    eng = FakeEngine()
    reqs = [S.Request(0, 5.0, (8, 8, 8), 100.0, 0.5, 1e-3, 10),
            S.Request(1, 50.0, (8, 8, 8), 100.0, 0.5, 1e-3, 10)]
    out = _server(eng, budget_bytes=10**9, quantum=4).serve(reqs)
    assert [o.admitted for o in out] == [5.0, 50.0]


def test_batching_beats_one_at_a_time_when_launches_dominate():
    """With a per-launch overhead and small runs, sharing launches raises throughput
    (the fake engine's cost model; the GPU numbers come from the bench)."""
    reqs = _reqs(n=60, gap=0.0005, steps=(50, 200))
    a = S.summarize(_server(FakeEngine(rate=1e7), budget_bytes=10**9, quantum=16).serve(reqs))
    b = S.summarize(_server(FakeEngine(rate=1e7), budget_bytes=10**9, batched=False).serve(reqs))
    assert a["mlups"] > 1.5 * b["mlups"]
    assert a["requests"] == b["requests"] == 60


def test_request_stream_is_seeded_and_in_range():
    a = S.request_stream(500, seed=7, steps=(2000, 20000))
    b = S.request_stream(500, seed=7, steps=(2000, 20000))
    assert a == b
    assert a[0].arrival == 0.0
    assert all(x.arrival <= y.arrival for x, y in zip(a, a[1:]))
    assert {r.grid for r in a} == set(S.GRIDS)
    assert all(100 <= r.re <= 4000 and 0.1 <= r.atwood <= 0.9 and 1e-3 <= r.sigma <= 1e-2
               and 2000 <= r.steps <= 20000 for r in a)


def test_poisson_arrivals_have_the_stated_mean_gap():
    r = S.request_stream(20000, seed=1, mean_interarrival=0.25)
    gaps = np.diff([x.arrival for x in r])
    assert abs(gaps.mean() - 0.25) < 0.01
    # exponential gaps: standard deviation equals the mean
    assert abs(gaps.std() - 0.25) < 0.01


def test_with_load_scales_the_gaps():
    reqs = S.request_stream(400, seed=2)
    svc = lambda r: r.updates / 1e9  # noqa: E731
    loaded = S.with_load(reqs, svc, 1.5)
    gaps = np.diff([r.arrival for r in loaded])
    mean_service = np.mean([svc(r) for r in reqs])
    assert gaps.mean() == pytest.approx(mean_service / 1.5, rel=1e-9)
    assert [r.steps for r in loaded] == [r.steps for r in reqs]


def test_summarize():
    outs = [S.Outcome(i, 0.0, 0.0, float(i + 1), 10, 100, True) for i in range(100)]
    s = S.summarize(outs)
    assert s["p50_s"] == pytest.approx(50.5)
    assert s["p99_s"] == pytest.approx(99.01)
    assert s["mlups"] == pytest.approx(100 * 10 * 100 / 100.0 / 1e6)
    assert s["unstable"] == 0


def test_footprint_grows_with_the_grid():
    from paper_1507_07294_gb300 import lbm
    sizes = []
    for g in S.GRIDS:
        w = S.workload_of(S.Request(0, 0.0, g, 1000.0, 0.5, 5e-3, 10), phi0=np.zeros(0))
        sizes.append(lbm.lbm_memory_bytes(*lbm.params_from_workload(w)))
    per_cell = [s / (g[0] * g[1] * g[2]) for s, g in zip(sizes, S.GRIDS)]
    # populations (22 + 3 slots x 2 arrays) and phi, mu: about 216 B per cell and more
    assert all(200 < b < 300 for b in per_cell)
    assert per_cell[-1] == pytest.approx(per_cell[-2], rel=0.02)


def test_large_run_cap():
    """With max_large = 1 at most one large run is open at a time; small requests pass
    a held-back large one; large requests keep their order among themselves."""
    reqs = _reqs(n=60, gap=0.0005, steps=(20, 200))
    big = 16 * 16 * 64

    class Counting(FakeEngine):
        def __init__(self):
            super().__init__()
            self.max_large_open = 0

        def open(self, r):
            h = super().open(r)
            self.max_large_open = max(self.max_large_open,
                                      sum(c >= big for (_, _, c) in self.open_runs))
            return h

    eng = Counting()
    srv = _server(eng, budget_bytes=10**9, max_runs=8, quantum=8, max_large=1,
                  large_cells=big)
    out = srv.serve(reqs)
    assert len(out) == 60 and eng.max_large_open == 1
    larges = sorted((o for o in out if o.cells >= big), key=lambda o: o.arrival)
    assert all(a.admitted <= b.admitted for a, b in zip(larges, larges[1:]))
    passed = [o for o in out if o.cells < big and any(
        l.arrival < o.arrival and l.admitted > o.admitted for l in larges)]
    assert passed, "small requests should overtake a large one held by the cap"
    with pytest.raises(ValueError):
        _server(FakeEngine(), budget_bytes=10**9, max_large=0)
