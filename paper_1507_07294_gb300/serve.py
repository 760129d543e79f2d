"""Continuous-batching request loop for many Rayleigh-Taylor runs on one GPU.

Requests (a grid, a Reynolds number, an Atwood number, a surface tension and a step
count) arrive over time.  The server keeps every admitted run's populations resident
in device memory, admits waiting requests first-come first-served whenever a slot and
enough of the device-memory budget are free (each run's footprint comes from
lbm_memory_bytes), and advances all admitted runs together in quanta of Q time steps
with one batched launch per pass (lbm_batch_step).  A run's first few steps are taken
alone (lbm_step) -- the first step after initialisation has its own time-derivative
rule (d_t(phi u) = 0) and the rest of that chunk aligns the run's remaining steps to a
multiple of Q, so that every admitted run takes part in every quantum.  Runs that are
done are read out (the order-parameter field plus the FP64 mass and momentum sums) and
their memory is returned to the budget.  The loop is pipelined (the next quantum is
queued before the host reads out the last one's finished runs), and every few quanta
each run's FP64 sums are checked so that a diverged run stops early.

The one-at-a-time baseline takes the same requests in arrival order and runs each to
completion alone with lbm_step, one run on the device at a time (same quanta, same
divergence checks).

Scheduling is host logic over an engine interface (open / step_alone / step_batch /
sync / finish / footprint), so it runs unchanged against a fake engine on the CPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

# grids of the serving workload, (nx, ny, nz): periodic x, y; walls at z
GRIDS: Tuple[Tuple[int, int, int], ...] = ((32, 32, 32), (64, 64, 64), (64, 64, 256),
                                           (128, 128, 512))


@dataclass
class Request:
    """One simulation run: a Rayleigh-Taylor problem (Sec. III C) on a W x W x nz grid."""

    rid: int
    arrival: float  # seconds after the stream starts
    grid: Tuple[int, int, int]
    re: float
    atwood: float
    sigma: float
    steps: int

    @property
    def cells(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    @property
    def updates(self) -> int:
        return self.cells * self.steps


@dataclass
class Outcome:
    """What the server reports for a finished request."""

    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int  # steps taken: fewer than requested when the run was stopped as diverged
    cells: int
    stable: bool
    result: object = field(default=None, repr=False)

    @property
    def latency(self) -> float:
        """Time to solution: from arrival to the result on the host."""
        return self.finished - self.arrival


def request_stream(n: int = 200, seed: int = 0, grids: Sequence[Tuple[int, int, int]] = GRIDS,
                   re: Tuple[float, float] = (100.0, 4000.0),
                   atwood: Tuple[float, float] = (0.1, 0.9),
                   sigma: Tuple[float, float] = (1e-3, 1e-2),
                   steps: Tuple[int, int] = (2000, 20000),
                   mean_interarrival: float = 1.0) -> List[Request]:
    """n seeded requests with Poisson arrivals (exponential gaps of the given mean); the
    grid uniform over `grids`, Re, At and sigma uniform over their ranges, the step count
    uniform over the integers in `steps`."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(mean_interarrival, size=n)
    gaps[0] = 0.0
    arrivals = np.cumsum(gaps)
    out = []
    for i in range(n):
        g = grids[int(rng.integers(len(grids)))]
        out.append(Request(rid=i, arrival=float(arrivals[i]), grid=tuple(int(v) for v in g),
                           re=float(rng.uniform(*re)), atwood=float(rng.uniform(*atwood)),
                           sigma=float(rng.uniform(*sigma)),
                           steps=int(rng.integers(steps[0], steps[1] + 1))))
    return out


def with_load(requests: Sequence[Request], service_time: Callable[[Request], float],
              load: float) -> List[Request]:
    """The same requests with arrival times rescaled so that the offered load is `load`
    times what one-at-a-time service sustains: the mean gap becomes mean(service) / load."""
    if load <= 0:
        raise ValueError("load must be positive")
    mean_service = float(np.mean([service_time(r) for r in requests]))
    gaps = np.diff([0.0] + [r.arrival for r in requests])
    mean_gap = float(np.mean(gaps[1:])) if len(gaps) > 1 else 1.0
    scale = (mean_service / load) / mean_gap if mean_gap > 0 else 0.0
    return [Request(r.rid, r.arrival * scale, r.grid, r.re, r.atwood, r.sigma, r.steps)
            for r in requests]


def summarize(outcomes: Sequence[Outcome], t_start: float = 0.0) -> Dict[str, float]:
    """p50 / p99 time to solution, aggregate MLUPS over the makespan, run counts."""
    if not outcomes:
        return {"requests": 0}
    lat = np.array([o.latency for o in outcomes])
    end = max(o.finished for o in outcomes)
    makespan = end - t_start
    updates = float(sum(o.cells * o.steps for o in outcomes))
    return {
        "requests": len(outcomes),
        "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()),
        "makespan_s": float(makespan),
        "mlups": updates / makespan / 1e6 if makespan > 0 else float("nan"),
        "unstable": int(sum(not o.stable for o in outcomes)),
    }


class Server:
    """Continuous batching: admit by slots and memory budget, advance all admitted runs
    in quanta of `quantum` steps with one batched launch per pass, retire finished runs.

    batched=False gives the one-at-a-time baseline: one run resident, stepped alone
    (lbm_step) in the same quanta and with the same divergence checks, so the two differ
    only in how many runs share the device.
    """

    def __init__(self, engine, budget_bytes: int, max_runs: int = 16, quantum: int = 64,
                 batched: bool = True, check_every: int = 2,
                 max_large: Optional[int] = None, large_cells: int = 0,
                 clock: Callable[[], float] = time.perf_counter,
                 sleep: Callable[[float], None] = time.sleep):
        """check_every: every that many quanta each stepping run's FP64 sums are
        enqueued (lbm_reduce_async); a run found non-finite is stopped and reported
        unstable without taking its remaining steps (0: never check).

        max_large: at most this many runs of at least `large_cells` cells on the device
        at once (None: no cap).  Large runs fill the GPU by themselves, so sharing it
        among many of them only stretches each; a large request held back by the cap
        lets later small requests pass it, and is admitted as soon as a large run
        leaves."""
        if quantum < 1 or max_runs < 1:
            raise ValueError("quantum and max_runs must be >= 1")
        if max_large is not None and max_large < 1:
            raise ValueError("max_large must be >= 1 or None")
        self.max_large = max_large
        self.large_cells = int(large_cells)
        self.check_every = check_every
        self.stopped = 0
        self.engine = engine
        self.budget = int(budget_bytes)
        self.max_runs = max_runs if batched else 1
        self.quantum = quantum
        self.batched = batched
        self.clock = clock
        self.sleep = sleep
        self.peak_bytes = 0
        self.peak_runs = 0
        self.quanta = 0

    def _is_large(self, r: Request) -> bool:
        return self.max_large is not None and r.cells >= self.large_cells

    def serve(self, requests: Sequence[Request]) -> List[Outcome]:
        """Serve the requests (arrival times relative to the call) and return their
        outcomes in finishing order.

        Pipelined: iteration k launches quantum k, then waits for quantum k - 1 and
        reads out the runs that finished in it, so the device always has the next
        quantum queued while the host reads results and admits requests.  A finished
        run keeps its slot and its memory until it has been read out."""
        pending = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        for r in pending:
            if self.engine.footprint(r) > self.budget:
                raise ValueError(f"request {r.rid} alone exceeds the memory budget")
        waiting: deque = deque()
        active: List[list] = []     # [request, handle, remaining steps, bytes, admitted at]
        inflight = None             # (fence of the last quantum, runs it finished)
        used = 0
        done: List[Outcome] = []
        t0 = self.clock()
        now = lambda: self.clock() - t0  # noqa: E731
        while pending or waiting or active or inflight:
            t = now()
            while pending and pending[0].arrival <= t:
                waiting.append(pending.popleft())
            # admission: first come first served while a slot and the budget allow; a
            # large request over the large-run cap is passed over, not waited for
            held_runs = active + (inflight[1] if inflight else [])
            held = len(held_runs)
            large = sum(self._is_large(a[0]) for a in held_runs)
            passed = deque()
            while waiting and held < self.max_runs:
                if (self.max_large is not None and self._is_large(waiting[0])
                        and large >= self.max_large):
                    passed.append(waiting.popleft())
                    continue
                need = self.engine.footprint(waiting[0])
                if used + need > self.budget:
                    break
                r = waiting.popleft()
                large += self._is_large(r)
                admitted = now()
                h = self.engine.open(r)
                used += need
                held += 1
                first = (r.steps - 1) % self.quantum + 1 if r.steps > 0 else 0
                if first:
                    self.engine.step_alone(h, first)
                active.append([r, h, r.steps - first, need, admitted])
            passed.extend(waiting)
            waiting = passed  # the passed-over large requests keep their place in line
            self.peak_bytes = max(self.peak_bytes, used)
            self.peak_runs = max(self.peak_runs, held)
            # launch this quantum (and, every check_every quanta, the divergence checks)
            stepping = [a for a in active if a[2] > 0]
            checked = []
            if stepping:
                if self.batched:
                    self.engine.step_batch([a[1] for a in stepping], self.quantum)
                else:
                    for a in stepping:
                        self.engine.step_alone(a[1], self.quantum)
                self.quanta += 1
                for a in stepping:
                    a[2] -= self.quantum
                if self.check_every and self.quanta % self.check_every == 0:
                    checked = [a for a in stepping if a[2] > 0]
                    for a in checked:
                        self.engine.check(a[1])
            finished = [a for a in active if a[2] <= 0]
            active = [a for a in active if a[2] > 0]
            # wait for the previous quantum; stop the runs its checks found diverged
            if inflight is not None:
                prev_fence, prev_finished, prev_checked = inflight
                if prev_fence is not None:
                    self.engine.wait(prev_fence)
                bad = {id(a) for a in prev_checked if self.engine.diverged(a[1])}
                if bad:
                    self.stopped += sum(id(a) in bad for a in active)
                    finished += [a for a in active if id(a) in bad]
                    active = [a for a in active if id(a) not in bad]
            fence = self.engine.fence([a[1] for a in stepping + finished]) \
                if stepping or finished else None
            # read out what the previous quantum finished
            if inflight is not None:
                for r, h, left, need, admitted in inflight[1]:
                    stable, result = self.engine.finish(h)
                    used -= need
                    done.append(Outcome(r.rid, r.arrival, admitted, now(), r.steps - max(left, 0),
                                        r.cells, stable, result))
            inflight = (fence, finished, checked) if fence is not None else None
            if inflight is None and not active and pending and not waiting:
                self.sleep(max(0.0, pending[0].arrival - now()))
        return done


# --------------------------------------------------------------------------------
# The GPU engine: runs are lbm Solvers on one stream, quanta are lbm_batch_step calls.
# --------------------------------------------------------------------------------

def workload_of(req: Request, phi0: Optional[np.ndarray] = None, steps: Optional[int] = None):
    """The Rayleigh-Taylor workload of a request (Eqs. 42-44 with sqrt(gW) = 0.04, D = 4,
    Pe = 50); phi0 may be passed in when already built for this grid."""
    from . import inputs as I
    nx, ny, nz = req.grid
    if nx != ny:
        raise ValueError("Rayleigh-Taylor grids are square in x, y")
    w = I.rayleigh_taylor(W=nx, Re=req.re, atwood=req.atwood, sigma=req.sigma, nz=nz,
                          steps=req.steps if steps is None else steps,
                          with_fields=phi0 is None)
    if phi0 is not None:
        w.phi0 = phi0
    return w


class GpuEngine:
    """Engine over the C-ABI library: one CUDA stream for every run and the batch."""

    def __init__(self, storage: Optional[int] = None, keep_phi: bool = True):
        import torch
        from . import lbm
        self.lbm = lbm
        self.torch = torch
        self.storage = lbm.LBM_STORAGE_FP32 if storage is None else storage
        # every run has a stream of its own (recycled when it finishes), so reading out
        # one run never waits behind another run's steps
        self._free_streams: List[object] = []
        self._stream_of: Dict[int, object] = {}
        self._checks: Dict[int, tuple] = {}  # divergence-check buffers (device, pinned host)
        # the shared launches run on a stream of their own, so that they overlap the
        # runs that take their own launches (lbm_batch_set_split)
        self.batch_stream = torch.cuda.Stream()
        self.batch = lbm.Batch(stream=self.batch_stream.cuda_stream)
        self.keep_phi = keep_phi
        self._phi0: Dict[Tuple[int, int, int], np.ndarray] = {}
        self._bytes: Dict[Tuple[int, int, int], int] = {}

    def phi0(self, grid) -> np.ndarray:
        from . import inputs as I
        if grid not in self._phi0:
            self._phi0[grid] = I.rt_interface(grid[0], grid[2], 4.0)
        return self._phi0[grid]

    def footprint(self, req: Request) -> int:
        if req.grid not in self._bytes:
            w = workload_of(req, phi0=np.zeros(0))
            g, p = self.lbm.params_from_workload(w, storage=self.storage)
            self._bytes[req.grid] = self.lbm.lbm_memory_bytes(g, p)
        return self._bytes[req.grid]

    def open(self, req: Request):
        w = workload_of(req, phi0=self.phi0(req.grid))
        st = self._free_streams.pop() if self._free_streams else self.torch.cuda.Stream()
        with self.torch.cuda.nvtx.range(f"admit {req.rid}"):
            s = self.lbm.Solver(w, stream=st.cuda_stream, storage=self.storage)
        self._stream_of[id(s)] = st
        return s

    def stream_of(self, solver):
        return self._stream_of[id(solver)]

    def step_alone(self, solver, n: int) -> None:
        solver.step(n)

    def step_batch(self, solvers, n: int) -> None:
        with self.torch.cuda.nvtx.range(f"quantum {len(solvers)} runs"):
            self.batch.step(solvers, n)

    def check(self, solver) -> None:
        """Enqueues the run's FP64 sums (lbm_reduce_async), written by the reduction
        straight into a page-locked host slot."""
        slot = self._checks.get(id(solver))
        if slot is None:
            slot = self.torch.zeros(5, dtype=self.torch.float64).pin_memory()
            self._checks[id(solver)] = slot
        self.lbm.lbm_reduce_async(solver.ctx, slot.data_ptr())

    def diverged(self, solver) -> bool:
        """Whether the last check of the run (read after its fence) found a non-finite
        value."""
        slot = self._checks.get(id(solver))
        return slot is not None and bool(slot[4].item() > 0)

    def fence(self, solvers):
        """Events marking everything launched so far on the runs' streams."""
        evs = []
        for s in solvers:
            e = self.torch.cuda.Event()
            e.record(self.stream_of(s))
            evs.append(e)
        return evs

    def wait(self, fence) -> None:
        for e in fence:
            e.synchronize()

    def sync(self) -> None:
        self.torch.cuda.synchronize()

    def finish(self, solver):
        """Reads the run's result; a non-finite state marks it unstable."""
        lbm = self.lbm
        with self.torch.cuda.nvtx.range("read-out"):
            try:
                totals = solver.reduce()
                stable = True
            except lbm.LbmError as e:
                if e.status != lbm.LBM_EUNSTABLE:
                    raise
                totals, stable = None, False
            phi = None
            if self.keep_phi:
                # a page-locked buffer (from PyTorch's cache of them), which the read-out
                # kernel fills directly
                buf = self.torch.empty(solver.ctx.n, dtype=self.torch.float64,
                                       pin_memory=True).numpy()
                phi = lbm.lbm_read_fields(solver.ctx, lbm.LBM_FIELD_PHI, out={"phi": buf})["phi"]
        solver.close()
        self._checks.pop(id(solver), None)
        self._free_streams.append(self._stream_of.pop(id(solver)))
        return stable, {"totals": totals, "phi": phi}

    def close(self) -> None:
        self.batch.close()


def service_time_model(engine: GpuEngine, grids: Sequence[Tuple[int, int, int]],
                       steps: int = 200) -> Dict[Tuple[int, int, int], Tuple[float, float]]:
    """Per grid: (seconds per time step alone, fixed seconds per run for open + read-out),
    measured on the device; used to set the offered load."""
    out = {}
    for g in grids:
        req = Request(-1, 0.0, tuple(g), 1000.0, 0.5, 5e-3, steps)
        t0 = time.perf_counter()
        s = engine.open(req)
        s.step(1)
        engine.sync()
        t1 = time.perf_counter()
        s.step(steps)
        engine.sync()
        t2 = time.perf_counter()
        engine.finish(s)
        t3 = time.perf_counter()
        out[tuple(g)] = ((t2 - t1) / steps, (t1 - t0) + (t3 - t2))
    return out


def tune_batch(engine: GpuEngine, grids: Sequence[Tuple[int, int, int]], quantum: int = 64,
               reps: int = 2) -> Dict[str, object]:
    """Autotunes the batch schedule on a mix of one run per grid, by coordinate descent
    over: the size split (runs of at least that many cells take their own launches;
    candidates in waves of stream-collide blocks), then for each pass its blocks
    (persistent, in blocks per SM, or 0 = one block per item) and the prefetch
    distance of the stream-collide pass.  Leaves the best settings on engine.batch and
    returns them with the measured quantum times (ms)."""
    torch = engine.torch
    b = engine.batch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    wave = sms * 4 * 256  # cells of one wave of stream-collide blocks (4 per SM, 256 cells each)
    runs = [engine.open(Request(-1, 0.0, tuple(g), 1000.0, 0.5, 5e-3, 1)) for g in grids]
    for s in runs:
        s.step(1)

    def timed() -> float:
        engine.step_batch(runs, quantum)  # capture + warm
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            engine.step_batch(runs, quantum)
            torch.cuda.synchronize()  # every run's stream and the batch's
            best = min(best, (time.perf_counter() - t0) * 1e3)
        return best

    knobs = [
        ("split_cells", b.set_split, [0] + [k * wave for k in (1, 2, 4, 8, 16)]),
        ("collide_blocks", lambda v: b.set_grid(2, v), [0, 4 * sms, 8 * sms]),
        ("collide_prefetch", lambda v: b.set_prefetch(2, v), [-1, 0, sms * 2]),
        ("phi_blocks", lambda v: b.set_grid(0, v), [0, 8 * sms, 16 * sms]),
        ("mu_blocks", lambda v: b.set_grid(1, v), [0, 6 * sms, 12 * sms]),
    ]
    log: Dict[str, object] = {}
    for name, setter, values in knobs:
        times = {}
        for v in values:
            setter(v)
            times[v] = timed()
        best = min(times, key=times.get)
        setter(best)
        log[name] = best
        log[name + "_ms"] = {str(k): round(t, 3) for k, t in times.items()}
    for s in runs:
        engine.finish(s)
    return log
