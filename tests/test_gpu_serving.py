"""Batched execution and the request loop on the GPU, through the C ABI.

A run advanced inside a batch (lbm_batch_step) runs the same per-cell device code on
the same state as when it is advanced alone (lbm_step), so its state must come out
bit for bit the same whatever else shares the launch.  The batched path is also checked
against the FP64 oracle at the coupled-path tolerances.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import inputs as I
from paper_1507_07294_gb300 import serve as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1507_07294_gb300 import lbm
    lbm.load_library()
    return lbm


def _mix():
    """Runs of uneven, ragged sizes; periodic and walled; with gravity and noise."""
    a = I.perturbed(I.droplet(n=16, R=5.0, nx=20, ny=18, nz=16), seed=11, u_amp=0.01, p_amp=1e-3)
    b = I.rayleigh_taylor(W=24, nz=40, Re=300.0, atwood=0.3, sigma=5e-3)
    b = I.perturbed(b, seed=12, u_amp=0.01, p_amp=1e-4)
    c = I.perturbed(I.rayleigh_taylor(W=37, nz=70, Re=1000.0, atwood=0.7, sigma=2e-3), seed=13,
                    u_amp=0.005)
    d = I.perturbed(I.droplet(n=33, R=9.0), seed=14, u_amp=0.005, p_amp=1e-4)
    return [a, b, c, d]


def _state(s):
    f, g, phiu, t = s.state()
    return f, g, phiu, t


def _assert_same(s1, s2):
    for x, y in zip(_state(s1)[:3], _state(s2)[:3]):
        assert np.array_equal(x, y)
    assert s1.t == s2.t


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_each_run_is_the_same_alone_and_in_the_mix(L, storage):
    st = {"fp32": L.LBM_STORAGE_FP32, "fp16": L.LBM_STORAGE_FP16, "bf16": L.LBM_STORAGE_BF16}[storage]
    ws = _mix()
    alone = [L.Solver(w, storage=st) for w in ws]
    for s in alone:
        s.step(23)
    mixed = [L.Solver(w, storage=st) for w in ws]
    with L.Batch() as b:
        for s in mixed:
            s.step(1)
        b.step(mixed, 7)
        b.step(mixed[1:3], 5)   # a subset
        for s in (mixed[0], mixed[3]):
            s.step(5)           # alone in between
        b.step(mixed, 10)
    for s1, s2 in zip(alone, mixed):
        _assert_same(s1, s2)
    for s in alone + mixed:
        s.close()


def test_batch_grid_sizes_do_not_change_results(L):
    ws = _mix()[:3]
    ref = [L.Solver(w) for w in ws]
    for s in ref:
        s.step(9)
    with L.Batch() as b:
        runs = [L.Solver(w) for w in ws]
        for s in runs:
            s.step(1)
        for p, n in ((0, 1), (1, 1), (2, 1)):  # one block per pass: every item strided
            b.set_grid(p, n)
            assert b.get_grid(p) == n
        b.step(runs, 4)
        for p, n in ((0, 1000), (1, 77), (2, 4096)):
            b.set_grid(p, n)
        b.set_prefetch(0, 0)
        b.set_prefetch(2, 5)
        b.step(runs, 2)
        for p in range(3):  # one block per item
            b.set_grid(p, 0)
        b.set_prefetch(0, -1)
        b.set_prefetch(2, -1)
        assert b.get_prefetch(2) == -1
        b.step(runs, 2)
        for s1, s2 in zip(ref, runs):
            _assert_same(s1, s2)
        with pytest.raises(L.LbmError):
            b.set_grid(3, 10)
        with pytest.raises(L.LbmError):
            b.set_grid(0, -1)
        with pytest.raises(L.LbmError):
            b.set_prefetch(1, 4)  # the chemical-potential pass does not prefetch
        for s in ref + runs:
            s.close()


def test_batched_path_matches_the_oracle(L):
    """Two runs through the batch for 100 steps against the FP64 oracle."""
    ws = [I.perturbed(I.droplet(n=32, R=8.0), seed=0, u_amp=0.005, p_amp=1e-4),
          I.perturbed(I.rayleigh_taylor(W=24, nz=50, Re=256.0), seed=5, u_amp=0.01, p_amp=1e-4)]
    runs = [L.Solver(w) for w in ws]
    with L.Batch() as b:
        for s in runs:
            s.step(1)
        b.step(runs, 99)
    for w, s in zip(ws, runs):
        gf = s.fields()
        o = O.Oracle(O.Params.from_workload(w))
        o.init(w.phi0, w.u0, w.p0)
        o.step(100)
        of = o.fields()
        assert np.abs(gf["phi"] - of["phi"]).max() <= 1e-5
        assert np.abs(gf["u"] - of["u"]).max() / w.U <= 1e-4
        s.close()


def test_batch_rejects_what_it_cannot_run(L):
    w = I.droplet(n=12, R=3.0)
    with L.Batch() as b:
        fresh = L.Solver(w)
        with pytest.raises(L.LbmError, match="no step"):
            b.step([fresh], 3)
        fresh.step(1)
        b.step([fresh], 0)  # zero steps: nothing happens
        assert fresh.t == 1
        with pytest.raises(L.LbmError, match="twice"):
            b.step([fresh, fresh], 2)
        aa = L.Solver(w, pattern=L.LBM_PATTERN_AA)
        aa.step(1)
        half = L.Solver(w, storage=L.LBM_STORAGE_FP16)
        half.step(1)
        wv = I.droplet(n=12, R=3.0)
        wv.srt_flow = True
        variant = L.Solver(wv)
        variant.step(1)
        track = L.Solver(I.deformation(n=16, period=100.0))
        track.step(1)
        for bad in (aa, variant, track):
            with pytest.raises(L.LbmError):
                b.step([fresh, bad], 2)
        with pytest.raises(L.LbmError, match="storage"):
            b.step([fresh, half], 2)
        assert fresh.t == 1  # refused calls change nothing
        for s in (fresh, aa, half, variant, track):
            s.close()


def test_serving_loop_results_equal_alone_runs(L):
    """A small request stream through the continuous-batching server: each finished
    run's phi equals the same request run alone from start to finish."""
    grids = ((16, 16, 16), (24, 24, 40), (16, 16, 64))
    reqs = S.request_stream(10, seed=4, grids=grids, steps=(5, 90), mean_interarrival=0.002)
    eng = S.GpuEngine()
    budget = 3 * max(eng.footprint(r) for r in reqs)
    srv = S.Server(eng, budget_bytes=budget, max_runs=4, quantum=16)
    out = srv.serve(reqs)
    assert sorted(o.rid for o in out) == list(range(10))
    assert srv.peak_bytes <= budget and srv.peak_runs <= 4
    assert srv.quanta > 0 and srv.peak_runs >= 2
    by = {r.rid: r for r in reqs}
    for o in out:
        r = by[o.rid]
        assert o.stable
        with L.Solver(S.workload_of(r)) as s:
            s.step(r.steps)
            phi = s.fields(L.LBM_FIELD_PHI)["phi"]
        assert np.array_equal(phi, o.result["phi"]), f"request {o.rid}"
        assert o.result["totals"][0] == pytest.approx(
            float(np.sum(S.workload_of(r).phi0)), abs=1e-6 * r.cells)
    summ = S.summarize(out)
    assert summ["requests"] == 10 and summ["p99_s"] >= summ["p50_s"] > 0
    eng.close()


def test_batch_tuner_leaves_its_choice_set(L):
    eng = S.GpuEngine()
    log = S.tune_batch(eng, ((16, 16, 16), (24, 24, 40)), quantum=4, reps=1)
    b = eng.batch
    assert b.get_split() == log["split_cells"]
    assert b.get_grid(2) == log["collide_blocks"]
    assert b.get_prefetch(2) == log["collide_prefetch"]
    assert b.get_grid(0) == log["phi_blocks"] and b.get_grid(1) == log["mu_blocks"]
    eng.close()


def test_split_runs_are_the_same_alone_and_in_the_mix(L):
    """With a size split the large runs take their own launches on their streams while
    the small ones share the batched launches on the batch's stream."""
    import torch
    ws = _mix()
    alone = [L.Solver(w) for w in ws]
    for s in alone:
        s.step(12)
    streams = [torch.cuda.Stream() for _ in ws]
    mixed = [L.Solver(w, stream=st.cuda_stream) for w, st in zip(ws, streams)]
    with L.Batch(stream=torch.cuda.Stream().cuda_stream) as b:
        b.set_split(30 * 30 * 30)  # the 37 x 37 x 70 and 33^3 runs go alone
        for s in mixed:
            s.step(1)
        b.step(mixed, 6)
        b.set_split(1)              # every run alone
        b.step(mixed, 2)
        b.set_split(0)              # every run shared
        b.step(mixed, 3)
    torch.cuda.synchronize()
    for s1, s2 in zip(alone, mixed):
        _assert_same(s1, s2)
    for s in alone + mixed:
        s.close()


def test_reduce_async_matches_reduce(L):
    import torch
    w = I.perturbed(I.droplet(n=20, R=6.0), seed=3, u_amp=0.01)
    with L.Solver(w) as s:
        s.step(5)
        buf = torch.full((5,), -1.0, dtype=torch.float64, device="cuda")
        L.lbm_reduce_async(s.ctx, buf.data_ptr())
        torch.cuda.synchronize()
        sum_phi, mom = s.reduce()
        got = buf.cpu().numpy()
        assert got[0] == sum_phi and np.array_equal(got[1:4], mom) and got[4] == 0
        with pytest.raises(L.LbmError, match="aligned"):
            L.lbm_reduce_async(s.ctx, buf.data_ptr() + 4)
        with pytest.raises(L.LbmError):
            L.lbm_reduce_async(s.ctx, 0)


def test_server_stops_a_diverging_run(L):
    """32^3, Re = 100, At = 0.9 (density ratio 19): the method itself diverges near step
    450 (the FP64 oracle too); the server's checks stop it well before its 3000 steps
    while the stable run alongside completes unchanged."""
    reqs = [S.Request(0, 0.0, (32, 32, 32), 100.0, 0.9, 1e-3, 3000),
            S.Request(1, 0.0, (32, 32, 32), 100.0, 0.3, 1e-3, 300)]
    eng = S.GpuEngine()
    srv = S.Server(eng, budget_bytes=10**10, quantum=32, check_every=1)
    out = {o.rid: o for o in srv.serve(reqs)}
    assert not out[0].stable and 300 <= out[0].steps < 1500 and srv.stopped == 1
    assert out[1].stable and out[1].steps == 300
    with L.Solver(S.workload_of(reqs[1])) as s:
        s.step(300)
        assert np.array_equal(s.fields(L.LBM_FIELD_PHI)["phi"], out[1].result["phi"])
    eng.close()


def test_batch_limits(L):
    """At most 256 runs per call; negative sizes and empty calls are refused."""
    w = I.droplet(n=4, R=1.5)
    runs = [L.Solver(w) for _ in range(257)]
    for s in runs:
        s.step(1)
    with L.Batch() as b:
        with pytest.raises(L.LbmError, match="256"):
            b.step(runs, 1)
        b.step(runs[:256], 1)
        with pytest.raises(L.LbmError):
            b.step([], 1)
        with pytest.raises(L.LbmError):
            b.set_split(-1)
        with pytest.raises(L.LbmError):
            b.step(runs[:2], -1)
    assert runs[0].t == 2 and runs[256].t == 1
    for s in runs:
        s.close()
