"""The serving loop's scheduling on the CPU, with a simulated engine and clock.

Checks the admission rules (budget, one block per beam on the device, arrival
order within a beam), continuous batching (blocks arriving while a step runs
are launched on the second stream before that step ends) and the latency
bookkeeping.
"""
import numpy as np
import pytest

from paper_2401_13834_gb300.serve import Server, SimEngine


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def make(budget, cost=1.0, reserves=(10,), nstreams=2, max_batch=64):
    clk = Clock()
    eng = SimEngine(lambda plan: plan["cost"], clk)
    srv = Server(eng, budget, max_batch=max_batch, nstreams=nstreams, clock=clk)
    ids = [srv.add_beam({"reserve": r, "cost": cost}) for r in reserves]
    return srv, eng, clk, ids


def run(srv, clk, dt=0.25, until=1e9):
    while not srv.idle() and clk.t < until:
        srv.pump()
        clk.t += dt


def test_plan_larger_than_budget_is_rejected():
    srv, _, _, _ = make(100)
    with pytest.raises(ValueError):
        srv.add_beam({"reserve": 101, "cost": 1.0})


def test_budget_never_exceeded_and_everything_completes():
    rng = np.random.default_rng(0)
    reserves = rng.integers(5, 40, size=12)
    srv, eng, clk, ids = make(100, reserves=reserves)
    peak = 0
    for step in range(200):
        if step < 120 and rng.random() < 0.6:
            srv.submit(int(rng.integers(0, 12)), block=None)
        srv.pump()
        peak = max(peak, srv.reserved)
        assert srv.reserved <= 100
        # the blocks on the device never exceed the budget either
        on_dev = sum(j.reserve for _, _, jobs in srv.inflight for j in jobs)
        assert on_dev <= 100
        clk.t += 0.3
    run(srv, clk)
    assert srv.idle()
    assert peak <= 100 and srv.peak_reserved <= 100
    assert all(j.done is not None for j in srv.completed)


def test_one_block_per_beam_on_the_device_and_order_kept():
    srv, eng, clk, ids = make(1000, reserves=(10, 10, 10))
    for k in range(5):
        for b in ids:
            srv.submit(b, block=None)
    run(srv, clk)
    for h in eng.launches:
        beams = [j.beam for j in h["jobs"]]
        assert len(beams) == len(set(beams))
    # every beam's blocks completed in order, each after the previous one finished
    for b in ids:
        js = sorted((j for j in srv.completed if j.beam == b), key=lambda j: j.seq)
        assert [j.seq for j in js] == list(range(5))
        for a, c in zip(js, js[1:]):
            assert c.launched >= a.done


def test_continuous_batching_overlaps_steps():
    """A block arriving while a step runs goes out on the other stream at once."""
    srv, eng, clk, ids = make(1000, cost=2.0, reserves=(10, 10))
    srv.submit(ids[0], block=None)
    srv.pump()                      # step 1 on stream 0, ends at t = 2
    clk.t = 0.5
    srv.submit(ids[1], block=None)
    srv.pump()                      # step 2 on stream 1, before step 1 ends
    assert len(srv.inflight) == 2
    assert {s for _, s, _ in srv.inflight} == {0, 1}
    assert eng.launches[1]["jobs"][0].launched == 0.5
    run(srv, clk, dt=0.5)
    lat = sorted(j.latency for j in srv.completed)
    assert lat == [2.0, 2.0]


def test_blocks_wait_for_memory_then_run():
    srv, eng, clk, ids = make(25, cost=1.0, reserves=(10, 10, 10))
    for b in ids:
        srv.submit(b, block=None)
    srv.pump()
    assert srv.reserved == 20 and len(srv.pending) == 1   # the third waits for memory
    run(srv, clk)
    assert len(srv.completed) == 3 and srv.peak_reserved <= 25


def test_max_batch_splits_steps():
    srv, eng, clk, ids = make(10 ** 6, reserves=(1,) * 10, max_batch=4, nstreams=1)
    for b in ids:
        srv.submit(b, block=None)
    run(srv, clk)
    assert [len(h["jobs"]) for h in eng.launches] == [4, 4, 2]


def test_stats():
    srv, eng, clk, ids = make(1000, cost=1.0, reserves=(10, 10))
    for b in ids:
        srv.submit(b, block=None)
    run(srv, clk)
    st = srv.stats(data_seconds=lambda j: 10.0)
    assert st["blocks"] == 2 and st["p50_latency_s"] == pytest.approx(2.0)   # one step of two jobs
    assert st["real_time_factor"] == pytest.approx(20.0 / st["span_s"])


def test_drain_deadline_on_a_hung_step():
    """A step that never finishes (made on the host) ends drain() with
    TimeoutError at the deadline instead of waiting forever."""
    srv, eng, clk, ids = make(1000, cost=1.0, reserves=(10,))
    eng.stall = True
    srv.submit(ids[0], block=None)

    class Tick:  # the server's clock advances as it polls
        def __call__(self):
            clk.t += 0.5
            return clk.t
    srv.clock = Tick()
    with pytest.raises(TimeoutError):
        srv.drain(timeout_s=10.0)
    assert len(srv.inflight) == 1            # the hung step is still accounted for


def test_beam_removed_mid_stream():
    srv, eng, clk, ids = make(15, cost=1.0, reserves=(10, 10))
    for k in range(3):
        srv.submit(ids[0], block=None)
        srv.submit(ids[1], block=None)
    srv.pump()                               # beam 0's first block admitted (budget fits one)
    dropped = srv.remove_beam(ids[1])
    assert len(dropped) == 3 and all(j.beam == ids[1] for j in dropped)
    with pytest.raises(ValueError):
        srv.submit(ids[1], block=None)
    run(srv, clk)
    assert sorted(j.seq for j in srv.completed) == [0, 1, 2]
    assert all(j.beam == ids[0] for j in srv.completed)


def test_malformed_block_refused_at_submit():
    clk = Clock()
    eng = SimEngine(lambda plan: 1.0, clk)
    srv = Server(eng, 100, clock=clk)
    b = srv.add_beam({"reserve": 10, "cost": 1.0, "block": "ok"})
    srv.submit(b, block="ok")
    with pytest.raises(ValueError):
        srv.submit(b, block="short")
    assert len(srv.pending) == 1
