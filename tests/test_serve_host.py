"""Host-side logic of the served form, with a fake executor and clock (no GPU):
HBM-budget admission, slot reuse, continuous batching of requests that arrive
while a round is running, latency accounting and percentiles."""
import numpy as np
import pytest

from paper_2506_09226_gb300 import datagen, serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4          # every look at the clock advances it
        return self.t


class FakeExecutor:
    """Rounds take `dur` seconds of fake time; one round at a time."""

    def __init__(self, clock, dur=0.01, cost=100):
        self.clock, self.dur, self.c = clock, dur, cost
        self.rounds, self.running = [], 0

    def cost(self, r):
        return self.c

    def can_launch(self):
        return self.running == 0

    def launch(self, reqs):
        self.rounds.append([r.rid for r in reqs])
        self.running += 1
        end = self.clock.t + self.dur
        ex = self

        class H:
            def done(self):
                return ex.clock.t >= end

            def close(self):
                ex.running -= 1
        return H()


def test_percentile_nearest_rank():
    xs = list(range(1, 101))
    assert serve.percentile(xs, 50) == 50 and serve.percentile(xs, 99) == 99
    assert serve.percentile([7.0], 99) == 7.0


def test_admission_budget_and_slots():
    a = serve.Admission(budget_bytes=250, slots=3)
    s1, s2 = a.try_admit(100), a.try_admit(100)
    assert s1 is not None and s2 is not None and s1 != s2
    assert a.try_admit(100) is None                       # budget
    a.release(s1, 100)
    s3 = a.try_admit(100)
    assert s3 not in (s1, s2) and a.used == 200 and a.busy == 2     # least recently used slot first
    a.release(s2, 100)
    a.release(s3, 100)
    assert a.try_admit(100) == s1
    b = serve.Admission(budget_bytes=10 ** 9, slots=1)
    assert b.try_admit(1) is not None and b.try_admit(1) is None   # slots


def test_continuous_batching_with_fake_executor():
    clock = FakeClock()
    trace = datagen.poisson_trace(1.0, 500.0, [10 ** 6], seed=3, n_lo=10, n_hi=100)
    ex = FakeExecutor(clock, dur=0.02)
    adm = serve.Admission(budget_bytes=10 ** 9, slots=10 ** 4)
    st = serve.serve_loop(trace, ex, adm, clock=clock, idle_sleep=0)
    assert len(st.latencies_ms) == len(trace)
    assert sorted(r for rd in ex.rounds for r in rd) == list(range(len(trace)))
    assert st.rounds == len(ex.rounds) < len(trace)       # arrivals during a round join the next one
    assert max(len(r) for r in ex.rounds) > 1
    assert min(st.latencies_ms) >= 0 and st.max_inflight >= max(len(r) for r in ex.rounds)
    assert adm.used == 0 and adm.busy == 0                # everything released


def test_admission_limits_inflight():
    clock = FakeClock()
    trace = [datagen.Arrival(0.0, 0, 0, 10, 100) for _ in range(50)]
    ex = FakeExecutor(clock, dur=0.01, cost=100)
    adm = serve.Admission(budget_bytes=1000, slots=10 ** 4)    # at most 10 in flight
    st = serve.serve_loop(trace, ex, adm, clock=clock, idle_sleep=0)
    assert len(st.latencies_ms) == 50 and st.max_inflight == 10
    assert all(len(r) <= 10 for r in ex.rounds) and len(ex.rounds) == 5


def test_poisson_trace_rate_and_ranges():
    tr = datagen.poisson_trace(20.0, 2000.0, [10 ** 9, 5 * 10 ** 8], seed=5)
    rate = len(tr) / 20.0
    assert abs(rate - 2000) < 5 * np.sqrt(2000 / 20.0) * 2
    assert all(0 <= a.offset and a.offset + a.n <= (10 ** 9 if a.shape == 0 else 5 * 10 ** 8) for a in tr)
    assert all(int(0.01 * 2557) - 1 <= a.date_hi <= int(0.9 * 2557) + 1 for a in tr)
    assert all(tr[i].t <= tr[i + 1].t for i in range(len(tr) - 1))


def test_row_cap_keeps_rounds_short():
    clock = FakeClock()
    sizes = [10, 10, 500, 10, 10, 10]
    trace = [datagen.Arrival(0.0, 0, 0, n, 100) for n in sizes]
    ex = FakeExecutor(clock, dur=0.01)
    adm = serve.Admission(budget_bytes=10 ** 9, slots=100)
    serve.serve_loop(trace, ex, adm, clock=clock, idle_sleep=0, row_cap=100)
    assert ex.rounds == [[0, 1], [2], [3, 4, 5]]        # oldest first; the big one alone


def test_cancel_frees_slot_and_budget():
    """Cancellation at each stage: before admission (dropped, never run),
    admitted but not launched (slot and budget returned at once, and a
    waiting request takes them), and in flight (kept until its round
    completes, then released, its result not counted)."""
    clock = FakeClock()
    # rounds of one request (row_cap): request 0 runs first; 1 and 2 wait
    trace = [datagen.Arrival(0.0, 0, 0, 10, 100) for _ in range(4)]
    ex = FakeExecutor(clock, dur=0.05, cost=100)
    adm = serve.Admission(budget_bytes=200, slots=2)        # two in flight at most
    released = []
    orig = adm.release

    def spy(slot, cost):
        released.append((round(clock.t, 4), slot))
        orig(slot, cost)
    adm.release = spy
    # 0 and 1 are admitted at once; 0 launches, 1 waits in `ready` behind the
    # running round; cancel 1 then (its slot goes to 2); cancel 3 before it
    # is admitted; cancel 0 while its round runs
    st = serve.serve_loop(trace, ex, adm, clock=clock, idle_sleep=0, row_cap=10,
                          cancel_at={1: 0.01, 3: 0.011, 0: 0.02})
    assert st.cancelled == 3
    launched = [r for rd in ex.rounds for r in rd]
    assert 1 not in launched and 3 not in launched          # never ran
    assert 0 in launched and 2 in launched
    assert len(st.latencies_ms) == 1 and st.rows == 10       # only request 2 counts
    assert adm.used == 0 and adm.busy == 0                  # everything released
    # request 1's slot came back before round 0 finished, and request 2 took it
    t_rel1 = [t for t, s in released][0]
    assert t_rel1 < 0.05
    assert ex.rounds[0] == [0] and ex.rounds[1] == [2]


def test_cancel_unknown_or_finished_is_ignored():
    clock = FakeClock()
    trace = [datagen.Arrival(0.0, 0, 0, 10, 100) for _ in range(3)]
    ex = FakeExecutor(clock, dur=0.001, cost=1)
    adm = serve.Admission(budget_bytes=10, slots=10)
    st = serve.serve_loop(trace, ex, adm, clock=clock, idle_sleep=0, cancel_at={2: 5.0})
    assert st.cancelled == 0 and len(st.latencies_ms) == 3
    assert adm.used == 0 and adm.busy == 0


def test_gc_paused_restores_the_collector():
    import gc
    assert gc.isenabled()
    with serve.gc_paused():
        assert not gc.isenabled()
    assert gc.isenabled() and gc.get_freeze_count() == 0
    try:
        with serve.gc_paused():
            raise RuntimeError("leaves the loop")
    except RuntimeError:
        pass
    assert gc.isenabled() and gc.get_freeze_count() == 0
