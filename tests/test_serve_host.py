"""Host logic of the continuous-batching server, with a fake pool (no GPU)."""
import itertools

import pytest

from paper_2104_00537_gb300 import serve


class FakeCase:
    def __init__(self, n, steps):
        self.n = n
        self.steps = steps  # steps needed to reach t_end


class FakePool:
    """Pool with a particle budget and slots; a case finishes after its steps."""

    def __init__(self, max_particles, max_cases, clock):
        self.max_p, self.max_c = max_particles, max_cases
        self.used_p = 0
        self.active = {}
        self.clock = clock
        self.admit_log = []
        self.max_concurrent = 0

    def try_admit(self, case, t_end):
        if len(self.active) >= self.max_c or self.used_p + case.n > self.max_p:
            return None
        slot = next(s for s in itertools.count() if s not in self.active)
        self.active[slot] = [case, 0]
        self.used_p += case.n
        self.admit_log.append((case, self.clock.t))
        self.max_concurrent = max(self.max_concurrent, len(self.active))
        return slot

    def pool_step(self, k):
        self.clock.t += 0.001 * k  # the device time of k steps
        done = []
        for s, v in self.active.items():
            v[1] += k
            if v[1] >= v[0].steps:
                done.append(s)
        return done

    def release(self, slot):
        case, _ = self.active.pop(slot)
        self.used_p -= case.n

    def get_state(self, slot):
        return {"slot": slot}


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


def make(reqs):
    return [serve.Request(i, a, FakeCase(n, s), 1.0) for i, (a, n, s) in enumerate(reqs)]


def test_requests_overlap_and_all_finish():
    clk = Clock()
    pool = FakePool(1000, 4, clk)
    reqs = make([(0.0, 300, 50), (0.01, 300, 50), (0.02, 300, 50), (0.5, 100, 10)])
    srv = serve.Server(pool, chunk=10, clock=clk, sleep=clk.sleep)
    srv.run(reqs)
    assert all(r.done > r.arrival for r in reqs)
    assert pool.max_concurrent == 3          # the three early requests ran together
    assert pool.used_p == 0 and not pool.active
    # the late request arrived after the others finished, so it did not wait
    assert reqs[3].admitted == pytest.approx(reqs[3].arrival)


def test_admission_waits_for_memory_fifo():
    clk = Clock()
    pool = FakePool(500, 8, clk)
    reqs = make([(0.0, 400, 30), (0.0, 400, 30), (0.0, 50, 30)])
    srv = serve.Server(pool, chunk=10, clock=clk, sleep=clk.sleep)
    srv.run(reqs)
    # FIFO: request 1 does not fit next to request 0; request 2 may not jump the queue
    assert reqs[1].admitted >= reqs[0].done
    assert reqs[2].admitted >= reqs[1].admitted
    assert pool.max_concurrent == 2


def test_plain_pool_serialises():
    clk = Clock()
    pool = FakePool(10 ** 6, 1, clk)
    reqs = make([(0.0, 10, 20), (0.0, 10, 20), (0.0, 10, 20)])
    serve.Server(pool, chunk=10, clock=clk, sleep=clk.sleep).run(reqs)
    assert pool.max_concurrent == 1
    assert reqs[0].done < reqs[1].done < reqs[2].done


def test_oversized_request_is_an_error():
    clk = Clock()
    pool = FakePool(100, 4, clk)
    with pytest.raises(RuntimeError):
        serve.Server(pool, chunk=10, clock=clk, sleep=clk.sleep).run(make([(0.0, 500, 10)]))


def test_percentiles():
    xs = list(range(1, 101))
    assert serve.percentile(xs, 50) == pytest.approx(50.5)
    assert serve.percentile(xs, 99) == pytest.approx(99.01)
    s = serve.summary(make([(0.0, 1, 1)] * 0), 1.0)
    assert s["requests"] == 0


def test_trace_is_seeded_and_poisson_shaped():
    from paper_2104_00537_gb300 import cases
    a = cases.sloshing_trace(40, rate=20.0, seed=3, n_min=2000, n_max=4000, t_end=0.1)
    b = cases.sloshing_trace(40, rate=20.0, seed=3, n_min=2000, n_max=4000, t_end=0.1)
    assert [x[0] for x in a] == [x[0] for x in b]
    gaps = [a[i + 1][0] - a[i][0] for i in range(len(a) - 1)]
    assert all(g > 0 for g in gaps)
    assert 0.02 < sum(gaps) / len(gaps) < 0.09  # mean 1/20 s
    assert all(2000 * 0.5 < c.n_fluid < 4000 * 1.6 for _, c, _ in a)
