"""Continuous-batching server loop over the libsph pool (host logic only).

Requests (SPH cases with an end time) arrive on a seeded Poisson trace.  The
server keeps one pool engine resident on the GPU; every loop iteration it

  1. moves requests whose arrival time has passed into the wait queue,
  2. admits waiting requests in FIFO order while the pool has a free slot and
     enough particle / cell-table memory (admission by free device memory:
     the pool's capacity is fixed from the free HBM when it is created),
  3. advances every admitted case by `chunk` Symplectic steps in one call
     (all cases share every kernel launch; each keeps its own dt and t),
  4. releases the cases that reached their end time and records their
     time-to-result (completion - arrival, queueing included).

So requests that arrive while others run are admitted as soon as a slot and
memory free up, and their work overlaps on the device with the running ones.
The same loop with a one-case pool is the plain one-case-at-a-time baseline.
The pool object only needs try_admit / pool_step / release / get_state, so the
loop is tested on the CPU with a fake pool.
"""
from collections import deque
from dataclasses import dataclass, field
import time


@dataclass
class Request:
    rid: int
    arrival: float           # seconds after the start of the run
    case: object             # cases.Case
    t_end: float             # simulated end time (s)
    admitted: float = -1.0
    done: float = -1.0
    slot: int = -1
    result: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def percentile(xs, q):
    """q-th percentile (0-100) by linear interpolation between order statistics."""
    s = sorted(xs)
    if not s:
        return float("nan")
    k = (len(s) - 1) * q / 100.0
    f = int(k)
    c = min(f + 1, len(s) - 1)
    return s[f] + (s[c] - s[f]) * (k - f)


class Server:
    def __init__(self, pool, chunk=10, clock=time.perf_counter, keep_results=False,
                 sleep=time.sleep):
        self.pool = pool
        self.chunk = int(chunk)
        self.clock = clock
        self.sleep = sleep
        self.keep_results = keep_results
        self.case_steps = 0

    def run(self, requests):
        """Serve the requests (sorted by arrival); returns them with times filled."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting = deque()
        active = {}
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting:
                r = waiting[0]
                slot = self.pool.try_admit(r.case, r.t_end)
                if slot is None:
                    break  # no slot or memory until a running case finishes
                waiting.popleft()
                r.slot = slot
                r.admitted = self.clock() - t0
                active[slot] = r
            if not active:
                if pending:  # idle until the next arrival
                    self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                    continue
                if waiting:
                    raise RuntimeError("request %d does not fit in an empty pool"
                                       % waiting[0].rid)
                break
            finished = self.pool.pool_step(self.chunk)
            self.case_steps += self.chunk * len(active)
            t_now = self.clock() - t0
            for slot in finished:
                r = active.pop(slot)
                r.done = t_now
                if self.keep_results:
                    r.result = self.pool.get_state(slot)
                self.pool.release(slot)
        return requests


def summary(requests, wall):
    lat = [r.latency for r in requests]
    return {"requests": len(requests), "wall_s": wall,
            "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
            "mean_s": sum(lat) / max(1, len(lat)),
            "throughput_req_s": len(requests) / wall if wall > 0 else float("nan")}
