"""Scheduler of the continuous-batching server, on CPU with a fake engine and a
virtual clock: admission by memory budget in arrival order, batches of one
(model, m, stage) group, stage order, and interleaving of requests that arrive
while others are in flight."""
import numpy as np
import pytest

from paper_2508_19525_b300.serving import Request, Server, STAGES, bucket, percentile


class FakeEngine:
    """Every iteration costs `base + per * batch` virtual seconds."""

    def __init__(self, clock, base=0.010, per=0.002, foot=100):
        self.clock, self.base, self.per, self.foot = clock, base, per, foot
        self.used_trace = []
        self.log = []
        self.server = None

    def footprint(self, r):
        return self.foot * (r.m // 16)

    def admit(self, r):
        self.log.append(("admit", r.rid))

    def run(self, key, batch):
        assert len({(r.model, r.m, r.stage) for r in batch}) == 1
        assert (batch[0].model, batch[0].m, batch[0].stage) == key
        self.log.append(("run", key, [r.rid for r in batch]))
        self.clock.t += self.base + self.per * len(batch)
        self.used_trace.append(self.server.used)

    def release(self, r):
        self.log.append(("release", r.rid))

    def idle(self, seconds):
        self.clock.t += max(seconds, 1e-6)


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def make_requests(n, rate, seed, buckets=(32, 64, 128)):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        seq = int(rng.integers(16, max(buckets) + 1))
        out.append(Request(rid=i, client_seed=100 + i, model="bert" if i % 2 else "gpt2", seq=seq,
                           m=bucket(seq, buckets), arrival=t))
    return out


def test_bucket():
    assert bucket(16, (32, 64)) == 32 and bucket(33, (32, 64)) == 64 and bucket(64, (64, 32)) == 64
    with pytest.raises(ValueError):
        bucket(65, (32, 64))


@pytest.mark.parametrize("rate,budget,max_batch", [(20, 10_000, 8), (200, 1500, 4), (1000, 800, 8)])
def test_every_request_finishes_within_budget(rate, budget, max_batch):
    clock = Clock()
    eng = FakeEngine(clock)
    srv = Server(eng, budget_bytes=budget, max_batch=max_batch)
    eng.server = srv
    reqs = make_requests(40, rate, seed=rate)
    done = srv.run(reqs, clock=clock)
    assert sorted(r.rid for r in done) == list(range(40))
    assert max(eng.used_trace) <= budget
    assert srv.used == 0
    for r in done:
        assert r.stage == STAGES and r.arrival <= r.admitted <= r.done
    # admission in arrival order
    admits = [e[1] for e in eng.log if e[0] == "admit"]
    assert admits == sorted(admits, key=lambda i: (reqs[i].arrival, i))
    # each request runs its stages in order, once each
    for r in reqs:
        stages = [e[1][2] for e in eng.log if e[0] == "run" and r.rid in e[2]]
        assert stages == list(range(STAGES))
    assert all(n <= max_batch for _, n in srv.iterations)


def test_requests_interleave_and_batch_under_load():
    clock = Clock()
    eng = FakeEngine(clock, base=0.05, per=0.001)
    srv = Server(eng, budget_bytes=100_000, max_batch=8)
    eng.server = srv
    reqs = make_requests(60, rate=400, seed=7, buckets=(64,))
    for r in reqs:
        r.model = "bert"
    srv.run(reqs, clock=clock)
    # under load, batches form, and stage-0 work of later arrivals runs between
    # the stages of earlier ones
    assert max(n for _, n in srv.iterations) > 1
    first_done = min(r.done for r in reqs)
    assert any(r.admitted < first_done and r.rid > 8 for r in reqs)
    lat = [r.latency for r in reqs]
    assert percentile(lat, 50) <= percentile(lat, 99)


def test_oversized_request_is_refused():
    clock = Clock()
    eng = FakeEngine(clock, foot=10_000)
    srv = Server(eng, budget_bytes=100)
    eng.server = srv
    with pytest.raises(ValueError):
        srv.run(make_requests(1, 10, seed=1), clock=clock)
