"""Host logic of the serving loop (admission by HBM budget, FIFO order,
continuous batching, retirement, latency bookkeeping) against a fake of the
library's group calls: no GPU needed."""
import itertools
import types

import pytest

from paper_2501_07465_gb300 import serve


class FakeLib:
    """Simulated simulations: a member advances one step per group step
    until it reaches its target (the contract of pic_group_step)."""

    def __init__(self):
        self.ids = itertools.count(1)
        self.sims = {}
        self.groups = {}
        self.max_members = 0
        self.events = []
        self.solo_steps = 0

    # group calls
    def pic_group_create(self, capacity, budget, stream, use_graph):
        g = next(self.ids)
        self.groups[g] = {"members": {}, "budget": budget}
        return g

    def pic_group_destroy(self, g):
        del self.groups[g]

    def pic_group_add(self, g, h, nsteps):
        G = self.groups[g]
        if G["budget"] and sum(self.sims[m]["bytes"] for m in G["members"]) + self.sims[h]["bytes"] > G["budget"]:
            raise AssertionError("server admitted past the budget")
        G["members"][h] = [0, nsteps]
        self.sims[h]["group"] = g
        self.events.append(("add", self.sims[h]["job"]))

    def pic_group_remove(self, g, h):
        del self.groups[g]["members"][h]
        self.sims[h]["group"] = None
        self.events.append(("remove", self.sims[h]["job"]))

    def pic_group_step(self, g, n):
        for h, (d, t) in self.groups[g]["members"].items():
            self.groups[g]["members"][h][0] = min(t, d + n)
        total = sum(len(G["members"]) for G in self.groups.values())
        self.max_members = max(self.max_members, total)

    def pic_group_sync(self, g):
        pass

    def pic_group_progress(self, g, h):
        d, t = self.groups[g]["members"][h]
        return d, t - d

    # simulation calls
    def pic_sync(self, h):
        pass

    def pic_memory_bytes(self, h):
        return self.sims[h]["bytes"]

    def pic_diagnostics(self, h):
        s = self.sims[h]
        d = self.groups[s["group"]]["members"][h][0] if s["group"] else s["steps"]
        return {"step": d, "job": s["job"]}

    def pic_step(self, h, n):
        assert self.sims[h]["group"] is None, "a group member stepped on its own"
        self.sims[h]["steps"] += n
        self.solo_steps += n

    def pic_destroy(self, h):
        assert self.sims[h]["group"] is None, "destroyed while in a group"
        del self.sims[h]

    def make_sim(self, wl, stream, tuning):
        h = next(self.ids)
        self.sims[h] = {"bytes": wl["bytes"], "job": wl["job"], "group": None, "steps": 0}
        return h


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(serve, "pic", lib)
    monkeypatch.setattr(serve, "runner", types.SimpleNamespace(
        make_sim=lib.make_sim, estimate_bytes=lambda wl: wl["bytes"]))
    monkeypatch.setattr(serve, "step_bytes", lambda wl: wl.get("cost", 0))
    return lib


def _jobs(spec):
    return [dict(job=k, name=f"j{k}", arrival=a, steps=s, bytes=b, grid=dict(dims=d))
            for k, (a, s, b, d) in enumerate(spec)]


class Clock:
    """Deterministic clock: every reading advances 1 ms."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


def _fake_stream(priority=0):
    return types.SimpleNamespace(cuda_stream=0)


class _FakeEvent:
    """A chunk completes as soon as it is enqueued."""

    def record(self, stream):
        pass

    def query(self):
        return True


def _server(**kw):
    return serve.Server(stream_factory=_fake_stream, event_factory=_FakeEvent, **kw)


def test_all_jobs_complete_with_their_step_counts(fake):
    jobs = _jobs([(0.0, 100, 10, 2), (0.0, 300, 10, 3), (0.001, 64, 10, 2), (0.002, 500, 10, 2)])
    srv = _server(hbm_budget=1000, chunk=64)
    done, s = srv.run(jobs, clock=Clock())
    srv.close()
    assert sorted(done) == [0, 1, 2, 3]
    for j in jobs:
        assert done[j["job"]]["result"]["step"] == j["steps"]
        assert done[j["job"]]["latency"] > 0
    assert fake.max_members >= 3  # jobs overlapped on the device
    assert s["p50_latency_s"] <= s["p99_latency_s"]


def test_budget_bounds_resident_bytes_and_keeps_fifo(fake):
    # three jobs of 60 bytes under a budget of 100: at most one resident
    jobs = _jobs([(0.0, 64, 60, 2), (0.0, 64, 60, 2), (0.0, 64, 60, 3)])
    srv = _server(hbm_budget=100, chunk=64)
    done, s = srv.run(jobs, clock=Clock())
    srv.close()
    assert s["peak_resident_bytes"] <= 100
    assert fake.max_members == 1
    adds = [j for e, j in fake.events if e == "add"]
    assert adds == [0, 1, 2]  # first come, first admitted


def test_job_larger_than_budget_is_an_error(fake):
    jobs = _jobs([(0.0, 64, 500, 2)])
    srv = _server(hbm_budget=100, chunk=64)
    with pytest.raises(RuntimeError):
        srv.run(jobs, clock=Clock())
    srv.close()


def test_latency_counts_from_arrival(fake):
    jobs = _jobs([(0.0, 64, 10, 2), (0.05, 64, 10, 2)])
    srv = _server(hbm_budget=1000, chunk=64)
    done, s = srv.run(jobs, clock=Clock())
    srv.close()
    assert done[1]["finish"] >= 0.05
    assert abs(done[1]["latency"] - (done[1]["finish"] - 0.05)) < 1e-12
    assert s["jobs"] == 2 and s["sims_per_hour"] > 0


def test_large_jobs_take_solo_lanes(fake):
    # job 1 is above the per-step cost threshold: stepped alone, in chunks
    jobs = _jobs([(0.0, 100, 10, 2), (0.0, 70, 10, 3), (0.0, 64, 10, 3)])
    jobs[1]["cost"] = 10 ** 12
    srv = _server(hbm_budget=1000, chunk=64, solo_chunk=32)
    done, s = srv.run(jobs, clock=Clock())
    srv.close()
    assert done[1]["lane"] == "solo" and done[0]["lane"] == done[2]["lane"] == "group"
    assert fake.solo_steps == 70
    assert done[1]["result"]["step"] == 70
    assert s["solo_jobs"] == 1
