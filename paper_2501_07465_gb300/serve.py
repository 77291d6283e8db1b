"""Serving loop: simulation jobs arrive over time, are admitted while their
device state fits an HBM budget, and advance concurrently (continuous
batching) until each has taken its own number of steps.

Jobs go to one of two kinds of lane, by their per-step cost (bytes a step
moves: 48 B per cell + 60 B per particle):
  * small jobs join the batch-engine group of their dimensionality (2D and 3D
    cannot share the particle tile): all members advance together, a chunk
    of steps at a time, with one particle and one field launch per step and
    CUDA-graph replay; the two groups run on high-priority streams so that
    their short kernels are scheduled ahead of the long ones;
  * large jobs, whose kernels fill the GPU on their own, each get a solo lane:
    their own stream, stepped by pic_step a chunk at a time.
The loop never waits for the whole device: every lane has at most one chunk
in flight, marked by a CUDA event; when a lane's event has completed the loop
retires that lane's finished jobs (the result function reads what the caller
wants, the handle leaves its group and is destroyed, its bytes are released)
and enqueues the lane's next chunk.  Arrived jobs are admitted first come,
first served while the resident bytes plus the job's estimated bytes stay
within the budget.  A job's latency runs from its arrival to the moment the
loop sees its last chunk complete.  The serial reference runs the same jobs
one at a time, in arrival order, through the plain single-simulation path
(pic_step).

    python -m paper_2501_07465_gb300.serve --jobs 40 --rate 2
"""
from __future__ import annotations

import argparse
import collections
import json
import time

from . import inputs, pic, runner

SOLO_BYTES = 64 << 20  # per-step bytes above which a job gets a lane of its own


def step_bytes(wl):
    return 48 * runner.cells(wl) + 60 * runner.particles(wl)


def diagnostics_result(h, wl):
    return pic.pic_diagnostics(h)


def fields_result(h, wl):
    """Diagnostics and the six field components (FP64 host arrays)."""
    d = pic.pic_diagnostics(h)
    d["fields"] = pic.pic_read_fields(h, 63, inputs.grid_shape(wl["grid"]["n"]))
    return d


def _pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q * (len(xs) - 1)))))
    return xs[k]


def _summary(jobs, done, t_first, t_last, mode):
    lat = [done[j["job"]]["latency"] for j in jobs]
    span = t_last - t_first
    return {"mode": mode, "jobs": len(jobs), "seconds": span,
            "sims_per_hour": len(jobs) / span * 3600 if span > 0 else None,
            "p50_latency_s": _pct(lat, 0.50), "p99_latency_s": _pct(lat, 0.99),
            "mean_latency_s": sum(lat) / len(lat)}


def _torch_stream(priority=0):
    import torch
    return torch.cuda.Stream(priority=priority)


def _torch_event():
    import torch
    return torch.cuda.Event()


class _Lane:
    def __init__(self, stream, group=None):
        self.stream = stream
        self.group = group
        self.members = {}  # handle -> [workload, bytes, steps left to enqueue (solo)]
        self.event = None  # completion of the chunk in flight


class Server:
    def __init__(self, hbm_budget=150e9, capacity=256, chunk=64, solo_chunk=32, use_graph=1,
                 tuning=None, result_fn=diagnostics_result, solo_bytes=SOLO_BYTES,
                 stream_factory=None, event_factory=None):
        self.stream_factory = stream_factory or _torch_stream
        self.event_factory = event_factory or _torch_event
        self.budget = int(hbm_budget)
        self.chunk = chunk
        self.solo_chunk = solo_chunk
        self.solo_bytes = solo_bytes
        self.tuning = tuning or {}
        self.result_fn = result_fn
        self.capacity = capacity
        self.loader = self.stream_factory(0)
        self.groups = {}
        for d in (2, 3):
            st = self.stream_factory(-1)
            self.groups[d] = _Lane(st, pic.pic_group_create(capacity, self.budget, st.cuda_stream,
                                                            use_graph))
        self.solos = []
        self.resident = 0
        self.peak_resident = 0
        self.peak_jobs = 0
        self.chunks = 0

    def close(self):
        for lane in list(self.groups.values()) + self.solos:
            for h in list(lane.members):
                if lane.group is not None:
                    pic.pic_group_remove(lane.group, h)
                pic.pic_destroy(h)
            lane.members.clear()
        for lane in self.groups.values():
            pic.pic_group_destroy(lane.group)
        self.groups = {}
        self.solos = []

    def _jobs_resident(self):
        return sum(len(l.members) for l in list(self.groups.values()) + self.solos)

    def _admit(self, queue):
        while queue:
            wl = queue[0]
            est = runner.estimate_bytes(wl)
            if self.resident + est > self.budget:
                if self._jobs_resident() == 0:
                    raise RuntimeError(f"{wl['name']} does not fit the HBM budget alone")
                return
            if step_bytes(wl) > self.solo_bytes:
                lane = _Lane(self.stream_factory(0))
                h = runner.make_sim(wl, lane.stream.cuda_stream, self.tuning.get(wl["grid"]["dims"]))
                self.solos.append(lane)
            else:
                lane = self.groups[wl["grid"]["dims"]]
                if len(lane.members) >= self.capacity:
                    return
                h = runner.make_sim(wl, self.loader.cuda_stream, self.tuning.get(wl["grid"]["dims"]))
                pic.pic_sync(h)
                pic.pic_group_add(lane.group, h, wl["steps"])  # waits for the lane's chunk
            b = pic.pic_memory_bytes(h)
            lane.members[h] = [wl, b, wl["steps"]]
            self.resident += b
            self.peak_resident = max(self.peak_resident, self.resident)
            self.peak_jobs = max(self.peak_jobs, self._jobs_resident())
            queue.popleft()

    def _launch(self, lane):
        if lane.group is not None:
            pic.pic_group_step(lane.group, self.chunk)
        else:
            (h, m), = lane.members.items()
            n = min(self.solo_chunk, m[2])
            pic.pic_step(h, n)
            m[2] -= n
        lane.event = self.event_factory()
        lane.event.record(lane.stream)
        self.chunks += 1

    def _retire(self, lane, t_end, done):
        for h in list(lane.members):
            wl, b, left = lane.members[h]
            if lane.group is not None:
                finished = pic.pic_group_progress(lane.group, h)[1] == 0
            else:
                finished = left == 0
            if not finished:
                continue
            del lane.members[h]
            res = self.result_fn(h, wl)
            if lane.group is not None:
                pic.pic_group_remove(lane.group, h)
            pic.pic_destroy(h)
            self.resident -= b
            done[wl["job"]] = {"latency": t_end - wl["arrival"], "finish": t_end, "result": res,
                               "bytes": b, "lane": "group" if lane.group is not None else "solo"}

    def run(self, jobs, clock=time.perf_counter, idle_sleep=1e-4):
        """Serve `jobs` (each with an "arrival" offset in seconds); returns
        (per-job records keyed by job id, summary)."""
        pending = collections.deque(sorted(jobs, key=lambda j: j["arrival"]))
        queue = collections.deque()
        done = {}
        t0 = clock()
        while len(done) < len(jobs):
            now = clock() - t0
            while pending and pending[0]["arrival"] <= now:
                queue.append(pending.popleft())
            self._admit(queue)
            progressed = False
            for lane in list(self.groups.values()) + self.solos:
                if lane.event is not None:
                    if not lane.event.query():
                        continue
                    lane.event = None
                    self._retire(lane, clock() - t0, done)
                    progressed = True
                if lane.members:
                    self._launch(lane)
                    progressed = True
            self.solos = [l for l in self.solos if l.members or l.event is not None]
            if not progressed:
                if self._jobs_resident() == 0 and pending and not queue:
                    time.sleep(max(0.0, pending[0]["arrival"] - (clock() - t0)))
                else:
                    time.sleep(idle_sleep)
        t_last = max(r["finish"] for r in done.values())
        s = _summary(jobs, done, min(j["arrival"] for j in jobs), t_last, "continuous batching")
        s.update(chunks=self.chunks, peak_resident_bytes=self.peak_resident,
                 peak_resident_jobs=self.peak_jobs, budget_bytes=self.budget, chunk=self.chunk,
                 solo_chunk=self.solo_chunk, solo_jobs=sum(1 for r in done.values()
                                                           if r["lane"] == "solo"))
        return done, s


def serve(jobs, **kw):
    srv = Server(**kw)
    try:
        return srv.run(jobs)
    finally:
        srv.close()


def serve_serial(jobs, tuning=None, result_fn=diagnostics_result, clock=time.perf_counter):
    """The same jobs one at a time through pic_step, in arrival order."""
    import torch
    st = torch.cuda.current_stream()
    done = {}
    t0 = clock()
    for wl in sorted(jobs, key=lambda j: j["arrival"]):
        wait = wl["arrival"] - (clock() - t0)
        if wait > 0:
            time.sleep(wait)
        h = runner.make_sim(wl, st.cuda_stream, (tuning or {}).get(wl["grid"]["dims"]))
        try:
            pic.pic_step(h, wl["steps"])
            pic.pic_sync(h)
            t_end = clock() - t0
            res = result_fn(h, wl)
        finally:
            pic.pic_destroy(h)
        done[wl["job"]] = {"latency": t_end - wl["arrival"], "finish": t_end, "result": res}
    t_last = max(r["finish"] for r in done.values())
    return done, _summary(jobs, done, min(j["arrival"] for j in jobs), t_last, "serial")


def serial_service_times(jobs, tuning=None, clock=time.perf_counter, sample_steps=None):
    """Each job run alone through pic_step, back to back, in arrival order:
    its service time (create, load, steps, diagnostics, destroy).  With
    sample_steps, a job longer than that runs sample_steps steps and its
    steps' time is scaled to its full step count (a step of one simulation
    costs the same all through its run; the sample spans whole re-sort
    intervals); the create, load, diagnostics and destroy are measured as
    they are."""
    import torch
    st = torch.cuda.current_stream()
    out = {}
    for wl in sorted(jobs, key=lambda j: j["arrival"]):
        t0 = clock()
        h = runner.make_sim(wl, st.cuda_stream, (tuning or {}).get(wl["grid"]["dims"]))
        try:
            pic.pic_sync(h)
            t1 = clock()
            n = wl["steps"] if not sample_steps else min(wl["steps"], sample_steps)
            pic.pic_step(h, n)
            pic.pic_sync(h)
            t2 = clock()
            diagnostics_result(h, wl)
        finally:
            pic.pic_destroy(h)
        t3 = clock()
        out[wl["job"]] = (t1 - t0) + (t2 - t1) * wl["steps"] / max(n, 1) + (t3 - t2)
    return out


def serial_queue(jobs, service):
    """One server, first come first served: job j starts when it has arrived
    and the previous job has finished, and takes its measured service time.
    The same summary as serve_serial, without running the jobs again (the
    service time of a job run alone does not depend on when it arrives)."""
    done = {}
    free_at = 0.0
    for wl in sorted(jobs, key=lambda j: j["arrival"]):
        start = max(wl["arrival"], free_at)
        free_at = start + service[wl["job"]]
        done[wl["job"]] = {"latency": free_at - wl["arrival"], "finish": free_at}
    t_last = max(r["finish"] for r in done.values())
    return done, _summary(jobs, done, min(j["arrival"] for j in jobs), t_last,
                          "serial (measured service times, FIFO)")


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--jobs", type=int, default=40)
    ap.add_argument("--rate", type=float, nargs="+", default=[2.0])
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--no-serial", action="store_true")
    args = ap.parse_args()
    import torch

    from . import build as libbuild
    libbuild.build()
    torch.cuda.set_device(0)
    pic.use_torch_allocator()
    for rate in args.rate:
        jobs = inputs.serve_jobs(args.jobs, rate)
        _, s = serve(jobs, hbm_budget=args.budget_gb * 1e9, chunk=args.chunk)
        line = {"rate_per_s": rate, "served": s}
        if not args.no_serial:
            _, line["serial"] = serve_serial(jobs)
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
