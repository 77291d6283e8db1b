"""Batched sweeps: many independent simulations advanced together by the
batch engine (pic_group_*: one particle launch and one field launch per step
for all members, CUDA-graph replay between re-sorts), against the plain
single-simulation path (pic_step on each simulation in turn).

Both runs build every simulation first (not timed) and then time the
stepping of all of them to their own step counts with CUDA events on the
stream they run on; sims/hour = simulations / timed seconds x 3600."""
from __future__ import annotations

from . import pic, runner


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_batch(workloads, tuning=None, use_graph=1, chunk=None, keep=False):
    """Step every workload to its own step count in one group.  Returns a
    dict with the timed seconds, sims/hour, particle-steps/s, kernel launches
    and (keep=True) the handles, still loaded, for inspection."""
    import torch
    st = torch.cuda.Stream()
    hs = []
    g = pic.pic_group_create(len(workloads), 0, st.cuda_stream, use_graph)
    try:
        psteps = 0
        for wl in workloads:
            h = runner.make_sim(wl, 0, tuning)
            hs.append(h)
            pic.pic_group_add(g, h, wl["steps"])
            psteps += sum(pic.pic_diagnostics(h)["count"]) * wl["steps"]
        torch.cuda.synchronize()
        nmax = max(wl["steps"] for wl in workloads)
        l0 = pic.pic_group_info(g)["launches"]
        e0, e1 = _events()
        e0.record(st)
        left = nmax
        while left > 0:  # the host never waits inside the timed region
            n = min(left, chunk or left)
            pic.pic_group_step(g, n)
            left -= n
        e1.record(st)
        e1.synchronize()
        pic.pic_group_sync(g)
        sec = e0.elapsed_time(e1) / 1e3
        info = pic.pic_group_info(g)
        for h, wl in zip(hs, workloads):
            d = pic.pic_diagnostics(h)
            if d["step"] != wl["steps"]:
                raise RuntimeError(f"{wl['name']}: {d['step']} steps, expected {wl['steps']}")
        out = {"sims": len(workloads), "seconds": sec, "sims_per_hour": len(workloads) / sec * 3600,
               "particle_steps_per_s": psteps / sec, "group_steps": nmax,
               "gpu_launches": info["launches"] - l0, "member_bytes": info["member_bytes"]}
    finally:
        pic.pic_group_destroy(g)
        if not keep:
            for h in hs:
                pic.pic_destroy(h)
    if keep:
        out["handles"] = hs
    return out


def run_serial(workloads, tuning=None, keep=False):
    """Step each workload alone (pic_step), one after the other, all on one
    stream."""
    import torch
    st = torch.cuda.current_stream()
    hs = []
    try:
        psteps = 0
        for wl in workloads:
            h = runner.make_sim(wl, st.cuda_stream, tuning)
            hs.append(h)
            psteps += sum(pic.pic_diagnostics(h)["count"]) * wl["steps"]
            pic.pic_get_timing(h)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record(st)
        for h, wl in zip(hs, workloads):
            pic.pic_step(h, wl["steps"])
        e1.record(st)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        launches = 0
        for h in hs:
            launches += pic.pic_get_timing(h)["kernel_launches"]
        out = {"sims": len(workloads), "seconds": sec, "sims_per_hour": len(workloads) / sec * 3600,
               "particle_steps_per_s": psteps / sec, "gpu_launches": launches}
    finally:
        if not keep:
            for h in hs:
                pic.pic_destroy(h)
    if keep:
        out["handles"] = hs
    return out
