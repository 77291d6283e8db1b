"""Serving and batched sweeps on the GPU: a job's result is the same alone
and in the served mix (continuous batching with other jobs of other sizes,
dimensionalities and species mixes), admission estimates bound the real
device bytes, the batched sweep runs every member to its own step count, and
the autotuner times candidates and caches its choice."""
import json

import numpy as np
import pytest

from paper_2501_07465_gb300 import inputs as I

from tests import pairs as PR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2501_07465_gb300 import pic
    pic.use_torch_allocator()
    yield


def _mix():
    s = I.SEED_BASE + 9
    jobs = [
        I.nanostructure2d(0, 64, "disk", 0.25, 5.0, 8, 500e-9, 150, s),
        I.nanostructure2d(1, 96, "bowtie", 0.2, 4.0, 6, 700e-9, 230, s),
        I._periodic_plasma(2, 2, 64, 120, s),
        I._metal3d(3, 64, 100, s),
        I._graphene(4, 64, 180, s),
        I._periodic_plasma(5, 3, 40, 90, s),
        I.nanostructure2d(6, 128, "rod", 0.3, 3.0, 4, 450e-9, 300, s),
    ]
    for k, wl in enumerate(jobs):
        wl["job"] = k
        wl["arrival"] = 0.004 * k
    return jobs


def test_alone_equals_mix():
    import torch

    from paper_2501_07465_gb300 import pic, runner, serve
    jobs = _mix()
    done, summ = serve.serve(jobs, hbm_budget=150e9, chunk=32, solo_chunk=16,
                             solo_bytes=30 << 20, result_fn=serve.fields_result)
    assert sorted(done) == list(range(len(jobs)))
    # continuous batching: several jobs were resident at once, in both kinds of lane
    assert summ["peak_resident_jobs"] >= 3
    assert summ["peak_resident_bytes"] > max(r["bytes"] for r in done.values())
    lanes = {r["lane"] for r in done.values()}
    assert lanes == {"group", "solo"}
    st = torch.cuda.current_stream().cuda_stream
    for wl in jobs:
        h = runner.make_sim(wl, st)
        try:
            pic.pic_step(h, wl["steps"])
            alone = serve.fields_result(h, wl)
        finally:
            pic.pic_destroy(h)
        mix = done[wl["job"]]["result"]
        assert mix["step"] == alone["step"] == wl["steps"]
        assert list(mix["count"]) == list(alone["count"])
        for c in range(6):
            a, b = mix["fields"][c], alone["fields"][c]
            if np.linalg.norm(b) > 0:
                assert PR.rel_l2(a, b) < 1e-4, (wl["name"], c, PR.rel_l2(a, b))
        for k, ke in enumerate(alone["kinetic"]):
            if ke > 0:
                assert abs(mix["kinetic"][k] - ke) <= 1e-5 * ke, (wl["name"], k)


def test_admission_estimate_bounds_device_bytes():
    from paper_2501_07465_gb300 import pic, runner
    for wl in _mix():
        h = runner.make_sim(wl, 0)
        try:
            got = pic.pic_memory_bytes(h)
        finally:
            pic.pic_destroy(h)
        est = runner.estimate_bytes(wl)
        assert got <= est <= 2 * got + (32 << 20), (wl["name"], got, est)


def test_tight_budget_serialises_but_completes():
    from paper_2501_07465_gb300 import runner, serve
    jobs = _mix()[:3]
    budget = max(runner.estimate_bytes(w) for w in jobs) + 1
    done, summ = serve.serve(jobs, hbm_budget=budget, chunk=64)
    assert sorted(done) == [0, 1, 2]
    assert summ["peak_resident_bytes"] <= budget
    for wl in jobs:
        assert done[wl["job"]]["result"]["step"] == wl["steps"]


def test_batch_sweep_and_serial_agree_on_step_counts():
    from paper_2501_07465_gb300 import batch, pic
    wls = I.batch2d(count=6)
    for wl in wls:
        wl["steps"] = wl["steps"] // 10
    b = batch.run_batch(wls, keep=True)
    s = batch.run_serial(wls, keep=True)
    try:
        for hb, hs, wl in zip(b["handles"], s["handles"], wls):
            db, ds = pic.pic_diagnostics(hb), pic.pic_diagnostics(hs)
            assert db["step"] == ds["step"] == wl["steps"]
            fb = PR.gpu_fields(hb, wl["grid"])
            fs = PR.gpu_fields(hs, wl["grid"])
            for c in range(6):
                if np.linalg.norm(fs[c]) > 0:
                    assert PR.rel_l2(fb[c], fs[c]) < 1e-4
    finally:
        for h in b["handles"] + s["handles"]:
            pic.pic_destroy(h)
    assert b["gpu_launches"] > 0 and s["gpu_launches"] > 0


def test_autotuner_times_and_caches(tmp_path, monkeypatch):
    from paper_2501_07465_gb300 import autotune
    monkeypatch.setenv("PIC_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    wls = I.batch2d(count=4)
    tiles = [(8, 8, 1), (16, 16, 1)]
    tun, entry = autotune.tune_group(wls, sample=4, steps=16, warm=16, tiles=tiles)
    assert not entry["cached"]
    assert tuple(tun["tile"]) in tiles
    assert len(entry["table"]) == len(tiles) + 2
    assert all(np.isfinite(r["ms"]) and r["ms"] > 0 for r in entry["table"])
    tun2, entry2 = autotune.tune_group(wls, sample=4, steps=16, warm=16, tiles=tiles)
    assert entry2["cached"] and tun2 == tun
    data = json.load(open(tmp_path / "tune.json"))
    assert len(data) == 1
