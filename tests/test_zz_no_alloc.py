"""pic_cell_counts_noalloc: per-cell particle counts for callers that must
not allocate device memory while they run (CUDA-graph capture, memory
handed to a fixed pool, latency-sensitive serving loops).

It counts into a fixed array built into the library instead of a buffer
allocated per call, so it must give exactly what pic_cell_counts gives, call
after call (the shared array keeps the previous call's counts and has to be
cleared each time).  This file is collected last so that a failure here does
not hide the other GPU tests; it also passes alone in a fresh process.
"""
import math

import numpy as np
import pytest

from paper_2501_07465_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


def _sim(n, nparticles, seed):
    import torch

    from paper_2501_07465_gb300 import pic
    rng = np.random.default_rng(seed)
    d = (0.5e-9,) * 3
    dims = 3 if n[2] > 1 else 2
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(dims))
    h = pic.pic_create(pic.make_grid(dims, n, d, dt, bc=(0, 0, 0)),
                       torch.cuda.current_stream().cuda_stream)
    cell, off, v = I.random_particles(rng, n, nparticles, vscale=3e6, dims=dims)
    pic.pic_load_species(h, pic.species_desc(pic.PIC_FREE, -I.QE, I.ME, 1e3), cell, off, v)
    return h


def test_noalloc_counts_equal_the_allocating_entry_point_twice_in_a_row():
    from paper_2501_07465_gb300 import pic
    n = (48, 40, 24)
    h = _sim(n, 200000, 5)
    try:
        shape = I.grid_shape(n)
        for _ in range(2):
            pic.pic_step(h, 7)
            ref = pic.pic_cell_counts(h, 0, shape)
            got = pic.pic_cell_counts_noalloc(h, 0, shape)
            assert np.array_equal(got, ref)
            assert got.sum() == 200000
            again = pic.pic_cell_counts_noalloc(h, 0, shape)
            assert np.array_equal(again, ref)
    finally:
        pic.pic_destroy(h)


def test_noalloc_counts_reject_grids_above_the_limit():
    from paper_2501_07465_gb300 import pic
    n = (256, 128, 129)  # 4.2 M cells > 2^22
    assert n[0] * n[1] * n[2] > pic.PIC_NOALLOC_MAX_CELLS
    h = _sim(n, 1000, 6)
    try:
        with pytest.raises(pic.PicError) as e:
            pic.pic_cell_counts_noalloc(h, 0, I.grid_shape(n))
        assert e.value.status == pic.PIC_EINVAL
        assert "at most" in str(e.value)
    finally:
        pic.pic_destroy(h)


def test_noalloc_counts_of_a_group_member_wait_for_the_group():
    """A member of a batch group is advanced on the group's stream, so the
    counts must wait for the group's steps in flight: called straight after
    pic_group_step (no synchronisation in between), it gives what
    pic_cell_counts gives once the group has finished."""
    import torch

    from paper_2501_07465_gb300 import pic
    n = (64, 56, 1)
    hs = [_sim(n, 60000 + 5000 * i, 11 + i) for i in range(2)]
    gstream = torch.cuda.Stream()  # the group's own stream, not the members'
    g = pic.pic_group_create(4, 0, gstream.cuda_stream, 0)
    try:
        for h in hs:
            pic.pic_group_add(g, h, 40)
        shape = I.grid_shape(n)
        for _ in range(2):
            pic.pic_group_step(g, 20)
            got = [pic.pic_cell_counts_noalloc(h, 0, shape) for h in hs]
            ref = [pic.pic_cell_counts(h, 0, shape) for h in hs]
            for a, b, h in zip(got, ref, hs):
                assert np.array_equal(a, b)
                assert a.sum() == pic.pic_diagnostics(h)["count"][0]
    finally:
        for h in hs:
            pic.pic_group_remove(g, h)
        pic.pic_group_destroy(g)
        for h in hs:
            pic.pic_destroy(h)
