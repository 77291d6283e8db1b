"""The 3D CIC particle phase on the default 8 x 8 x 4 tile takes a kernel
whose loop finishes only the moves that stay in their cell: a move that
crosses a cell face is completed after the loop from a per-tile list, and a
particle that has drifted out of its tile's box (or that overflows the
list) from a global list by a second kernel.  These cases drive every one
of those paths hard -- fast particles, no re-sort for many steps, thousands
of crossing moves per tile -- and check the result against the FP64 oracle
and against the generic kernel (a tile that the lean kernel does not take).
"""
import math

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
    yield


def _fast_plasma(rng, n=(24, 24, 16), ppc=16, vscale=6e7, bc=(0, 0, 0)):
    """A 3D plasma of free electrons moving ~0.06 cell a step along each
    axis (so a sixth of the moves cross a face), plus a bound species at its
    anchors (ions at the loaded positions: the Gauss residual starts at 0)."""
    d = (0.5e-9,) * 3
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(3))
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=bc, pml_cells=4 if any(bc) else 0)
    N = int(np.prod(n)) * ppc
    w = 5.9e28 * d[0] ** 3 / ppc
    cell, off, v = I.random_particles(rng, n, N, vscale=vscale)
    cb, anc, disp, vb = I.random_bound(rng, n, N // 4, dscale=0.0, vscale=2e4)
    w0 = 2 * np.pi * I.C_LIGHT / 400e-9
    species = [
        dict(kind=I.FREE, q=-I.QE, m=I.ME, w=w, cell=cell, off=off, v=v, background=1),
        dict(kind=I.BOUND, q=-I.QE, m=I.ME, w=0.5 * w, cell=cb, anchor_off=anc, disp=disp, v=vb,
             omega0=(w0, w0, w0), gamma=(1e14,) * 3, background=1),
    ]
    return grid, species


def test_lean_kernel_runs_on_the_default_tile_and_not_on_others():
    """Two kernels a particle phase on the 8 x 8 x 4 tile (the loop and the
    global completion), one on any other tile but the sheet tile 16 x 8 x 1."""
    from paper_2501_07465_gb300 import pic
    rng = np.random.default_rng(3)
    grid, species = _fast_plasma(rng, n=(16, 16, 8), ppc=2)
    per_step = {}
    for tile in ((8, 8, 4), (8, 8, 5)):
        h = PR.gpu_sim(grid, None, species, tuning=dict(tile=tile, sort_interval=1000,
                                                       no_overlap=1))
        try:
            pic.pic_step(h, 1)
            pic.pic_get_timing(h)  # reset the counters
            pic.pic_step(h, 4)
            per_step[tile] = pic.pic_get_timing(h)["kernel_launches"] / 4
        finally:
            pic.pic_destroy(h)
    assert per_step[(8, 8, 4)] == per_step[(8, 8, 5)] + 1


def test_crossing_and_drifted_particles_match_the_oracle():
    """16 ppc at ~0.06 cell a step: about a thousand crossing moves per tile
    and step (the shared list of 256 overflows into the global one) and,
    with no re-sort for 30 steps, particles more than a cell out of their
    tile (the global list).  Velocities and positions after one step within
    1e-5, fields within 1e-5 after one step and 1e-3 after 30, per-cell
    counts exact, Gauss's law at FP32 roundoff."""
    from paper_2501_07465_gb300 import pic
    rng = np.random.default_rng(5)
    grid, species = _fast_plasma(rng)
    n = grid["n"]
    s = PR.oracle_sim(grid, None, species)
    s.step(1)
    Xo = s.species(0)[0]
    s.close()
    keep = np.flatnonzero(~PR.near_face(Xo, 3, 1e-5))
    species[0] = dict(species[0], cell=species[0]["cell"][keep], off=species[0]["off"][keep],
                      v=species[0]["v"][keep])
    s = PR.oracle_sim(grid, None, species)
    h = PR.gpu_sim(grid, None, species, tuning=dict(tile=(8, 8, 4), sort_interval=1000,
                                                   no_overlap=1))
    try:
        PR.compare_one_step(pic, h, s, grid, species)
        pic.pic_step(h, 29)
        s.step(29)
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
        _, Vo, _, _ = s.species(0)
        rd = pic.pic_read_species(h, 0, keep.size)
        rel = np.linalg.norm(rd["v"] - Vo, axis=1) / np.linalg.norm(Vo, axis=1)
        assert np.quantile(rel, 0.99) < 1e-4
        diag = pic.pic_diagnostics(h)
        assert diag["count"] == [keep.size, species[1]["cell"].size]
        qs = I.QE * 5.9e28 / 16 / I.EPS0
        assert diag["gauss_max"] < 1e-5 * qs
    finally:
        pic.pic_destroy(h)
        s.close()


def test_lean_and_generic_kernels_agree():
    """The same fast plasma on the default tile (lean kernel) and on an
    8 x 8 x 2 tile (generic kernel): fields within 1e-5 after 10 steps
    without a re-sort, velocities within 1e-5."""
    from paper_2501_07465_gb300 import pic
    rng = np.random.default_rng(8)
    grid, species = _fast_plasma(rng, n=(32, 24, 16), ppc=8, bc=(1, 1, 1))
    out = []
    for tile in ((8, 8, 4), (8, 8, 2)):
        h = PR.gpu_sim(grid, None, species, tuning=dict(tile=tile, sort_interval=1000))
        try:
            pic.pic_step(h, 10)
            out.append((PR.gpu_fields(h, grid), pic.pic_read_species(h, 0, species[0]["cell"].size),
                        pic.pic_diagnostics(h)))
        finally:
            pic.pic_destroy(h)
    (fa, ra, da), (fb, rb, db) = out
    for c in range(6):
        if np.linalg.norm(fb[c]) > 0:
            assert PR.rel_l2(fa[c], fb[c]) < 1e-5, c
    assert PR.vel_rel(ra["v"], rb["v"], 1e5) < 1e-5
    assert da["count"] == db["count"]


def test_sheet_tile_agrees_with_the_generic_kernel():
    """The sheet tile 16 x 8 x 1 (lean kernel) against 16 x 8 x 2 (generic
    kernel) on fast free electrons filling a 48 x 40 x 12 periodic box, no
    re-sort for 10 steps (crossings, drifted particles): fields and
    velocities within 1e-5, counts equal."""
    from paper_2501_07465_gb300 import pic
    rng = np.random.default_rng(9)
    grid, species = _fast_plasma(rng, n=(48, 40, 12), ppc=8)
    out = []
    for tile in ((16, 8, 1), (16, 8, 2)):
        h = PR.gpu_sim(grid, None, species, tuning=dict(tile=tile, sort_interval=1000))
        try:
            pic.pic_step(h, 10)
            out.append((PR.gpu_fields(h, grid), pic.pic_read_species(h, 0, species[0]["cell"].size),
                        pic.pic_diagnostics(h)))
        finally:
            pic.pic_destroy(h)
    (fa, ra, da), (fb, rb, db) = out
    for c in range(6):
        if np.linalg.norm(fb[c]) > 0:
            assert PR.rel_l2(fa[c], fb[c]) < 1e-5, c
    assert PR.vel_rel(ra["v"], rb["v"], 1e5) < 1e-5
    assert da["count"] == db["count"]
