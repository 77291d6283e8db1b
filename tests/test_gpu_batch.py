"""The batch engine: simulations advanced together (one particle launch and
one field launch per step for all members, CUDA-graph replay) give what each
simulation gives alone, each member stops after its own step count, and
admission respects the HBM budget."""
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


def _case(k, n):
    """A 2D nanostructure: a disk, rod or bowtie of FD free + bound electrons."""
    rng = np.random.default_rng(100 + k)
    d = (0.5e-9,) * 3
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(2))
    shape = (n, n + 8 * (k % 3), 1)
    c = (shape[0] / 2, shape[1] / 2)
    if k % 3 == 0:
        mask = I.disk_mask2d(shape, c, n / 4)
    elif k % 3 == 1:
        mask = I.rod_mask2d(shape, c, n / 2, n / 6)
    else:
        mask = I.bowtie_mask2d(shape, c, n / 4, 4 + k % 5)
    grid = dict(dims=2, n=shape, d=d, dt=dt, bc=(1, 1, 0), pml_cells=8,
                src=dict(inc_axis=0, pol_axis=1, src_index=10, E0=5e9,
                         omega=2 * np.pi * I.C_LIGHT / (400e-9 + 50e-9 * k), tau=2e-16, t0=1e-16))
    w0 = 2 * np.pi * I.C_LIGHT / 400e-9
    cell, off, v = I.random_particles(rng, shape, 3000 + 500 * k, mask=mask, vscale=1.5e6, dims=2)
    cb, anc, disp, vb = I.random_bound(rng, shape, 2000, mask=mask, dscale=0.0, vscale=1e4)
    anc[:, 2] = 0.5
    w = 5.9e28 * d[0] ** 3 / 8
    species = [dict(kind=I.FREE, q=-I.QE, m=I.ME, w=w, cell=cell, off=off, v=v),
               dict(kind=I.BOUND, q=-I.QE, m=I.ME, w=0.5 * w, cell=cb, anchor_off=anc, disp=disp,
                    v=vb, omega0=(w0,) * 3, gamma=(1e14,) * 3)]
    return grid, mask, species


def _state(h, grid, species):
    from paper_2501_07465_gb300 import pic
    f = PR.gpu_fields(h, grid)
    v = pic.pic_read_species(h, 0, species[0]["cell"].size)["v"]
    return f, v


@pytest.mark.parametrize("use_graph", [0, 1])
def test_group_matches_alone(use_graph):
    import torch

    from paper_2501_07465_gb300 import pic
    sizes = [40, 64, 52, 96, 72]
    targets = [70, 45, 70, 23, 64]
    cases = [_case(k, n) for k, n in enumerate(sizes)]
    tuning = dict(sort_interval=8)
    alone = []
    for (grid, mask, species), t in zip(cases, targets):
        h = PR.gpu_sim(grid, mask, species, tuning=tuning)
        pic.pic_step(h, t)
        alone.append(_state(h, grid, species))
        pic.pic_destroy(h)
    stream = torch.cuda.current_stream().cuda_stream
    g = pic.pic_group_create(8, 0, stream, use_graph)
    hs = []
    try:
        for (grid, mask, species), t in zip(cases, targets):
            h = PR.gpu_sim(grid, mask, species, tuning=tuning)
            pic.pic_group_add(g, h, t)
            hs.append(h)
        pic.pic_group_step(g, 30)
        pic.pic_group_step(g, 50)   # every member reaches its target
        pic.pic_group_sync(g)
        for k, ((grid, mask, species), h) in enumerate(zip(cases, hs)):
            assert pic.pic_group_progress(g, h) == (targets[k], 0)
            f, v = _state(h, grid, species)
            fa, va = alone[k]
            for c in range(6):
                if np.linalg.norm(fa[c]) > 0:
                    assert PR.rel_l2(f[c], fa[c]) < 1e-4, (k, c, PR.rel_l2(f[c], fa[c]))
            rel = np.linalg.norm(v - va, axis=1) / np.linalg.norm(va, axis=1)
            assert np.quantile(rel, 0.99) < 1e-4
            assert pic.pic_diagnostics(h)["step"] == targets[k]
        info = pic.pic_group_info(g)
        assert info["members"] == len(sizes)
        assert info["launches"] > 0
    finally:
        pic.pic_group_destroy(g)
        for h in hs:
            pic.pic_destroy(h)


def test_group_budget_and_membership():
    import torch

    from paper_2501_07465_gb300 import pic
    stream = torch.cuda.current_stream().cuda_stream
    grid, mask, species = _case(0, 48)
    h1 = PR.gpu_sim(grid, mask, species)
    h2 = PR.gpu_sim(grid, mask, species)
    b1 = pic.pic_memory_bytes(h1)
    g = pic.pic_group_create(4, int(1.5 * b1), stream, 1)
    try:
        pic.pic_group_add(g, h1, 10)
        with pytest.raises(pic.PicError) as e:
            pic.pic_group_add(g, h2, 10)
        assert e.value.status == pic.PIC_EBUDGET
        with pytest.raises(pic.PicError) as e:
            pic.pic_step(h1, 1)  # members step through their group
        assert e.value.status == pic.PIC_ESTATE
        pic.pic_group_step(g, 4)
        pic.pic_group_remove(g, h1)
        pic.pic_group_add(g, h2, 10)
        pic.pic_group_step(g, 4)
        pic.pic_group_sync(g)
        pic.pic_step(h1, 2)  # a released simulation steps on its own again
        assert pic.pic_diagnostics(h1)["step"] == 6
        assert pic.pic_group_progress(g, h2) == (4, 6)
    finally:
        pic.pic_group_destroy(g)
        pic.pic_destroy(h1)
        pic.pic_destroy(h2)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_group_with_boundary_variants_matches_alone(use_graph):
    """Members with the variants a batch takes -- open edges with the
    work-function barrier (Sec. 3), bound electrons with a diagonal gamma,
    diffuse reflection at the material edges (Sec. 3; the draws keyed on the
    member's own step index, which a captured epoch advances on the device),
    a per-cell permittivity (Eq. consteps) -- beside a plain member: one
    persistent launch (the variant batch kernel) and one batched field
    launch give each the result it gets alone (fields 1e-4, 99 % of
    velocities 1e-4; the diffuse member's reflections and per-cell counts
    exactly)."""
    import torch

    from paper_2501_07465_gb300 import pic
    sizes, targets = [40, 64, 52, 48, 56], [40, 33, 40, 40, 37]
    cases = [_case(k, n) for k, n in enumerate(sizes)]
    cases[2][2][1]["gamma"] = (1e14, 3e14, 5e13)
    g4, m4, _ = cases[4]
    eps = np.where(m4 > 0, 3.5, 1.0).astype(np.float32)
    eps[:, :, : g4["n"][0] // 4] = 2.0

    def setup(h, k):
        if k == 1:
            pic.pic_set_particle_bc(h, pic.PIC_EDGE_OPEN)
            pic.pic_set_work_function(h, 4.5)
        elif k == 3:
            pic.pic_set_particle_bc(h, pic.PIC_EDGE_REFLECT, 0.5, 1234567)
        elif k == 4:
            pic.pic_set_permittivity(h, eps)

    tuning = dict(sort_interval=8)
    alone, refl, counts = [], [], []
    for k, ((grid, mask, species), t) in enumerate(zip(cases, targets)):
        h = PR.gpu_sim(grid, mask, species, tuning=tuning)
        setup(h, k)
        pic.pic_step(h, t)
        alone.append(_state(h, grid, species))
        refl.append(pic.pic_diagnostics(h)["reflections"][0])
        counts.append(pic.pic_cell_counts(h, 0, I.grid_shape(grid["n"])))
        pic.pic_destroy(h)
    assert refl[3] > 0  # the diffuse member does reflect
    stream = torch.cuda.current_stream().cuda_stream
    g = pic.pic_group_create(8, 0, stream, use_graph)
    hs = []
    try:
        for k, ((grid, mask, species), t) in enumerate(zip(cases, targets)):
            h = PR.gpu_sim(grid, mask, species, tuning=tuning)
            setup(h, k)
            pic.pic_group_add(g, h, t)
            hs.append(h)
        pic.pic_group_step(g, 40)
        pic.pic_group_sync(g)
        for k, ((grid, mask, species), h) in enumerate(zip(cases, hs)):
            f, v = _state(h, grid, species)
            fa, va = alone[k]
            for c in range(6):
                if np.linalg.norm(fa[c]) > 0:
                    assert PR.rel_l2(f[c], fa[c]) < 1e-4, (k, c, PR.rel_l2(f[c], fa[c]))
            rel = np.linalg.norm(v - va, axis=1) / np.linalg.norm(va, axis=1)
            assert np.quantile(rel, 0.99) < 1e-4
            if k == 3:
                assert pic.pic_diagnostics(h)["reflections"][0] == refl[3]
                assert np.array_equal(pic.pic_cell_counts(h, 0, I.grid_shape(grid["n"])),
                                      counts[3])
    finally:
        pic.pic_group_destroy(g)
        for h in hs:
            pic.pic_destroy(h)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_group_of_tsc_members_matches_alone(use_graph):
    """Members with TSC shapes (Sec. 4.1's W at order 2 for the free
    electrons; the group runs the TSC batch kernel with the wider staged
    box) give what each gives alone (fields 1e-4, 99 % of velocities 1e-4);
    a CIC simulation cannot join a TSC group."""
    import torch

    from paper_2501_07465_gb300 import pic
    sizes, targets = [40, 56, 48], [36, 30, 36]
    cases = [_case(k, n) for k, n in enumerate(sizes)]
    tuning = dict(sort_interval=8)

    def make(grid, mask, species):
        h = PR.gpu_sim(grid, mask, [], tuning=tuning)
        pic.pic_set_shape_order(h, 2)
        for sp in species:
            desc = pic.species_desc(sp["kind"], sp["q"], sp["m"], sp.get("w", 0.0),
                                    omega0=sp.get("omega0", (0, 0, 0)),
                                    gamma=sp.get("gamma", (0, 0, 0)), v_F=sp.get("v_F", 0.0),
                                    background=sp.get("background", 0))
            pic.pic_load_species(h, desc, cell=sp["cell"], off=sp.get("off"), v=sp["v"],
                                 anchor_off=sp.get("anchor_off"), disp=sp.get("disp"))
        return h

    alone = []
    for (grid, mask, species), t in zip(cases, targets):
        h = make(grid, mask, species)
        pic.pic_step(h, t)
        alone.append(_state(h, grid, species))
        pic.pic_destroy(h)
    stream = torch.cuda.current_stream().cuda_stream
    g = pic.pic_group_create(4, 0, stream, use_graph)
    hs = []
    try:
        for (grid, mask, species), t in zip(cases, targets):
            h = make(grid, mask, species)
            pic.pic_group_add(g, h, t)
            hs.append(h)
        grid, mask, species = cases[0]
        hc = PR.gpu_sim(grid, mask, species, tuning=tuning)
        try:
            with pytest.raises(pic.PicError) as e:
                pic.pic_group_add(g, hc, 5)
            assert e.value.status == pic.PIC_EINVAL
        finally:
            pic.pic_destroy(hc)
        pic.pic_group_step(g, 36)
        pic.pic_group_sync(g)
        for k, ((grid, mask, species), h) in enumerate(zip(cases, hs)):
            assert pic.pic_group_progress(g, h) == (targets[k], 0)
            f, v = _state(h, grid, species)
            fa, va = alone[k]
            for c in range(6):
                if np.linalg.norm(fa[c]) > 0:
                    assert PR.rel_l2(f[c], fa[c]) < 1e-4, (k, c, PR.rel_l2(f[c], fa[c]))
            rel = np.linalg.norm(v - va, axis=1) / np.linalg.norm(va, axis=1)
            assert np.quantile(rel, 0.99) < 1e-4
    finally:
        pic.pic_group_destroy(g)
        for h in hs:
            pic.pic_destroy(h)
