"""GPU parity of TSC (order-2) shapes for the free and Dirac particles
(the shape function W of Sec. 4.1 at the next order; bound particles keep
CIC): one step against the oracle particle by particle, fields after tens of
steps, Gauss's law at roundoff on the device, and argument checks."""
import math

import numpy as np
import pytest

from oracle import oracle as O
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


def _pic():
    from paper_2501_07465_gb300 import pic
    return pic


def _tsc_sims(grid, mask, species, tuning=None):
    """The same case with TSC shapes in the oracle and on the device."""
    pic = _pic()
    s = O.OracleSim(**PR.oracle_grid(grid))
    s.set_shape_order(2)
    if mask is not None:
        s.set_mask(mask)
    n = tuple(grid["n"])
    for sp in species:
        X, V, D = PR.species_arrays_for_oracle(sp, n)
        s.add_species(sp["kind"], sp["q"], sp["m"], sp["w"], X, V, D=D,
                      omega0=sp.get("omega0", (0, 0, 0)), gamma=sp.get("gamma", (0, 0, 0)),
                      vF=sp.get("v_F", 0.0), bg=sp.get("background", 0))
    h = PR.gpu_sim(grid, mask, [], tuning=tuning)
    pic.pic_set_shape_order(h, 2)
    for sp in species:
        desc = pic.species_desc(sp["kind"], sp["q"], sp["m"], sp.get("w", 0.0),
                                omega0=sp.get("omega0", (0, 0, 0)), gamma=sp.get("gamma", (0, 0, 0)),
                                v_F=sp.get("v_F", 0.0), background=sp.get("background", 0))
        pic.pic_load_species(h, desc, cell=sp["cell"], off=sp.get("off"), v=sp["v"],
                             anchor_off=sp.get("anchor_off"), disp=sp.get("disp"))
    return s, h


def _guard(grid, mask, species):
    """Drop free particles that end the first oracle step within 1e-5 cell
    of a face (FP32 and FP64 may cross differently there)."""
    s, h = _tsc_sims(grid, mask, species)
    _pic().pic_destroy(h)
    s.step(1)
    Xo = s.species(0)[0]
    s.close()
    ok = ~PR.near_face(Xo, grid["dims"], 1e-5)
    assert ok.mean() > 0.99
    keep = np.flatnonzero(ok)
    sp0 = dict(species[0], cell=species[0]["cell"][keep], off=species[0]["off"][keep],
               v=species[0]["v"][keep])
    return [sp0] + list(species[1:])


@pytest.mark.parametrize("overlap,mode", [(1, 2), (0, 2), (1, 1)])
def test_tsc_sphere_matches_oracle(overlap, mode):
    """The metal sphere (CPML, plane wave) with TSC free electrons and CIC
    bound electrons: one step particle by particle (1e-5), per-cell counts
    and reflections exact, fields 1e-5; 30 more steps: fields 1e-3."""
    rng = np.random.default_rng(81)
    grid, mask, species = PR.sphere_case(rng)
    species = _guard(grid, mask, species)
    pic = _pic()
    s, h = _tsc_sims(grid, mask, species, tuning=dict(no_overlap=1 - overlap, field_mode=mode))
    try:
        nro = PR.compare_one_step(pic, h, s, grid, species)
        assert nro > 0
        pic.pic_step(h, 30)
        s.step(30)
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
    finally:
        pic.pic_destroy(h)
        s.close()


@pytest.mark.parametrize("tile", [(16, 8, 1), (7, 5, 1), (2, 2, 1)])
def test_tsc_periodic_2d_matches_oracle(tile):
    """2D3V periodic plasma with TSC, ragged and tiny tiles (more particles
    on the slow path), sorting every 4 steps: velocities after one step
    (1e-5), fields after 1 (1e-5) and 60 steps (1e-3), kinetic energy 1e-5."""
    rng = np.random.default_rng(82)
    n = (50, 37, 1)
    d = (0.1e-9, 0.1e-9, 0.1e-9)
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(2))
    grid = dict(dims=2, n=n, d=d, dt=dt, bc=(0, 0, 0))
    cell, off, v = I.random_particles(rng, n, 20000, vscale=2e6, dims=2)
    w = 8.5e28 * np.prod(d) / 16
    species = [dict(kind=I.FREE, q=-I.QE, m=I.ME, w=w, cell=cell, off=off, v=v, background=2)]
    pic = _pic()
    s, h = _tsc_sims(grid, None, species, tuning=dict(tile=tile, sort_interval=4))
    try:
        pic.pic_step(h, 1)
        s.step(1)
        _, Vo, _, _ = s.species(0)
        rd = pic.pic_read_species(h, 0, cell.size)
        assert PR.vel_rel(rd["v"], Vo, 1e5) < 1e-5
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            if np.linalg.norm(s.field(c)) > 0:
                assert PR.rel_l2(got[c], s.field(c)) < 1e-5, c
        pic.pic_step(h, 59)
        s.step(59)
        got = PR.gpu_fields(h, grid)
        for c in (0, 1, 2, 5):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
        assert abs(pic.pic_diagnostics(h)["kinetic"][0] / s.diag()["kinetic"][0] - 1) < 1e-5
    finally:
        pic.pic_destroy(h)
        s.close()


def test_tsc_keeps_gauss_law_on_the_device():
    """Periodic sphere, ions at the loaded positions (so the start is
    neutral), TSC free + CIC bound electrons: after 40 steps the device's
    Gauss residual div E - rho/eps0 (rho with each species' own shape) stays
    at FP32 roundoff of one macro-particle's charge density."""
    rng = np.random.default_rng(83)
    grid, mask, species = PR.sphere_case(rng)
    grid["bc"] = (0, 0, 0)
    grid["src"] = None
    species[1]["disp"] = np.zeros_like(species[1]["disp"])
    pic = _pic()
    s, h = _tsc_sims(grid, mask, species)
    try:
        pic.pic_step(h, 40)
        dg = pic.pic_diagnostics(h)
        qs = I.QE * 5.9e28 / 8 / I.EPS0
        assert dg["gauss_max"] < 1e-5 * qs
        assert dg["field_E"] > 0
    finally:
        pic.pic_destroy(h)
        s.close()


def test_shape_order_arguments():
    """Orders other than 1 and 2 are refused (PIC_EINVAL), as is a change
    after species are loaded (PIC_ESTATE); a group takes a TSC simulation
    and then refuses a CIC one (its members share one shape order)."""
    pic = _pic()
    n = (8, 8, 8)
    grid = dict(dims=3, n=n, d=(1e-9,) * 3, dt=1e-18, bc=(0, 0, 0))
    rng = np.random.default_rng(6)
    cell, off, v = I.random_particles(rng, n, 100)
    h = PR.gpu_sim(grid, None, [])
    g = None
    try:
        for bad in (0, 3, -1):
            with pytest.raises(pic.PicError) as e:
                pic.pic_set_shape_order(h, bad)
            assert e.value.status == pic.PIC_EINVAL
        pic.pic_set_shape_order(h, 2)
        desc = pic.species_desc(I.FREE, -I.QE, I.ME, 1.0)
        pic.pic_load_species(h, desc, cell=cell, off=off, v=v)
        with pytest.raises(pic.PicError) as e:
            pic.pic_set_shape_order(h, 1)
        assert e.value.status == pic.PIC_ESTATE
        g = pic.pic_group_create(4)
        pic.pic_group_add(g, h, 1)
        hc = PR.gpu_sim(grid, None, [])
        try:
            pic.pic_load_species(hc, desc, cell=cell, off=off, v=v)
            with pytest.raises(pic.PicError) as e:
                pic.pic_group_add(g, hc, 1)
            assert e.value.status == pic.PIC_EINVAL
        finally:
            pic.pic_destroy(hc)
        pic.pic_group_remove(g, h)
    finally:
        if g is not None:
            pic.pic_group_destroy(g)
        pic.pic_destroy(h)
