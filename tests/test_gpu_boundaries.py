"""GPU parity of the particle boundary variants of Sec. 3: the work-function
barrier (an external electrostatic field that only the particles see), open
material edges, and diffusive reflection.

Bars as in the other parity tests: per-particle velocities and positions
within 1e-5 (relative / cells) after one step, fields within 1e-5 relative
L2 after one step and 1e-3 after tens of steps.  The diffuse draws use the
same Philox counter on both sides, so which particles reflect diffusely is
bit-exact on inputs where no particle ends within 1e-5 cell of a face.
"""
import math

import numpy as np
import pytest

from paper_2501_07465_gb300 import inputs as I

from tests import pairs as PR

pytestmark = pytest.mark.gpu

EXT_BITS = 512 | 1024 | 2048


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


# ---------------------------------------------------------------------------
# the barrier field
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,bc", [(3, (1, 0, 1)), (3, (0, 0, 0)), (2, (0, 1, 0))])
def test_work_function_field_matches_oracle(dims, bc):
    """The barrier built on the device from the mask equals the oracle's
    (FP64, rounded once to FP32): sphere / disk masks that touch periodic and
    non-periodic faces."""
    pic = _pic()
    if dims == 3:
        n = (37, 29, 23)
        mask = I.sphere_mask(n, 12.5, center=(20.0, 14.5, 3.0))
    else:
        n = (61, 43, 1)
        mask = I.disk_mask2d(n, (30.5, 5.0), 17.0)
    d = (0.3e-9, 0.35e-9, 0.4e-9)
    grid = dict(dims=dims, n=n, d=d, dt=0.4 * d[0] / (I.C_LIGHT * math.sqrt(dims)), bc=bc,
                pml_cells=3)
    W = 4.25
    s = PR.oracle_sim(grid, mask, [])
    want = np.stack(s.work_function_field(W))
    h = PR.gpu_sim(grid, mask, [])
    try:
        with pytest.raises(pic.PicError) as e:
            pic.pic_read_fields(h, EXT_BITS, I.grid_shape(n))
        assert e.value.status == pic.PIC_ESTATE
        pic.pic_set_work_function(h, W)
        got = pic.pic_read_fields(h, EXT_BITS, I.grid_shape(n))
        scale = np.abs(want).max()
        assert scale > 0
        assert np.all(np.abs(got - want) <= 2.0 ** -23 * np.abs(want))
        assert np.count_nonzero(got) == np.count_nonzero(want)
        pic.pic_set_work_function(h, 0.0)  # removes it
        with pytest.raises(pic.PicError):
            pic.pic_read_fields(h, EXT_BITS, I.grid_shape(n))
    finally:
        pic.pic_destroy(h)
        s.close()


def test_boundary_variant_arguments():
    """Sizes, NaN / infinite fields, |W| > 1e3 eV, unknown edge rules,
    p outside [0, 1] and open edges with a diffuse share are refused with
    PIC_EINVAL; an external field round-trips at FP32; a group takes a
    simulation with an external field or with a diffuse share, whose
    surface rule then stays fixed while it is a member (PIC_ESTATE)."""
    pic = _pic()
    n = (8, 8, 8)
    grid = dict(dims=3, n=n, d=(1e-9,) * 3, dt=1e-18, bc=(0, 0, 0))
    rng = np.random.default_rng(3)
    E = rng.normal(size=(3,) + I.grid_shape(n)) * 1e9
    h = PR.gpu_sim(grid, None, [])
    g = None
    try:
        pic.pic_set_external_field(h, E)
        got = pic.pic_read_fields(h, EXT_BITS, I.grid_shape(n))
        assert np.array_equal(got, E.astype(np.float32).astype(np.float64))
        got_y = pic.pic_read_fields(h, pic.PIC_EXTY, I.grid_shape(n))
        assert np.array_equal(got_y[0], got[1])
        for bad in (E[:, :4], E * np.nan, E * np.inf):
            with pytest.raises(pic.PicError) as e:
                pic.pic_set_external_field(h, bad)
            assert e.value.status == pic.PIC_EINVAL
        for W in (float("nan"), 1.5e3, -2e3):
            with pytest.raises(pic.PicError) as e:
                pic.pic_set_work_function(h, W)
            assert e.value.status == pic.PIC_EINVAL
        for args in ((2, 0.0), (-1, 0.0), (0, -0.1), (0, 1.5), (0, float("nan")), (1, 0.2)):
            with pytest.raises(pic.PicError) as e:
                pic.pic_set_particle_bc(h, *args)
            assert e.value.status == pic.PIC_EINVAL
        with pytest.raises(pic.PicError) as e:
            pic.pic_write_fields(h, pic.PIC_EXTX, E[0])
        assert e.value.status == pic.PIC_EINVAL
        g = pic.pic_group_create(4)
        pic.pic_group_add(g, h, 1)
        with pytest.raises(pic.PicError) as e:
            pic.pic_set_external_field(h, None)  # not while in a group
        assert e.value.status == pic.PIC_ESTATE
        pic.pic_group_remove(g, h)
        pic.pic_set_external_field(h, None)
        pic.pic_set_particle_bc(h, pic.PIC_EDGE_REFLECT, 0.5, 9)
        pic.pic_group_add(g, h, 1)  # a diffuse member steps in its group
        with pytest.raises(pic.PicError) as e:
            pic.pic_set_particle_bc(h, pic.PIC_EDGE_OPEN, 0.0, 0)  # not while in a group
        assert e.value.status == pic.PIC_ESTATE
        pic.pic_group_remove(g, h)
        pic.pic_set_particle_bc(h, pic.PIC_EDGE_OPEN, 0.0, 0)
    finally:
        if g is not None:
            pic.pic_group_destroy(g)
        pic.pic_destroy(h)


# ---------------------------------------------------------------------------
# particles against the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("overlap,mode", [(1, 2), (0, 2), (1, 1), (0, 3)])
def test_potential_wall_matches_oracle(overlap, mode):
    """The potential-wall surface: open edges plus the work-function barrier
    (W = 4.3 eV) on the metal sphere (free and bound electrons, CPML, a
    plane-wave source).  One step matches the oracle particle by particle;
    after 30 more steps the fields match to 1e-3 and some electrons have left
    the sphere (open edges) with no material-edge reflection."""
    rng = np.random.default_rng(51)
    grid, mask, species = PR.sphere_case(rng)
    W = 4.3

    def setup(s):
        s.set_external_field(s.work_function_field(W))
        s.set_particle_bc(open_edges=True)

    species = PR.guarded_species(grid, mask, species, setup)
    pic = _pic()
    s = PR.oracle_sim(grid, mask, species)
    setup(s)
    h = PR.gpu_sim(grid, mask, species, tuning=dict(no_overlap=1 - overlap, field_mode=mode))
    pic.pic_set_work_function(h, W)
    pic.pic_set_particle_bc(h, pic.PIC_EDGE_OPEN)
    try:
        nro = PR.compare_one_step(pic, h, s, grid, species)
        assert nro == 0
        pic.pic_step(h, 30)
        s.step(30)
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
        Xo, Vo, _, _ = s.species(0)
        rd = pic.pic_read_species(h, 0, species[0]["cell"].size)
        rel = np.linalg.norm(rd["v"] - Vo, axis=1) / np.linalg.norm(Vo, axis=1)
        assert np.quantile(rel, 0.99) < 1e-4
        out_gpu = int((mask.ravel()[rd["cell"]] == 0).sum())
        c = np.floor(Xo).astype(int)
        out_orc = int((mask[c[:, 2], c[:, 1], c[:, 0]] == 0).sum())
        assert out_gpu > 0
        assert abs(out_gpu - out_orc) <= max(3, 0.01 * out_orc)
    finally:
        pic.pic_destroy(h)
        s.close()


@pytest.mark.parametrize("overlap,p", [(1, 0.5), (0, 1.0)])
def test_diffuse_reflection_matches_oracle(overlap, p):
    """Conditional reflection with a diffuse share p on the metal sphere
    (hot electrons loaded in its surface shell): the same particles reflect
    diffusely on both sides and leave with the same velocities (1e-5) after
    one step; after 20 more steps 99 % of the velocities agree to 1e-4 and
    every electron is still in the metal."""
    rng = np.random.default_rng(52)
    grid, mask, species = PR.sphere_case(rng, vscale=2e7, shell=True)
    seed = 0x1234_5678_9ABC

    def setup(s):
        s.set_particle_bc(p_diffuse=p, seed=seed)

    species = PR.guarded_species(grid, mask, species, setup)
    pic = _pic()
    s = PR.oracle_sim(grid, mask, species)
    setup(s)
    h = PR.gpu_sim(grid, mask, species, tuning=dict(no_overlap=1 - overlap, field_mode=2))
    pic.pic_set_particle_bc(h, pic.PIC_EDGE_REFLECT, p, seed)
    try:
        nro = PR.compare_one_step(pic, h, s, grid, species)
        assert nro > 40
        pic.pic_step(h, 20)
        s.step(20)
        Xo, Vo, _, nro = s.species(0)
        rd = pic.pic_read_species(h, 0, species[0]["cell"].size)
        rel = np.linalg.norm(rd["v"] - Vo, axis=1) / np.linalg.norm(Vo, axis=1)
        assert np.quantile(rel, 0.99) < 1e-4
        assert np.all(mask.ravel()[rd["cell"]] == 1)
        diag = pic.pic_diagnostics(h)
        assert abs(int(diag["reflections"][0]) - nro) <= max(3, 0.01 * nro)
    finally:
        pic.pic_destroy(h)
        s.close()


def test_diffuse_dirac_disk_matches_oracle():
    """Dirac carriers in a 2D nanodisk with fully diffuse edges: the in-plane
    2D law on both sides -- same velocities after one step (1e-5), v_z = 0
    and |v| = v_F after 30 steps."""
    rng = np.random.default_rng(53)
    n = (48, 40, 1)
    d = (1e-9, 1e-9, 1e-9)
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(2))
    mask = I.disk_mask2d(n, (24.0, 20.0), 15.0)
    grid = dict(dims=2, n=n, d=d, dt=dt, bc=(1, 1, 0), pml_cells=4)
    vF = 3e7  # fast enough that many carriers meet the edge within a few steps
    m_d = (0.2 * I.QE / 1e6) / (2 * 1e6)
    cell, off, _ = I.random_particles(rng, n, 8000, mask=mask, dims=2,
                                      cells=rng.choice(PR.shell_cells(mask), size=8000))
    phi = rng.uniform(0, 2 * np.pi, cell.size)
    v = np.stack([vF * np.cos(phi), vF * np.sin(phi), np.zeros_like(phi)], 1).astype(np.float32)
    w = 1e25 * np.prod(d) / 32
    species = [dict(kind=I.DIRAC, q=-I.QE, m=m_d, v_F=vF, w=w, cell=cell, off=off, v=v,
                    background=1)]
    seed = 42

    def setup(s):
        s.set_particle_bc(p_diffuse=1.0, seed=seed)

    species = PR.guarded_species(grid, mask, species, setup)
    pic = _pic()
    s = PR.oracle_sim(grid, mask, species)
    setup(s)
    h = PR.gpu_sim(grid, mask, species)
    pic.pic_set_particle_bc(h, pic.PIC_EDGE_REFLECT, 1.0, seed)
    try:
        nro = PR.compare_one_step(pic, h, s, grid, species)
        assert nro > 20
        pic.pic_step(h, 29)
        s.step(29)
        rd = pic.pic_read_species(h, 0, species[0]["cell"].size)
        sp = np.linalg.norm(rd["v"].astype(np.float64), axis=1)
        assert np.abs(sp / vF - 1).max() <= 4 * 2.0 ** -23
        assert np.all(rd["v"][:, 2] == 0)
        assert np.all(mask.ravel()[rd["cell"]] == 1)
    finally:
        pic.pic_destroy(h)
        s.close()


def test_zero_external_field_changes_nothing():
    """An all-zero external field selects the kernel with the boundary
    variants but adds exact zeros: velocities after one step are bit-equal to
    the plain kernel's."""
    rng = np.random.default_rng(54)
    grid, mask, species = PR.sphere_case(rng, nfree=4000, nbound=2000)
    pic = _pic()
    h0 = PR.gpu_sim(grid, mask, species)
    h1 = PR.gpu_sim(grid, mask, species)
    zero = np.zeros((3,) + I.grid_shape(grid["n"]))
    pic.pic_set_external_field(h1, zero)
    try:
        pic.pic_step(h0, 1)
        pic.pic_step(h1, 1)
        for k, bound in ((0, False), (1, True)):
            r0 = pic.pic_read_species(h0, k, species[k]["cell"].size, bound=bound)
            r1 = pic.pic_read_species(h1, k, species[k]["cell"].size, bound=bound)
            assert np.array_equal(r0["v"], r1["v"])
        f0 = PR.gpu_fields(h0, grid)
        f1 = PR.gpu_fields(h1, grid)
        for c in range(6):
            assert PR.rel_l2(f1[c], f0[c]) < 1e-6
    finally:
        pic.pic_destroy(h0)
        pic.pic_destroy(h1)


# ---------------------------------------------------------------------------
# closed forms at sizes beyond the oracle's
# ---------------------------------------------------------------------------

def test_potential_wall_energy_on_gpu():
    """Electrons of negligible weight bouncing in a periodic slab with open
    edges and a W = 4 eV barrier: with normal energy K < W they stay within
    the slab and its barrier layer; with K > W they cross.  At every readback
    the normal kinetic energy is K inside the slab and K - W in the vacuum
    (away from the 1.5-cell barrier layers).  Tolerance from FP32: a kick
    rounds v to half an ulp, and across a barrier layer of N steps the kicks
    are nearly constant, so the roundings add up to |dK| / K <= 2 N 2^-23
    per crossing (N <= 2000 here: 5e-4); the run makes at most four
    crossings -> 2e-3 K."""
    pic = _pic()
    n = (24, 8, 8)
    d = (0.45e-9, 0.5e-9, 0.4e-9)
    dt = 0.5 * min(d) / (I.C_LIGHT * math.sqrt(3))
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=(0, 0, 0))
    mask = np.zeros(I.grid_shape(n), np.uint8)
    mask[:, :, 6:14] = 1
    W = 4.0
    ratios = np.array([0.3, 0.5, 0.9, 1.1, 1.5, 2.0, 3.0, 0.7])
    npart = ratios.size
    v0 = np.sqrt(2 * ratios * W * I.QE / I.ME)
    cx = np.full(npart, 10)
    cy = np.arange(npart) % 8
    cz = np.arange(npart) // 8 + 3
    cell = (cx + n[0] * (cy + n[1] * cz)).astype(np.int32)
    off = np.full((npart, 3), 0.5, np.float32)
    v = np.zeros((npart, 3), np.float32)
    v[:, 0] = v0
    species = [dict(kind=I.FREE, q=-I.QE, m=I.ME, w=1e-12, cell=cell, off=off, v=v)]
    h = PR.gpu_sim(grid, mask, species)
    pic.pic_set_work_function(h, W)
    pic.pic_set_particle_bc(h, pic.PIC_EDGE_OPEN)
    seen_vac = np.zeros(npart, bool)
    try:
        for _ in range(300):
            pic.pic_step(h, 100)
            rd = pic.pic_read_species(h, 0, npart)
            x = PR.gpu_positions(rd, n)[:, 0]
            Kx = 0.5 * I.ME * rd["v"][:, 0].astype(np.float64) ** 2 / (W * I.QE)
            inside = (x > 8.0) & (x < 12.0)
            vac = (x > 16.0) | (x < 4.0)
            tol = 2e-3 * ratios
            assert np.all(np.abs(Kx[inside] - ratios[inside]) < tol[inside])
            assert np.all(np.abs(Kx[vac] - (ratios[vac] - 1)) < tol[vac])
            assert not np.any(vac & (ratios < 1))
            seen_vac |= vac
        assert np.all(seen_vac == (ratios > 1))
        assert pic.pic_diagnostics(h)["reflections"][0] == 0
    finally:
        pic.pic_destroy(h)


@pytest.mark.parametrize("kind", [I.FREE, I.DIRAC])
def test_diffuse_lambert_law_on_gpu(kind):
    """One million particles crossing a planar material edge in one step
    with p = 1: speed kept (FP32), re-emitted inward, and the moments of
    Lambert's law -- 3D: E[cos] = 2/3, E[cos^2] = 1/2, uniform azimuth;
    Dirac sheet: E[cos] = pi/4, E[sin] = 0, v_z = 0 -- within 4 sigma."""
    pic = _pic()
    rng = np.random.default_rng(55)
    dims = 3 if kind == I.FREE else 2
    n = (32, 64, 64) if dims == 3 else (32, 512, 1)
    d = (0.5e-9,) * 3
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(dims))
    grid = dict(dims=dims, n=n, d=d, dt=dt, bc=(0, 0, 0))
    mask = np.zeros(I.grid_shape(n), np.uint8)
    mask[:, :, :16] = 1
    N = 1 << 20
    cy = rng.integers(0, n[1], N)
    cz = rng.integers(0, n[2], N)
    cell = (15 + n[0] * (cy + n[1] * cz)).astype(np.int32)
    vF = 1e6
    if kind == I.DIRAC:
        th = rng.uniform(-1.2, 1.2, N)
        v = np.stack([vF * np.cos(th), vF * np.sin(th), np.zeros(N)], 1)
    else:
        v = rng.normal(size=(N, 3)) * 2e5
        v[:, 0] = 0.1 * d[0] / dt * (1 + rng.random(N))
    # start where the face at x = 16 is met 5 % .. 95 % into the step, away
    # from the transverse faces
    step_x = v[:, 0] * dt / d[0]
    off = np.column_stack([1 - (0.05 + 0.9 * rng.random(N)) * step_x,
                           0.25 + 0.5 * rng.random(N),
                           0.25 + 0.5 * rng.random(N) if dims == 3 else np.full(N, 0.5)])
    off = off.astype(np.float32)
    v = v.astype(np.float32)
    m = (0.2 * I.QE / vF) / (2 * vF) if kind == I.DIRAC else I.ME
    species = [dict(kind=kind, q=-I.QE, m=m, w=1e-12, cell=cell, off=off, v=v, v_F=vF)]
    h = PR.gpu_sim(grid, mask, species)
    pic.pic_set_particle_bc(h, pic.PIC_EDGE_REFLECT, 1.0, 2024)
    try:
        pic.pic_step(h, 1)
        rd = pic.pic_read_species(h, 0, N)
        assert pic.pic_diagnostics(h)["reflections"][0] == N
        V = rd["v"].astype(np.float64)
        sp0 = np.linalg.norm(v.astype(np.float64), axis=1)
        sp = np.linalg.norm(V, axis=1)
        assert np.abs(sp / sp0 - 1).max() < 1e-6
        ct = -V[:, 0] / sp
        assert np.all(ct >= 0)
        if kind == I.FREE:
            assert abs(ct.mean() - 2 / 3) < 4 * math.sqrt(1 / 18 / N)
            assert abs((ct ** 2).mean() - 0.5) < 4 * math.sqrt(1 / 12 / N)
            ph = np.arctan2(V[:, 2], V[:, 1])
            for f in (np.cos(ph), np.sin(ph), np.cos(2 * ph)):
                assert abs(f.mean()) < 4 * math.sqrt(0.5 / N)
        else:
            assert np.all(V[:, 2] == 0)
            assert abs(ct.mean() - math.pi / 4) < 4 * math.sqrt((2 / 3 - math.pi ** 2 / 16) / N)
            assert abs((V[:, 1] / sp).mean()) < 4 * math.sqrt(1 / 3 / N)
        X = PR.gpu_positions(rd, n)
        assert np.all(X[:, 0] < 16.0)
    finally:
        pic.pic_destroy(h)
