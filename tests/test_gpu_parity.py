"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances: per-particle velocity within 1e-5 relative after one step;
fields within 1e-5 relative L2 after one step and 1e-3 after 100 steps;
integer results (per-cell counts, reflection counts) bit-exact on inputs
where no particle ends within 1e-5 cell of a face (the oracle decides in
FP64, the GPU in FP32: such particles may legitimately cross differently).
"""
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


def _ov(overlap):
    """Tuning of the field work beside the particle phase: 0 none, 1 the B
    pass beside it, 2 both field passes beside it (the current applied after
    the join; the library's default)."""
    return dict(no_overlap=0 if overlap else 1, field_overlap=overlap)


def _pic():
    from paper_2501_07465_gb300 import pic
    return pic


def _vel_rel(vg, vo, floor):
    return np.max(np.linalg.norm(vg - vo, axis=1) / np.maximum(np.linalg.norm(vo, axis=1), floor))


# ---------------------------------------------------------------------------
# fields only (a8)
# ---------------------------------------------------------------------------

def _plane_wave_fields(grid):
    n = grid["n"]
    nz, ny, nx = I.grid_shape(n)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rng = np.random.default_rng(3)
    f = {}
    for c in range(6):
        f[c] = (rng.normal(size=(nz, ny, nx)) * (1e6 if c < 3 else 1e6 / I.C_LIGHT) +
                np.sin(2 * np.pi * (i / nx + 2 * j / ny)) * (1e7 if c < 3 else 0.0))
    return f


_FIELD_GRIDS = [(3, (0, 0, 0), False), (3, (1, 1, 1), True), (3, (0, 0, 1), True),
                (2, (1, 0, 0), True), (2, (1, 1, 0), False), (2, (0, 0, 0), True)]
# the default split passes on every grid; the fused (1) and one-pass (3)
# field modes, which the step does not use by default, one case each
_FIELD_CASES = ([g + r for g in _FIELD_GRIDS
                 for r in ((45, 0, 0, 2), (44, 0, 0, 2), (64, 0, 0, 2), (44, 0, 1, 2))] +
                [(3, (1, 1, 1), True, 44, 0, 1, 1), (2, (1, 0, 0), True, 45, 1, 0, 1),
                 (3, (1, 1, 1), True, 45, 0, 0, 3)])


@pytest.mark.parametrize("dims,bc,src,nx,plain,overlap,mode", _FIELD_CASES)
def test_field_update_matches_oracle(dims, bc, src, nx, plain, overlap, mode):
    """mode 2: the split B / E passes (overlap = 1: B beside the particle
    phase).  mode 1, the fused update: nx = 44 and 64 take the TMA-fed kernel
    (row pitch a multiple of 16 B; 44 leaves a ragged last block), nx = 45 and
    plain = 1 the plain-load one; overlap = 1 runs it beside the particle phase
    with the separate current pass.  mode 3, the one-pass streaming update:
    nx = 45 and 70 leave ragged warps (lane 31 and lane 0 take their x
    neighbours from memory, beyond-grid lanes only shuffle), overlap = 1 runs
    it beside the particle phase with the separate current pass."""
    n = (nx, 20, 36) if dims == 3 else (nx + 25, 41, 1)
    if dims == 2 and nx % 4 == 0:
        n = (nx + 24, 41, 1)
    d = (1e-9, 0.8e-9, 1.1e-9)
    dt = 0.45 * min(d[:dims]) / (I.C_LIGHT * math.sqrt(dims))
    grid = dict(dims=dims, n=n, d=d, dt=dt, bc=bc, pml_cells=6)
    if src:
        inc = 2 if bc == (0, 0, 1) else 0
        grid["src"] = dict(inc_axis=inc, pol_axis=1 if inc != 1 else 0, src_index=9, E0=1e8,
                           omega=2 * np.pi * I.C_LIGHT / 30e-9, tau=4e-17, t0=6e-17)
    fields = _plane_wave_fields(grid)
    pic = _pic()
    h = PR.gpu_sim(grid, None, [], fields=fields,
                   tuning=dict(field_plain=plain, no_overlap=1 - overlap, field_mode=mode))
    s = PR.oracle_sim(grid, None, [], fields=fields)
    try:
        for nsteps, tol in ((1, 1e-5), (99, 1e-3)):
            pic.pic_step(h, nsteps)
            s.step(nsteps)
            got = PR.gpu_fields(h, grid)
            for c in range(6):
                ref = s.field(c)
                assert PR.rel_l2(got[c], ref) < tol, (c, nsteps, PR.rel_l2(got[c], ref))
    finally:
        pic.pic_destroy(h)
        s.close()


# ---------------------------------------------------------------------------
# particles: free, bound, Dirac, reflection (a2-a7)
# ---------------------------------------------------------------------------

def _sphere_case(rng, n=(30, 26, 22), radius=8.0, nfree=6000, nbound=4000, bc=(1, 1, 1),
                 vscale=4e6, dscale=2e-12):
    d = (0.5e-9,) * 3
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(3))
    mask = I.sphere_mask(n, radius)
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=bc, pml_cells=4,
                src=dict(inc_axis=0, pol_axis=1, src_index=6, E0=3e9,
                         omega=2 * np.pi * I.C_LIGHT / 20e-9, tau=3e-17, t0=2e-17))
    w = 5.9e28 * d[0] ** 3 / 8
    cell, off, v = I.random_particles(rng, n, nfree, mask=mask, vscale=vscale)
    cb, anc, disp, vb = I.random_bound(rng, n, nbound, mask=mask, dscale=dscale, vscale=2e4)
    w0 = 2 * np.pi * I.C_LIGHT / 400e-9
    species = [
        dict(kind=I.FREE, q=-I.QE, m=I.ME, w=w, cell=cell, off=off, v=v, background=1),
        dict(kind=I.BOUND, q=-I.QE, m=I.ME, w=0.5 * w, cell=cb, anchor_off=anc, disp=disp, v=vb,
             omega0=(w0, w0, w0), gamma=(1e14,) * 3, background=1),
    ]
    return grid, mask, species


@pytest.mark.parametrize("n,overlap,mode", [((30, 26, 22), 0, 2), ((32, 28, 24), 0, 2),
                                            ((32, 28, 24), 1, 2), ((32, 28, 24), 2, 2),
                                            ((30, 26, 22), 2, 2), ((32, 28, 24), 1, 1),
                                            ((30, 26, 22), 0, 3)])
def test_sphere_one_step_particles_fields_counts(n, overlap, mode):
    rng = np.random.default_rng(11)
    grid, mask, species = _sphere_case(rng, n=n)
    pic = _pic()
    n = grid["n"]
    s = PR.oracle_sim(grid, mask, species)
    s.step(1)
    Xo, Vo, Do, nro = s.species(0)
    # guard: no free particle may end within 1e-5 cell of a face
    ok = ~PR.near_face(Xo, 3, 1e-5)
    assert ok.mean() > 0.99
    keep = np.flatnonzero(ok)
    sp = [dict(species[0], cell=species[0]["cell"][keep], off=species[0]["off"][keep],
               v=species[0]["v"][keep]), species[1]]
    s.close()
    s = PR.oracle_sim(grid, mask, sp)
    h = PR.gpu_sim(grid, mask, sp, tuning=dict(keep_J=1, field_mode=mode, **_ov(overlap)))
    try:
        pic.pic_step(h, 1)
        s.step(1)
        Xo, Vo, _, nro = s.species(0)
        rd = pic.pic_read_species(h, 0, keep.size)
        assert _vel_rel(rd["v"], Vo, 1e5) < 1e-5
        dX = PR.periodic_delta(PR.gpu_positions(rd, n), Xo, n, 3)
        assert np.abs(dX).max() < 1e-5
        Xb, Vb, Db, _ = s.species(1)
        rb = pic.pic_read_species(h, 1, sp[1]["cell"].size, bound=True)
        assert _vel_rel(rb["v"], Vb, 1e3) < 1e-5
        assert np.abs(rb["disp"] - Db).max() < 1e-5 * np.abs(Db).max()
        diag = pic.pic_diagnostics(h)
        assert diag["reflections"][0] == nro
        assert nro > 0
        for k in range(2):
            assert np.array_equal(pic.pic_cell_counts(h, k, I.grid_shape(n)), s.cell_counts(k))
        got = PR.gpu_fields(h, grid, comps=range(9))
        for c in range(6):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-5, c
        # J of the deposit (the soft-source sheet is applied inside the field
        # kernel on the GPU and through J in the oracle: leave its plane out)
        src_plane = grid["src"]["src_index"]
        for c in range(3):
            jg, jo = got[6 + c].copy(), s.field(6 + c)
            jg[:, :, src_plane] = 0
            jo[:, :, src_plane] = 0
            assert PR.rel_l2(jg, jo) < 1e-5, ("J", c)
    finally:
        pic.pic_destroy(h)
        s.close()


@pytest.mark.parametrize("n,overlap,mode", [((30, 26, 22), 0, 2), ((36, 26, 22), 0, 2),
                                            ((36, 26, 22), 1, 2), ((36, 26, 22), 2, 2),
                                            ((36, 26, 22), 1, 1), ((36, 26, 22), 0, 3)])
def test_sphere_hundred_steps(n, overlap, mode):
    rng = np.random.default_rng(12)
    grid, mask, species = _sphere_case(rng, n=n, vscale=1.5e6)
    pic = _pic()
    n = grid["n"]
    s = PR.oracle_sim(grid, mask, species)
    h = PR.gpu_sim(grid, mask, species, tuning=dict(sort_interval=16, field_mode=mode,
                                                   **_ov(overlap)))
    try:
        pic.pic_step(h, 100)
        s.step(100)
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
        Xo, Vo, _, nro = s.species(0)
        rd = pic.pic_read_species(h, 0, species[0]["cell"].size)
        rel = np.linalg.norm(rd["v"] - Vo, axis=1) / np.linalg.norm(Vo, axis=1)
        assert np.quantile(rel, 0.99) < 1e-4
        diag = pic.pic_diagnostics(h)
        assert diag["count"] == [species[0]["cell"].size, species[1]["cell"].size]
        # every particle is still inside the material
        c = rd["cell"]
        assert np.all(mask.ravel()[c] == 1)
        assert abs(int(diag["reflections"][0]) - nro) <= max(3, 0.01 * nro)
    finally:
        pic.pic_destroy(h)
        s.close()


@pytest.mark.parametrize("tile,overlap,mode", [((32, 32, 1), 0, 2), ((16, 8, 1), 0, 2),
                                               ((7, 5, 1), 0, 2), ((16, 8, 1), 1, 2),
                                               ((16, 8, 1), 1, 1), ((16, 8, 1), 0, 3)])
def test_free_2d_periodic(tile, overlap, mode):
    """2D3V periodic plasma, ragged tiles, sorting every 4 steps."""
    rng = np.random.default_rng(21)
    n = (50, 37, 1)
    d = (0.1e-9, 0.1e-9, 0.1e-9)
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(2))
    grid = dict(dims=2, n=n, d=d, dt=dt, bc=(0, 0, 0))
    cell, off, v = I.random_particles(rng, n, 20000, vscale=2e6, dims=2)
    w = 8.5e28 * np.prod(d) / 16
    species = [dict(kind=I.FREE, q=-I.QE, m=I.ME, w=w, cell=cell, off=off, v=v, background=2)]
    pic = _pic()
    s = PR.oracle_sim(grid, None, species)
    h = PR.gpu_sim(grid, None, species, tuning=dict(tile=tile, sort_interval=4, no_overlap=1 - overlap,
                                                    field_mode=mode))
    try:
        pic.pic_step(h, 1)
        s.step(1)
        _, Vo, _, _ = s.species(0)
        rd = pic.pic_read_species(h, 0, cell.size)
        assert _vel_rel(rd["v"], Vo, 1e5) < 1e-5
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            if np.linalg.norm(s.field(c)) > 0:
                assert PR.rel_l2(got[c], s.field(c)) < 1e-5, c
        pic.pic_step(h, 99)
        s.step(99)
        got = PR.gpu_fields(h, grid)
        for c in (0, 1, 2, 5):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
        d0 = pic.pic_diagnostics(h)
        od = s.diag()
        assert abs(d0["kinetic"][0] / od["kinetic"][0] - 1) < 1e-5
    finally:
        pic.pic_destroy(h)
        s.close()


@pytest.mark.parametrize("tile", [(8, 8, 4), (16, 8, 1)])
def test_dirac_sheet_speed_and_parity(tile):
    """A one-cell sheet of Dirac carriers (Sec. 5) with CPML in z and a
    normally incident pulse, on the default tile and on the sheet tile
    16 x 8 x 1 (both taken by the lean kernel; 40 x 36 cells leave ragged
    tiles): velocities after one step within 1e-5 of the oracle, |v| = v_F
    to 2 ulp and v_z = 0 after 50, fields within 1e-3."""
    rng = np.random.default_rng(31)
    n = (40, 36, 16)
    d = (1e-9,) * 3
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(3))
    mask = I.sheet_mask(n, 8)
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=(0, 0, 1), pml_cells=4,
                src=dict(inc_axis=2, pol_axis=0, src_index=5, E0=1e8,
                         omega=2 * np.pi * I.C_LIGHT / 30e-9, tau=4e-17, t0=3e-17))
    vF = 1e6
    m_d = (0.2 * I.QE / vF) / (2 * vF)
    cell, off, _ = I.random_particles(rng, n, 20000, mask=mask)
    phi = rng.uniform(0, 2 * np.pi, cell.size)
    v = np.stack([vF * np.cos(phi), vF * np.sin(phi), np.zeros_like(phi)], 1).astype(np.float32)
    w = 1e25 * np.prod(d) / 32
    species = [dict(kind=I.DIRAC, q=-I.QE, m=m_d, v_F=vF, w=w, cell=cell, off=off, v=v,
                    background=1)]
    pic = _pic()
    s = PR.oracle_sim(grid, mask, species)
    h = PR.gpu_sim(grid, mask, species, tuning=dict(tile=tile))
    try:
        pic.pic_step(h, 1)
        s.step(1)
        rd = pic.pic_read_species(h, 0, cell.size)
        _, Vo, _, _ = s.species(0)
        assert _vel_rel(rd["v"], Vo, vF) < 1e-5
        pic.pic_step(h, 49)
        s.step(49)
        rd = pic.pic_read_species(h, 0, cell.size)
        sp = np.linalg.norm(rd["v"].astype(np.float64), axis=1)
        assert np.abs(sp / vF - 1).max() <= 2 * 2.0 ** -23
        assert np.all(rd["v"][:, 2] == 0)
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
    finally:
        pic.pic_destroy(h)
        s.close()


# ---------------------------------------------------------------------------
# loader (a1), diagnostics (a10), edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,dims,quiet", [(I.FREE, 3, 0), (I.FREE, 2, 1), (I.DIRAC, 3, 0),
                                             (I.BOUND, 3, 1)])
def test_fd_loader_matches_oracle(kind, dims, quiet):
    n = (20, 18, 12) if dims == 3 else (24, 20, 1)
    d = (0.5e-9,) * 3
    dt = 0.4 * d[0] / (I.C_LIGHT * math.sqrt(dims))
    mask = I.sphere_mask(n, 7.0) if dims == 3 else None
    if kind == I.DIRAC:
        mask = I.sheet_mask(n, 6)
    grid = dict(dims=dims, n=n, d=d, dt=dt, bc=(0, 0, 0))
    vF = 1e6
    m = (0.2 * I.QE / vF) / (2 * vF) if kind == I.DIRAC else I.ME
    sp = dict(kind=kind, q=-I.QE, m=m, v_F=vF if kind == I.DIRAC else 0.0, density=5.9e28,
              E_F=(0.2 if kind == I.DIRAC else 5.5) * I.QE, T=300.0, ppc=8 if dims == 3 else 16,
              quiet=quiet, seed=12345, stream=3, omega0=(4e15,) * 3, gamma=(1e14,) * 3)
    cell, off, v = O.fd_load(dims, n, mask, kind, m, sp["E_F"], 300.0, sp["v_F"], sp["ppc"],
                             quiet, 12345, 3)
    pic = _pic()
    h = PR.gpu_sim(grid, mask, [sp])
    try:
        rd = pic.pic_read_species(h, 0, cell.size, bound=kind == I.BOUND)
        assert np.array_equal(rd["cell"], cell)
        if kind == I.BOUND:
            assert np.array_equal(rd["anchor_off"], off)
            assert np.all(rd["v"] == 0)
        else:
            assert np.abs(rd["off"] - off).max() < 6e-8
            vo = v.astype(np.float32)
            scale = np.abs(v).max()
            assert np.abs(rd["v"] - vo).max() <= 2e-7 * scale
    finally:
        pic.pic_destroy(h)


def test_diagnostics_match_oracle():
    rng = np.random.default_rng(41)
    grid, mask, species = _sphere_case(rng, bc=(0, 0, 0), dscale=0.0)
    grid = dict(grid)
    grid.pop("src")
    grid["pml_cells"] = 0
    pic = _pic()
    s = PR.oracle_sim(grid, mask, species)
    h = PR.gpu_sim(grid, mask, species)
    try:
        for it in range(3):
            dg = pic.pic_diagnostics(h)
            do = s.diag()
            for k in range(2):
                assert abs(dg["kinetic"][k] / do["kinetic"][k] - 1) < 1e-6
            if do["field_E"] > 0:
                assert abs(dg["field_E"] / do["field_E"] - 1) < 1e-4
            qs = I.QE * 5.9e28 / 8 / I.EPS0
            # charge conservation: the residual stays at FP32 roundoff
            assert dg["gauss_max"] < 1e-5 * qs
            assert do["gauss_max"] < 1e-10 * qs
            pic.pic_step(h, 5)
            s.step(5)
    finally:
        pic.pic_destroy(h)
        s.close()


def test_empty_species_and_no_particles():
    n = (16, 16, 16)
    d = (0.5e-9,) * 3
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(3))
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=(0, 0, 0))
    species = [dict(kind=I.FREE, q=-I.QE, m=I.ME, w=1.0, cell=np.zeros(0, np.int32),
                     off=np.zeros((0, 3), np.float32), v=np.zeros((0, 3), np.float32))]
    pic = _pic()
    h = PR.gpu_sim(grid, None, species)
    try:
        pic.pic_step(h, 3)
        dg = pic.pic_diagnostics(h)
        assert dg["count"] == [0]
        assert dg["field_E"] == 0.0
    finally:
        pic.pic_destroy(h)


def test_abi_rejects_bad_arguments():
    pic = _pic()
    g = pic.make_grid(3, (16, 16, 16), (0.5e-9,) * 3, 1e-15)  # far above the Yee limit
    with pytest.raises(pic.PicError) as e:
        pic.pic_create(g)
    assert e.value.status == pic.PIC_EDTLIMIT
    g = pic.make_grid(2, (16, 16, 4), (0.5e-9,) * 3, 1e-19)
    with pytest.raises(pic.PicError) as e:
        pic.pic_create(g)
    assert e.value.status == pic.PIC_EINVAL
    g = pic.make_grid(3, (16, 16, 16), (0.5e-9,) * 3, 5e-19)
    h = pic.pic_create(g)
    try:
        bad = pic.species_desc(pic.PIC_BOUND, -I.QE, I.ME, 1.0, omega0=(1e15,) * 3,
                               gamma=(1e14, -2e14, 1e14))
        with pytest.raises(pic.PicError):
            pic.pic_load_species(h, bad, cell=np.zeros(1, np.int32),
                                 anchor_off=np.zeros((1, 3)), v=np.zeros((1, 3), np.float32))
        ok = pic.species_desc(pic.PIC_FREE, -I.QE, I.ME, 1.0)
        with pytest.raises(pic.PicError):
            pic.pic_load_species(h, ok, cell=np.array([16 ** 3], np.int32),
                                 off=np.zeros((1, 3), np.float32), v=np.zeros((1, 3), np.float32))
        with pytest.raises(pic.PicError):
            pic.pic_load_species(h, ok, cell=np.array([0], np.int32),
                                 off=np.ones((1, 3), np.float32), v=np.zeros((1, 3), np.float32))
        # a bound species with an enormous plasma density violates Eq. dtlimit
        with pytest.raises(pic.PicError) as e:
            pic.pic_load_species(h, ok, density=1e40, E_F=5 * I.QE, T=0.0, ppc=1, seed=1)
        assert e.value.status == pic.PIC_EDTLIMIT
    finally:
        pic.pic_destroy(h)


# ---------------------------------------------------------------------------
# long-run observables (within 1 %)
# ---------------------------------------------------------------------------

def _fit_frequency(t, y, w_guess):
    best = None
    for w in np.linspace(0.8 * w_guess, 1.2 * w_guess, 4001):
        A = np.stack([np.cos(w * t), np.sin(w * t), np.ones_like(t)], 1)
        coef, *_ = np.linalg.lstsq(A, y, rcond=None)
        r = np.sum((A @ coef - y) ** 2)
        if best is None or r < best[0]:
            best = (r, w)
    return best[1]


def test_langmuir_frequency_on_gpu():
    """The full 64 x 64, 16 ppc Langmuir workload, run ~2.2 plasma periods:
    w_p = sqrt(n e^2/(eps0 m)) within 1 % (Bohm-Gross shift 0.26 %)."""
    wl = I.langmuir2d()
    g = wl["grid"]
    nx, ny = g["n"][0], g["n"][1]
    dx = g["d"][0]
    sp = wl["species"][0]
    cell, off, v = O.fd_load(2, g["n"], None, I.FREE, I.ME, sp["E_F"], sp["T"], 0.0, 16, 1,
                             sp["seed"], 0)
    X = I.langmuir_ripple(I.cell_coords(cell, g["n"]) + off, nx, dx, wl["ripple"])
    cellr = (np.floor(X[:, 1]).astype(np.int64) * nx + np.floor(X[:, 0]).astype(np.int64))
    offr = (X - np.floor(X)).astype(np.float32)
    offr[:, 2] = 0.5
    w = sp["density"] * dx ** 3 / 16
    species = [dict(kind=I.FREE, q=-I.QE, m=I.ME, w=w, cell=cellr.astype(np.int32), off=offr,
                    v=v.astype(np.float32), background=2)]
    Ex = I.langmuir_initial_Ex(nx, ny, dx, sp["density"], wl["ripple"])
    pic = _pic()
    h = PR.gpu_sim(g, None, species, fields={0: Ex})
    wp = math.sqrt(sp["density"] * I.QE ** 2 / (I.EPS0 * I.ME))
    nsteps = int(2.2 * 2 * math.pi / (wp * g["dt"]))
    t, y = [], []
    i = np.arange(nx)
    k = 2 * math.pi / (nx * dx)
    try:
        for it in range(nsteps // 20):
            pic.pic_step(h, 20)
            E = pic.pic_read_fields(h, pic.PIC_EX, I.grid_shape(g["n"]))[0, 0].mean(axis=0)
            y.append(2 / nx * np.sum(E * np.sin(k * (i + 0.5) * dx)))
            t.append((it + 1) * 20 * g["dt"])
    finally:
        pic.pic_destroy(h)
    wfit = _fit_frequency(np.array(t), np.array(y), wp)
    assert abs(wfit / wp - 1) < 0.01


def test_bound_only_current_parity():
    """The bound current comes from displacements of ~1e-5 cell per step; it
    must match the oracle's J to 1e-5 even where free electrons are absent."""
    rng = np.random.default_rng(51)
    n = (24, 20, 18)
    d = (0.5e-9,) * 3
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(3))
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=(0, 0, 0))
    cb, anc, disp, vb = I.random_bound(rng, n, 30000, dscale=3e-12, vscale=3e4)
    w0 = 2 * np.pi * I.C_LIGHT / 400e-9
    # the workload's bound density: n_b = 2.95e28 m^-3 over the particles per cell
    w = 2.95e28 * np.prod(d) * np.prod(n) / cb.size
    species = [dict(kind=I.BOUND, q=-I.QE, m=I.ME, w=w, cell=cb, anchor_off=anc, disp=disp,
                    v=vb, omega0=(w0, w0, w0), gamma=(1e14,) * 3)]
    pic = _pic()
    s = PR.oracle_sim(grid, None, species)
    h = PR.gpu_sim(grid, None, species, tuning=dict(keep_J=1))
    try:
        for it in range(3):
            pic.pic_step(h, 1)
            s.step(1)
            got = PR.gpu_fields(h, grid, comps=(6, 7, 8))
            ref = np.stack([s.field(6 + c) for c in range(3)])
            assert PR.rel_l2(got, ref) < 1e-5, (it, PR.rel_l2(got, ref))
    finally:
        pic.pic_destroy(h)
        s.close()


def test_bound_medium_resonance_and_damping_on_gpu():
    """A uniform Lorentz medium (periodic, 16 ppc bound electrons at the
    sphere workload's w0, gamma and N_b = 0.5 n) started from a k-mode
    displacement rings at w_L = sqrt(w0^2 + w_pb^2 - gamma^2/4) within 1 %
    and its amplitude decays as exp(-gamma t / 2) within 5 % (Sec. 4, Eq.
    modlorentz; the dielectric response of Eq. lordielectric)."""
    nb = 0.5 * 5.9e28
    nx, ny = 32, 2
    dx = 0.5e-9
    dt = 0.5 * dx / (I.C_LIGHT * math.sqrt(2))
    w0, gam = 4.709e15, 1e14
    grid = dict(dims=2, n=(nx, ny, 1), d=(dx, dx, dx), dt=dt, bc=(0, 0, 0))
    cell, off, v = O.fd_load(2, (nx, ny, 1), None, O.KIND_BOUND, I.ME, 0, 0, 0, 16, True, 3, 0)
    X = I.cell_coords(cell, (nx, ny, 1)) + off
    k = 2 * math.pi / (nx * dx)
    D = np.zeros_like(X)
    D[:, 0] = 1e-12 * np.sin(k * X[:, 0] * dx)
    w = nb * dx ** 3 / 16
    species = [dict(kind=I.BOUND, q=-I.QE, m=I.ME, w=w, cell=cell.astype(np.int32),
                    anchor_off=off.astype(np.float64), disp=D.astype(np.float32),
                    v=v.astype(np.float32), omega0=(w0,) * 3, gamma=(gam,) * 3, background=1)]
    i = np.arange(nx)
    Ex = -nb * (-I.QE) * 1e-12 * np.sin(k * (i + 0.5) * dx) / I.EPS0
    pic = _pic()
    h = PR.gpu_sim(grid, None, species, fields={0: np.broadcast_to(Ex, (1, ny, nx)).copy()})
    wpb2 = nb * I.QE ** 2 / (I.EPS0 * I.ME)
    wL = math.sqrt(w0 ** 2 + wpb2 - gam ** 2 / 4)
    nsteps = int(3 * 2 * math.pi / (wL * dt))
    t, y = [], []
    try:
        for it in range(nsteps // 5):
            pic.pic_step(h, 5)
            E = pic.pic_read_fields(h, pic.PIC_EX, I.grid_shape(grid["n"]))[0, 0].mean(axis=0)
            y.append(2 / nx * np.sum(E * np.sin(k * (i + 0.5) * dx)))
            t.append((it + 1) * 5 * dt)
    finally:
        pic.pic_destroy(h)
    t, y = np.array(t), np.array(y)
    wfit = _fit_frequency(t, y * np.exp(gam * t / 2), wL)
    assert abs(wfit / wL - 1) < 0.01
    A = np.stack([np.cos(wL * t), np.sin(wL * t)], 1)
    half = len(t) // 2
    a1 = np.linalg.lstsq(A[:half], y[:half], rcond=None)[0]
    a2 = np.linalg.lstsq(A[half:], y[half:], rcond=None)[0]
    ratio = np.linalg.norm(a2) / np.linalg.norm(a1)
    pred = math.exp(-gam / 2 * (t[half:].mean() - t[:half].mean()))
    assert abs(ratio / pred - 1) < 0.05


@pytest.mark.parametrize("overlap", [0, 1])
def test_tma_b_pass_interior_blocks(overlap):
    """The split update with the TMA-fed B pass on the interior field blocks
    (3D, CPML 6 on every face, 96 x 40 x 64 cells: blocks at x 32-63, y 8-31,
    z 16-31 take it, next to CPML blocks on every side) matches the oracle
    after 1 and 30 steps and the plain-load path (no TMA) to roundoff."""
    n = (96, 40, 64)
    d = (1e-9, 0.8e-9, 1.1e-9)
    dt = 0.45 * min(d) / (I.C_LIGHT * math.sqrt(3))
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=(1, 1, 1), pml_cells=6,
                src=dict(inc_axis=0, pol_axis=1, src_index=9, E0=1e8,
                         omega=2 * np.pi * I.C_LIGHT / 30e-9, tau=4e-17, t0=6e-17))
    fields = _plane_wave_fields(grid)
    pic = _pic()
    h = PR.gpu_sim(grid, None, [], fields=fields,
                   tuning=dict(no_overlap=1 - overlap, field_mode=2))
    hp = PR.gpu_sim(grid, None, [], fields=fields,
                    tuning=dict(no_overlap=1 - overlap, field_mode=2, field_plain=1))
    s = PR.oracle_sim(grid, None, [], fields=fields)
    try:
        for nsteps, tol in ((1, 1e-5), (29, 1e-4)):
            pic.pic_step(h, nsteps)
            pic.pic_step(hp, nsteps)
            s.step(nsteps)
            got = PR.gpu_fields(h, grid)
            plain = PR.gpu_fields(hp, grid)
            for c in range(6):
                assert PR.rel_l2(got[c], s.field(c)) < tol, (c, nsteps)
                assert PR.rel_l2(got[c], plain[c]) < 1e-6, (c, nsteps)
        pic.pic_sync(h)
    finally:
        pic.pic_destroy(h)
        pic.pic_destroy(hp)
        s.close()


def test_tma_wait_timeout_is_latched_and_the_device_recovers():
    """The bounded waits of the TMA-fed B pass: with a limit of one poll the
    pass gives up on its copies, latches PIC_ETIMEOUT (reported by pic_sync),
    still waits -- at the full bound -- for the copies it has in flight before
    each CTA exits, and the handle is destroyed cleanly.  A fresh handle then
    runs the same grid normally and matches the oracle."""
    n = (96, 40, 64)
    d = (1e-9, 0.8e-9, 1.1e-9)
    dt = 0.45 * min(d) / (I.C_LIGHT * math.sqrt(3))
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=(1, 1, 1), pml_cells=6)
    fields = _plane_wave_fields(grid)
    pic = _pic()
    h = PR.gpu_sim(grid, None, [], fields=fields, tuning=dict(field_mode=2, wait_polls=1))
    try:
        pic.pic_step(h, 3)
        with pytest.raises(pic.PicError) as e:
            pic.pic_sync(h)
        assert e.value.status == pic.PIC_ETIMEOUT
    finally:
        pic.pic_destroy(h)
    h = PR.gpu_sim(grid, None, [], fields=fields, tuning=dict(field_mode=2))
    s = PR.oracle_sim(grid, None, [], fields=fields)
    try:
        pic.pic_step(h, 3)
        pic.pic_sync(h)
        s.step(3)
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-5, c
    finally:
        pic.pic_destroy(h)
        s.close()


@pytest.mark.parametrize("overlap", [0, 1])
def test_tma_passes_with_current_3d_periodic(overlap):
    """3D periodic plasma (64 x 24 x 40 cells, free electrons everywhere):
    the interior field blocks go through the TMA-fed B pass while the E pass
    applies the deposited current of every block.  Fields match the oracle
    after 1 step (1e-5) and 20 steps (1e-3), and the plain-load path (no
    TMA) to 1e-5 (atomics order the current sums differently)."""
    rng = np.random.default_rng(31)
    n = (64, 24, 40)
    d = (0.1e-9, 0.1e-9, 0.1e-9)
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(3))
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=(0, 0, 0))
    cell, off, v = I.random_particles(rng, n, 120000, vscale=2e6)
    w = 8.5e28 * np.prod(d) / 2
    species = [dict(kind=I.FREE, q=-I.QE, m=I.ME, w=w, cell=cell, off=off, v=v, background=2)]
    pic = _pic()
    s = PR.oracle_sim(grid, None, species)
    h = PR.gpu_sim(grid, None, species, tuning=dict(no_overlap=1 - overlap, field_mode=2))
    hp = PR.gpu_sim(grid, None, species,
                    tuning=dict(no_overlap=1 - overlap, field_mode=2, field_plain=1))
    try:
        for nsteps, tol in ((1, 1e-5), (19, 1e-3)):
            pic.pic_step(h, nsteps)
            pic.pic_step(hp, nsteps)
            s.step(nsteps)
            got = PR.gpu_fields(h, grid)
            plain = PR.gpu_fields(hp, grid)
            for c in range(6):
                ref = s.field(c)
                if np.linalg.norm(ref) > 0:
                    assert PR.rel_l2(got[c], ref) < tol, (c, nsteps)
                    assert PR.rel_l2(got[c], plain[c]) < 1e-5, (c, nsteps)
        pic.pic_sync(h)
    finally:
        pic.pic_destroy(h)
        pic.pic_destroy(hp)
        s.close()


@pytest.mark.parametrize("overlap", [0, 1])
def test_permittivity_matches_oracle(overlap):
    """Eq. consteps with a per-cell eps_r: the metal sphere (free and bound
    electrons, CPML, plane-wave source) with a dielectric slab (eps_r = 2.5)
    through it and a second one (eps_r = 6) in vacuum.  Fields match the
    oracle after 1 step (1e-5) and 40 steps (1e-3); the Gauss residual on D
    stays at roundoff (FP32 on the GPU, FP64 in the oracle)."""
    rng = np.random.default_rng(41)
    # no initial bound displacement: ions at the anchors neutralise the start,
    # so the Gauss residual on D begins (and must stay) at roundoff
    grid, mask, species = _sphere_case(rng, n=(32, 28, 24), bc=(0, 0, 0), dscale=0.0)
    grid["src"] = None
    n = grid["n"]
    eps = np.ones((n[2], n[1], n[0]), np.float32)
    eps[:, :, 12:18] = 2.5
    eps[:, 2:6, 24:29] = 6.0
    pic = _pic()
    s = PR.oracle_sim(grid, mask, species)
    s.set_permittivity(eps.astype(np.float64))
    h = PR.gpu_sim(grid, mask, species, tuning=dict(no_overlap=1 - overlap, field_mode=2))
    pic.pic_set_permittivity(h, eps)
    try:
        for nsteps, tol in ((1, 1e-5), (39, 1e-3)):
            pic.pic_step(h, nsteps)
            s.step(nsteps)
            got = PR.gpu_fields(h, grid)
            for c in range(6):
                ref = s.field(c)
                if np.linalg.norm(ref) > 0:
                    assert PR.rel_l2(got[c], ref) < tol, (c, nsteps, PR.rel_l2(got[c], ref))
        dg = pic.pic_diagnostics(h)
        od = s.diag()
        qs = I.QE * 5.9e28 / 8 / I.EPS0  # one macro-particle's charge density / eps0
        assert od["gauss_max"] < 1e-10 * qs
        assert dg["gauss_max"] < 1e-5 * qs
        assert abs(dg["field_E"] / od["field_E"] - 1) < 1e-3
    finally:
        pic.pic_destroy(h)
        s.close()


def test_dielectric_half_space_fresnel_on_gpu():
    """The Fresnel pin of the oracle run by the GPU path: a pulse in vacuum on
    an eps_r = 4 half-space reflects 1/3 and transmits 2/3 of its amplitude
    within 2 %."""
    nx = 1200
    n = (nx, 2, 1)
    d = (1e-9, 1e-9, 1e-9)
    dt = 0.5 * 1e-9 / (I.C_LIGHT * math.sqrt(2))
    tau = 0.25e-15
    grid = dict(dims=2, n=n, d=d, dt=dt, bc=(1, 0, 0), pml_cells=16,
                src=dict(inc_axis=0, pol_axis=1, src_index=40, E0=1e8,
                         omega=2 * math.pi * I.C_LIGHT / 80e-9, tau=tau, t0=3 * tau))
    eps = np.ones((1, 2, nx), np.float32)
    eps[..., 700:] = 4.0
    pic = _pic()
    h = PR.gpu_sim(grid, None, [])
    pic.pic_set_permittivity(h, eps)
    pa, pb = 200, 800
    nsteps = int((3 * tau * I.C_LIGHT / 1e-9 + 1560) / (I.C_LIGHT * dt / 1e-9))
    t, ea, eb = [], [], []
    try:
        for it in range(nsteps):
            pic.pic_step(h, 1)
            E = pic.pic_read_fields(h, pic.PIC_EY, I.grid_shape(n))[0, 0, 0]
            t.append((it + 1) * dt)
            ea.append(abs(E[pa]))
            eb.append(abs(E[pb]))
    finally:
        pic.pic_destroy(h)
    t, ea, eb = np.array(t), np.array(ea), np.array(eb)
    split = 3 * tau + (pa - 40 + 500) * 1e-9 / I.C_LIGHT
    inc, ref, tra = ea[t < split].max(), ea[t > split].max(), eb.max()
    assert abs(ref / inc - 1 / 3) < 0.02 / 3
    assert abs(tra / inc - 2 / 3) < 0.02 * 2 / 3


def test_permittivity_arguments():
    """Wrong size, non-positive or NaN values and the fused field modes are
    refused with PIC_EINVAL / PIC_ESTATE; NULL returns to vacuum."""
    pic = _pic()
    n = (8, 8, 8)
    grid = dict(dims=3, n=n, d=(1e-9,) * 3, dt=1e-18, bc=(0, 0, 0))
    h = PR.gpu_sim(grid, None, [])
    try:
        good = np.full((8, 8, 8), 2.0, np.float32)
        for bad in (np.full(10, 2.0, np.float32), -good, good * np.nan, good * 0):
            with pytest.raises(pic.PicError) as e:
                pic.pic_set_permittivity(h, bad)
            assert e.value.status == pic.PIC_EINVAL
        pic.pic_set_permittivity(h, good)
        with pytest.raises(pic.PicError) as e:
            pic.pic_set_tuning(h, field_mode=3)
        assert e.value.status == pic.PIC_EINVAL
        pic.pic_set_permittivity(h, None)
        pic.pic_set_tuning(h, field_mode=1)
        with pytest.raises(pic.PicError) as e:
            pic.pic_set_permittivity(h, good)
        assert e.value.status == pic.PIC_ESTATE
    finally:
        pic.pic_destroy(h)


def test_lorentz_half_space_reflection_spectrum_on_gpu():
    """The bound species as a dielectric (Sec. 4, Eq. lordielectric): a pulse
    reflected by a half-space of Lorentz-bound electrons has the spectrum
    |r(omega)| = |(1 - n)/(1 + n)|, n^2 = 1 + w_pb^2 / (w0^2 - w^2 - i gamma w),
    within 1 % over w = 0.34 .. 0.66 w0 (|r| about 0.44) -- the closed-form
    counterpart of the paper's comparison with a full-wave solver."""
    grid, mask, sp, steps, prm = PR.lorentz_half_space_case()
    pic = _pic()
    h = PR.gpu_sim(grid, mask, [sp])
    trace = np.zeros(steps)
    try:
        for it in range(steps):
            pic.pic_step(h, 1)
            trace[it] = pic.pic_read_fields(h, pic.PIC_EY, I.grid_shape(grid["n"]))[0, 0, 0, 100]
    finally:
        pic.pic_destroy(h)
    err, band = PR.lorentz_reflection_error(trace, **prm)
    assert band.min() < 0.36 * prm["w0"] and band.max() > 0.64 * prm["w0"]
    assert err < 0.01, err


def test_a_smaller_box_created_later_does_not_refuse_a_larger_one():
    """The particle kernels' shared-memory limit is a property of the kernel,
    not of one simulation: a simulation with a large staged box (16 x 16 x 8
    tile) still steps after one with a small box (4 x 4 x 2) was created,
    and both match what they give alone."""
    rng = np.random.default_rng(41)
    n = (24, 20, 16)
    d = (0.5e-9,) * 3
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(3))
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=(0, 0, 0))
    cell, off, v = I.random_particles(rng, n, 20000, vscale=2e6)
    species = [dict(kind=I.FREE, q=-I.QE, m=I.ME, w=1e3, cell=cell, off=off, v=v)]
    pic = _pic()
    big = PR.gpu_sim(grid, None, species, tuning=dict(tile=(16, 16, 8)))
    small = PR.gpu_sim(grid, None, species, tuning=dict(tile=(4, 4, 2)))
    s = PR.oracle_sim(grid, None, species)
    try:
        pic.pic_step(big, 3)
        pic.pic_step(small, 3)
        s.step(3)
        for h in (big, small):
            pic.pic_sync(h)
            got = PR.gpu_fields(h, grid)
            for c in range(6):
                if np.linalg.norm(s.field(c)) > 0:
                    assert PR.rel_l2(got[c], s.field(c)) < 1e-4, c
    finally:
        pic.pic_destroy(big)
        pic.pic_destroy(small)
        s.close()
