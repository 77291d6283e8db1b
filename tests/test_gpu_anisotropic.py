"""GPU parity of bound species with diagonal binding and damping tensors
(Eq. modlorentz with omega0 = diag(w0x, w0y, w0z), gamma = diag(gx, gy, gz);
the general 3x3 solve of the modified Boris rotation, Appendix A.2).

Bars as in the other parity tests: one step against the oracle particle by
particle (1e-5), fields 1e-5 after one step and 1e-3 after 30 steps; and at
a size beyond the oracle, the per-axis closed forms of a uniform Lorentz
medium.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_07465_gb300 import inputs as I

from tests import pairs as PR

pytestmark = pytest.mark.gpu

W0 = (4.709e15, 3.2e15, 6.0e15)
GAMMA = (1e14, 3e14, 5e13)


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


@pytest.mark.parametrize("overlap,mode", [(1, 2), (0, 2), (1, 1)])
def test_anisotropic_bound_matches_oracle(overlap, mode):
    """The metal sphere with bound electrons of diagonal omega0 and gamma,
    driven by the plane-wave source (so B couples the axes in the rotation):
    one step matches the oracle particle by particle, 30 more steps match in
    the fields (1e-3) and in 99 % of the bound velocities (1e-4)."""
    rng = np.random.default_rng(61)
    grid, mask, species = PR.sphere_case(rng, omega0=W0, gamma=GAMMA)
    species = PR.guarded_species(grid, mask, species, lambda s: None)
    pic = _pic()
    s = PR.oracle_sim(grid, mask, species)
    h = PR.gpu_sim(grid, mask, species, tuning=dict(no_overlap=1 - overlap, field_mode=mode))
    try:
        PR.compare_one_step(pic, h, s, grid, species)
        pic.pic_step(h, 30)
        s.step(30)
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
        _, Vb, Db, _ = s.species(1)
        rb = pic.pic_read_species(h, 1, species[1]["cell"].size, bound=True)
        rel = np.linalg.norm(rb["v"] - Vb, axis=1) / np.maximum(np.linalg.norm(Vb, axis=1), 1e3)
        assert np.quantile(rel, 0.99) < 1e-4
    finally:
        pic.pic_destroy(h)
        s.close()


@pytest.mark.parametrize("tile", [(8, 8, 4), (8, 8, 2)])
def test_isotropic_gamma_unchanged_by_the_variant_kernel(tile):
    """Equal gamma entries keep the closed-form solve in both kernels: with
    an all-zero external field (which selects the variant kernel) the bound
    velocities after one step are bit-equal to the plain kernel's -- the
    lean kernel of the default tile and the generic one of another tile.
    The first step sees no field, so the comparison isolates the push."""
    rng = np.random.default_rng(62)
    grid, mask, species = PR.sphere_case(rng, nfree=2000, nbound=4000)
    pic = _pic()
    h0 = PR.gpu_sim(grid, mask, species, tuning=dict(tile=tile))
    h1 = PR.gpu_sim(grid, mask, species, tuning=dict(tile=tile))
    pic.pic_set_external_field(h1, np.zeros((3,) + I.grid_shape(grid["n"])))
    try:
        pic.pic_step(h0, 1)
        pic.pic_step(h1, 1)
        r0 = pic.pic_read_species(h0, 1, species[1]["cell"].size, bound=True)
        r1 = pic.pic_read_species(h1, 1, species[1]["cell"].size, bound=True)
        assert np.array_equal(r0["v"], r1["v"]) and np.array_equal(r0["disp"], r1["disp"])
    finally:
        pic.pic_destroy(h0)
        pic.pic_destroy(h1)


def _fit_frequency(t, y, w_guess):
    ws = np.linspace(0.9 * w_guess, 1.1 * w_guess, 4001)
    best, wbest = -1.0, w_guess
    for w in ws:
        A = np.stack([np.cos(w * t), np.sin(w * t)], 1)
        c = np.linalg.lstsq(A, y, rcond=None)[0]
        r = np.linalg.norm(A @ c)
        if r > best:
            best, wbest = r, w
    return wbest


@pytest.mark.parametrize("axis", [0, 1])
def test_anisotropic_medium_rings_per_axis(axis):
    """A uniform Lorentz medium with diagonal omega0 and gamma (2D periodic,
    16 ppc bound electrons, N_b = 0.5 x 5.9e28 m^-3) started from a k-mode
    displacement along `axis`: the longitudinal mode rings at
    sqrt(w0_a^2 + w_pb^2 - gamma_a^2/4) within 1 % and decays as
    exp(-gamma_a t / 2) within 5 % -- the two axes differ by 6 % in
    frequency and 3x in damping."""
    nb = 0.5 * 5.9e28
    nk, nt = 32, 2
    n = (nk, nt, 1) if axis == 0 else (nt, nk, 1)
    dx = 0.5e-9
    dt = 0.5 * dx / (I.C_LIGHT * math.sqrt(2))
    w0, gam = W0[axis], GAMMA[axis]
    grid = dict(dims=2, n=n, d=(dx, dx, dx), dt=dt, bc=(0, 0, 0))
    cell, off, v = O.fd_load(2, n, None, O.KIND_BOUND, I.ME, 0, 0, 0, 16, True, 3, 0)
    X = I.cell_coords(cell, n) + off
    k = 2 * math.pi / (nk * dx)
    D = np.zeros_like(X)
    D[:, axis] = 1e-12 * np.sin(k * X[:, axis] * dx)
    w = nb * dx ** 3 / 16
    species = [dict(kind=I.BOUND, q=-I.QE, m=I.ME, w=w, cell=cell.astype(np.int32),
                    anchor_off=off.astype(np.float64), disp=D.astype(np.float32),
                    v=v.astype(np.float32), omega0=W0, gamma=GAMMA, background=1)]
    i = np.arange(nk)
    Ek = -nb * (-I.QE) * 1e-12 * np.sin(k * (i + 0.5) * dx) / I.EPS0
    E0 = np.broadcast_to(Ek, (1, nt, nk)) if axis == 0 else np.broadcast_to(Ek[:, None], (1, nk, nt))
    pic = _pic()
    h = PR.gpu_sim(grid, None, species, fields={axis: E0.copy()})
    wpb2 = nb * I.QE ** 2 / (I.EPS0 * I.ME)
    wL = math.sqrt(w0 ** 2 + wpb2 - gam ** 2 / 4)
    nsteps = int(6 * 2 * math.pi / (wL * dt))
    t, y = [], []
    bit = pic.PIC_EX if axis == 0 else pic.PIC_EY
    try:
        for it in range(nsteps // 5):
            pic.pic_step(h, 5)
            E = pic.pic_read_fields(h, bit, I.grid_shape(n))[0, 0]
            prof = E.mean(axis=0) if axis == 0 else E.mean(axis=1)
            y.append(2 / nk * np.sum(prof * np.sin(k * (i + 0.5) * dx)))
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


def test_gamma_arguments():
    """Negative or NaN gamma entries are refused with PIC_EINVAL; a group
    takes a simulation with an anisotropic gamma."""
    pic = _pic()
    n = (8, 8, 8)
    grid = dict(dims=3, n=n, d=(1e-9,) * 3, dt=1e-18, bc=(0, 0, 0))
    rng = np.random.default_rng(5)
    cb, anc, disp, vb = I.random_bound(rng, n, 100)
    h = PR.gpu_sim(grid, None, [])
    g = None
    try:
        for gam in ((-1e14, 0, 0), (float("nan"),) * 3, (0, float("inf"), 0)):
            desc = pic.species_desc(I.BOUND, -I.QE, I.ME, 1.0, omega0=W0, gamma=gam)
            with pytest.raises(pic.PicError) as e:
                pic.pic_load_species(h, desc, cell=cb, v=vb, anchor_off=anc, disp=disp)
            assert e.value.status == pic.PIC_EINVAL
        desc = pic.species_desc(I.BOUND, -I.QE, I.ME, 1.0, omega0=W0, gamma=GAMMA)
        pic.pic_load_species(h, desc, cell=cb, v=vb, anchor_off=anc, disp=disp)
        g = pic.pic_group_create(4)
        pic.pic_group_add(g, h, 1)
        pic.pic_group_remove(g, h)
    finally:
        if g is not None:
            pic.pic_group_destroy(g)
        pic.pic_destroy(h)


def _rotated_tensor():
    """Omega^2 = R diag(W0^2) R^T for a rotation about z then x: the diagonal
    (as omega0) and the off-diagonal entries (xy, xz, yz)."""
    a, b = 0.7, -0.4
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    R = Rz @ Rx
    W2 = R @ np.diag(np.array(W0) ** 2) @ R.T
    return tuple(np.sqrt(np.diag(W2))), np.array([W2[0, 1], W2[0, 2], W2[1, 2]])


@pytest.mark.parametrize("overlap", [1, 0])
def test_binding_tensor_matches_oracle(overlap):
    """Bound electrons with a full (rotated) binding tensor in the driven
    metal sphere: one step particle by particle (1e-5), 30 more steps in the
    fields (1e-3) and 99 % of the bound velocities (1e-4)."""
    rng = np.random.default_rng(63)
    omega0, off = _rotated_tensor()
    grid, mask, species = PR.sphere_case(rng, omega0=omega0, gamma=GAMMA)
    species = PR.guarded_species(grid, mask, species, lambda s: s.set_binding_offdiag(1, off))
    pic = _pic()
    s = PR.oracle_sim(grid, mask, species)
    s.set_binding_offdiag(1, off)
    h = PR.gpu_sim(grid, mask, species, tuning=dict(no_overlap=1 - overlap, field_mode=2))
    pic.pic_set_binding_tensor(h, 1, off)
    try:
        PR.compare_one_step(pic, h, s, grid, species)
        pic.pic_step(h, 30)
        s.step(30)
        got = PR.gpu_fields(h, grid)
        for c in range(6):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
        _, Vb, _, _ = s.species(1)
        rb = pic.pic_read_species(h, 1, species[1]["cell"].size, bound=True)
        rel = np.linalg.norm(rb["v"] - Vb, axis=1) / np.maximum(np.linalg.norm(Vb, axis=1), 1e3)
        assert np.quantile(rel, 0.99) < 1e-4
    finally:
        pic.pic_destroy(h)
        s.close()


def test_binding_tensor_arguments():
    """A tensor that is not positive definite, NaN entries or a free species
    are refused (PIC_EINVAL); a tensor too stiff for dt (Eq. dtlimit with the
    Gershgorin bound of its largest eigenvalue) gives PIC_EDTLIMIT."""
    pic = _pic()
    n = (8, 8, 8)
    grid = dict(dims=3, n=n, d=(1e-9,) * 3, dt=1e-18, bc=(0, 0, 0))
    rng = np.random.default_rng(7)
    cb, anc, disp, vb = I.random_bound(rng, n, 50)
    cell, off, v = I.random_particles(rng, n, 50)
    h = PR.gpu_sim(grid, None, [])
    try:
        pic.pic_load_species(h, pic.species_desc(I.FREE, -I.QE, I.ME, 1.0), cell=cell, off=off,
                             v=v)
        pic.pic_load_species(h, pic.species_desc(I.BOUND, -I.QE, I.ME, 1.0, omega0=W0,
                                                 gamma=GAMMA),
                             cell=cb, v=vb, anchor_off=anc, disp=disp)
        w = np.array(W0) ** 2
        for k, bad in ((1, [w[0], 0, 0]), (1, [0, float("nan"), 0]), (0, [1e30, 0, 0])):
            with pytest.raises(pic.PicError) as e:
                pic.pic_set_binding_tensor(h, k, bad)
            assert e.value.status == pic.PIC_EINVAL
        pic.pic_set_binding_tensor(h, 1, [0.5 * math.sqrt(w[0] * w[1]), 0, 0])  # accepted
    finally:
        pic.pic_destroy(h)
    # stiff binding: omega0 = 1.3e18 s^-1 loads (Eq. dtlimit: 1.2e-18 s >
    # dt), but with all off-diagonal entries 0.9 omega0^2 (positive
    # definite, eigenvalues 2.8 and 0.1 omega0^2) the limit drops to
    # 8.3e-19 s
    h = PR.gpu_sim(grid, None, [])
    try:
        w0 = 1.3e18
        pic.pic_load_species(h, pic.species_desc(I.BOUND, -I.QE, I.ME, 1.0, omega0=(w0,) * 3),
                             cell=cb, v=vb, anchor_off=anc, disp=disp)
        with pytest.raises(pic.PicError) as e:
            pic.pic_set_binding_tensor(h, 0, [0.9 * w0 ** 2] * 3)
        assert e.value.status == pic.PIC_EDTLIMIT
    finally:
        pic.pic_destroy(h)


def test_binding_tensor_counts_in_later_species_dt_limit():
    """Eq. dtlimit for a species loaded after a binding tensor uses the
    tensor's bound, not the diagonal omega0^2 alone.  dx = 1 nm, dt = 1e-18 s:
    the limit holds while omega_b^2 + omega_p^2 < 2.92e36 s^-2.  The bound
    species (omega0 = 1e18 s^-1) with off-diagonal entries 0.5 omega0^2 has
    the Gershgorin bound 2e36 (accepted); a free species adding
    omega_p^2 = 1.2e36 then exceeds the limit (it would pass against the
    diagonal 1e36)."""
    pic = _pic()
    n = (8, 8, 8)
    grid = dict(dims=3, n=n, d=(1e-9,) * 3, dt=1e-18, bc=(0, 0, 0))
    rng = np.random.default_rng(8)
    cb, anc, disp, vb = I.random_bound(rng, n, 50)
    cell, off, v = I.random_particles(rng, n, 50)
    w0 = 1e18
    dens = 1.2e36 * I.ME * I.EPS0 / I.QE ** 2
    for with_tensor in (False, True):
        h = PR.gpu_sim(grid, None, [])
        try:
            pic.pic_load_species(h, pic.species_desc(I.BOUND, -I.QE, I.ME, 1.0,
                                                     omega0=(w0,) * 3),
                                 cell=cb, v=vb, anchor_off=anc, disp=disp, density=1.0)
            if with_tensor:
                pic.pic_set_binding_tensor(h, 0, [0.5 * w0 ** 2] * 3)
                with pytest.raises(pic.PicError) as e:
                    pic.pic_load_species(h, pic.species_desc(I.FREE, -I.QE, I.ME, 1.0),
                                         cell=cell, off=off, v=v, density=dens)
                assert e.value.status == pic.PIC_EDTLIMIT
            else:
                pic.pic_load_species(h, pic.species_desc(I.FREE, -I.QE, I.ME, 1.0),
                                     cell=cell, off=off, v=v, density=dens)
        finally:
            pic.pic_destroy(h)
