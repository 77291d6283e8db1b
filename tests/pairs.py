"""Helpers for parity tests: run the same seeded inputs through the CUDA
path (via the C ABI binding) and through the FP64 oracle."""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O
from paper_2501_07465_gb300 import inputs as I

FIELD_BITS = [1, 2, 4, 8, 16, 32]


def oracle_grid(grid):
    g = dict(grid)
    src = g.pop("src", None)
    if src:
        g.update(src=True, **src)
    return g


def species_arrays_for_oracle(sp, n):
    """Explicit species dict -> (X, V, D) for the oracle."""
    if sp["kind"] == I.BOUND:
        X = I.cell_coords(sp["cell"], n) + sp["anchor_off"]
        D = np.asarray(sp.get("disp", np.zeros_like(X)), np.float64)
    else:
        X = I.positions(sp["cell"], sp["off"], n)
        D = None
    return X, np.asarray(sp["v"], np.float64), D


def oracle_sim(grid, mask, species, fields=None):
    s = O.OracleSim(**oracle_grid(grid))
    n = tuple(grid["n"])
    if mask is not None:
        s.set_mask(mask)
    for sp in species:
        if "cell" not in sp:  # loader request: the oracle draws its own particles
            cell, off, v = O.fd_load(grid["dims"], n, mask, sp["kind"], sp["m"], sp.get("E_F", 0.0),
                                     sp.get("T", 0.0), sp.get("v_F", 0.0), sp["ppc"],
                                     sp.get("quiet", 0), sp["seed"], sp.get("stream", 0))
            w = sp["density"] * np.prod(grid["d"]) / sp["ppc"]
            X = I.cell_coords(cell, n) + off
            if sp["kind"] == I.BOUND:
                s.add_species(sp["kind"], sp["q"], sp["m"], w, X, v, D=np.zeros_like(X),
                              omega0=sp.get("omega0", (0, 0, 0)), gamma=sp.get("gamma", (0, 0, 0)),
                              bg=sp.get("background", 0))
            else:
                s.add_species(sp["kind"], sp["q"], sp["m"], w, X, v, vF=sp.get("v_F", 0.0),
                              bg=sp.get("background", 0))
            continue
        X, V, D = species_arrays_for_oracle(sp, n)
        s.add_species(sp["kind"], sp["q"], sp["m"], sp["w"], X, V, D=D,
                      omega0=sp.get("omega0", (0, 0, 0)), gamma=sp.get("gamma", (0, 0, 0)),
                      vF=sp.get("v_F", 0.0), bg=sp.get("background", 0))
    if fields:
        for comp, arr in fields.items():
            s.set_field(comp, arr)
    return s


def gpu_sim(grid, mask, species, fields=None, tuning=None):
    import torch

    from paper_2501_07465_gb300 import pic
    pic.use_torch_allocator()
    g = pic.make_grid(grid["dims"], grid["n"], grid["d"], grid["dt"], bc=grid.get("bc", (0, 0, 0)),
                      pml_cells=grid.get("pml_cells", 0), src=grid.get("src"))
    h = pic.pic_create(g, torch.cuda.current_stream().cuda_stream)
    if tuning:
        pic.pic_set_tuning(h, **tuning)
    if mask is not None:
        pic.pic_set_material_mask(h, mask)
    for sp in species:
        desc = pic.species_desc(sp["kind"], sp["q"], sp["m"], sp.get("w", 0.0),
                                omega0=sp.get("omega0", (0, 0, 0)), gamma=sp.get("gamma", (0, 0, 0)),
                                v_F=sp.get("v_F", 0.0), background=sp.get("background", 0))
        if "cell" in sp:
            pic.pic_load_species(h, desc, cell=sp["cell"], off=sp.get("off"), v=sp["v"],
                                 anchor_off=sp.get("anchor_off"), disp=sp.get("disp"),
                                 density=sp.get("density", 0.0))
        else:
            pic.pic_load_species(h, desc, density=sp["density"], E_F=sp.get("E_F", 0.0),
                                 T=sp.get("T", 0.0), ppc=sp["ppc"], quiet=sp.get("quiet", 0),
                                 seed=sp["seed"], stream=sp.get("stream", 0))
    if fields:
        which = 0
        arrs = []
        for comp in sorted(fields):
            which |= FIELD_BITS[comp]
            arrs.append(fields[comp])
        pic.pic_write_fields(h, which, np.stack(arrs))
    return h


def gpu_fields(h, grid, comps=range(6)):
    from paper_2501_07465_gb300 import pic
    which = 0
    for c in comps:
        which |= FIELD_BITS[c] if c < 6 else (64 << (c - 6))
    return pic.pic_read_fields(h, which, I.grid_shape(grid["n"]))


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def gpu_positions(rd, n):
    """Readback dict -> positions in cell units (float64)."""
    if "off" in rd:
        return I.positions(rd["cell"], rd["off"], n)
    return I.cell_coords(rd["cell"], n) + rd["anchor_off"]


def periodic_delta(a, b, n, dims):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    for ax in range(dims):
        L = n[ax]
        d[:, ax] = (d[:, ax] + L / 2) % L - L / 2
    return d


def near_face(X, dims, tol=1e-4):
    """True where a position lies within tol (cells) of a cell face."""
    f = np.asarray(X, np.float64)[:, :dims] % 1.0
    return np.any((f < tol) | (f > 1 - tol), axis=1)


# ---------------------------------------------------------------------------
# the Lorentz half-space reflection case (Sec. 4, Eq. lordielectric)
# ---------------------------------------------------------------------------

def lorentz_reflection_error(trace, dt, tau, dx, w0, gam, wpb2):
    """|r(omega)| of the reflected over the incident pulse at the probe (100
    cells from the source sheet at 40, the half-space from 500) against
    Fresnel with the bound species' eps(omega) in the exact discrete form of
    the leapfrog oscillator (Eq. dispersion1 read with sin terms), over the
    band where the incident spectrum exceeds 20 % of its peak."""
    t = (np.arange(trace.size) + 1) * dt
    split = 3 * tau + (60 + 400) * dx / I.C_LIGHT
    inc = np.fft.rfft(np.where(t < split, trace, 0.0), 1 << 16)
    ref = np.fft.rfft(np.where(t >= split, trace, 0.0), 1 << 16)
    w = 2 * np.pi * np.fft.rfftfreq(1 << 16, dt)
    band = np.abs(inc) > 0.2 * np.abs(inc).max()
    den = w0 ** 2 * dt ** 2 - 4 * np.sin(w * dt / 2) ** 2 - 1j * gam * dt * np.sin(w * dt)
    n = np.sqrt((1 + wpb2 * dt ** 2 / den).astype(complex))
    n = np.where(n.imag < 0, -n, n)
    r_th = np.abs((1 - n) / (1 + n))
    r = np.abs(ref) / np.maximum(np.abs(inc), 1e-300)
    return float(np.abs(r[band] / r_th[band] - 1).max()), w[band]


def lorentz_half_space_case():
    """A 2D3V grid (1600 x 2 cells of 10 nm, CPML along x) with bound
    electrons (the sphere workload's w0, gamma and N_b, 4 ppc quiet lattice,
    ions at the anchors) filling x in [500, 1400) cells, and an 800 nm pulse
    (FWHM 4 fs) launched from x = 40."""
    nx, dx = 1600, 10e-9
    dt = 0.5 * dx / (I.C_LIGHT * math.sqrt(2))
    w0, gam, nb = 2 * np.pi * I.C_LIGHT / 400e-9, 1e14, 0.5 * 5.9e28
    tau = 4e-15
    grid = dict(dims=2, n=(nx, 2, 1), d=(dx,) * 3, dt=dt, bc=(1, 0, 0), pml_cells=16,
                src=dict(inc_axis=0, pol_axis=1, src_index=40, E0=1e7,
                         omega=2 * np.pi * I.C_LIGHT / 800e-9, tau=tau, t0=3 * tau))
    mask = np.zeros((1, 2, nx), np.uint8)
    mask[..., 500:1400] = 1
    sp = dict(kind=I.BOUND, q=-I.QE, m=I.ME, density=nb, ppc=4, quiet=1, seed=7, E_F=0.0, T=0.0,
              omega0=(w0,) * 3, gamma=(gam,) * 3, background=1)
    steps = int((3 * tau + 860 * dx / I.C_LIGHT + 6 * tau + 20e-15) / dt)
    wpb2 = nb * I.QE ** 2 / (I.EPS0 * I.ME)
    return grid, mask, sp, steps, dict(dt=dt, tau=tau, dx=dx, w0=w0, gam=gam, wpb2=wpb2)

# ---------------------------------------------------------------------------
# the metal-sphere parity case shared by the GPU tests
# ---------------------------------------------------------------------------

def vel_rel(vg, vo, floor):
    """Largest per-particle velocity difference relative to max(|v|, floor)."""
    return np.max(np.linalg.norm(vg - vo, axis=1) / np.maximum(np.linalg.norm(vo, axis=1), floor))


def shell_cells(mask):
    """Material cells with a vacuum face neighbour (outside the grid counts
    as vacuum), as linear indices."""
    m = np.asarray(mask, bool)
    pad = np.pad(m, 1, constant_values=False)
    vac_nb = np.zeros_like(m)
    for ax in range(3):
        if m.shape[ax] == 1:
            continue
        for sh in (-1, 1):
            vac_nb |= ~np.take(np.roll(pad, sh, axis=ax), range(1, m.shape[ax] + 1), axis=ax)[
                tuple(slice(1, -1) if a != ax else slice(None) for a in range(3))]
    return np.flatnonzero((m & vac_nb).ravel())


def sphere_case(rng, n=(32, 28, 24), nfree=6000, nbound=3000, vscale=4e6, shell=False,
                omega0=None, gamma=(1e14,) * 3):
    """A metal sphere (radius 8 cells of 0.5 nm) of free and bound
    electrons with ions at the loaded positions, CPML on every face and a
    plane-wave source; shell=True loads the free electrons in the surface
    shell.  omega0 defaults to 2 pi c / 400 nm on every axis."""
    d = (0.5e-9,) * 3
    dt = 0.5 * d[0] / (I.C_LIGHT * math.sqrt(3))
    mask = I.sphere_mask(n, 8.0)
    grid = dict(dims=3, n=n, d=d, dt=dt, bc=(1, 1, 1), pml_cells=4,
                src=dict(inc_axis=0, pol_axis=1, src_index=6, E0=3e9,
                         omega=2 * np.pi * I.C_LIGHT / 20e-9, tau=3e-17, t0=2e-17))
    w = 5.9e28 * d[0] ** 3 / 8
    cells = rng.choice(shell_cells(mask), size=nfree) if shell else None
    cell, off, v = I.random_particles(rng, n, nfree, mask=mask, vscale=vscale, cells=cells)
    cb, anc, disp, vb = I.random_bound(rng, n, nbound, mask=mask, dscale=2e-12, vscale=2e4)
    w0 = 2 * np.pi * I.C_LIGHT / 400e-9
    species = [
        dict(kind=I.FREE, q=-I.QE, m=I.ME, w=w, cell=cell, off=off, v=v, background=1),
        dict(kind=I.BOUND, q=-I.QE, m=I.ME, w=0.5 * w, cell=cb, anchor_off=anc, disp=disp, v=vb,
             omega0=tuple(omega0) if omega0 is not None else (w0, w0, w0), gamma=tuple(gamma),
             background=1),
    ]
    return grid, mask, species


def guarded_species(grid, mask, species, setup):
    """Drop the free particles that end the first oracle step within 1e-5
    cell of a face (FP32 and FP64 may cross differently there)."""
    s = oracle_sim(grid, mask, species)
    setup(s)
    s.step(1)
    Xo = s.species(0)[0]
    s.close()
    ok = ~near_face(Xo, grid["dims"], 1e-5)
    assert ok.mean() > 0.99
    keep = np.flatnonzero(ok)
    sp0 = dict(species[0], cell=species[0]["cell"][keep], off=species[0]["off"][keep],
               v=species[0]["v"][keep])
    return [sp0] + list(species[1:])


def compare_one_step(pic, h, s, grid, species):
    """One step on both sides: velocities (1e-5 relative) and positions
    (1e-5 cell) of species 0, velocities and displacements of the bound
    species 1 if any, reflection count, per-cell counts (exact) and fields
    (1e-5 relative L2).  Returns the oracle's reflection count."""
    n = grid["n"]
    pic.pic_step(h, 1)
    s.step(1)
    Xo, Vo, _, nro = s.species(0)
    rd = pic.pic_read_species(h, 0, species[0]["cell"].size)
    assert vel_rel(rd["v"], Vo, 1e5) < 1e-5
    dX = periodic_delta(gpu_positions(rd, n), Xo, n, grid["dims"])
    assert np.abs(dX).max() < 1e-5
    if len(species) > 1:
        Xb, Vb, Db, _ = s.species(1)
        rb = pic.pic_read_species(h, 1, species[1]["cell"].size, bound=True)
        assert vel_rel(rb["v"], Vb, 1e3) < 1e-5
        assert np.abs(rb["disp"] - Db).max() < 1e-5 * np.abs(Db).max()
    diag = pic.pic_diagnostics(h)
    assert diag["reflections"][0] == nro
    for k in range(len(species)):
        assert np.array_equal(pic.pic_cell_counts(h, k, I.grid_shape(n)), s.cell_counts(k))
    got = gpu_fields(h, grid)
    for c in range(6):
        ref = s.field(c)
        if np.linalg.norm(ref) > 0:
            assert rel_l2(got[c], ref) < 1e-5, c
    return nro
