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
