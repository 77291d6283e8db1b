"""Helpers for parity tests: run the same seeded inputs through the CUDA
path (via the C ABI binding) and through the FP64 oracle."""
from __future__ import annotations

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
