"""Building simulations from workload descriptions (the dictionaries of
`inputs`): one pic_create, the material mask, then each species through the
library's Fermi-Dirac loader.  Used by the autotuner, the serving loop and
the benchmark; all work runs in the CUDA library."""
from __future__ import annotations

import numpy as np

from . import pic


def grid_desc(wl):
    g = wl["grid"]
    return pic.make_grid(g["dims"], g["n"], g["d"], g["dt"], bc=g.get("bc", (0, 0, 0)),
                         pml_cells=g.get("pml_cells", 0), src=g.get("src"))


def make_sim(wl, stream=0, tuning=None, shape_order=1):
    """A loaded simulation handle for workload `wl` on CUDA stream `stream`
    (free and Dirac particles with CIC, or TSC for shape_order 2)."""
    h = pic.pic_create(grid_desc(wl), stream)
    try:
        if tuning:
            pic.pic_set_tuning(h, **tuning)
        if shape_order != 1:
            pic.pic_set_shape_order(h, shape_order)
        if wl.get("mask") is not None:
            pic.pic_set_material_mask(h, wl["mask"])
        for sp in wl["species"]:
            desc = pic.species_desc(sp["kind"], sp["q"], sp["m"], 0.0,
                                    omega0=sp.get("omega0", (0, 0, 0)),
                                    gamma=sp.get("gamma", (0, 0, 0)), v_F=sp.get("v_F", 0.0),
                                    background=sp.get("background", 0))
            pic.pic_load_species(h, desc, density=sp["density"], E_F=sp["E_F"], T=sp["T"],
                                 ppc=sp["ppc"], quiet=sp["quiet"], seed=sp["seed"],
                                 stream=sp["stream"])
    except Exception:
        pic.pic_destroy(h)
        raise
    return h


def cells(wl):
    return int(np.prod(wl["grid"]["n"]))


def material_cells(wl):
    return cells(wl) if wl.get("mask") is None else int(np.count_nonzero(wl["mask"]))


def particles(wl):
    """Macro-particles the loader places (ppc per material cell per species)."""
    return sum(sp["ppc"] * material_cells(wl) for sp in wl["species"])


def estimate_bytes(wl):
    """Device bytes a simulation of `wl` will hold (an upper estimate used
    for admission before the handle exists): ping-pong E and B, J, the
    material mask, CPML coefficients and memory terms, and per particle the
    double-buffered SoA state (cell, id, offsets, velocities; bound: FP64 and
    FP32 anchors and displacements) and its slot in the deferred-particle
    list, plus 16 MB of fixed tables."""
    g = wl["grid"]
    nc = cells(wl)
    per_cell = 4 * (12 + 3) + 1 + 8 * 2
    pml = g.get("pml_cells", 0)
    slab = 0
    if pml:
        n = g["n"]
        for a in range(g["dims"]):
            if g.get("bc", (0, 0, 0))[a] == 1:
                slab += 2 * pml * nc // n[a]
    b = nc * per_cell + slab * 4 * 8
    for sp in wl["species"]:
        np_ = sp["ppc"] * material_cells(wl)
        b += np_ * (2 * (4 + 4 + 24) + (2 * (24 + 12 + 12) if sp["kind"] == 1 else 0) + 8 + 8)
    return int(b + (16 << 20))
