"""The Fermi-Dirac relaxation study of Sec. 2: bulk electron plasma loaded
with FD momenta relaxes toward a Maxwell-Boltzmann tail in a collisionless
PIC run; the apparent temperature beta of the high-energy tail
(counts ~ exp(-E / beta)) grows as A sqrt(t), and A depends on the
particles per cell.

The runs go through the batch engine (all density / ppc cases advanced by
the same launches) and the kinetic-energy histogram of the library
(pic_energy_histogram); the fits are host-side analysis of those counts.

Tail reading: bins whose lower edge lies at or above E_F + 2 kT0 (kT0 the
loading temperature) with at least 5 counts, least squares of ln(count)
against the bin centre weighted by the counts (Poisson), beta = -1 / slope.
The growth law is fitted as beta(t) = A sqrt(t) over the samples t > 0.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I
from . import pic, runner

EV = I.QE


def tail_beta(counts, e_max, e_lo, min_count=5):
    """Apparent temperature (J) of the tail of a kinetic-energy histogram
    (nbins bins of width e_max / nbins plus an overflow entry): weighted
    least squares of ln(count) on the bin centres at or above e_lo.  Returns
    (beta, number of bins used); beta is nan with fewer than 3 bins."""
    c = np.asarray(counts, dtype=np.float64)[:-1]
    nb = c.size
    w = e_max / nb
    lo = np.arange(nb) * w
    sel = (lo >= e_lo) & (c >= min_count)
    if sel.sum() < 3:
        return float("nan"), int(sel.sum())
    x = lo[sel] + 0.5 * w
    y = np.log(c[sel])
    wt = c[sel]
    xm = np.sum(wt * x) / wt.sum()
    ym = np.sum(wt * y) / wt.sum()
    slope = np.sum(wt * (x - xm) * (y - ym)) / np.sum(wt * (x - xm) ** 2)
    return (-1.0 / slope if slope < 0 else float("inf")), int(sel.sum())


def sqrt_law(t, beta):
    """Least-squares A of beta = A sqrt(t) over t > 0, and the R^2 of the fit."""
    t = np.asarray(t, np.float64)
    b = np.asarray(beta, np.float64)
    sel = (t > 0) & np.isfinite(b)
    st = np.sqrt(t[sel])
    A = float(np.sum(st * b[sel]) / np.sum(st * st))
    res = b[sel] - A * st
    tot = b[sel] - b[sel].mean()
    r2 = 1.0 - float(np.sum(res ** 2) / max(np.sum(tot ** 2), 1e-300))
    return A, r2


def run(densities=(2e28, 4e28, 6e28), ppcs=(16, 32, 64, 128), t_end_fs=20.0, samples=20,
        T_eV=0.0375, nbins=3000, stream=0, use_graph=1, tile=(2, 2, 2), shape_order=1):
    """All density x ppc cases in one batch group, sampled `samples` times
    over t_end_fs.  Particle tile 2 x 2 x 2 cells: at 16-128 particles per
    cell the default 8 x 8 x 4 tile holds up to 32 k particles depositing
    into one shared current box (6x slower, measured).  shape_order 2: TSC
    for the electrons (the group then runs the TSC batch kernel).
    Returns a dict: per case beta(t) (eV), A (eV / sqrt(fs)), R^2, and the
    whole job's particle-steps / s."""
    wls = [I.bulk_cube(n, p, T_eV=T_eV) for n in densities for p in ppcs]
    dt = wls[0]["grid"]["dt"]
    nsteps = int(round(t_end_fs * 1e-15 / dt))
    chunk = max(1, nsteps // samples)
    hs, g = [], None
    try:
        for wl in wls:
            hs.append(runner.make_sim(wl, stream, dict(tile=tuple(tile)) if tile else None,
                                      shape_order))
        counts = [int(sum(pic.pic_diagnostics(h)["count"])) for h in hs]
        g = pic.pic_group_create(len(hs), 0, stream, use_graph)
        for h in hs:
            pic.pic_group_add(g, h, nsteps)
        EF = [wl["species"][0]["E_F"] for wl in wls]
        emax = [3.0 * e for e in EF]
        e_lo = [e + 2 * T_eV * EV for e in EF]
        t_fs = [0.0]
        beta = [[tail_beta(pic.pic_energy_histogram(h, 0, emax[k], nbins), emax[k], e_lo[k])[0]
                 for k, h in enumerate(hs)]]
        done = 0
        wall = 0.0
        while done < nsteps:
            n = min(chunk, nsteps - done)
            t0 = time.perf_counter()
            pic.pic_group_step(g, n)
            pic.pic_group_sync(g)
            wall += time.perf_counter() - t0
            done += n
            t_fs.append(done * dt * 1e15)
            beta.append([tail_beta(pic.pic_energy_histogram(h, 0, emax[k], nbins), emax[k],
                                   e_lo[k])[0] for k, h in enumerate(hs)])
        beta = np.array(beta) / EV
        cases = []
        for k, wl in enumerate(wls):
            A, r2 = sqrt_law(t_fs, beta[:, k])
            cases.append({"density": wl["species"][0]["density"], "ppc": wl["species"][0]["ppc"],
                          "particles": counts[k], "E_F_eV": EF[k] / EV,
                          "beta_eV": [round(float(b), 5) for b in beta[:, k]],
                          "A_eV_per_sqrt_fs": A, "r2": r2})
        return {"t_fs": [round(t, 4) for t in t_fs], "steps": nsteps, "dt": dt,
                "cases": cases, "wall_s": wall, "tile": list(tile) if tile else None,
                "shape": "TSC" if shape_order == 2 else "CIC",
                "particle_steps_per_s": sum(counts) * nsteps / wall}
    finally:
        if g is not None:
            pic.pic_group_destroy(g)
        for h in hs:
            pic.pic_destroy(h)
