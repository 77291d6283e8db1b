"""The collective check of the Dirac carriers (Sec. 5): a sheet of massless
carriers pushed with the averaged transverse mass m_d = p_F / (2 v_F) must
oscillate as a 2D plasmon of mass m_pl = 2 m_d = p_F / v_F per carrier.

The sheet lies in one node plane of a grid that is periodic on all three
axes, starts with a current ripple at wavenumber q (inputs.dirac_sheet_ring)
and rings; the in-plane E on the sheet, projected on the ripple, is fitted
by a single frequency and compared with the closed form

  w^2 = n_s e^2 kappa coth(kappa L_z / 2) g(q v_F / w) / (2 eps0 m_pl),

where kappa = sqrt(q^2 - w^2 / c^2) is the field's decay rate off the sheet
(retardation), coth(kappa L_z / 2) sums the sheet's periodic images along z,
and g(s) = 2 (1 / sqrt(1 - s^2) - 1) / s^2 = 1 + 3 s^2 / 4 + ... is the
kinetic correction of carriers that all move at v_F (collisionless
response of a ring of velocities).  For a free-standing sheet (L_z -> inf)
at small q v_F / w and w << c q it is w^2 = n_s e^2 q / (2 eps0 m_pl).
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs as I


def closed_form_omega(n_s, q, m_pl, L_z, v_F):
    """The plasmon frequency of the model above (rad/s), by fixed-point
    iteration."""
    w2 = n_s * I.QE ** 2 * q / (2 * I.EPS0 * m_pl)
    for _ in range(100):
        kap = math.sqrt(q * q - w2 / I.C_LIGHT ** 2)
        s2 = (q * v_F) ** 2 / w2
        g = 2.0 * (1.0 / math.sqrt(1.0 - s2) - 1.0) / s2 if s2 > 1e-12 else 1.0 + 0.75 * s2
        w2 = n_s * I.QE ** 2 * kap / math.tanh(kap * L_z / 2) * g / (2 * I.EPS0 * m_pl)
    return math.sqrt(w2)


def fit_frequency(t, y, w_guess, span=0.3, samples=6001):
    """Least-squares fit of y = a cos(w t) + b sin(w t) + c over w in
    [w_guess (1 - span), w_guess (1 + span)]."""
    t = np.asarray(t, np.float64)
    y = np.asarray(y, np.float64)
    best = None
    for w in np.linspace((1 - span) * w_guess, (1 + span) * w_guess, samples):
        A = np.stack([np.cos(w * t), np.sin(w * t), np.ones_like(t)], 1)
        coef, *_ = np.linalg.lstsq(A, y, rcond=None)
        r = float(np.sum((A @ coef - y) ** 2))
        if best is None or r < best[0]:
            best = (r, w)
    return best[1]


def sheet_case(mode, n_s=1e16, E_F_eV=0.2, v_F=1e6, nx=64, ny=2, nz=32, dx=10e-9, ppc_side=4):
    """Grid, species and closed-form frequency of a ringing sheet: the
    graphene parameters of the sheet workload (n_s, E_F, v_F) on a coarse
    periodic grid, mode wavelengths nx / mode cells along x."""
    dt = 0.5 * dx / (I.C_LIGHT * math.sqrt(3))
    p_F = E_F_eV * I.QE / v_F
    m_d = p_F / (2 * v_F)
    q = 2 * math.pi * mode / (nx * dx)
    k0 = nz // 2
    cell, off, v, ppc = I.dirac_sheet_ring(nx, ny, k0, q, dx, v_F, ppc_side)
    grid = dict(dims=3, n=(nx, ny, nz), d=(dx, dx, dx), dt=dt, bc=(0, 0, 0), pml_cells=0)
    species = [dict(kind=I.DIRAC, q=-I.QE, m=m_d, v_F=v_F, w=n_s * dx * dx / ppc, cell=cell,
                    off=off, v=v, background=1)]
    w = closed_form_omega(n_s, q, 2 * m_d, nz * dx, v_F)
    return dict(grid=grid, species=species, omega=w, q=q, k0=k0, mode=mode, n_s=n_s,
                m_pl=2 * m_d, v_F=v_F)


def ring_gpu(case, stream, periods=1.5, samples=300):
    """Run a sheet case on the GPU path and fit its frequency.  Returns
    (w_fit, w_closed, steps, seconds)."""
    import time

    from . import pic
    g = case["grid"]
    h = pic.pic_create(pic.make_grid(3, g["n"], g["d"], g["dt"], bc=g["bc"]), stream)
    try:
        pic.pic_set_tuning(h, tile=(8, g["n"][1], 4))
        sp = case["species"][0]
        pic.pic_load_species(h, pic.species_desc(sp["kind"], sp["q"], sp["m"], sp["w"],
                                                 v_F=sp["v_F"], background=1),
                             cell=sp["cell"], off=sp["off"], v=sp["v"])
        nx, ny, nz = g["n"]
        w = case["omega"]
        nsteps = int(periods * 2 * math.pi / (w * g["dt"]))
        every = max(1, nsteps // samples)
        xi = (np.arange(nx) + 0.5) * g["d"][0]
        proj = np.cos(case["q"] * xi)
        t, y = [], []
        t0 = time.perf_counter()
        for it in range(nsteps // every):
            pic.pic_step(h, every)
            Ex = pic.pic_read_fields(h, 1, (nz, ny, nx))[0]
            y.append(float(np.sum(Ex[case["k0"]].mean(axis=0) * proj)))
            t.append((it + 1) * every * g["dt"])
        secs = time.perf_counter() - t0
    finally:
        pic.pic_destroy(h)
    return fit_frequency(t, y, w), w, (nsteps // every) * every, secs
