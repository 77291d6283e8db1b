"""Host-side analysis of the relaxation study (Sec. 2): the tail fit and
the square-root growth law, checked on exact data."""
import math

import numpy as np

from paper_2501_07465_gb300 import relax


def test_tail_fit_recovers_an_exact_exponential():
    """Counts proportional to exp(-E / beta) over the bins (any prefactor)
    give beta back to roundoff; bins below e_lo and under 5 counts are
    left out."""
    nb, e_max = 400, 10.0
    centres = (np.arange(nb) + 0.5) * e_max / nb
    for beta in (0.3, 1.0, 2.5):
        c = np.append(1e9 * np.exp(-centres / beta), 0)
        c[:40] = 1e12  # a Fermi sea below e_lo must not matter
        got, used = relax.tail_beta(c, e_max, e_lo=1.0, min_count=0)
        assert abs(got / beta - 1) < 1e-9 and used == nb - 40
    c = np.zeros(nb + 1)
    assert math.isnan(relax.tail_beta(c, e_max, 1.0)[0])


def test_sqrt_law_on_exact_data():
    t = np.linspace(0, 20, 21)
    A, r2 = relax.sqrt_law(t, 0.37 * np.sqrt(t))
    assert abs(A - 0.37) < 1e-12 and abs(r2 - 1) < 1e-12
    A, r2 = relax.sqrt_law(t, 0.37 * np.sqrt(t) + 0.05 * np.cos(t))
    assert abs(A - 0.37) < 0.02 and r2 < 1


def test_workload_fermi_energy_agrees_with_the_oracle():
    """The bulk-cube workload's E_F (Sec. 2, exponent 2/3) equals the
    oracle's pinned Fermi energy for the study's three densities."""
    from oracle import oracle as O
    from paper_2501_07465_gb300 import inputs as I
    for n in (2e28, 4e28, 6e28):
        wl = I.bulk_cube(n, 32)
        assert abs(wl["species"][0]["E_F"] / O.fermi_energy(n, I.ME) - 1) < 1e-12
