"""The OpenMP build of the oracle (used only to time it on all host cores)
computes what the serial build computes: same particles, same fields, up to
the order in which the deposit's FP64 contributions to J are summed."""
import numpy as np

from oracle import oracle as O
from paper_2501_07465_gb300 import inputs as I

from tests import pairs as PR


def test_openmp_build_matches_the_serial_build():
    rng = np.random.default_rng(77)
    grid, mask, species = PR.sphere_case(rng, n=(20, 18, 16), nfree=3000, nbound=1500)
    a = PR.oracle_sim(grid, mask, species)
    b = O.OracleSim(parallel=True, **PR.oracle_grid(grid))
    b.set_mask(mask)
    for sp in species:
        X, V, D = PR.species_arrays_for_oracle(sp, tuple(grid["n"]))
        b.add_species(sp["kind"], sp["q"], sp["m"], sp["w"], X, V, D=D,
                      omega0=sp.get("omega0", (0, 0, 0)), gamma=sp.get("gamma", (0, 0, 0)),
                      vF=sp.get("v_F", 0.0), bg=sp.get("background", 0))
    a.step(20)
    b.step(20)
    for c in range(6):
        fa, fb = a.field(c), b.field(c)
        assert np.linalg.norm(fa - fb) <= 1e-12 * max(np.linalg.norm(fa), 1e-300), c
    for k in range(len(species)):
        Xa, Va, Da, ra = a.species(k)
        Xb, Vb, Db, rb = b.species(k)
        assert np.abs(Xa - Xb).max() < 1e-12
        assert np.abs(Va - Vb).max() <= 1e-10 * np.abs(Va).max()
        assert ra == rb
    assert O.threads(parallel=True) >= 1
    assert O.threads(parallel=False) == 1
    a.close()
    b.close()
