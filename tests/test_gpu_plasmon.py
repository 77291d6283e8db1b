"""The Dirac carriers' collective check on the GPU path (Sec. 5): a sheet
of massless carriers pushed with m_d = p_F / (2 v_F) rings at the 2D plasmon
frequency of mass p_F / v_F, at two wavenumbers, and follows the oracle step
by step on the same seeded sheet."""
import math

import numpy as np
import pytest

from paper_2501_07465_gb300 import inputs as I

from tests import pairs as PR
from tests.test_oracle_pins import sheet_plasmon_closed_form

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


@pytest.mark.parametrize("mode", [1, 2])
def test_sheet_plasmon_frequency_on_gpu(mode):
    """The sheet of the oracle pin (n_s = 4e17 m^-2, E_F = 0.2 eV, v_F = 1e6,
    10 nm cells, 64 x 2 x 32 periodic): fitted frequency within 1 % of the
    closed form; |v| = v_F and v_z = 0 throughout."""
    import torch

    from paper_2501_07465_gb300 import pic, plasmon
    case = plasmon.sheet_case(mode, n_s=4e17)
    g = case["grid"]
    w_test = sheet_plasmon_closed_form(case["n_s"], case["q"], case["m_pl"], g["n"][2] * g["d"][2],
                                       case["v_F"])
    assert abs(case["omega"] / w_test - 1) < 1e-12
    wfit, w, steps, _ = plasmon.ring_gpu(case, torch.cuda.current_stream().cuda_stream)
    assert abs(wfit / w_test - 1) < 0.01, (mode, wfit, w_test, steps)


def test_sheet_plasmon_follows_the_oracle():
    """The same sheet (mode 1) on both paths: velocities within 1e-5 after
    one step, fields within 1e-3 relative L2 after one step and after 200,
    |v| = v_F to 2 ulp and v_z = 0 on the GPU.

    The field bound is wider than the workloads' 1e-5 because of what this
    input asks of FP32: a carrier moves v_F dt / dx = 9.6e-4 cells per step,
    which FP32 offsets near 0.5 resolve only to ulp / move = 6e-5, and the
    quiet ring start cancels all but the drift share (~5 %) of each cell's
    current, so J -- the only source of E here -- carries a relative error of
    a few 1e-4 (measured 1.0e-4 after one step)."""
    from paper_2501_07465_gb300 import pic, plasmon
    case = plasmon.sheet_case(1, n_s=4e17)
    grid, species = case["grid"], case["species"]
    s = PR.oracle_sim(grid, None, species)
    h = PR.gpu_sim(grid, None, species, tuning=dict(tile=(8, grid["n"][1], 4)))
    n = species[0]["cell"].size
    try:
        pic.pic_step(h, 1)
        s.step(1)
        rd = pic.pic_read_species(h, 0, n)
        _, Vo, _, _ = s.species(0)
        assert np.max(np.linalg.norm(rd["v"] - Vo, axis=1)) / 1e6 < 1e-5
        # the mode carries E_x, E_z and B_y; E_y, B_x and B_z hold only
        # rounding noise (1e-6 of the mode's fields in FP64), so they are
        # checked against the mode's scale instead of each other
        got = PR.gpu_fields(h, grid)
        assert PR.rel_l2(got[0], s.field(0)) < 1e-3
        pic.pic_step(h, 199)
        s.step(199)
        got = PR.gpu_fields(h, grid)
        for c in (0, 2, 4):
            assert PR.rel_l2(got[c], s.field(c)) < 1e-3, c
        for c, scale in ((1, got[0]), (3, got[4]), (5, got[4])):
            assert np.linalg.norm(got[c]) < 1e-3 * np.linalg.norm(scale), c
        rd = pic.pic_read_species(h, 0, n)
        sp = np.linalg.norm(rd["v"].astype(np.float64), axis=1)
        assert np.abs(sp / 1e6 - 1).max() <= 2 * 2.0 ** -23
        assert np.all(rd["v"][:, 2] == 0)
        assert np.all(rd["off"][:, 2] == 0)
    finally:
        pic.pic_destroy(h)
        s.close()
