"""The C-ABI library loads on a machine without a GPU and exports every
function declared in include/pic.h; the Python binding declares exactly
those names (no compute calls here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_07465_gb300 import build, pic
    build.build()
    return pic.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pic_create", "pic_load_species", "pic_set_material_mask", "pic_step",
                     "pic_read_fields", "pic_diagnostics", "pic_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2501_07465_gb300 import pic
    out = subprocess.run(["nm", "-D", "--defined-only", pic.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for name in _declared():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_binding_covers_the_header_exactly(lib):
    from paper_2501_07465_gb300 import pic
    assert sorted(pic.SIGNATURES) == _declared()


def test_last_error_without_handle_is_a_string(lib):
    from paper_2501_07465_gb300 import pic
    assert isinstance(pic.pic_last_error(None), str)


def test_library_is_built_for_sm_103a(lib):
    from paper_2501_07465_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
