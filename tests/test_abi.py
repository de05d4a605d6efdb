"""The C-ABI library builds, loads and exports every entry point of include/cdi.h.

Host-only helpers (Eq. 17/24 condition, Eq. 25-28 time steps) are exercised
without a GPU; nothing here launches a kernel.
"""
import ctypes
import os
import re

import pytest

from paper_1803_01262_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "cdi.h")).read()
    return sorted(set(re.findall(r"CDI_API\s+(?:const\s+)?\w+\s*\*?\s*(cdi_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libcdi():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("cdi_create_grid", "cdi_set_velocity", "cdi_step", "cdi_mass_and_bounds",
              "cdi_step_adjoint", "cdi_check_condition", "cdi_max_dt"):
        assert s in syms


def test_library_exports_every_declared_symbol(libcdi):
    for s in declared_symbols():
        assert hasattr(libcdi, s), s


def test_binding_signatures_cover_header():
    from paper_1803_01262_gb300 import cdi
    assert set(declared_symbols()) <= set(cdi.SIGNATURES)


def test_check_condition_host():
    from paper_1803_01262_gb300 import cdi
    assert cdi.check_condition(1.0, 1.0, 0.1, 3)           # on the crossover line, A = 0.1
    assert cdi.check_condition(1.5, 0.5, 0.25, 2)          # Table 2 point 1
    assert not cdi.check_condition(0.9, 0.9, 0.1, 2)       # point 5 is below Eq. 17
    assert not cdi.check_condition(1.0, 1.0, 0.2, 3)       # A > 1/6
    assert cdi.check_condition(0.5, float("inf"), 0.1, 2)  # pure reinitialisation, eps = dx/2
    with pytest.raises(cdi.CDIError):
        cdi.check_condition(-1.0, 1.0, 0.1, 3)


def test_max_dt_host():
    from paper_1803_01262_gb300 import cdi
    dx, eps, g = 0.02, 0.02, 1.5
    e = dx * dx / (g * eps)
    assert cdi.max_dt(dx, eps, g, 3, cdi.CDI_EULER) == pytest.approx(e / 6)
    assert cdi.max_dt(dx, eps, g, 3, cdi.CDI_RK2) == pytest.approx(e / 6)
    assert cdi.max_dt(dx, eps, g, 2, cdi.CDI_RK3) == pytest.approx(2.51 * e / 8)
    assert cdi.max_dt(dx, eps, g, 2, cdi.CDI_RK4) == pytest.approx(2.79 * e / 8)  # Eq. 31


def test_product_does_not_import_oracle():
    """The CUDA path's sources never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1803_01262_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
