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


def test_max_dt_mixed_host():
    """Below-line step: min(diffusive limit, c dx / (sum of component maxima + D_f gamma)),
    c = 2.83 for RK4 (Eq. 32, so min(Eq. 31, Eq. 32) in 2D), c = 1 for Euler."""
    from paper_1803_01262_gb300 import cdi
    dx = 2.0 / 50
    c = 2.0 ** 0.5 / 2
    for eoh, gu in ((1.5, 0.5), (1.0, 1.0), (0.7, 0.7), (0.55, 0.3), (2.0, 3.0)):
        eps, g = eoh * dx, gu
        eq31 = 2.79 * dx * dx / (8 * g * eps)
        eq32 = 2.83 * dx / (c + c + 2 * g)
        assert cdi.max_dt_mixed(dx, eps, g, (c, c), cdi.CDI_RK4) == pytest.approx(min(eq31, eq32), rel=1e-15)
        eul = min(dx * dx / (4 * g * eps), dx / (c + c + 2 * g))
        assert cdi.max_dt_mixed(dx, eps, g, (c, c), cdi.CDI_EULER) == pytest.approx(eul, rel=1e-15)
    # far below the line (eps/dx 0.55, gamma/u 0.3) the advective limit of Eq. 32 binds;
    # at Table 2's point 7 (0.7, 0.7) Eq. 32 as printed exceeds Eq. 31, which then binds;
    # above the line (point 1: 1.5, 0.5) Eq. 31 binds
    assert cdi.max_dt_mixed(dx, 0.55 * dx, 0.3, (c, c), cdi.CDI_RK4) == pytest.approx(
        2.83 * dx / (2 * c + 0.6), rel=1e-15)
    assert cdi.max_dt_mixed(dx, 0.7 * dx, 0.7, (c, c), cdi.CDI_RK4) == pytest.approx(
        2.79 * dx * dx / (8 * 0.7 * 0.7 * dx), rel=1e-15)
    assert cdi.max_dt_mixed(dx, 1.5 * dx, 0.5, (c, c), cdi.CDI_RK4) == pytest.approx(
        2.79 * dx * dx / (8 * 0.5 * 1.5 * dx), rel=1e-15)
    # 1D: Eq. 10 at the crossover line, dx / (u + gamma)
    assert cdi.max_dt_mixed(0.01, 0.01, 1.0, (1.0,), cdi.CDI_EULER) == pytest.approx(
        min(0.01 * 0.01 / (2 * 0.01), 0.01 / 2.0))
    for bad in (cdi.CDI_RK2, cdi.CDI_RK3):
        with pytest.raises(cdi.CDIError):
            cdi.max_dt_mixed(dx, dx, 1.0, (c, c), bad)
    with pytest.raises(cdi.CDIError):
        cdi.max_dt_mixed(dx, dx, 1.0, (-1.0, c), cdi.CDI_EULER)
