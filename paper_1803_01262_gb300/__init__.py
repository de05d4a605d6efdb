"""GB300 (sm_103a) implementation of the explicit conservative diffuse
interface (CDI) phase-field step of Mirjalili, Ivey & Mani (arXiv 1803.01262).

Submodules:
  build   -- nvcc build of the CUDA library (_lib/libcdi.so, C ABI in include/cdi.h)
  cdi     -- ctypes binding of the C ABI (Grid, check_condition, max_dt)
  inputs  -- seeded synthetic phase fields and divergence-free face velocities

Attributes of ``cdi`` are re-exported lazily so that importing ``inputs``
does not load torch or the CUDA library.
"""

_LAZY = {"Grid", "CDIError", "check_condition", "max_dt", "lib"}


def __getattr__(name):
    if name in _LAZY:
        from . import cdi
        return getattr(cdi, name)
    raise AttributeError(name)
