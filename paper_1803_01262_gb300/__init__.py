"""GB300 (sm_103a) implementation of the explicit conservative diffuse
interface (CDI) phase-field step of Mirjalili, Ivey & Mani (arXiv 1803.01262).

Submodules:
  build        -- nvcc build of the CUDA library (_lib/libcdi.so, C ABI in include/cdi.h)
  cdi          -- ctypes binding of the C ABI (Grid, Batch, check_condition, max_dt,
                  max_dt_mixed)
  inputs       -- seeded synthetic phase fields and divergence-free face velocities
  autograd     -- checkpointed differentiable rollouts and the sphere inverse problem
  phase        -- phase-diagram sweeps of the (eps/dx, gamma/|u|) plane as one batch
  state_io     -- on-disk state for resuming long runs, JSON-lines run records
  profile_step -- fixed-configuration runs for profiler captures

Attributes of ``cdi`` are re-exported lazily so that importing ``inputs``
does not load torch or the CUDA library.
"""

_LAZY = {"Grid", "CDIError", "check_condition", "max_dt", "max_dt_mixed", "lib"}


def __getattr__(name):
    if name in _LAZY:
        from . import cdi
        return getattr(cdi, name)
    raise AttributeError(name)
