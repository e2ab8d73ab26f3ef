"""GB300-native (sm_103a) even-odd Wilson-Dirac operator for SU(2) gauge links.

The hot path of arXiv:2411.18511 ("Scaling SU(2) to 1000 GPUs using HiRep"):
the hopping operator D_eo / D_oe for fundamental and adjoint fermions, the
even-odd Schur operator and CG solves on it, behind the C ABI of
``libhirep_gb300.so`` (``include/hirep_gb300.h``).  ``hr`` is the ctypes
binding; ``fields`` holds device-buffer helpers; ``autograd`` wraps the
operator and the solve as ``torch.autograd.Function``.
"""

from . import hr  # noqa: F401
from .hr import HrError, Context  # noqa: F401


def build(force: bool = False) -> str:
    """Compile libhirep_gb300.so for sm_103a (in-tree) and return its path."""
    from . import _build
    return _build.build(force=force)
