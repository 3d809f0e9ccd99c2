"""GB300-native (sm_103a) near-circulant splitting (NCS) for TV-CT and TV-PET.

Ryu, Ko, Won, "Splitting with Near-Circulant Linear Systems: Applications to
Total Variation CT and PET" (arXiv 1810.13100).  The compute path is the CUDA
library libncs.so (C ABI in include/ncs.h); this package is its thin Python
binding.  PyTorch supplies device memory and streams only.
"""
from .binding import (  # noqa: F401
    Plan,
    Batch,
    Cone,
    ConePlan,
    UNet,
    NCSError,
    load_library,
    status_string,
    LIB_PATH,
    NCS_OK,
    NCS_NOT_CONVERGED,
)


def build(force: bool = False) -> str:
    """Compile libncs.so in-tree for sm_103a and return its path."""
    from . import _build
    return _build.build(force=force)
