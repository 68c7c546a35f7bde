"""GB300-native (sm_103a) VDS hot path: Gaussian-kernel density and free-energy
gradient passes, explicit/implicit particle steps, stress, bandwidth selection
and the POD machinery, behind a C-ABI library (``include/vds.h``).

Importing this package does not load the CUDA library; ``from
paper_2603_12550_gb300 import vds`` (or ``load()``) does, and raises if the
compiled library is missing.
"""
__all__ = ["load"]


def load():
    from . import vds  # noqa: F401  (loads the shared library)
    return vds
