"""GB300-native DPar2: two-stage randomized-SVD compression of irregular
dense tensors and ALS on the compressed slices (arXiv 2203.12798).

The compute path is the CUDA library libdpar2.so (include/dpar2.h); this
package builds it (``build``) and binds it (``api``).
"""
from .build import LIB, build  # noqa: F401


def load():
    """Import the binding (raises if libdpar2.so has not been built)."""
    from . import api

    api.lib()
    return api
