"""GB300-native explicit OTM material-point update (arXiv 2206.08772, Algorithm 1).

The compute path is the CUDA library libotm.so (include/otm.h), built in-tree for sm_103a by
``paper_2206_08772_gb300.build.build()``. This package only marshals arguments.
"""
from . import _lib  # noqa: F401
from ._lib import OTMError, header_functions, load  # noqa: F401


def __getattr__(name):
    # torch-dependent parts are imported lazily so that the build step needs no GPU
    if name in ("OTM", "support_search", "lme", "return_map", "make_params", "material_struct"):
        from . import otm as _otm
        return getattr(_otm, name)
    raise AttributeError(name)
