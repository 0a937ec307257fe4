"""GB300 (sm_103a) implementation of the coupled LBM-PIBM-DEM time step of the
particulate immersed boundary method (Zhang et al., arXiv:1407.6704).

The step runs in ``libpibm.so`` (CUDA, built by ``build.build()``) behind the C
ABI of ``include/pibm.h``; ``Pibm`` is its Python binding and ``inputs`` holds
the seeded synthetic workloads.
"""
from ._lib import PibmError  # noqa: F401


def Pibm(*args, **kwargs):  # noqa: N802 - thin constructor alias, imports torch lazily
    from .pibm import Pibm as _P
    return _P(*args, **kwargs)
