"""KFAC for PINN losses on GB300 (sm_103a): Python binding of libkfacpinn.so.

The compute path lives entirely in the CUDA library behind the C-ABI of
include/kfac_pinn.h; this package only marshals arguments.  Importing the
package does not load the library; constructing KfacPinn does, and fails
loudly if it has not been built (paper_2405_15603_gb300.build.build()).
"""
from ._lib import KfacError, EXPORTS  # noqa: F401


def __getattr__(name):
    if name in ("KfacPinn", "make_config", "param_count"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
