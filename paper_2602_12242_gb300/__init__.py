"""GB300 (sm_103a) implementation of the per-stage hot path of the MagneX
micromagnetics method: H_eff, LLG right-hand side, RK4/Euler stepping with the
FFT demag convolution, behind the C ABI of include/mx.h.

The compute lives in ``_build/libmx.so`` (built by ``build.build()``); this
package only marshals arguments.  Importing it does not load the library;
the first call does, and fails loudly if the library is missing.
"""
from ._lib import (MX_EULER, MX_RK4, MX_TERM_ALL, MX_TERM_ANIS, MX_TERM_DEMAG, MX_TERM_DMI,  # noqa: F401
                   MX_TERM_EXCH, MX_TERM_ZEEMAN, MxError)

__all__ = ["Context", "MxError"]


def __getattr__(name):
    if name in ("Context", "to_dev4", "from_dev4"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
