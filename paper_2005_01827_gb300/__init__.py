"""GB300-native batched LISA log-likelihood for massive-black-hole-binary templates.

The computation (Katz et al. 2020, Sec. II and II.A) lives in the CUDA library
``liblisalike.so`` behind the C ABI of ``include/lisa_like.h``; ``lisalike`` is its
ctypes binding.  Build with ``python -m paper_2005_01827_gb300.build``.
"""
from . import lisalike  # noqa: F401
from .lisalike import (LISA_PREC_FP64, LISA_PREC_SPLIT, MODES6, LisaError,  # noqa: F401
                       LisaLike, dl_from_z, psd_aet)

__all__ = ["lisalike", "LisaLike", "LisaError", "dl_from_z", "psd_aet", "MODES6",
           "LISA_PREC_FP64", "LISA_PREC_SPLIT"]
