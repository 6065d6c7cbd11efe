"""GB300-native parametric interior-point NMPC (arXiv 2606.04725 hot path).

The compute path is the CUDA library libnmpc.so (include/nmpc.h); this
package only marshals arguments to it.
"""
from ._lib import (MODEL_DISTILLATION, MODEL_DISTILLATION_DAE, MODEL_PAPER_PLATE, MODEL_PLATE,  # noqa: F401
                   MODEL_TOY, ORDER_AUTO, KKT_HYKKT, KKT_LIFTED,
                   ORDER_NATURAL, ORDER_ND,
                   NmpcError, Solver, Structure, autotune, lib, options, unpack_duals)
from .build import build  # noqa: F401
