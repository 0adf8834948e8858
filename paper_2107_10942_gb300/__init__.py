"""Q2X for GB300: multipole coefficients of layer potentials over simplices
(Gumerov, Kaneko & Duraiswami, arXiv 2107.10942) by the paper's O(1)-per-moment
recursions, in hand-written CUDA kernels for sm_103a behind a C ABI
(include/q2x.h).  This package is the thin Python binding over that ABI."""
from ._lib import Q2XError  # noqa: F401
from .q2x import (Plan, NORM_COEFF, NORM_MOMENT, FP64, FP32_MIXED, DENSITY_CONST,  # noqa: F401
                  DENSITY_LINEAR, n_coef)
