"""GB300 (sm_103a) contour-integral solver for split-form nonlinear eigenvalue problems.

The numerical work lives in the CUDA library libnepciss.so (C ABI in include/nep_ciss.h);
``binding`` marshals arguments to it. Build with ``paper_1910_11712_gb300.build.build()``.
"""
from . import binding  # noqa: F401
from .binding import Plan, Split, ciss_solve  # noqa: F401
