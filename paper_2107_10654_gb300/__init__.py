"""GB300 (sm_103a) sketched Tucker core update by ridge leverage score sampling.

The CUDA library libtucker.so (include/tucker.h) implements the hot path of
Fahrbach, Ghadiri and Fu's ALS-RS: per-factor leverage scores, product-
distribution sampling of Kronecker rows, dedupe, gather, the fused Kronecker
Gram/right-hand side and the FP64 ridge solve, beside the exact core update,
ALS sweeps and the adjoint.  This package is its thin Python binding.
"""
from .tucker import (TuckerError, Handle, Samples, CooTensor, tucker_leverage_scores,  # noqa: F401
                     tucker_sample_rows, tucker_core_update_sketched, tucker_core_update_exact,
                     tucker_als_sweep, tucker_ridge_loss, tucker_core_solve_adjoint,
                     tucker_sample_rows_noalloc, tucker_sketched_gram, tucker_set_solver)
from .autograd import SketchedCoreSolve  # noqa: F401
from ._lib import load as load_library, LIB_PATH  # noqa: F401
