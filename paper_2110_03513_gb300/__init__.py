"""GB300 (sm_103a) componentwise boosting: Python binding of the C ABI in include/cwb.h.

The functions named ``cwb_*`` mirror the C entry points one to one (argument
marshalling only); :class:`Model` is a small convenience wrapper built on
them.  Every step of the method runs in the CUDA library; importing this
package fails loudly if ``libcwb.so`` has not been built.
"""
from .binding import (  # noqa: F401
    BINS_EXACT, BINS_SQRT, BL_CATEGORICAL, BL_CATEGORICAL_BINARY, BL_LINEAR, BL_PSPLINE, LOSS_BINOMIAL, LOSS_L2, OPT_ACWB, OPT_CWB, OPT_HCWB,
    Batch, CwbError, Model, Server, cwb_create, cwb_fit, cwb_force_selection, cwb_free, cwb_get_bin_index, cwb_get_coefficients,
    cwb_get_criteria, cwb_get_fitted, cwb_get_learner_info, cwb_get_learner_matrices, cwb_get_trace,
    cwb_get_profile, cwb_get_residuals, cwb_get_scatter_plan, cwb_last_error, cwb_predict, cwb_predict_noalloc, cwb_profile, cwb_synchronize, learner, library_path, load_library,
    cwb_create_many, cwb_shard_create, cwb_shard_finish, cwb_shard_rows, cwb_shard_scatter, cwb_shard_sizes, cwb_shard_solve, cwb_shard_stats,
)
from .sharded import ShardedFit, split_rows, torch_allreduce, torch_allreduce_tensor  # noqa: F401
