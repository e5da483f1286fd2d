"""GB300-native KKT factor/solve and interior-point method for arrowhead LPs.

The compute path is the in-tree CUDA library ``libahlp.so`` (C ABI in
include/ahlp.h); this package is its thin Python binding.  Importing it
without the built library raises ImportError -- there is no CPU fallback.
"""
from ._lib import (  # noqa: F401
    AHLPError,
    Options,
    PREC_FP64,
    PREC_MIXED,
    Problem,
    STATUS,
    arrowhead_lp_create,
    autotune,
    batch_layout,
    default_options,
    ipm_solve,
    kkt_adjoint_solve,
    kkt_factor,
    kkt_factor_kernel_times,
    kkt_schur_dense,
    kkt_solve,
    kkt_stage_times,
    kkt_update_jobs,
    tile_sparse_jobs,
    launch_count,
    transfer_bytes,
    lib_path,
    load,
    recover,
    set_cb,
    set_options,
)

load()
