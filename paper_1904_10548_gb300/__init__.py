"""GB300 (sm_103a) solver for scenario-based stochastic MPC of drinking-water
networks: the accelerated proximal gradient method on the Fenchel dual
(arXiv 1904.10548, §4), behind the C ABI of include/rapidnet.h.

All computation runs in ``librapidnet.so`` (hand-written CUDA); this
package only marshals arguments.  Build the library with
``__graft_entry__.build()`` (or ``python -m paper_1904_10548_gb300.build``).
"""
from ._binding import (  # noqa: F401
    Factor, RapidNetError, Server, load, rapidnet_dual_gradient_device, rapidnet_dual_gradient_noalloc, rapidnet_factor,
    rapidnet_factor_free, rapidnet_factor_info, rapidnet_last_error, rapidnet_solve,
    rapidnet_solve_device, rapidnet_solve_batch, solve_batch, scenario_tree, pernode_matrices,
    RN_PREC_FP64, RN_PREC_MIXED, RN_PREC_FP32, RN_OK, RN_NOT_CONVERGED, RN_ERR_UNSUPPORTED,
    RN_FACTOR_AUTO, RN_FACTOR_SHARED, RN_FACTOR_PER_NODE,
    STATUS_NAMES, EXPORTS, LIB_PATH,
)
