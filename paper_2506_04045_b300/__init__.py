"""B300-native fuzzy clustering (arXiv 2506.04045): parallel FISTA / GPA for
min ||S - U U^T||_F^2 over row-stochastic U, as hand-written sm_103a kernels
behind the C ABI of include/cluster.h.  This package is the thin Python
binding of that library."""
from .binding import (  # noqa: F401
    CSR, Options, Report, Solver, Batch, Server, ClusterError, load, lib_path, last_error, default_options,
    objective, objective_static, hessian_apply, csr_from_edges, make_csr,
    OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, EMAXITER, ETIMEOUT, EAGAIN,
    FP32, MIXED_BF16, STEP_CONST, STEP_INV_L_FROB, STEP_INV_L_SPEC,
    STOP_LOSS, STOP_PG_REL, STOP_PG_ABS, STOP_NONE,
)
