"""CPU oracle for IPT (test infrastructure; see ipt_oracle's header)."""
from .ipt_oracle import *  # noqa: F401,F403
from .ipt_oracle import (OK, MAXITER, DIVERGED, DEGENERATE_THETA, INVALID_ARG,  # noqa: F401
                         partition, unit_columns, inverse_gaps, ipt_map, residual,
                         initial_residual_norm, ipt_solve, ipt_solve_csr,
                         rs_corrections, chart_jacobian, acx_differences, acx_sigma,
                         acx_update, ipt_solve_acx, ipt_solve_acx_csr)
from . import damping  # noqa: F401,E402
from . import anderson  # noqa: F401,E402
