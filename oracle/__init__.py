"""CPU oracle for the PDHG hot path (test infrastructure only; see ``oracle.pdhg``)."""
from .pdhg import (DEFAULTS, OracleLP, OracleResult, default_eta, default_omega,  # noqa: F401
                   finite_bound_norm, fixed_point_residual, halpern, kkt, p_fun, p_norm_sq,
                   pdhg_step, pid_omega, power_sigma_max, proj_negS, proj_S, proj_X,
                   restart_decision, solve)
