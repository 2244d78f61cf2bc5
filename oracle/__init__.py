"""FP64 CPU oracle (test infrastructure only; see tgv_oracle's header)."""
from .tgv_oracle import *  # noqa: F401,F403
from .tgv_oracle import (Flow, RK_A, RK_B, DIAG_NAMES, d1, d2, shift, grid,  # noqa: F401
                         conserved, primitives, initial_condition, convective,
                         pressure_terms, viscous_terms, residual, rk_substep,
                         rk3_step, run, diagnostics, kinetic_energy, vorticity,
                         final_ke, grad_final_ke, rhs_vjp, rhs_jvp)
