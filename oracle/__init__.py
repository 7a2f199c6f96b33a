"""CPU FP64 oracle for the compact finite-difference derivative path.

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by the
benchmark's CPU-baseline leg, never by the GPU product path.  It shares no code with
the CUDA library; see ``tds_oracle.c`` for what each function computes and which
passage of the paper it follows.
"""
from .oracle import (  # noqa: F401
    build, bands, rhs_lines, deriv_lines, deriv_adjoint_lines, tridiag_solve,
    lines_view, from_lines_view, to_layout, from_layout, deriv, deriv_adjoint,
    layout_lines_count, grid_spacing, transport_term_lines, transport_term,
    transport_rhs, filter_lines, filter_adjoint_lines, interp_lines, interp_adjoint_lines,
    apply_op, FILTER, INTERP,
)
