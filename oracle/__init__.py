"""CPU oracle for the spectral D-bar CGO solve -- test infrastructure only.

Imported by tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg;
never by the product path.
"""
from .dbar_oracle import (CGOProblem, Grid, W, W_closed, W_series, dbar_inverse,  # noqa: F401
                          dft2, dft_last_axis, gmres, h_of_S, solve_cgo, taylor_coeffs)
