"""Tolerance of a GPU preconditioner apply against the oracle's, when the two sides' blocks
differ (test helper; no arithmetic of the method).

The GPU assembles the per-voxel blocks B_n from its sufficient statistics, the oracle from
Y and X directly; the parity tests bound their difference per entry (1e-12 of the largest W
block; for the A system, whose blocks are differences of lagged y'y products that cancel,
1e-12 of the largest lambda-weighted y'y sum). To first order y = M^-1 x then moves by at
most ||M^-1|| ||dM|| ||y||. Every preconditioner here satisfies M >= blockdiag(B_n): the
block-Jacobi blocks are B_n + diag(scale) deg_n; symmetric SOR with 0 < omega < 2 and the
symmetric V-cycle satisfy M >= B~ >= blockdiag(B_n), because the prior part of B~ is
positive semidefinite. So ||M^-1|| <= 1 / min_n lambda_min(B_n), and a block perturbation
of at most e per entry has spectral norm at most D e; the factor 10 covers the constants of
dM in dB (M is a product of block factors for SOR and the V-cycle), and 1e-12 the rounding
of the two evaluation orders.
"""
import numpy as np


def apply_tolerance(blocks, entry_err):
    """Relative-L2 tolerance for y = M^-1 x given the oracle's blocks (N, D, D) and the bound
    on the GPU blocks' per-entry error."""
    D = blocks.shape[1]
    lam_min = np.linalg.eigvalsh(blocks).min()
    return 1e-12 + 10.0 * D * entry_err / lam_min
