"""The reduced-basis preconditioner in the FP64 oracle (test infrastructure: imported only
by the tests).

Section 3.3 names a preconditioner built by the reduced basis method and a low-rank
approximation of the Jacobian, and leaves its construction to the paper's references.
The reading implemented by the library and written out plainly here: for a reduced
basis, the columns of V (n x k, any basis of the subspace), and the Jacobian J,
    C = V ((J V)^T J V)^{-1} (J V)^T,     P^{-1} r = C r + B^{-1} (r - J C r),
with B the block-Jacobi matrix (the exact element-diagonal blocks of J). C r is the
minimal-residual solve of J x = r over span(V) (J C is the orthogonal projector onto
span(J V)); it does not depend on which basis of the subspace V holds.
"""
from __future__ import annotations

import numpy as np


def block_jacobi_inverse(J, nloc):
    """B^{-1}: the inverses of the nloc x nloc diagonal blocks of the dense J."""
    n = J.shape[0]
    Binv = np.zeros_like(J)
    for s in range(0, n, nloc):
        Binv[s:s + nloc, s:s + nloc] = np.linalg.inv(J[s:s + nloc, s:s + nloc])
    return Binv


def rb_apply(J, Binv, V, r):
    """P^{-1} r for the reduced basis V (n x k; k = 0 gives block-Jacobi alone)."""
    if V is None or V.shape[1] == 0:
        return Binv @ r
    JV = J @ V
    c = V @ np.linalg.solve(JV.T @ JV, JV.T @ r)
    return c + Binv @ (r - J @ c)
