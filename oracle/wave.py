"""The wave model of Section 2.1 in the FP64 oracle (test infrastructure: imported only
by the tests).

The wave model replaces Eq. 1a, q + grad u = 0, by dq/dt + grad u = 0, keeps Eq. 1b,
m du/dt + div f = s, and couples the ODE of Eq. 2, alpha dw/dt + beta w = s_w, to
recover the displacement. With f = kappa q (kappa = c^2), s = 0 and s_w = u this is the
scalar wave equation w_tt = c^2 lap w, u = w_t, q = -grad w.

The LDG semi-discretisation of Eq. 1a's left side is the oracle's own q-stage map
Q(u), the LDG form of -grad u, so the semi-discrete system is
    M du/dt = -R_s(u, q),    dq/dt = Q(u),    alpha dw/dt + beta w = u,
with R_s the oracle's residual of Eq. 1b at given q (no time term, no source). Here it
is written out plainly: the operator L of d/dt (u, q) = L (u, q) is assembled column by
column from those maps, and a DIRK step (Section 2.2) solves each stage of the coupled
system with a dense factorisation. No elimination of q is used.
"""
from __future__ import annotations

import numpy as np

from . import dirk_tableau


def wave_operator(o):
    """Dense L with d/dt (u, q) = L (u, q) for the oracle `o` (a Poisson oracle of case
    zero: kappa = c^2, tau the jump penalty), and the mass matrix M."""
    n = o.ndof
    nq = o.mesh.n_elem * o.ncu * o.nd * o.npe
    M = np.empty((n, n))
    Au = np.empty((n, n))
    Aq = np.empty((n, nq))
    Qm = np.empty((nq, n))
    zq = np.zeros(nq)
    zu = np.zeros(n)
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = o.mass(e)
        Au[:, k] = o.residual_with_q(e, zq)
        Qm[:, k] = o.q(e)
    for k in range(nq):
        e = np.zeros(nq)
        e[k] = 1.0
        Aq[:, k] = o.residual_with_q(zu, e)
    Minv = np.linalg.inv(M)
    L = np.block([[-Minv @ Au, -Minv @ Aq], [Qm, np.zeros((nq, nq))]])
    return L, M


def wave_step(L, n, u, q, w, dt, scheme, alpha=1.0, beta=0.0, solve=None):
    """One DIRK step of d/dt y = L y, y = (u, q), with w from alpha dw/dt + beta w = u:
    stage i solves (I - dt a_ii L) Y_i = y + dt sum_{j<i} a_ij K_j, K_i = L Y_i, and
    alpha Kw_i + beta (w + dt sum_{j<=i} a_ij Kw_j) = U_i; then y + dt sum_i b_i K_i.
    `solve(a, rhs)`, if given, solves (I - a L) Y = rhs (a factorisation kept by the
    caller); otherwise a dense solve per stage."""
    A, b, c = dirk_tableau(scheme)
    s = len(b)
    y = np.concatenate([u, q])
    I = np.eye(len(y))
    K, Kw = [], []
    for i in range(s):
        rhs = y + dt * sum(A[i][j] * K[j] for j in range(i))
        a = dt * A[i][i]
        Y = solve(a, rhs) if solve is not None else np.linalg.solve(I - a * L, rhs)
        K.append(L @ Y)
        if w is not None:
            wh = w + dt * sum(A[i][j] * Kw[j] for j in range(i))
            Kw.append((Y[:n] - beta * wh) / (alpha + beta * dt * A[i][i]))
    y1 = y + dt * sum(b[i] * K[i] for i in range(s))
    w1 = None if w is None else w + dt * sum(b[i] * Kw[i] for i in range(s))
    return y1[:n], y1[n:], w1


def quad_node_coords(o):
    """Physical coordinates [E][n_pe][2] of the nodes of an oracle on quadrilaterals
    (bilinear map of the element's vertices, in the lexicographic vertex order)."""
    nodes = o.ref_rules()[0][:, :2]
    s, t = (nodes[:, 0] + 1.0) / 2.0, (nodes[:, 1] + 1.0) / 2.0
    N = np.stack([(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t], axis=1)     # [npe][4]
    return np.einsum("pv,evd->epd", N, o.mesh.xyz)
