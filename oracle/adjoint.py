"""Adjoint sensitivities for the oracle (test infrastructure only; see package header).

The paper has no adjoint; this is implicit differentiation of the converged
discrete solution, written from its definition. With A psi = b the LD / S_N
system of Eq. trop (A = L_h - S_h, b the mass-weighted source) and a scalar
objective J(psi):

    A^T lambda = dJ/dpsi,         dJ/dp = -lambda^T (dA/dp) psi.

Per cell i, with m_i = (h_i/6)[[2,1],[1,2]] acting on the two LD nodes:
    dA/dsigma_t,i    =  m_i (x) I_N
    dA/dsigma_s,l,i  = -m_i (x) M[:, l] D[l, :]        (S = M diag(sigma_s) D)
so
    dJ/dsigma_t,i   = -sum_{a,b} m_ab sum_n lambda_{i,a,n} psi_{i,b,n}
    dJ/dsigma_s,l,i = +sum_{a,b} m_ab (sum_n M[n,l] lambda_{i,a,n}) phi_{l,i,b}.

Objectives: the right-boundary exit current J = sum_{mu_n>0} w_n mu_n psi_{K,R,n}
(default), or a linear functional J = <g, phi> of the flux moments (the
vector-Jacobian product used by automatic differentiation).
The transposed system is solved with a sparse LU of A^T itself, so nothing here
relies on the structure of A^T that the GPU path uses.
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import iterations as it
from . import transport as tr


def exit_current_right(prob, psi):
    """J = sum over mu_n > 0 of w_n mu_n psi at the right node of the last cell."""
    mu, w, _, _ = it.tables(prob["N"], prob["L"])
    return tr.exit_currents(mu, w, psi)[1]


def dJ_dpsi(prob, g_phi=None):
    """Gradient of the objective with respect to psi, shape (K, 2, N)."""
    N, L = prob["N"], prob["L"]
    mu, w, D, _ = it.tables(N, L)
    K = prob["h"].size
    s = np.zeros((K, 2, N))
    if g_phi is None:
        pos = mu > 0
        s[-1, 1, pos] = w[pos] * mu[pos]
    else:
        s = np.einsum("ln,kal->kan", D, g_phi)          # d<g, D psi>/dpsi = D^T g
    return s


def gradients(prob, g_phi=None):
    """(J, dJ/dsigma_t [K], dJ/dsigma_s [K, L+1], psi, lambda) at the discrete solution.

    Forward: the direct solve of A psi = b. Adjoint: sparse LU of A^T.
    J is the exit current (g_phi None) or <g_phi, phi>.
    """
    N, L = prob["N"], prob["L"]
    mu, w, D, M = it.tables(N, L)
    K = prob["h"].size
    A = it.transport_matrix(prob, mu, w)
    phi, psi = it.direct_solve(prob, return_psi=True)
    s = dJ_dpsi(prob, g_phi)
    lam = spla.splu(A.T.tocsc()).solve(s.ravel()).reshape(K, 2, N)
    J = exit_current_right(prob, psi) if g_phi is None else float(np.sum(g_phi * phi))
    m = np.array([[2.0, 1.0], [1.0, 2.0]])
    h6 = prob["h"] / 6.0
    lam_psi = np.einsum("kan,kbn->kab", lam, psi)                     # sum_n lambda_a psi_b
    d_st = -h6 * np.einsum("ab,kab->k", m, lam_psi)
    lam_t = np.einsum("nl,kan->kal", M, lam)                          # sum_n M[n,l] lambda_n
    d_ss = h6[:, None] * np.einsum("ab,kal,kbl->kl", m, lam_t, phi)
    return J, d_st, d_ss, psi, lam
