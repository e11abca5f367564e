"""Iterative solvers for the oracle (test infrastructure only; see package header).

A slab problem is a dict with
  N, L            quadrature order (even) and scattering order (L <= N-1)
  h[K]            cell widths
  sigma_t[K]      total cross section per cell
  sigma_s[K,L+1]  Legendre moments sigma_{s,l} per cell (Eq. treq)
  Q[K,2,L+1]      external source as Legendre moments at the two LD nodes; the
                  angular source is q_n = sum_l (2l+1)/2 P_l(mu_n) Q_l, so an
                  isotropic scalar source of strength S has Q_0 = S (q_n = S/2)
  bc              'vacuum' (default), 'reflective', or a (left, right) pair of them
  psi_inc         optional (2, N) incoming angular flux at the vacuum edges (row 0:
                  left edge, read for mu > 0; row 1: right edge, read for mu < 0);
                  absent = no incoming flux (Eq. trans-equation-bc)
The state of every iteration is the flux moments phi[K,2,L+1] at the LD nodes.

Convergence test (Eq. iterate): the paper iterates while
||phi_l^{m+1} - phi_l^m||_inf exceeds a tolerance without saying relative or
absolute or which l; the reading used here is the relative change of the scalar
flux, max|phi_0^{m+1} - phi_0^m| / max|phi_0^{m+1}| < tol.
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import quadrature as qd
from . import transport as tr


def tables(N, L):
    """mu, w, D (L+1 x N), M (N x L+1) for an S_N set and scattering order L (Eqs. phi-mom, treq)."""
    mu, w = qd.gauss_legendre(N)
    return mu, w, qd.moment_operator(mu, w, L), qd.expansion_operator(mu, L)


def moments(D, psi):
    """phi[K,2,l] = sum_n D[l,n] psi[K,2,n] (Eq. phi-mom)."""
    return np.einsum("ln,kan->kal", D, psi)


def scattering_source(M, sigma_s, phi, Q=None):
    """Nodal angular source q_n = sum_l M[n,l] (sigma_{s,l} phi_l + Q_l) (Eq. treq, S psi + q)."""
    src = sigma_s[:, None, :] * phi
    if Q is not None:
        src = src + Q
    return np.einsum("nl,kal->kan", M, src)


def _streaming_inverse(prob, mu):
    """Return a function (q, incident) -> L_h^{-1} q (Eq. trsi left-hand side) with
    the problem's incoming boundary fluxes when incident is True (the source
    sweeps) and none when False (sweeps of an error or Krylov vector).

    Both edges vacuum: the upwind sweep. A reflective edge: a sparse LU of the
    global streaming matrix (the sweep would need lagged boundary values there).
    """
    h, st = prob["h"], prob["sigma_t"]
    bc = tr.bc_sides(prob.get("bc", "vacuum"))
    inc = prob.get("psi_inc")
    K, N = h.size, mu.size
    if bc == ("vacuum", "vacuum"):
        def sweep(q, incident=False):
            if incident and inc is not None:
                return tr.sweep(mu, st, h, q, psi_in_left=inc[0], psi_in_right=inc[1])
            return tr.sweep(mu, st, h, q)
        return sweep
    Kc = st[:, None, None] * np.eye(N)[None]
    lu = spla.splu(tr.assemble(mu, h, Kc, bc=bc))
    src = tr.incident_source(mu, K, inc, bc)

    def solve(q, incident=False):
        rhs = tr.mass_weight(h, q) + (src if incident else 0.0)
        return lu.solve(rhs.ravel()).reshape(K, 2, N)
    return solve


def fp_matrix(prob, mu, w, laplacian="mpd"):
    """Sparse LD form of the FP operator F = mu d/dz + sigma_a - sigma_tr/2 A_FP (Eqs. fpop,
    fp-mpd-oper, wd-eq-oper), with sigma_a = sigma_t - sigma_{s,0} and
    sigma_tr = sigma_{s,0} - sigma_{s,1} (Sec. 2), same BCs as the transport problem
    applied homogeneously to the correction."""
    N = mu.size
    A_fp = qd.angular_laplacian(mu, w, laplacian)
    sa = prob["sigma_t"] - prob["sigma_s"][:, 0]
    s1 = prob["sigma_s"][:, 1] if prob["sigma_s"].shape[1] > 1 else np.zeros_like(sa)
    str_ = prob["sigma_s"][:, 0] - s1
    Kc = sa[:, None, None] * np.eye(N)[None] - 0.5 * str_[:, None, None] * A_fp[None]
    return tr.assemble(mu, prob["h"], Kc, bc=prob.get("bc", "vacuum"))


def transport_matrix(prob, mu, w):
    """Sparse LD form of L - S (Eq. trop) with S = M diag(sigma_s) D per cell."""
    N, L = prob["N"], prob["L"]
    _, _, D, M = tables(N, L)
    Kc = prob["sigma_t"][:, None, None] * np.eye(N)[None] \
        - np.einsum("nl,kl,lm->knm", M, prob["sigma_s"], D)
    return tr.assemble(mu, prob["h"], Kc, bc=prob.get("bc", "vacuum"))


def rel_change(phi_new, phi_old):
    """Relative change of the scalar flux (reading of Eq. iterate, module docstring)."""
    return np.max(np.abs(phi_new[..., 0] - phi_old[..., 0])) / np.max(np.abs(phi_new[..., 0]))


def source_iteration(prob, tol=1e-10, max_it=100000, phi0=None, history=False):
    """Source iteration L psi^{m+1} = S psi^m + q (Eq. trsi), on moments.

    Returns (phi, iterations, list of relative changes).
    Pinned by: the infinite-medium closed form phi_0^m = (S/sigma_t) sum_{k<m} c^k and
    the spectral-radius bound max_l sigma_{s,l}/sigma_t (Sec. 2.1; P4, P11).
    """
    N, L = prob["N"], prob["L"]
    mu, w, D, M = tables(N, L)
    Linv = _streaming_inverse(prob, mu)
    K = prob["h"].size
    phi = np.zeros((K, 2, L + 1)) if phi0 is None else np.array(phi0, dtype=np.float64)
    hist = []
    for it in range(1, max_it + 1):
        psi = Linv(scattering_source(M, prob["sigma_s"], phi, prob["Q"]), incident=True)
        phi_new = moments(D, psi)
        e = rel_change(phi_new, phi)
        hist.append(e)
        phi = phi_new
        if e < tol:
            break
    return (phi, it, hist) if history else (phi, it)


def fpsa_source_iteration(prob, laplacian="mpd", tol=1e-10, max_it=10000, phi0=None,
                          history=False, return_psi=False):
    """FPSA source iteration (Eqs. predict, correct, iterate).

    Predict:  L psi^{m+1/2} = S psi^m + q                        (sweep)
    Correct:  psi^{m+1} = psi^{m+1/2} + F^{-1} S (psi^{m+1/2} - psi^m)
    with F the LD / S_N FP operator using the MPD or WFD angular Laplacian,
    factorized once by sparse LU (the paper factorizes the FP stiffness matrix
    with an LU 'factorize' object, Sec. 4) and solved each iteration. Only the
    moments l <= L of the corrected flux feed the next scattering source, so the
    state carried is phi^{m+1} = phi^{m+1/2} + D F^{-1} S (psi^{m+1/2} - psi^m).
    Returns (phi, iterations[, history][, psi]) where psi is the corrected angular
    flux of the last iteration.
    Pinned by: one-iteration convergence for P_L-equivalent moments with N = L+1
    (Eq. fsa_pl_eq, P5); fixed point equal to the direct solve (P7); infinite-medium
    one-step convergence (P4).
    """
    N, L = prob["N"], prob["L"]
    mu, w, D, M = tables(N, L)
    K = prob["h"].size
    Linv = _streaming_inverse(prob, mu)
    F = spla.splu(fp_matrix(prob, mu, w, laplacian))
    phi = np.zeros((K, 2, L + 1)) if phi0 is None else np.array(phi0, dtype=np.float64)
    hist = []
    psi = None
    for it in range(1, max_it + 1):
        psi_half = Linv(scattering_source(M, prob["sigma_s"], phi, prob["Q"]), incident=True)
        phi_half = moments(D, psi_half)
        r = scattering_source(M, prob["sigma_s"], phi_half - phi)      # S (psi^{m+1/2} - psi^m)
        ups = F.solve(tr.mass_weight(prob["h"], r).ravel()).reshape(K, 2, N)
        psi = psi_half + ups
        phi_new = phi_half + moments(D, ups)
        e = rel_change(phi_new, phi)
        hist.append(e)
        phi = phi_new
        if e < tol:
            break
    out = (phi, it)
    if history:
        out = out + (hist,)
    if return_psi:
        out = out + (psi,)
    return out


def fpsa_iteration_matrix(prob, laplacian="mpd"):
    """Dense matrix G of one homogeneous FPSA iteration on the flux moments, phi -> phi'
    (Eqs. predict, correct with zero source and zero incoming flux), columns in the
    order of phi.ravel() ([cell][node][l]); small problems only (one iteration per
    column). Its spectral radius is the asymptotic error reduction per iteration.
    Pinned by: on a uniform slab with reflective edges it equals the angularly-discrete
    Fourier analysis (oracle.fourier) at lambda = 0 exactly and, for a supremum at
    lambda > 0, to third order in the cell width (tests/test_oracle_fourier.py).
    """
    N, L = prob["N"], prob["L"]
    mu, w, D, M = tables(N, L)
    K = prob["h"].size
    Linv = _streaming_inverse(prob, mu)
    F = spla.splu(fp_matrix(prob, mu, w, laplacian))
    n = K * 2 * (L + 1)
    G = np.zeros((n, n))
    for j in range(n):
        phi = np.zeros(n)
        phi[j] = 1.0
        phi = phi.reshape(K, 2, L + 1)
        psi_half = Linv(scattering_source(M, prob["sigma_s"], phi), incident=False)
        phi_half = moments(D, psi_half)
        r = scattering_source(M, prob["sigma_s"], phi_half - phi)
        ups = F.solve(tr.mass_weight(prob["h"], r).ravel()).reshape(K, 2, N)
        G[:, j] = (phi_half + moments(D, ups)).ravel()
    return G


def direct_solve(prob, return_psi=False):
    """The discrete solution itself: (L_h - S_h) psi = m q + (incoming boundary fluxes) by
    sparse LU (the fixed point that SI and FPSA converge to; unique for sigma_a > 0)."""
    N, L = prob["N"], prob["L"]
    mu, w, D, M = tables(N, L)
    K = prob["h"].size
    A = transport_matrix(prob, mu, w)
    b = tr.mass_weight(prob["h"], scattering_source(M, np.zeros_like(prob["sigma_s"]),
                                                   np.zeros((K, 2, L + 1)), prob["Q"])) \
        + tr.incident_source(mu, K, prob.get("psi_inc"), prob.get("bc", "vacuum"))
    psi = spla.splu(A).solve(b.ravel()).reshape(K, 2, N)
    phi = moments(D, psi)
    return (phi, psi) if return_psi else phi


def fpsa_gmres(prob, laplacian="mpd", restart=30, tol=1e-10, max_it=10000, history=False):
    """Restarted GMRES(restart) with right FPSA preconditioning (Sec. 4, 'FPSA-preconditioned GMRES').

    FPSA source iteration is the Richardson iteration
        phi^{m+1} = phi^m + (I + C) (b - (I - T) phi^m)
    for the moment equation (I - T) phi = b, with the source-iteration operator
    T = D L^{-1} M Sigma, b = D L^{-1} M Q (Eq. trsi) and the FP correction
    C = D F^{-1} (m (x) M Sigma) (Eq. correct). GMRES is applied to the right-
    preconditioned system (I - T)(I + C) u = b from u = 0 and returns
    phi = (I + C) u. Arnoldi by modified Gram-Schmidt, the least-squares problem by
    Givens rotations; stop when ||b - (I - T) phi|| / ||b|| < tol (2-norm over all
    moments). Returns (phi, iterations[, residual history]).
    Pinned by: the fixed point equals the direct solve; full GMRES (restart >=
    dimension) terminates within the dimension; residuals never increase within a
    cycle; fewer iterations than FPSA source iteration on forward-peaked slabs.
    """
    N, L = prob["N"], prob["L"]
    mu, w, D, M = tables(N, L)
    K = prob["h"].size
    Linv = _streaming_inverse(prob, mu)
    F = spla.splu(fp_matrix(prob, mu, w, laplacian))
    ss = prob["sigma_s"]
    shape = (K, 2, L + 1)

    def T(v):
        return moments(D, Linv(scattering_source(M, ss, v)))

    def C(v):
        return moments(D, F.solve(tr.mass_weight(prob["h"], scattering_source(M, ss, v)).ravel()).reshape(K, 2, N))

    def A(u):
        z = u + C(u)
        return z - T(z)

    b = moments(D, Linv(scattering_source(M, np.zeros_like(ss), np.zeros(shape), prob["Q"]), incident=True))
    bnorm = np.linalg.norm(b)
    u = np.zeros(shape)
    hist = []
    it = 0
    while it < max_it:
        r = b - A(u)
        beta = np.linalg.norm(r)
        if beta / bnorm < tol:
            break
        V = [r / beta]
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j = 0
        for j in range(restart):
            wv = A(V[j])
            for i in range(j + 1):
                H[i, j] = np.sum(wv * V[i])
                wv = wv - H[i, j] * V[i]
            hnext = np.linalg.norm(wv)
            H[j + 1, j] = hnext
            for i in range(j):                      # apply the earlier rotations to column j
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j], H[j + 1, j] = den, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            hist.append(abs(g[j + 1]) / bnorm)
            if hist[-1] < tol or it >= max_it or hnext == 0.0:
                break
            V.append(wv / hnext)
        y = np.linalg.solve(np.triu(H[:j + 1, :j + 1]), g[:j + 1])
        for i in range(j + 1):
            u = u + y[i] * V[i]
        if hist and hist[-1] < tol:
            break
    phi = u + C(u)
    return (phi, it, hist) if history else (phi, it)
