"""LD-in-space discretization for the oracle (test infrastructure only; see package header).

The paper discretizes space with linear-discontinuous (LD) finite elements
(Sec. 2.2) but prints no LD equations. Reading used here (and by the CUDA path,
written independently there): Galerkin LD with the linear Lagrange basis
b_L = (z_R - z)/h, b_R = (z - z_L)/h on each cell, consistent (not lumped) mass,
upwind numerical flux at cell edges, and a source that is linear in the cell
with nodal values q_L, q_R. Testing the per-ordinate equation
mu dpsi/dz + sigma psi = q (the L operator of Eq. trop-operator) against b_L, b_R
gives, for one cell of width h and ordinate mu:

    [G(mu) + sigma m] [psi_L, psi_R]^T = m [q_L, q_R]^T + |mu| psi_in e_up

    G(mu) = [[mu/2 - mu [mu<0],  mu/2              ],
             [-mu/2,             -mu/2 + mu [mu>0] ]]
    m     = (h/6) [[2, 1], [1, 2]]

with e_up the upwind node (L for mu > 0, R for mu < 0) and psi_in the upwind
neighbour's outflow value (or the boundary value). For mu > 0 this is
(mu/2 + sigma h/3) psi_L + (mu/2 + sigma h/6) psi_R = mu psi_in + h (2 q_L + q_R)/6
(-mu/2 + sigma h/6) psi_L + (mu/2 + sigma h/3) psi_R = h (q_L + 2 q_R)/6.

Every operator of the form  mu d/dz + K(z)  with K an N x N angular matrix per
cell (K = sigma_t I for L, K = sigma_t I - M diag(sigma_s) D for L - S of Eq. trop,
K = sigma_a I - sigma_tr/2 A_FP for the FP operator F of Eqs. fpop, fp-mpd-oper,
wd-eq-oper) is discretized the same way: block (a, b) of cell i is
G(mu)_ab delta + m_ab K_i.

Unknown ordering of the global vectors: index (i, a, n) -> (2 i + a) N + n with
cell i, node a in {0 = L, 1 = R}, ordinate n (mu ascending).
"""

import numpy as np
import scipy.sparse as sp


def mass_matrix(h):
    """Consistent LD mass matrix m = (h/6)[[2,1],[1,2]] of one cell."""
    return (h / 6.0) * np.array([[2.0, 1.0], [1.0, 2.0]])


def streaming_block(mu):
    """G(mu) of the module docstring: the LD upwind streaming block, shape (2, 2)."""
    pos = 1.0 if mu > 0 else 0.0
    neg = 1.0 - pos
    return np.array([[mu / 2.0 - mu * neg, mu / 2.0],
                     [-mu / 2.0, -mu / 2.0 + mu * pos]])


def sweep(mu, sigma_t, h, q, psi_in_left=None, psi_in_right=None):
    """Upwind LD sweep: solve L psi = q ordinate by ordinate, cell by cell (Eq. trsi, Sec. 2.2).

    q: nodal angular source, shape (K, 2, N). psi_in_left: incoming values at
    the left edge for mu > 0 (shape (N,), entries for mu < 0 ignored);
    psi_in_right likewise at the right edge for mu < 0. Default: vacuum (0).
    Returns psi, shape (K, 2, N). Each cell is one 2 x 2 system per ordinate
    (module docstring), solved by Cramer's rule for all ordinates of one
    direction at once; cells are visited in the upwind order of that direction.
    Pinned by: pure-absorber attenuation = product of Pade[1/2] factors (P3),
    agreement with the sparse global matrix of ``assemble`` (brute force),
    particle balance (P8).
    """
    K, _, N = q.shape
    psi = np.zeros((K, 2, N))
    inL = np.zeros(N) if psi_in_left is None else np.asarray(psi_in_left, dtype=np.float64)
    inR = np.zeros(N) if psi_in_right is None else np.asarray(psi_in_right, dtype=np.float64)
    for forward in (True, False):
        sel = mu > 0 if forward else mu < 0
        if not np.any(sel):
            continue
        m = mu[sel]
        G = np.array([streaming_block(x) for x in m])          # (n_dir, 2, 2)
        inflow = (inL if forward else inR)[sel].copy()
        for i in (range(K) if forward else range(K - 1, -1, -1)):
            mass = mass_matrix(h[i])
            T = G + sigma_t[i] * mass[None, :, :]
            rhs = mass @ q[i][:, sel]                            # (2, n_dir)
            if forward:
                rhs[0] += m * inflow
            else:
                rhs[1] += -m * inflow
            det = T[:, 0, 0] * T[:, 1, 1] - T[:, 0, 1] * T[:, 1, 0]
            psi[i, 0, sel] = (rhs[0] * T[:, 1, 1] - T[:, 0, 1] * rhs[1]) / det
            psi[i, 1, sel] = (T[:, 0, 0] * rhs[1] - T[:, 1, 0] * rhs[0]) / det
            inflow = psi[i, 1, sel] if forward else psi[i, 0, sel]
    return psi


def bc_sides(bc):
    """(left, right) edge conditions from 'vacuum', 'reflective' or a pair of them."""
    if isinstance(bc, str):
        bc = (bc, bc)
    left, right = bc
    for side in (left, right):
        if side not in ("vacuum", "reflective"):
            raise ValueError(f"unknown boundary condition {side!r}")
    return left, right


def assemble(mu, h, Kcell, bc="vacuum"):
    """Global sparse matrix of  mu d/dz + K  in LD (module docstring), shape (2KN, 2KN).

    Kcell: per-cell angular matrices, shape (K, N, N). bc (per edge, see
    ``bc_sides``): 'vacuum' (the incoming flux is a given boundary value, which
    belongs to the right-hand side -- zero in Eq. trans-equation-bc; a beam sets
    one ordinate, see ``incident_source``) or 'reflective' (incoming psi(mu) =
    outgoing psi(-mu) at that edge: the infinite-medium and symmetric-slab special
    cases of the tests and the mirrored half-slab).
    """
    left, right = bc_sides(bc)
    K, N, _ = Kcell.shape
    rows, cols, vals = [], [], []

    def idx(i, a, n):
        return (2 * i + a) * N + n

    for i in range(K):
        mass = mass_matrix(h[i])
        for a in range(2):
            for b in range(2):
                blk = mass[a, b] * Kcell[i]
                r = idx(i, a, 0) + np.arange(N)
                c = idx(i, b, 0) + np.arange(N)
                rr, cc = np.meshgrid(r, c, indexing="ij")
                rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(blk.ravel())
        for n in range(N):
            G = streaming_block(mu[n])
            for a in range(2):
                for b in range(2):
                    if G[a, b] != 0.0:
                        rows.append([idx(i, a, n)]); cols.append([idx(i, b, n)]); vals.append([G[a, b]])
            # upwind coupling: the inflow moves to the left-hand side with sign -|mu|
            if mu[n] > 0:
                if i > 0:
                    rows.append([idx(i, 0, n)]); cols.append([idx(i - 1, 1, n)]); vals.append([-mu[n]])
                elif left == "reflective":
                    rows.append([idx(0, 0, n)]); cols.append([idx(0, 0, N - 1 - n)]); vals.append([-mu[n]])
            else:
                if i < K - 1:
                    rows.append([idx(i, 1, n)]); cols.append([idx(i + 1, 0, n)]); vals.append([mu[n]])
                elif right == "reflective":
                    rows.append([idx(K - 1, 1, n)]); cols.append([idx(K - 1, 1, N - 1 - n)]); vals.append([mu[n]])
    A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(2 * K * N, 2 * K * N))
    A.sum_duplicates()
    return A


def incident_source(mu, K, psi_inc, bc="vacuum"):
    """Right-hand-side contribution of given incoming boundary fluxes, shape (K, 2, N).

    psi_inc: shape (2, N), the incoming angular flux at the left edge (row 0,
    read for mu_n > 0) and at the right edge (row 1, read for mu_n < 0). In the
    cell equations of the module docstring the inflow enters as |mu| psi_in at
    the upwind node of the boundary cell. Reflective edges take no given inflow.
    """
    left, right = bc_sides(bc)
    N = mu.size
    out = np.zeros((K, 2, N))
    if psi_inc is None:
        return out
    psi_inc = np.asarray(psi_inc, dtype=np.float64)
    pos, neg = mu > 0, mu < 0
    if left == "vacuum":
        out[0, 0, pos] = mu[pos] * psi_inc[0, pos]
    if right == "vacuum":
        out[K - 1, 1, neg] = -mu[neg] * psi_inc[1, neg]
    return out


def beam_incident(mu, w, side="left"):
    """Unit beam: unit incoming partial current carried by the most normal incoming
    ordinate only, psi = 1 / (w_n |mu_n|) (the paper's beam source of Sec. 4 gives
    no formula; this is the reading). Returns psi_inc of shape (2, N)."""
    N = mu.size
    out = np.zeros((2, N))
    n = N - 1 if side == "left" else 0
    out[0 if side == "left" else 1, n] = 1.0 / (w[n] * abs(mu[n]))
    return out


def mass_weight(h, q):
    """Apply the cell mass matrix node-wise: (m_i (x) I_N) q_i for every cell. q: (K, 2, N)."""
    out = np.empty_like(q)
    out[:, 0, :] = (h / 6.0)[:, None] * (2.0 * q[:, 0, :] + q[:, 1, :])
    out[:, 1, :] = (h / 6.0)[:, None] * (q[:, 0, :] + 2.0 * q[:, 1, :])
    return out


def exit_currents(mu, w, psi):
    """Outgoing partial currents (J_left, J_right) = sum |mu_n| w_n psi_n over outgoing ordinates."""
    neg = mu < 0
    pos = mu > 0
    jl = np.sum(w[neg] * np.abs(mu[neg]) * psi[0, 0, neg])
    jr = np.sum(w[pos] * mu[pos] * psi[-1, 1, pos])
    return jl, jr
