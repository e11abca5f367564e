"""Seeded synthetic slab problems (shared by the tests, the bench and the oracle checks).

This module builds INPUTS only: cell widths, cross sections, scattering-kernel
Legendre moments and external sources. It holds none of the solver's arithmetic
and imports neither the oracle nor the CUDA binding.

A problem is a dict:
  N, L            S_N order (even) and scattering order, L <= N-1
  h[K]            cell widths [cm]
  sigma_t[K]      total cross section [1/cm]
  sigma_s[K,L+1]  scattering moments sigma_{s,l} = sigma_{s,0} f_l
  Q[K,2,L+1]      external source moments at the two LD nodes of every cell
                  (isotropic scalar source S -> Q_0 = S; angular source S/2)
  bc              'vacuum' (both edges), 'reflective', or a (left, right) pair of them
  psi_inc         optional [2][N] incoming fluxes at the vacuum edges (row 0 left edge,
                  read for mu > 0; row 1 right edge, read for mu < 0)
Batched / multi-right-hand-side problems carry Q[R,K,2,L+1].

Scattering kernels (Sec. 1 and Sec. 4 of the paper name them; their moment
values are external data there):
  Henyey-Greenstein   f_l = g^l
  screened Rutherford sigma_s(mu0) ~ (1 - mu0 + 2 eta)^-2, normalised;
                      f_l = -4 eta (1+eta) Q_l'(1+2 eta) = l (Q_{l-1}(a) - a Q_l(a)),
                      a = 1 + 2 eta, Q_l the Legendre function of the second kind.
"""

import math

import numpy as np

SEED_BASE = 13013


def hg_moments(g, L):
    """Henyey-Greenstein kernel moments f_l = g^l, l = 0..L."""
    return np.asarray(g, dtype=np.float64) ** np.arange(L + 1)


def srk_moments(eta, L):
    """Screened-Rutherford moments f_l = l (Q_{l-1}(a) - a Q_l(a)), a = 1 + 2 eta, f_0 = 1.

    Q_0(a) = atanh(1/a) and Q_1 = a Q_0 - 1, then Bonnet's recurrence
    (l+1) Q_{l+1} = (2l+1) a Q_l - l Q_{l-1}. Forward recurrence of the decaying
    solution amplifies rounding by about (a + sqrt(a^2-1))^{2l}, which stays
    below 3 for the (eta, L) pairs used here (eta >= 1e-6, L <= 255).
    """
    a = 1.0 + 2.0 * eta
    Qf = np.zeros(L + 2)
    Qf[0] = 0.5 * math.log1p(2.0 / (a - 1.0))       # atanh(1/a) = 0.5 ln((a+1)/(a-1))
    Qf[1] = a * Qf[0] - 1.0
    for l in range(1, L + 1):
        Qf[l + 1] = ((2 * l + 1) * a * Qf[l] - l * Qf[l - 1]) / (l + 1)
    f = np.empty(L + 1)
    f[0] = 1.0
    for l in range(1, L + 1):
        f[l] = l * (Qf[l - 1] - a * Qf[l])
    return f


def slab(K, N, L, width, sigma_t, sigma_s, source):
    """Assemble a problem dict from per-cell arrays (broadcast scalars to K cells)."""
    h = np.full(K, width / K)
    st = np.broadcast_to(np.asarray(sigma_t, dtype=np.float64), (K,)).copy()
    ss = np.broadcast_to(np.asarray(sigma_s, dtype=np.float64), (K, L + 1)).copy()
    Q = np.zeros((K, 2, L + 1))
    Q[:, :, 0] = np.broadcast_to(np.asarray(source, dtype=np.float64), (K,))[:, None]
    return dict(N=N, L=L, h=h, sigma_t=st, sigma_s=ss, Q=Q, bc="vacuum")


def plain_hg_slab(K=200, N=16, L=15, g=0.9):
    """Plain FP64 workload: 1 cm, K uniform cells, S_N, HG g expanded to L moments,
    sigma_t = 101/cm, sigma_s0 = 100/cm, uniform isotropic unit source, vacuum."""
    return slab(K, N, L, 1.0, 101.0, 100.0 * hg_moments(g, L), 1.0)


def precision_srk_slab(K=2000, N=64, L=63, eta=1e-5, sigma_s0=1000.0, sigma_a=0.01):
    """Precision workload: 1 cm, K cells, S_N, screened Rutherford (eta) to L moments,
    sigma_s0 = 1000/cm, sigma_a = 0.01/cm, isotropic unit source in the left half only."""
    src = np.where(np.arange(K) < K // 2, 1.0, 0.0)
    return slab(K, N, L, 1.0, sigma_s0 + sigma_a, sigma_s0 * srk_moments(eta, L), src)


def random_slab(K, N, L, seed, kernel="hg", regions=3, thick=(1.0, 300.0), c=(0.5, 0.999),
                width=1.0, ragged_h=True, nrhs=None):
    """Small heterogeneous test slab: `regions` material regions with seeded
    sigma_t (log-uniform in `thick`), scattering ratio c, HG g in [0.5, 0.95] or
    SRK eta in [1e-5, 1e-3]; seeded positive cell widths summing to `width`;
    seeded nonnegative linear sources (different at the two nodes). With nrhs,
    Q has a leading right-hand-side axis."""
    rng = np.random.default_rng(SEED_BASE + seed)
    hw = rng.uniform(0.5, 1.5, K) if ragged_h else np.ones(K)
    h = width * hw / hw.sum()
    bounds = np.sort(rng.choice(np.arange(1, K), size=min(regions - 1, K - 1), replace=False)) \
        if K > 1 else np.array([], dtype=int)
    reg = np.searchsorted(bounds, np.arange(K), side="right")
    nreg = reg.max() + 1
    st_r = np.exp(rng.uniform(np.log(thick[0]), np.log(thick[1]), nreg))
    c_r = rng.uniform(c[0], c[1], nreg)
    if kernel == "hg":
        f_r = np.stack([hg_moments(g, L) for g in rng.uniform(0.5, 0.95, nreg)])
    else:
        f_r = np.stack([srk_moments(e, L) for e in np.exp(rng.uniform(np.log(1e-5), np.log(1e-3), nreg))])
    st = st_r[reg]
    ss = (c_r * st_r)[reg][:, None] * f_r[reg]
    shape = (K, 2) if nrhs is None else (nrhs, K, 2)
    Q = np.zeros(shape + (L + 1,))
    Q[..., 0] = rng.uniform(0.0, 1.0, shape)
    if L >= 1:
        Q[..., 1] = rng.uniform(-0.2, 0.2, shape) * Q[..., 0]
    return dict(N=N, L=L, h=h, sigma_t=st, sigma_s=ss, Q=Q, bc="vacuum")


def mirrored_half_slab(K, N, L, seed, side):
    """A seeded heterogeneous half slab with a reflective edge on `side`, and the
    symmetric slab of 2K cells (vacuum both edges) that it is one half of. The mirror
    image of a cell has its cross sections and width, and its nodal source values in
    reversed node order; only even source moments are used so that the source is
    reflection-symmetric in angle. Returns (half, full, slice of the half in full)."""
    p = random_slab(K, N, L, seed=seed, kernel="hg", thick=(2, 40), c=(0.5, 0.95))
    p["Q"][..., 1::2] = 0.0
    mir = {k: p[k][::-1].copy() for k in ("h", "sigma_t", "sigma_s")}
    mir["Q"] = p["Q"][::-1, ::-1].copy()
    full = dict(N=N, L=L, bc="vacuum")
    first, second = (mir, p) if side == "left" else (p, mir)
    for k in ("h", "sigma_t", "sigma_s", "Q"):
        full[k] = np.concatenate([first[k], second[k]])
    half = dict(p, bc=("reflective", "vacuum") if side == "left" else ("vacuum", "reflective"))
    part = slice(K, 2 * K) if side == "left" else slice(0, K)
    return half, full, part


def pl_equivalent_slab(K, N, seed):
    """P_L-equivalent scattering moments sigma_{s,l} = sigma_{s,0} - sigma_tr/2 l(l+1)
    (Eq. fsa_pl_eq) with L = N-1 in a seeded heterogeneous slab."""
    L = N - 1
    rng = np.random.default_rng(SEED_BASE + 100 + seed)
    h = rng.uniform(0.5, 1.5, K); h /= h.sum()
    st = np.exp(rng.uniform(np.log(2.0), np.log(50.0), K))
    s0 = st * rng.uniform(0.8, 0.99, K)
    s_tr = s0 * rng.uniform(0.001, 0.02, K)
    l = np.arange(L + 1)
    ss = s0[:, None] - 0.5 * s_tr[:, None] * (l * (l + 1))[None, :]
    Q = np.zeros((K, 2, L + 1))
    Q[:, :, 0] = rng.uniform(0.0, 1.0, (K, 2))
    return dict(N=N, L=L, h=h, sigma_t=st, sigma_s=ss, Q=Q, bc="vacuum")


def batch_slabs(B, seed, N_choices=(16, 32, 64, 128), K_range=(100, 5000)):
    """Batching workload: B independent 1 cm slabs with seeded uneven sizes: K uniform
    on K_range, N drawn from N_choices with L = N-1, two material regions (cells
    [0, K/2) and the rest) each with HG g ~ U[0.8, 0.99], c ~ U[0.9, 0.999] and
    sigma_t log-uniform on [1, 1000]/cm; isotropic unit source; vacuum."""
    rng = np.random.default_rng(SEED_BASE + 3 + seed)
    out = []
    for _ in range(B):
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        N = int(rng.choice(N_choices))
        L = N - 1
        g = rng.uniform(0.8, 0.99, 2)
        c = rng.uniform(0.9, 0.999, 2)
        st = np.exp(rng.uniform(0.0, np.log(1000.0), 2))
        reg = (np.arange(K) >= K // 2).astype(int)
        ss = (c * st)[reg][:, None] * np.stack([hg_moments(x, L) for x in g])[reg]
        p = slab(K, N, L, 1.0, st[reg], ss, 1.0)
        out.append(p)
    return out


def differentiation_slab(K=1000, N=128, L=127, eta=1e-6, sigma_s0=1000.0, sigma_a=0.01, noise=0.05, seed=0):
    """Differentiation workload: 1 cm, K cells, S_N, screened Rutherford (eta) to L moments,
    base sigma_s0 = 1000/cm, sigma_a = 0.01/cm, isotropic unit source, vacuum; per-cell
    seeded lognormal noise: sigma_a,i = sigma_a exp(noise z_i), sigma_s,l,i = sigma_s,l exp(noise z'_i)
    (one z' per cell for all l, so each cell keeps a valid kernel shape), sigma_t,i = sigma_a,i + sigma_s0,i."""
    rng = np.random.default_rng(SEED_BASE + 4 + seed)
    z = rng.standard_normal(K)
    zp = rng.standard_normal(K)
    sa = sigma_a * np.exp(noise * z)
    ss = (sigma_s0 * srk_moments(eta, L))[None, :] * np.exp(noise * zp)[:, None]
    return slab(K, N, L, 1.0, sa + ss[:, 0], ss, 1.0)


def scale_slab(K=20000, N=256, L=255, g=0.99, c=0.9999, sigma_t=100.0, nrhs=64, seed=0):
    """Scale workload: 1 cm, K cells, S_N, HG g to L moments, sigma_t = 100/cm, c = 0.9999,
    nrhs seeded nonnegative isotropic sources Q ~ U[0, 1) per (rhs, cell), vacuum."""
    rng = np.random.default_rng(SEED_BASE + 5 + seed)
    p = slab(K, N, L, 1.0, sigma_t, c * sigma_t * hg_moments(g, L), 0.0)
    Q = np.zeros((nrhs, K, 2, L + 1))
    Q[..., 0] = rng.uniform(0.0, 1.0, (nrhs, K))[:, :, None]
    p["Q"] = Q
    return p
