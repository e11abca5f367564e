"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerance: converged scalar flux within 1e-9 relative (max-norm, relative to
max|phi_0|) of the oracle; both sides iterate to a relative change of 1e-13 so
the iteration error is far below the bound. Moments l >= 1 are compared with the
same absolute scale.
"""
import numpy as np
import pytest

from oracle import iterations as oit
from paper_1907_13013_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def binding():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1907_13013_gb300 import binding as b
    return b


def relerr(phi, ref):
    return np.abs(phi - ref).max() / np.abs(ref[..., 0]).max()


def oracle(p, method, lap="mpd", tol=1e-13, max_it=5000):
    if method == "si":
        return oit.source_iteration(p, tol=tol, max_it=max_it)
    return oit.fpsa_source_iteration(p, lap, tol=tol, max_it=max_it)


@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_plain_hg_slab_fpsa(binding, lap):
    p = inputs.plain_hg_slab()
    ctx = binding.context_for(p, laplacian=lap)
    phi, st = ctx.solve("fpsa", tol=1e-13, max_iterations=500)
    ref, n = oracle(p, "fpsa", lap)
    assert relerr(phi[0], ref) < TOL
    assert abs(st["iterations"] - n) <= 1
    # direct discrete solution (the fixed point itself)
    assert relerr(phi[0], oit.direct_solve(p)) < TOL


def test_plain_hg_slab_si_iterates_match(binding):
    # identical iterate counts: both sides run exactly 40 SI iterations from zero
    p = inputs.plain_hg_slab()
    ctx = binding.context_for(p)
    phi, st = ctx.solve("si", tol=0.0, max_iterations=40, raise_on_notconv=False)
    ref, _ = oit.source_iteration(p, tol=0.0, max_it=40)
    assert st["iterations"] == 40
    assert relerr(phi[0], ref) < 1e-12


@pytest.mark.parametrize("N,K,seed,kernel", [(2, 5, 0, "hg"), (4, 1, 1, "hg"), (8, 2, 2, "srk"),
                                             (8, 3, 3, "hg"), (16, 33, 4, "srk"), (32, 64, 5, "hg"),
                                             (64, 97, 6, "srk")])
@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_random_slabs(binding, N, K, seed, kernel, lap):
    p = inputs.random_slab(K, N, N - 1, seed=seed, kernel=kernel, thick=(1, 300), c=(0.5, 0.999))
    ctx = binding.context_for(p, laplacian=lap)
    phi, st = ctx.solve("fpsa", tol=1e-13, max_iterations=2000)
    ref, n = oracle(p, "fpsa", lap)
    assert relerr(phi[0], ref) < TOL, (relerr(phi[0], ref), st)


def test_truncated_expansion_L_below_N_minus_1(binding):
    p = inputs.random_slab(40, 16, 5, seed=7, kernel="hg")
    ctx = binding.context_for(p)
    phi, st = ctx.solve("fpsa", tol=1e-13, max_iterations=2000)
    ref, n = oracle(p, "fpsa")
    assert phi.shape == (1, 40, 2, 6)
    assert relerr(phi[0], ref) < TOL


def test_batch_ragged_instances_and_rhs(binding):
    # several instances of different cell counts and R = 3 right-hand sides in one context
    R = 3
    probs = [inputs.random_slab(K, 16, 15, seed=20 + i, kernel="srk", nrhs=R) for i, K in enumerate([1, 7, 64, 33, 2])]
    ctx = binding.context_for(probs)
    phi, st = ctx.solve("fpsa", tol=1e-13, max_iterations=2000)
    off = 0
    for p in probs:
        K = p["h"].size
        for r in range(R):
            pr = dict(p, Q=p["Q"][r])
            ref, _ = oracle(pr, "fpsa")
            assert relerr(phi[r, off:off + K], ref) < TOL
        off += K


def test_pl_equivalent_one_iteration(binding):
    # Eq. fsa_pl_eq: P_L-equivalent moments with N = L+1 converge in one FPSA iteration (MPD)
    p = inputs.pl_equivalent_slab(50, 16, 3)
    ctx = binding.context_for(p, laplacian="mpd")
    phi, st = ctx.solve("fpsa", tol=0.0, max_iterations=1, raise_on_notconv=False)
    assert relerr(phi[0], oit.direct_solve(p)) < 1e-10


def test_device_pointers_and_phi0(binding):
    import torch
    p = inputs.random_slab(30, 8, 7, seed=8)
    ctx = binding.context_for(p)
    dev = torch.device("cuda:0")
    st_ = torch.tensor(p["sigma_t"], device=dev)
    ss = torch.tensor(p["sigma_s"], device=dev)
    q = torch.tensor(p["Q"][None], device=dev)
    ctx.set_xs(st_, ss, q)
    out = torch.zeros((1, 30, 2, 8), dtype=torch.float64, device=dev)
    ctx.solve("fpsa", tol=1e-13, out=out)
    ref, _ = oracle(p, "fpsa")
    assert relerr(out.cpu().numpy()[0], ref) < TOL
    # restarting from the converged moments converges at once (resume = pass back the iterate)
    out2 = torch.zeros_like(out)
    _, st = ctx.solve("fpsa", tol=1e-11, out=out2, phi0=out.clone())
    assert st["iterations"] <= 2


def test_error_paths(binding):
    p = inputs.random_slab(10, 8, 7, seed=9)
    ctx = binding.Context([10], p["h"], 8, 7)
    with pytest.raises(binding.FpsaError) as e:
        ctx.solve()
    assert e.value.code == binding.ESTATE
    bad = p["sigma_t"].copy(); bad[3] = -1.0
    with pytest.raises(binding.FpsaError) as e:
        ctx.set_xs(bad, p["sigma_s"], p["Q"][None])
    assert e.value.code == binding.EINVAL
    nan = p["Q"][None].copy(); nan[0, 2, 1, 0] = np.nan
    with pytest.raises(binding.FpsaError) as e:
        ctx.set_xs(p["sigma_t"], p["sigma_s"], nan)
    assert e.value.code == binding.ENONFINITE
    ctx.set_xs(p["sigma_t"], p["sigma_s"], p["Q"][None])
    with pytest.raises(binding.FpsaError) as e:
        ctx.solve("si", tol=1e-14, max_iterations=3)
    assert e.value.code == binding.ENOTCONV


def read_golden(name):
    import os
    vals, its = [], {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            if line.startswith("#"):
                if "iterations to relative change" in line:
                    key = line.split("change")[1].split(":")[0].strip().split()[0]
                    its[key] = int(line.rsplit(":", 1)[1])
                continue
            vals.append(float(line))
    return np.array(vals), its


@pytest.mark.parametrize("name,factory", [("plain_hg_slab", inputs.plain_hg_slab),
                                          ("precision_srk_slab", inputs.precision_srk_slab)])
@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_full_size_against_golden(binding, name, factory, lap):
    # Full-size workloads in the benchmark's launch configuration, against the stored oracle flux.
    p = factory()
    ref, its = read_golden("%s_fpsa_%s_phi0.txt" % (name, lap))
    ctx = binding.context_for(p, laplacian=lap)
    phi, st = ctx.solve("fpsa", tol=1e-10)
    assert abs(st["iterations"] - its["1e-10"]) <= 1, (st, its)
    phi0 = phi[0, :, :, 0].ravel()
    assert np.abs(phi0 - ref).max() / np.abs(ref).max() < TOL
    phi, st = ctx.solve("fpsa", tol=1e-13)
    assert np.abs(phi[0, :, :, 0].ravel() - ref).max() / np.abs(ref).max() < 1e-11


# ---------------------------------------------------------------------------
# Mixed precision: FP32 sweeps / contractions / BCR inside FP64 refinement.
# The converged flux must still be within 1e-9 of the FP64 oracle.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,K,seed,kernel", [(2, 5, 0, "hg"), (8, 3, 3, "hg"), (16, 33, 4, "srk"),
                                             (32, 64, 5, "hg"), (64, 97, 6, "srk")])
@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_mixed_random_slabs(binding, N, K, seed, kernel, lap):
    p = inputs.random_slab(K, N, N - 1, seed=seed, kernel=kernel, thick=(1, 300), c=(0.5, 0.999))
    ctx = binding.context_for(p, laplacian=lap, precision="mixed")
    phi, st = ctx.solve("fpsa", tol=1e-12, max_iterations=100)
    ref, n = oracle(p, "fpsa", lap)
    assert relerr(phi[0], ref) < TOL, (relerr(phi[0], ref), st)


@pytest.mark.parametrize("N,K,seed,c", [(16, 120, 8, (0.9, 0.9999)), (64, 200, 9, (0.99, 0.99999))])
def test_mixed_adaptive_inner_count(binding, N, K, seed, c):
    # the adaptive inner count (inner_iterations 0) reaches the oracle's solution in no more
    # refinement steps than a fixed count of 4 and with inner iterations in [4, 16] per step
    p = inputs.random_slab(K, N, N - 1, seed=seed, kernel="srk", thick=(5, 500), c=c)
    ctx = binding.context_for(p, laplacian="wfd", precision="mixed")
    phi_a, st_a = ctx.solve("fpsa", tol=1e-12, max_iterations=100)
    phi_f, st_f = ctx.solve("fpsa", tol=1e-12, max_iterations=100, inner_iterations=4)
    ref = oit.direct_solve(p)
    assert relerr(phi_a[0], ref) < TOL and relerr(phi_f[0], ref) < TOL
    assert st_a["outer_iterations"] <= st_f["outer_iterations"], (st_a, st_f)
    assert st_a["sweeps"] <= 16 * (st_a["outer_iterations"] - 1), st_a


def test_mixed_batch_and_si(binding):
    R = 2
    probs = [inputs.random_slab(K, 8, 7, seed=40 + i, kernel="hg", c=(0.3, 0.8), nrhs=R) for i, K in enumerate([1, 9, 40])]
    for method in ("fpsa", "si"):
        ctx = binding.context_for(probs, precision="mixed")
        phi, st = ctx.solve(method, tol=1e-12, max_iterations=200, inner_iterations=8)
        off = 0
        for p in probs:
            K = p["h"].size
            for r in range(R):
                ref = oit.direct_solve(dict(p, Q=p["Q"][r]))
                assert relerr(phi[r, off:off + K], ref) < TOL, (method, relerr(phi[r, off:off + K], ref))
            off += K


@pytest.mark.parametrize("name,factory", [("plain_hg_slab", inputs.plain_hg_slab),
                                          ("precision_srk_slab", inputs.precision_srk_slab)])
@pytest.mark.parametrize("lap", ["mpd", "wfd"])
def test_mixed_full_size_against_golden(binding, name, factory, lap):
    p = factory()
    ref, its = read_golden("%s_fpsa_%s_phi0.txt" % (name, lap))
    ctx = binding.context_for(p, laplacian=lap, precision="mixed")
    phi, st = ctx.solve("fpsa", tol=1e-10, max_iterations=50)
    err = np.abs(phi[0, :, :, 0].ravel() - ref).max() / np.abs(ref).max()
    assert err < TOL, (err, st)


# ---------------------------------------------------------------------------
# Adjoint: gradients of the exit current / of a moment functional with respect to
# every per-cell sigma_t and sigma_s,l, against the oracle adjoint (sparse LU of A^T).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("objective", ["exit", "vjp"])
@pytest.mark.parametrize("N,K,seed,kernel", [(8, 13, 1, "srk"), (16, 40, 2, "hg"), (64, 60, 3, "srk")])
def test_adjoint_against_oracle(binding, precision, objective, N, K, seed, kernel):
    from oracle import adjoint as oadj
    p = inputs.random_slab(K, N, N - 1, seed=seed, kernel=kernel, thick=(1, 200), c=(0.6, 0.99))
    g = np.random.default_rng(seed).standard_normal((K, 2, N)) if objective == "vjp" else None
    J, d_st, d_ss, _, _ = oadj.gradients(p, g)
    ctx = binding.context_for(p, precision=precision)
    ctx.solve("fpsa", tol=1e-13, max_iterations=500)
    gt, gs, Jg, st = ctx.adjoint(dJ_dphi=None if g is None else g[None], tol=1e-13)
    if g is None:
        assert abs(Jg[0, 0] - J) < 1e-10 * abs(J)
    assert np.abs(gt - d_st).max() < 1e-8 * np.abs(d_st).max()
    assert np.abs(gs - d_ss).max() < 1e-8 * np.abs(d_ss).max()


def test_adjoint_central_differences_and_batch(binding):
    # two instances x two rhs: gradients are summed over rhs, instances are independent
    R = 2
    probs = [inputs.random_slab(K, 16, 15, seed=50 + i, kernel="srk", thick=(2, 100), c=(0.8, 0.99), nrhs=R)
             for i, K in enumerate([30, 17])]
    ctx = binding.context_for(probs)
    ctx.solve("fpsa", tol=1e-13)
    gt, gs, J, _ = ctx.adjoint(tol=1e-13)
    st = np.concatenate([p["sigma_t"] for p in probs])
    ss = np.concatenate([p["sigma_s"] for p in probs])
    q = np.concatenate([p["Q"] for p in probs], axis=1)

    def Jtot(st_, ss_):
        ctx.set_xs(st_, ss_, q)
        ctx.solve("fpsa", tol=1e-14, max_iterations=2000)
        return ctx.adjoint(tol=1e-6)[2].sum()

    assert J.shape == (R, 2)
    rng = np.random.default_rng(0)
    for i in rng.choice(st.size, 5, replace=False):
        d = 1e-6 * st[i]
        a = st.copy(); a[i] += d
        b = st.copy(); b[i] -= d
        fd = (Jtot(a, ss) - Jtot(b, ss)) / (2 * d)
        assert abs(fd - gt[i]) < 1e-4 * np.abs(gt).max()
        l = int(rng.integers(0, 16))
        d = 1e-6 * max(abs(ss[i, l]), 1e-2)
        a = ss.copy(); a[i, l] += d
        b = ss.copy(); b[i, l] -= d
        fd = (Jtot(st, a) - Jtot(st, b)) / (2 * d)
        assert abs(fd - gs[i, l]) < 1e-4 * np.abs(gs).max()


def test_autograd_function(binding):
    import torch
    from oracle import adjoint as oadj
    p = inputs.random_slab(25, 16, 15, seed=77, kernel="hg", thick=(1, 50), c=(0.7, 0.98))
    dev = torch.device("cuda:0")
    ctx = binding.Context([25], p["h"], 16, 15)
    st = torch.tensor(p["sigma_t"], device=dev, requires_grad=True)
    ss = torch.tensor(p["sigma_s"], device=dev, requires_grad=True)
    q = torch.tensor(p["Q"][None], device=dev)
    w = torch.tensor(np.random.default_rng(3).standard_normal((1, 25, 2, 16)), device=dev)
    phi = binding.FPSASolve.apply(ctx, st, ss, q, 1e-13)
    loss = (phi * w).sum()
    loss.backward()
    J, d_st, d_ss, _, _ = oadj.gradients(p, w[0].cpu().numpy())
    assert abs(loss.item() - J) < 1e-9 * abs(J)
    assert np.abs(st.grad.cpu().numpy() - d_st).max() < 1e-8 * np.abs(d_st).max()
    assert np.abs(ss.grad.cpu().numpy() - d_ss).max() < 1e-8 * np.abs(d_ss).max()


def test_adjoint_requires_forward(binding):
    p = inputs.random_slab(10, 8, 7, seed=9)
    ctx = binding.context_for(p)
    with pytest.raises(binding.FpsaError) as e:
        ctx.adjoint()
    assert e.value.code == binding.ESTATE


# ---------------------------------------------------------------------------
# Tensor-core (tcgen05, split BF16 x3) contractions in the FP32 inner solves.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,K,seed", [(16, 70, 11), (32, 65, 12), (64, 150, 13)])
@pytest.mark.parametrize("contraction", ["tensor", "simt"])
def test_mixed_contraction_engines(binding, N, K, seed, contraction):
    p = inputs.random_slab(K, N, N - 1, seed=seed, kernel="srk", thick=(1, 300), c=(0.5, 0.999))
    ctx = binding.context_for(p, precision="mixed")
    phi, st = ctx.solve("fpsa", tol=1e-12, max_iterations=100, contraction=contraction)
    ref, n = oracle(p, "fpsa")
    assert relerr(phi[0], ref) < TOL, (relerr(phi[0], ref), st)


def test_tensor_contraction_refused_when_N_does_not_qualify(binding):
    p = inputs.random_slab(10, 8, 7, seed=14)
    ctx = binding.context_for(p, precision="mixed")
    with pytest.raises(binding.FpsaError) as e:
        ctx.solve("fpsa", tol=1e-12, contraction="tensor")
    assert e.value.code == binding.ENOTSUP


def test_tensor_contraction_batch_rhs_ragged_tail(binding):
    # 3 instances x 2 rhs, 2*sumK = 2*(61+3+70) = 268 columns: tiles straddle instances and end ragged
    R = 2
    probs = [inputs.random_slab(K, 32, 31, seed=60 + i, kernel="hg", nrhs=R) for i, K in enumerate([61, 3, 70])]
    ctx = binding.context_for(probs, precision="mixed")
    phi, st = ctx.solve("fpsa", tol=1e-12, max_iterations=100, contraction="tensor")
    off = 0
    for p in probs:
        K = p["h"].size
        for r in range(R):
            ref = oit.direct_solve(dict(p, Q=p["Q"][r]))
            assert relerr(phi[r, off:off + K], ref) < TOL
        off += K


# ---------------------------------------------------------------------------
# Large angular orders: 2N > 128 uses the recursive block-Schur inversion
# (N = 96: one Schur level with shared-memory Gauss-Jordan leaves; N = 128, 256:
# register Gauss-Jordan leaves of 128), N = 80 the one-CTA shared-memory inversion.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,K,seed", [(80, 9, 21), (96, 10, 22), (128, 12, 23), (256, 5, 24)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_N(binding, N, K, seed, precision):
    p = inputs.random_slab(K, N, N - 1, seed=seed, kernel="srk", thick=(5, 500), c=(0.8, 0.999))
    ctx = binding.context_for(p, precision=precision)
    phi, st = ctx.solve("fpsa", tol=1e-12, max_iterations=200)
    ref = oit.direct_solve(p)
    assert relerr(phi[0], ref) < TOL, (relerr(phi[0], ref), st)
    assert st["pivot_growth"] < 1e8


# ---------------------------------------------------------------------------
# Differentiation workload (K = 1000, S128, SRK eta = 1e-6, +-5% lognormal noise):
# full-size GPU adjoint against central differences on 20 seeded cells (step 1e-6
# relative, both perturbed solves to a relative change of 1e-13), and mixed vs FP64
# gradients; oracle
# adjoint parity on a reduced slab built with the same recipe.
# ---------------------------------------------------------------------------
def exit_current_weights(N):
    from oracle import quadrature as qd
    mu, w = qd.gauss_legendre(N)
    M = qd.expansion_operator(mu, N - 1)
    pos = mu > 0
    return (w[pos] * mu[pos]) @ M[pos]


def test_differentiation_workload_oracle_parity_reduced(binding):
    from oracle import adjoint as oadj
    p = inputs.differentiation_slab(K=40)
    J, d_st, d_ss, _, _ = oadj.gradients(p)
    for precision in ("fp64", "mixed"):
        ctx = binding.context_for(p, precision=precision)
        ctx.solve("fpsa", tol=1e-13, max_iterations=500)
        gt, gs, Jg, _ = ctx.adjoint(tol=1e-13)
        assert abs(Jg[0, 0] - J) < 1e-9 * abs(J)
        assert np.abs(gt - d_st).max() < 1e-6 * np.abs(d_st).max()
        assert np.abs(gs - d_ss).max() < 1e-6 * np.abs(d_ss).max()


def test_differentiation_workload_full_size_central_differences(binding):
    p = inputs.differentiation_slab()
    K, N, L = p["h"].size, p["N"], p["L"]
    cJ = exit_current_weights(N)
    ctx = binding.context_for(p, precision="fp64")
    ctx.solve("fpsa", tol=1e-13, max_iterations=1000)
    gt, gs, Jg, st = ctx.adjoint(tol=1e-13, max_iterations=1000)
    ctxm = binding.context_for(p, precision="mixed")
    ctxm.solve("fpsa", tol=1e-13, max_iterations=300)
    gtm, gsm, _, _ = ctxm.adjoint(tol=1e-13, max_iterations=300)
    assert np.abs(gtm - gt).max() < 1e-6 * np.abs(gt).max()
    assert np.abs(gsm - gs).max() < 1e-6 * np.abs(gs).max()
    q = p["Q"][None]

    def J(st_, ss_):
        ctx.set_xs(st_, ss_, q)
        phi, _ = ctx.solve("fpsa", tol=1e-13, max_iterations=1000)
        return float(phi[0, K - 1, 1] @ cJ)

    assert abs(J(p["sigma_t"], p["sigma_s"]) - Jg[0, 0]) < 1e-12 * abs(Jg[0, 0])
    rng = np.random.default_rng(2026)
    cells = rng.choice(K, 20, replace=False)
    for i in cells:
        d = 1e-6 * p["sigma_t"][i]
        a = p["sigma_t"].copy(); a[i] += d
        b = p["sigma_t"].copy(); b[i] -= d
        fd = (J(a, p["sigma_s"]) - J(b, p["sigma_s"])) / (2 * d)
        assert abs(fd - gt[i]) < 1e-4 * np.abs(gt).max(), (i, fd, gt[i])
        l = int(rng.integers(0, L + 1))
        d = 1e-6 * abs(p["sigma_s"][i, l])
        a = p["sigma_s"].copy(); a[i, l] += d
        b = p["sigma_s"].copy(); b[i, l] -= d
        fd = (J(p["sigma_t"], a) - J(p["sigma_t"], b)) / (2 * d)
        assert abs(fd - gs[i, l]) < 1e-4 * np.abs(gs).max(), (i, l, fd, gs[i, l])


# ---------------------------------------------------------------------------
# Scale workload (K = 20000, S256, L = 255, HG g = 0.99, c = 0.9999, 64 rhs):
# full size in mixed precision, checked by particle balance per right-hand side
# (emission = absorption + leakage, exact for the LD solution); oracle parity on a
# reduced slab built with the same recipe.
# ---------------------------------------------------------------------------
def balance_defect(p, phi, r):
    from oracle import quadrature as qd
    N, L = p["N"], p["L"]
    mu, w = qd.gauss_legendre(N)
    M = qd.expansion_operator(mu, L)
    pos, neg = mu > 0, mu < 0
    jr = (w[pos] * mu[pos]) @ (M[pos] @ phi[r, -1, 1])
    jl = (w[neg] * -mu[neg]) @ (M[neg] @ phi[r, 0, 0])
    h = p["h"]
    Q = p["Q"][r]
    sa = p["sigma_t"] - p["sigma_s"][:, 0]
    emission = np.sum(h * (Q[:, 0, 0] + Q[:, 1, 0]) / 2)
    absorption = np.sum(sa * h * (phi[r, :, 0, 0] + phi[r, :, 1, 0]) / 2)
    return abs(emission - absorption - jl - jr) / emission


def test_scale_workload_reduced_oracle_parity(binding):
    p = inputs.scale_slab(K=24, nrhs=3)
    ctx = binding.context_for(p, precision="mixed")
    phi, st = ctx.solve("fpsa", tol=1e-12, max_iterations=200)
    for r in range(3):
        ref = oit.direct_solve(dict(p, Q=p["Q"][r]))
        assert relerr(phi[r], ref) < TOL
        assert balance_defect(p, phi, r) < 1e-9


def test_scale_workload_full_size(binding):
    p = inputs.scale_slab()
    ctx = binding.context_for(p, precision="mixed")
    phi, st = ctx.solve("fpsa", tol=1e-10, max_iterations=200)
    assert st["status"] == 0 and np.all(np.isfinite(phi))
    for r in (0, 17, 63):
        assert balance_defect(p, phi, r) < 1e-7, (r, balance_defect(p, phi, r), st)


# ---------------------------------------------------------------------------
# Batching workload (the recipe of inputs.batch_slabs at reduced sizes): uneven K
# and N in {16, 32, 64, 128}, grouped by N into contexts on concurrent streams.
# ---------------------------------------------------------------------------
def test_batching_workload_reduced(binding):
    from paper_1907_13013_gb300 import batch
    probs = inputs.batch_slabs(48, seed=1, K_range=(20, 160))
    solver = batch.BatchSolver(probs, precision="mixed", laplacian="wfd", budget_bytes=64 << 20)
    assert len(solver.waves) > 4  # the small budget forces several waves per group
    phis, stats = solver.solve(tol=1e-12, max_iterations=200)
    assert sum(s["instances"] for s in stats) == len(probs)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(probs), 8, replace=False):
        p = probs[i]
        ref = oit.direct_solve(p)
        assert relerr(phis[i], ref) < TOL, (i, p["N"], p["h"].size)


def window_residual(p, phi, cells):
    """Residual of the discrete LD transport equations (the oracle's L_h - S_h and m q,
    Eq. trop) at the given cells, relative to the largest |L_h - S_h| |psi| + |m q| of
    the window: each cell is checked on the 3-cell window around it, whose rows for
    the middle cell are exactly the full slab's (psi = M phi is exact for L = N - 1).
    A perturbation of phi by 1e-9 of max|phi_0| (the parity bound) raises this measure
    to about 2e-7 on the Batching recipe; the converged solution gives about 1e-15."""
    from oracle import transport as tr
    N, L = p["N"], p["L"]
    mu, w, D, M = oit.tables(N, L)
    K = p["h"].size
    worst = 0.0
    for i in cells:
        a, b = max(i - 1, 0), min(i + 2, K)
        sub = dict(p, h=p["h"][a:b], sigma_t=p["sigma_t"][a:b], sigma_s=p["sigma_s"][a:b], Q=p["Q"][a:b],
                   bc="vacuum")
        A = oit.transport_matrix(sub, mu, w)
        psi = np.einsum("nl,kal->kan", M, phi[a:b]).ravel()
        bv = tr.mass_weight(sub["h"], oit.scattering_source(M, np.zeros_like(sub["sigma_s"]),
                                                            np.zeros_like(phi[a:b]), sub["Q"])).ravel()
        r = A @ psi - bv
        scale = abs(A) @ np.abs(psi) + np.abs(bv)
        rows = slice((i - a) * 2 * N, (i - a + 1) * 2 * N)
        worst = max(worst, float(np.max(np.abs(r[rows])) / np.max(scale)))
    return worst


def test_batching_recipe_full_size_sampled(binding):
    """The first 128 slabs of the seeded 4096-slab Batching recipe (K up to 5000, every N)
    through the batch driver at the bench's tolerance: for each N its largest slab and
    one more, the LD equations at the edges, the region boundary and seeded interior
    cells (window_residual), the particle balance of every slab, and the oracle's
    direct solution for each N's smallest slab."""
    from paper_1907_13013_gb300 import batch
    probs = inputs.batch_slabs(128, seed=0)
    phis, stats = batch.BatchSolver(probs, precision="mixed", laplacian="wfd").solve(tol=1e-10, max_iterations=200)
    assert all(s["status"] == 0 for s in stats)
    rng = np.random.default_rng(5)
    tabs = {}
    for N in (16, 32, 64, 128):
        idx = [i for i, p in enumerate(probs) if p["N"] == N]
        assert idx
        by_k = sorted(idx, key=lambda i: probs[i]["h"].size)
        for i in (by_k[-1], by_k[len(by_k) // 2]):
            p = probs[i]
            K = p["h"].size
            cells = [0, K - 1, K // 2 - 1, K // 2] + [int(x) for x in rng.integers(1, K - 1, 3)]
            res = window_residual(p, np.asarray(phis[i]), cells)
            assert res < 1e-7, (N, K, res)
        small = by_k[0]
        if probs[small]["h"].size <= 1200:
            ref = oit.direct_solve(probs[small])
            assert relerr(np.asarray(phis[small]), ref) < TOL, (N, probs[small]["h"].size)
        if N not in tabs:
            tabs[N] = binding.tables(N, N - 1, "wfd")
    for p, phi in zip(probs, phis):
        mu, w, M = tabs[p["N"]]["mu"], tabs[p["N"]]["w"], tabs[p["N"]]["M"]
        phi = np.asarray(phi)
        jr = (w[mu > 0] * mu[mu > 0]) @ (M[mu > 0] @ phi[-1, 1])
        jl = (w[mu < 0] * -mu[mu < 0]) @ (M[mu < 0] @ phi[0, 0])
        sa = p["sigma_t"] - p["sigma_s"][:, 0]
        emission = np.sum(p["h"] * (p["Q"][:, 0, 0] + p["Q"][:, 1, 0]) / 2)
        absorption = np.sum(sa * p["h"] * (phi[:, 0, 0] + phi[:, 1, 0]) / 2)
        assert abs(emission - absorption - jl - jr) < 1e-9 * emission


# ---------------------------------------------------------------------------
# FPSA-preconditioned GMRES(m) (FP64), against the oracle's GMRES and direct solve.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("lap", ["mpd", "wfd"])
@pytest.mark.parametrize("N,K,seed,restart", [(8, 30, 71, 30), (16, 60, 72, 5), (64, 40, 73, 30)])
def test_gmres_against_oracle(binding, lap, N, K, seed, restart):
    p = inputs.random_slab(K, N, N - 1, seed=seed, kernel="srk", thick=(5, 300), c=(0.9, 0.999))
    ctx = binding.context_for(p, laplacian=lap)
    phi, st = ctx.solve("gmres", tol=1e-12, max_iterations=500, restart=restart)
    ref = oit.direct_solve(p)
    assert relerr(phi[0], ref) < TOL
    _, n_or = oit.fpsa_gmres(p, lap, restart=restart, tol=1e-12)
    assert abs(st["iterations"] - n_or) <= 2, (st["iterations"], n_or)


def test_gmres_batch_systems_and_adjoint(binding):
    R = 2
    probs = [inputs.random_slab(K, 16, 15, seed=80 + i, kernel="hg", c=(0.8, 0.99), nrhs=R) for i, K in enumerate([25, 9])]
    ctx = binding.context_for(probs)
    phi, st = ctx.solve("gmres", tol=1e-12, max_iterations=300)
    off = 0
    for p in probs:
        K = p["h"].size
        for r in range(R):
            assert relerr(phi[r, off:off + K], oit.direct_solve(dict(p, Q=p["Q"][r]))) < TOL
        off += K
    gt, gs, J, _ = ctx.adjoint(method="gmres", tol=1e-13)   # adjoint solve by GMRES too
    gt2, gs2, _, _ = ctx.adjoint(method="fpsa", tol=1e-13)
    assert np.abs(gt - gt2).max() < 1e-8 * np.abs(gt2).max()


def test_gmres_phi0_rule(binding):
    p = inputs.random_slab(10, 8, 7, seed=90)
    ctx = binding.context_for(p)
    with pytest.raises(binding.FpsaError) as e:
        ctx.solve("gmres", tol=1e-10, phi0=np.zeros((1, 10, 2, 8)))
    assert e.value.code == binding.ENOTSUP


# GMRES in MIXED precision: FP32 GMRES(m) inner solves of the correction equation
# inside the FP64 refinement loop reach the FP64 fixed point.
@pytest.mark.parametrize("lap", ["mpd", "wfd"])
@pytest.mark.parametrize("N,K,seed,restart", [(16, 60, 74, 30), (64, 40, 75, 30), (32, 50, 76, 4)])
def test_gmres_mixed_against_oracle(binding, lap, N, K, seed, restart):
    p = inputs.random_slab(K, N, N - 1, seed=seed, kernel="srk", thick=(5, 300), c=(0.9, 0.999))
    ctx = binding.context_for(p, laplacian=lap, precision="mixed")
    phi, st = ctx.solve("gmres", tol=1e-12, max_iterations=60, restart=restart)
    assert relerr(phi[0], oit.direct_solve(p)) < TOL
    assert st["outer_iterations"] <= 12, st


def test_gmres_mixed_batch_and_adjoint(binding):
    R = 2
    probs = [inputs.random_slab(K, 16, 15, seed=80 + i, kernel="hg", c=(0.8, 0.99), nrhs=R) for i, K in enumerate([25, 9])]
    ctx = binding.context_for(probs, precision="mixed")
    phi, st = ctx.solve("gmres", tol=1e-12, max_iterations=60)
    off = 0
    for p in probs:
        K = p["h"].size
        for r in range(R):
            assert relerr(phi[r, off:off + K], oit.direct_solve(dict(p, Q=p["Q"][r]))) < TOL
        off += K
    gt, gs, J, _ = ctx.adjoint(method="gmres", tol=1e-12)
    ref = binding.context_for(probs)
    ref.solve("fpsa", tol=1e-13)
    gt2, gs2, _, _ = ref.adjoint(method="fpsa", tol=1e-13)
    assert np.abs(gt - gt2).max() < 1e-8 * np.abs(gt2).max()
    assert np.abs(gs - gs2).max() < 1e-8 * np.abs(gs2).max()
