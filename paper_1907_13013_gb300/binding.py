"""Thin ctypes binding of libfpsa.so (argument marshalling only).

Every step of the solve runs in the library's CUDA kernels; this module only
packs descriptors, passes host (numpy) or device (torch CUDA tensor) pointers
and the current torch stream, and unpacks results. It raises if the library
is missing: there is no CPU fallback.

Names follow the C ABI in include/fpsa.h: fpsa_create, fpsa_set_xs,
fpsa_solve, fpsa_adjoint, fpsa_get_tuning / fpsa_set_tuning / fpsa_autotune,
fpsa_destroy, fpsa_strerror, fpsa_last_error.
"""

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfpsa.so")

OK, EINVAL, ENOMEM, ENONFINITE, ENOTCONV, EPIVOT, ETIMEOUT, ECUDA, ENOTSUP, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
LAPLACIAN = {"mpd": 0, "wfd": 1}
PRECISION = {"fp64": 0, "mixed": 1}
METHOD = {"si": 0, "fpsa": 1, "gmres": 2}
CONTRACTION = {"auto": 0, "simt": 1, "tensor": 2}
BC = {"vacuum": 0, "reflective": 1}
MEM_HOST, MEM_DEVICE = 0, 1
MAX_ORDINATES = 256


class FpsaDesc(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int32), ("n_ordinates", ctypes.c_int32),
                ("n_moments", ctypes.c_int32), ("n_rhs", ctypes.c_int32),
                ("n_cells", ctypes.POINTER(ctypes.c_int32)), ("h", ctypes.POINTER(ctypes.c_double)),
                ("laplacian", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("bc", ctypes.POINTER(ctypes.c_int32))]


class FpsaOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("max_iterations", ctypes.c_int32), ("tol", ctypes.c_double),
                ("inner_iterations", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("contraction", ctypes.c_int32), ("restart", ctypes.c_int32)]


class FpsaStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("outer_iterations", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("rel_change", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("cell_angles", ctypes.c_double),
                ("pivot_growth", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FpsaTuning(ctypes.Structure):
    _fields_ = [("sweep_cells_per_thread", ctypes.c_int32), ("solve_blocks_per_sm", ctypes.c_int32),
                ("solve_max_slices", ctypes.c_int32), ("factor_engine", ctypes.c_int32),
                ("solve_engine", ctypes.c_int32), ("residual_engine", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


PHASES = ["sweep", "contract", "bcr_solve", "bcr_invert", "bcr_schur", "assemble", "convergence", "residual"]


class FpsaProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 8), ("timed", ctypes.c_int64 * 8), ("ms", ctypes.c_double * 8)]

    def as_dict(self):
        return {ph: {"launches": int(self.launches[i]), "timed": int(self.timed[i]), "ms": float(self.ms[i])}
                for i, ph in enumerate(PHASES)}


EXPORTS = ["fpsa_create", "fpsa_set_xs", "fpsa_solve", "fpsa_destroy", "fpsa_strerror", "fpsa_last_error",
           "fpsa_profile_enable", "fpsa_profile_read", "fpsa_sweep_noalloc", "fpsa_adjoint",
           "fpsa_set_incident", "fpsa_get_tuning", "fpsa_set_tuning", "fpsa_autotune", "fpsa_tables",
           "fpsa_set_limits"]
NOALLOC_MAX_CELL_ANGLES = 131072

_lib = None


def load():
    """Load libfpsa.so once (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfpsa.so not built (run __graft_entry__.build()); no CPU fallback exists")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p
    lib.fpsa_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(FpsaDesc)]
    lib.fpsa_create.restype = ctypes.c_int
    lib.fpsa_set_xs.argtypes = [vp, dp, dp, dp, i32]
    lib.fpsa_set_xs.restype = ctypes.c_int
    lib.fpsa_solve.argtypes = [vp, ctypes.POINTER(FpsaOpts), dp, dp, i32, ctypes.POINTER(FpsaStats)]
    lib.fpsa_solve.restype = ctypes.c_int
    lib.fpsa_destroy.argtypes = [vp]
    lib.fpsa_destroy.restype = None
    lib.fpsa_strerror.argtypes = [ctypes.c_int]
    lib.fpsa_strerror.restype = ctypes.c_char_p
    lib.fpsa_last_error.argtypes = [vp]
    lib.fpsa_last_error.restype = ctypes.c_char_p
    lib.fpsa_profile_enable.argtypes = [vp, i32]
    lib.fpsa_profile_enable.restype = ctypes.c_int
    lib.fpsa_profile_read.argtypes = [vp, ctypes.POINTER(FpsaProfile)]
    lib.fpsa_profile_read.restype = ctypes.c_int
    lib.fpsa_adjoint.argtypes = [vp, ctypes.POINTER(FpsaOpts), dp, dp, dp, dp, i32, ctypes.POINTER(FpsaStats)]
    lib.fpsa_adjoint.restype = ctypes.c_int
    lib.fpsa_set_incident.argtypes = [vp, dp, i32]
    lib.fpsa_set_incident.restype = ctypes.c_int
    lib.fpsa_get_tuning.argtypes = [vp, ctypes.POINTER(FpsaTuning)]
    lib.fpsa_get_tuning.restype = ctypes.c_int
    lib.fpsa_set_tuning.argtypes = [vp, ctypes.POINTER(FpsaTuning)]
    lib.fpsa_set_tuning.restype = ctypes.c_int
    lib.fpsa_autotune.argtypes = [vp, ctypes.POINTER(FpsaOpts), i32, ctypes.POINTER(FpsaTuning),
                                  ctypes.POINTER(ctypes.c_double)]
    lib.fpsa_autotune.restype = ctypes.c_int
    lib.fpsa_tables.argtypes = [i32, i32, i32, dp, dp, dp, dp, dp]
    lib.fpsa_tables.restype = ctypes.c_int
    lib.fpsa_set_limits.argtypes = [vp, ctypes.c_int64, ctypes.c_double]
    lib.fpsa_set_limits.restype = ctypes.c_int
    lib.fpsa_sweep_noalloc.argtypes = [i32, i32, dp, dp, dp, dp, vp]
    lib.fpsa_sweep_noalloc.restype = ctypes.c_int
    lib.fpsa_solve_batch.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(FpsaOpts), ctypes.POINTER(dp), i32,
                                     ctypes.POINTER(FpsaStats)]
    lib.fpsa_solve_batch.restype = ctypes.c_int
    _lib = lib
    return lib


class FpsaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (load().fpsa_strerror(code).decode(), code, msg))
        self.code = code


def _ptr(x):
    """(pointer, mem kind, keepalive) of a numpy array (host) or torch CUDA tensor (device)."""
    if isinstance(x, np.ndarray):
        a = np.ascontiguousarray(x, dtype=np.float64)
        return a.ctypes.data, MEM_HOST, a
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("device arrays must be contiguous float64 torch tensors")
        return x.data_ptr(), (MEM_DEVICE if x.is_cuda else MEM_HOST), x
    raise TypeError("expected numpy array or torch tensor")


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


class Context:
    """One fpsa_ctx: B slab instances sharing (N, L), ragged cell counts, R right-hand sides."""

    def __init__(self, n_cells, h, N, L, n_rhs=1, laplacian="mpd", precision="fp64", device=0, stream=None,
                 bc=None):
        """bc: None / 'vacuum' / 'reflective' / a (left, right) pair for every instance, or a
        list with one of those per instance."""
        lib = load()
        self.n_cells = np.ascontiguousarray(np.atleast_1d(n_cells), dtype=np.int32)
        self.h = np.ascontiguousarray(h, dtype=np.float64)
        self.N, self.L, self.R = int(N), int(L), int(n_rhs)
        self.B = int(self.n_cells.size)
        self.sumK = int(self.n_cells.sum())
        if self.h.size != self.sumK:
            raise ValueError("h must hold sum(n_cells) widths")
        self.stream = _stream_handle(stream)
        self.bc = _bc_array(bc, self.B)
        d = FpsaDesc(self.B, self.N, self.L + 1, self.R,
                     self.n_cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     self.h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     LAPLACIAN[laplacian], PRECISION[precision], int(device), ctypes.c_void_p(self.stream),
                     self.bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if self.bc is not None else None)
        self._h = ctypes.c_void_p()
        rc = lib.fpsa_create(ctypes.byref(self._h), ctypes.byref(d))
        if rc != OK:
            raise FpsaError(rc, "fpsa_create: " + lib.fpsa_last_error(None).decode())
        self._lib = lib

    def _check(self, rc, what):
        if rc != OK:
            raise FpsaError(rc, "%s: %s" % (what, self._lib.fpsa_last_error(self._h).decode()))

    def set_xs(self, sigma_t, sigma_s, q):
        """sigma_t [sumK], sigma_s [sumK][L+1], q [R][sumK][2][L+1] (numpy host or torch cuda float64)."""
        ps = [_ptr(x) for x in (sigma_t, sigma_s, q)]
        mems = {m for _, m, _ in ps}
        if len(mems) != 1:
            raise TypeError("sigma_t, sigma_s and q must all be host or all device")
        self._check(self._lib.fpsa_set_xs(self._h, ps[0][0], ps[1][0], ps[2][0], mems.pop()), "fpsa_set_xs")

    def set_incident(self, psi_inc):
        """Incoming angular fluxes at the vacuum edges, psi_inc [R][B][2][N] (numpy or torch
        cuda float64): [r][b][0] at the left edge (read for mu > 0), [r][b][1] at the right
        edge (read for mu < 0). None clears them."""
        if psi_inc is None:
            self._check(self._lib.fpsa_set_incident(self._h, None, MEM_HOST), "fpsa_set_incident")
            return
        if tuple(psi_inc.shape) != (self.R, self.B, 2, self.N):
            raise ValueError("psi_inc must have shape (R, B, 2, N)")
        pi, mem, keep = _ptr(psi_inc)
        self._check(self._lib.fpsa_set_incident(self._h, pi, mem), "fpsa_set_incident")

    def solve(self, method="fpsa", tol=1e-10, max_iterations=10000, out=None, phi0=None,
              inner_iterations=0, inner_tol=0.0, check_every=1, raise_on_notconv=True, contraction="auto",
              restart=0):
        """Returns (phi, stats dict). phi [R][sumK][2][L+1]: into `out` if given (numpy or torch
        cuda), else a new numpy array."""
        if out is None:
            out = np.zeros((self.R, self.sumK, 2, self.L + 1))
        po, mem, keep = _ptr(out)
        if phi0 is not None:
            p0, m0, keep0 = _ptr(phi0)
            if m0 != mem:
                raise TypeError("phi0 and out must be of the same memory kind")
        else:
            p0 = None
        o = FpsaOpts(METHOD[method], int(max_iterations), float(tol), int(inner_iterations), float(inner_tol),
                     int(check_every), CONTRACTION[contraction], int(restart))
        st = FpsaStats()
        rc = self._lib.fpsa_solve(self._h, ctypes.byref(o), po, p0, mem, ctypes.byref(st))
        if rc != OK and not (rc == ENOTCONV and not raise_on_notconv):
            self._check(rc, "fpsa_solve")
        if isinstance(out, np.ndarray) and keep is not out:
            out[...] = keep
        return out, st.as_dict()

    def adjoint(self, dJ_dphi=None, method="fpsa", tol=1e-12, max_iterations=10000, out_sigma_t=None,
                out_sigma_s=None, inner_iterations=0, check_every=1, contraction="auto"):
        """Gradients of J with respect to sigma_t [sumK] and sigma_s [sumK][L+1] at the last
        converged solve (fpsa_adjoint). dJ_dphi None: J = exit current through the right edge,
        summed over instances and rhs; else the vector-Jacobian product with dJ_dphi
        [R][sumK][2][L+1]. Returns (dJ_dsigma_t, dJ_dsigma_s, J [R][B] or None, stats)."""
        dev = out_sigma_t is not None and not isinstance(out_sigma_t, np.ndarray)
        if out_sigma_t is None:
            out_sigma_t = np.zeros(self.sumK)
        if out_sigma_s is None:
            out_sigma_s = (np.zeros((self.sumK, self.L + 1)) if isinstance(out_sigma_t, np.ndarray)
                           else out_sigma_t.new_zeros((self.sumK, self.L + 1)))
        pt, mem, kt = _ptr(out_sigma_t)
        ps, ms, ks = _ptr(out_sigma_s)
        pg = None
        if dJ_dphi is not None:
            pg, mg, kg = _ptr(dJ_dphi)
            if mg != mem:
                raise TypeError("dJ_dphi and the outputs must be of the same memory kind")
        J = None
        pj = None
        if mem == MEM_HOST:
            J = np.zeros((self.R, self.B))
            pj = J.ctypes.data
        o = FpsaOpts(METHOD[method], int(max_iterations), float(tol), int(inner_iterations), 0.0, int(check_every),
                     CONTRACTION[contraction], 0)
        st = FpsaStats()
        rc = self._lib.fpsa_adjoint(self._h, ctypes.byref(o), pg, pt, ps, pj, mem, ctypes.byref(st))
        self._check(rc, "fpsa_adjoint")
        if isinstance(out_sigma_t, np.ndarray) and kt is not out_sigma_t:
            out_sigma_t[...] = kt
        if isinstance(out_sigma_s, np.ndarray) and ks is not out_sigma_s:
            out_sigma_s[...] = ks
        return out_sigma_t, out_sigma_s, (J if dJ_dphi is None else None), st.as_dict()

    def get_tuning(self):
        """Launch shapes in effect (fpsa_get_tuning), as a dict of the fpsa_tuning fields."""
        t = FpsaTuning()
        self._check(self._lib.fpsa_get_tuning(self._h, ctypes.byref(t)), "fpsa_get_tuning")
        return t.as_dict()

    def set_tuning(self, tuning=None):
        """Request launch shapes (fpsa_set_tuning): a dict of fpsa_tuning fields (missing or
        0: the library's choice); None restores every library choice."""
        if tuning is None:
            self._check(self._lib.fpsa_set_tuning(self._h, None), "fpsa_set_tuning")
            return
        t = FpsaTuning(*(int(tuning.get(k, 0)) for k, _ in FpsaTuning._fields_))
        self._check(self._lib.fpsa_set_tuning(self._h, ctypes.byref(t)), "fpsa_set_tuning")

    def autotune(self, method="fpsa", tol=1e-10, max_iterations=10000, inner_iterations=0, inner_tol=0.0,
                 check_every=1, contraction="auto", restart=0, repeats=3):
        """Time candidate launch shapes on solves with these options and keep the fastest
        (fpsa_autotune). Returns (shapes dict, milliseconds per solve)."""
        o = FpsaOpts(METHOD[method], int(max_iterations), float(tol), int(inner_iterations), float(inner_tol),
                     int(check_every), CONTRACTION[contraction], int(restart))
        t = FpsaTuning()
        ms = ctypes.c_double(0.0)
        self._check(self._lib.fpsa_autotune(self._h, ctypes.byref(o), int(repeats), ctypes.byref(t),
                                            ctypes.byref(ms)), "fpsa_autotune")
        return t.as_dict(), ms.value

    def set_limits(self, wait_polls=0, growth_limit=0.0):
        """Limits of the failure checks (fpsa_set_limits): polls of a BCR dataflow wait before
        it gives up (FPSA_ETIMEOUT) and the pivot-growth limit of fpsa_set_xs (FPSA_EPIVOT);
        0 restores each default."""
        self._check(self._lib.fpsa_set_limits(self._h, int(wait_polls), float(growth_limit)), "fpsa_set_limits")

    def profile_enable(self, on=True):
        """Reset the launch counters; with on, bracket every launch with CUDA events."""
        self._check(self._lib.fpsa_profile_enable(self._h, 1 if on else 0), "fpsa_profile_enable")

    def profile_read(self):
        """Per kernel class: launches, timed launches and summed event milliseconds."""
        p = FpsaProfile()
        self._check(self._lib.fpsa_profile_read(self._h, ctypes.byref(p)), "fpsa_profile_read")
        return p.as_dict()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.fpsa_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tables(N, L, laplacian="mpd"):
    """The library's S_N tables (fpsa_tables; host only, no GPU): dict of mu [N], w [N],
    D [L+1][N], M [N][L+1] and the angular Laplacian A [N][N]."""
    out = {"mu": np.zeros(N), "w": np.zeros(N), "D": np.zeros((L + 1, N)), "M": np.zeros((N, L + 1)),
           "A": np.zeros((N, N))}
    rc = load().fpsa_tables(int(N), int(L + 1), LAPLACIAN[laplacian], *(out[k].ctypes.data for k in
                                                                     ("mu", "w", "D", "M", "A")))
    if rc != OK:
        raise FpsaError(rc, "fpsa_tables (N=%d, L=%d)" % (N, L))
    return out


def sweep_noalloc(N, h, sigma_t, q, psi, stream=None):
    """One LD sweep psi = L^{-1} q of a single slab through fpsa_sweep_noalloc, the entry point
    that allocates no device memory (for callers that cannot call cudaMalloc). h, sigma_t [K],
    q, psi [K][2][N] are contiguous float64 CUDA tensors; the work is enqueued on `stream`
    (default: torch's current stream) and not synchronised."""
    import torch
    for x in (h, sigma_t, q, psi):
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise TypeError("sweep_noalloc takes contiguous float64 CUDA tensors")
    K = int(h.numel())
    rc = load().fpsa_sweep_noalloc(int(N), K, h.data_ptr(), sigma_t.data_ptr(), q.data_ptr(), psi.data_ptr(),
                                   ctypes.c_void_p(_stream_handle(stream)))
    if rc != OK:
        raise FpsaError(rc, "fpsa_sweep_noalloc (N=%d, K=%d)" % (N, K))
    return psi


def solve_batch(contexts, method="fpsa", tol=1e-10, max_iterations=10000, inner_iterations=0,
                contraction="auto", raise_on_notconv=True):
    """fpsa_solve_batch: the MIXED solves of several contexts (e.g. the (N, L) groups of a
    batch of slabs) as one CUDA graph launch. Returns ([phi per context, numpy
    [R][sumK][2][L+1]], [stats dict per context])."""
    lib = load()
    n = len(contexts)
    outs = [np.zeros((c.R, c.sumK, 2, c.L + 1)) for c in contexts]
    handles = (ctypes.c_void_p * n)(*[c._h.value for c in contexts])
    ptrs = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
    st = (FpsaStats * n)()
    o = FpsaOpts(METHOD[method], int(max_iterations), float(tol), int(inner_iterations), 0.0, 1,
                 CONTRACTION[contraction], 0)
    rc = lib.fpsa_solve_batch(handles, n, ctypes.byref(o), ptrs, MEM_HOST, st)
    stats = [s.as_dict() for s in st]
    if rc != OK and not (rc == ENOTCONV and not raise_on_notconv):
        bad = next((i for i, s in enumerate(stats) if s["status"] != OK), 0)
        raise FpsaError(rc, "fpsa_solve_batch: " + lib.fpsa_last_error(handles[bad]).decode())
    return outs, stats


def _bc_array(bc, B):
    """[B][2] int32 edge conditions, or None when every edge is vacuum."""
    if bc is None:
        return None
    per = bc if isinstance(bc, list) else [bc] * B
    if len(per) != B:
        raise ValueError("one boundary condition entry per instance")
    out = np.zeros((B, 2), dtype=np.int32)
    for b, x in enumerate(per):
        pair = (x, x) if isinstance(x, str) else tuple(x)
        out[b] = [BC[pair[0]], BC[pair[1]]]
    return out if out.any() else None


def context_for(problems, n_rhs=None, **kw):
    """Context + set_xs for a list of problem dicts (see inputs.py) sharing N and L; the
    problems' edge conditions ('bc') and incoming fluxes ('psi_inc', [2][N] shared by all
    right-hand sides or [R][2][N]) are passed on."""
    probs = problems if isinstance(problems, (list, tuple)) else [problems]
    N, L = probs[0]["N"], probs[0]["L"]
    K = [p["h"].size for p in probs]
    h = np.concatenate([p["h"] for p in probs])
    st = np.concatenate([p["sigma_t"] for p in probs])
    ss = np.concatenate([p["sigma_s"] for p in probs])
    Qs = [p["Q"] if p["Q"].ndim == 4 else p["Q"][None] for p in probs]
    R = Qs[0].shape[0] if n_rhs is None else n_rhs
    q = np.concatenate(Qs, axis=1)
    if "bc" not in kw and any(p.get("bc", "vacuum") != "vacuum" for p in probs):
        kw["bc"] = [p.get("bc", "vacuum") for p in probs]
    ctx = Context(K, h, N, L, n_rhs=R, **kw)
    try:
        ctx.set_xs(st, ss, q)
        if any(p.get("psi_inc") is not None for p in probs):
            inc = np.zeros((R, len(probs), 2, N))
            for b, p in enumerate(probs):
                if p.get("psi_inc") is not None:
                    inc[:, b] = np.broadcast_to(p["psi_inc"], (R, 2, N))
            ctx.set_incident(inc)
    except BaseException:
        ctx.close()  # the context's device memory goes now, not when it is collected
        raise
    return ctx


class FPSASolve:
    """torch.autograd.Function wrapper: phi = solve(sigma_t, sigma_s, q) on a Context, with
    backward = fpsa_adjoint (implicit differentiation of the converged fixed point; no
    iteration history is stored). Inputs are contiguous float64 CUDA tensors:
    sigma_t [sumK], sigma_s [sumK][L+1], q [R][sumK][2][L+1]; returns phi [R][sumK][2][L+1].
    Gradients flow to sigma_t and sigma_s (q is treated as a constant)."""

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(actx, fctx, sigma_t, sigma_s, q, tol, max_iterations):
                    fctx.set_xs(sigma_t.detach(), sigma_s.detach(), q.detach())
                    phi = torch.empty((fctx.R, fctx.sumK, 2, fctx.L + 1), dtype=torch.float64, device=sigma_t.device)
                    fctx.solve("fpsa", tol=tol, max_iterations=max_iterations, out=phi)
                    fctx._generation = getattr(fctx, "_generation", 0) + 1
                    actx.fctx = fctx
                    actx.gen = fctx._generation
                    actx.tol, actx.max_iterations = tol, max_iterations
                    actx.save_for_backward(sigma_t.detach(), sigma_s.detach(), q.detach())
                    return phi

                @staticmethod
                def backward(actx, grad_phi):
                    fctx = actx.fctx
                    sigma_t, sigma_s, q = actx.saved_tensors
                    if getattr(fctx, "_generation", 0) != actx.gen:
                        # the context has solved something else since: restore this forward state
                        fctx.set_xs(sigma_t, sigma_s, q)
                        fctx.solve("fpsa", tol=actx.tol, max_iterations=actx.max_iterations,
                                   out=torch.empty((fctx.R, fctx.sumK, 2, fctx.L + 1), dtype=torch.float64,
                                                   device=sigma_t.device))
                        fctx._generation += 1
                        actx.gen = fctx._generation
                    d_st = torch.empty_like(sigma_t)
                    d_ss = torch.empty_like(sigma_s)
                    fctx.adjoint(dJ_dphi=grad_phi.contiguous(), tol=min(actx.tol, 1e-12), out_sigma_t=d_st,
                                 out_sigma_s=d_ss)
                    return None, d_st, d_ss, None, None, None

            cls._fn = _F
        return cls._fn

    @classmethod
    def apply(cls, fctx, sigma_t, sigma_s, q, tol=1e-12, max_iterations=10000):
        return cls.function().apply(fctx, sigma_t, sigma_s, q, tol, max_iterations)
