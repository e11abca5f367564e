/*
 * fpsa.h -- C ABI of the GB300 FPSA source-iteration library (libfpsa.so).
 *
 * Computes the steady, mono-energetic 1D slab S_N transport problem of
 * arXiv:1907.13013, Sec. 2 (Eq. treq with Eq. trans-equation-bc):
 *
 *   mu dpsi/dz + sigma_t psi = sum_{l<=L} (2l+1)/2 sigma_{s,l} P_l(mu) phi_l + q
 *
 * discretized with S_N Gauss-Legendre in angle and linear-discontinuous (LD)
 * Galerkin finite elements (consistent mass, upwind edges) in space (Sec. 2.2),
 * and solves it by source iteration (Eq. trsi) or by Fokker-Planck synthetic
 * acceleration (Eqs. predict, correct, iterate) whose correction operator is the
 * FP operator F = mu d/dz + sigma_a - sigma_tr/2 L_FP (Eq. fpop) with the MPD
 * (Eq. fp-mpd) or WFD (Eq. w_wfd) angular Laplacian, sigma_a = sigma_t - sigma_{s,0}
 * and sigma_tr = sigma_{s,0} - sigma_{s,1}.
 *
 * Conventions used by every entry point
 *   - Ordinates mu_1 < ... < mu_N (Gauss-Legendre, weights sum to 2).
 *   - A context holds B independent slab instances sharing (N, L); instance b
 *     has K_b cells. Cells of all instances are concatenated instance-major:
 *     global cell g in [0, sumK), instance b owning [off_b, off_b + K_b).
 *   - Every instance is solved for R right-hand sides (sources) at once.
 *   - Moments at the two LD nodes of a cell: node 0 = left edge, 1 = right edge.
 *   - Layouts are row-major with the LAST index contiguous:
 *       sigma_t [sumK]                 sigma_s [sumK][L+1]
 *       q       [R][sumK][2][L+1]      phi     [R][sumK][2][L+1]
 *     q holds source MOMENTS: the angular source is
 *     q_n = sum_l (2l+1)/2 P_l(mu_n) q_l, so an isotropic scalar source S is q_0 = S.
 *   - Boundary conditions, per instance and edge (fpsa_desc.bc): vacuum with a
 *     given incoming flux (zero unless set by fpsa_set_incident; Eq.
 *     trans-equation-bc) or reflective.
 *   - Ownership: the caller owns every pointer it passes; the library copies
 *     inputs into device buffers it owns and writes results into the caller's
 *     buffers before returning (the context stream is synchronised).
 *   - Errors: every int-returning call returns FPSA_OK (0) or a negative code;
 *     nothing throws across the ABI. fpsa_last_error() gives the message of the
 *     last failing call on a context.
 *   - Threading: one context must not be used from two threads at once.
 */
#ifndef FPSA_H
#define FPSA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FPSA_OK          0
#define FPSA_EINVAL     -1   /* bad argument (sizes, layout, cross sections) */
#define FPSA_ENOMEM     -2   /* device allocation failed */
#define FPSA_ENONFINITE -3   /* a NaN/Inf appeared in an input or iterate */
#define FPSA_ENOTCONV   -4   /* max_iterations reached before tol */
#define FPSA_EPIVOT     -5   /* FP block factorization: zero/non-finite pivot or growth above limit */
#define FPSA_ETIMEOUT   -6   /* a bounded device wait ran out */
#define FPSA_ECUDA      -7   /* a CUDA runtime call failed */
#define FPSA_ENOTSUP    -8   /* configuration outside what the library supports */
#define FPSA_ESTATE     -9   /* call order violated (e.g. solve before set_xs) */

enum fpsa_laplacian { FPSA_LAPLACIAN_MPD = 0, FPSA_LAPLACIAN_WFD = 1 };
enum fpsa_precision { FPSA_PRECISION_FP64 = 0, FPSA_PRECISION_MIXED = 1 };
enum fpsa_method    { FPSA_METHOD_SI = 0, FPSA_METHOD_FPSA = 1, FPSA_METHOD_GMRES = 2 };
enum fpsa_mem       { FPSA_MEM_HOST = 0, FPSA_MEM_DEVICE = 1 };
/* Edge conditions. VACUUM: the incoming flux is given (zero unless set by
 * fpsa_set_incident; Eq. trans-equation-bc). REFLECT: incoming psi(mu) = outgoing
 * psi(-mu) at that edge (the symmetry plane of a slab twice as wide). */
enum fpsa_bc        { FPSA_BC_VACUUM = 0, FPSA_BC_REFLECT = 1 };

typedef struct fpsa_ctx fpsa_ctx;

typedef struct {
    int32_t n_instances;      /* B >= 1 */
    int32_t n_ordinates;      /* N: even, 2 <= N <= FPSA_MAX_ORDINATES */
    int32_t n_moments;        /* L+1: 1 <= L+1 <= N */
    int32_t n_rhs;            /* R >= 1 */
    const int32_t *n_cells;   /* host [B]: K_b >= 1 */
    const double *h;          /* host [sumK]: cell widths > 0 */
    int32_t laplacian;        /* enum fpsa_laplacian */
    int32_t precision;        /* enum fpsa_precision */
    int32_t device;           /* CUDA device ordinal */
    void *stream;             /* cudaStream_t the library launches on; NULL = legacy default */
    const int32_t *bc;        /* host [B][2]: (left, right) enum fpsa_bc per instance; NULL = all vacuum */
} fpsa_desc;

typedef struct {
    int32_t method;           /* enum fpsa_method */
    int32_t max_iterations;   /* cap on transport sweeps (FP64) / refinement steps (MIXED) */
    double tol;               /* SI / FPSA, and every method in MIXED: stop when
                                 max|phi_0^{m+1}-phi_0^m| / max|phi_0^{m+1}| < tol between
                                 iterates (MIXED: between FP64 refinement steps), the worst
                                 instance/right-hand side deciding (Eq. iterate);
                                 GMRES in FP64: stop when every (rhs, instance) system has
                                 ||b - (I-T) phi||_2 / ||b||_2 < tol on the moments */
    int32_t inner_iterations; /* MIXED, SI / FPSA: FP32 iterations per FP64 refinement step;
                                 0 = adaptive (FPSA): 4 per step, and where the first step
                                 shows the FP64 residual taking longer than one inner
                                 iteration (timed by CUDA events), later steps take as many
                                 as the observed contraction per inner iteration needs to
                                 bring the error below tol (at least 4, at most 16, and no
                                 more than keep a step's reduction above 1e-6, the FP32
                                 floor); fpsa_solve_batch: 0 = 4 every step. MIXED, GMRES:
                                 cap on the FP32 Krylov iterations per refinement step
                                 (0 = the restart length) */
    double inner_tol;         /* MIXED, GMRES: relative residual target of each FP32 inner
                                 GMRES solve (0 = default 1e-5); unused otherwise */
    int32_t check_every;      /* test convergence every this many iterations (0 = 1) */
    int32_t contraction;      /* MIXED inner contractions (SI, FPSA and the inner GMRES solves of
                                 GMRES-IR): 0 = auto (tensor cores when N is a
                                 multiple of 16 and <= 128, or a multiple of 32 and <= 256), 1 = SIMT
                                 FP32, 2 = tensor cores (tcgen05, split BF16 x3; FPSA_ENOTSUP if N
                                 does not qualify) */
    int32_t restart;          /* GMRES restart length m (0 = 30) */
} fpsa_opts;

typedef struct {
    int32_t status;           /* same as the return value of fpsa_solve */
    int32_t iterations;       /* FP64: FPSA/SI iterations (GMRES: Krylov iterations); MIXED:
                                 total inner iterations (GMRES: inner Krylov iterations) */
    int32_t outer_iterations; /* MIXED: FP64 refinement steps; FP64: = iterations */
    int32_t sweeps;           /* transport sweeps launched (each covers all instances and rhs) */
    double rel_change;        /* last tested relative change of phi_0 */
    double setup_ms;          /* last fpsa_set_xs: upload + FP assembly + block factorization */
    double solve_ms;          /* this fpsa_solve, wall clock on the host */
    double cell_angles;       /* sum_b K_b * N * R * sweeps */
    double pivot_growth;      /* max over FP blocks of max|A^{-1}| * max|A| (FP64 check) */
} fpsa_stats;

/* Kernel classes for the built-in profiler. */
enum fpsa_phase {
    FPSA_PHASE_SWEEP = 0,       /* LD transport sweep */
    FPSA_PHASE_CONTRACT = 1,    /* moment / scattering-source contractions (+ fused updates) */
    FPSA_PHASE_BCR_SOLVE = 2,   /* block cyclic reduction forward / backward solve */
    FPSA_PHASE_BCR_INVERT = 3,  /* block inversion of eliminated cells (factorization) */
    FPSA_PHASE_BCR_SCHUR = 4,   /* Schur updates of kept cells (factorization) */
    FPSA_PHASE_ASSEMBLE = 5,    /* FP block assembly and sweep coefficients */
    FPSA_PHASE_CONVERGENCE = 6, /* convergence reduction */
    FPSA_PHASE_RESIDUAL = 7,    /* FP64 refinement residual and update (MIXED) */
    FPSA_N_PHASES = 8
};

typedef struct {
    int64_t launches[FPSA_N_PHASES];  /* kernel launches since the last reset (always counted) */
    int64_t timed[FPSA_N_PHASES];     /* launches bracketed by CUDA events while profiling was on */
    double ms[FPSA_N_PHASES];         /* summed event time of the timed launches */
} fpsa_profile;

/* Reset the counters; on != 0 additionally brackets every kernel launch with a
 * pair of CUDA events on the context stream (adds host-side launch overhead). */
int fpsa_profile_enable(fpsa_ctx *ctx, int32_t on);

/* Synchronise the context stream and return the counters since the last reset. */
int fpsa_profile_read(fpsa_ctx *ctx, fpsa_profile *out);

/* Largest N the library supports. */
#define FPSA_MAX_ORDINATES 256

/* Create a context: validates the descriptor, builds the S_N tables (mu_n, w_n,
 * D = [w_n P_l(mu_n)], M = [(2l+1)/2 P_l(mu_n)], the MPD or WFD Laplacian;
 * Sec. 2.2 Eqs. phi-mom, treq, fp-mpd, w_wfd), copies h and allocates every
 * device buffer. *out is NULL on failure. Sets and keeps desc->device current. */
int fpsa_create(fpsa_ctx **out, const fpsa_desc *desc);

/* Load cross sections and sources (layouts above; mem = enum fpsa_mem says
 * whether the three pointers are host or device memory), then assemble the LD
 * FP operator per cell (2N x 2N diagonal blocks, N/2 x N/2 upwind couplings;
 * Eqs. fpop, fp-mpd-oper, wd-eq-oper) and factor it by block cyclic reduction.
 * Requires sigma_t > 0, 0 <= sigma_{s,0} <= sigma_t, finite values.
 * Returns FPSA_EPIVOT if a block is singular or its growth check fails, and
 * FPSA_ETIMEOUT if a bounded device wait of the factorization ran out (the
 * dataflow factorization and the coarse inverse of a single-slab solve wait on
 * counters and copies with limits). */
int fpsa_set_xs(fpsa_ctx *ctx, const double *sigma_t, const double *sigma_s,
                const double *q, int32_t mem);

/* Given incoming angular fluxes at the vacuum edges, psi_inc [R][B][2][N] of kind
 * mem: [r][b][0][n] is the inflow at the left edge (read for mu_n > 0), [r][b][1][n]
 * at the right edge (read for mu_n < 0); other entries and reflective edges are
 * ignored. A unit beam (Sec. 4's beam source) is 1/(w_n |mu_n|) on the most normal
 * incoming ordinate. NULL clears them (no incoming flux). They enter the transport
 * source of fpsa_solve only (fpsa_adjoint solves with homogeneous edges). Values are
 * copied; a later fpsa_solve is needed before fpsa_adjoint. Host values must be
 * finite (FPSA_ENONFINITE). */
int fpsa_set_incident(fpsa_ctx *ctx, const double *psi_inc, int32_t mem);

/* Iterate to convergence (opts may be NULL: FPSA, tol 1e-10, 10000 iterations).
 * Methods: source iteration (Eq. trsi); FPSA source iteration (Eqs. predict,
 * correct, iterate); GMRES(m) on the moment equation (I - T) phi = b with right
 * preconditioning by the FP correction, (I - T)(I + C) u = b, phi = (I + C) u,
 * T = D L^{-1} M Sigma, C = D F^{-1} (m (x) M Sigma) (Sec. 4's FPSA-preconditioned
 * GMRES). MIXED runs every method inside FP64 iterative refinement of psi: SI and
 * FPSA as inner_iterations FP32 iterations, GMRES as one FP32 GMRES(m) solve of the
 * moment correction equation per refinement step (GMRES-IR) plus one sweep for the
 * angular correction; GMRES with phi0 is FPSA_ENOTSUP in FP64.
 * phi: output [R][sumK][2][L+1]; phi0: optional initial moments, same layout
 * (NULL = zero). Both pointers are of kind mem. stats may be NULL.
 * Returns FPSA_ENOTCONV (with phi holding the last iterate) if max_iterations
 * is reached. */
int fpsa_solve(fpsa_ctx *ctx, const fpsa_opts *opts, double *phi, const double *phi0,
               int32_t mem, fpsa_stats *stats);

/* Solve the problems of n contexts together as ONE launch of a CUDA graph: the
 * Batching pattern, where slabs of different orders N (one context per (N, L)
 * group) are solved at once. Every context must be MIXED precision, on the same
 * device, after a successful fpsa_set_xs; methods SI or FPSA (Eqs. trsi; predict,
 * correct, iterate). The graph holds, per context, the start of its FP64
 * refinement (zero state, first residual) and a device-side while loop whose body
 * is one refinement step (inner_iterations FP32 iterations, default 4, the FP64
 * accumulation and residual) and whose test is the stopping rule of fpsa_solve
 * (relative change of phi_0 below tol, or max_iterations refinement steps, or a
 * bounded wait that ran out, or a non-finite change), evaluated on the GPU; the
 * contexts' loops are independent branches of the graph and run concurrently. The
 * inner iteration count is fixed (fpsa_solve shortens the confirming step to one
 * inner iteration), so a context may take one step more than fpsa_solve would;
 * the iterates differ by rounding order only. The kernels are launched without
 * programmatic dependent launch inside the graph. phi[i]: output [R][sumK][2][L+1]
 * of context i, of kind mem (no phi0: every solve starts from zero). stats: NULL
 * or an array of n (solve_ms is the wall time of the whole call). The graph is
 * built, run and destroyed inside the call; it allocates a stream and the graph.
 * Returns the first failing status (each stats[i].status tells which), FPSA_ENOTSUP
 * if this CUDA driver refuses the graph (e.g. a conditional node). Contexts must not
 * be used by other threads during the call. */
int fpsa_solve_batch(fpsa_ctx *const *ctxs, int32_t n, const fpsa_opts *opts, double *const *phi,
                     int32_t mem, fpsa_stats *stats);

/* Sensitivities of an objective J of the converged solution with respect to every
 * per-cell sigma_t and sigma_s,l, by implicit differentiation of the discrete
 * fixed point (the paper has no adjoint; the system is Eq. trop in LD / S_N form,
 * A psi = b with A = L_h - S_h). No iteration history is used: A^T lambda = dJ/dpsi
 * is solved through the identity A^T = W Pi A Pi W^{-1} (W = diag(w_n) per node,
 * Pi = ordinate reversal; the transposed upwind sweep of mu is the sweep of -mu and
 * S, MPD and WFD are w-self-adjoint and reversal-symmetric), i.e. as the forward
 * FPSA iteration A x = Pi W^{-1} dJ/dpsi with the same factors (reverse-direction
 * sweeps and transposed FP corrections in the original ordinates), then
 *   dJ/dsigma_t,g   = -sum_{a,b} m_ab sum_{l<N} (2l+1)/2 (-1)^l x_{l,a} phi_{l,b}
 *   dJ/dsigma_s,l,g = +sum_{a,b} m_ab (2l+1)/2 (-1)^l x_{l,a} phi_{l,b}
 * with m = (h_g/6)[[2,1],[1,2]], summed over right-hand sides.
 * Requires the last fpsa_solve since fpsa_set_xs to have returned FPSA_OK
 * (FPSA_ESTATE otherwise); its moments are kept by the context.
 *   opts:        iteration settings of the adjoint solve (NULL: FPSA, tol 1e-12)
 *   dJ_dphi:     NULL -> J = sum over rhs and instances of the right-boundary exit
 *                current sum_{mu_n>0} w_n mu_n psi_n(z_1); else the vector-Jacobian
 *                product with dJ_dphi [R][sumK][2][L+1]
 *   dJ_dsigma_t: output [sumK]; dJ_dsigma_s: output [sumK][L+1]
 *   J:           optional output [R][B], the exit currents of the forward solution
 * All array pointers are of kind mem. Returns FPSA_ENOTCONV if the adjoint solve
 * does not converge. */
int fpsa_adjoint(fpsa_ctx *ctx, const fpsa_opts *opts, const double *dJ_dphi, double *dJ_dsigma_t,
                 double *dJ_dsigma_s, double *J, int32_t mem, fpsa_stats *stats);

/* ---------------------------------------------------------------------------
 * Launch shapes and their autotuner. The paper has no counterpart: these choose
 * how the kernels of one iteration are laid out on the GPU, never what they
 * compute (every shape gives the same iterates up to rounding order). A zero
 * field means the library's own choice.
 */
typedef struct {
    int32_t sweep_cells_per_thread; /* transport sweep: consecutive cells a lane carries
                                       (a segment is 8 such chunks); at least the library's
                                       choice for the context (its smallest: that bounds the
                                       segment maps it allocated), at most 1 << 20 */
    int32_t solve_blocks_per_sm;    /* BCR solve: resident blocks per SM of its cooperative
                                       grid, 1..4 (capped by the kernel's occupancy) */
    int32_t solve_max_slices;       /* BCR solve: most row slices one block-row of a level is
                                       split into, 1, 2 or 4 */
    int32_t factor_engine;          /* BCR factorization of the next fpsa_set_xs: 1 = SIMT
                                       Gauss-Jordan (and SIMT block GEMMs), 2 = tensor cores
                                       (only for FP32 factors (MIXED), else FPSA_ENOTSUP:
                                       2N = 128, blocked Gauss-Jordan with tcgen05 trailing
                                       updates in split BF16; 2N = 256 or 512, the recursive
                                       block inversion's h x h products as tcgen05 split-BF16
                                       GEMMs, its 128 x 128 leaves by Gauss-Jordan); 0 = tensor
                                       cores where they apply, else SIMT. Factors differ by
                                       rounding only (the pivots are chosen in FP32 either
                                       way) */
    int32_t solve_engine;           /* BCR solve (the FP solve of every iteration; the
                                       factorization itself is unchanged): 1 = the dataflow
                                       solve on the FP32/FP64 cores (right-hand sides 8 at a
                                       time), 2 = tensor cores (each unit one split-BF16 tcgen05
                                       GEMM of A^{-1} by 64 right-hand sides, so every factor
                                       is read once per 64 of them; only for FP32 factors
                                       (MIXED) with 2N a multiple of 128 up to 512 and at least
                                       16 right-hand sides, else FPSA_ENOTSUP; such a context
                                       keeps a second, split copy of its factors, the same
                                       size as the FP32 ones); 0 = tensor cores where they
                                       apply, else the dataflow solve. Solutions differ by
                                       rounding only */
    int32_t residual_engine;        /* MIXED, the FP64 refinement residual's two contractions
                                       (phi = D psi, s = M (Sigma phi + Q)): 1 = FP64 FMA
                                       cores, 2 = tensor cores computing them exactly at FP64
                                       working accuracy (each column and operator row as a
                                       56-bit fixed-point number in eight balanced
                                       base-128 digits, each exact in BF16; the 36
                                       digit-pair products summed exactly in
                                       FP32 and recombined in FP64; N a multiple of 32 up to
                                       256, else FPSA_ENOTSUP); 0 = tensor cores where they
                                       apply, else FP64 cores. Results differ by rounding
                                       only */
} fpsa_tuning;

/* The shapes in effect (zero fields resolved to the values used). */
int fpsa_get_tuning(const fpsa_ctx *ctx, fpsa_tuning *out);

/* Request shapes for the following solves (t == NULL: all library choices).
 * sweep_cells_per_thread below the context's smallest is raised to it and
 * solve_blocks_per_sm above the occupancy is lowered to it; other values out of
 * the ranges above return FPSA_EINVAL and leave the shapes unchanged. */
int fpsa_set_tuning(fpsa_ctx *ctx, const fpsa_tuning *t);

/* Time fpsa_solve(ctx, opts, ...) on the loaded cross sections for candidate
 * shapes and keep the fastest: first every (solve_blocks_per_sm, solve_max_slices)
 * pair with the library's sweep shape, then sweep_cells_per_thread = c, 2c, 4c, 8c
 * (c the smallest; while the segments per slab still drop) with that solve
 * shape. Each candidate is solved once untimed and then `repeats` times (>= 1)
 * between CUDA events on the context stream; its time is the fastest of those.
 * best (may be NULL) receives the chosen shapes, best_ms (may be NULL) their time
 * in milliseconds. Requires fpsa_set_xs (FPSA_ESTATE). Any status other than
 * FPSA_OK from a trial solve ends the search, restores the shapes held before the
 * call and is returned. Afterwards the context is as after an fpsa_solve (its
 * moments are kept for fpsa_adjoint). */
int fpsa_autotune(fpsa_ctx *ctx, const fpsa_opts *opts, int32_t repeats, fpsa_tuning *best, double *best_ms);

/* The S_N tables a context builds, for N = n_ordinates and L = n_moments - 1
 * (same limits as fpsa_create), host-side only (no CUDA call; Sec. 2.2):
 *   mu [N], w [N]   Gauss-Legendre ordinates (ascending) and weights: the roots of
 *                   P_N and 2 / ((1 - mu^2) P_N'(mu)^2)
 *   D  [L+1][N]     D[l][n] = w_n P_l(mu_n)            (Eq. phi-mom)
 *   M  [N][L+1]     M[n][l] = (2l+1)/2 P_l(mu_n)       (Eq. treq)
 *   A  [N][N]       the angular Laplacian: MPD F = M diag(-l(l+1)) D over l < N
 *                   (Eq. fp-mpd) or WFD W (Eq. w_wfd), per `laplacian`
 * Every output is a caller-owned host array; any may be NULL (not written).
 * Returns FPSA_EINVAL for N odd, < 2 or > FPSA_MAX_ORDINATES, n_moments outside
 * [1, N] or an unknown laplacian. */
int fpsa_tables(int32_t n_ordinates, int32_t n_moments, int32_t laplacian, double *mu, double *w, double *D,
                double *M, double *A);

/* Limits of the failure checks, for callers that need the error paths to fire on
 * ordinary inputs (tests of FPSA_ETIMEOUT and FPSA_EPIVOT handling; the paper has no
 * counterpart). wait_polls: how many times a polling thread of the BCR dataflow
 * kernels (the factorization of fpsa_set_xs and the solve of every iteration) tests
 * a counter it waits on before it gives up, records the failure and goes on with
 * the data it has; the call then returns FPSA_ETIMEOUT (its results are not valid).
 * growth_limit: fpsa_set_xs returns FPSA_EPIVOT when the pivot growth
 * max|A| max|A^{-1}| of an eliminated block (fpsa_stats.pivot_growth) exceeds it.
 * 0 restores each default (2^25 polls, about a second; growth 1e14). A context
 * whose call returned FPSA_ETIMEOUT or FPSA_EPIVOT stays usable: after
 * fpsa_set_xs failed, call it again (fpsa_solve needs a successful one); after
 * fpsa_solve failed, solve again. Waits on copies and tensor-core completions are
 * bounded by time (2 s) and not affected. Negative values return FPSA_EINVAL. */
int fpsa_set_limits(fpsa_ctx *ctx, int64_t wait_polls, double growth_limit);

/* Release every device buffer of the context (NULL is allowed). */
void fpsa_destroy(fpsa_ctx *ctx);

/* Static text for a status code. */
const char *fpsa_strerror(int code);

/* Message of the last failing call on ctx ("" if none); valid until the next call.
 * With ctx == NULL: why the last fpsa_create on this thread failed in a CUDA call
 * ("" after a successful create or an argument error). */
const char *fpsa_last_error(const fpsa_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Allocation-free transport sweep. The paper has no counterpart: this is a
 * service entry point for callers that cannot call cudaMalloc -- code running
 * inside another framework's memory pool or under its allocator lock, or a
 * process whose device memory is reserved up front.
 *
 * Computes one LD upwind sweep psi = L^{-1} q (the transport operator
 * mu d/dz + sigma_t in the LD discretization above, zero incoming flux at both
 * edges) for ONE slab of n_cells cells and n_ordinates Gauss-Legendre ordinates.
 * All five array pointers are DEVICE memory owned by the caller:
 *   h [K], sigma_t [K]          cell widths and total cross sections
 *   q [K][2][N]                 nodal ANGULAR source (values at the ordinates)
 *   psi [K][2][N]               output angular flux
 * The per-(cell, ordinate) coefficient scratch lives in a fixed __device__
 * array of FPSA_SWEEP_NOALLOC_MAX_CELL_ANGLES x 6 doubles (6.3 MB) that every GPU
 * loading the library holds until the process exits; no call allocates device
 * memory. K * N above that limit, or N > 256, returns FPSA_ENOTSUP; malformed
 * arguments return FPSA_EINVAL; a refused launch returns FPSA_ECUDA (the launch's
 * own status: an error left pending by earlier, unrelated work is not cleared).
 * Work is enqueued on `stream` (cudaStream_t, NULL = legacy default) and the
 * call returns without synchronising. The first call on a device does a one-time
 * set-up with that device current: it looks up the arrays' device addresses and
 * copies the ordinate tables of every even N <= 256 into a second fixed array
 * (a synchronous copy); make that first call before any stream capture. Later
 * calls copy nothing from host memory. All calls share the one scratch array and
 * leave their coefficients in it (each call rewrites every coefficient it reads
 * before the sweep): calls whose work overlaps on the GPU (e.g. on two streams)
 * race and must be serialised by the caller.
 */
#define FPSA_SWEEP_NOALLOC_MAX_CELL_ANGLES 131072
int fpsa_sweep_noalloc(int32_t n_ordinates, int32_t n_cells, const double *h, const double *sigma_t,
                       const double *q, double *psi, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FPSA_H */
