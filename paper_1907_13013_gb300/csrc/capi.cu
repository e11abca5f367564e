// C ABI and host driver of the FPSA library (declarations and contracts in include/fpsa.h).
//
// One FPSA source iteration (Eqs. predict, correct, iterate of arXiv:1907.13013)
// is, per sweep, the launch sequence
//   k_sweep            psi^{m+1/2} = L^{-1} q                      (LD upwind sweep)
//   k_fp_rhs           phi^{m+1/2} = D psi^{m+1/2};  rhs = m (x) M Sigma (phi^{m+1/2} - phi^m)
//   k_bcr_solve_flow   upsilon = F^{-1} rhs (all reduction levels in one cooperative launch)
//   k_update_scatter   phi^{m+1} = phi^{m+1/2} + D upsilon; q = M (Sigma phi^{m+1} + Q)
// with the convergence maxima of Eq. iterate accumulated in k_update_scatter.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fpsa_internal.h"
#include "kernels.cuh"
#include "tc_contract.cuh"
#include "bcr_large.cuh"
#include "bgemm_tc.cuh"
#include "residual_tc.cuh"
#include "bcr_factor_tc.cuh"
#include "bcr_solve_tc.cuh"
#include "gmres.cuh"

using namespace fpsa;

namespace {

// segmented sweep: cells per thread (at least 4) so that no slab needs more than
// kSegMax segments of kSegWarps * cpt cells
inline int sweep_cells_per_thread(const Geometry &g) {
    const int per = kSegMax * kSegWarps;
    return std::max(4, (g.Kmax + per - 1) / per);
}
inline int sweep_segments(const Geometry &g) {
    const int len = kSegWarps * sweep_cells_per_thread(g);
    return (g.Kmax + len - 1) / len;
}
constexpr int kContractThreads = 256;
constexpr int kInvertThreads = 512;
constexpr int kSolveThreads = 256;  // one (item, rhs) unit per block (the staged solve: its compute groups' threads)

template <typename T>
struct PathBuffers {
    T *DT = nullptr, *MT = nullptr;          // D^T [n][l], M^T [l][n]
    T *sigma_s = nullptr;                    // [sumK][N] (zero for l >= L+1)
    T *Q = nullptr;                          // [R][sumK][2][N]
    T *coef = nullptr;                       // [sumK][6][N]
    T *A = nullptr, *Bc = nullptr, *Cc = nullptr;
    T *phi = nullptr, *phi_half = nullptr, *q = nullptr, *psi = nullptr, *rhs = nullptr;
    T *qang = nullptr;                       // MIXED inner path: nodal residual source [R][sumK][2][N]
    T *ybuf = nullptr;                       // BCR solve: intermediate y, then the solution [R][sumK][2N]
    T *cmap = nullptr, *smap = nullptr;      // segmented sweep: chunk and segment maps (k_sweep_maps)
    T *G = nullptr;                          // coarse step of the BCR solve: inverse of the coarse system [n][n]
    // recursive block inversion (2N too large for one CTA): per-depth scratch X, Y
    std::vector<T *> inv_scratch;
    double *inv_amax = nullptr;
};

}  // namespace

constexpr double kGrowthLimit = 1e14;  // default pivot-growth limit of the FP block factorization

struct fpsa_ctx {
    Geometry geo;
    Tables tab;
    int laplacian = 0, precision = 0, device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    bool xs_ready = false;
    double setup_ms = 0.0, pivot_growth = 0.0;
    std::vector<void *> allocs;

    int32_t *d_off = nullptr, *d_K = nullptr, *d_cell_inst = nullptr, *d_slot_base = nullptr;
    int32_t *d_bc = nullptr;     // [B][2] edge conditions; NULL when every edge is vacuum
    double *d_in_st = nullptr, *d_in_ss = nullptr, *d_in_q = nullptr;  // fpsa_set_xs staging of host inputs
    int *d_xs_err = nullptr;     // [2] validation of fpsa_set_xs
    // BCR solve dataflow counters, double-buffered: [parity][cnt | done][rhs chunks][sumK];
    // each solve uses one parity and zeroes the other for the next solve
    int *d_flow = nullptr;
    size_t flow_n = 0;                      // counters per array (rhs chunks x sumK)
    int flow_parity = 0;
    bool solve_pdl = true;                  // cooperative launch with programmatic serialization accepted
    int *d_factor_cnt = nullptr;            // dataflow factorization counters [sumK]
    double *d_inc = nullptr;     // [R][B][2][N] given incoming edge fluxes (FP64)
    bool has_inc = false;
    float *d_Afp32 = nullptr, *d_mu32 = nullptr;  // angular Laplacian and mu rounded to FP32 (FP32 assembly)
    double *d_mu = nullptr, *d_Afp = nullptr, *d_h = nullptr, *d_sigma_t = nullptr, *d_s0 = nullptr,
           *d_s1 = nullptr;
    std::vector<BcrItem *> d_levels;
    BcrItem *d_roots = nullptr;
    BcrItem *d_items_all = nullptr;  // levels concatenated, then roots (cooperative solve)
    LevelTable lvt[2] = {};          // per element type (row slicing depends on the vector width)
    int coop_grid[2] = {0, 0};       // cooperative BCR solve grid for float [0] / double [1]
    int solve_per_sm[2] = {0, 0};    // resident blocks per SM of the cooperative BCR solve (occupancy)
    int n_sm = 0;
    int sweep_cpt = 0;               // cells per thread of the segmented sweep in effect
    fpsa_tuning tuning = {};         // requested launch shapes (0: the library's choice)
    int factor_grid[2] = {0, 0};     // cooperative dataflow factorization grid (0: per-level launches)
    int factor_tc_grid = 0;          // grid of the tensor-core factorization (FP32, 2N = 128), 0: unavailable
    bool bgemm_tc_able = false;      // FP32, 2N = 256 or 512: recursive inversion's GEMMs on tensor cores
    unsigned char *d_res_ops = nullptr;  // MIXED: digit slices of D and M, then their row exponents
    rtc::Ops res_ops = {};               // (NULL D: the tensor-core residual does not apply)
    // tensor-core BCR solve (FP32 factors, 2N a multiple of 128 up to 512, R >= 16)
    int tcs_rt = 0;                  // right-hand sides per unit; 0: unavailable
    int tcs_grid = 0;                // two CTAs per SM
    unsigned char *d_tcs_A = nullptr;  // the factors split to BF16 hi / lo in the core-matrix layout
    float *d_tcs_g = nullptr;        // per-CTA backward coupling vectors
    int *d_tcs_queue = nullptr;      // unit counters, one per parity of d_flow
    unsigned long long *d_conv = nullptr, *d_growth = nullptr;
    int *d_status = nullptr;
    double *d_result = nullptr;
    int *d_steps = nullptr;      // refinement steps taken by a batch graph's loop
    cudaEvent_t ad_ev[4] = {};   // MIXED: first residual and first inner step, timed once per solve
    double *h_result = nullptr;  // pinned

    // adjoint
    bool fwd_ready = false;      // d_phi_fwd holds the last converged forward moments
    double *d_phi_fwd = nullptr, *d_adj_src = nullptr, *d_gphi = nullptr;  // [R][sumK][2][N]
    double *d_Pm = nullptr, *d_cJ = nullptr;                              // (-1)^l P_l(mu_n), exit-current weights
    double *d_J = nullptr, *d_grad_t = nullptr, *d_grad_s = nullptr;

    // GMRES: Krylov basis and work vectors (double for FP64 contexts, float for the
    // inner solves of MIXED), allocated at first use
    int gm_restart = 0;
    unsigned char *gm_V = nullptr, *gm_u = nullptr, *gm_w = nullptr, *gm_b = nullptr;
    double *gm_partial = nullptr, *gm_dots = nullptr, *gm_coef = nullptr, *gm_alpha = nullptr;
    long long *gm_seg_begin = nullptr, *gm_seg_end = nullptr;
    int gm_nchunks = 0;

    PathBuffers<double> p64;  // FP64 path; for MIXED: FP64 tables, psi (refined iterate), phi
    PathBuffers<float> p32;   // MIXED: the FP32 inner FPSA solve
    // tensor-core contractions of the FP32 inner solve
    bool tc_able = false;               // N multiple of 16, 16 <= N <= 128, or tc_big
    bool tc_big = false;                // N multiple of 32 in (128, 256]: operators streamed
    bool gm_use_tc = false;             // this solve's GMRES contractions on tensor cores (MIXED)
    unsigned char *d_tc_ops = nullptr;  // D_hi, D_lo, M_hi, M_lo (BF16, core-matrix layout)
    // [0]: a bounded device wait ran out (tensor-core or BCR dataflow); [1]: the polls a
    // BCR dataflow wait makes before it gives up (fpsa_set_limits)
    int *d_dev_err = nullptr, *h_flag = nullptr;
    double growth_limit = kGrowthLimit;  // fpsa_set_xs: FPSA_EPIVOT above this pivot growth
    int tc_grid = 0;

    // built-in profiler: launch counters (always) and event pairs (when on)
    bool prof_on = false;
    int64_t launches[FPSA_N_PHASES] = {};
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_rec;  // (phase, index of start event)
    size_t ev_used = 0;
};

namespace {

thread_local std::string g_create_error;  // why the last fpsa_create on this thread failed

// The dynamic shared-memory limit of a kernel is process-wide state, while
// contexts with different N (possibly on different host threads) need different
// sizes: only ever raise it, under a lock, so no context lowers another's.
std::mutex g_attr_mutex;
std::map<std::pair<const void *, int>, int> g_attr_max;

cudaError_t raise_smem_limit(const void *func, int bytes) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    int &cur = g_attr_max[{func, dev}];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// Launch bracket: counts every launch of a kernel class and, while profiling is
// on, records a CUDA event pair around it on the context stream.
struct Launch {
    fpsa_ctx *c;
    int phase;
    Launch(fpsa_ctx *ctx, int ph) : c(ctx), phase(ph) {
        c->launches[ph]++;
        if (!c->prof_on) return;
        if (c->ev_used + 2 > c->ev_pool.size())
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                c->ev_pool.push_back(e);
            }
        c->ev_rec.push_back({ph, (int)c->ev_used});
        cudaEventRecord(c->ev_pool[c->ev_used], c->stream);
        c->ev_used += 2;
    }
    ~Launch() {
        if (c->prof_on) cudaEventRecord(c->ev_pool[c->ev_rec.back().second + 1], c->stream);
    }
};

int fail(fpsa_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? FPSA_ENOMEM : FPSA_ECUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

template <typename P>
cudaError_t dalloc(fpsa_ctx *ctx, P **p, size_t count) {
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(P));
    if (e != cudaSuccess) return e;
    ctx->allocs.push_back(v);
    *p = static_cast<P *>(v);
    return cudaSuccess;
}

template <typename T>
size_t contract_smem(int N) { return 2 * 2 * (size_t)kContractCells * N * sizeof(T); }

// shared memory of the Schur update kernel: X and two staged operands, (N/2)^2 each,
// or X alone when staging does not fit
template <typename T>
bool schur_staged(int N) { return (size_t)3 * (N / 2) * (N / 2) * sizeof(T) <= 227 * 1024 - 1024; }
template <typename T>
size_t schur_smem(int N) { return (size_t)(schur_staged<T>(N) ? 3 : 1) * (N / 2) * (N / 2) * sizeof(T); }

// usable dynamic shared memory per CTA (227 KB opt-in, less room for static shared memory)
constexpr size_t kSmemLimit = 227 * 1024 - 1024;

// columns of the coarse inverse per block of k_bcr_coarse_inverse, and its shared memory
constexpr int kCoarseCols = 16;
size_t coarse_inverse_smem_bytes(int N, int m, int esize) {
    return esize == 8 ? coarse_inverse_values<double>(N, m, kCoarseCols) * 8 : coarse_inverse_values<float>(N, m, kCoarseCols) * 4;
}
template <typename T>
size_t coarse_inverse_smem(int N, const LevelTable &lv) {
    return coarse_inverse_values<T>(N, lv.coarse_m, kCoarseCols) * sizeof(T);
}

// Coarse step of the staged BCR solve (one instance, one right-hand side): the
// lowest level c whose coarse cells (local index a multiple of 2^c) number at most
// N/4 (so that their right-hand sides fit a coupling area), when at least two
// reduction levels lie above it; G rows per unit: the largest power of two dividing
// 2N whose rows fit the staged solve's column buffer ((2N)^2 values). Sets
// coarse_level = -1 otherwise.
void plan_coarse(LevelTable &lv, const Geometry &g, int esize) {
    lv.coarse_level = -1;
    lv.coarse_m = lv.coarse_K = lv.coarse_rpu = lv.coarse_units = 0;
    const int N = g.N, n2 = 2 * N, K = g.B == 1 ? g.sumK : 0;
    if (g.B != 1 || g.R != 1 || !bcr_slice_staged(N, esize) || !bcr_couplings_staged(N, esize)) return;
    if (n2 > 256 / (kCoarseCols / 8)) return;
    for (int c = 1; c + 2 <= g.n_levels; ++c) {
        const int m = (K + (1 << c) - 1) >> c;
        if (m > N / 4) continue;
        const int n = m * n2;
        if (n % kCoarseCols) return;
        // G rows of a unit land in the column buffer of the staged solve: (2N)^2 values
        const size_t buf = (size_t)n2 * n2 * esize;
        int rpu = 1;
        while (rpu * 2 <= n2 && n2 % (rpu * 2) == 0 && (size_t)rpu * 2 * n * esize <= buf) rpu *= 2;
        if ((size_t)rpu * n * esize > buf) return;
        if (coarse_inverse_smem_bytes(N, m, esize) > kSmemLimit) return;
        lv.coarse_level = c;
        lv.coarse_m = m;
        lv.coarse_K = K;
        lv.coarse_rpu = rpu;
        lv.coarse_units = n / rpu;
        return;
    }
}

// right-hand sides per BCR solve unit
int solve_rc(int R) { return R >= 8 ? 8 : (R >= 4 ? 4 : (R >= 2 ? 2 : 1)); }

// copy stages of the staged-slice BCR solve: as many as fit one block's shared memory
// (at most kMaxSolveStages); 0 when the slices are not staged
template <typename T>
int solve_stages(int N, int RC) {
    if (!bcr_slice_staged(N, (int)sizeof(T))) return 0;
    const size_t base = (size_t)kSolveGroups * bcr_stage_base_values<T>(N, kSolveThreads / kSolveGroups, RC) * sizeof(T);
    const size_t stage = (size_t)bcr_stage_values<T>(N, RC) * sizeof(T);
    const int ns = (int)((kSmemLimit - base) / stage);
    return std::max(1, std::min(kMaxSolveStages, ns));
}

// shared memory of the cooperative BCR solve: the unit scratch and, when one unit's
// A^{-1} slice fits, the copy stages
template <typename T>
size_t solve_smem(int N, int RC) {
    if (bcr_slice_staged(N, (int)sizeof(T)))
        return ((size_t)kSolveGroups * bcr_stage_base_values<T>(N, kSolveThreads / kSolveGroups, RC) +
                (size_t)solve_stages<T>(N, RC) * bcr_stage_values<T>(N, RC)) *
               sizeof(T);
    return (size_t)bcr_unit_smem_values(N, kSolveThreads, VecOf<T>::V, RC, (int)sizeof(T)) * sizeof(T);
}

// threads of a cooperative BCR solve block: the staged solve adds a service warp per compute group
template <typename T>
int solve_threads(int N) {
    return bcr_slice_staged(N, (int)sizeof(T)) ? kSolveThreads + 32 * kSolveGroups : kSolveThreads;
}

template <typename T>
const void *coop_kernel(int RC, int N) {
    if (bcr_slice_staged(N, (int)sizeof(T))) {
        constexpr int NT = kSolveThreads + 32 * kSolveGroups;
        switch (RC) {
            case 8: return (const void *)k_bcr_solve_flow_s<T, NT, 8>;
            case 4: return (const void *)k_bcr_solve_flow_s<T, NT, 4>;
            case 2: return (const void *)k_bcr_solve_flow_s<T, NT, 2>;
            default: return (const void *)k_bcr_solve_flow_s<T, NT, 1>;
        }
    }
    switch (RC) {
        case 8: return (const void *)k_bcr_solve_flow<T, kSolveThreads, 8>;
        case 4: return (const void *)k_bcr_solve_flow<T, kSolveThreads, 4>;
        case 2: return (const void *)k_bcr_solve_flow<T, kSolveThreads, 2>;
        default: return (const void *)k_bcr_solve_flow<T, kSolveThreads, 1>;
    }
}

// the tensor-core solve for RT right-hand sides per unit
const void *tcs_kernel(int RT) {
    switch (RT) {
        case 16: return (const void *)k_bcr_solve_tc<16>;
        case 32: return (const void *)k_bcr_solve_tc<32>;
        case 48: return (const void *)k_bcr_solve_tc<48>;
        default: return (const void *)k_bcr_solve_tc<64>;
    }
}

template <typename T>
size_t invert_smem(int N) {
    const int n2 = 2 * N;
    return ((size_t)n2 * (n2 + 1) + n2) * sizeof(T) + (size_t)n2 * sizeof(int);
}

// full: every buffer of an FPSA iteration in precision T. Otherwise only the tables,
// cross sections, sources and the psi / phi state (the FP64 side of MIXED).

// Does one CTA invert an n x n block directly (registers for n in {32, 64, 128},
// else shared memory)? (Routing 128 x 128 FP32 blocks through one block-Schur
// level with 64 x 64 leaves was measured slower: the elimination steps are
// latency bound, so halving their length does not pay for the extra GEMMs.)
template <typename T>
bool cta_invertible(int n) {
    return n == 32 || n == 64 || n == 128 || invert_smem<T>(n / 2) <= kSmemLimit;
}

template <typename T>
int alloc_path(fpsa_ctx *ctx, PathBuffers<T> &p, bool full) {
    const Geometry &g = ctx->geo;
    const size_t N = g.N, ang = (size_t)g.R * g.sumK * 2 * N;
    const int h2 = g.N / 2;
    CK(dalloc(ctx, &p.DT, N * N));
    CK(dalloc(ctx, &p.MT, N * N));
    CK(dalloc(ctx, &p.sigma_s, (size_t)g.sumK * N));
    CK(dalloc(ctx, &p.phi, ang));
    CK(dalloc(ctx, &p.psi, ang));
    {
        const int nseg = sweep_segments(g);
        CK(dalloc(ctx, &p.smap, (size_t)g.R * g.B * nseg * N * 2));
        CK(dalloc(ctx, &p.cmap, (size_t)g.R * g.B * nseg * kSegWarps * N * 2));
    }
    if (full) {
        CK(dalloc(ctx, &p.coef, (size_t)g.sumK * 6 * N));
        CK(dalloc(ctx, &p.A, (size_t)g.sumK * 4 * N * N));
        CK(dalloc(ctx, &p.Bc, (size_t)g.n_slots * h2 * h2));
        CK(dalloc(ctx, &p.Cc, (size_t)g.n_slots * h2 * h2));
        CK(dalloc(ctx, &p.phi_half, ang));
        CK(dalloc(ctx, &p.q, ang));
        CK(dalloc(ctx, &p.rhs, ang));
        CK(dalloc(ctx, &p.ybuf, ang));

        const LevelTable &lvp = ctx->lvt[sizeof(T) == 8 ? 1 : 0];
        if (lvp.coarse_level >= 0) {
            const size_t n = (size_t)lvp.coarse_m * 2 * N;
            CK(dalloc(ctx, &p.G, n * n));
            CK(raise_smem_limit((const void *)k_bcr_coarse_inverse<T, kCoarseCols>, (int)coarse_inverse_smem<T>(g.N, lvp)));
        }
        // scratch of the recursive block inversion: X and Y per recursion depth
        for (int n = 2 * g.N; !cta_invertible<T>(n); n /= 2) {
            T *s = nullptr;
            CK(dalloc(ctx, &s, (size_t)2 * kLargeChunk * (n / 2) * (n / 2)));
            p.inv_scratch.push_back(s);
        }
        if (!p.inv_scratch.empty()) {
            CK(dalloc(ctx, &p.inv_amax, kLargeChunk));
            CK(raise_smem_limit((const void *)k_binv_smem_rm<T>, (int)kSmemLimit));
        }
        CK(raise_smem_limit((const void *)k_bcr_schur<T>, (int)schur_smem<T>(g.N)));
    }
    {
        const int cs = (int)contract_smem<T>(g.N);
        CK(raise_smem_limit((const void *)k_scatter<T>, cs));
        CK(raise_smem_limit((const void *)k_fp_rhs<T>, cs));
        CK(raise_smem_limit((const void *)k_update_scatter<T>, cs));
        CK(raise_smem_limit((const void *)k_expand<T>, cs));
        CK(raise_smem_limit((const void *)k_fp_rhs_moments<T>, cs));
        CK(raise_smem_limit((const void *)k_moments_axpy<T>, cs));
        if (sizeof(T) == 8)
            CK(raise_smem_limit((const void *)k_mixed_residual, cs));
    }
    if (full && ctx->precision == FPSA_PRECISION_MIXED) {
        CK(dalloc(ctx, &p.qang, ang));
    } else {
        CK(dalloc(ctx, &p.Q, ang));
    }
    std::vector<T> DT(N * N), MT(N * N);
    for (size_t l = 0; l < N; ++l)
        for (size_t n = 0; n < N; ++n) {
            DT[n * N + l] = (T)ctx->tab.D[l * N + n];
            MT[l * N + n] = (T)ctx->tab.M[n * N + l];
        }
    CK(cudaMemcpy(p.DT, DT.data(), N * N * sizeof(T), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p.MT, MT.data(), N * N * sizeof(T), cudaMemcpyHostToDevice));
    if (invert_smem<T>(g.N) <= kSmemLimit)
        CK(raise_smem_limit((const void *)k_bcr_invert<T>, (int)invert_smem<T>(g.N)));
    return FPSA_OK;
}

// Does the recursive inversion of this context run its block GEMMs on the tensor
// cores? (FP32 factors with 2N = 256 or 512, unless the SIMT engine is requested.)
bool bgemm_on_tc(const fpsa_ctx *ctx) { return ctx->bgemm_tc_able && ctx->tuning.factor_engine != 1; }

// C = alpha A B + beta C for the h x h blocks of a batch of ne items: tcgen05 split
// BF16 GEMMs for FP32 blocks with h = 128 or 256 where the context allows it, else
// the SIMT kernel.
template <typename T>
void bgemm(fpsa_ctx *ctx, int h, T alpha, BMat<T> A, BMat<T> B, T beta, BMat<T> C, const BcrItem *items, int ne) {
    cudaStream_t st = ctx->stream;
    if constexpr (sizeof(T) == sizeof(float)) {
        if (bgemm_on_tc(ctx) && (h == 128 || h == 256)) {
            if (h == 256)
                k_bgemm_tc<256><<<dim3(2, ne), bgt::kThreads, bgt::smem_bytes(256), st>>>(alpha, A, B, beta, C,
                                                                                          items, ctx->d_dev_err);
            else
                k_bgemm_tc<128><<<dim3(1, ne), bgt::kThreads, bgt::smem_bytes(128), st>>>(alpha, A, B, beta, C,
                                                                                          items, ctx->d_dev_err);
            return;
        }
    }
    const dim3 gg((h + 63) / 64, (h + 63) / 64, ne);
    k_bgemm<T><<<gg, 256, 0, st>>>(h, alpha, A, B, beta, C, items);
}

// In-place inverse (row-major) of the n x n blocks M of a batch of ne items,
// recursing by block Schur complements down to CTA-sized blocks.
template <typename T>
int invert_inplace(fpsa_ctx *ctx, PathBuffers<T> &p, BMat<T> M, int n, const BcrItem *items, int ne, int depth) {
    cudaStream_t st = ctx->stream;
    if (n == 128) {
        k_binv_reg_rm<T, 128><<<ne, 512, 0, st>>>(M, items, ctx->d_status);
    } else if (n == 64) {
        k_binv_reg_rm<T, 64><<<ne, 512, 0, st>>>(M, items, ctx->d_status);
    } else if (n == 32) {
        k_binv_reg_rm<T, 32><<<ne, 512, 0, st>>>(M, items, ctx->d_status);
    } else if (invert_smem<T>(n / 2) <= kSmemLimit) {
        k_binv_smem_rm<T><<<ne, kInvertThreads, invert_smem<T>(n / 2), st>>>(M, n, items, ctx->d_status);
    } else {
        const int h = n / 2;
        if (depth >= (int)p.inv_scratch.size()) return fail(ctx, FPSA_ENOTSUP, "block inversion scratch missing");
        const BMat<T> A11 = M.sub(0, 0), A12 = M.sub(0, h), A21 = M.sub(h, 0), A22 = M.sub(h, h);
        T *s = p.inv_scratch[depth];
        const BMat<T> X{s, (long long)h * h, h, 0}, Y{s + (size_t)kLargeChunk * h * h, (long long)h * h, h, 0};
        int rc = invert_inplace(ctx, p, A11, h, items, ne, depth + 1);  // A11 <- P
        if (rc) return rc;
        bgemm(ctx, h, T(1), A11, A12, T(0), X, items, ne);    // X = P A12
        bgemm(ctx, h, T(1), A21, A11, T(0), Y, items, ne);    // Y = A21 P
        bgemm(ctx, h, T(-1), A21, X, T(1), A22, items, ne);   // A22 <- S = A22 - A21 X
        rc = invert_inplace(ctx, p, A22, h, items, ne, depth + 1);  // A22 <- Q = S^{-1}
        if (rc) return rc;
        bgemm(ctx, h, T(-1), X, A22, T(0), A12, items, ne);   // A12 <- -X Q
        bgemm(ctx, h, T(-1), A22, Y, T(0), A21, items, ne);   // A21 <- -Q Y
        bgemm(ctx, h, T(-1), X, A21, T(1), A11, items, ne);   // A11 <- P - X A21
    }
    CK(cudaGetLastError());
    return FPSA_OK;
}

// Invert the eliminated blocks of `items` (ni of them) in place, transposed, with
// the FP64 growth check: one CTA per block when it fits, else the recursive path.
template <typename T>
// with_schur: the level's Schur updates are fused into the register-tile inversion
// kernel when it is used; *fused reports whether they were (else the caller launches
// k_bcr_schur).
int invert_level(fpsa_ctx *ctx, PathBuffers<T> &p, const BcrItem *items, int ni, bool with_schur = false,
                 bool *fused = nullptr) {
    const int N = ctx->geo.N, n2 = 2 * N;
    cudaStream_t st = ctx->stream;
    Launch L_(ctx, FPSA_PHASE_BCR_INVERT);
    const int staged = with_schur ? (schur_staged<T>(N) ? 1 : 0) : -1;
    const size_t ssm = with_schur ? schur_smem<T>(N) : 0;
    const bool reg = (n2 == 128 && cta_invertible<T>(128)) || n2 == 64 || n2 == 32;
    if (fused) *fused = reg && with_schur;
    if (n2 == 128 && cta_invertible<T>(128)) {
        k_bcr_invert_reg<T, 128><<<ni, 512, ssm, st>>>(p.A, items, ctx->d_growth, ctx->d_status, p.Bc, p.Cc, staged);
    } else if (n2 == 64) {
        k_bcr_invert_reg<T, 64><<<ni, 512, ssm, st>>>(p.A, items, ctx->d_growth, ctx->d_status, p.Bc, p.Cc, staged);
    } else if (n2 == 32) {
        k_bcr_invert_reg<T, 32><<<ni, 512, ssm, st>>>(p.A, items, ctx->d_growth, ctx->d_status, p.Bc, p.Cc, staged);
    } else if (cta_invertible<T>(n2)) {
        k_bcr_invert<T><<<ni, kInvertThreads, invert_smem<T>(ctx->geo.N), st>>>(p.A, items, n2, ctx->d_growth,
                                                                               ctx->d_status);
    } else {
        const BMat<T> M{p.A, (long long)n2 * n2, n2, 1};
        for (int c0 = 0; c0 < ni; c0 += kLargeChunk) {
            const int ne = std::min(kLargeChunk, ni - c0);
            k_bamax<T><<<ne, 256, 0, st>>>(M, n2, items + c0, p.inv_amax);
            int rc = invert_inplace(ctx, p, M, n2, items + c0, ne, 0);
            if (rc) return rc;
            k_btranspose<T><<<ne, 256, 0, st>>>(M, n2, items + c0, p.inv_amax, ctx->d_growth, ctx->d_status);
        }
    }
    CK(cudaGetLastError());
    return FPSA_OK;
}

// Tensor-core operands of the FP32 inner contractions: D and M (as FP32 values)
// split into BF16 hi / lo, stored as the B operands of Out = X Op^T in the
// K-major core-matrix layout (Op_D[l][n] = D[l][n], Op_M[n][l] = M[n][l]).
// Digit slices of D and M for the tensor-core FP64 residual (MIXED, N a multiple of 32
// up to 256): computed once on the host, layout of rtc::block_offset, exponents after.
int setup_residual_tc(fpsa_ctx *ctx) {
    const int N = ctx->geo.N;
    if (ctx->precision != FPSA_PRECISION_MIXED || !rtc::applies(N)) return FPSA_OK;
    const size_t nn = (size_t)N * N;
    const size_t sl = (size_t)(N / rtc::oc_of(N)) * (N / rtc::KC) * rtc::b_block_bytes(N);
    std::vector<unsigned char> host(2 * sl + 2 * N * sizeof(int32_t));
    std::vector<double> M(nn);  // M stored [n][l] already: rows n, K = l
    for (size_t i = 0; i < nn; ++i) M[i] = ctx->tab.M[i];
    int32_t *eD = reinterpret_cast<int32_t *>(host.data() + 2 * sl), *eM = eD + N;
    rtc::slice_operator(ctx->tab.D.data(), N, host.data(), eD);
    rtc::slice_operator(M.data(), N, host.data() + sl, eM);
    CK(dalloc(ctx, &ctx->d_res_ops, host.size()));
    CK(cudaMemcpy(ctx->d_res_ops, host.data(), host.size(), cudaMemcpyHostToDevice));
    ctx->res_ops.D = ctx->d_res_ops;
    ctx->res_ops.M = ctx->d_res_ops + sl;
    ctx->res_ops.eD = reinterpret_cast<const int32_t *>(ctx->d_res_ops + 2 * sl);
    ctx->res_ops.eM = ctx->res_ops.eD + N;
    CK(raise_smem_limit((const void *)k_mixed_residual_tc, (int)rtc::smem_bytes(N)));
    return FPSA_OK;
}

int setup_tc(fpsa_ctx *ctx) {
    const int N = ctx->geo.N;
    // N <= 128: the operators stay in shared memory; N in (128, 256], a multiple of 32:
    // they are streamed in K-chunks (chunk-major layout)
    ctx->tc_big = N > 128 && N <= 256 && N % tc::kChunkK == 0;
    ctx->tc_able = ((N % 16 == 0) && N >= 16 && N <= 128) || ctx->tc_big;
    if (!ctx->tc_able) return FPSA_OK;
    const size_t nn = (size_t)N * N;
    std::vector<__nv_bfloat16> ops(4 * nn);
    for (int o = 0; o < N; ++o)
        for (int k = 0; k < N; ++k) {
            const size_t off = (ctx->tc_big ? tc::chunk_offset(o, k, N) : tc::kmajor_offset(o, k, N)) / 2;
            const float d = (float)ctx->tab.D[(size_t)o * N + k];
            const float m = (float)ctx->tab.M[(size_t)o * N + k];
            const __nv_bfloat16 dh = __float2bfloat16_rn(d), mh = __float2bfloat16_rn(m);
            ops[off] = dh;
            ops[nn + off] = __float2bfloat16_rn(d - __bfloat162float(dh));
            ops[2 * nn + off] = mh;
            ops[3 * nn + off] = __float2bfloat16_rn(m - __bfloat162float(mh));
        }
    CK(dalloc(ctx, &ctx->d_tc_ops, 4 * nn * sizeof(__nv_bfloat16)));
    CK(cudaMemcpy(ctx->d_tc_ops, ops.data(), ops.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    if (ctx->tc_big) {
        const int smem = (int)tc::BigPlan::make(N).total;
        CK(raise_smem_limit((const void *)k_tc_fp_rhs_big, smem));
        CK(raise_smem_limit((const void *)k_tc_update_scatter_big, smem));
        CK(raise_smem_limit((const void *)k_tc_fp_rhs_moments<true>, smem));
        CK(raise_smem_limit((const void *)k_tc_moments_axpy<true>, smem));
        ctx->tc_grid = nsm;  // one CTA per SM (its shared memory)
        return FPSA_OK;
    }
    const int smem = (int)tc::Plan::make(N).total;
    CK(raise_smem_limit((const void *)k_tc_fp_rhs, smem));
    CK(raise_smem_limit((const void *)k_tc_update_scatter, smem));
    CK(raise_smem_limit((const void *)k_tc_fp_rhs_tile, smem));
    CK(raise_smem_limit((const void *)k_tc_update_scatter_tile, smem));
    CK(raise_smem_limit((const void *)k_tc_fp_rhs_moments<false>, smem));
    CK(raise_smem_limit((const void *)k_tc_moments_axpy<false>, smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_update_scatter, 128, smem));
    ctx->tc_grid = std::max(1, std::min(per_sm, 2)) * nsm;
    return FPSA_OK;
}

// Upload per-path cross sections / sources (padded to N moments); with full, also the
// sweep coefficients, the FP operator assembly and its block factorization.
// The dataflow factorization kernel for blocks of n2 x n2 (register-tiled inversion), or NULL.
template <typename T>
const void *factor_kernel(int n2) {
    if (n2 == 128 && cta_invertible<T>(128)) return (const void *)k_bcr_factor_flow<T, 128>;
    if (n2 == 64) return (const void *)k_bcr_factor_flow<T, 64>;
    if (n2 == 32) return (const void *)k_bcr_factor_flow<T, 32>;
    return nullptr;
}

template <typename T>
int setup_path(fpsa_ctx *ctx, PathBuffers<T> &p, bool full) {
    const Geometry &g = ctx->geo;
    const int N = g.N, h2 = N / 2;
    cudaStream_t st = ctx->stream;
    if (!full) return FPSA_OK;
    {
        const size_t tot = (size_t)g.sumK * N;
        {
            Launch L_(ctx, FPSA_PHASE_ASSEMBLE);
            k_sweep_coef<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(ctx->d_mu, ctx->d_h, ctx->d_sigma_t, N,
                                                                            g.sumK, p.coef);
        }
        CK(cudaGetLastError());
    }
    CK(cudaMemsetAsync(p.Bc, 0, (size_t)g.n_slots * h2 * h2 * sizeof(T), st));
    CK(cudaMemsetAsync(p.Cc, 0, (size_t)g.n_slots * h2 * h2 * sizeof(T), st));
    {
        Launch L_(ctx, FPSA_PHASE_ASSEMBLE);
        const T *afp, *muT;
        if constexpr (sizeof(T) == sizeof(double)) {
            afp = ctx->d_Afp;
            muT = ctx->d_mu;
        } else {
            afp = ctx->d_Afp32;
            muT = ctx->d_mu32;
        }
        k_fp_assemble<T><<<g.sumK, dim3(32, 8), 0, st>>>(muT, afp, ctx->d_h, ctx->d_sigma_t, ctx->d_s0, ctx->d_s1,
                                                 ctx->d_cell_inst, ctx->d_off, ctx->d_K, ctx->d_slot_base, N, p.A, p.Bc,
                                                 p.Cc, ctx->d_bc);
    }
    CK(cudaGetLastError());
    const int e = sizeof(T) == 8 ? 1 : 0;
    const bool tc_factor = e == 0 && ctx->factor_tc_grid > 0 && ctx->tuning.factor_engine != 1;
    if (tc_factor) {
        // every level and the roots in one cooperative launch, inversions on tensor cores
        const LevelTable &lv = ctx->lvt[e];
        float *A = reinterpret_cast<float *>(p.A), *Bc = reinterpret_cast<float *>(p.Bc),
              *Cc = reinterpret_cast<float *>(p.Cc);
        const BcrItem *items = ctx->d_items_all;
        int n_items = lv.off[g.n_levels] + lv.n_roots;
        unsigned long long *growth = ctx->d_growth;
        int *status = ctx->d_status, *cnt = ctx->d_factor_cnt, *err = ctx->d_dev_err;
        int *queue = ctx->d_factor_cnt + g.sumK;  // the work queue's next item
        CK(cudaMemsetAsync(cnt, 0, ((size_t)g.sumK + 1) * sizeof(int), st));
        Launch L_(ctx, FPSA_PHASE_BCR_INVERT);
        k_bcr_factor_tc<<<ctx->factor_tc_grid, tcf::kThreads, tcf::Smem::total, st>>>(A, items, n_items, Bc, Cc,
                                                                                    growth, status, cnt, err, queue);
    } else if (ctx->factor_grid[e] > 0) {
        // every level and the roots in one cooperative launch (dataflow between items)
        const LevelTable &lv = ctx->lvt[e];
        T *A = p.A, *Bc = p.Bc, *Cc = p.Cc;
        const BcrItem *items = ctx->d_items_all;
        int n_items = lv.off[g.n_levels] + lv.n_roots;
        unsigned long long *growth = ctx->d_growth;
        int *status = ctx->d_status, *cnt = ctx->d_factor_cnt, *err = ctx->d_dev_err;
        int staged = schur_staged<T>(N) ? 1 : 0;
        void *args[] = {(void *)&A,      (void *)&items,  (void *)&n_items, (void *)&Bc,  (void *)&Cc,
                        (void *)&growth, (void *)&status, (void *)&cnt,     (void *)&err, (void *)&staged};
        CK(cudaMemsetAsync(cnt, 0, (size_t)g.sumK * sizeof(int), st));
        Launch L_(ctx, FPSA_PHASE_BCR_INVERT);
        CK(cudaLaunchCooperativeKernel(factor_kernel<T>(2 * N), dim3(ctx->factor_grid[e]), dim3(512), args,
                                       schur_smem<T>(N), st));
    }
    for (int l = 0; l < g.n_levels && ctx->factor_grid[e] == 0 && !tc_factor; ++l) {
        const int ni = (int)g.levels[l].size();
        if (!ni) continue;
        bool fused = false;
        int rc = invert_level(ctx, p, ctx->d_levels[l], ni, true, &fused);
        if (rc) return rc;
        CK(cudaGetLastError());
        if (!fused) {
            Launch L_(ctx, FPSA_PHASE_BCR_SCHUR);
            k_bcr_schur<T><<<ni, 256, schur_smem<T>(N), st>>>(p.A, p.Bc, p.Cc, ctx->d_levels[l], N,
                                                              schur_staged<T>(N) ? 1 : 0);
        }
        CK(cudaGetLastError());
    }
    if (ctx->factor_grid[e] == 0 && !tc_factor) {
        int rc = invert_level(ctx, p, ctx->d_roots, g.B);
        if (rc) return rc;
    }
    CK(cudaGetLastError());
    if (e == 0 && ctx->d_tcs_A) {  // the factors once more, split for the tensor-core solve
        Launch L_(ctx, FPSA_PHASE_BCR_INVERT);
        tcs::k_bcr_factor_split<<<(unsigned)((size_t)g.sumK * (2 * N / tcs::kK)), 256, 0, st>>>(
            reinterpret_cast<const float *>(p.A), ctx->d_tcs_A, 2 * N);
        CK(cudaGetLastError());
    }
    if (p.G) {
        const LevelTable &lv = ctx->lvt[sizeof(T) == 8 ? 1 : 0];
        const int n = lv.coarse_m * 2 * N;
        Launch L_(ctx, FPSA_PHASE_BCR_INVERT);
        k_bcr_coarse_inverse<T, kCoarseCols><<<n / kCoarseCols, 256, coarse_inverse_smem<T>(N, lv), st>>>(
            p.A, p.Bc, p.Cc, ctx->d_items_all, lv, N, p.G, ctx->d_dev_err);
        CK(cudaGetLastError());
    }
    return FPSA_OK;
}

// Set while a batch graph is captured on this thread: kernels are launched without the
// programmatic-dependent-launch attribute (plain graph edges between them).
thread_local bool g_plain_launch = false;

// Launch with programmatic dependent launch allowed: the kernel's blocks may be
// scheduled while the previous kernel in the stream drains, and the kernel waits
// for it (griddepcontrol.wait, before touching its outputs or overwriting its
// inputs), so launch latency and the kernel's own prologue overlap the tail.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = g_plain_launch ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// psi = L^{-1} q for every (ordinate, instance, rhs) with the given incoming edge
// fluxes inc (NULL: none): the segmented sweep (chunk / segment maps, then the
// re-sweep from each segment's inflow; reflective edges take their whole-slab maps
// from the segment maps).
template <typename T>
int sweep(fpsa_ctx *ctx, PathBuffers<T> &p, const T *q, T *psi, const T *inc) {
    const Geometry &g = ctx->geo;
    const int cpt = ctx->sweep_cpt, nseg = (g.Kmax + kSegWarps * cpt - 1) / (kSegWarps * cpt);
    const dim3 grid(2 * ((g.N / 2 + 31) / 32), nseg, g.R * g.B);
    {
        Launch L_(ctx, FPSA_PHASE_SWEEP);
        CK(launch_pdl(k_sweep_maps<T>, grid, dim3(kSegWarps * 32), 0, ctx->stream, q, (const T *)p.coef, ctx->d_off,
                      ctx->d_K, g.N, g.sumK, g.B, cpt, nseg, p.cmap, p.smap));
    }
    {
        Launch L_(ctx, FPSA_PHASE_SWEEP);
        CK(launch_pdl(k_sweep_apply<T>, grid, dim3(kSegWarps * 32), 0, ctx->stream, q, psi, (const T *)p.coef,
                      ctx->d_off, ctx->d_K, g.N, g.sumK, g.B, cpt, nseg, (const T *)p.cmap, (const T *)p.smap, inc,
                      (const int32_t *)ctx->d_bc));
    }
    CK(cudaGetLastError());
    return FPSA_OK;
}

// Launch shape of the cooperative BCR solve from the requested tuning: the grid
// (resident blocks per SM, at most the occupancy and 4 by default, times the SMs)
// and the row slices per item at each level: an item's 2N rows (in vectors of V)
// are split into S in {1, 2, 4} slices (quadrant-aligned) of >= 2 vectors while the
// level's units still fit in one pass of the grid, S at most the requested cap.
// The coarse-step plan does not depend on either.
void plan_solve_shape(fpsa_ctx *ctx) {
    const Geometry &g = ctx->geo;
    const int RC = solve_rc(g.R), nchunk = (g.R + RC - 1) / RC;
    const int bpsm = ctx->tuning.solve_blocks_per_sm > 0 ? ctx->tuning.solve_blocks_per_sm : 4;
    const int smax = ctx->tuning.solve_max_slices > 0 ? ctx->tuning.solve_max_slices : 4;
    for (int e = 0; e < 2; ++e) {
        ctx->coop_grid[e] = std::min(bpsm, ctx->solve_per_sm[e]) * ctx->n_sm;
        const int V = e ? VecOf<double>::V : VecOf<float>::V;
        const int vecs = 2 * g.N / V;
        LevelTable &lv = ctx->lvt[e];
        for (int l = 0; l <= g.n_levels; ++l) {
            const int items = l < g.n_levels ? (int)g.levels[l].size() : g.B;
            int S = 1;
            while (2 * S <= smax && vecs % (2 * S) == 0 && vecs / (2 * S) >= 2 &&
                   (long long)items * nchunk * 2 * S <= ctx->coop_grid[e])
                S *= 2;
            lv.slices[l] = S;
        }
    }
}

// F u = rhs by block cyclic reduction over the stored factors: one cooperative
// launch (forward levels, roots, backward levels); the solution is left in p.ybuf.
// No memset precedes it (its counters were zeroed by the previous solve), so it can
// be launched as a programmatic dependent of the kernel before it.
// The tensor-core solve (k_bcr_solve_tc): an ordinary launch of two CTAs per SM
// that takes its units from a queue; counters as the cooperative solve's.
int bcr_solve_tc(fpsa_ctx *ctx, PathBuffers<float> &p, float *rhs) {
    const Geometry &g = ctx->geo;
    const size_t n = ctx->flow_n;
    int *cnt = ctx->d_flow + 2 * n * ctx->flow_parity, *done = cnt + n;
    int *zero_next = ctx->d_flow + 2 * n * (1 - ctx->flow_parity);
    int *queue = ctx->d_tcs_queue + ctx->flow_parity, *queue_next = ctx->d_tcs_queue + (1 - ctx->flow_parity);
    ctx->flow_parity ^= 1;
    const int RT = ctx->tcs_rt;
    const size_t smem = tcs::Plan::make(2 * g.N, RT).total;
    Launch L_(ctx, FPSA_PHASE_BCR_SOLVE);
    auto go = [&](auto kern) {
        return launch_pdl(kern, dim3(ctx->tcs_grid), dim3(tcs::kThreads), smem, ctx->stream,
                          (const unsigned char *)ctx->d_tcs_A, (const float *)p.Bc, (const float *)p.Cc,
                          (const BcrItem *)ctx->d_items_all, ctx->lvt[0], rhs, p.ybuf, ctx->d_tcs_g, g.N, g.sumK,
                          g.R, cnt, done, queue, ctx->d_dev_err, zero_next, (long long)(2 * n), queue_next);
    };
    switch (RT) {
        case 16: CK(go(k_bcr_solve_tc<16>)); break;
        case 32: CK(go(k_bcr_solve_tc<32>)); break;
        case 48: CK(go(k_bcr_solve_tc<48>)); break;
        default: CK(go(k_bcr_solve_tc<64>)); break;
    }
    return FPSA_OK;
}

template <typename T>
int bcr_solve(fpsa_ctx *ctx, PathBuffers<T> &p, T *rhs) {
    if constexpr (sizeof(T) == sizeof(float))
        if (ctx->tcs_rt && ctx->tuning.solve_engine != 1) return bcr_solve_tc(ctx, p, rhs);
    const Geometry &g = ctx->geo;
    int N = g.N, sumK = g.sumK, R = g.R;
    const BcrItem *items = ctx->d_items_all;
    LevelTable lv = ctx->lvt[sizeof(T) == 8 ? 1 : 0];
    const T *A = p.A, *Bc = p.Bc, *Cc = p.Cc;
    T *Y = p.ybuf;
    const size_t n = ctx->flow_n;
    int *cnt = ctx->d_flow + 2 * n * ctx->flow_parity, *done = cnt + n, *err = ctx->d_dev_err;
    int *zero_next = ctx->d_flow + 2 * n * (1 - ctx->flow_parity);
    long long nzero = (long long)(2 * n);
    ctx->flow_parity ^= 1;
    const T *G = p.G;
    void *args[] = {(void *)&A,   (void *)&Bc,  (void *)&Cc,   (void *)&items, (void *)&lv,
                    (void *)&rhs, (void *)&Y,   (void *)&N,    (void *)&sumK,  (void *)&R,
                    (void *)&cnt, (void *)&done, (void *)&err, (void *)&G,     (void *)&zero_next, (void *)&nzero};
    const int grid = ctx->coop_grid[sizeof(T) == 8 ? 1 : 0];
    const int RC = solve_rc(R);
    const void *kern = coop_kernel<T>(RC, N);
    Launch L_(ctx, FPSA_PHASE_BCR_SOLVE);
    if (g_plain_launch) {  // captured into a batch graph: a cooperative kernel node
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(solve_threads<T>(N));
        cfg.dynamicSmemBytes = solve_smem<T>(N, RC);
        cfg.stream = ctx->stream;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeCooperative;
        attr.val.cooperative = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelExC(&cfg, kern, args));
        return FPSA_OK;
    }
    if (ctx->solve_pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(solve_threads<T>(N));
        cfg.dynamicSmemBytes = solve_smem<T>(N, RC);
        cfg.stream = ctx->stream;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        if (cudaLaunchKernelExC(&cfg, kern, args) == cudaSuccess) return FPSA_OK;
        (void)cudaGetLastError();  // the combination is refused: plain cooperative launches from now on
        ctx->solve_pdl = false;
    }
    CK(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(solve_threads<T>(N)), args, solve_smem<T>(N, RC),
                                   ctx->stream));
    return FPSA_OK;
}

template <typename T>
// Qm: source moments (may be NULL), Qa: nodal angular source (may be NULL), inc:
// incoming edge fluxes (may be NULL). phi_out may be NULL (the iterate stays in p.phi).
int solve_fp64(fpsa_ctx *ctx, PathBuffers<T> &p, const fpsa_opts &o, const double *phi0, int mem, double *phi_out,
               fpsa_stats &stats, const T *Qm, const T *Qa, const T *inc) {
    const Geometry &g = ctx->geo;
    const int N = g.N, L1 = g.L1;
    cudaStream_t st = ctx->stream;
    const size_t ncol = (size_t)g.R * g.sumK * 2;
    const size_t csm = contract_smem<T>(N);
    const dim3 cgrid((g.sumK + kContractCells - 1) / kContractCells, g.R);
    const bool fpsa = o.method == FPSA_METHOD_FPSA;

    if (phi0) {
        CK(cudaMemsetAsync(p.phi, 0, ncol * N * sizeof(T), st));
        CK(cudaMemcpy2DAsync(p.phi, N * sizeof(T), phi0, L1 * sizeof(double), L1 * sizeof(double), ncol,
                             mem == FPSA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    } else {
        CK(cudaMemsetAsync(p.phi, 0, ncol * N * sizeof(T), st));
    }
    CK(cudaMemsetAsync(ctx->d_conv, 0, (size_t)g.R * g.B * 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(ctx->d_dev_err, 0, sizeof(int), st));
    {
        Launch L_(ctx, FPSA_PHASE_CONTRACT);
        k_scatter<T><<<cgrid, kContractThreads, csm / 2, st>>>(p.phi, p.sigma_s, Qm, p.MT, p.q, N, g.sumK, Qa);
    }
    CK(cudaGetLastError());
    const int every = o.check_every > 0 ? o.check_every : 1;
    int status = FPSA_ENOTCONV;
    double e = INFINITY;
    int it = 0;
    for (it = 1; it <= o.max_iterations; ++it) {
        int rc0 = sweep(ctx, p, p.q, p.psi, inc);
        if (rc0) return rc0;
        if (fpsa) {
            {
                Launch L_(ctx, FPSA_PHASE_CONTRACT);
                k_fp_rhs<T><<<cgrid, kContractThreads, csm, st>>>(p.psi, p.phi, p.phi_half, p.sigma_s, ctx->d_h, p.DT,
                                                                   p.MT, p.rhs, N, g.sumK);
            }
            int rc = bcr_solve(ctx, p, p.rhs);
            if (rc) return rc;
            {
                Launch L_(ctx, FPSA_PHASE_CONTRACT);
                k_update_scatter<T><<<cgrid, kContractThreads, csm, st>>>(p.ybuf, p.phi_half, p.phi, p.sigma_s, Qm, p.DT,
                                                                           p.MT, p.q, ctx->d_cell_inst, g.B, ctx->d_conv,
                                                                           N, g.sumK, Qa);
            }
        } else {
            {
                Launch L_(ctx, FPSA_PHASE_CONTRACT);
                k_update_scatter<T><<<cgrid, kContractThreads, csm, st>>>(p.psi, (const T *)nullptr, p.phi, p.sigma_s,
                                                                           Qm, p.DT, p.MT, p.q, ctx->d_cell_inst, g.B,
                                                                           ctx->d_conv, N, g.sumK, Qa);
            }
        }
        CK(cudaGetLastError());
        if (it % every == 0 || it == o.max_iterations) {
            {
                Launch L_(ctx, FPSA_PHASE_CONVERGENCE);
                k_conv_finalize<<<1, 256, 0, st>>>(ctx->d_conv, g.R * g.B, ctx->d_result);
            }
            CK(cudaMemcpyAsync(ctx->h_result, ctx->d_result, sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(ctx->h_flag, ctx->d_dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            e = ctx->h_result[0];
            if (*ctx->h_flag) {
                status = fail(ctx, FPSA_ETIMEOUT, "a bounded device wait ran out (BCR dataflow)");
                break;
            }
            if (std::isnan(e)) {
                status = fail(ctx, FPSA_ENONFINITE, "non-finite iterate at iteration " + std::to_string(it));
                break;
            }
            if (e < o.tol) {
                status = FPSA_OK;
                break;
            }
        }
    }
    if (it > o.max_iterations) it = o.max_iterations;
    stats.iterations = it;
    stats.outer_iterations = it;
    stats.sweeps = it;
    stats.rel_change = e;
    if (phi_out)
        CK(cudaMemcpy2DAsync(phi_out, L1 * sizeof(double), p.phi, N * sizeof(T), L1 * sizeof(double), ncol,
                             mem == FPSA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    if (status == FPSA_ENOTCONV)
        fail(ctx, FPSA_ENOTCONV, "not converged after " + std::to_string(o.max_iterations) + " iterations");
    return status;
}

// MIXED: FP64 iterative refinement on the GPU around FP32 FPSA inner solves.
//   outer k:  phi = D psi64, convergence test of phi_0 against the previous outer
//             iterate (Eq. iterate), residual source dq (FP64, stored FP32)
//   inner:    `inner` FPSA iterations (Eqs. predict, correct) on L dpsi = S dpsi + dq
//             from dpsi = 0, all in FP32: sweep, contractions, BCR solve
//   update:   psi64 += psi_half + upsilon of the last inner iteration (FP64)
// With the GMRES method the inner solve is FP32 GMRES(m) on the moment form of the
// correction equation (to a relative residual of inner_tol, at most inner_cap Krylov
// iterations), followed by one sweep for the angular correction.
template <typename T>
int gmres_core(fpsa_ctx *ctx, PathBuffers<T> &p, int m, double tol, int max_it, const T *Qm, const T *Qa,
               const T *inc, int &it, int &sweeps, double &worst);

// Launch plan of the MIXED path's inner contractions (tensor cores or SIMT FP32).
struct MixedPlan {
    dim3 cgrid;
    size_t ncol, nang;
    bool use_tc, tc_big, tc_full;
    TcOps tcops;
    int tc_blocks;
    size_t tc_smem;
};

int mixed_plan(fpsa_ctx *ctx, const fpsa_opts &o, MixedPlan &mp) {
    const Geometry &g = ctx->geo;
    const int N = g.N;
    if (o.contraction == 2 && !ctx->tc_able)
        return fail(ctx, FPSA_ENOTSUP,
                    "tensor-core contractions need N a multiple of 16 and <= 128, or a multiple of 32 and <= 256");
    mp.cgrid = dim3((g.sumK + kContractCells - 1) / kContractCells, g.R);
    mp.ncol = (size_t)g.R * g.sumK * 2;
    mp.nang = mp.ncol * N;
    mp.use_tc = ctx->tc_able && o.contraction != 1;
    mp.tcops = TcOps{ctx->d_tc_ops, ctx->d_tc_ops + 2 * (size_t)N * N * sizeof(__nv_bfloat16)};
    const int tc_tiles = ((2 * g.sumK + 127) / 128) * g.R;
    mp.tc_blocks = std::max(1, std::min(tc_tiles, ctx->tc_grid));
    mp.tc_big = ctx->tc_big;
    mp.tc_smem = mp.tc_big ? tc::BigPlan::make(N).total : tc::Plan::make(N).total;
    mp.tc_full = !mp.tc_big && tc::Plan::make(N).full;
    return FPSA_OK;
}

// The FP64 residual of a refinement step: phi = D psi64, the convergence maxima, the
// residual source of the next inner solve (k_mixed_residual), then the relative change
// of phi_0 into d_result (k_conv_finalize).
int mixed_residual_launch(fpsa_ctx *ctx, const MixedPlan &mp, const double *Qm, const double *Qa, const double *inc,
                          bool gmres) {
    const Geometry &g = ctx->geo;
    const int N = g.N;
    cudaStream_t st = ctx->stream;
    PathBuffers<double> &p = ctx->p64;
    PathBuffers<float> &f = ctx->p32;
    // auto: the tensor cores where the 64-cell tiles fill the GPU (one CTA per SM holds all
    // of its tensor memory); below that the FP64 kernel's finer blocks finish sooner
    const bool res_tc = ctx->res_ops.D && (ctx->tuning.residual_engine == 2 ||
                                           (ctx->tuning.residual_engine == 0 &&
                                            (long long)((g.sumK + 63) / 64) * g.R >= ctx->n_sm));
    if (res_tc) {
        Launch L_(ctx, FPSA_PHASE_RESIDUAL);
        CK(launch_pdl(k_mixed_residual_tc, dim3((g.sumK + 63) / 64, g.R), dim3(rtc::kThreads),
                      (size_t)rtc::smem_bytes(N), st, (const double *)p.psi, p.phi, (const double *)p.sigma_s, Qm,
                      ctx->res_ops, (const double *)ctx->d_sigma_t, (const double *)ctx->d_h,
                      (const double *)ctx->d_mu, (const int32_t *)ctx->d_cell_inst, (const int32_t *)ctx->d_off,
                      (const int32_t *)ctx->d_K, g.B, ctx->d_conv, f.qang, N, g.sumK, Qa, inc,
                      (const int32_t *)ctx->d_bc, gmres ? (float *)nullptr : f.q, gmres ? (float *)nullptr : f.phi,
                      ctx->d_dev_err));
    } else {
        Launch L_(ctx, FPSA_PHASE_RESIDUAL);
        CK(launch_pdl(k_mixed_residual, mp.cgrid, dim3(kContractThreads), contract_smem<double>(N), st, p.psi, p.phi,
                      p.sigma_s, Qm, p.DT, p.MT, ctx->d_sigma_t, ctx->d_h, ctx->d_mu, ctx->d_cell_inst, ctx->d_off,
                      ctx->d_K, g.B, ctx->d_conv, f.qang, N, g.sumK, Qa, inc, ctx->d_bc,
                      gmres ? (float *)nullptr : f.q, gmres ? (float *)nullptr : f.phi));
    }
    {
        Launch L_(ctx, FPSA_PHASE_CONVERGENCE);
        CK(launch_pdl(k_conv_finalize, dim3(1), dim3(256), 0, st, ctx->d_conv, g.R * g.B, ctx->d_result));
    }
    CK(cudaGetLastError());
    return FPSA_OK;
}

// inner_k FP32 FPSA (fpsa) or SI iterations of the correction equation from zero
// (f.phi = 0 and f.q = f.qang were written by the residual kernel), then
// psi64 += dpsi (FP64). Adds the sweeps launched to `sweeps`.
int mixed_inner_launch(fpsa_ctx *ctx, const MixedPlan &mp, int inner_k, bool fpsa, int &sweeps) {
    const Geometry &g = ctx->geo;
    const int N = g.N;
    cudaStream_t st = ctx->stream;
    PathBuffers<double> &p = ctx->p64;
    PathBuffers<float> &f = ctx->p32;
    const dim3 cgrid = mp.cgrid;
    const bool use_tc = mp.use_tc, tc_big = mp.tc_big, tc_full = mp.tc_full;
    const int tc_blocks = mp.tc_blocks;
    const size_t tc_smem = mp.tc_smem;
    const TcOps tcops = mp.tcops;
    for (int j = 1; j <= inner_k; ++j) {
        int rcs = sweep(ctx, f, f.q, f.psi, (const float *)nullptr);
        if (rcs) return rcs;
        ++sweeps;
        const float *vin = f.psi, *base = nullptr;
        if (fpsa) {
            {
                Launch L_(ctx, FPSA_PHASE_CONTRACT);
                if (use_tc && tc_big)
                    CK(launch_pdl(k_tc_fp_rhs_big, dim3(tc_blocks), dim3(128), tc_smem, st, (const float *)f.psi,
                                  (const float *)f.phi, f.phi_half, (const float *)f.sigma_s,
                                  (const double *)ctx->d_h, tcops, f.rhs, N, g.sumK, g.R, ctx->d_dev_err));
                else if (use_tc && tc_full)
                    CK(launch_pdl(k_tc_fp_rhs_tile, dim3(tc_blocks), dim3(128), tc_smem, st, (const float *)f.psi,
                                  (const float *)f.phi, f.phi_half, (const float *)f.sigma_s,
                                  (const double *)ctx->d_h, tcops, f.rhs, N, g.sumK, g.R, ctx->d_dev_err));
                else if (use_tc)
                    k_tc_fp_rhs<<<tc_blocks, 128, tc_smem, st>>>(f.psi, f.phi, f.phi_half, f.sigma_s, ctx->d_h,
                                                                 tcops, f.rhs, N, g.sumK, g.R, ctx->d_dev_err);
                else
                    k_fp_rhs<float><<<cgrid, kContractThreads, contract_smem<float>(N), st>>>(
                        f.psi, f.phi, f.phi_half, f.sigma_s, ctx->d_h, f.DT, f.MT, f.rhs, N, g.sumK);
            }
            int rc = bcr_solve(ctx, f, f.rhs);
            if (rc) return rc;
            vin = f.ybuf;
            base = f.phi_half;
        }
        if (j < inner_k) {
            Launch L_(ctx, FPSA_PHASE_CONTRACT);
            if (use_tc && tc_big)
                CK(launch_pdl(k_tc_update_scatter_big, dim3(tc_blocks), dim3(128), tc_smem, st, vin, base, f.phi,
                              (const float *)f.sigma_s, tcops, f.q, (const float *)f.qang, N, g.sumK, g.R,
                              ctx->d_dev_err));
            else if (use_tc && tc_full)
                CK(launch_pdl(k_tc_update_scatter_tile, dim3(tc_blocks), dim3(128), tc_smem, st, vin, base, f.phi,
                              (const float *)f.sigma_s, tcops, f.q, (const float *)f.qang, N, g.sumK, g.R,
                              ctx->d_dev_err));
            else if (use_tc)
                k_tc_update_scatter<<<tc_blocks, 128, tc_smem, st>>>(vin, base, f.phi, f.sigma_s, tcops, f.q,
                                                                     f.qang, N, g.sumK, g.R, ctx->d_dev_err);
            else
                k_update_scatter<float><<<cgrid, kContractThreads, contract_smem<float>(N), st>>>(
                    vin, base, f.phi, f.sigma_s, (const float *)nullptr, f.DT, f.MT, f.q, ctx->d_cell_inst, g.B,
                    (unsigned long long *)nullptr, N, g.sumK, f.qang);
        }
    }
    {
        Launch L_(ctx, FPSA_PHASE_RESIDUAL);
        CK(launch_pdl(k_mixed_accumulate, dim3(4 * 152), dim3(256), 0, st, p.psi, (const float *)f.psi,
                      fpsa ? (const float *)f.ybuf : (const float *)nullptr, mp.nang));
    }
    CK(cudaGetLastError());
    return FPSA_OK;
}

int solve_mixed(fpsa_ctx *ctx, const fpsa_opts &o, const double *phi0, int mem, double *phi_out, fpsa_stats &stats,
                const double *Qm, const double *Qa, const double *inc) {
    const Geometry &g = ctx->geo;
    const int N = g.N, L1 = g.L1;
    cudaStream_t st = ctx->stream;
    PathBuffers<double> &p = ctx->p64;
    PathBuffers<float> &f = ctx->p32;
    MixedPlan mp;
    int rcp = mixed_plan(ctx, o, mp);
    if (rcp) return rcp;
    const size_t ncol = mp.ncol, nang = mp.nang;
    const dim3 cgrid = mp.cgrid;
    const int inner = o.inner_iterations > 0 ? o.inner_iterations : 4;
    const bool adaptive = o.inner_iterations <= 0;
    constexpr int kInnerMax = 16;
    int k_before = 0, k_last = 0;  // inner iterations of the last two steps
    const bool fpsa = o.method == FPSA_METHOD_FPSA, gmres = o.method == FPSA_METHOD_GMRES;
    const int m = o.restart > 0 ? o.restart : 30;
    const int inner_cap = o.inner_iterations > 0 ? o.inner_iterations : m;
    const double inner_tol = o.inner_tol > 0 ? o.inner_tol : 1e-5;
    int krylov = 0;
    ctx->gm_use_tc = mp.use_tc;  // the inner GMRES solves of GMRES-IR too
    CK(cudaMemsetAsync(ctx->d_dev_err, 0, sizeof(int), st));

    CK(cudaMemsetAsync(p.phi, 0, nang * sizeof(double), st));
    if (phi0) {
        CK(cudaMemcpy2DAsync(p.phi, N * sizeof(double), phi0, L1 * sizeof(double), L1 * sizeof(double), ncol,
                             mem == FPSA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
        Launch L_(ctx, FPSA_PHASE_RESIDUAL);
        k_expand<double><<<cgrid, kContractThreads, contract_smem<double>(N) / 2, st>>>(p.phi, p.MT, p.psi, N, g.sumK);
    } else {
        CK(cudaMemsetAsync(p.psi, 0, nang * sizeof(double), st));
    }
    CK(cudaMemsetAsync(ctx->d_conv, 0, (size_t)g.R * g.B * 2 * sizeof(unsigned long long), st));
    int status = FPSA_ENOTCONV;
    double e = INFINITY, e_prev = INFINITY;
    int outer = 0, sweeps = 0;
    // the adaptive inner count pays only where a residual costs more than an inner
    // iteration: both are timed once, on the first refinement step (event pairs)
    bool adaptive_on = false;
    const bool time_first = adaptive && fpsa;
    if (time_first && !ctx->ad_ev[0])
        for (int i = 0; i < 4; ++i) CK(cudaEventCreate(&ctx->ad_ev[i]));
    for (outer = 1; outer <= o.max_iterations + 1; ++outer) {
        if (time_first && outer == 1) CK(cudaEventRecord(ctx->ad_ev[0], st));
        int rcr = mixed_residual_launch(ctx, mp, Qm, Qa, inc, gmres);
        if (rcr) return rcr;
        if (time_first && outer == 1) CK(cudaEventRecord(ctx->ad_ev[1], st));
        CK(cudaMemcpyAsync(ctx->h_result, ctx->d_result, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ctx->h_flag, ctx->d_dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        e = ctx->h_result[0];
        if (*ctx->h_flag) {
            status = fail(ctx, FPSA_ETIMEOUT, "a bounded device wait ran out (tensor-core contraction or BCR dataflow)");
            break;
        }
        if (std::isnan(e)) {
            status = fail(ctx, FPSA_ENONFINITE, "non-finite iterate at refinement step " + std::to_string(outer));
            break;
        }
        if ((outer > 1 || phi0) && e < o.tol) {
            status = FPSA_OK;
            break;
        }
        if (outer > o.max_iterations) break;
        if (gmres) {
            // inner FP32 GMRES on the correction equation (moments), then the angular
            // correction dpsi = L^{-1} (M Sigma dphi + dq) by one more sweep
            int git = 0, gsw = 0;
            double gres = 0.0;
            int rc = gmres_core<float>(ctx, f, m, inner_tol, inner_cap, (const float *)nullptr, f.qang,
                                       (const float *)nullptr, git, gsw, gres);
            if (rc != FPSA_OK && rc != FPSA_ENOTCONV) return rc;
            krylov += git;
            sweeps += gsw + 1;
            {
                Launch L_(ctx, FPSA_PHASE_CONTRACT);
                k_scatter<float><<<cgrid, kContractThreads, contract_smem<float>(N) / 2, st>>>(
                    f.phi, f.sigma_s, (const float *)nullptr, f.MT, f.q, N, g.sumK, f.qang);
            }
            rc = sweep(ctx, f, f.q, f.psi, (const float *)nullptr);
            if (rc) return rc;
            {
                Launch L_(ctx, FPSA_PHASE_RESIDUAL);
                CK(launch_pdl(k_mixed_accumulate, dim3(4 * 152), dim3(256), 0, st, p.psi, (const float *)f.psi,
                              (const float *)nullptr, nang));
            }
            CK(cudaGetLastError());
            continue;
        }
        // inner FP32 solve of the correction from zero. When the last two refinement
        // changes predict that the remaining error (geometric extrapolation) is already
        // below tol, one inner iteration suffices for the step that confirms it: the
        // stopping test itself is unchanged. With the adaptive count (inner_iterations
        // 0), a step takes as many inner iterations as the observed contraction per
        // inner iteration needs to bring that error below tol, at most kInnerMax and no
        // more than keep the step's reduction above the FP32 floor (1e-6): fewer FP64
        // residuals where they are expensive relative to an inner iteration.
        // The change e measured now is the size of the previous step's correction, i.e. the
        // error before that step, so e / e_prev is the contraction of the step before it
        // (k_before inner iterations) and the error now is e times the contraction of the
        // previous step (k_last inner iterations).
        int inner_k = inner;
        if (outer > 1 && e_prev > e && e > 0.0) {
            const double r = e / e_prev;
            if (!adaptive || k_before == 0) {
                if (e * r / (1.0 - r) < o.tol) inner_k = 1;
            } else {
                const double lrho = std::log(r) / k_before;  // log of the contraction per inner iteration
                const double err = e * std::exp(lrho * k_last), rk = std::exp(lrho * inner);
                if (err / (1.0 - rk) < o.tol) {
                    inner_k = 1;
                } else {
                    const int need = (int)std::ceil(std::log(o.tol / err) / lrho);
                    const int floor32 = (int)std::floor(std::log(1e-6) / lrho);
                    inner_k = std::max(inner, std::min({need, floor32, kInnerMax}));
                }
            }
        }
        e_prev = e;
        k_before = k_last;
        k_last = inner_k;
        if (time_first && outer == 2) {  // the first step's events have completed (synchronised above)
            float t_res = 0.f, t_step = 0.f;
            if (cudaEventElapsedTime(&t_res, ctx->ad_ev[0], ctx->ad_ev[1]) == cudaSuccess &&
                cudaEventElapsedTime(&t_step, ctx->ad_ev[2], ctx->ad_ev[3]) == cudaSuccess)
                adaptive_on = t_res * inner > t_step;  // residual slower than one inner iteration
            (void)cudaGetLastError();
        }
        if (!adaptive_on && inner_k > inner) inner_k = inner;
        k_last = inner_k;
        if (time_first && outer == 1) CK(cudaEventRecord(ctx->ad_ev[2], st));
        int rci = mixed_inner_launch(ctx, mp, inner_k, fpsa, sweeps);
        if (rci) return rci;
        if (time_first && outer == 1) CK(cudaEventRecord(ctx->ad_ev[3], st));
    }
    stats.iterations = gmres ? krylov : sweeps;
    stats.outer_iterations = std::min(outer, o.max_iterations + 1);
    stats.sweeps = sweeps;
    stats.rel_change = e;
    if (phi_out)
        CK(cudaMemcpy2DAsync(phi_out, L1 * sizeof(double), p.phi, N * sizeof(double), L1 * sizeof(double), ncol,
                             mem == FPSA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    if (status == FPSA_ENOTCONV)
        fail(ctx, FPSA_ENOTCONV, "not converged after " + std::to_string(o.max_iterations) + " refinement steps");
    return status;
}


// Lazily allocate the GMRES work space for restart length m. The basis and work
// vectors hold the precision of the Krylov solve (FP64 contexts: double; MIXED:
// float, the inner solve of the refinement loop); dots are always FP64.
int gmres_alloc(fpsa_ctx *ctx, int m) {
    if (ctx->gm_restart >= m) return FPSA_OK;
    const Geometry &g = ctx->geo;
    const size_t n = (size_t)g.R * g.sumK * 2 * g.N;
    const size_t es = ctx->precision == FPSA_PRECISION_FP64 ? sizeof(double) : sizeof(float);
    const int nsys = g.R * g.B;
    if (ctx->gm_V) {  // grow: release the old basis (the allocations list keeps the pointer)
        CK(cudaFree(ctx->gm_V));
        ctx->allocs.erase(std::find(ctx->allocs.begin(), ctx->allocs.end(), (void *)ctx->gm_V));
        ctx->gm_V = nullptr;
    }
    CK(dalloc(ctx, &ctx->gm_V, (size_t)(m + 1) * n * es));
    if (!ctx->gm_u) {
        CK(dalloc(ctx, &ctx->gm_u, n * es));
        CK(dalloc(ctx, &ctx->gm_w, n * es));
        CK(dalloc(ctx, &ctx->gm_b, n * es));
        CK(dalloc(ctx, &ctx->gm_seg_begin, nsys));
        CK(dalloc(ctx, &ctx->gm_seg_end, nsys));
        std::vector<long long> sb(nsys), se(nsys);
        long long maxlen = 0;
        for (int r = 0; r < g.R; ++r)
            for (int b = 0; b < g.B; ++b) {
                const int s = r * g.B + b;
                sb[s] = ((long long)r * g.sumK + g.off[b]) * 2 * g.N;
                se[s] = sb[s] + (long long)g.K[b] * 2 * g.N;
                maxlen = std::max(maxlen, se[s] - sb[s]);
            }
        CK(cudaMemcpy(ctx->gm_seg_begin, sb.data(), nsys * sizeof(long long), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->gm_seg_end, se.data(), nsys * sizeof(long long), cudaMemcpyHostToDevice));
        ctx->gm_nchunks = (int)((maxlen + kDotChunk - 1) / kDotChunk);
    }
    if (ctx->gm_partial) {
        for (double *q : {ctx->gm_partial, ctx->gm_dots, ctx->gm_coef, ctx->gm_alpha}) {
            CK(cudaFree(q));
            ctx->allocs.erase(std::find(ctx->allocs.begin(), ctx->allocs.end(), (void *)q));
        }
    }
    CK(dalloc(ctx, &ctx->gm_partial, (size_t)nsys * ctx->gm_nchunks * (m + 1)));
    CK(dalloc(ctx, &ctx->gm_dots, (size_t)nsys * (m + 1)));
    CK(dalloc(ctx, &ctx->gm_coef, (size_t)nsys * (m + 1)));
    CK(dalloc(ctx, &ctx->gm_alpha, nsys));
    ctx->gm_restart = m;
    return FPSA_OK;
}

// out[s][i] = <V_i, w>_s for i < nv, all systems s (FP64 sums); result copied to host hdots.
template <typename T>
int gm_dots(fpsa_ctx *ctx, const T *V, int nv, const T *w, std::vector<double> &hdots) {
    const Geometry &g = ctx->geo;
    const int nsys = g.R * g.B;
    const size_t n = (size_t)g.R * g.sumK * 2 * g.N;
    cudaStream_t st = ctx->stream;
    {
        Launch L_(ctx, FPSA_PHASE_CONVERGENCE);
        k_seg_dots<T><<<dim3(ctx->gm_nchunks, nsys), kDotThreads, 0, st>>>(V, n, nv, w, ctx->gm_seg_begin, ctx->gm_seg_end,
                                                                   ctx->gm_nchunks, ctx->gm_partial);
    }
    {
        Launch L_(ctx, FPSA_PHASE_CONVERGENCE);
        k_seg_dots_finish<<<(nsys * nv + 255) / 256, 256, 0, st>>>(ctx->gm_partial, nsys, ctx->gm_nchunks, nv,
                                                                    ctx->gm_dots);
    }
    CK(cudaGetLastError());
    hdots.resize((size_t)nsys * nv);
    CK(cudaMemcpyAsync(hdots.data(), ctx->gm_dots, hdots.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ctx->h_flag, ctx->d_dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*ctx->h_flag) return fail(ctx, FPSA_ETIMEOUT, "a bounded device wait ran out (BCR dataflow)");
    return FPSA_OK;
}

// y = alpha_s x + sum_i coef[s][i] V_i (alpha NULL: y = sum ...; x NULL: x = y),
// coefficients from the host.
template <typename T>
int gm_combine(fpsa_ctx *ctx, T *y, const std::vector<double> *alpha, const T *V, int nv,
               const std::vector<double> &coef, const T *x = nullptr) {
    const Geometry &g = ctx->geo;
    const int nsys = g.R * g.B;
    const size_t n = (size_t)g.R * g.sumK * 2 * g.N;
    cudaStream_t st = ctx->stream;
    if (nv) CK(cudaMemcpyAsync(ctx->gm_coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    if (alpha)
        CK(cudaMemcpyAsync(ctx->gm_alpha, alpha->data(), alpha->size() * sizeof(double), cudaMemcpyHostToDevice, st));
    {
        Launch L_(ctx, FPSA_PHASE_CONVERGENCE);
        k_seg_combine<T><<<dim3(ctx->gm_nchunks, nsys), kDotThreads, 0, st>>>(
            y, alpha ? ctx->gm_alpha : nullptr, x ? x : y, V, n, nv, ctx->gm_coef, ctx->gm_seg_begin,
            ctx->gm_seg_end);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));  // the host vectors are reused right away
    return FPSA_OK;
}

// The GMRES operator's contractions, on tensor cores for the FP32 inner solve of
// GMRES-IR when ctx->gm_use_tc (set per solve from the options), else SIMT:
//   gm_fp_rhs:  rhs = m (x) M Sigma v
//   gm_update:  out = base + D y;  q = M Sigma out
//   gm_axpy:    out = base + sign D psi  (base may be NULL or alias out)
template <typename T>
int gm_fp_rhs(fpsa_ctx *ctx, PathBuffers<T> &p, const T *v, T *rhs) {
    const Geometry &g = ctx->geo;
    const int N = g.N;
    cudaStream_t st = ctx->stream;
    Launch L_(ctx, FPSA_PHASE_CONTRACT);
    if constexpr (sizeof(T) == sizeof(float)) {
        if (ctx->gm_use_tc) {
            const TcOps ops{ctx->d_tc_ops, ctx->d_tc_ops + 2 * (size_t)N * N * sizeof(__nv_bfloat16)};
            const int blocks = std::max(1, std::min(((2 * g.sumK + 127) / 128) * g.R, ctx->tc_grid));
            if (ctx->tc_big)
                CK(launch_pdl(k_tc_fp_rhs_moments<true>, dim3(blocks), dim3(128), (size_t)tc::BigPlan::make(N).total, st,
                              (const float *)v, (const float *)p.sigma_s, (const double *)ctx->d_h, ops, (float *)rhs, N,
                              g.sumK, g.R, ctx->d_dev_err));
            else
                CK(launch_pdl(k_tc_fp_rhs_moments<false>, dim3(blocks), dim3(128), (size_t)tc::Plan::make(N).total, st,
                              (const float *)v, (const float *)p.sigma_s, (const double *)ctx->d_h, ops, (float *)rhs, N,
                              g.sumK, g.R, ctx->d_dev_err));
            return FPSA_OK;
        }
    }
    const dim3 cgrid((g.sumK + kContractCells - 1) / kContractCells, g.R);
    k_fp_rhs_moments<T><<<cgrid, kContractThreads, contract_smem<T>(N), st>>>(v, p.sigma_s, ctx->d_h, p.MT, rhs, N,
                                                                               g.sumK);
    CK(cudaGetLastError());
    return FPSA_OK;
}

template <typename T>
int gm_update(fpsa_ctx *ctx, PathBuffers<T> &p, const T *y, const T *base, T *out) {
    const Geometry &g = ctx->geo;
    const int N = g.N;
    cudaStream_t st = ctx->stream;
    Launch L_(ctx, FPSA_PHASE_CONTRACT);
    if constexpr (sizeof(T) == sizeof(float)) {
        if (ctx->gm_use_tc) {
            const TcOps ops{ctx->d_tc_ops, ctx->d_tc_ops + 2 * (size_t)N * N * sizeof(__nv_bfloat16)};
            const int blocks = std::max(1, std::min(((2 * g.sumK + 127) / 128) * g.R, ctx->tc_grid));
            const float *qnull = nullptr;
            if (ctx->tc_big)
                CK(launch_pdl(k_tc_update_scatter_big, dim3(blocks), dim3(128), (size_t)tc::BigPlan::make(N).total,
                              st, (const float *)y, (const float *)base, (float *)out, (const float *)p.sigma_s, ops,
                              (float *)p.q, qnull, N, g.sumK, g.R, ctx->d_dev_err));
            else if (tc::Plan::make(N).full)
                CK(launch_pdl(k_tc_update_scatter_tile, dim3(blocks), dim3(128), (size_t)tc::Plan::make(N).total, st,
                              (const float *)y, (const float *)base, (float *)out, (const float *)p.sigma_s, ops,
                              (float *)p.q, qnull, N, g.sumK, g.R, ctx->d_dev_err));
            else
                CK(launch_pdl(k_tc_update_scatter, dim3(blocks), dim3(128), (size_t)tc::Plan::make(N).total, st,
                              (const float *)y, (const float *)base, (float *)out, (const float *)p.sigma_s, ops,
                              (float *)p.q, qnull, N, g.sumK, g.R, ctx->d_dev_err));
            return FPSA_OK;
        }
    }
    const dim3 cgrid((g.sumK + kContractCells - 1) / kContractCells, g.R);
    k_update_scatter<T><<<cgrid, kContractThreads, contract_smem<T>(N), st>>>(
        y, base, out, p.sigma_s, (const T *)nullptr, p.DT, p.MT, p.q, ctx->d_cell_inst, g.B,
        (unsigned long long *)nullptr, N, g.sumK, (const T *)nullptr);
    CK(cudaGetLastError());
    return FPSA_OK;
}

template <typename T>
int gm_axpy(fpsa_ctx *ctx, PathBuffers<T> &p, const T *psi, const T *base, T sign, T *out) {
    const Geometry &g = ctx->geo;
    const int N = g.N;
    cudaStream_t st = ctx->stream;
    Launch L_(ctx, FPSA_PHASE_CONTRACT);
    if constexpr (sizeof(T) == sizeof(float)) {
        if (ctx->gm_use_tc) {
            const TcOps ops{ctx->d_tc_ops, ctx->d_tc_ops + 2 * (size_t)N * N * sizeof(__nv_bfloat16)};
            const int blocks = std::max(1, std::min(((2 * g.sumK + 127) / 128) * g.R, ctx->tc_grid));
            if (ctx->tc_big)
                CK(launch_pdl(k_tc_moments_axpy<true>, dim3(blocks), dim3(128), (size_t)tc::BigPlan::make(N).total, st,
                              (const float *)psi, (const float *)base, (float)sign, ops, (float *)out, N, g.sumK, g.R,
                              ctx->d_dev_err));
            else
                CK(launch_pdl(k_tc_moments_axpy<false>, dim3(blocks), dim3(128), (size_t)tc::Plan::make(N).total, st,
                              (const float *)psi, (const float *)base, (float)sign, ops, (float *)out, N, g.sumK, g.R,
                              ctx->d_dev_err));
            return FPSA_OK;
        }
    }
    const dim3 cgrid((g.sumK + kContractCells - 1) / kContractCells, g.R);
    k_moments_axpy<T><<<cgrid, kContractThreads, contract_smem<T>(N), st>>>(psi, base, sign, p.DT, out, N, g.sumK);
    CK(cudaGetLastError());
    return FPSA_OK;
}

// out = (I - T)(I + C) v  (out may not alias v)
template <typename T>
int gm_apply(fpsa_ctx *ctx, PathBuffers<T> &p, const T *v, T *out) {
    int rc = gm_fp_rhs(ctx, p, v, p.rhs);
    if (rc) return rc;
    rc = bcr_solve(ctx, p, p.rhs);
    if (rc) return rc;
    rc = gm_update(ctx, p, (const T *)p.ybuf, v, out);  // out = z = v + D upsilon;  q = M Sigma z
    if (rc) return rc;
    rc = sweep(ctx, p, p.q, p.psi, (const T *)nullptr);
    if (rc) return rc;
    return gm_axpy(ctx, p, (const T *)p.psi, (const T *)out, T(-1), out);  // out = z - D psi
}

// GMRES(m) with right FPSA preconditioning in precision T, batched over (rhs, instance)
// systems: (I - T)(I + C) u = b, b = D L^{-1} (M Qm + Qa) with the incoming edge
// fluxes inc (the applications of T take none), from u = 0; on return p.phi
// holds phi = (I + C) u. Stops when every system's relative residual 2-norm (the
// Givens estimate, and the true residual at each restart) is below tol, or after
// max_it Krylov iterations (FPSA_ENOTCONV, no message: the caller decides).
template <typename T>
int gmres_core(fpsa_ctx *ctx, PathBuffers<T> &p, int m, double tol, int max_it, const T *Qm, const T *Qa,
               const T *inc, int &it, int &sweeps, double &worst) {
    const Geometry &g = ctx->geo;
    const int N = g.N, nsys = g.R * g.B;
    const size_t n = (size_t)g.R * g.sumK * 2 * N;
    cudaStream_t st = ctx->stream;
    int rc = gmres_alloc(ctx, m);
    if (rc) return rc;
    CK(cudaMemsetAsync(ctx->d_dev_err, 0, sizeof(int), st));
    T *V = reinterpret_cast<T *>(ctx->gm_V), *u = reinterpret_cast<T *>(ctx->gm_u),
      *w = reinterpret_cast<T *>(ctx->gm_w), *b = reinterpret_cast<T *>(ctx->gm_b);
    const size_t csm = contract_smem<T>(N);
    const dim3 cgrid((g.sumK + kContractCells - 1) / kContractCells, g.R);
    // b = D L^{-1} (M Qm + Qa)
    CK(cudaMemsetAsync(u, 0, n * sizeof(T), st));
    {
        Launch L_(ctx, FPSA_PHASE_CONTRACT);
        k_scatter<T><<<cgrid, kContractThreads, csm / 2, st>>>(u, p.sigma_s, Qm, p.MT, p.q, N, g.sumK, Qa);
    }
    rc = sweep(ctx, p, p.q, p.psi, inc);
    if (rc) return rc;
    rc = gm_axpy(ctx, p, (const T *)p.psi, (const T *)nullptr, T(1), b);
    if (rc) return rc;
    std::vector<double> dots, bnorm(nsys), coef, alpha(nsys), c1(nsys, 1.0);
    rc = gm_dots(ctx, b, 1, b, dots);
    if (rc) return rc;
    for (int s = 0; s < nsys; ++s) bnorm[s] = std::sqrt(dots[s]);
    it = 0;
    sweeps = 1;
    worst = INFINITY;
    int status = FPSA_ENOTCONV;
    while (it < max_it) {
        // r = b - A' u  (u = 0 on the first cycle)
        if (it > 0) {
            rc = gm_apply(ctx, p, u, w);
            if (rc) return rc;
            ++sweeps;
            std::vector<double> one(nsys, -1.0);
            rc = gm_combine(ctx, V, &c1, w, 1, one, (const T *)b);  // V_0 = b - A' u
            if (rc) return rc;
        } else {
            CK(cudaMemcpyAsync(V, b, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
        }
        rc = gm_dots(ctx, V, 1, V, dots);
        if (rc) return rc;
        std::vector<double> beta(nsys);
        worst = 0.0;
        for (int s = 0; s < nsys; ++s) {
            beta[s] = std::sqrt(dots[s]);
            worst = std::max(worst, bnorm[s] > 0 ? beta[s] / bnorm[s] : 0.0);
            alpha[s] = beta[s] > 0 ? 1.0 / beta[s] : 0.0;
        }
        if (!std::isfinite(worst)) return fail(ctx, FPSA_ENONFINITE, "non-finite GMRES residual");
        if (worst < tol) { status = FPSA_OK; break; }
        rc = gm_combine(ctx, V, &alpha, V, 0, coef);  // V_0 = r / beta
        if (rc) return rc;
        // Arnoldi with classical Gram-Schmidt applied twice, Givens rotations per system
        std::vector<double> H((size_t)nsys * (m + 1) * m, 0.0), cs((size_t)nsys * m), sn((size_t)nsys * m),
            gvec((size_t)nsys * (m + 1), 0.0);
        for (int s = 0; s < nsys; ++s) gvec[(size_t)s * (m + 1)] = beta[s];
        auto Hs = [&](int s, int i, int j) -> double & { return H[((size_t)s * (m + 1) + i) * m + j]; };
        int j = 0, jdone = 0;
        for (j = 0; j < m && it < max_it; ++j) {
            rc = gm_apply(ctx, p, V + (size_t)j * n, w);
            if (rc) return rc;
            ++sweeps;
            std::vector<double> hsum((size_t)nsys * (j + 1), 0.0);
            for (int pass = 0; pass < 2; ++pass) {
                rc = gm_dots(ctx, V, j + 1, w, dots);
                if (rc) return rc;
                std::vector<double> neg(dots.size());
                for (size_t q = 0; q < dots.size(); ++q) {
                    neg[q] = -dots[q];
                    hsum[q] += dots[q];
                }
                rc = gm_combine(ctx, w, &c1, V, j + 1, neg);
                if (rc) return rc;
            }
            rc = gm_dots(ctx, w, 1, w, dots);
            if (rc) return rc;
            worst = 0.0;
            for (int s = 0; s < nsys; ++s) {
                const double hnext = std::sqrt(dots[s]);
                for (int i = 0; i <= j; ++i) Hs(s, i, j) = hsum[(size_t)s * (j + 1) + i];
                for (int i = 0; i < j; ++i) {
                    const double c = cs[(size_t)s * m + i], sv = sn[(size_t)s * m + i];
                    const double t = c * Hs(s, i, j) + sv * Hs(s, i + 1, j);
                    Hs(s, i + 1, j) = -sv * Hs(s, i, j) + c * Hs(s, i + 1, j);
                    Hs(s, i, j) = t;
                }
                const double den = std::hypot(Hs(s, j, j), hnext);
                const double c = den > 0 ? Hs(s, j, j) / den : 1.0, sv = den > 0 ? hnext / den : 0.0;
                cs[(size_t)s * m + j] = c;
                sn[(size_t)s * m + j] = sv;
                Hs(s, j, j) = den;
                double *gs = &gvec[(size_t)s * (m + 1)];
                gs[j + 1] = -sv * gs[j];
                gs[j] = c * gs[j];
                worst = std::max(worst, bnorm[s] > 0 ? std::fabs(gs[j + 1]) / bnorm[s] : 0.0);
                alpha[s] = hnext > 0 ? 1.0 / hnext : 0.0;
            }
            ++it;
            jdone = j + 1;
            if (!std::isfinite(worst)) return fail(ctx, FPSA_ENONFINITE, "non-finite GMRES residual");
            if (worst < tol) break;
            if (j + 1 < m) {  // V_{j+1} = w / h_{j+1,j}
                rc = gm_combine(ctx, V + (size_t)(j + 1) * n, &alpha, V, 0, coef, (const T *)w);
                if (rc) return rc;
            }
        }
        // u += sum_i y_i V_i, y from the triangular least-squares system per system
        std::vector<double> y((size_t)nsys * jdone, 0.0);
        for (int s = 0; s < nsys; ++s)
            for (int i = jdone - 1; i >= 0; --i) {
                double acc = gvec[(size_t)s * (m + 1) + i];
                for (int k2 = i + 1; k2 < jdone; ++k2) acc -= Hs(s, i, k2) * y[(size_t)s * jdone + k2];
                y[(size_t)s * jdone + i] = Hs(s, i, i) != 0.0 ? acc / Hs(s, i, i) : 0.0;
            }
        rc = gm_combine(ctx, u, &c1, V, jdone, y);
        if (rc) return rc;
        if (worst < tol) { status = FPSA_OK; break; }
    }
    // phi = (I + C) u
    rc = gm_fp_rhs(ctx, p, (const T *)u, p.rhs);
    if (rc) return rc;
    rc = bcr_solve(ctx, p, p.rhs);
    if (rc) return rc;
    rc = gm_update(ctx, p, (const T *)p.ybuf, (const T *)u, p.phi);
    if (rc) return rc;
    return status;
}

// GMRES(m) with right FPSA preconditioning, FP64 (Sec. 4).
int solve_gmres(fpsa_ctx *ctx, const fpsa_opts &o, const double *phi0, int mem, double *phi_out, fpsa_stats &stats,
                const double *Qm, const double *Qa, const double *inc) {
    PathBuffers<double> &p = ctx->p64;
    const Geometry &g = ctx->geo;
    const size_t ncol = (size_t)g.R * g.sumK * 2;
    if (phi0) return fail(ctx, FPSA_ENOTSUP, "GMRES starts from zero (phi0 not supported)");
    int it = 0, sweeps = 0;
    double worst = INFINITY;
    const int status = gmres_core<double>(ctx, p, o.restart > 0 ? o.restart : 30, o.tol, o.max_iterations, Qm, Qa,
                                          inc, it, sweeps, worst);
    if (status != FPSA_OK && status != FPSA_ENOTCONV) return status;
    stats.iterations = it;
    stats.outer_iterations = it;
    stats.sweeps = sweeps;
    stats.rel_change = worst;
    if (phi_out)
        CK(cudaMemcpy2DAsync(phi_out, g.L1 * sizeof(double), p.phi, g.N * sizeof(double), g.L1 * sizeof(double), ncol,
                             mem == FPSA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (status == FPSA_ENOTCONV)
        fail(ctx, FPSA_ENOTCONV, "GMRES not converged after " + std::to_string(it) + " iterations");
    return status;
}

}  // namespace

// One device-side loop test of a batch graph (Eq. iterate): after a refinement step's
// residual, count the step and keep looping while the relative change of phi_0 is at
// least tol, no bounded wait ran out, the change is finite and fewer than max_steps
// corrections were made.
__global__ void k_batch_cond(cudaGraphConditionalHandle handle, const double *__restrict__ e,
                             const int *__restrict__ err, int *__restrict__ steps, double tol, int max_steps) {
    if (threadIdx.x == 0) {
        const int s = ++*steps;
        const double v = *e;
        const bool go = *err == 0 && !isnan(v) && !(v < tol) && s < max_steps;
        cudaGraphSetConditional(handle, go ? 1u : 0u);
    }
}

// Capture one context's MIXED solve into graph G as a prologue node (zero state,
// first residual) followed by a while node whose body is one refinement step
// (inner FP32 iterations, accumulation, residual, loop test). Launches go to the
// capture stream cs; the context's own stream and profiler are restored afterwards.
int capture_mixed_loop(fpsa_ctx *ctx, const MixedPlan &mp, const fpsa_opts &o, int inner, cudaGraph_t G,
                       cudaStream_t cs) {
    const Geometry &g = ctx->geo;
    PathBuffers<double> &p = ctx->p64;
    const bool fpsa = o.method == FPSA_METHOD_FPSA;
    const double *inc = ctx->has_inc ? ctx->d_inc : nullptr;
    cudaStream_t own = ctx->stream;
    const bool prof = ctx->prof_on;
    ctx->stream = cs;
    ctx->prof_on = false;
    g_plain_launch = true;
    int rc = FPSA_OK;
    cudaGraph_t pg = nullptr;
    cudaGraphNode_t pnode = nullptr, wnode = nullptr;
    auto restore = [&]() {
        ctx->stream = own;
        ctx->prof_on = prof;
        g_plain_launch = false;
    };
    auto end_capture_on_error = [&]() {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(cs, &junk);
        if (junk) cudaGraphDestroy(junk);
        (void)cudaGetLastError();
    };
    // prologue: zero state, first residual (its change is never tested: no phi0)
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        restore();
        return fail(ctx, FPSA_ECUDA, "batch graph: stream capture refused");
    }
    int sw = 0;
    if (cudaMemsetAsync(ctx->d_dev_err, 0, sizeof(int), cs) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_steps, 0, sizeof(int), cs) != cudaSuccess ||
        cudaMemsetAsync(p.phi, 0, mp.nang * sizeof(double), cs) != cudaSuccess ||
        cudaMemsetAsync(p.psi, 0, mp.nang * sizeof(double), cs) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_conv, 0, (size_t)g.R * g.B * 2 * sizeof(unsigned long long), cs) != cudaSuccess) {
        end_capture_on_error();
        restore();
        return fail(ctx, FPSA_ECUDA, "batch graph: capture of the prologue failed");
    }
    rc = mixed_residual_launch(ctx, mp, p.Q, nullptr, inc, false);
    if (rc) {
        end_capture_on_error();
        restore();
        return rc;
    }
    if (cudaStreamEndCapture(cs, &pg) != cudaSuccess || !pg) {
        (void)cudaGetLastError();
        restore();
        return fail(ctx, FPSA_ECUDA, "batch graph: capture of the prologue failed");
    }
    cudaGraphConditionalHandle handle;
    cudaGraphNodeParams cp = {};
    bool ok = cudaGraphAddChildGraphNode(&pnode, G, nullptr, 0, pg) == cudaSuccess;
    cudaGraphDestroy(pg);
    ok = ok && cudaGraphConditionalHandleCreate(&handle, G, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&wnode, G, &pnode, nullptr, 1, &cp) == cudaSuccess;
    }
    if (!ok || cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        (void)cudaGetLastError();
        restore();
        return fail(ctx, FPSA_ENOTSUP, "batch graph: conditional while node refused");
    }
    // body: the BCR solves alternate their counter halves; with an odd number of them per
    // step the first one's half is zeroed at the top of the step (it is otherwise zeroed
    // by the step before)
    if (fpsa && inner % 2 == 1) {
        const int par = ctx->flow_parity;
        ok = cudaMemsetAsync(ctx->d_flow + 2 * ctx->flow_n * par, 0, 2 * ctx->flow_n * sizeof(int), cs) == cudaSuccess;
        if (ctx->d_tcs_queue) ok = ok && cudaMemsetAsync(ctx->d_tcs_queue + par, 0, sizeof(int), cs) == cudaSuccess;
        if (!ok) {
            end_capture_on_error();
            restore();
            return fail(ctx, FPSA_ECUDA, "batch graph: capture of the loop body failed");
        }
    }
    rc = mixed_inner_launch(ctx, mp, inner, fpsa, sw);
    if (!rc) rc = mixed_residual_launch(ctx, mp, p.Q, nullptr, inc, false);
    if (!rc) {
        k_batch_cond<<<1, 32, 0, cs>>>(handle, ctx->d_result, ctx->d_dev_err, ctx->d_steps, o.tol, o.max_iterations);
        if (cudaGetLastError() != cudaSuccess) rc = fail(ctx, FPSA_ECUDA, "batch graph: loop test launch failed");
    }
    if (rc) {
        end_capture_on_error();
        restore();
        return rc;
    }
    cudaGraph_t body_out = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &body_out);
    restore();
    if (ce != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, FPSA_ENOTSUP, std::string("batch graph: loop body capture failed: ") + cudaGetErrorString(ce));
    }
    return FPSA_OK;
}

extern "C" {

const char *fpsa_strerror(int code) {
    switch (code) {
        case FPSA_OK: return "ok";
        case FPSA_EINVAL: return "invalid argument";
        case FPSA_ENOMEM: return "device out of memory";
        case FPSA_ENONFINITE: return "non-finite value";
        case FPSA_ENOTCONV: return "iteration did not converge";
        case FPSA_EPIVOT: return "FP block factorization failed (pivot or growth)";
        case FPSA_ETIMEOUT: return "bounded device wait timed out";
        case FPSA_ECUDA: return "CUDA runtime error";
        case FPSA_ENOTSUP: return "configuration not supported by the library";
        case FPSA_ESTATE: return "call order violated";
        default: return "unknown status";
    }
}

const char *fpsa_last_error(const fpsa_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void fpsa_destroy(fpsa_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (void *p : ctx->allocs) cudaFree(p);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->ad_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->h_result) cudaFreeHost(ctx->h_result);
    if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
    delete ctx;
}

int fpsa_create(fpsa_ctx **out, const fpsa_desc *d) {
    if (!out) return FPSA_EINVAL;
    *out = nullptr;
    if (!d || !d->n_cells || !d->h) return FPSA_EINVAL;
    if (d->n_instances < 1 || d->n_rhs < 1 || d->n_ordinates < 2 || d->n_ordinates % 2 ||
        d->n_moments < 1 || d->n_moments > d->n_ordinates)
        return FPSA_EINVAL;
    if (d->laplacian != FPSA_LAPLACIAN_MPD && d->laplacian != FPSA_LAPLACIAN_WFD) return FPSA_EINVAL;
    if (d->precision != FPSA_PRECISION_FP64 && d->precision != FPSA_PRECISION_MIXED) return FPSA_EINVAL;
    if (d->n_ordinates > FPSA_MAX_ORDINATES) return FPSA_ENOTSUP;
    long long sumK = 0;
    for (int b = 0; b < d->n_instances; ++b) {
        if (d->n_cells[b] < 1) return FPSA_EINVAL;
        sumK += d->n_cells[b];
    }
    if (sumK > (1ll << 30)) return FPSA_EINVAL;
    for (long long c = 0; c < sumK; ++c)
        if (!(d->h[c] > 0.0) || !std::isfinite(d->h[c])) return FPSA_EINVAL;
    bool any_reflect = false;
    if (d->bc)
        for (int e = 0; e < 2 * d->n_instances; ++e) {
            if (d->bc[e] != FPSA_BC_VACUUM && d->bc[e] != FPSA_BC_REFLECT) return FPSA_EINVAL;
            any_reflect |= d->bc[e] == FPSA_BC_REFLECT;
        }

    fpsa_ctx *ctx = new fpsa_ctx();
    ctx->laplacian = d->laplacian;
    ctx->precision = d->precision;
    ctx->device = d->device;
    ctx->stream = static_cast<cudaStream_t>(d->stream);
    auto bail = [&](int rc) {
        fpsa_destroy(ctx);
        return rc;
    };
    if (cudaSetDevice(d->device) != cudaSuccess) return bail(FPSA_ECUDA);
    build_tables(d->n_ordinates, d->n_moments, d->laplacian, ctx->tab);
    build_geometry(d->n_cells, d->n_instances, d->n_ordinates, d->n_moments, d->n_rhs, ctx->geo);
    const Geometry &g = ctx->geo;
    int rc = [&]() -> int {
        CK(dalloc(ctx, &ctx->d_off, g.B));
        CK(dalloc(ctx, &ctx->d_K, g.B));
        CK(dalloc(ctx, &ctx->d_cell_inst, g.sumK));
        CK(dalloc(ctx, &ctx->d_slot_base, g.sumK));
        CK(dalloc(ctx, &ctx->d_mu, g.N));
        CK(dalloc(ctx, &ctx->d_Afp, (size_t)g.N * g.N));
        CK(dalloc(ctx, &ctx->d_h, g.sumK));
        CK(dalloc(ctx, &ctx->d_sigma_t, g.sumK));
        CK(dalloc(ctx, &ctx->d_s0, g.sumK));
        CK(dalloc(ctx, &ctx->d_s1, g.sumK));
        CK(dalloc(ctx, &ctx->d_conv, (size_t)g.R * g.B * 2));
        CK(dalloc(ctx, &ctx->d_in_st, g.sumK));
        CK(dalloc(ctx, &ctx->d_in_ss, (size_t)g.sumK * g.L1));
        CK(dalloc(ctx, &ctx->d_in_q, (size_t)g.R * g.sumK * 2 * g.L1));
        CK(dalloc(ctx, &ctx->d_xs_err, 2));
        CK(dalloc(ctx, &ctx->d_dev_err, 2));
        {
            const int e0[2] = {0, (int)kFlowSpinLimit};
            CK(cudaMemcpy(ctx->d_dev_err, e0, sizeof(e0), cudaMemcpyHostToDevice));
        }
        CK(cudaMallocHost(&ctx->h_flag, sizeof(int)));
        {
            const int nchunk = (g.R + solve_rc(g.R) - 1) / solve_rc(g.R);
            ctx->flow_n = (size_t)nchunk * g.sumK;
            CK(dalloc(ctx, &ctx->d_flow, 4 * ctx->flow_n));
            CK(cudaMemset(ctx->d_flow, 0, 4 * ctx->flow_n * sizeof(int)));
            CK(dalloc(ctx, &ctx->d_factor_cnt, (size_t)g.sumK + 1));  // + the tensor-core factorization's queue
        }
        CK(dalloc(ctx, &ctx->d_growth, 1));
        CK(dalloc(ctx, &ctx->d_status, 1));
        CK(dalloc(ctx, &ctx->d_result, 2));
        CK(dalloc(ctx, &ctx->d_steps, 1));
        CK(cudaMallocHost(&ctx->h_result, 2 * sizeof(double)));
        CK(cudaMemcpy(ctx->d_off, g.off.data(), g.B * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_K, g.K.data(), g.B * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_cell_inst, g.cell_inst.data(), g.sumK * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_slot_base, g.slot_base.data(), g.sumK * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_mu, ctx->tab.mu.data(), g.N * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_Afp, ctx->tab.Afp.data(), (size_t)g.N * g.N * sizeof(double), cudaMemcpyHostToDevice));
        {
            std::vector<float> a32(ctx->tab.Afp.begin(), ctx->tab.Afp.end());
            CK(dalloc(ctx, &ctx->d_Afp32, a32.size()));
            CK(cudaMemcpy(ctx->d_Afp32, a32.data(), a32.size() * sizeof(float), cudaMemcpyHostToDevice));
            std::vector<float> m32(ctx->tab.mu.begin(), ctx->tab.mu.end());
            CK(dalloc(ctx, &ctx->d_mu32, m32.size()));
            CK(cudaMemcpy(ctx->d_mu32, m32.data(), m32.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
        CK(cudaMemcpy(ctx->d_h, d->h, g.sumK * sizeof(double), cudaMemcpyHostToDevice));
        if (any_reflect) {
            CK(dalloc(ctx, &ctx->d_bc, 2 * g.B));
            CK(cudaMemcpy(ctx->d_bc, d->bc, 2 * g.B * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
        ctx->d_levels.assign(g.n_levels, nullptr);
        for (int l = 0; l < g.n_levels; ++l) {
            CK(dalloc(ctx, &ctx->d_levels[l], g.levels[l].size()));
            CK(cudaMemcpy(ctx->d_levels[l], g.levels[l].data(), g.levels[l].size() * sizeof(BcrItem),
                          cudaMemcpyHostToDevice));
        }
        CK(dalloc(ctx, &ctx->d_roots, g.B));
        CK(cudaMemcpy(ctx->d_roots, g.roots.data(), g.B * sizeof(BcrItem), cudaMemcpyHostToDevice));
        {
            const size_t nang = (size_t)g.R * g.sumK * 2 * g.N;
            CK(dalloc(ctx, &ctx->d_phi_fwd, nang));
            CK(dalloc(ctx, &ctx->d_adj_src, nang));
            CK(dalloc(ctx, &ctx->d_gphi, nang));
            CK(dalloc(ctx, &ctx->d_Pm, (size_t)g.N * g.N));
            CK(dalloc(ctx, &ctx->d_cJ, g.N));
            CK(dalloc(ctx, &ctx->d_J, (size_t)g.R * g.B));
            CK(dalloc(ctx, &ctx->d_grad_t, g.sumK));
            CK(dalloc(ctx, &ctx->d_grad_s, (size_t)g.sumK * g.L1));
            // P_l(mu_n) = D[l][n] / w_n
            std::vector<double> Pm((size_t)g.N * g.N), cJ(g.N, 0.0);
            for (int n = 0; n < g.N; ++n)
                for (int l = 0; l < g.N; ++l) {
                    const double P = ctx->tab.D[(size_t)l * g.N + n] / ctx->tab.w[n];
                    Pm[(size_t)n * g.N + l] = (l & 1) ? -P : P;
                    if (ctx->tab.mu[n] > 0.0) cJ[l] += ctx->tab.w[n] * ctx->tab.mu[n] * (l + 0.5) * P;
                }
            CK(cudaMemcpy(ctx->d_Pm, Pm.data(), Pm.size() * sizeof(double), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(ctx->d_cJ, cJ.data(), cJ.size() * sizeof(double), cudaMemcpyHostToDevice));
        }
        {
            std::vector<BcrItem> all;
            for (int l = 0; l < g.n_levels; ++l) all.insert(all.end(), g.levels[l].begin(), g.levels[l].end());
            all.insert(all.end(), g.roots.begin(), g.roots.end());
            CK(dalloc(ctx, &ctx->d_items_all, all.size()));
            CK(cudaMemcpy(ctx->d_items_all, all.data(), all.size() * sizeof(BcrItem), cudaMemcpyHostToDevice));
            int nsm = 0, per_sm = 0;
            CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
            const int RC = solve_rc(g.R);
            CK(raise_smem_limit((const void *)coop_kernel<float>(RC, g.N), (int)solve_smem<float>(g.N, RC)));
            CK(raise_smem_limit((const void *)coop_kernel<double>(RC, g.N), (int)solve_smem<double>(g.N, RC)));
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coop_kernel<float>(RC, g.N),
                                                             solve_threads<float>(g.N), solve_smem<float>(g.N, RC)));
            ctx->solve_per_sm[0] = std::max(1, per_sm);
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coop_kernel<double>(RC, g.N),
                                                             solve_threads<double>(g.N), solve_smem<double>(g.N, RC)));
            ctx->solve_per_sm[1] = std::max(1, per_sm);
            ctx->n_sm = nsm;
            for (int e = 0; e < 2; ++e) {
                const void *fk = e ? factor_kernel<double>(2 * g.N) : factor_kernel<float>(2 * g.N);
                const size_t fsm = e ? schur_smem<double>(g.N) : schur_smem<float>(g.N);
                int fper = 0;
                if (fk) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fper, fk, 512, fsm));
                ctx->factor_grid[e] = (fk && fper > 0) ? nsm : 0;  // one block per SM
            }
            if (2 * g.N == tcf::kN2 && ctx->precision == FPSA_PRECISION_MIXED) {
                // up to 4 CTAs per SM (4 x 128 TMEM columns), as occupancy allows
                // 4 CTAs per SM (the shared memory of each admits no more, so their 4 x 128
                // TMEM columns fit; the runtime's occupancy estimate for kernels that allocate
                // tensor memory is one CTA per SM, so it is not consulted: the launch is not
                // cooperative and takes its items from a queue)
                CK(raise_smem_limit((const void *)k_bcr_factor_tc, (int)tcf::Smem::total));
                CK(cudaFuncSetAttribute((const void *)k_bcr_factor_tc,
                                        cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
                ctx->factor_tc_grid = 4 * nsm;
            }
            if ((2 * g.N == 256 || 2 * g.N == 512) && ctx->precision == FPSA_PRECISION_MIXED) {
                // the recursive block inversion's GEMMs (h = 128, 256) on the tensor cores:
                // two (h = 256) or three (h = 128) CTAs per SM by shared memory, so their
                // tensor-memory columns always fit
                CK(raise_smem_limit((const void *)k_bgemm_tc<256>, (int)bgt::smem_bytes(256)));
                CK(raise_smem_limit((const void *)k_bgemm_tc<128>, (int)bgt::smem_bytes(128)));
                ctx->bgemm_tc_able = true;
            }
            if (ctx->precision == FPSA_PRECISION_MIXED && tcs::applies(2 * g.N, g.R)) {
                // the tensor-core BCR solve: a split copy of the factors, two CTAs per SM
                ctx->tcs_rt = tcs::rhs_tile(g.R);
                ctx->tcs_grid = 2 * nsm;
                CK(dalloc(ctx, &ctx->d_tcs_A, (size_t)g.sumK * tcs::cell_bytes(2 * g.N)));
                CK(dalloc(ctx, &ctx->d_tcs_g, (size_t)ctx->tcs_grid * ctx->tcs_rt * g.N));
                CK(dalloc(ctx, &ctx->d_tcs_queue, 2));
                CK(cudaMemset(ctx->d_tcs_queue, 0, 2 * sizeof(int)));
                const void *k = tcs_kernel(ctx->tcs_rt);
                CK(raise_smem_limit(k, (int)tcs::Plan::make(2 * g.N, ctx->tcs_rt).total));
                CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
            }
            for (int e = 0; e < 2; ++e) {
                LevelTable &lv = ctx->lvt[e];
                lv.n_levels = g.n_levels;
                lv.n_roots = g.B;
                lv.n_stages = e ? solve_stages<double>(g.N, RC) : solve_stages<float>(g.N, RC);
                plan_coarse(lv, g, e ? (int)sizeof(double) : (int)sizeof(float));
                int off = 0;
                for (int l = 0; l <= g.n_levels; ++l) {
                    lv.off[l] = off;
                    off += l < g.n_levels ? (int)g.levels[l].size() : g.B;
                }
            }
            ctx->sweep_cpt = sweep_cells_per_thread(g);
            plan_solve_shape(ctx);
        }
        if (ctx->precision == FPSA_PRECISION_FP64) return alloc_path(ctx, ctx->p64, true);
        int r2 = alloc_path(ctx, ctx->p64, false);
        if (r2) return r2;
        r2 = alloc_path(ctx, ctx->p32, true);
        if (r2) return r2;
        r2 = setup_residual_tc(ctx);
        if (r2) return r2;
        return setup_tc(ctx);
    }();
    if (rc != FPSA_OK) {
        g_create_error = ctx->err;
        return bail(rc);
    }
    g_create_error.clear();
    *out = ctx;
    return FPSA_OK;
}

int fpsa_set_xs(fpsa_ctx *ctx, const double *sigma_t, const double *sigma_s, const double *q, int32_t mem) {
    if (!ctx) return FPSA_EINVAL;
    if (!sigma_t || !sigma_s || !q) return fail(ctx, FPSA_EINVAL, "null input pointer");
    if (mem != FPSA_MEM_HOST && mem != FPSA_MEM_DEVICE) return fail(ctx, FPSA_EINVAL, "bad mem kind");
    CK(cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    const Geometry &g = ctx->geo;
    const size_t nss = (size_t)g.sumK * g.L1, nq = (size_t)g.R * g.sumK * 2 * g.L1;
    cudaStream_t s = ctx->stream;
    ctx->xs_ready = false;
    ctx->fwd_ready = false;
    const double *st_in = sigma_t, *ss_in = sigma_s, *q_in = q;
    if (mem == FPSA_MEM_HOST) {  // one upload of the caller's arrays; conversion happens on the device
        CK(cudaMemcpyAsync(ctx->d_in_st, sigma_t, g.sumK * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->d_in_ss, sigma_s, nss * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->d_in_q, q, nq * sizeof(double), cudaMemcpyHostToDevice, s));
        st_in = ctx->d_in_st;
        ss_in = ctx->d_in_ss;
        q_in = ctx->d_in_q;
    }
    const int big = 0x7fffffff;
    CK(cudaMemcpyAsync(ctx->d_xs_err, &big, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->d_xs_err + 1, 0, sizeof(int), s));
    CK(cudaMemsetAsync(ctx->d_growth, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s));
    CK(cudaMemsetAsync(ctx->d_dev_err, 0, sizeof(int), s));
    const bool mixed = ctx->precision == FPSA_PRECISION_MIXED;
    {
        Launch L_(ctx, FPSA_PHASE_ASSEMBLE);
        k_prepare_xs<<<4 * 152, 256, 0, s>>>(st_in, ss_in, q_in, g.N, g.L1, g.sumK, g.R, ctx->p64.sigma_s,
                                              mixed ? ctx->p32.sigma_s : nullptr, ctx->p64.Q, nullptr, ctx->d_sigma_t,
                                              ctx->d_s0, ctx->d_s1, ctx->d_xs_err, ctx->d_xs_err + 1);
    }
    CK(cudaGetLastError());
    int err[2];
    CK(cudaMemcpyAsync(err, ctx->d_xs_err, sizeof(err), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (err[0] != big) {
        const int c = err[0] / 4, check = err[0] % 4;
        if (check == 0) return fail(ctx, FPSA_EINVAL, "sigma_t must be finite and > 0 (cell " + std::to_string(c) + ")");
        if (check == 1) return fail(ctx, FPSA_ENONFINITE, "non-finite sigma_s at cell " + std::to_string(c));
        return fail(ctx, FPSA_EINVAL, "need 0 <= sigma_s0 <= sigma_t (cell " + std::to_string(c) + ")");
    }
    if (err[1]) return fail(ctx, FPSA_ENONFINITE, "non-finite source moment");
    int rc = mixed ? setup_path(ctx, ctx->p32, true) : setup_path(ctx, ctx->p64, true);
    if (rc) return rc;
    unsigned long long growth = 0;
    int status = 0, dev_err = 0;
    CK(cudaMemcpyAsync(&growth, ctx->d_growth, sizeof(growth), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&status, ctx->d_status, sizeof(status), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&dev_err, ctx->d_dev_err, sizeof(dev_err), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (dev_err) return fail(ctx, FPSA_ETIMEOUT, "a bounded device wait of the factorization ran out");
    double gr;
    std::memcpy(&gr, &growth, sizeof(gr));
    ctx->pivot_growth = gr;
    ctx->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (status || !std::isfinite(gr) || gr > ctx->growth_limit)
        return fail(ctx, FPSA_EPIVOT, "FP block factorization failed: growth " + std::to_string(gr));
    ctx->xs_ready = true;
    return FPSA_OK;
}

int fpsa_set_incident(fpsa_ctx *ctx, const double *psi_inc, int32_t mem) {
    if (!ctx) return FPSA_EINVAL;
    if (mem != FPSA_MEM_HOST && mem != FPSA_MEM_DEVICE) return fail(ctx, FPSA_EINVAL, "bad mem kind");
    CK(cudaSetDevice(ctx->device));
    const Geometry &g = ctx->geo;
    const size_t n = (size_t)g.R * g.B * 2 * g.N;
    ctx->fwd_ready = false;
    if (!psi_inc) {
        ctx->has_inc = false;
        return FPSA_OK;
    }
    if (mem == FPSA_MEM_HOST)
        for (size_t i = 0; i < n; ++i)
            if (!std::isfinite(psi_inc[i])) return fail(ctx, FPSA_ENONFINITE, "non-finite incoming flux");
    if (!ctx->d_inc) CK(dalloc(ctx, &ctx->d_inc, n));
    CK(cudaMemcpyAsync(ctx->d_inc, psi_inc, n * sizeof(double),
                       mem == FPSA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->has_inc = true;
    return FPSA_OK;
}

int fpsa_set_limits(fpsa_ctx *ctx, int64_t wait_polls, double growth_limit) {
    if (!ctx) return FPSA_EINVAL;
    if (wait_polls < 0 || wait_polls > 0x7fffffffll) return fail(ctx, FPSA_EINVAL, "wait_polls outside [0, 2^31 - 1]");
    if (!(growth_limit >= 0.0)) return fail(ctx, FPSA_EINVAL, "growth_limit must be >= 0");
    CK(cudaSetDevice(ctx->device));
    const int limit = wait_polls > 0 ? (int)wait_polls : (int)kFlowSpinLimit;
    CK(cudaMemcpyAsync(ctx->d_dev_err + 1, &limit, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->growth_limit = growth_limit > 0.0 ? growth_limit : kGrowthLimit;
    return FPSA_OK;
}

int fpsa_profile_enable(fpsa_ctx *ctx, int32_t on) {
    if (!ctx) return FPSA_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < FPSA_N_PHASES; ++k) ctx->launches[k] = 0;
    ctx->ev_rec.clear();
    ctx->ev_used = 0;
    ctx->prof_on = on != 0;
    return FPSA_OK;
}

int fpsa_profile_read(fpsa_ctx *ctx, fpsa_profile *out) {
    if (!ctx || !out) return FPSA_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    std::memset(out, 0, sizeof(*out));
    for (int k = 0; k < FPSA_N_PHASES; ++k) out->launches[k] = ctx->launches[k];
    for (const auto &r : ctx->ev_rec) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev_pool[r.second], ctx->ev_pool[r.second + 1]));
        out->ms[r.first] += ms;
        out->timed[r.first] += 1;
    }
    return FPSA_OK;
}

int fpsa_solve(fpsa_ctx *ctx, const fpsa_opts *opts, double *phi, const double *phi0, int32_t mem,
               fpsa_stats *stats) {
    if (!ctx) return FPSA_EINVAL;
    if (!phi) return fail(ctx, FPSA_EINVAL, "null phi");
    if (mem != FPSA_MEM_HOST && mem != FPSA_MEM_DEVICE) return fail(ctx, FPSA_EINVAL, "bad mem kind");
    if (!ctx->xs_ready) return fail(ctx, FPSA_ESTATE, "fpsa_set_xs must succeed before fpsa_solve");
    fpsa_opts o{FPSA_METHOD_FPSA, 10000, 1e-10, 0, 0.0, 1, 0, 0};
    if (opts) o = *opts;
    if (o.method != FPSA_METHOD_SI && o.method != FPSA_METHOD_FPSA && o.method != FPSA_METHOD_GMRES)
        return fail(ctx, FPSA_EINVAL, "bad method");
    if (o.max_iterations < 1 || !(o.tol >= 0.0) || o.restart < 0) return fail(ctx, FPSA_EINVAL, "bad max_iterations / tol / restart");
    CK(cudaSetDevice(ctx->device));
    fpsa_stats s{};
    const auto t0 = std::chrono::steady_clock::now();
    ctx->fwd_ready = false;
    const double *inc = ctx->has_inc ? ctx->d_inc : nullptr;
    int rc = o.method == FPSA_METHOD_GMRES && ctx->precision == FPSA_PRECISION_FP64
                 ? solve_gmres(ctx, o, phi0, mem, phi, s, ctx->p64.Q, nullptr, inc)
                 : ctx->precision == FPSA_PRECISION_FP64
                 ? solve_fp64(ctx, ctx->p64, o, phi0, mem, phi, s, (const double *)ctx->p64.Q, (const double *)nullptr,
                              inc)
                 : solve_mixed(ctx, o, phi0, mem, phi, s, ctx->p64.Q, nullptr, inc);
    if (rc == FPSA_OK) {
        // keep the converged moments (all N) for fpsa_adjoint
        const size_t nang = (size_t)ctx->geo.R * ctx->geo.sumK * 2 * ctx->geo.N;
        CK(cudaMemcpyAsync(ctx->d_phi_fwd, ctx->p64.phi, nang * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->fwd_ready = true;
    }
    s.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    s.status = rc;
    s.setup_ms = ctx->setup_ms;
    s.pivot_growth = ctx->pivot_growth;
    s.cell_angles = (double)ctx->geo.sumK * ctx->geo.N * ctx->geo.R * s.sweeps;
    if (stats) *stats = s;
    return rc;
}

int fpsa_solve_batch(fpsa_ctx *const *ctxs, int32_t n, const fpsa_opts *opts, double *const *phi, int32_t mem,
                     fpsa_stats *stats) {
    if (!ctxs || n < 1) return FPSA_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return FPSA_EINVAL;
    fpsa_ctx *c0 = ctxs[0];
    if (!phi) return fail(c0, FPSA_EINVAL, "null phi array");
    if (mem != FPSA_MEM_HOST && mem != FPSA_MEM_DEVICE) return fail(c0, FPSA_EINVAL, "bad mem kind");
    fpsa_opts o{FPSA_METHOD_FPSA, 10000, 1e-10, 0, 0.0, 1, 0, 0};
    if (opts) o = *opts;
    if (o.method != FPSA_METHOD_SI && o.method != FPSA_METHOD_FPSA)
        return fail(c0, FPSA_ENOTSUP, "fpsa_solve_batch: method must be SI or FPSA");
    if (o.max_iterations < 1 || !(o.tol >= 0.0)) return fail(c0, FPSA_EINVAL, "bad max_iterations / tol");
    for (int i = 0; i < n; ++i) {
        fpsa_ctx *c = ctxs[i];
        if (!phi[i]) return fail(c, FPSA_EINVAL, "null phi");
        if (c->precision != FPSA_PRECISION_MIXED)
            return fail(c, FPSA_ENOTSUP, "fpsa_solve_batch: MIXED precision contexts only");
        if (c->device != c0->device) return fail(c, FPSA_EINVAL, "fpsa_solve_batch: contexts on different devices");
        if (!c->xs_ready) return fail(c, FPSA_ESTATE, "fpsa_set_xs must succeed before fpsa_solve_batch");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(c, FPSA_EINVAL, "fpsa_solve_batch: a context appears twice");
    }
    fpsa_ctx *ctx = c0;  // error messages of CUDA failures go to the first context
    CK(cudaSetDevice(c0->device));
    const auto t0 = std::chrono::steady_clock::now();
    const int inner = o.inner_iterations > 0 ? o.inner_iterations : 4;
    std::vector<MixedPlan> plans(n);
    for (int i = 0; i < n; ++i) {
        ctxs[i]->fwd_ready = false;
        int rc = mixed_plan(ctxs[i], o, plans[i]);
        if (rc) return rc;
        CK(cudaStreamSynchronize(ctxs[i]->stream));  // earlier work of every context is done
    }
    cudaStream_t cs = nullptr;
    cudaGraph_t G = nullptr;
    cudaGraphExec_t X = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    auto cleanup = [&]() {
        if (X) cudaGraphExecDestroy(X);
        if (G) cudaGraphDestroy(G);
        if (cs) cudaStreamDestroy(cs);
    };
#define CKB(x)                                                                             \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            cudaStreamSynchronize(cs);                                                     \
            cleanup();                                                                     \
            return fail(c0, FPSA_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
        }                                                                                  \
    } while (0)
    if (cudaGraphCreate(&G, 0) != cudaSuccess) {
        cleanup();
        return fail(c0, FPSA_ECUDA, "cudaGraphCreate failed");
    }
    for (int i = 0; i < n; ++i) {
        int rc = capture_mixed_loop(ctxs[i], plans[i], o, inner, G, cs);
        if (rc) {
            cleanup();
            return rc;
        }
    }
    cudaError_t ce = cudaGraphInstantiate(&X, G, 0);
    if (ce != cudaSuccess) {
        (void)cudaGetLastError();
        cleanup();
        return fail(c0, FPSA_ENOTSUP, std::string("batch graph instantiation failed: ") + cudaGetErrorString(ce));
    }
    ce = cudaGraphLaunch(X, cs);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(cs);
    if (ce != cudaSuccess) {
        cleanup();
        return fail(c0, FPSA_ECUDA, std::string("batch graph launch failed: ") + cudaGetErrorString(ce));
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    int worst = FPSA_OK;
    for (int i = 0; i < n; ++i) {
        fpsa_ctx *c = ctxs[i];
        const Geometry &g = c->geo;
        double e = 0.0;
        int err = 0, steps = 0;
        CKB(cudaMemcpy(&e, c->d_result, sizeof(double), cudaMemcpyDeviceToHost));
        CKB(cudaMemcpy(&err, c->d_dev_err, sizeof(int), cudaMemcpyDeviceToHost));
        CKB(cudaMemcpy(&steps, c->d_steps, sizeof(int), cudaMemcpyDeviceToHost));
        int status = FPSA_OK;
        if (err) status = fail(c, FPSA_ETIMEOUT, "a bounded device wait ran out (tensor-core contraction or BCR dataflow)");
        else if (std::isnan(e)) status = fail(c, FPSA_ENONFINITE, "non-finite iterate in the batch graph");
        else if (!(e < o.tol))
            status = fail(c, FPSA_ENOTCONV, "not converged after " + std::to_string(o.max_iterations) + " refinement steps");
        const size_t ncol = (size_t)g.R * g.sumK * 2;
        CKB(cudaMemcpy2DAsync(phi[i], g.L1 * sizeof(double), c->p64.phi, g.N * sizeof(double), g.L1 * sizeof(double),
                             ncol, mem == FPSA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, cs));
        if (status == FPSA_OK) {
            CKB(cudaMemcpyAsync(c->d_phi_fwd, c->p64.phi, ncol * g.N * sizeof(double), cudaMemcpyDeviceToDevice, cs));
            c->fwd_ready = true;
        }
        if (stats) {
            fpsa_stats s{};
            s.status = status;
            s.outer_iterations = steps + 1;
            s.sweeps = steps * inner;
            s.iterations = s.sweeps;
            s.rel_change = e;
            s.setup_ms = c->setup_ms;
            s.solve_ms = ms;
            s.pivot_growth = c->pivot_growth;
            s.cell_angles = (double)g.sumK * g.N * g.R * s.sweeps;
            stats[i] = s;
        }
        if (status != FPSA_OK && worst == FPSA_OK) worst = status;
    }
    ce = cudaStreamSynchronize(cs);
    cleanup();
    if (ce != cudaSuccess) return fail(c0, FPSA_ECUDA, cudaGetErrorString(ce));
    return worst;
#undef CKB
}

int fpsa_adjoint(fpsa_ctx *ctx, const fpsa_opts *opts, const double *dJ_dphi, double *dJ_dsigma_t,
                 double *dJ_dsigma_s, double *J, int32_t mem, fpsa_stats *stats) {
    if (!ctx) return FPSA_EINVAL;
    if (!dJ_dsigma_t || !dJ_dsigma_s) return fail(ctx, FPSA_EINVAL, "null gradient output");
    if (mem != FPSA_MEM_HOST && mem != FPSA_MEM_DEVICE) return fail(ctx, FPSA_EINVAL, "bad mem kind");
    if (!ctx->fwd_ready) return fail(ctx, FPSA_ESTATE, "fpsa_adjoint needs a converged fpsa_solve since the last fpsa_set_xs");
    fpsa_opts o{FPSA_METHOD_FPSA, 10000, 1e-12, 0, 0.0, 1, 0, 0};
    if (opts) o = *opts;
    if (o.method != FPSA_METHOD_SI && o.method != FPSA_METHOD_FPSA && o.method != FPSA_METHOD_GMRES)
        return fail(ctx, FPSA_EINVAL, "bad method");
    if (o.max_iterations < 1 || !(o.tol >= 0.0) || o.restart < 0)
        return fail(ctx, FPSA_EINVAL, "bad max_iterations / tol / restart");
    CK(cudaSetDevice(ctx->device));
    const Geometry &g = ctx->geo;
    const int N = g.N, L1 = g.L1;
    const size_t ncol = (size_t)g.R * g.sumK * 2, nang = ncol * N;
    cudaStream_t st = ctx->stream;
    const auto t0 = std::chrono::steady_clock::now();
    const cudaMemcpyKind h2d = mem == FPSA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind d2h = mem == FPSA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (dJ_dphi) {
        CK(cudaMemsetAsync(ctx->d_gphi, 0, nang * sizeof(double), st));
        CK(cudaMemcpy2DAsync(ctx->d_gphi, N * sizeof(double), dJ_dphi, L1 * sizeof(double), L1 * sizeof(double), ncol,
                             h2d, st));
    }
    {
        Launch L_(ctx, FPSA_PHASE_RESIDUAL);
        k_adjoint_source<<<4 * 152, 256, 0, st>>>(dJ_dphi ? ctx->d_gphi : nullptr, ctx->d_Pm, ctx->d_mu, ctx->d_h,
                                                  ctx->d_cell_inst, ctx->d_off, ctx->d_K, N, g.sumK, g.R,
                                                  ctx->d_adj_src);
    }
    {
        Launch L_(ctx, FPSA_PHASE_RESIDUAL);
        k_exit_current<<<dim3(g.B, g.R), 32, 0, st>>>(ctx->d_phi_fwd, ctx->d_cJ, ctx->d_off, ctx->d_K, N, g.sumK, g.B,
                                                       ctx->d_J);
    }
    CK(cudaGetLastError());
    fpsa_stats s{};
    // A x = Pi W^{-1} dJ/dpsi with the forward machinery and factors
    // (homogeneous edges: the given incoming fluxes belong to the forward source only)
    int rc = o.method == FPSA_METHOD_GMRES && ctx->precision == FPSA_PRECISION_FP64
                 ? solve_gmres(ctx, o, nullptr, mem, nullptr, s, nullptr, ctx->d_adj_src, nullptr)
                 : ctx->precision == FPSA_PRECISION_FP64
                 ? solve_fp64(ctx, ctx->p64, o, nullptr, mem, nullptr, s, (const double *)nullptr,
                              (const double *)ctx->d_adj_src, (const double *)nullptr)
                 : solve_mixed(ctx, o, nullptr, mem, nullptr, s, nullptr, ctx->d_adj_src, nullptr);
    if (rc != FPSA_OK) return rc;
    {
        Launch L_(ctx, FPSA_PHASE_RESIDUAL);
        k_adjoint_grad<<<g.sumK, 128, 0, st>>>(ctx->d_phi_fwd, ctx->p64.phi, ctx->d_h, N, L1, g.sumK, g.R,
                                               ctx->d_grad_t, ctx->d_grad_s);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dJ_dsigma_t, ctx->d_grad_t, g.sumK * sizeof(double), d2h, st));
    CK(cudaMemcpyAsync(dJ_dsigma_s, ctx->d_grad_s, (size_t)g.sumK * L1 * sizeof(double), d2h, st));
    if (J) CK(cudaMemcpyAsync(J, ctx->d_J, (size_t)g.R * g.B * sizeof(double), d2h, st));
    CK(cudaStreamSynchronize(st));
    s.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    s.status = rc;
    s.setup_ms = ctx->setup_ms;
    s.pivot_growth = ctx->pivot_growth;
    s.cell_angles = (double)g.sumK * g.N * g.R * s.sweeps;
    if (stats) *stats = s;
    return FPSA_OK;
}


int fpsa_tables(int32_t n_ordinates, int32_t n_moments, int32_t laplacian, double *mu, double *w, double *D,
                double *M, double *A) {
    const int N = n_ordinates, L1 = n_moments;
    if (N < 2 || N % 2 || N > FPSA_MAX_ORDINATES || L1 < 1 || L1 > N) return FPSA_EINVAL;
    if (laplacian != FPSA_LAPLACIAN_MPD && laplacian != FPSA_LAPLACIAN_WFD) return FPSA_EINVAL;
    Tables t;
    build_tables(N, L1, laplacian, t);
    if (mu) std::copy(t.mu.begin(), t.mu.end(), mu);
    if (w) std::copy(t.w.begin(), t.w.end(), w);
    if (D) std::copy(t.D.begin(), t.D.begin() + (size_t)L1 * N, D);  // rows l < L+1
    if (M)
        for (int n = 0; n < N; ++n)
            for (int l = 0; l < L1; ++l) M[(size_t)n * L1 + l] = t.M[(size_t)n * N + l];
    if (A) std::copy(t.Afp.begin(), t.Afp.end(), A);
    return FPSA_OK;
}

int fpsa_get_tuning(const fpsa_ctx *ctx, fpsa_tuning *out) {
    if (!ctx || !out) return FPSA_EINVAL;
    const int e = ctx->precision == FPSA_PRECISION_FP64 ? 1 : 0;
    out->sweep_cells_per_thread = ctx->sweep_cpt;
    out->solve_blocks_per_sm = ctx->coop_grid[e] / std::max(1, ctx->n_sm);
    out->solve_max_slices = ctx->tuning.solve_max_slices > 0 ? ctx->tuning.solve_max_slices : 4;
    out->factor_engine = ((ctx->factor_tc_grid > 0 || ctx->bgemm_tc_able) && ctx->tuning.factor_engine != 1) ? 2 : 1;
    out->solve_engine = (ctx->tcs_rt > 0 && ctx->tuning.solve_engine != 1) ? 2 : 1;
    out->residual_engine =
        (ctx->res_ops.D && (ctx->tuning.residual_engine == 2 ||
                            (ctx->tuning.residual_engine == 0 &&
                             (long long)((ctx->geo.sumK + 63) / 64) * ctx->geo.R >= ctx->n_sm))) ? 2 : 1;
    return FPSA_OK;
}

int fpsa_set_tuning(fpsa_ctx *ctx, const fpsa_tuning *t) {
    if (!ctx) return FPSA_EINVAL;
    fpsa_tuning r{};
    if (t) r = *t;
    if (r.sweep_cells_per_thread < 0 || r.sweep_cells_per_thread > (1 << 20))
        return fail(ctx, FPSA_EINVAL, "sweep_cells_per_thread outside [0, 1 << 20]");
    if (r.solve_blocks_per_sm < 0 || r.solve_blocks_per_sm > 4)
        return fail(ctx, FPSA_EINVAL, "solve_blocks_per_sm outside [0, 4]");
    if (r.solve_max_slices != 0 && r.solve_max_slices != 1 && r.solve_max_slices != 2 && r.solve_max_slices != 4)
        return fail(ctx, FPSA_EINVAL, "solve_max_slices not 0, 1, 2 or 4");
    if (r.factor_engine < 0 || r.factor_engine > 2) return fail(ctx, FPSA_EINVAL, "factor_engine not 0, 1 or 2");
    if (r.factor_engine == 2 && ctx->factor_tc_grid == 0 && !ctx->bgemm_tc_able)
        return fail(ctx, FPSA_ENOTSUP, "tensor-core factorization needs FP32 factors (MIXED) with 2N = 128, 256 or 512");
    if (r.solve_engine < 0 || r.solve_engine > 2) return fail(ctx, FPSA_EINVAL, "solve_engine not 0, 1 or 2");
    if (r.residual_engine < 0 || r.residual_engine > 2)
        return fail(ctx, FPSA_EINVAL, "residual_engine not 0, 1 or 2");
    if (r.residual_engine == 2 && !ctx->res_ops.D)
        return fail(ctx, FPSA_ENOTSUP, "tensor-core residual needs MIXED precision and N a multiple of 32 up to 256");
    if (r.solve_engine == 2 && ctx->tcs_rt == 0)
        return fail(ctx, FPSA_ENOTSUP,
                    "tensor-core BCR solve needs FP32 factors (MIXED), 2N a multiple of 128 up to 512 and at least "
                    "16 right-hand sides");
    // the segment maps were allocated for the smallest cells-per-thread (most segments)
    const int cmin = sweep_cells_per_thread(ctx->geo);
    ctx->sweep_cpt = std::max(cmin, r.sweep_cells_per_thread);
    ctx->tuning = r;
    plan_solve_shape(ctx);
    return FPSA_OK;
}

int fpsa_autotune(fpsa_ctx *ctx, const fpsa_opts *opts, int32_t repeats, fpsa_tuning *best, double *best_ms) {
    if (!ctx) return FPSA_EINVAL;
    if (repeats < 1) return fail(ctx, FPSA_EINVAL, "repeats < 1");
    if (!ctx->xs_ready) return fail(ctx, FPSA_ESTATE, "fpsa_set_xs must succeed before fpsa_autotune");
    CK(cudaSetDevice(ctx->device));
    const Geometry &g = ctx->geo;
    struct Scratch {  // released on every return
        double *phi = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Scratch() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            if (phi) cudaFree(phi);
        }
    } sc;
    CK(cudaMalloc(&sc.phi, (size_t)g.R * g.sumK * 2 * g.L1 * sizeof(double)));
    CK(cudaEventCreate(&sc.e0));
    CK(cudaEventCreate(&sc.e1));
    const fpsa_tuning saved = ctx->tuning;
    // fastest of `repeats` timed solves after one untimed solve with shapes t
    auto trial = [&](const fpsa_tuning &t, double &ms) -> int {
        int rc = fpsa_set_tuning(ctx, &t);
        ms = INFINITY;
        for (int i = 0; rc == FPSA_OK && i <= repeats; ++i) {
            CK(cudaEventRecord(sc.e0, ctx->stream));
            rc = fpsa_solve(ctx, opts, sc.phi, nullptr, FPSA_MEM_DEVICE, nullptr);
            if (rc != FPSA_OK) break;
            CK(cudaEventRecord(sc.e1, ctx->stream));
            CK(cudaEventSynchronize(sc.e1));
            float f = 0.f;
            CK(cudaEventElapsedTime(&f, sc.e0, sc.e1));
            if (i > 0) ms = std::min(ms, (double)f);
        }
        return rc;
    };
    auto give_up = [&](int rc) {
        const std::string msg = ctx->err;
        fpsa_set_tuning(ctx, &saved);
        ctx->err = msg;
        return rc;
    };
    fpsa_tuning bt{};
    double bms = INFINITY;
    const int bmax = std::min(4, ctx->solve_per_sm[ctx->precision == FPSA_PRECISION_FP64 ? 1 : 0]);
    for (int b = 1; b <= bmax; ++b)
        for (int s = 1; s <= 4; s *= 2) {
            const fpsa_tuning t{0, b, s, saved.factor_engine, saved.solve_engine, saved.residual_engine};
            double ms = 0.0;
            const int rc = trial(t, ms);
            if (rc != FPSA_OK) return give_up(rc);
            if (ms < bms) bms = ms, bt = t;
        }
    const int cmin = sweep_cells_per_thread(g);
    auto segments = [&](int c) { return (g.Kmax + kSegWarps * c - 1) / (kSegWarps * c); };
    for (int k = 1; k <= 3 && segments(cmin << k) < segments(cmin << (k - 1)); ++k) {
        fpsa_tuning t = bt;
        t.sweep_cells_per_thread = cmin << k;
        double ms = 0.0;
        const int rc = trial(t, ms);
        if (rc != FPSA_OK) return give_up(rc);
        if (ms < bms) bms = ms, bt = t;
    }
    // keep the winner (the context's moments are those of the last trial solve)
    const int rc = fpsa_set_tuning(ctx, &bt);
    if (rc != FPSA_OK) return give_up(rc);
    if (best) fpsa_get_tuning(ctx, best);
    if (best_ms) *best_ms = bms;
    return FPSA_OK;
}

}  // extern "C"
