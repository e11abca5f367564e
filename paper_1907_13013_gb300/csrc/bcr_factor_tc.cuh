// Block cyclic reduction factorization with the block inversions on tensor cores
// (FP32 factors of the mixed-precision path, 2N = 128; sm_100a / sm_103a, inline PTX).
//
// Same dataflow as k_bcr_factor_flow (items of every level and the roots in one
// cooperative launch, each waiting on a per-cell counter for the Schur updates of
// the levels below it, then inverting its 2N x 2N block, updating its kept
// neighbours and bumping their counters), with the inversion restructured as a
// blocked Gauss-Jordan elimination whose trailing updates are tcgen05 MMAs:
//
//   The block X (128 x 128 FP32) lives in tensor memory, row r in TMEM lane r,
//   column c in TMEM column c of the CTA's 128-column allocation. The 128 threads
//   (4 warps, one per TMEM lane quarter) each own one row.
//   For each panel q of 16 columns:
//     1. the panel's columns are read from TMEM into registers (16 per thread) and
//        eliminated by Gauss-Jordan with partial pivoting, one column per step:
//        every warp max-reduces a key carrying |x| (to 16 mantissa bits) and the row
//        index, the warp's candidate row publishes its 16 panel values, one block
//        barrier, every thread picks the best of the 4 candidates and updates its
//        row (pivot rows are never moved: row p_k is step k's pivot row). (One warp
//        eliminating the whole panel alone, synchronised by shuffles only, measured
//        twice as slow: its 64 values per lane leave the warp latency-bound.)
//     2. the panel now holds W = E[:, P] (E the product of the panel's elementary
//        row operations, P its pivot rows), and every other column y becomes
//          E y = y + (W - S_P) y[P],   S_P[r][j] = [r == P_j],
//        a rank-16 update: D (the other TMEM columns) += A B with A = W - S_P
//        (128 x 16) and B = the pivot rows' old values (16 x 128), issued by one
//        thread as tcgen05.mma kind::f16 in split BF16 (x = x_hi + x_lo, three
//        products hi*hi + hi*lo + lo*hi, the dropped lo*lo term ~2^-16 relative);
//        the panel's own columns are set to W by tcgen05.st;
//     3. the update is issued as two commits: the next panel's 16 columns first,
//        then the rest, so the next panel's elimination starts while the bulk of
//        the update still runs.
//   At the end X[row][col] = A^{-1}[iperm[row]][perm[col]] (perm[k] = p_k); the
//   transposed inverse the BCR solve reads, At[c][r] = A^{-1}[r][c], is written
//   through shared memory with coalesced rows.
// The pivot choices and the panel arithmetic are FP32; only the trailing updates
// go through the BF16 split. The factors are the preconditioner of the FP32 inner
// solve of the mixed-precision refinement, so this changes its rate, not the
// converged solution. Growth check as in the SIMT kernels (FP64 product of the FP32
// max|A| and max|A^{-1}|).
//
// Every mbarrier wait is bounded (2 s): on timeout the CTA records err[0] = 1,
// waits (bounded) for its own MMAs still in flight and stops taking items; the
// dataflow counter waits give up after err[1] polls (then record err[0] = 1 and
// go on). TMEM: 128 columns per CTA; the launch keeps at most 4 CTAs on an SM
// (their shared memory), so every allocation is granted at once.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "bulk_copy.cuh"
#include "kernels.cuh"
#include "tc_contract.cuh"

namespace fpsa {
namespace tcf {

constexpr int kN2 = 128;          // block size (2N)
constexpr int kPanel = 16;        // columns per panel (one K-step of kind::f16)
constexpr int kPanels = kN2 / kPanel;
constexpr int kThreads = 128;     // one row per thread
constexpr int kStageLd = 36;      // padded row of a 32-column staging chunk
constexpr int kOutLd = kN2 + 4;   // padded row of the output staging buffer
constexpr uint32_t kOpBytes = (uint32_t)kN2 * kPanel * 2;  // one BF16 operand, 128 x 16

// Shared-memory layout of one CTA (bytes). The union area is used in turn by the
// input staging, the panel operands and pivot rows, and the output staging with the
// inverse's coupling quadrants (then the Schur products); the coupling blocks the
// Schur updates multiply arrive in their own area during the inversion.
struct Smem {
    static constexpr uint32_t a_hi = 0, a_lo = a_hi + kOpBytes, b_hi = a_lo + kOpBytes, b_lo = b_hi + kOpBytes;
    static constexpr uint32_t prf = b_lo + kOpBytes;                    // [16][128] FP32 pivot rows
    static constexpr uint32_t ops_end = prf + kPanel * kN2 * 4;         // 24 KB
    static constexpr uint32_t stage_in = 4u * 32 * kStageLd * 4;        // input staging, 18 KB
    static constexpr uint32_t so = 0;                                   // output staging [32][kOutLd]
    static constexpr uint32_t quad = 32u * kOutLd * 4;                  // A^{-1}[L- u R+, L+ u R-], [64][64]
    static constexpr uint32_t prod = 0;                                 // Schur products X1..X4, [4][32][32]
    static constexpr uint32_t out_end = quad + 64u * 64 * 4;            // 32.5 KB
    static constexpr uint32_t union_bytes = ops_end > out_end ? (ops_end > stage_in ? ops_end : stage_in)
                                                               : (out_end > stage_in ? out_end : stage_in);
    static constexpr uint32_t cpl = union_bytes;                        // B_j, C_j, B_i, C_i: [4][32][32]
    // pivot search: keys [2][4], candidate rows [2][4][16]; perm, iperm; reductions
    static constexpr uint32_t keys = cpl + 4u * 32 * 32 * 4;
    static constexpr uint32_t rows = keys + 2 * 4 * 4;
    static constexpr uint32_t perm = rows + 2 * 4 * kPanel * 4;
    static constexpr uint32_t iperm = perm + kN2 * 4;
    static constexpr uint32_t red = iperm + kN2 * 4;                     // 4 doubles
    static constexpr uint32_t bars = red + 4 * 8;                        // 3 mbarriers
    static constexpr uint32_t tslot = bars + 3 * 8;
    static constexpr uint32_t next = tslot + 4;                          // the item taken from the queue
    static constexpr uint32_t used = next + 4;
    // at least this much per CTA, so that no more than 4 CTAs share an SM (4 x 128
    // TMEM columns)
    static constexpr uint32_t total = used > 48 * 1024 ? used : 48 * 1024;
};
static_assert(Smem::so + 32u * kOutLd * 4 <= Smem::quad && Smem::prod + 4u * 32 * 32 * 4 <= Smem::quad,
              "output staging and Schur products stay below the coupling quadrants");
static_assert(Smem::total + 1024 <= 57 * 1024 && 5 * (Smem::total + 1024) > 228 * 1024,
              "4 CTAs per SM fit, 5 do not");

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 FP32 columns of this thread's lane without the wait (tmem_ld16 of the
// contraction kernels waits at once).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// D[:, n0 .. n0 + n) += (A_hi + A_lo)(B_hi + B_lo) restricted to the three leading
// products, K = 16; A 128 x 16 and B (rows n0 ..) 16 x n in the K-major core-matrix
// layout (8-row groups 256 B apart). One thread.
__device__ __forceinline__ void issue_panel_update(uint32_t tmem, const unsigned char *sm, int n0, int n) {
    const uint32_t idesc = tc::idesc_bf16(128, n);
    const uint32_t base = tc::smem_u32(sm);
    const uint32_t boff = (uint32_t)(n0 / 8) * 256u;
    const uint64_t ah = tc::smem_desc(base + Smem::a_hi, 128, 256), al = tc::smem_desc(base + Smem::a_lo, 128, 256);
    const uint64_t bh = tc::smem_desc(base + Smem::b_hi + boff, 128, 256),
                   bl = tc::smem_desc(base + Smem::b_lo + boff, 128, 256);
    const uint32_t d = tmem + (uint32_t)n0;
    tc::mma_bf16(d, ah, bh, idesc, 1u);
    tc::mma_bf16(d, ah, bl, idesc, 1u);
    tc::mma_bf16(d, al, bh, idesc, 1u);
}

// Stage rows [32 w, 32 w + 32) x columns [32 cc, 32 cc + 32) of the block at Ag
// (coalesced 16-byte loads through the warp's padded staging rows) into this warp's
// TMEM lane quarter; returns max |value|. Whole warp.
__device__ __forceinline__ float load_chunk(const float *Ag, unsigned char *sm, uint32_t trow, int cc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *st = reinterpret_cast<float *>(sm) + w * 32 * kStageLd;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int f = lane + 32 * k, row = f >> 3, qd = f & 7;
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(Ag + (size_t)(32 * w + row) * kN2 + 32 * cc) + qd);
        *reinterpret_cast<float4 *>(st + row * kStageLd + 4 * qd) = v;
    }
    __syncwarp();
    float v[32], amax = 0.f;
#pragma unroll
    for (int qd = 0; qd < 8; ++qd) {
        const float4 x = *reinterpret_cast<const float4 *>(st + lane * kStageLd + 4 * qd);
        v[4 * qd] = x.x; v[4 * qd + 1] = x.y; v[4 * qd + 2] = x.z; v[4 * qd + 3] = x.w;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) amax = fmaxf(amax, fabsf(v[i]));
    tmem_st16(trow + 32 * cc, v);
    tmem_st16(trow + 32 * cc + 16, v + 16);
    __syncwarp();  // the chunk's reads before the next chunk's writes
    return amax;
}

// The chunks a lower-level neighbour's Schur update writes: A[L+, L-] (rows 32..63 =
// warp 1, columns 0..31 = chunk 0) and A[R-, R+] (rows 64..95 = warp 2, chunk 3).
__device__ __forceinline__ bool updated_chunk(int w, int cc) { return (w == 1 && cc == 0) || (w == 2 && cc == 3); }

// Invert the 128 x 128 block already in TMEM (rows in lanes); write the transposed
// inverse to Ag and the quadrants A^{-1}[L- u R+, L+ u R-] the Schur updates use
// into shared memory (Smem::quad, [64][64], rows L- then R+, columns L+ then R-).
// amax: this thread's max |A| from the loads. Returns false if an MMA wait ran out
// (the caller stops; bar_b's pending phase, pb, then covers every MMA still in
// flight: its commit is always the CTA's latest). pa / pb: the phases of the two
// update barriers (carried across items).
__device__ __forceinline__ bool tc_invert_block(float *Ag, unsigned char *sm, uint32_t tmem, uint64_t *bar_a,
                                                uint64_t *bar_b, uint32_t &pa, uint32_t &pb, float amax,
                                                unsigned long long *growth, int *status) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t trow = tmem + ((uint32_t)(32 * w) << 16);  // this warp's lane quarter, column 0
    int *perm = reinterpret_cast<int *>(sm + Smem::perm);
    int *iperm = reinterpret_cast<int *>(sm + Smem::iperm);
    double *s_red = reinterpret_cast<double *>(sm + Smem::red);
    float *prf = reinterpret_cast<float *>(sm + Smem::prf);
    bool bad = false;
    // wait (bounded) for the phase of bar with the given parity; the parity advances
    // only when it completed, so after a failure the pending phase is still named
    auto wait_phase = [](uint64_t *bar, uint32_t &parity) {
        const bool ok = tc::mbar_wait(bar, parity);
        tc::tc_fence_after();
        if (!__syncthreads_and(ok)) return false;
        parity ^= 1u;
        return true;
    };
    unsigned *s_key = reinterpret_cast<unsigned *>(sm + Smem::keys);  // [2][4]
    float *s_row = reinterpret_cast<float *>(sm + Smem::rows);        // [2][4][16]
    bool used = false;  // row t has been a pivot row
    for (int q = 0; q < kPanels; ++q) {
        if (q > 0) {  // the update of this panel's columns (first commit of panel q - 1)
            if (!wait_phase(bar_a, pa)) return false;
        }
        float xp[kPanel];
        {
            uint32_t r[16];
            tmem_ld16_nowait(trow + kPanel * q, r);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < kPanel; ++j) xp[j] = __uint_as_float(r[j]);
        }
        // ---- Gauss-Jordan on the panel, one column per step, all 4 warps (row t per thread)
#pragma unroll
        for (int j = 0; j < kPanel; ++j) {
            const int k = kPanel * q + j, par = k & 1;
            const unsigned mag = (__float_as_uint(xp[j]) & 0x7fffffffu) >> 7;
            const unsigned key = used ? 0u : (((mag + 1u) << 7) | (unsigned)t);
            const unsigned wmax = __reduce_max_sync(0xffffffffu, key);
            if (lane == 0) s_key[par * 4 + w] = wmax;
            if (key == wmax && wmax != 0u) {
                float *dst = s_row + (par * 4 + w) * kPanel;
#pragma unroll
                for (int qd = 0; qd < 4; ++qd)
                    *reinterpret_cast<float4 *>(dst + 4 * qd) =
                        make_float4(xp[4 * qd], xp[4 * qd + 1], xp[4 * qd + 2], xp[4 * qd + 3]);
            }
            __syncthreads();
            const uint4 kk = *reinterpret_cast<const uint4 *>(s_key + par * 4);
            unsigned best = kk.x;
            int pw = 0;
            if (kk.y > best) { best = kk.y; pw = 1; }
            if (kk.z > best) { best = kk.z; pw = 2; }
            if (kk.w > best) { best = kk.w; pw = 3; }
            const int p = (int)(best & 127u);
            float rv[kPanel];
            {
                const float *src = s_row + (par * 4 + pw) * kPanel;
#pragma unroll
                for (int qd = 0; qd < 4; ++qd) {
                    const float4 x = *reinterpret_cast<const float4 *>(src + 4 * qd);
                    rv[4 * qd] = x.x; rv[4 * qd + 1] = x.y; rv[4 * qd + 2] = x.z; rv[4 * qd + 3] = x.w;
                }
            }
            const float pv = rv[j];
            if (best == 0u || pv == 0.f || !isfinite(pv)) bad = true;
            float inv;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(pv));
            inv = inv * fmaf(-pv, inv, 2.f);  // one Newton step for 1/pv
            if (t == p) {
#pragma unroll
                for (int jj = 0; jj < kPanel; ++jj) xp[jj] = (jj == j) ? inv : rv[jj] * inv;
                used = true;
                perm[k] = t;
                iperm[t] = k;
            } else {
                const float f = xp[j] * inv;
#pragma unroll
                for (int jj = 0; jj < kPanel; ++jj) xp[jj] = (jj == j) ? -f : fmaf(-f, rv[jj], xp[jj]);
            }
        }
        if (q > 0) {  // the rest of panel q - 1's update: X current everywhere, operands free
            if (!wait_phase(bar_b, pb)) return false;
        }
        // ---- the panel's columns become W; A operand = W - S_P (row t's pivot step, if in the panel)
        const int ks = iperm[t] - kPanel * q;  // step of row t within this panel, if any (own entry)
        const bool piv = ks >= 0 && ks < kPanel;
        {
            float a[kPanel];
#pragma unroll
            for (int j = 0; j < kPanel; ++j) a[j] = (piv && j == ks) ? xp[j] - 1.f : xp[j];
            tmem_st16(trow + kPanel * q, xp);
            tc::store_split_row16(sm + Smem::a_hi, sm + Smem::a_lo, t, 0, a, kPanel);
        }
        // ---- B operand: the panel's pivot rows (old values) across all columns, 32 columns per wait
        if (__any_sync(0xffffffffu, piv)) {
            float *dst = prf + (piv ? ks : 0) * kN2;
#pragma unroll 1
            for (int cc = 0; cc < 4; ++cc) {
                uint32_t r[32];
                tmem_ld16_nowait(trow + 32 * cc, r);
                tmem_ld16_nowait(trow + 32 * cc + 16, r + 16);
                tmem_wait_ld();
                if (piv) {
#pragma unroll
                    for (int qd = 0; qd < 8; ++qd)
                        *reinterpret_cast<float4 *>(dst + 32 * cc + 4 * qd) =
                            make_float4(__uint_as_float(r[4 * qd]), __uint_as_float(r[4 * qd + 1]),
                                        __uint_as_float(r[4 * qd + 2]), __uint_as_float(r[4 * qd + 3]));
                }
            }
        }
        __syncthreads();
        {
            float b[kPanel];
#pragma unroll
            for (int jj = 0; jj < kPanel; ++jj) b[jj] = prf[jj * kN2 + t];  // column t of the pivot rows
            tc::store_split_row16(sm + Smem::b_hi, sm + Smem::b_lo, t, 0, b, kPanel);
        }
        tmem_wait_st();
        tc::fence_async_smem();
        tc::tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc::tc_fence_after();
            if (q + 1 < kPanels) {
                issue_panel_update(tmem, sm, kPanel * (q + 1), kPanel);
                tc::mma_commit(bar_a);
            }
            if (q > 0) issue_panel_update(tmem, sm, 0, kPanel * q);
            if (q + 2 < kPanels) issue_panel_update(tmem, sm, kPanel * (q + 2), kN2 - kPanel * (q + 2));
            tc::mma_commit(bar_b);
        }
    }
    if (!wait_phase(bar_b, pb)) return false;

    // ---- output: At[perm[col]][iperm[row]] = X[row][col], 32 columns at a time through shared memory;
    // the quadrants of the Schur updates are kept
    float ainv = 0.f;
    {
        float *so = reinterpret_cast<float *>(sm + Smem::so);
        float *quad = reinterpret_cast<float *>(sm + Smem::quad);
        const int ir = iperm[t] & (kN2 - 1);  // a permutation of 0..127 (masked: never outside the buffer)
        for (int cc = 0; cc < 4; ++cc) {
            uint32_t r[32];
            tmem_ld16_nowait(trow + 32 * cc, r);
            tmem_ld16_nowait(trow + 32 * cc + 16, r + 16);
            tmem_wait_ld();
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const float x = __uint_as_float(r[jj]);
                ainv = fmaxf(ainv, fabsf(x));
                if (!isfinite(x)) bad = true;
                so[jj * kOutLd + ir] = x;
            }
            __syncthreads();
            // staged row jj is column c = perm[32 cc + jj] of A^{-1}
            for (int jj = w; jj < 32; jj += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(so + jj * kOutLd + 4 * lane);
                reinterpret_cast<float4 *>(Ag + (size_t)(perm[32 * cc + jj] & (kN2 - 1)) * kN2)[lane] = v;
            }
            for (int idx = t; idx < 32 * 64; idx += kThreads) {
                const int jj = idx >> 6, rr = idx & 63;  // rows L- (rr < 32) then R+
                const int c = perm[32 * cc + jj] & (kN2 - 1);
                if (c >= 32 && c < 96) quad[rr * 64 + (c - 32)] = so[jj * kOutLd + (rr < 32 ? rr : rr + 64)];
            }
            __syncthreads();
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        ainv = fmaxf(ainv, __shfl_xor_sync(0xffffffffu, ainv, o));
    }
    if (lane == 0) s_red[w] = (double)amax;
    __syncthreads();
    const double am = fmax(fmax(s_red[0], s_red[1]), fmax(s_red[2], s_red[3]));
    if (growth && lane == 0) atomicMax(growth, dkey((double)ainv * am));
    if (bad) atomicExch(status, 1);
    tc::tc_fence_before();
    __syncthreads();  // s_red and perm are reused by the next step
    tc::tc_fence_after();
    return true;
}

// out[i][l] (op)= sum_k M[i][k] V[k][l] for 32 x 32 blocks, one warp: lane l owns
// column l (M read by broadcast, V by consecutive lanes). mode 0: out = sum (shared
// memory), 1: out -= sum (global, a read-modify-write by this warp alone), 2: out =
// -sum (global).
__device__ __forceinline__ void warp_mm32(const float *M, int ldm, const float *V, int ldv, float *out, int ldo,
                                          int mode) {
    const int lane = threadIdx.x & 31;
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        const float v = V[k * ldv + lane];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = fmaf(M[i * ldm + k], v, acc[i]);
    }
    if (mode == 1) {
        float old[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) old[i] = __ldcg(out + (size_t)i * ldo + lane);
#pragma unroll
        for (int i = 0; i < 32; ++i) out[(size_t)i * ldo + lane] = old[i] - acc[i];
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) out[(size_t)i * ldo + lane] = mode == 2 ? -acc[i] : acc[i];
    }
}

}  // namespace tcf

// The factorization dataflow of k_bcr_factor_flow with tensor-core inversions (FP32,
// 2N = 128): one 128-thread CTA per item at a time, up to 4 CTAs per SM. CTAs take
// the items in their order (levels ascending, roots last) from a work queue (*queue,
// zero at launch): every item a CTA waits for has a lower index and was taken by a
// CTA that is already running, so the launch needs no co-residency guarantee (it is
// an ordinary launch, not a cooperative one). An item
// stages the parts of its block that no lower level updates into TMEM before it
// waits for its counter, then the two updated chunks; its coupling blocks arrive by
// bulk copy during the inversion, and the Schur updates of its kept neighbours are
// formed from shared memory (the inverse's quadrants kept by the output pass), one
// 32 x 32 product per warp:
//   right j = i+s:  X1 = B_j A^{-1}[R+,R-];  A_j[L+,L-] -= X1 C_i;  X2 = B_j A^{-1}[R+,L+];  B_j' = -X2 B_i
//   left  j = i-s:  X3 = C_j A^{-1}[L-,L+];  A_j[R-,R+] -= X3 B_i;  X4 = C_j A^{-1}[L-,R-];
//                   C_j' = -X4 C_i  (0 if i has no right neighbour)
__global__ void __launch_bounds__(tcf::kThreads, 4) k_bcr_factor_tc(float *__restrict__ A,
                                                                     const BcrItem *__restrict__ items, int n_items,
                                                                     float *__restrict__ Bc, float *__restrict__ Cc,
                                                                     unsigned long long *__restrict__ growth,
                                                                     int *__restrict__ status, int *cnt, int *err,
                                                                     int *queue) {
    using namespace tcf;
    extern __shared__ __align__(128) unsigned char smem_ftc[];
    unsigned char *sm = smem_ftc;
    uint64_t *bar_a = reinterpret_cast<uint64_t *>(sm + Smem::bars), *bar_b = bar_a + 1, *bar_c = bar_a + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + Smem::tslot);
    float *cpl = reinterpret_cast<float *>(sm + Smem::cpl);  // [0] B_j, [1] C_j, [2] B_i, [3] C_i
    constexpr int hh = 32 * 32;
    if (threadIdx.x == 0) {
        tc::mbar_init(bar_a, 1);
        tc::mbar_init(bar_b, 1);
        tc::mbar_init(bar_c, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tslot, (uint32_t)kN2);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const uint32_t trow = tmem + ((uint32_t)(32 * w) << 16);
    const unsigned limit = flow_spin_limit(err);
    uint32_t pa = 0, pb = 0, pc = 0;
    int *s_next = reinterpret_cast<int *>(sm + Smem::next);
    for (;;) {
        if (t == 0) *s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int ii = *s_next;
        if (ii >= n_items) break;
        const BcrItem it = items[ii];
        float *Ag = A + (size_t)it.cell * kN2 * kN2;
        int *iperm = reinterpret_cast<int *>(sm + Smem::iperm);
        iperm[t] = -1;  // rows not yet pivots (ordered before any read by the barriers below)
        // the chunks no lower level updates, before the wait
        float amax = 0.f;
        for (int cc = 0; cc < 4; ++cc)
            if (!updated_chunk(w, cc)) amax = fmaxf(amax, load_chunk(Ag, sm, trow, cc));
        FlowSync fs{};
        fs.err = err;
        fs.limit = limit;
        int want = 0;
        for (int lp = 0; lp < it.level; ++lp)
            want += (it.local >= (1 << lp)) + (it.local + (1 << lp) < it.K_inst);
        if (want) {
            fs.wait0 = cnt + it.cell;
            fs.want0 = want;
        }
        flow_wait(&fs);
        const bool has_r = it.right >= 0, has_l = it.left >= 0;
        if (t == 0 && (has_r || has_l)) {  // the couplings, final now: in flight during the inversion
            constexpr uint32_t hb = hh * 4;
            tc::fence_async_smem();
            tc::mbar_arrive_expect_tx(bar_c, 2 * hb + (has_r ? hb : 0u) + (has_l ? hb : 0u));
            if (has_r) tc::bulk_copy_g2s(cpl, Bc + (size_t)it.s_right * hh, hb, bar_c);
            if (has_l) tc::bulk_copy_g2s(cpl + hh, Cc + (size_t)it.s_left * hh, hb, bar_c);
            tc::bulk_copy_g2s(cpl + 2 * hh, Bc + (size_t)it.s_cell * hh, hb, bar_c);
            tc::bulk_copy_g2s(cpl + 3 * hh, Cc + (size_t)it.s_cell * hh, hb, bar_c);
        }
        for (int cc = 0; cc < 4; ++cc)
            if (updated_chunk(w, cc)) amax = fmaxf(amax, load_chunk(Ag, sm, trow, cc));
        tmem_wait_st();
        tc::tc_fence_before();
        __syncthreads();  // staging area reused by the operands; TMEM writes done
        tc::tc_fence_after();
        if (!tc_invert_block(Ag, sm, tmem, bar_a, bar_b, pa, pb, amax, growth, status)) {
            // an MMA did not complete in time: record it, let any MMA and copy still in
            // flight land (bounded) and stop taking items
            if (t == 0) atomicExch(err, 1);
            tc::mbar_wait(bar_b, pb);
            if (has_r || has_l) tc::mbar_wait(bar_c, pc);
            break;
        }
        if (has_r || has_l) {
            const bool ok = tc::mbar_wait(bar_c, pc);
            if (!__syncthreads_and(ok)) {
                if (t == 0) atomicExch(err, 1);
                break;
            }
            pc ^= 1u;
            const float *quad = reinterpret_cast<const float *>(sm + Smem::quad);  // [64][64]
            float *X = reinterpret_cast<float *>(sm + Smem::prod);                // [4][32][32]
            // wave 1: X1 = B_j Q[R+][R-], X2 = B_j Q[R+][L+], X3 = C_j Q[L-][L+], X4 = C_j Q[L-][R-]
            if (w < 2 ? has_r : has_l) {
                const float *Mj = cpl + (w < 2 ? 0 : hh);
                const int r0 = w < 2 ? 32 : 0, c0 = (w == 0 || w == 3) ? 32 : 0;
                warp_mm32(Mj, 32, quad + r0 * 64 + c0, 64, X + w * hh, 32, 0);
            }
            __syncthreads();
            // wave 2: A_j[L+,L-] -= X1 C_i; B_j' = -X2 B_i; A_j[R-,R+] -= X3 B_i; C_j' = -X4 C_i
            constexpr int n2 = kN2, Lm = 0, Lp = 32, Rm = 64, Rp = 96;
            if (w == 0 && has_r)
                warp_mm32(X, 32, cpl + 3 * hh, 32, A + (size_t)it.right * n2 * n2 + Lp * n2 + Lm, n2, 1);
            if (w == 1 && has_r) warp_mm32(X + hh, 32, cpl + 2 * hh, 32, Bc + (size_t)it.s_right_next * hh, 32, 2);
            if (w == 2 && has_l)
                warp_mm32(X + 2 * hh, 32, cpl + 2 * hh, 32, A + (size_t)it.left * n2 * n2 + Rm * n2 + Rp, n2, 1);
            if (w == 3 && has_l) {
                float *Cn = Cc + (size_t)it.s_left_next * hh;
                if (has_r) warp_mm32(X + 3 * hh, 32, cpl + 3 * hh, 32, Cn, 32, 2);
                else
                    for (int i = 0; i < 32; ++i) Cn[i * 32 + lane] = 0.f;
            }
            if (has_r) fs.sig0 = cnt + it.right;
            if (has_l) fs.sig1 = cnt + it.left;
            flow_signal(&fs);
        }
        __syncthreads();  // shared memory reused by the block's next item
    }
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, (uint32_t)kN2);
}

}  // namespace fpsa
