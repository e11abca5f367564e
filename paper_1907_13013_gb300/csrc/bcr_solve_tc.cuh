// Block cyclic reduction solve with many right-hand sides on tensor cores (the
// FP32 factors of the mixed-precision path; 2N a multiple of 128 up to 512, at
// least 16 right-hand sides).
//
// The dataflow solve k_bcr_solve_flow applies an eliminated cell's A^{-1} to at
// most 8 right-hand sides per unit, so with R of them every factor is read R / 8
// times per solve. Here a unit is one (cell, phase, tile of RT <= 64 right-hand
// sides), and its product is one GEMM on the tensor cores:
//   forward  Y_i = A_i^{-1} r_i                            [2N x RT]
//   backward u_i = Y_i - A_i^{-1}[:, N/2 : 3N/2] g_i,
//            g_i = [B_i u_left[3N/2 : 2N] ; C_i u_right[0 : N/2]]
// (the same reduction, pushes and counters as k_bcr_solve_flow, one row slice).
// A_i^{-1} is operand A (2N/128 tiles of 128 rows, M = 128), the right-hand sides
// operand B (N = RT), accumulated in FP32 in tensor memory ((2N/128) x RT
// columns). Precision: split BF16 with three products, as the contractions
//   A x ~= A_hi x_hi + A_hi x_lo + A_lo x_hi.
// Each factor is stored a second time for this solve, already split and in the
// K-major core-matrix layout (k_bcr_factor_split), as 2N/16 chunks of 16 columns
// (hi [2N x 16] then lo); a chunk is one bulk asynchronous copy (the TMA engine)
// into one of two shared-memory stages, so a unit streams its factor once while
// the previous chunk is multiplied. The right-hand-side chunk of each K-step is
// split by the CTA's threads from FP32 (loaded one chunk ahead) into the stage
// beside it. The coupling products (N/2 x N/2 blocks, a few percent of the
// flops) run on the FP32 cores, one row per thread.
//
// Units are taken from a work queue in phase order (forward levels, roots,
// backward levels): a unit depends only on units with lower indices, every one of
// which is held by a running CTA, so every wait ends and an ordinary launch
// suffices (two CTAs per SM: the shared-memory request admits no third, so their
// 2 x 256 tensor-memory columns always fit). The copies of a CTA's next unit are
// issued while the current one finishes. Every wait is bounded; on a timeout the
// CTA records the error, lets its copies and products land (bounded), frees its
// tensor memory and stops taking units, and the other CTAs' waits give up as soon
// as they see the error flag.
#pragma once

#include "kernels.cuh"
#include "tc_contract.cuh"

namespace fpsa {
namespace tcs {

constexpr int kThreads = 128;
constexpr int kK = 16;                     // factor columns per streamed chunk: one MMA K-step
constexpr int kMaxRT = 64;                 // right-hand sides per unit
constexpr int kMaxN2 = 512;
constexpr uint32_t kMinSmem = 80u * 1024u;  // > 228 KB / 3: at most two CTAs per SM

__host__ __device__ constexpr int rhs_tile(int R) { return R >= kMaxRT ? kMaxRT : (R + 15) / 16 * 16; }
__host__ __device__ constexpr bool applies(int n2, int R) { return n2 % 128 == 0 && n2 <= kMaxN2 && R >= 16; }
// bytes of one chunk of a split factor (hi + lo, 2N x 16 BF16 each) and of a cell's
__host__ __device__ constexpr uint32_t chunk_bytes(int n2) { return (uint32_t)n2 * kK * 4u; }
__host__ __device__ constexpr size_t cell_bytes(int n2) { return (size_t)n2 * n2 * 4u; }
// one K-step of the right-hand sides: hi + lo, RT x 16 BF16 each
__host__ __device__ constexpr uint32_t rhs_bytes(int RT) { return (uint32_t)RT * kK * 4u; }
// row stride (floats) of the coupling vectors in shared memory, [RT][N/2 + 4]
__host__ __device__ constexpr int aux_ld(int n2) { return n2 / 4 + 4; }

// Shared memory: two stages (factor chunk, then right-hand-side chunk), the
// coupling vectors, 5 mbarriers (full[2], empty[2], drain), the tensor-memory slot
// and the CTA's current unit.
struct Plan {
    uint32_t stage, aux, bars, total;
    __host__ __device__ static Plan make(int n2, int RT) {
        Plan p;
        p.stage = chunk_bytes(n2) + rhs_bytes(RT);
        p.aux = 2 * p.stage;
        p.bars = (p.aux + (uint32_t)RT * aux_ld(n2) * 4u + 15u) & ~15u;
        p.total = p.bars + 64;
        if (p.total < kMinSmem) p.total = kMinSmem;
        return p;
    }
};

// out = the split copy of the stored inverses (FP32, transposed: Mt[col][row] =
// A^{-1}[row][col]): block (cell, kc) writes columns 16 kc .. 16 kc + 15 as hi and lo
// BF16 in the K-major core-matrix layout, element (row, k) of a part at
// kmajor_offset(row, k, 16). Consecutive threads take consecutive rows, so every
// column is read coalesced; each thread writes 16 bytes of each part.
__global__ void __launch_bounds__(256) k_bcr_factor_split(const float *__restrict__ A, unsigned char *__restrict__ out,
                                                          int n2) {
    const int nkc = n2 / kK;
    const int cell = blockIdx.x / nkc, kc = blockIdx.x - cell * nkc;
    const float *Mt = A + (size_t)cell * n2 * n2 + (size_t)kc * kK * n2;
    unsigned char *o = out + (size_t)cell * cell_bytes(n2) + (size_t)kc * chunk_bytes(n2);
    for (int i = threadIdx.x; i < 2 * n2; i += blockDim.x) {
        const int row = i % n2, half = i / n2;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat16 h0, l0, h1, l1;
            tc::split_bf16(Mt[(size_t)(8 * half + 2 * j) * n2 + row], h0, l0);
            tc::split_bf16(Mt[(size_t)(8 * half + 2 * j + 1) * n2 + row], h1, l1);
            hi[j] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lo[j] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        const uint32_t off = tc::kmajor_offset(row, 8 * half, kK);
        *reinterpret_cast<uint4 *>(o + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4 *>(o + (size_t)n2 * kK * 2 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// acc[r] = sum_k M[p][k] v[r][k] for row p = threadIdx.x < h2: M row-major h2 x h2
// in global memory, v [RT][ld] in shared memory (read by the whole warp at once).
template <int RT>
__device__ __forceinline__ void coupling_rows(const float *__restrict__ M, const float *v, int h2, int ld,
                                              float (&acc)[RT]) {
    const int p = threadIdx.x;
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[r] = 0.f;
    const float4 *Mr = reinterpret_cast<const float4 *>(M + (size_t)p * h2);
    for (int k4 = 0; k4 < h2 / 4; ++k4) {
        const float4 m = __ldg(Mr + k4);
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const float4 a = *reinterpret_cast<const float4 *>(v + r * ld + 4 * k4);
            acc[r] = fmaf(m.x, a.x, acc[r]);
            acc[r] = fmaf(m.y, a.y, acc[r]);
            acc[r] = fmaf(m.z, a.z, acc[r]);
            acc[r] = fmaf(m.w, a.w, acc[r]);
        }
    }
}

// v[r][k] = src[r * stride + k] (r < nrc, else 0) for r < RT, k < h2
template <int RT>
__device__ __forceinline__ void load_vectors(float *v, const float *src, size_t stride, int nrc, int h2, int ld) {
    for (int i = threadIdx.x; i < RT * h2; i += kThreads) {
        const int r = i / h2, k = i - r * h2;
        v[r * ld + k] = r < nrc ? __ldcg(src + (size_t)r * stride + k) : 0.f;
    }
}

// The dataflow wait of a unit (thread 0 polls; bounded), giving up at once when
// another CTA has recorded an error.
__device__ __forceinline__ void flow_wait_tc(const FlowSync &fs) {
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int *c = k ? fs.wait1 : fs.wait0;
            const int want = k ? fs.want1 : fs.want0;
            if (!c) continue;
            unsigned spins = 0;
            while (ld_acquire_gpu(c) < want) {
                if (++spins > fs.limit || *(volatile int *)fs.err != 0) {
                    atomicExch(fs.err, 1);
                    break;
                }
                if (spins > 256) __nanosleep(32);
            }
        }
    }
    __syncthreads();
}

struct Unit {
    int item, ch, bwd, nkc, kc0;
};

}  // namespace tcs

// The solve: units as above over the concatenated item array of lv; counters
// cnt / done per (tile of RT right-hand sides, cell), zero at launch, as in
// k_bcr_solve_flow (one slice per item); queue: this launch's unit counter (zero
// at launch). zero_next / queue_next: the other parity's counters, zeroed for the
// following solve. gs: per-CTA scratch of the backward coupling vectors g
// (gridDim.x x RT x N floats).
template <int RT>
__global__ void __launch_bounds__(tcs::kThreads) k_bcr_solve_tc(
    const unsigned char *__restrict__ Atc, const float *__restrict__ Bc, const float *__restrict__ Cc,
    const BcrItem *__restrict__ items, LevelTable lv, float *rhs, float *Y, float *gs, int N, int sumK, int R,
    int *cnt, int *done, int *queue, int *err, int *zero_next, long long nzero, int *queue_next) {
    using namespace tcs;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < nzero; i += (long long)gridDim.x * kThreads)
        zero_next[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *queue_next = 0;
    tc::grid_dependency_wait();
    extern __shared__ __align__(128) unsigned char smem_tcs[];
    const int n2 = 2 * N, h2 = N / 2, hh = h2 * h2, MT = n2 / 128, ald = aux_ld(n2);
    const Plan pl = Plan::make(n2, RT);
    const uint32_t cbytes = chunk_bytes(n2);
    float *aux = reinterpret_cast<float *>(smem_tcs + pl.aux);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_tcs + pl.bars), *empty = full + 2, *drain = full + 4;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(full + 5);
    int *s_unit = reinterpret_cast<int *>(tslot + 1);
    const int t = threadIdx.x;
    if (t == 0) {
        for (int i = 0; i < 5; ++i) tc::mbar_init(full + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint32_t tcols = tc::tmem_cols_for(MT * RT);
    if (t < 32) {
        tc::tmem_alloc(tslot, tcols);
        tc::tmem_relinquish();
    }
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    const int nch = (R + RT - 1) / RT, nl = lv.n_levels, P = 2 * nl;
    const size_t rstride = (size_t)sumK * n2;
    const unsigned limit = flow_spin_limit(err);
    auto level_of = [&](int ph) { return ph <= nl ? ph : 2 * nl - ph; };
    auto phase_units = [&](int ph) {
        const int l = level_of(ph);
        return (l < nl ? lv.off[l + 1] - lv.off[l] : lv.n_roots) * nch;
    };
    int total = 0;
    for (int ph = 0; ph <= P; ++ph) total += phase_units(ph);
    auto decode = [&](int u, Unit &d) {
        int ph = 0, start = 0;
        while (u >= start + phase_units(ph)) {
            start += phase_units(ph);
            ++ph;
        }
        const int w = u - start;
        d.ch = w % nch;
        d.item = lv.off[level_of(ph)] + w / nch;
        d.bwd = ph > nl;
        d.nkc = d.bwd ? N / kK : n2 / kK;
        d.kc0 = d.bwd ? h2 / kK : 0;
    };

    // thread 0: the stream of factor chunks, unit after unit in the order this CTA
    // takes them; chunk q of the stream goes to stage q & 1
    Unit cur{}, nxt{};
    int nxt_u = -1;
    uint32_t cur_base = 0, issued = 0, waited = 0;
    auto chunk_src = [&](const Unit &d, int c) {
        return Atc + (size_t)items[d.item].cell * cell_bytes(n2) + (size_t)(d.kc0 + c) * cbytes;
    };
    auto issue = [&](uint32_t q) {  // thread 0: request chunk q of the stream, if it exists
        const unsigned char *src;
        if (q < cur_base + (uint32_t)cur.nkc) {
            src = chunk_src(cur, (int)(q - cur_base));
        } else {
            if (nxt_u < 0) {
                nxt_u = atomicAdd(queue, 1);
                if (nxt_u < total) decode(nxt_u, nxt);
            }
            if (nxt_u >= total) return;
            src = chunk_src(nxt, (int)(q - cur_base - (uint32_t)cur.nkc));
        }
        const int s = q & 1;
        tc::mbar_arrive_expect_tx(&full[s], cbytes);
        tc::bulk_copy_g2s(smem_tcs + s * pl.stage, src, cbytes, &full[s]);
        issued = q + 1;
    };

    if (t == 0) *s_unit = atomicAdd(queue, 1);
    __syncthreads();
    int u = *s_unit;
    Unit d{};
    if (u < total) decode(u, d);
    if (t == 0 && u < total) {
        cur = d;
        issue(0);
        issue(1);
    }
    const uint32_t idesc = tc::idesc_bf16(128, RT);
    const int br = t >> 1, bh = t & 1;  // right-hand-side split: row br, k-half bh of a chunk
    const int w = t >> 5, lane = t & 31;
    const uint32_t lane_base = (uint32_t)(w * 32) << 16;
    uint32_t q = 0;  // stream index of the chunk being consumed
    bool ok = true;
    while (u < total) {
        const BcrItem it = items[d.item];
        const int r0 = d.ch * RT, nrc = min(RT, R - r0);
        int *cnt_c = cnt + (size_t)d.ch * sumK, *done_c = done + (size_t)d.ch * sumK;
        FlowSync fs{};
        fs.err = err;
        fs.limit = limit;
        if (!d.bwd) {
            int want = 0;
            for (int lp = 0; lp < it.level; ++lp)
                want += (it.local >= (1 << lp)) + (it.local + (1 << lp) < it.K_inst);
            if (want) {
                fs.wait0 = cnt_c + it.cell;
                fs.want0 = want;
            }
        } else {
            fs.wait0 = done_c + it.left;
            fs.want0 = 1;
            if (it.right >= 0) {
                fs.wait1 = done_c + it.right;
                fs.want1 = 1;
            }
        }
        flow_wait_tc(fs);
        const float *bsrc;
        size_t bstride;
        if (!d.bwd) {
            bsrc = rhs + (size_t)r0 * rstride + (size_t)it.cell * n2;
            bstride = rstride;
        } else {
            // g = [B_i u_left[3N/2 : 2N] ; C_i u_right[0 : N/2]] into this CTA's scratch, [RT][N]
            float *g = gs + (size_t)blockIdx.x * RT * N;
            float acc[RT];
            load_vectors<RT>(aux, Y + (size_t)r0 * rstride + (size_t)it.left * n2 + N + h2, rstride, nrc, h2, ald);
            __syncthreads();
            if (t < h2) {
                coupling_rows<RT>(Bc + (size_t)it.s_cell * hh, aux, h2, ald, acc);
#pragma unroll
                for (int r = 0; r < RT; ++r) g[(size_t)r * N + t] = acc[r];
            }
            __syncthreads();
            if (it.right >= 0) {
                load_vectors<RT>(aux, Y + (size_t)r0 * rstride + (size_t)it.right * n2, rstride, nrc, h2, ald);
                __syncthreads();
                if (t < h2) {
                    coupling_rows<RT>(Cc + (size_t)it.s_cell * hh, aux, h2, ald, acc);
#pragma unroll
                    for (int r = 0; r < RT; ++r) g[(size_t)r * N + h2 + t] = acc[r];
                }
            } else if (t < h2) {
#pragma unroll
                for (int r = 0; r < RT; ++r) g[(size_t)r * N + h2 + t] = 0.f;
            }
            __syncthreads();
            bsrc = g;
            bstride = N;
        }

        // the GEMM: chunk by chunk, the right-hand sides split into the stage beside the factor chunk
        float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
        auto load_b = [&](int c) {
            if (br < nrc) {
                const float4 *s = reinterpret_cast<const float4 *>(bsrc + (size_t)br * bstride + c * kK + 8 * bh);
                v0 = __ldcg(s);
                v1 = __ldcg(s + 1);
            } else {
                v0 = v1 = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        if (br < RT) load_b(0);
        bool fail = false;
        for (int c = 0; c < d.nkc; ++c, ++q) {
            const int s = q & 1;
            unsigned char *stg = smem_tcs + s * pl.stage, *bs = stg + cbytes;
            if (q >= 2) ok = ok && tc::mbar_wait(&empty[s], ((q >> 1) - 1) & 1);  // chunk q - 2's products are done
            if (br < RT) {
                const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    __nv_bfloat16 h0, l0, h1, l1;
                    tc::split_bf16(x[2 * j], h0, l0);
                    tc::split_bf16(x[2 * j + 1], h1, l1);
                    hi[j] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    lo[j] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
                const uint32_t off = tc::kmajor_offset(br, 8 * bh, kK);
                *reinterpret_cast<uint4 *>(bs + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4 *>(bs + (size_t)RT * kK * 2 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                if (c + 1 < d.nkc) load_b(c + 1);
            }
            tc::fence_async_smem();  // the st.shared above, before the tensor core reads them
            if (__syncthreads_or(!ok)) {
                fail = true;
                break;
            }
            if (t == 0) {
                ok = tc::mbar_wait(&full[s], (q >> 1) & 1);
                if (ok) {
                    waited = q + 1;
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(stg), b0 = tc::smem_u32(bs);
                    const uint64_t bhd = tc::smem_desc(b0, 128, 256), bld = tc::smem_desc(b0 + RT * kK * 2, 128, 256);
                    for (int m = 0; m < MT; ++m) {
                        const uint64_t ahd = tc::smem_desc(a0 + 4096u * m, 128, 256);
                        const uint64_t ald_ = tc::smem_desc(a0 + (uint32_t)n2 * kK * 2 + 4096u * m, 128, 256);
                        const uint32_t dt = tmem + (uint32_t)(m * RT);
                        tc::mma_bf16(dt, ahd, bhd, idesc, c > 0 ? 1u : 0u);
                        tc::mma_bf16(dt, ahd, bld, idesc, 1u);
                        tc::mma_bf16(dt, ald_, bhd, idesc, 1u);
                    }
                    tc::mma_commit(&empty[s]);
                    // the stage is refilled with chunk q + 2 once these products have read it
                    ok = tc::mbar_wait(&empty[s], (q >> 1) & 1);
                    if (ok) issue(q + 2);
                }
            }
        }
        if (fail || __syncthreads_or(!ok)) break;
        // every product of the unit has completed (the last chunk's commit)
        const uint32_t ql = q - 1;
        ok = tc::mbar_wait(&empty[ql & 1], (ql >> 1) & 1);
        if (__syncthreads_or(!ok)) break;
        tc::tc_fence_after();
        if (!d.bwd) {
            const bool push_r = it.right >= 0, push_l = it.left >= 0;
            float v[16];
            for (int m = 0; m < MT; ++m) {
                const int row = 128 * m + 32 * w + lane;
                for (int c16 = 0; c16 < RT / 16; ++c16) {
                    tc::tmem_ld16(tmem + lane_base + (uint32_t)(m * RT + 16 * c16), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int r = 16 * c16 + j;
                        if (r < nrc) Y[(size_t)(r0 + r) * rstride + (size_t)it.cell * n2 + row] = v[j];
                        if (push_r && row >= N + h2) aux[r * ald + row - N - h2] = v[j];
                    }
                }
            }
            float acc[RT];
            if (push_r) {  // r_right[N/2 : N] -= B_right Y_i[3N/2 : 2N]
                __syncthreads();
                if (t < h2) {
                    coupling_rows<RT>(Bc + (size_t)it.s_right * hh, aux, h2, ald, acc);
                    float *o = rhs + (size_t)r0 * rstride + (size_t)it.right * n2 + h2 + t;
#pragma unroll
                    for (int r = 0; r < RT; ++r)
                        if (r < nrc) atomicAdd(o + (size_t)r * rstride, -acc[r]);
                }
            }
            if (push_l) {  // r_left[N : 3N/2] -= C_left Y_i[0 : N/2]
                __syncthreads();
                if (32 * w < h2) {
                    for (int c16 = 0; c16 < RT / 16; ++c16) {
                        tc::tmem_ld16(tmem + lane_base + (uint32_t)(16 * c16), v);
                        const int row = 32 * w + lane;
                        if (row < h2)
#pragma unroll
                            for (int j = 0; j < 16; ++j) aux[(16 * c16 + j) * ald + row] = v[j];
                    }
                }
                __syncthreads();
                if (t < h2) {
                    coupling_rows<RT>(Cc + (size_t)it.s_left * hh, aux, h2, ald, acc);
                    float *o = rhs + (size_t)r0 * rstride + (size_t)it.left * n2 + N + t;
#pragma unroll
                    for (int r = 0; r < RT; ++r)
                        if (r < nrc) atomicAdd(o + (size_t)r * rstride, -acc[r]);
                }
            }
            if (push_r) fs.sig0 = cnt_c + it.right;
            if (push_l) fs.sig1 = cnt_c + it.left;
            else fs.sig2 = done_c + it.cell;  // a root: its solution is final
        } else {
            float v[16];
            for (int m = 0; m < MT; ++m) {
                const int row = 128 * m + 32 * w + lane;
                for (int c16 = 0; c16 < RT / 16; ++c16) {
                    tc::tmem_ld16(tmem + lane_base + (uint32_t)(m * RT + 16 * c16), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int r = 16 * c16 + j;
                        if (r < nrc) {
                            float *y = Y + (size_t)(r0 + r) * rstride + (size_t)it.cell * n2 + row;
                            *y = __ldcg(y) - v[j];
                        }
                    }
                }
            }
            fs.sig0 = done_c + it.cell;
        }
        tc::tc_fence_before();  // the accumulator reads, before the next unit's products
        flow_signal(&fs);
        // the next unit: already taken by the copy stream, or taken now
        if (t == 0) {
            if (nxt_u < 0) {
                nxt_u = atomicAdd(queue, 1);
                if (nxt_u < total) decode(nxt_u, nxt);
            }
            *s_unit = nxt_u;
            if (nxt_u < total) {
                cur_base += (uint32_t)cur.nkc;
                cur = nxt;
                // a unit taken here (not by the stream) has no chunk in flight yet
                if (issued < cur_base + 1) issue(cur_base);
                if (issued < cur_base + 2) issue(cur_base + 1);
            }
            nxt_u = -1;
        }
        __syncthreads();
        u = *s_unit;
        if (u < total) decode(u, d);
    }
    if (!ok || u < total) {
        // a wait gave up: let this CTA's copies and products land (bounded), record the error
        if (t == 0) {
            for (uint32_t j = waited; j < issued; ++j)
                if (!tc::mbar_wait(&full[j & 1], (j >> 1) & 1)) break;
            tc::mma_commit(drain);
            (void)tc::mbar_wait(drain, 0);
            atomicExch(err, 1);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tmem, tcols);
}

}  // namespace fpsa
