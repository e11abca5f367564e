// Tensor-core (tcgen05) angular contractions for the FP32 inner solves of the
// mixed-precision path (sm_100a / sm_103a, inline PTX).
//
// A contraction over a tile of 128 columns (64 cells x 2 LD nodes) is the GEMM
//   Out[c][o] = sum_k X[c][k] Op[o][k],   c < 128, o, k < N,
// with Op = D (phi = D psi, Eq. phi-mom) or Op = M (q = M src, Eq. treq).
// Precision: split BF16 with three products. x = x_hi + x_lo with
// x_hi = bf16(x), x_lo = bf16(x - x_hi) (likewise for Op), and
//   x Op ~= x_hi Op_hi + x_hi Op_lo + x_lo Op_hi
// accumulated in FP32 in tensor memory (the dropped x_lo Op_lo term is ~2^-16
// relative). One elected thread issues tcgen05.mma (M = 128, N = N, K = 16 per
// instruction, cta_group::1, kind::f16, A and B both BF16); completion is
// signalled through an mbarrier by tcgen05.commit; the four warps read their 32
// accumulator lanes back with tcgen05.ld.
//
// Shared-memory operand layout (no swizzle, K-major): an R x K BF16 operand is a
// grid of 8 x 8 "core matrices" (8 rows of 16 bytes, 128 contiguous bytes);
// element (row, k) sits at byte
//   ((row / 8) * (K / 8) + k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2,
// so core matrices adjacent in K are 128 B apart (leading byte offset) and
// adjacent 8-row groups K * 16 B apart (stride byte offset). A K-step of 16
// starts 256 B further. The constant operands (D, M) are stored in global memory
// already split and in this layout and are staged with one bulk asynchronous
// copy (cp.async.bulk, the TMA engine) per CTA.
//
// Every wait on an mbarrier is bounded; on timeout the kernel records an error
// flag, releases its tensor memory and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "bulk_copy.cuh"

namespace fpsa {
namespace tc {

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {  // whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator,
// both operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row, k) in the K-major no-swizzle layout with K columns
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int row, int k, int K) {
    return (uint32_t)((((row >> 3) * (K >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Staged global I/O: a tile's 128 columns are 128 contiguous rows of N floats in
// global memory; they move through padded shared buffers [128][kStageLd] in
// k-chunks of kStageK with coalesced 16-byte accesses, and each thread then reads
// or writes its own row (the accumulator lane layout) without bank conflicts.
constexpr int kStageK = 16;
constexpr int kStageLd = kStageK + 4;
constexpr uint32_t kStageBytes = 128u * kStageLd * 4;

// Shared-memory plan of one contraction CTA for N (multiple of 16, <= 128):
//   opD_hi, opD_lo, opM_hi, opM_lo: N x N BF16 each (constant operands)
//   x_hi, x_lo:                     128 x N BF16 each (the column tile)
//   stage[3]:                       [128][kStageLd] FP32 each (staged I/O)
//   bars: 2 mbarriers (bulk copy, MMA), tmem slot
struct Plan {
    uint32_t op_bytes, x_bytes, stage_bytes, total;
    bool full;  // whole-tile staging ([128][N + 4] FP32 per buffer, N <= 64)
    __host__ __device__ static Plan make(int N) {
        Plan p;
        p.op_bytes = (uint32_t)N * N * 2;
        p.x_bytes = 128u * N * 2;
        p.full = N <= 64;
        p.stage_bytes = p.full ? 128u * (N + 4) * 4 : kStageBytes;
        p.total = 4 * p.op_bytes + 2 * p.x_bytes + 3 * p.stage_bytes + 64;
        return p;
    }
};

// Whole-tile staging: asynchronous 16-byte copies of rows [0, nrows) of src (row
// length N floats, N a multiple of 4) into st[row][0..N) with row stride N + 4
// (conflict-free row reads); rows >= nrows are zero-filled. Not committed here.
__device__ __forceinline__ void tile_load_async(float *st, const float *src, int N, int nrows) {
    const int Q = N / 4, ld = N + 4;
    for (int f = threadIdx.x; f < 128 * Q; f += 128) {
        const int row = f / Q, q = f - row * Q;
        float *dst = st + row * ld + 4 * q;
        if (row < nrows)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)),
                         "l"(src + (size_t)row * N + 4 * q)
                         : "memory");
        else
            *reinterpret_cast<float4 *>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPending>
__device__ __forceinline__ void async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NPending) : "memory"); }

// dst[row * N + k] = st[row][k] for rows < nrows, coalesced 16-byte stores.
__device__ __forceinline__ void tile_store(const float *st, float *dst, int N, int nrows) {
    const int Q = N / 4, ld = N + 4;
    for (int f = threadIdx.x; f < 128 * Q; f += 128) {
        const int row = f / Q, q = f - row * Q;
        if (row < nrows)
            reinterpret_cast<float4 *>(dst + (size_t)row * N)[q] =
                *reinterpret_cast<const float4 *>(st + row * ld + 4 * q);
    }
}

// st[row][0..kStageK) = src[row * N + k0 ..] for rows < nrows, 0 above (all 128 threads).
__device__ __forceinline__ void stage_in(float *st, const float *src, int N, int nrows, int k0) {
    constexpr int Q = kStageK / 4;  // float4 per row chunk
    for (int f = threadIdx.x; f < 128 * Q; f += 128) {
        const int row = f / Q, q = f - row * Q;
        const float4 v = row < nrows ? __ldg(reinterpret_cast<const float4 *>(src + (size_t)row * N + k0) + q)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4 *>(st + row * kStageLd + 4 * q) = v;
    }
}

// dst[row * N + k0 ..] = st[row][0..kStageK) for rows < nrows (all 128 threads).
__device__ __forceinline__ void stage_out(const float *st, float *dst, int N, int nrows, int k0) {
    constexpr int Q = kStageK / 4;
    for (int f = threadIdx.x; f < 128 * Q; f += 128) {
        const int row = f / Q, q = f - row * Q;
        if (row < nrows)
            reinterpret_cast<float4 *>(dst + (size_t)row * N + k0)[q] =
                *reinterpret_cast<const float4 *>(st + row * kStageLd + 4 * q);
    }
}

// 16 floats of row `row` from k0 in a padded buffer of row stride ld (16-byte aligned rows).
__device__ __forceinline__ void row_get16_ld(const float *st, int ld, int row, int k0, float *v) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 x = *reinterpret_cast<const float4 *>(st + row * ld + k0 + 4 * q);
        v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
}
__device__ __forceinline__ void row_put16_ld(float *st, int ld, int row, int k0, const float *v) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4 *>(st + row * ld + k0 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2],
                                                                            v[4 * q + 3]);
}

__device__ __forceinline__ void row_get16(const float *st, int row, float *v) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 x = *reinterpret_cast<const float4 *>(st + row * kStageLd + 4 * q);
        v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
}

__device__ __forceinline__ void row_put16(float *st, int row, const float *v) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4 *>(st + row * kStageLd + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2],
                                                                              v[4 * q + 3]);
}

__host__ __device__ constexpr uint32_t tmem_cols_for(int N) { return N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u)); }

// Issue Out = X Op over K = N for the tile in x_hi / x_lo against op_hi / op_lo
// (three products per K-step), then commit to bar. Called by one thread.
__device__ __forceinline__ void issue_split_gemm(uint32_t tmem, const unsigned char *x_hi, const unsigned char *x_lo,
                                                 const unsigned char *op_hi, const unsigned char *op_lo, int N,
                                                 uint64_t *bar) {
    const uint32_t idesc = idesc_bf16(128, N);
    const uint32_t sbo = (uint32_t)N * 16;  // (K / 8) core matrices of 128 B per 8-row group
    const uint32_t xh = smem_u32(x_hi), xl = smem_u32(x_lo), oh = smem_u32(op_hi), ol = smem_u32(op_lo);
    for (int s = 0; s < N / 16; ++s) {
        const uint32_t ko = 256u * s;
        const uint64_t a_hi = smem_desc(xh + ko, 128, sbo), a_lo = smem_desc(xl + ko, 128, sbo);
        const uint64_t b_hi = smem_desc(oh + ko, 128, sbo), b_lo = smem_desc(ol + ko, 128, sbo);
        mma_bf16(tmem, a_hi, b_hi, idesc, s > 0 ? 1u : 0u);
        mma_bf16(tmem, a_hi, b_lo, idesc, 1u);
        mma_bf16(tmem, a_lo, b_hi, idesc, 1u);
    }
    mma_commit(bar);
}

// Write 16 FP32 values of tile row c, columns k0..k0+15 (k0 a multiple of 8), into
// x_hi / x_lo: two 16-byte stores per half (one core-matrix row each).
__device__ __forceinline__ void store_split_row16(unsigned char *x_hi, unsigned char *x_lo, int c, int k0,
                                                  const float *v, int N) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) split_bf16(v[8 * half + i], h[i], l[i]);
        const uint32_t off = kmajor_offset(c, k0 + 8 * half, N);
        *reinterpret_cast<uint4 *>(x_hi + off) = *reinterpret_cast<const uint4 *>(h);
        *reinterpret_cast<uint4 *>(x_lo + off) = *reinterpret_cast<const uint4 *>(l);
    }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Fused FPSA contraction kernels on tensor cores (FP32 data), persistent over
// 128-column tiles. Columns are (cell, node) pairs of one rhs: column index
// j = 2 g + a within rhs r. 128 threads: thread t owns tile row t (accumulator
// lane t); global reads and writes go through the staged, coalesced k-chunks.
//   k_tc_fp_rhs:        phi_half = D psi;  rhs = m (x) M Sigma (phi_half - phi)
//   k_tc_update_scatter: phi = phi_base + D v;  q = M (Sigma phi) + q_ang
// err is set to 1 if an mbarrier wait ran out (the kernel then stops).
// ---------------------------------------------------------------------------
struct TcOps {
    const unsigned char *D;  // D_hi then D_lo, N x N BF16 each, K-major core-matrix layout
    const unsigned char *M;  // M_hi then M_lo
};

// Common prologue: smem carve-up, TMEM allocation, operand staging. Returns false on timeout.
struct TcCta {
    unsigned char *opD_hi, *opD_lo, *opM_hi, *opM_lo, *x_hi, *x_lo;
    float *stA, *stB, *stC;
    uint64_t *bar_copy, *bar_mma;
    uint32_t *tmem_slot;
    uint32_t tmem;
    uint32_t mma_phase;
};

__device__ __forceinline__ bool tc_cta_setup(TcCta &s, unsigned char *smem, const TcOps &ops, int N, int *err,
                                             bool wait_ops = true) {
    const tc::Plan pl = tc::Plan::make(N);
    s.opD_hi = smem;
    s.opD_lo = smem + pl.op_bytes;
    s.opM_hi = smem + 2 * pl.op_bytes;
    s.opM_lo = smem + 3 * pl.op_bytes;
    s.x_hi = smem + 4 * pl.op_bytes;
    s.x_lo = s.x_hi + pl.x_bytes;
    s.stA = reinterpret_cast<float *>(s.x_lo + pl.x_bytes);
    s.stB = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(s.stA) + pl.stage_bytes);
    s.stC = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(s.stB) + pl.stage_bytes);
    unsigned char *tail = reinterpret_cast<unsigned char *>(s.stC) + pl.stage_bytes;
    s.bar_copy = reinterpret_cast<uint64_t *>(tail);
    s.bar_mma = s.bar_copy + 1;
    s.tmem_slot = reinterpret_cast<uint32_t *>(s.bar_mma + 1);
    s.mma_phase = 0;
    if (threadIdx.x == 0) {
        tc::mbar_init(s.bar_copy, 1);
        tc::mbar_init(s.bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(s.tmem_slot, tc::tmem_cols_for(N));
        tc::tmem_relinquish();
    }
    __syncthreads();
    tc::tc_fence_after();
    s.tmem = *s.tmem_slot;
    if (threadIdx.x == 0) {
        tc::mbar_arrive_expect_tx(s.bar_copy, 4 * pl.op_bytes);
        tc::bulk_copy_g2s(s.opD_hi, ops.D, 2 * pl.op_bytes, s.bar_copy);
        tc::bulk_copy_g2s(s.opM_hi, ops.M, 2 * pl.op_bytes, s.bar_copy);
    }
    if (!wait_ops) return true;
    const bool ok = tc::mbar_wait(s.bar_copy, 0);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    return ok;
}

// Wait for the operator copy started by tc_cta_setup(..., wait_ops = false).
__device__ __forceinline__ bool tc_wait_ops(TcCta &s, int *err) {
    const bool ok = tc::mbar_wait(s.bar_copy, 0);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    return ok;
}

__device__ __forceinline__ void tc_cta_teardown(TcCta &s, int N) {
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(s.tmem, tc::tmem_cols_for(N));
}

// Run one split GEMM on the tile already in x_hi / x_lo against (op_hi, op_lo);
// afterwards the accumulator lanes are ready for tcgen05.ld. Returns false on timeout.
__device__ __forceinline__ bool tc_gemm(TcCta &s, const unsigned char *op_hi, const unsigned char *op_lo, int N,
                                        int *err) {
    tc::fence_async_smem();  // the tile's st.shared must be visible to the tensor core
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::tc_fence_after();
        tc::issue_split_gemm(s.tmem, s.x_hi, s.x_lo, op_hi, op_lo, N, s.bar_mma);
    }
    const bool ok = tc::mbar_wait(s.bar_mma, s.mma_phase);
    s.mma_phase ^= 1u;
    tc::tc_fence_after();
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    return ok;
}

__global__ void __launch_bounds__(128) k_tc_fp_rhs(const float *__restrict__ psi_half, const float *__restrict__ phi,
                                                   float *__restrict__ phi_half, const float *__restrict__ sigma_s,
                                                   const double *__restrict__ h, TcOps ops,
                                                   float *__restrict__ rhs, int N, int sumK, int R, int *err) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    TcCta s;
    const bool ok0 = tc_cta_setup(s, smem_tc, ops, N, err);
    tc::grid_dependency_wait();  // the inputs come from the previous kernel
    const int t = threadIdx.x;
    const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
    const int tiles_per_r = (2 * sumK + 127) / 128;
    const int ntiles = tiles_per_r * R;
    bool ok = ok0;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int r = tile / tiles_per_r, j0 = (tile % tiles_per_r) * 128;
        const int ncols = min(128, 2 * sumK - j0), ncell = (ncols + 1) >> 1;
        const bool live = t < ncols;
        const int g = (j0 + t) >> 1;
        const size_t cb = ((size_t)r * sumK * 2 + j0) * N;  // the tile's first element
        const float *sig = sigma_s + (size_t)(j0 >> 1) * N;
        // A = psi columns
        for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
            tc::stage_in(s.stA, psi_half + cb, N, ncols, k0);
            __syncthreads();
            float v[16];
            tc::row_get16(s.stA, t, v);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
            __syncthreads();
        }
        if (!(ok = tc_gemm(s, s.opD_hi, s.opD_lo, N, err))) break;
        // phi_half = D psi; next A = Sigma (phi_half - phi)
        for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
            tc::stage_in(s.stA, phi + cb, N, ncols, k0);
            tc::stage_in(s.stB, sig, N, ncell, k0);
            float a[16];
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
            __syncthreads();
            float ph[16], sg[16], v[16];
            tc::row_get16(s.stA, t, ph);
            tc::row_get16(s.stB, t >> 1, sg);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = live ? sg[i] * (a[i] - ph[i]) : 0.f;
            tc::row_put16(s.stC, t, a);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
            __syncthreads();
            tc::stage_out(s.stC, phi_half + cb, N, ncols, k0);
        }
        if (!(ok = tc_gemm(s, s.opM_hi, s.opM_lo, N, err))) break;
        // rhs = m (x) r: node partner is the adjacent lane (column j ^ 1)
        const float w = live ? (float)(h[g] / 6.0) : 0.f;
        for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
            float a[16], o[16];
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float other = __shfl_xor_sync(0xffffffffu, a[i], 1);  // r at the other node
                o[i] = w * (2.f * a[i] + other);
            }
            __syncthreads();  // stC of the previous chunk has been written out
            tc::row_put16(s.stC, t, o);
            __syncthreads();
            tc::stage_out(s.stC, rhs + cb, N, ncols, k0);
        }
    }
    tc_cta_teardown(s, N);
}

__global__ void __launch_bounds__(128) k_tc_update_scatter(const float *__restrict__ v_in,
                                                           const float *__restrict__ phi_base,
                                                           float *__restrict__ phi, const float *__restrict__ sigma_s,
                                                           TcOps ops, float *__restrict__ q,
                                                           const float *__restrict__ qang, int N, int sumK, int R,
                                                           int *err) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    TcCta s;
    const bool ok0 = tc_cta_setup(s, smem_tc, ops, N, err);
    tc::grid_dependency_wait();  // the inputs come from the previous kernel
    const int t = threadIdx.x;
    const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
    const int tiles_per_r = (2 * sumK + 127) / 128;
    const int ntiles = tiles_per_r * R;
    bool ok = ok0;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int r = tile / tiles_per_r, j0 = (tile % tiles_per_r) * 128;
        const int ncols = min(128, 2 * sumK - j0), ncell = (ncols + 1) >> 1;
        const bool live = t < ncols;
        const size_t cb = ((size_t)r * sumK * 2 + j0) * N;
        const float *sig = sigma_s + (size_t)(j0 >> 1) * N;
        for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
            tc::stage_in(s.stA, v_in + cb, N, ncols, k0);
            __syncthreads();
            float v[16];
            tc::row_get16(s.stA, t, v);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
            __syncthreads();
        }
        if (!(ok = tc_gemm(s, s.opD_hi, s.opD_lo, N, err))) break;
        // phi = phi_base + D v; next A = Sigma phi
        for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
            if (phi_base) tc::stage_in(s.stA, phi_base + cb, N, ncols, k0);
            tc::stage_in(s.stB, sig, N, ncell, k0);
            float a[16];
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
            __syncthreads();
            float pb[16], sg[16], v[16];
            if (phi_base) tc::row_get16(s.stA, t, pb);
            tc::row_get16(s.stB, t >> 1, sg);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                a[i] += phi_base ? pb[i] : 0.f;
                v[i] = live ? sg[i] * a[i] : 0.f;
            }
            tc::row_put16(s.stC, t, a);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
            __syncthreads();
            tc::stage_out(s.stC, phi + cb, N, ncols, k0);
        }
        if (!(ok = tc_gemm(s, s.opM_hi, s.opM_lo, N, err))) break;
        // q = M (Sigma phi) + q_ang
        for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
            if (qang) tc::stage_in(s.stA, qang + cb, N, ncols, k0);
            float a[16];
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
            __syncthreads();
            if (qang) {
                float qa[16];
                tc::row_get16(s.stA, t, qa);
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] += qa[i];
            }
            tc::row_put16(s.stC, t, a);
            __syncthreads();
            tc::stage_out(s.stC, q + cb, N, ncols, k0);
        }
    }
    tc_cta_teardown(s, N);
}

// Whole-tile variants for N <= 64: every global input of a tile is requested by
// asynchronous copies as soon as its buffer is free (the psi / v tile and the phi and
// sigma tiles at the start, overlapping the operator copy and the first GEMM), and
// outputs leave through the staging buffers with coalesced 16-byte stores.
//   stA: psi / v tile, then the outputs;  stB: phi / phi_base, then q_ang;  stC: sigma rows
__global__ void __launch_bounds__(128) k_tc_fp_rhs_tile(const float *__restrict__ psi_half,
                                                        const float *__restrict__ phi, float *__restrict__ phi_half,
                                                        const float *__restrict__ sigma_s, const double *__restrict__ h,
                                                        TcOps ops, float *__restrict__ rhs, int N, int sumK, int R,
                                                        int *err) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    TcCta s;
    const int t = threadIdx.x, ld = N + 4;
    const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
    const int tiles_per_r = (2 * sumK + 127) / 128;
    const int ntiles = tiles_per_r * R;
    bool ok = tc_cta_setup(s, smem_tc, ops, N, err, false);
    tc::grid_dependency_wait();  // the inputs come from the previous kernel
    bool first = true;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int r = tile / tiles_per_r, j0 = (tile % tiles_per_r) * 128;
        const int ncols = min(128, 2 * sumK - j0), ncell = (ncols + 1) >> 1;
        const bool live = t < ncols;
        const int g = (j0 + t) >> 1;
        const size_t cb = ((size_t)r * sumK * 2 + j0) * N;
        tc::tile_load_async(s.stA, psi_half + cb, N, ncols);
        tc::async_commit();
        tc::tile_load_async(s.stB, phi + cb, N, ncols);
        tc::tile_load_async(s.stC, sigma_s + (size_t)(j0 >> 1) * N, N, ncell);
        tc::async_commit();
        if (first && !(ok = tc_wait_ops(s, err))) break;
        first = false;
        tc::async_wait<1>();
        __syncthreads();
        for (int k0 = 0; k0 < N; k0 += 16) {
            float v[16];
            tc::row_get16_ld(s.stA, ld, t, k0, v);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
        }
        if (!(ok = tc_gemm(s, s.opD_hi, s.opD_lo, N, err))) break;
        tc::async_wait<0>();
        __syncthreads();
        // phi_half = D psi -> stA; next A = Sigma (phi_half - phi)
        for (int k0 = 0; k0 < N; k0 += 16) {
            float a[16], ph[16], sg[16], v[16];
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
            tc::row_get16_ld(s.stB, ld, t, k0, ph);
            tc::row_get16_ld(s.stC, ld, t >> 1, k0, sg);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = live ? sg[i] * (a[i] - ph[i]) : 0.f;
            tc::row_put16_ld(s.stA, ld, t, k0, a);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
        }
        __syncthreads();
        tc::tile_store(s.stA, phi_half + cb, N, ncols);
        if (!(ok = tc_gemm(s, s.opM_hi, s.opM_lo, N, err))) break;
        // rhs = m (x) r: node partner is the adjacent lane (column j ^ 1)
        const float w = live ? (float)(h[g] / 6.0) : 0.f;
        for (int k0 = 0; k0 < N; k0 += 16) {
            float a[16], o[16];
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float other = __shfl_xor_sync(0xffffffffu, a[i], 1);
                o[i] = w * (2.f * a[i] + other);
            }
            tc::row_put16_ld(s.stA, ld, t, k0, o);
        }
        __syncthreads();
        tc::tile_store(s.stA, rhs + cb, N, ncols);
        __syncthreads();  // stA / stB / stC free for the next tile's copies
    }
    if (first) tc_wait_ops(s, err);  // no copy may land after the CTA has gone
    tc::async_wait<0>();
    tc_cta_teardown(s, N);
}

__global__ void __launch_bounds__(128) k_tc_update_scatter_tile(const float *__restrict__ v_in,
                                                                const float *__restrict__ phi_base,
                                                                float *__restrict__ phi,
                                                                const float *__restrict__ sigma_s, TcOps ops,
                                                                float *__restrict__ q, const float *__restrict__ qang,
                                                                int N, int sumK, int R, int *err) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    TcCta s;
    const int t = threadIdx.x, ld = N + 4;
    const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
    const int tiles_per_r = (2 * sumK + 127) / 128;
    const int ntiles = tiles_per_r * R;
    bool ok = tc_cta_setup(s, smem_tc, ops, N, err, false);
    tc::grid_dependency_wait();  // the inputs come from the previous kernel
    bool first = true;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int r = tile / tiles_per_r, j0 = (tile % tiles_per_r) * 128;
        const int ncols = min(128, 2 * sumK - j0), ncell = (ncols + 1) >> 1;
        const bool live = t < ncols;
        const size_t cb = ((size_t)r * sumK * 2 + j0) * N;
        tc::tile_load_async(s.stA, v_in + cb, N, ncols);
        tc::async_commit();
        if (phi_base) tc::tile_load_async(s.stB, phi_base + cb, N, ncols);
        tc::tile_load_async(s.stC, sigma_s + (size_t)(j0 >> 1) * N, N, ncell);
        tc::async_commit();
        if (first && !(ok = tc_wait_ops(s, err))) break;
        first = false;
        tc::async_wait<1>();
        __syncthreads();
        for (int k0 = 0; k0 < N; k0 += 16) {
            float v[16];
            tc::row_get16_ld(s.stA, ld, t, k0, v);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
        }
        if (!(ok = tc_gemm(s, s.opD_hi, s.opD_lo, N, err))) break;
        tc::async_wait<0>();
        __syncthreads();
        // phi = phi_base + D v -> stA; next A = Sigma phi
        for (int k0 = 0; k0 < N; k0 += 16) {
            float a[16], pb[16], sg[16], v[16];
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
            if (phi_base) tc::row_get16_ld(s.stB, ld, t, k0, pb);
            tc::row_get16_ld(s.stC, ld, t >> 1, k0, sg);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                a[i] += phi_base ? pb[i] : 0.f;
                v[i] = live ? sg[i] * a[i] : 0.f;
            }
            tc::row_put16_ld(s.stA, ld, t, k0, a);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
        }
        __syncthreads();
        if (qang) {  // stB is free now: the q_ang tile arrives during the second GEMM
            tc::tile_load_async(s.stB, qang + cb, N, ncols);
        }
        tc::async_commit();
        tc::tile_store(s.stA, phi + cb, N, ncols);
        if (!(ok = tc_gemm(s, s.opM_hi, s.opM_lo, N, err))) break;
        tc::async_wait<0>();
        __syncthreads();
        // q = M (Sigma phi) + q_ang
        for (int k0 = 0; k0 < N; k0 += 16) {
            float a[16];
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
            if (qang) {
                float qa[16];
                tc::row_get16_ld(s.stB, ld, t, k0, qa);
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] += qa[i];
            }
            tc::row_put16_ld(s.stA, ld, t, k0, a);
        }
        __syncthreads();
        tc::tile_store(s.stA, q + cb, N, ncols);
        __syncthreads();
    }
    if (first) tc_wait_ops(s, err);  // no copy may land after the CTA has gone
    tc::async_wait<0>();
    tc_cta_teardown(s, N);
}

// ---------------------------------------------------------------------------
// Streamed-operator variants for N > 128 (N a multiple of 32, at most 256): the
// operators (2 N^2 BF16 values each, split hi / lo) no longer fit shared memory next
// to the column tile, so each GEMM streams them through three buffers in K-chunks of
// 32 (an operator is stored chunk-major in global memory, [N / 32 chunks][N rows][32]
// in the K-major core-matrix layout, so a chunk is one bulk copy; the operators are
// shared by every tile and stay in L2); a buffer is refilled once the MMAs of the
// chunk before the current one have read it, so two copies stay in flight while a
// chunk is multiplied. The column tile (the A operand, 128 x N) is split from FP32
// rows that each thread reads straight from global memory (row t of the tile is the
// thread's accumulator lane), and every epilogue reads and writes its row the same
// way, four 16-byte accesses per 16 columns and no block barrier between k-chunks,
// several k-chunks of loads in flight per thread. The accumulator is N FP32 columns
// of TMEM (M = 128, N = 256 per instruction).
// ---------------------------------------------------------------------------
namespace tc {
constexpr int kChunkK = 32;
constexpr int kBigBufs = 3;
// byte offset of element (row, k) of an N x N operator in the chunk-major layout
__host__ __device__ __forceinline__ uint32_t chunk_offset(int row, int k, int N) {
    return (uint32_t)(k / kChunkK) * (uint32_t)N * kChunkK * 2u + kmajor_offset(row, k % kChunkK, kChunkK);
}
// Shared-memory plan of a streamed CTA: x_hi, x_lo (128 x N BF16 each), three chunk
// buffers of hi + lo (N x 32 BF16 each), 7 mbarriers, tmem slot.
struct BigPlan {
    uint32_t x_bytes, chunk_bytes, total;
    __host__ __device__ static BigPlan make(int N) {
        BigPlan p;
        p.x_bytes = 128u * N * 2;
        p.chunk_bytes = (uint32_t)N * kChunkK * 2;  // one part (hi or lo) of one chunk
        p.total = 2 * p.x_bytes + 2 * kBigBufs * p.chunk_bytes + 128;
        return p;
    }
};

// 16 consecutive floats at p (16-byte aligned) through L2, or zeros.
__device__ __forceinline__ void ld_row16(const float *p, bool live, float *v) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 x = live ? __ldcg(reinterpret_cast<const float4 *>(p) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
}
__device__ __forceinline__ void st_row16(float *p, const float *v) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        reinterpret_cast<float4 *>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
// Row t of the tile (N floats at src, zeros when not live), scaled elementwise by
// scale (N floats, NULL: none), split into x_hi / x_lo; 64 columns of loads in flight.
__device__ __forceinline__ void load_split_row(const float *src, const float *scale, bool live, int N,
                                               unsigned char *x_hi, unsigned char *x_lo, int t) {
    for (int k0 = 0; k0 < N; k0 += 64) {
        float v[4][16], sc[4][16];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = live && k0 + 16 * j < N;
            ld_row16(src + k0 + 16 * j, in, v[j]);
            if (scale) ld_row16(scale + k0 + 16 * j, in, sc[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (k0 + 16 * j >= N) break;
            if (scale) {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[j][i] *= sc[j][i];
            }
            store_split_row16(x_hi, x_lo, t, k0 + 16 * j, v[j], N);
        }
    }
}
}  // namespace tc

struct TcBig {
    unsigned char *x_hi, *x_lo, *ch[tc::kBigBufs];  // ch[b]: hi then lo of buffer b
    uint64_t *full, *empty, *bar_mma;               // full[kBigBufs], empty[kBigBufs]
    uint32_t *tmem_slot;
    uint32_t tmem, mma_phase;
    uint32_t fills[tc::kBigBufs], reqs[tc::kBigBufs], commits[tc::kBigBufs];  // thread 0's view
};

__device__ __forceinline__ void tc_big_setup(TcBig &s, unsigned char *smem, int N) {
    const tc::BigPlan pl = tc::BigPlan::make(N);
    s.x_hi = smem;
    s.x_lo = smem + pl.x_bytes;
    for (int b = 0; b < tc::kBigBufs; ++b) {
        s.ch[b] = smem + 2 * pl.x_bytes + 2 * b * pl.chunk_bytes;
        s.fills[b] = s.reqs[b] = s.commits[b] = 0;
    }
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * pl.x_bytes + 2 * tc::kBigBufs * pl.chunk_bytes);
    s.full = bars;
    s.empty = bars + tc::kBigBufs;
    s.bar_mma = bars + 2 * tc::kBigBufs;
    s.tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * tc::kBigBufs + 1);
    s.mma_phase = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * tc::kBigBufs + 1; ++i) tc::mbar_init(bars + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(s.tmem_slot, tc::tmem_cols_for(N));
        tc::tmem_relinquish();
    }
    __syncthreads();
    tc::tc_fence_after();
    s.tmem = *s.tmem_slot;
}

// Out = X Op^T over K = N with the tile in x_hi / x_lo and the operator (hi, lo:
// chunk-major in global memory) streamed chunk by chunk; returns false on a timeout.
// Thread 0 runs the pipeline: chunks 0..2 are requested at once; after the MMAs of
// chunk c are issued, the buffer of chunk c - 1 is refilled with chunk c + 2 once
// those earlier MMAs have read it (its empty barrier), so the tensor core is not held
// up by the copy just requested. Every wait is bounded.
__device__ __forceinline__ bool tc_gemm_streamed(TcBig &s, const unsigned char *op_hi, const unsigned char *op_lo,
                                                 int N, int *err) {
    constexpr int NB = tc::kBigBufs;
    tc::fence_async_smem();  // the tile's st.shared must be visible to the tensor core
    tc::tc_fence_before();
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) {
        tc::tc_fence_after();
        const int nch = N / tc::kChunkK;
        const uint32_t cb = (uint32_t)N * tc::kChunkK * 2;
        auto request = [&](int c) {
            const int b = c % NB;
            tc::mbar_arrive_expect_tx(&s.full[b], 2 * cb);
            tc::bulk_copy_g2s(s.ch[b], op_hi + (size_t)c * cb, cb, &s.full[b]);
            tc::bulk_copy_g2s(s.ch[b] + cb, op_lo + (size_t)c * cb, cb, &s.full[b]);
            ++s.reqs[b];
        };
        int issued = 0;
        while (issued < nch && issued < NB) request(issued++);
        const uint32_t idesc = tc::idesc_bf16(128, N);
        const uint32_t xh = tc::smem_u32(s.x_hi), xl = tc::smem_u32(s.x_lo);
        const uint32_t sbo_x = (uint32_t)N * 16, sbo_b = tc::kChunkK * 16;
        for (int c = 0; c < nch && ok; ++c) {
            const int b = c % NB;
            ok = tc::mbar_wait(&s.full[b], s.fills[b] & 1u);
            if (!ok) break;
            ++s.fills[b];
            tc::tc_fence_after();
            const uint32_t oh = tc::smem_u32(s.ch[b]), ol = oh + cb;
            for (int j = 0; j < tc::kChunkK / 16; ++j) {
                const uint32_t ka = 256u * (uint32_t)(c * (tc::kChunkK / 16) + j), kb = 256u * (uint32_t)j;
                const uint64_t a_hi = tc::smem_desc(xh + ka, 128, sbo_x), a_lo = tc::smem_desc(xl + ka, 128, sbo_x);
                const uint64_t b_hi = tc::smem_desc(oh + kb, 128, sbo_b), b_lo = tc::smem_desc(ol + kb, 128, sbo_b);
                tc::mma_bf16(s.tmem, a_hi, b_hi, idesc, (c > 0 || j > 0) ? 1u : 0u);
                tc::mma_bf16(s.tmem, a_hi, b_lo, idesc, 1u);
                tc::mma_bf16(s.tmem, a_lo, b_hi, idesc, 1u);
            }
            tc::mma_commit(&s.empty[b]);
            ++s.commits[b];
            if (c >= 1 && issued < nch) {  // chunk c - 1 + NB into the buffer of chunk c - 1
                const int bp = (c - 1) % NB;
                ok = tc::mbar_wait(&s.empty[bp], (s.commits[bp] - 1u) & 1u);
                if (!ok) break;
                request(issued++);
            }
        }
        tc::mma_commit(s.bar_mma);
        // every buffer's last commit has landed (its phases stay in step for the next
        // GEMM), and on a timeout no requested copy is still landing (bounded)
        for (int b = 0; b < NB; ++b) {
            if (s.commits[b] > 0 && !tc::mbar_wait(&s.empty[b], (s.commits[b] - 1u) & 1u)) ok = false;
            while (s.fills[b] < s.reqs[b]) {
                if (!tc::mbar_wait(&s.full[b], s.fills[b] & 1u)) {
                    ok = false;
                    break;
                }
                ++s.fills[b];
            }
        }
    }
    ok = __syncthreads_and(ok) != 0;
    // every MMA issued has completed before the accumulator is read or the CTA ends (bounded)
    const bool done = tc::mbar_wait(s.bar_mma, s.mma_phase);
    s.mma_phase ^= 1u;
    tc::tc_fence_after();
    ok = __syncthreads_and(ok && done) != 0;
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    return ok;
}

__device__ __forceinline__ void tc_big_teardown(TcBig &s, int N) {
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(s.tmem, tc::tmem_cols_for(N));
}

// k_tc_fp_rhs with streamed operators (N > 128).
__global__ void __launch_bounds__(128) k_tc_fp_rhs_big(const float *__restrict__ psi_half,
                                                       const float *__restrict__ phi, float *__restrict__ phi_half,
                                                       const float *__restrict__ sigma_s,
                                                       const double *__restrict__ h, TcOps ops,
                                                       float *__restrict__ rhs, int N, int sumK, int R, int *err) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    TcBig s;
    tc_big_setup(s, smem_tc, N);
    tc::grid_dependency_wait();  // the inputs come from the previous kernel
    const int t = threadIdx.x;
    const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
    const int tiles_per_r = (2 * sumK + 127) / 128;
    const int ntiles = tiles_per_r * R;
    const size_t opb = (size_t)N * N * 2;  // bytes of one part of one operator
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int r = tile / tiles_per_r, j0 = (tile % tiles_per_r) * 128;
        const int ncols = min(128, 2 * sumK - j0);
        const bool live = t < ncols;
        const int g = live ? (j0 + t) >> 1 : 0;
        const size_t row = ((size_t)r * sumK * 2 + j0 + t) * N;  // this thread's column of the tile
        tc::load_split_row(psi_half + row, nullptr, live, N, s.x_hi, s.x_lo, t);
        if (!(ok = tc_gemm_streamed(s, ops.D, ops.D + opb, N, err))) break;
        // phi_half = D psi_half; next A = Sigma (phi_half - phi)
        const float *sig = sigma_s + (size_t)g * N;
        for (int k0 = 0; k0 < N; k0 += 16) {
            float a[16], ph[16], sg[16], v[16];
            tc::ld_row16(phi + row + k0, live, ph);
            tc::ld_row16(sig + k0, live, sg);
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = live ? sg[i] * (a[i] - ph[i]) : 0.f;
            if (live) tc::st_row16(phi_half + row + k0, a);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
        }
        if (!(ok = tc_gemm_streamed(s, ops.M, ops.M + opb, N, err))) break;
        // rhs = m (x) r: the node partner is the adjacent lane (column j ^ 1)
        const float w = live ? (float)(h[g] / 6.0) : 0.f;
        for (int k0 = 0; k0 < N; k0 += 16) {
            float a[16], o[16];
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float other = __shfl_xor_sync(0xffffffffu, a[i], 1);
                o[i] = w * (2.f * a[i] + other);
            }
            if (live) tc::st_row16(rhs + row + k0, o);
        }
    }
    tc_big_teardown(s, N);
}

// k_tc_update_scatter with streamed operators (N > 128).
__global__ void __launch_bounds__(128) k_tc_update_scatter_big(const float *__restrict__ v_in,
                                                               const float *__restrict__ phi_base,
                                                               float *__restrict__ phi,
                                                               const float *__restrict__ sigma_s, TcOps ops,
                                                               float *__restrict__ q, const float *__restrict__ qang,
                                                               int N, int sumK, int R, int *err) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    TcBig s;
    tc_big_setup(s, smem_tc, N);
    tc::grid_dependency_wait();  // the inputs come from the previous kernel
    const int t = threadIdx.x;
    const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
    const int tiles_per_r = (2 * sumK + 127) / 128;
    const int ntiles = tiles_per_r * R;
    const size_t opb = (size_t)N * N * 2;
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int r = tile / tiles_per_r, j0 = (tile % tiles_per_r) * 128;
        const int ncols = min(128, 2 * sumK - j0);
        const bool live = t < ncols;
        const int g = live ? (j0 + t) >> 1 : 0;
        const size_t row = ((size_t)r * sumK * 2 + j0 + t) * N;
        tc::load_split_row(v_in + row, nullptr, live, N, s.x_hi, s.x_lo, t);
        if (!(ok = tc_gemm_streamed(s, ops.D, ops.D + opb, N, err))) break;
        // phi = phi_base + D v (read before written: phi_base may alias phi); next A = Sigma phi
        const float *sig = sigma_s + (size_t)g * N;
        for (int k0 = 0; k0 < N; k0 += 16) {
            float a[16], pb[16], sg[16], v[16];
            tc::ld_row16(phi_base ? phi_base + row + k0 : nullptr, live && phi_base, pb);
            tc::ld_row16(sig + k0, live, sg);
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                a[i] += pb[i];
                v[i] = live ? sg[i] * a[i] : 0.f;
            }
            if (live) tc::st_row16(phi + row + k0, a);
            tc::store_split_row16(s.x_hi, s.x_lo, t, k0, v, N);
        }
        if (!(ok = tc_gemm_streamed(s, ops.M, ops.M + opb, N, err))) break;
        // q = M (Sigma phi) + q_ang
        for (int k0 = 0; k0 < N; k0 += 16) {
            float a[16], qa[16];
            tc::ld_row16(qang ? qang + row + k0 : nullptr, live && qang, qa);
            tc::tmem_ld16(s.tmem + lane_base + k0, a);
#pragma unroll
            for (int i = 0; i < 16; ++i) a[i] += qa[i];
            if (live) tc::st_row16(q + row + k0, a);
        }
    }
    tc_big_teardown(s, N);
}

// ---------------------------------------------------------------------------
// Tensor-core contractions of the GMRES operator (the FP32 inner solve of GMRES-IR),
// one GEMM each, with the operators either in shared memory (N <= 128) or streamed
// (N > 128); TcEngine picks the form at compile time.
//   k_tc_fp_rhs_moments:  rhs = m (x) M Sigma v      (v: moments)
//   k_tc_moments_axpy:    out = base + sign D psi   (base may be NULL or alias out)
// ---------------------------------------------------------------------------
template <bool kBig>
struct TcEngine {
    TcCta a;
    TcBig b;
    float *stA, *stB, *stC;
    unsigned char *x_hi, *x_lo;
    uint32_t tmem;
    __device__ __forceinline__ bool setup(unsigned char *smem, const TcOps &ops, int N, int *err) {
        bool ok = true;
        if constexpr (kBig) {  // global I/O straight from the threads' rows: no staging buffers
            tc_big_setup(b, smem, N);
            stA = stB = stC = nullptr;
            x_hi = b.x_hi; x_lo = b.x_lo; tmem = b.tmem;
        } else {
            ok = tc_cta_setup(a, smem, ops, N, err);
            stA = a.stA; stB = a.stB; stC = a.stC; x_hi = a.x_hi; x_lo = a.x_lo; tmem = a.tmem;
        }
        return ok;
    }
    __device__ __forceinline__ bool gemm(const TcOps &ops, bool use_d, int N, int *err) {
        if constexpr (kBig) {
            const unsigned char *o = use_d ? ops.D : ops.M;
            return tc_gemm_streamed(b, o, o + (size_t)N * N * 2, N, err);
        } else {
            return tc_gemm(a, use_d ? a.opD_hi : a.opM_hi, use_d ? a.opD_lo : a.opM_lo, N, err);
        }
    }
    __device__ __forceinline__ void teardown(int N) {
        if constexpr (kBig) tc_big_teardown(b, N);
        else tc_cta_teardown(a, N);
    }
};

template <bool kBig>
__global__ void __launch_bounds__(128) k_tc_fp_rhs_moments(const float *__restrict__ v,
                                                           const float *__restrict__ sigma_s,
                                                           const double *__restrict__ h, TcOps ops,
                                                           float *__restrict__ rhs, int N, int sumK, int R, int *err) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    TcEngine<kBig> e;
    bool ok = e.setup(smem_tc, ops, N, err);
    tc::grid_dependency_wait();  // the inputs come from the previous kernel
    const int t = threadIdx.x;
    const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
    const int tiles_per_r = (2 * sumK + 127) / 128;
    const int ntiles = tiles_per_r * R;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int r = tile / tiles_per_r, j0 = (tile % tiles_per_r) * 128;
        const int ncols = min(128, 2 * sumK - j0), ncell = (ncols + 1) >> 1;
        const bool live = t < ncols;
        const int g = (j0 + t) >> 1;
        const size_t cb = ((size_t)r * sumK * 2 + j0) * N;
        const float *sig = sigma_s + (size_t)(j0 >> 1) * N;
        // A = Sigma v
        if constexpr (kBig) {
            tc::load_split_row(v + cb + (size_t)t * N, sigma_s + (size_t)(live ? g : 0) * N, live, N, e.x_hi,
                               e.x_lo, t);
        } else {
            for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
                tc::stage_in(e.stA, v + cb, N, ncols, k0);
                tc::stage_in(e.stB, sig, N, ncell, k0);
                __syncthreads();
                float vv[16], sg[16], a[16];
                tc::row_get16(e.stA, t, vv);
                tc::row_get16(e.stB, t >> 1, sg);
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] = live ? sg[i] * vv[i] : 0.f;
                tc::store_split_row16(e.x_hi, e.x_lo, t, k0, a, N);
                __syncthreads();
            }
        }
        if (!(ok = e.gemm(ops, false, N, err))) break;
        // rhs = m (x) r: node partner is the adjacent lane (column j ^ 1)
        const float w = live ? (float)(h[g] / 6.0) : 0.f;
        for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
            float a[16], o[16];
            tc::tmem_ld16(e.tmem + lane_base + k0, a);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float other = __shfl_xor_sync(0xffffffffu, a[i], 1);
                o[i] = w * (2.f * a[i] + other);
            }
            if constexpr (kBig) {
                if (live) tc::st_row16(rhs + cb + (size_t)t * N + k0, o);
            } else {
                __syncthreads();  // stC of the previous chunk has been written out
                tc::row_put16(e.stC, t, o);
                __syncthreads();
                tc::stage_out(e.stC, rhs + cb, N, ncols, k0);
            }
        }
    }
    e.teardown(N);
}

template <bool kBig>
__global__ void __launch_bounds__(128) k_tc_moments_axpy(const float *__restrict__ psi, const float *base, float sign,
                                                         TcOps ops, float *out, int N, int sumK, int R, int *err) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    TcEngine<kBig> e;
    bool ok = e.setup(smem_tc, ops, N, err);
    tc::grid_dependency_wait();  // the inputs come from the previous kernel
    const int t = threadIdx.x;
    const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
    const int tiles_per_r = (2 * sumK + 127) / 128;
    const int ntiles = tiles_per_r * R;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int r = tile / tiles_per_r, j0 = (tile % tiles_per_r) * 128;
        const int ncols = min(128, 2 * sumK - j0);
        const size_t cb = ((size_t)r * sumK * 2 + j0) * N;
        if constexpr (kBig) {
            tc::load_split_row(psi + cb + (size_t)t * N, nullptr, t < ncols, N, e.x_hi, e.x_lo, t);
        } else {
            for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
                tc::stage_in(e.stA, psi + cb, N, ncols, k0);
                __syncthreads();
                float vv[16];
                tc::row_get16(e.stA, t, vv);
                tc::store_split_row16(e.x_hi, e.x_lo, t, k0, vv, N);
                __syncthreads();
            }
        }
        if (!(ok = e.gemm(ops, true, N, err))) break;
        // out = base + sign D psi (base read chunk by chunk before out is written: it may alias)
        for (int k0 = 0; k0 < N; k0 += tc::kStageK) {
            if constexpr (kBig) {
                const bool live = t < ncols;
                const size_t row = cb + (size_t)t * N + k0;
                float a[16], bs[16];
                tc::ld_row16(base ? base + row : nullptr, live && base, bs);
                tc::tmem_ld16(e.tmem + lane_base + k0, a);
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] = bs[i] + sign * a[i];
                if (live) tc::st_row16(out + row, a);
            } else {
                if (base) tc::stage_in(e.stA, base + cb, N, ncols, k0);
                float a[16];
                tc::tmem_ld16(e.tmem + lane_base + k0, a);
                __syncthreads();
                float bs[16];
                if (base) tc::row_get16(e.stA, t, bs);
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] = (base ? bs[i] : 0.f) + sign * a[i];
                tc::row_put16(e.stC, t, a);
                __syncthreads();
                tc::stage_out(e.stC, out + cb, N, ncols, k0);
            }
        }
    }
    e.teardown(N);
}

}  // namespace fpsa
