// Block GEMMs of the recursive block inversion on the tensor cores (FP32 factors
// of the mixed-precision path with 2N = 256 or 512, Sec. 4's factorized FP operator).
//
// The recursive block-Schur inversion of `bcr_large.cuh` spends almost all of its
// flops in six products of h x h blocks per level of recursion (h = 2N / 2, 2N / 4,
// down to 128). Here each product
//   C = alpha A B + beta C        (n x n blocks of a batch, n = 128 or 256)
// is one tcgen05 GEMM per 128-row tile of C: M = 128, N = n, accumulated in FP32 in
// tensor memory (n columns). Precision: split BF16 with three products, as in the
// contractions, A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped terms are
// about 2^-17 of each product); the factors are the FP correction's preconditioner,
// so this changes the convergence rate by rounding only, never the fixed point.
//
// K is streamed in chunks of 32 through two shared-memory stages: the CTA's 256
// threads load a chunk of A (128 rows x 32, row-major, k contiguous) and of B
// (32 rows x n, col contiguous) from global memory into registers one chunk ahead,
// split them and store both as K-major BF16 operands in the core-matrix layout (B
// transposed on the way, so the B operand is the N x K matrix B^T). A stage is
// overwritten only after the MMAs that read it have signalled its mbarrier. Every
// wait is bounded; on a timeout the CTA records the error, waits (bounded) for its
// products in flight, frees its tensor memory and returns without writing C.
#pragma once

#include "bcr_large.cuh"
#include "tc_contract.cuh"

namespace fpsa {
namespace bgt {

constexpr int kThreads = 256;
constexpr int kKc = 32;  // K columns of a streamed chunk: two MMA K-steps of 16
// one part (hi or lo) of an A chunk (128 x 32 BF16) and of a B chunk (n x 32 BF16)
__host__ __device__ constexpr uint32_t a_bytes() { return 128u * kKc * 2u; }
__host__ __device__ constexpr uint32_t b_bytes(int n) { return (uint32_t)n * kKc * 2u; }
// a stage: A_hi, A_lo, B_hi, B_lo
__host__ __device__ constexpr uint32_t stage_bytes(int n) { return 2u * (a_bytes() + b_bytes(n)); }
// two stages, 3 mbarriers (stage 0, stage 1, done) and the tensor-memory slot
__host__ __device__ constexpr uint32_t smem_bytes(int n) { return 2u * stage_bytes(n) + 64u; }

}  // namespace bgt

// grid (n / 128 row tiles, batch elements), 256 threads; C never aliases A or B.
template <int NB>
__global__ void __launch_bounds__(bgt::kThreads) k_bgemm_tc(float alpha, BMat<float> A, BMat<float> B, float beta,
                                                            BMat<float> C, const BcrItem *__restrict__ items,
                                                            int *__restrict__ err) {
    static_assert(NB == 128 || NB == 256, "n must be 128 or 256");
    using namespace bgt;
    extern __shared__ __align__(128) unsigned char smem_bg[];
    constexpr uint32_t SB = stage_bytes(NB);
    constexpr int NCH = NB / kKc;
    const int e = blockIdx.y, rt = blockIdx.x;
    const float *a = bmat_ptr(A, items, e) + (size_t)rt * 128 * A.ld;
    const float *b = bmat_ptr(B, items, e);
    float *c = bmat_ptr(C, items, e) + (size_t)rt * 128 * C.ld;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_bg + 2 * SB);  // stage[0], stage[1], done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3);
    const int t = threadIdx.x;
    if (t == 0) {
        for (int i = 0; i < 3; ++i) tc::mbar_init(bars + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (t < 32) {
        tc::tmem_alloc(tslot, (uint32_t)NB);
        tc::tmem_relinquish();
    }
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    // A: thread t loads row t / 2, k-half t % 2 of the chunk (16 values); B: column
    // t % NB, k range (t / NB) * KB .. + KB of the chunk
    constexpr int KB = kKc * NB / kThreads;  // 32 (NB = 256) or 16 (NB = 128)
    const int arow = t >> 1, akh = t & 1;
    const int bcol = t % NB, bk0 = (t / NB) * KB;
    float ra[16], rb[KB];
    auto load = [&](int ch) {
        const int k0 = ch * kKc;
        const float4 *src = reinterpret_cast<const float4 *>(a + (size_t)arow * A.ld + k0 + 16 * akh);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = __ldg(src + q);
            ra[4 * q] = v.x; ra[4 * q + 1] = v.y; ra[4 * q + 2] = v.z; ra[4 * q + 3] = v.w;
        }
        const float *bs = b + (size_t)(k0 + bk0) * B.ld + bcol;
#pragma unroll
        for (int k = 0; k < KB; ++k) rb[k] = __ldg(bs + (size_t)k * B.ld);
    };
    auto split8 = [](const float *v, uint4 &hi, uint4 &lo) {
        __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) tc::split_bf16(v[i], h[i], l[i]);
        hi = *reinterpret_cast<const uint4 *>(h);
        lo = *reinterpret_cast<const uint4 *>(l);
    };
    auto store = [&](int s) {
        unsigned char *st = smem_bg + s * SB;
        unsigned char *bh = st + 2 * a_bytes(), *bl = bh + b_bytes(NB);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint4 hi, lo;
            split8(ra + 8 * half, hi, lo);
            const uint32_t off = tc::kmajor_offset(arow, 16 * akh + 8 * half, kKc);
            *reinterpret_cast<uint4 *>(st + off) = hi;
            *reinterpret_cast<uint4 *>(st + a_bytes() + off) = lo;
        }
#pragma unroll
        for (int g = 0; g < KB / 8; ++g) {
            uint4 hi, lo;
            split8(rb + 8 * g, hi, lo);
            const uint32_t off = tc::kmajor_offset(bcol, bk0 + 8 * g, kKc);
            *reinterpret_cast<uint4 *>(bh + off) = hi;
            *reinterpret_cast<uint4 *>(bl + off) = lo;
        }
    };

    const uint32_t idesc = tc::idesc_bf16(128, NB);
    constexpr uint32_t kSbo = kKc * 16;  // 8-row groups of a K = 32 operand are 512 B apart
    uint32_t uses[2] = {0u, 0u};         // commits issued on each stage's mbarrier
    bool ok = true;
    load(0);
    for (int ch = 0; ch < NCH; ++ch) {
        const int s = ch & 1;
        // the stage is free once the MMAs of chunk ch - 2 have read it
        if (uses[s] > 0) ok = tc::mbar_wait(&bars[s], (uses[s] - 1u) & 1u);
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        store(s);
        tc::fence_async_smem();  // the st.shared above must be visible to the tensor core
        tc::tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc::tc_fence_after();
            const uint32_t ah = tc::smem_u32(smem_bg + s * SB), al = ah + a_bytes(), bh = al + a_bytes(),
                           bl = bh + b_bytes(NB);
#pragma unroll
            for (int j = 0; j < kKc / 16; ++j) {
                const uint32_t ko = 256u * j;
                const uint64_t dah = tc::smem_desc(ah + ko, 128, kSbo), dal = tc::smem_desc(al + ko, 128, kSbo);
                const uint64_t dbh = tc::smem_desc(bh + ko, 128, kSbo), dbl = tc::smem_desc(bl + ko, 128, kSbo);
                tc::mma_bf16(tmem, dah, dbh, idesc, (ch > 0 || j > 0) ? 1u : 0u);
                tc::mma_bf16(tmem, dah, dbl, idesc, 1u);
                tc::mma_bf16(tmem, dal, dbh, idesc, 1u);
            }
            tc::mma_commit(&bars[s]);
        }
        ++uses[s];
        if (ch + 1 < NCH) load(ch + 1);  // global loads in flight while the MMAs run
    }
    // every MMA issued has completed before tensor memory is read or freed (bounded)
    if (t == 0) tc::mma_commit(&bars[2]);
    bool done = tc::mbar_wait(&bars[2], 0u);
    for (int s = 0; s < 2; ++s)
        if (uses[s] > 0) done = tc::mbar_wait(&bars[s], (uses[s] - 1u) & 1u) && done;
    tc::tc_fence_after();
    ok = __syncthreads_and(ok && done) != 0;
    if (ok) {
        // epilogue: warp w reads accumulator lanes 32 (w % 4) .. + 31 (tile rows) and
        // column half w / 4
        const int q = (t >> 5) & 3, hc = t >> 7;
        const int row = 32 * q + (t & 31);
        float *crow = c + (size_t)row * C.ld;
#pragma unroll 1
        for (int c0 = hc * (NB / 2); c0 < (hc + 1) * (NB / 2); c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
            float4 *dst = reinterpret_cast<float4 *>(crow + c0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float4 o = make_float4(alpha * v[4 * i], alpha * v[4 * i + 1], alpha * v[4 * i + 2],
                                       alpha * v[4 * i + 3]);
                if (beta != 0.f) {
                    const float4 old = dst[i];
                    o.x = fmaf(beta, old.x, o.x);
                    o.y = fmaf(beta, old.y, o.y);
                    o.z = fmaf(beta, old.z, o.z);
                    o.w = fmaf(beta, old.w, o.w);
                }
                dst[i] = o;
            }
        }
    } else if (t == 0) {
        atomicExch(err, 1);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tmem, (uint32_t)NB);
}

}  // namespace fpsa
