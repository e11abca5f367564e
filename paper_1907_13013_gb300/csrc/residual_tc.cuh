// The FP64 refinement residual of the mixed-precision path with its two angular
// contractions on the tensor cores, exact to FP64 working accuracy.
//
// k_mixed_residual computes, per column (cell, node, rhs) of the FP64 iterate psi,
//   phi = D psi,   x = Sigma phi + Q,   s = M x (Eqs. phi-mom, treq),
// then the LD transport residual of that column. GB300's FP64 rate (about 1.2 TFLOP/s)
// makes the two N x N contractions the whole cost of the kernel. Here each contraction
// is an exact integer computation on the BF16 tensor cores:
//   - every row r of the input (a column's N values) is scaled by its own power of two,
//     x~ = x 2^-e_r with |x~| < 1 (e_r from frexp of max |x|), and written as the 56-bit
//     fixed-point integer q = rint(x~ 2^56); q = sign * sum_i dig_i 2^(49 - 7 i), i < 8,
//     with 7-bit digits dig_i in [0, 127]: x~ = sum_i s_i 2^(-7 (i + 1)), s_i = sign dig_i;
//   - every row o of the operator likewise (host side, once per context): t_j, e_o;
//   - x~ . op~ = sum_d 2^(-7 (d + 2)) A_d with A_d = sum_{i + j = d} sum_k s_i t_j over
//     the 36 digit pairs with i + j <= 7 (the dropped pairs weigh 2^-70 or less).
// Every product s_i t_j is an integer of magnitude below 2^14 and, for i + j = d >= 1,
// below 2^13; over K <= 256 terms and d + 1 pairs every partial sum stays an integer of
// magnitude at most 2^24, so the FP32 accumulation of the BF16 products in tensor
// memory is exact (A_d in its own accumulator, 8 x OC TMEM columns). The A_d are then
// combined in FP64, scaled by 2^(e_r + e_o): the only roundings are the 56-bit
// truncation of each row relative to its largest entry and the FP64 combination, i.e.
// the accuracy of an FP64 dot product.
//
// One CTA per tile of 64 cells x 2 nodes = 128 columns (tensor-memory lane = column),
// 128 threads. For each output chunk of OC = 64 rows (32 where 64 does not divide N)
// and each K-chunk of 32:
// thread 0 copies the operator's 8 digit slices of that block (OC x 32 BF16 each,
// stored K-major in the core-matrix layout, one bulk copy), every thread writes the 8
// digit slices of its column's 32 inputs (K-major), and thread 0 issues the 72 MMAs
// (36 pairs, two K-steps; M = 128, N = OC, K = 16). Waits are bounded; on a timeout
// the CTA records the error, waits (bounded) for its copies and products, frees its
// tensor memory and stops.
#pragma once

#include "kernels.cuh"
#include "tc_contract.cuh"

namespace fpsa {
namespace rtc {

constexpr int S = 8;    // digit slices: 56-bit fixed point per row
constexpr int KC = 32;  // K per chunk: two MMA K-steps
constexpr int kThreads = 128;
// output rows per chunk: 64 where they divide N, else 32 (N is a multiple of 32)
__host__ __device__ constexpr int oc_of(int N) { return N % 64 == 0 ? 64 : 32; }
__host__ __device__ constexpr uint32_t a_slice_bytes() { return 128u * KC * 2u; }
__host__ __device__ constexpr uint32_t b_slice_bytes(int N) { return (uint32_t)oc_of(N) * KC * 2u; }
__host__ __device__ constexpr uint32_t b_block_bytes(int N) { return S * b_slice_bytes(N); }
__host__ __device__ constexpr uint32_t smem_bytes(int N) { return S * a_slice_bytes() + b_block_bytes(N) + 64u; }
__host__ __device__ constexpr uint32_t tmem_cols(int N) { return (uint32_t)(S * oc_of(N)) <= 256u ? 256u : 512u; }
__host__ __device__ constexpr bool applies(int N) { return N % KC == 0 && N >= KC && N <= 256; }
// byte offset of operator block (oc, kc) in the stored digit slices
__host__ __device__ constexpr size_t block_offset(int N, int oc, int kc) {
    return ((size_t)oc * (N / KC) + kc) * b_block_bytes(N);
}

// The operator's digit slices (host side): op [No][K] row-major (No = K = N), out sized
// (N / OC) (N / KC) b_block_bytes(N) bytes, exps [N]. Same digits as the device side.
inline void slice_operator(const double *op, int N, unsigned char *out, int32_t *exps) {
    const int OC = oc_of(N);
    for (int o = 0; o < N; ++o) {
        double mx = 0.0;
        for (int k = 0; k < N; ++k) mx = std::fmax(mx, std::fabs(op[(size_t)o * N + k]));
        int e = 0;
        if (mx > 0.0) std::frexp(mx, &e);
        exps[o] = e;
        for (int k = 0; k < N; ++k) {
            const long long q = std::llrint(std::ldexp(op[(size_t)o * N + k], 56 - e));
            const unsigned long long u = (unsigned long long)(q < 0 ? -q : q);
            unsigned char *blk = out + block_offset(N, o / OC, k / KC);
            const uint32_t off = tc::kmajor_offset(o % OC, k % KC, KC);
            for (int j = 0; j < S; ++j) {
                const int dig = (int)((u >> (49 - 7 * j)) & 127u);
                const __nv_bfloat16 b = __float2bfloat16_rn((float)(q < 0 ? -dig : dig));
                std::memcpy(blk + j * b_slice_bytes(N) + off, &b, 2);
            }
        }
    }
}

struct Ops {
    const unsigned char *D, *M;  // digit slices of D (rows l) and M (rows n)
    const int32_t *eD, *eM;      // their row exponents
};

// 2^n as a double, for n in the normal range (exact)
__device__ __forceinline__ double pow2(int n) { return __longlong_as_double((long long)(n + 1023) << 52); }

// 8 FP64 inputs -> their 8 digit slices (BF16, one 16-byte row chunk per slice) at
// element offset off of the K-major A-operand slices; scale = 2^(56 - e) (exact).
__device__ __forceinline__ void slice8(const double *x, double scale, unsigned char *As, uint32_t off) {
    long long q[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) q[i] = __double2ll_rn(x[i] * scale);
#pragma unroll
    for (int j = 0; j < S; ++j) {
        __align__(16) __nv_bfloat16 b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const unsigned long long u = (unsigned long long)(q[i] < 0 ? -q[i] : q[i]);
            const int dig = (int)((u >> (49 - 7 * j)) & 127u);
            b[i] = __int2bfloat16_rn(q[i] < 0 ? -dig : dig);
        }
        *reinterpret_cast<uint4 *>(As + j * a_slice_bytes() + off) = *reinterpret_cast<const uint4 *>(b);
    }
}

}  // namespace rtc

// Same arguments and results as k_mixed_residual (plus the operators' digit slices and
// the error word); grid (ceil(sumK / 64), R), 128 threads.
__global__ void __launch_bounds__(rtc::kThreads) k_mixed_residual_tc(
    const double *__restrict__ psi, double *__restrict__ phi, const double *__restrict__ sigma_s,
    const double *__restrict__ Qext, rtc::Ops ops, const double *__restrict__ sigma_t, const double *__restrict__ h,
    const double *__restrict__ mu, const int32_t *__restrict__ cell_inst, const int32_t *__restrict__ off,
    const int32_t *__restrict__ Kc, int B, unsigned long long *__restrict__ conv, float *__restrict__ dq, int N,
    int sumK, const double *__restrict__ Qang, const double *__restrict__ psi_inc, const int32_t *__restrict__ bc,
    float *__restrict__ q32, float *__restrict__ phi32, int *__restrict__ err) {
    using namespace rtc;
    extern __shared__ __align__(128) unsigned char smem_rt[];
    unsigned char *As = smem_rt;
    unsigned char *Bs = smem_rt + S * a_slice_bytes();
    uint64_t *bar_b = reinterpret_cast<uint64_t *>(Bs + b_block_bytes(N)), *bar_m = bar_b + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_m + 1);
    const int t = threadIdx.x;
    const int OC = oc_of(N);
    const uint32_t ncols_t = tmem_cols(N);
    if (t == 0) {
        tc::mbar_init(bar_b, 1);
        tc::mbar_init(bar_m, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (t < 32) {
        tc::tmem_alloc(tslot, ncols_t);
        tc::tmem_relinquish();
    }
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    tc::grid_dependency_wait();  // inputs of the previous kernel (programmatic dependent launch)

    const int r = blockIdx.y, g0 = blockIdx.x * 64;
    const int ncell = min(64, sumK - g0), ncols = 2 * ncell;
    const bool live = t < ncols;
    const int g = g0 + (live ? t >> 1 : 0), a = t & 1;
    const size_t colbase = ((size_t)r * sumK + g0) * 2;
    const size_t row = (colbase + (live ? t : 0)) * N;  // this thread's column
    const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
    uint32_t pb = 0, pm = 0;
    bool ok = true;

    // One exact contraction out[o] = sum_k op[o][k] in(k) of this thread's column, in
    // output chunks of OC; `in8(k0, x)` loads the FP64 inputs k0 .. k0 + 7 (16-byte
    // loads, all issued before use), `epi(o, value)` consumes each output. e_in: the
    // column's exponent.
    auto contract = [&](const unsigned char *opsl, const int32_t *eop, int e_in, auto in8, auto epi) {
        const uint32_t idesc = tc::idesc_bf16(128, OC);
        const double scale = pow2(56 - e_in), p_in = pow2(e_in - 14);
        for (int oc = 0; oc < N / OC && ok; ++oc) {
            for (int kc = 0; kc < N / KC; ++kc) {
                if (t == 0) {
                    tc::mbar_arrive_expect_tx(bar_b, b_block_bytes(N));
                    tc::bulk_copy_g2s(Bs, opsl + block_offset(N, oc, kc), b_block_bytes(N), bar_b);
                }
                {
                    double x[KC / 8][8];
#pragma unroll
                    for (int g8 = 0; g8 < KC / 8; ++g8) in8(kc * KC + g8 * 8, x[g8]);
#pragma unroll
                    for (int g8 = 0; g8 < KC / 8; ++g8) slice8(x[g8], scale, As, tc::kmajor_offset(t, g8 * 8, KC));
                }
                tc::fence_async_smem();  // the slices' st.shared must be visible to the tensor core
                tc::tc_fence_before();
                __syncthreads();
                if (t == 0) {
                    bool okb = tc::mbar_wait(bar_b, pb);
                    if (okb) {
                        tc::tc_fence_after();
                        const uint32_t as = tc::smem_u32(As), bs = tc::smem_u32(Bs);
                        for (int d = 0; d < S; ++d)
                            for (int i = 0; i <= d; ++i) {
                                const int j = d - i;
#pragma unroll
                                for (int ks = 0; ks < KC / 16; ++ks) {
                                    const uint64_t ad = tc::smem_desc(as + i * a_slice_bytes() + 256u * ks, 128, KC * 16);
                                    const uint64_t bd =
                                        tc::smem_desc(bs + j * b_slice_bytes(N) + 256u * ks, 128, KC * 16);
                                    tc::mma_bf16(tmem + (uint32_t)(d * OC), ad, bd, idesc,
                                                 (kc > 0 || i > 0 || ks > 0) ? 1u : 0u);
                                }
                            }
                    } else {
                        atomicExch(err, 1);
                        tc::mbar_wait(bar_b, pb);  // the copy must not land after the CTA has gone (bounded)
                    }
                    tc::mma_commit(bar_m);  // also when nothing was issued: the phase completes
                }
                pb ^= 1u;
                const bool okm = tc::mbar_wait(bar_m, pm);
                pm ^= 1u;
                tc::tc_fence_after();
                ok = __syncthreads_and(okm && *(volatile int *)err == 0) != 0;
                if (!ok) break;
            }
            if (!ok) break;
            // epilogue: value(o) = 2^(e_in + e_o - 14) sum_d 2^(-7 d) A_d(o), Horner from d = 7
            for (int o16 = 0; o16 < OC; o16 += 16) {
                double hsum[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) hsum[i] = 0.0;
                for (int d = S - 1; d >= 0; --d) {
                    float v[16];
                    tc::tmem_ld16(tmem + lane_base + (uint32_t)(d * OC + o16), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) hsum[i] = fma(hsum[i], 0.0078125, (double)v[i]);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int o = oc * OC + o16 + i;
                    epi(o, hsum[i] * p_in * pow2(eop[o]));
                }
            }
            tc::tc_fence_before();  // the accumulator reads precede the next chunk's MMAs
            __syncthreads();
        }
    };
    auto row_exponent = [&](auto in8) {
        double mx = 0.0;
        for (int k0 = 0; k0 < N; k0 += 32) {
            double x[4][8];
#pragma unroll
            for (int j = 0; j < 4; ++j) in8(k0 + 8 * j, x[j]);
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 8; ++i) mx = fmax(mx, fabs(x[j][i]));
        }
        int e = 0;
        if (mx > 0.0) frexp(mx, &e);
        return e;
    };
    auto ld8 = [&](const double *p, double *x, bool coherent) {  // 8 doubles, 16-byte aligned
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double2 v = coherent ? __ldcg(reinterpret_cast<const double2 *>(p) + i)
                                       : __ldg(reinterpret_cast<const double2 *>(p) + i);
            x[2 * i] = v.x;
            x[2 * i + 1] = v.y;
        }
    };

    // phi = D psi (FP64 output), convergence maxima of phi_0
    const double *ps = psi + row;
    auto in_psi = [&](int k0, double *x) {
        if (live) ld8(ps + k0, x, false);
        else
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = 0.0;
    };
    const int e_psi = row_exponent(in_psi);
    const int slot = (r * B + cell_inst[g]) * 2;
    contract(ops.D, ops.eD, e_psi, in_psi, [&](int l, double pn) {
        if (!live) return;
        const size_t e = row + l;
        if (l == 0) {
            atomicMax(conv + slot, dkey(pn - phi[e]));
            atomicMax(conv + slot + 1, dkey(pn));
        }
        phi[e] = pn;
    });
    // s = M x, x = Sigma phi + Q (FP64 per element, as written above by this thread)
    const double *sg = sigma_s + (size_t)g * N;
    auto in_x = [&](int k0, double *x) {  // phi as written by this thread above: read through L2
        if (!live) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = 0.0;
            return;
        }
        double sv[8], pv[8], qv[8];
        ld8(sg + k0, sv, false);
        ld8(phi + row + k0, pv, true);
        if (Qext) ld8(Qext + row + k0, qv, false);
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = sv[i] * pv[i] + (Qext ? qv[i] : 0.0);
    };
    const int e_x = row_exponent(in_x);
    // the LD residual of this column's node, given both nodes' scattering source s
    const int b = cell_inst[g], loc = g - off[b];
    const double hh = h[g], st = sigma_t[g], w = 2.0 / hh;
    const double *psr = psi + (size_t)r * sumK * 2 * N;
    contract(ops.M, ops.eM, e_x, in_x, [&](int n, double s_own) {
        if (Qang && live) s_own += Qang[row + n];
        const double s_other = __shfl_xor_sync(0xffffffffu, s_own, 1);
        if (!live) return;
        const double sL = a ? s_other : s_own, sR = a ? s_own : s_other;
        const double m = mu[n];
        const double pL = psr[((size_t)2 * g) * N + n], pR = psr[((size_t)2 * g + 1) * N + n];
        double tL, tR;
        if (m > 0.0) {
            double pin;
            if (loc > 0) pin = psr[((size_t)2 * (g - 1) + 1) * N + n];
            else if (bc && bc[2 * b] == kBcReflect) pin = psr[((size_t)2 * g) * N + (N - 1 - n)];
            else pin = psi_inc ? psi_inc[(((size_t)r * B + b) * 2) * N + n] : 0.0;
            tL = 0.5 * m * (pL + pR) - m * pin;
            tR = 0.5 * m * (pR - pL);
        } else {
            double pin;
            if (loc < Kc[b] - 1) pin = psr[((size_t)2 * (g + 1)) * N + n];
            else if (bc && bc[2 * b + 1] == kBcReflect) pin = psr[((size_t)2 * g + 1) * N + (N - 1 - n)];
            else pin = psi_inc ? psi_inc[(((size_t)r * B + b) * 2 + 1) * N + n] : 0.0;
            tL = 0.5 * m * (pR - pL);
            tR = -0.5 * m * (pL + pR) + m * pin;
        }
        const float v = a ? (float)(sR - st * pR - w * (2.0 * tR - tL)) : (float)(sL - st * pL - w * (2.0 * tL - tR));
        const size_t e = row + n;
        dq[e] = v;
        if (q32) q32[e] = v;
        if (phi32) phi32[e] = 0.f;
    });
    if (!ok && t == 0) atomicExch(err, 1);
    tc::tc_fence_before();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tmem, ncols_t);
}

}  // namespace fpsa
