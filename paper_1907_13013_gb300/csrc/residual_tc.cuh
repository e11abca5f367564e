// The FP64 refinement residual of the mixed-precision path with its two angular
// contractions on the tensor cores, exact to FP64 working accuracy.
//
// k_mixed_residual computes, per column (cell, node, rhs) of the FP64 iterate psi,
//   phi = D psi,   x = Sigma phi + Q,   s = M x (Eqs. phi-mom, treq),
// then the LD transport residual of that column. GB300's FP64 rate (about 1.2 TFLOP/s)
// makes the two N x N contractions the whole cost of the kernel. Here each contraction
// is an exact integer computation on the BF16 tensor cores:
//   - every row r of the input (a column's N values) is scaled by its own power of two,
//     x~ = x 2^-e_r with |x~| < 1 (e_r the frexp exponent of max |x|), and written as the
//     56-bit fixed-point integer q = x~ 2^56 rounded to nearest (taken from the bits of x
//     with integer operations), split into balanced base-128 digits:
//     q = sum_{i < 8} s_i 2^(49 - 7 i) with s_0 in [-128, 128] and s_i in [-64, 63] for
//     i >= 1 (each exact in BF16), i.e. x~ = sum_i s_i 2^(-7 (i + 1));
//   - every row o of the operator likewise (host side, once per context): t_j, e_o;
//   - x~ . op~ = sum_d 2^(-7 (d + 2)) A_d with A_d = sum_{i + j = d} sum_k s_i t_j over
//     the 36 digit pairs with i + j <= 7 (the dropped pairs weigh 2^-70 or less).
// A product s_i t_j is an integer of magnitude at most 2^14 (i = j = 0), 2^13 (one
// index 0) or 2^12; the pairs of a diagonal d contribute at most (d + 3) 2^12 per k
// (2^14 for d <= 1), so over K <= 256 terms the sum of the magnitudes of a diagonal's
// products, and hence every partial sum in any order, is an integer of magnitude at
// most 10 x 2^20 < 2^24: the FP32 accumulation of the BF16 products in tensor memory
// is exact (A_d in its own accumulator, 8 x OC TMEM columns). The A_d are then
// combined in FP64, scaled by 2^(e_r + e_o): the only roundings are the 56-bit
// truncation of each row relative to its largest entry and the FP64 combination, i.e.
// the accuracy of an FP64 dot product.
//
// One CTA per tile of 64 cells x 2 nodes = 128 columns (tensor-memory lane = column)
// and per SM (it holds all 512 TMEM columns), 256 threads: two per column, each taking
// half of every K-chunk and of every output chunk. For each output chunk of OC = 64
// rows (32 where 64 does not divide N) and each K-chunk of 32, in two pipelined stages:
// thread 0 copies the operator's 8 digit slices of that block (OC x 32 BF16 each,
// stored K-major in the core-matrix layout, one bulk copy), the threads write the 8
// digit slices of their columns' 32 inputs (K-major), and thread 0 issues the 72 MMAs
// (36 pairs, two K-steps; M = 128, N = OC, K = 16) while the next chunk is prepared.
// Waits are bounded; on a timeout the CTA records the error, waits (bounded) for its
// copies and products, frees its tensor memory and stops.
#pragma once

#include "kernels.cuh"
#include "tc_contract.cuh"

namespace fpsa {
namespace rtc {

constexpr int S = 8;    // digit slices: 56-bit fixed point per row
constexpr int KC = 32;  // K per chunk: two MMA K-steps
constexpr int kThreads = 256;  // two threads per column (tensor-memory lane), halves of K and of the outputs
// output rows per chunk: 64 where they divide N, else 32 (N is a multiple of 32)
__host__ __device__ constexpr int oc_of(int N) { return N % 64 == 0 ? 64 : 32; }
__host__ __device__ constexpr uint32_t a_slice_bytes() { return 128u * KC * 2u; }
__host__ __device__ constexpr uint32_t b_slice_bytes(int N) { return (uint32_t)oc_of(N) * KC * 2u; }
__host__ __device__ constexpr uint32_t b_block_bytes(int N) { return S * b_slice_bytes(N); }
// two stages of (A slices, B block), then 4 mbarriers, the tensor-memory slot and the
// row-maximum exchange; at least 120 KB, so that one CTA per SM is resident: a second
// one would only wait in tcgen05.alloc for the first one's tensor memory (all 512
// columns), which measured a hundred times slower
__host__ __device__ constexpr uint32_t stage_bytes(int N) { return S * a_slice_bytes() + b_block_bytes(N); }
__host__ __device__ constexpr uint32_t smem_bytes(int N) {
    return 2 * stage_bytes(N) + 64u + 256u * 8u < 120u * 1024u ? 120u * 1024u : 2 * stage_bytes(N) + 64u + 256u * 8u;
}
__host__ __device__ constexpr uint32_t tmem_cols(int N) { return (uint32_t)(S * oc_of(N)) <= 256u ? 256u : 512u; }
__host__ __device__ constexpr bool applies(int N) { return N % KC == 0 && N >= KC && N <= 256; }
// byte offset of operator block (oc, kc) in the stored digit slices
__host__ __device__ constexpr size_t block_offset(int N, int oc, int kc) {
    return ((size_t)oc * (N / KC) + kc) * b_block_bytes(N);
}

// Balanced base-128 digits of q (|q| <= 2^56): q = sum_{j < 8} s[j] 2^(49 - 7 j) with
// s[0] in [-128, 128] and s[j] in [-64, 63] for j >= 1. With the bias
// b = 64 sum_{j >= 1} 2^(49 - 7 j) (< 2^49), q + b = s[0] 2^49 + sum_{j >= 1} (s[j] + 64)
// 2^(49 - 7 j) with every s[j] + 64 in [0, 127]: the plain base-128 digits of the low 49
// bits of q + b, less 64, and its arithmetic shift by 49.
__host__ __device__ __forceinline__ void balanced_digits(long long q, int *sd) {
    constexpr long long bias =
        64LL * ((1LL << 42) + (1LL << 35) + (1LL << 28) + (1LL << 21) + (1LL << 14) + (1LL << 7) + 1LL);
    const long long r = q + bias;
    sd[0] = (int)(r >> 49);
#pragma unroll
    for (int j = 1; j < S; ++j) sd[j] = (int)((r >> (49 - 7 * j)) & 127) - 64;
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
            int sd[S];
            balanced_digits(q, sd);
            unsigned char *blk = out + block_offset(N, o / OC, k / KC);
            const uint32_t off = tc::kmajor_offset(o % OC, k % KC, KC);
            for (int j = 0; j < S; ++j) {
                const __nv_bfloat16 b = __float2bfloat16_rn((float)sd[j]);
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

// x 2^(56 - e) rounded to an integer (|x| < 2^e), from the bits of x with integer
// operations only (the FP64 pipe is the resource this kernel avoids); zeros and
// subnormals (below 2^-1022) give 0.
__device__ __forceinline__ long long fixed56(double x, int e) {
    const long long bits = __double_as_longlong(x);
    const int E = (int)((bits >> 52) & 0x7FF);
    if (E == 0) return 0;
    const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = E - 1019 - e;  // x 2^(56 - e) = mant 2^sh, sh <= 3
    long long q = 0;
    if (sh >= 0) q = mant << sh;
    else if (sh > -54) q = (mant + (1LL << (-sh - 1))) >> -sh;
    return bits < 0 ? -q : q;
}

// 8 FP64 inputs -> their 8 digit slices (BF16, one 16-byte row chunk per slice) at
// element offset off of the K-major A-operand slices; e: the row's exponent.
__device__ __forceinline__ void slice8(const double *x, int e, unsigned char *As, uint32_t off) {
    int sd[8][S];
#pragma unroll
    for (int i = 0; i < 8; ++i) balanced_digits(fixed56(x[i], e), sd[i]);
#pragma unroll
    for (int j = 0; j < S; ++j) {
        __align__(16) __nv_bfloat16 b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) b[i] = __int2bfloat16_rn(sd[i][j]);
        *reinterpret_cast<uint4 *>(As + j * a_slice_bytes() + off) = *reinterpret_cast<const uint4 *>(b);
    }
}

}  // namespace rtc

// Same arguments and results as k_mixed_residual (plus the operators' digit slices and
// the error word); grid (ceil(sumK / 64), R), 256 threads: thread t and t + 128 share
// column t % 128 (its tensor-memory lane), each slicing half of every K-chunk and
// finishing half of every output chunk. The K-chunks of a contraction are pipelined
// through two stages: the MMAs of one chunk run while the next chunk is sliced and its
// operator block copied.
__global__ void __launch_bounds__(rtc::kThreads, 1) k_mixed_residual_tc(
    const double *__restrict__ psi, double *__restrict__ phi, const double *__restrict__ sigma_s,
    const double *__restrict__ Qext, rtc::Ops ops, const double *__restrict__ sigma_t, const double *__restrict__ h,
    const double *__restrict__ mu, const int32_t *__restrict__ cell_inst, const int32_t *__restrict__ off,
    const int32_t *__restrict__ Kc, int B, unsigned long long *__restrict__ conv, float *__restrict__ dq, int N,
    int sumK, const double *__restrict__ Qang, const double *__restrict__ psi_inc, const int32_t *__restrict__ bc,
    float *__restrict__ q32, float *__restrict__ phi32, int *__restrict__ err) {
    using namespace rtc;
    extern __shared__ __align__(128) unsigned char smem_rt[];
    const uint32_t SB = stage_bytes(N);
    unsigned char *stg[2] = {smem_rt, smem_rt + SB};  // A slices, then the B block
    uint64_t *bar_b = reinterpret_cast<uint64_t *>(smem_rt + 2 * SB), *bar_m = bar_b + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_m + 2);
    unsigned long long *s_max = reinterpret_cast<unsigned long long *>(smem_rt + 2 * SB + 64);
    const int t = threadIdx.x, tr = t & 127, half = t >> 7;
    const int OC = oc_of(N), nkc = N / KC, nit = (N / OC) * nkc;
    const uint32_t ncols_t = tmem_cols(N);
    if (t == 0) {
        for (int i = 0; i < 4; ++i) tc::mbar_init(bar_b + i, 1);
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
    const bool live = tr < ncols;
    const int g = g0 + (live ? tr >> 1 : 0), a = tr & 1;
    const size_t colbase = ((size_t)r * sumK + g0) * 2;
    const size_t row = (colbase + (live ? tr : 0)) * N;  // this thread's column
    const uint32_t lane_base = (uint32_t)((t & 127) & ~31) << 16;
    uint32_t fb[2] = {0u, 0u}, cm[2] = {0u, 0u};  // completed copy phases / MMA commits per stage
    bool ok = true;

    auto ld8 = [&](const double *p, double *x, bool coherent) {  // 8 doubles, 16-byte aligned
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double2 v = coherent ? __ldcg(reinterpret_cast<const double2 *>(p) + i)
                                       : __ldg(reinterpret_cast<const double2 *>(p) + i);
            x[2 * i] = v.x;
            x[2 * i + 1] = v.y;
        }
    };
    // frexp exponent of the row's largest magnitude: each half scans its half of the row
    // (integer compares of the magnitude bits, which order non-negative doubles) and the
    // two meet in shared memory; 0 for a row of zeros
    auto row_exponent = [&](auto in8) {
        unsigned long long mx = 0;
        for (int k0 = half * (N / 2); k0 < (half + 1) * (N / 2); k0 += 16) {
            double x[2][8];
            in8(k0, x[0]);
            in8(k0 + 8, x[1]);
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const unsigned long long u =
                        (unsigned long long)__double_as_longlong(x[j][i]) & 0x7FFFFFFFFFFFFFFFull;
                    mx = u > mx ? u : mx;
                }
        }
        s_max[t] = mx;
        __syncthreads();
        const unsigned long long m2 = s_max[t ^ 128];
        mx = m2 > mx ? m2 : mx;
        __syncthreads();  // s_max is reused by the next call
        const int E = (int)(mx >> 52);
        return E ? E - 1022 : 0;
    };

    // One exact contraction out[o] = sum_k op[o][k] in(k) of this thread's column, in
    // output chunks of OC; `in8(k0, x)` loads the FP64 inputs k0 .. k0 + 7 (16-byte
    // loads), `epi16(o0, v)` consumes outputs o0 .. o0 + 15 (every thread calls it for
    // its half of each output chunk). e_in: the column's exponent.
    auto contract = [&](const unsigned char *opsl, const int32_t *eop, int e_in, auto in8, auto epi16) {
        const uint32_t idesc = tc::idesc_bf16(128, OC);
        const double p_in = pow2(e_in - 14);
        auto issue_copy = [&](int it, int b) {
            if (t == 0) {
                tc::mbar_arrive_expect_tx(&bar_b[b], b_block_bytes(N));
                tc::bulk_copy_g2s(stg[b] + S * a_slice_bytes(), opsl + block_offset(N, it / nkc, it % nkc),
                                  b_block_bytes(N), &bar_b[b]);
            }
        };
        auto slice_chunk = [&](int it, int b) {  // this thread's 16 inputs of the chunk
            const int k0 = (it % nkc) * KC + half * 16;
            double x[2][8];
            if (live) {
                in8(k0, x[0]);
                in8(k0 + 8, x[1]);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) x[0][i] = x[1][i] = 0.0;
            }
            slice8(x[0], e_in, stg[b], tc::kmajor_offset(tr, half * 16, KC));
            slice8(x[1], e_in, stg[b], tc::kmajor_offset(tr, half * 16 + 8, KC));
            tc::fence_async_smem();  // the slices' st.shared must be visible to the tensor core
        };
        auto wait_mma = [&](int b) {  // the last commit on stage b has completed (bounded)
            return cm[b] == 0 || tc::mbar_wait(&bar_m[b], (cm[b] - 1u) & 1u);
        };
        issue_copy(0, 0);
        slice_chunk(0, 0);
        tc::tc_fence_before();
        __syncthreads();
        for (int it = 0; it < nit; ++it) {
            const int b = it & 1, kc = it % nkc, oc = it / nkc;
            if (t == 0) {
                bool okb = tc::mbar_wait(&bar_b[b], fb[b]);
                if (okb) {
                    tc::tc_fence_after();
                    const uint32_t as = tc::smem_u32(stg[b]), bs = as + S * a_slice_bytes();
                    for (int d = 0; d < S; ++d)
                        for (int i = 0; i <= d; ++i) {
                            const int j = d - i;
#pragma unroll
                            for (int ks = 0; ks < KC / 16; ++ks) {
                                const uint64_t ad = tc::smem_desc(as + i * a_slice_bytes() + 256u * ks, 128, KC * 16);
                                const uint64_t bd = tc::smem_desc(bs + j * b_slice_bytes(N) + 256u * ks, 128, KC * 16);
                                tc::mma_bf16(tmem + (uint32_t)(d * OC), ad, bd, idesc,
                                             (kc > 0 || i > 0 || ks > 0) ? 1u : 0u);
                            }
                        }
                } else {
                    atomicExch(err, 1);
                    tc::mbar_wait(&bar_b[b], fb[b]);  // the copy must not land after the CTA has gone (bounded)
                }
                tc::mma_commit(&bar_m[b]);  // also when nothing was issued: the phase completes
            }
            fb[b] ^= 1u;
            ++cm[b];
            if (it + 1 < nit) {
                const int nb = b ^ 1;
                ok = wait_mma(nb) && ok;  // stage nb's previous MMAs (iteration it - 1) have read it
                issue_copy(it + 1, nb);
                slice_chunk(it + 1, nb);
                tc::tc_fence_before();
                ok = __syncthreads_and(ok && *(volatile int *)err == 0) != 0;
                if (!ok) break;
            }
            if (kc == nkc - 1) {
                // epilogue of output chunk oc: value(o) = 2^(e_in + e_o - 14) sum_d 2^(-7 d) A_d(o).
                // The A_d are exact integers (|A_d| <= 2^24): hi = sum_{d < 4} A_d 2^(7 (3 - d))
                // and lo = sum_{d >= 4} A_d 2^(7 (7 - d)) are exact 64-bit integers (below 2^46),
                // so sum_d 2^(-7 d) A_d = hi 2^-21 + lo 2^-49 with one FP64 rounding
                ok = wait_mma(b) && ok;
                tc::tc_fence_after();
                for (int o16 = half * (OC / 2); o16 < (half + 1) * (OC / 2); o16 += 16) {
                    long long hi[16], lo[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) hi[i] = lo[i] = 0;
                    for (int d = 0; d < S; ++d) {
                        float v[16];
                        tc::tmem_ld16(tmem + lane_base + (uint32_t)(d * OC + o16), v);
                        const int sh = 7 * ((d < 4 ? 3 : 7) - d);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const long long q = (long long)__float2int_rn(v[i]) << sh;
                            if (d < 4) hi[i] += q;
                            else lo[i] += q;
                        }
                    }
                    double val[16];
                    const int o0 = oc * OC + o16;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        val[i] = fma((double)hi[i], 4.76837158203125e-07, (double)lo[i] * 1.7763568394002505e-15) *
                                 p_in * pow2(eop[o0 + i]);
                    epi16(o0, val);
                }
                tc::tc_fence_before();  // the accumulator reads precede the next chunk's MMAs
                ok = __syncthreads_and(ok && *(volatile int *)err == 0) != 0;
                if (!ok) break;
            }
        }
        if (!ok && t == 0) {  // nothing may land after the CTA has gone (bounded)
            for (int b = 0; b < 2; ++b) wait_mma(b);
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
    contract(ops.D, ops.eD, e_psi, in_psi, [&](int l0, const double *pn) {
        if (!live) return;
        double *dst = phi + row + l0;
        if (l0 == 0) {
            atomicMax(conv + slot, dkey(pn[0] - dst[0]));
            atomicMax(conv + slot + 1, dkey(pn[0]));
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) reinterpret_cast<double2 *>(dst)[i] = make_double2(pn[2 * i], pn[2 * i + 1]);
    });
    __syncthreads();  // the phi halves written by both threads of a column are read below
    // s = M x, x = Sigma phi + Q (FP64 per element; phi read through L2)
    const double *sg = sigma_s + (size_t)g * N;
    auto in_x = [&](int k0, double *x) {
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
    const int e_x = ok ? row_exponent(in_x) : 0;
    // the LD residual of this column's node for 16 ordinates, given both nodes' scattering
    // source s (the partner node is the adjacent lane); the 16 ordinates share the sign of mu
    // (N / 2 is a multiple of 16)
    const int b = cell_inst[g], loc = g - off[b];
    const double hh = h[g], st = sigma_t[g], w = 2.0 / hh;
    const double *psr = psi + (size_t)r * sumK * 2 * N;
    if (ok) contract(ops.M, ops.eM, e_x, in_x, [&](int n0, const double *s) {
        double sown[16], sL[16], sR[16];
        if (Qang && live) {
            double qa[16];
            ld8(Qang + row + n0, qa, false);
            ld8(Qang + row + n0 + 8, qa + 8, false);
#pragma unroll
            for (int i = 0; i < 16; ++i) sown[i] = s[i] + qa[i];
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) sown[i] = s[i];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const double so = __shfl_xor_sync(0xffffffffu, sown[i], 1);
            sL[i] = a ? so : sown[i];
            sR[i] = a ? sown[i] : so;
        }
        if (!live) return;
        double m[16], pL[16], pR[16], pin[16];
        ld8(mu + n0, m, false);
        ld8(mu + n0 + 8, m + 8, false);
        ld8(psr + ((size_t)2 * g) * N + n0, pL, false);
        ld8(psr + ((size_t)2 * g) * N + n0 + 8, pL + 8, false);
        ld8(psr + ((size_t)2 * g + 1) * N + n0, pR, false);
        ld8(psr + ((size_t)2 * g + 1) * N + n0 + 8, pR + 8, false);
        const bool pos = n0 >= N / 2;  // mu_n > 0 for n >= N / 2 (ascending, symmetric)
        if (pos ? loc > 0 : loc < Kc[b] - 1) {  // the upwind neighbour's outflow node
            const double *src = psr + (pos ? ((size_t)2 * (g - 1) + 1) : ((size_t)2 * (g + 1))) * N + n0;
            ld8(src, pin, false);
            ld8(src + 8, pin + 8, false);
        } else if (bc && bc[2 * b + (pos ? 0 : 1)] == kBcReflect) {  // the mirror ordinate's outflow
            const double *node = psr + ((size_t)2 * g + (pos ? 0 : 1)) * N;
#pragma unroll
            for (int i = 0; i < 16; ++i) pin[i] = node[N - 1 - (n0 + i)];
        } else if (psi_inc) {
            const double *src = psi_inc + (((size_t)r * B + b) * 2 + (pos ? 0 : 1)) * N + n0;
            ld8(src, pin, false);
            ld8(src + 8, pin + 8, false);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) pin[i] = 0.0;
        }
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            double tL, tR;
            if (pos) {
                tL = 0.5 * m[i] * (pL[i] + pR[i]) - m[i] * pin[i];
                tR = 0.5 * m[i] * (pR[i] - pL[i]);
            } else {
                tL = 0.5 * m[i] * (pR[i] - pL[i]);
                tR = -0.5 * m[i] * (pL[i] + pR[i]) + m[i] * pin[i];
            }
            v[i] = a ? (float)(sR[i] - st * pR[i] - w * (2.0 * tR - tL))
                     : (float)(sL[i] - st * pL[i] - w * (2.0 * tL - tR));
        }
        float4 *dd = reinterpret_cast<float4 *>(dq + row + n0);
#pragma unroll
        for (int i = 0; i < 4; ++i) dd[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        if (q32) {
            float4 *dq2 = reinterpret_cast<float4 *>(q32 + row + n0);
#pragma unroll
            for (int i = 0; i < 4; ++i) dq2[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
        if (phi32) {
            float4 *dp = reinterpret_cast<float4 *>(phi32 + row + n0);
#pragma unroll
            for (int i = 0; i < 4; ++i) dp[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    });
    if (!ok && t == 0) atomicExch(err, 1);
    tc::tc_fence_before();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tmem, ncols_t);
}

}  // namespace fpsa
