// Kernels of the FPSA-preconditioned GMRES(m) solver (Sec. 4 compares GMRES with
// and without the FP preconditioner; FPSA source iteration is the Richardson
// iteration with the same preconditioner).
//
// Unknowns: the flux moments, [R][sumK][2][N] like phi. The operator is
//   A' u = (I - T)(I + C) u,  T v = D L^{-1} M Sigma v,  C v = D F^{-1} (m (x) M Sigma v),
// solved from u = 0 for b = D L^{-1} (M Q + q_ang); phi = (I + C) u. Every
// (right-hand side, instance) pair is its own linear system, so inner products are
// segmented: system s = r * B + b owns the contiguous range of cells of instance b
// in right-hand side r. Reductions are two-pass (per-chunk partial sums, then a
// fixed-order sum) so results are bitwise reproducible.
#pragma once

#include "kernels.cuh"

namespace fpsa {

// rhs = m (x) M (Sigma v) per cell (the FP right-hand side of C v, Eq. correct).
template <typename T>
__global__ void k_fp_rhs_moments(const T *__restrict__ v, const T *__restrict__ sigma_s,
                                 const double *__restrict__ h, const T *__restrict__ MT, T *__restrict__ rhs, int N,
                                 int sumK) {
    extern __shared__ unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);
    T *Ys = Xs + 2 * kContractCells * N;
    const int r = blockIdx.y;
    const int g0 = blockIdx.x * kContractCells;
    const int ncell = min(kContractCells, sumK - g0);
    const int ncols = 2 * ncell;
    const size_t colbase = ((size_t)r * sumK + g0) * 2;
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) {
        const int c = idx / N, l = idx - c * N;
        Xs[idx] = sigma_s[(size_t)(g0 + c / 2) * N + l] * v[colbase * N + idx];
    }
    __syncthreads();
    block_contract(Xs, N, MT, N, ncols, Ys, N);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncell * N; idx += blockDim.x) {
        const int cl = idx / N, n = idx - cl * N;
        const T w = (T)(h[g0 + cl] / 6.0);
        const T r0 = Ys[(2 * cl) * N + n], r1 = Ys[(2 * cl + 1) * N + n];
        rhs[(colbase + 2 * cl) * N + n] = w * (T(2) * r0 + r1);
        rhs[(colbase + 2 * cl + 1) * N + n] = w * (r0 + T(2) * r1);
    }
}

// out = base + sign * D psi (moments of a sweep; base may be NULL).
template <typename T>
__global__ void k_moments_axpy(const T *__restrict__ psi, const T *__restrict__ base, T sign,
                               const T *__restrict__ DT, T *__restrict__ out, int N, int sumK) {
    extern __shared__ unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);
    T *Ys = Xs + 2 * kContractCells * N;
    const int r = blockIdx.y;
    const int g0 = blockIdx.x * kContractCells;
    const int ncols = 2 * min(kContractCells, sumK - g0);
    const size_t colbase = ((size_t)r * sumK + g0) * 2;
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) Xs[idx] = psi[colbase * N + idx];
    __syncthreads();
    block_contract(Xs, N, DT, N, ncols, Ys, N);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) {
        const size_t e = colbase * N + idx;
        out[e] = (base ? base[e] : T(0)) + sign * Ys[idx];
    }
}

// Segmented multi-dot, pass 1: for system s and vectors V_0..V_{nv-1} (stride vstride),
// partial[s][chunk][i] = sum over the chunk of the segment of V_i * w.
// Grid: (chunks, nsys), kDotThreads threads; segments [seg_begin[s], seg_end[s]), whole
// 16-byte words (every segment starts and ends on a multiple of 2N elements). A thread
// keeps its kDotChunk / kDotThreads elements of w in registers (16-byte loads,
// interleaved across the block so every load instruction is coalesced) and streams
// the vectors four at a time, so each V_i is read once with all of a thread's loads in
// flight together. FP64 vectors accumulate in FP64; FP32 vectors (the inner solves of
// GMRES-IR) in FP32 over a thread's 32 products, then in FP64 across threads and
// chunks (the FP64 rate of this GPU is far below what one FMA per loaded element
// needs). The sum order is fixed, so results are bitwise reproducible.
constexpr int kDotChunk = 8192;
constexpr int kDotThreads = 256;
template <typename T>
__global__ void __launch_bounds__(kDotThreads) k_seg_dots(const T *__restrict__ V, size_t vstride, int nv,
                                                          const T *__restrict__ w,
                                                          const long long *__restrict__ seg_begin,
                                                          const long long *__restrict__ seg_end, int nchunks,
                                                          double *__restrict__ partial) {
    using VT = typename VecOf<T>::type;
    constexpr int VW = VecOf<T>::V, NW = kDotChunk / VW / kDotThreads;
    __shared__ double red[4][kDotThreads / 32];
    const int s = blockIdx.y, ch = blockIdx.x, t = threadIdx.x;
    const long long b0 = seg_begin[s] + (long long)ch * kDotChunk;
    const long long b1 = min(seg_end[s], b0 + kDotChunk);
    const int nwords = b1 > b0 ? (int)((b1 - b0) / VW) : 0;
    const long long wb = b0 / VW;
    VT wv[NW];
#pragma unroll
    for (int u = 0; u < NW; ++u) {
        const int idx = t + kDotThreads * u;
        if (idx < nwords) wv[u] = __ldg(reinterpret_cast<const VT *>(w) + wb + idx);
    }
    for (int i0 = 0; i0 < nv; i0 += 4) {
        double acc[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            T a = T(0);
            if (i0 + g < nv) {
                const VT *vp = reinterpret_cast<const VT *>(V + (size_t)(i0 + g) * vstride) + wb;
#pragma unroll
                for (int u = 0; u < NW; ++u) {
                    const int idx = t + kDotThreads * u;
                    if (idx < nwords) {
                        const VT x = __ldg(vp + idx);
                        if constexpr (VW == 4) {
                            a = fma(x.x, wv[u].x, a); a = fma(x.y, wv[u].y, a);
                            a = fma(x.z, wv[u].z, a); a = fma(x.w, wv[u].w, a);
                        } else {
                            a = fma(x.x, wv[u].x, a); a = fma(x.y, wv[u].y, a);
                        }
                    }
                }
            }
            acc[g] = (double)a;
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            for (int o = 16; o > 0; o >>= 1) acc[g] += __shfl_xor_sync(0xffffffffu, acc[g], o);
            if ((t & 31) == 0) red[g][t >> 5] = acc[g];
        }
        __syncthreads();
        if (t < 4 && i0 + t < nv) {
            double sum = 0.0;
            for (int k = 0; k < kDotThreads / 32; ++k) sum += red[t][k];
            partial[((size_t)s * nchunks + ch) * nv + i0 + t] = sum;
        }
        __syncthreads();
    }
}

// Pass 2: out[s][i] = sum over chunks in order.
static __global__ void k_seg_dots_finish(const double *__restrict__ partial, int nsys, int nchunks, int nv,
                                         double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nsys * nv) return;
    const int s = t / nv, i = t - s * nv;
    double acc = 0.0;
    for (int c = 0; c < nchunks; ++c) acc += partial[((size_t)s * nchunks + c) * nv + i];
    out[(size_t)s * nv + i] = acc;
}

// y = alpha_s x + sum_i coef[s][i] V_i on the segment of system s (coef stride nv;
// alpha NULL: no x term; x may alias y). Grid and chunks as k_seg_dots; each thread
// holds its 32 elements and streams the vectors. FP32 vectors combine in FP32.
template <typename T>
__global__ void __launch_bounds__(kDotThreads) k_seg_combine(T *y, const double *__restrict__ alpha, const T *x,
                                                             const T *__restrict__ V, size_t vstride, int nv,
                                                             const double *__restrict__ coef,
                                                             const long long *__restrict__ seg_begin,
                                                             const long long *__restrict__ seg_end) {
    using VT = typename VecOf<T>::type;
    constexpr int VW = VecOf<T>::V, NW = kDotChunk / VW / kDotThreads;
    const int s = blockIdx.y, ch = blockIdx.x, t = threadIdx.x;
    const long long b0 = seg_begin[s] + (long long)ch * kDotChunk;
    const long long b1 = min(seg_end[s], b0 + kDotChunk);
    const int nwords = b1 > b0 ? (int)((b1 - b0) / VW) : 0;
    const long long wb = b0 / VW;
    VT acc[NW];
    const T al = alpha ? (T)alpha[s] : T(0);
#pragma unroll
    for (int u = 0; u < NW; ++u) {
        const int idx = t + kDotThreads * u;
        VT a;
        if constexpr (VW == 4) a = make_float4(0.f, 0.f, 0.f, 0.f);
        else a = make_double2(0.0, 0.0);
        if (alpha && idx < nwords) {
            const VT xv = reinterpret_cast<const VT *>(x)[wb + idx];
            if constexpr (VW == 4) a = make_float4(al * xv.x, al * xv.y, al * xv.z, al * xv.w);
            else a = make_double2(al * xv.x, al * xv.y);
        }
        acc[u] = a;
    }
    for (int i = 0; i < nv; ++i) {
        const T c = (T)coef[(size_t)s * nv + i];
        const VT *vp = reinterpret_cast<const VT *>(V + (size_t)i * vstride) + wb;
#pragma unroll
        for (int u = 0; u < NW; ++u) {
            const int idx = t + kDotThreads * u;
            if (idx < nwords) {
                const VT v = __ldg(vp + idx);
                if constexpr (VW == 4) {
                    acc[u].x = fma(c, v.x, acc[u].x); acc[u].y = fma(c, v.y, acc[u].y);
                    acc[u].z = fma(c, v.z, acc[u].z); acc[u].w = fma(c, v.w, acc[u].w);
                } else {
                    acc[u].x = fma(c, v.x, acc[u].x); acc[u].y = fma(c, v.y, acc[u].y);
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NW; ++u) {
        const int idx = t + kDotThreads * u;
        if (idx < nwords) reinterpret_cast<VT *>(y)[wb + idx] = acc[u];
    }
}

}  // namespace fpsa
