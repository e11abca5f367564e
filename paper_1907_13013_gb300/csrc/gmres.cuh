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
// partial[s][chunk][i] = sum over the chunk of the segment of V_i * w (FP64).
// Grid: (chunks, nsys); segments [seg_begin[s], seg_end[s]).
constexpr int kDotChunk = 8192;
template <typename T>
__global__ void k_seg_dots(const T *__restrict__ V, size_t vstride, int nv, const T *__restrict__ w,
                           const long long *__restrict__ seg_begin, const long long *__restrict__ seg_end,
                           int nchunks, double *__restrict__ partial) {
    __shared__ double red[32];
    const int s = blockIdx.y, ch = blockIdx.x;
    const long long b0 = seg_begin[s] + (long long)ch * kDotChunk;
    const long long b1 = min(seg_end[s], b0 + kDotChunk);
    for (int i = 0; i < nv; ++i) {
        double acc = 0.0;
        for (long long e = b0 + threadIdx.x; e < b1; e += blockDim.x)
            acc += (double)V[(size_t)i * vstride + e] * (double)w[e];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
            partial[((size_t)s * nchunks + ch) * nv + i] = t;
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

// y[e] = alpha_s * y[e] + sum_i coef[s][i] * V_i[e] (coef stride nv; alpha NULL: no y term),
// where s = col_sys[e / N] is the system of the column holding element e.
template <typename T>
__global__ void k_seg_combine(T *__restrict__ y, const double *__restrict__ alpha, const T *__restrict__ V,
                              size_t vstride, int nv, const double *__restrict__ coef,
                              const int32_t *__restrict__ col_sys, int N, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int s = col_sys[e / N];
        double acc = alpha ? alpha[s] * (double)y[e] : 0.0;
        for (int i = 0; i < nv; ++i) acc += coef[(size_t)s * nv + i] * (double)V[(size_t)i * vstride + e];
        y[e] = (T)acc;
    }
}

}  // namespace fpsa
