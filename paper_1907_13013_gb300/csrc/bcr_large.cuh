// Block cyclic reduction factorization for FP blocks larger than one CTA can
// invert in registers / shared memory (2N > 128): in-place recursive block-Schur
// inversion of each eliminated cell's 2N x 2N block,
//   [[A11, A12], [A21, A22]]^{-1}: P = A11^{-1}, X = P A12, Y = A21 P,
//   S = A22 - A21 X, Q = S^{-1},
//   A12 <- -X Q,  A21 <- -Q Y,  A11 <- P - X A21,  A22 <- Q,
// recursing on A11 and S until blocks are <= 128 (then Gauss-Jordan with partial
// pivoting, `gj_reg_body` / `gj_smem_body`). No pivoting crosses the halves; the
// FP blocks are well conditioned (the L-node half is |H|/2 + (h/3) K with
// K = sigma_a I - sigma_tr/2 A_FP), and the FP64 growth check of the whole block
// (max|A| max|A^{-1}|) guards every case. The inverse is finally transposed in
// place to the layout the BCR solve reads. All operations are batched over the
// eliminated cells of one level (a chunk of at most kLargeChunk at a time).
#pragma once

#include "kernels.cuh"

namespace fpsa {

constexpr int kLargeChunk = 1024;

// Matrix e of a batch: base + idx(e) * stride, row-major with leading dimension ld;
// idx(e) = items[e].cell (by_cell) or e.
template <typename T>
struct BMat {
    T *base;
    long long stride;
    int ld;
    int by_cell;
    __host__ __device__ BMat sub(int r0, int c0) const { return BMat{base + (long long)r0 * ld + c0, stride, ld, by_cell}; }
};

template <typename T>
__device__ __forceinline__ T *bmat_ptr(const BMat<T> &m, const BcrItem *items, int e) {
    return m.base + (long long)(m.by_cell ? items[e].cell : e) * m.stride;
}

template <typename T, int N2>
__global__ void __launch_bounds__(512) k_binv_reg_rm(BMat<T> M, const BcrItem *__restrict__ items,
                                                     int *__restrict__ status) {
    T *p = bmat_ptr(M, items, blockIdx.x);
    if constexpr (sizeof(T) == 4) gj_panel_body<N2>(p, M.ld, p, M.ld, false, nullptr, status);
    else gj_reg_body<T, N2>(p, M.ld, p, M.ld, false, nullptr, status);
}

template <typename T>
__global__ void k_binv_smem_rm(BMat<T> M, int n, const BcrItem *__restrict__ items, int *__restrict__ status) {
    T *p = bmat_ptr(M, items, blockIdx.x);
    gj_smem_body(p, M.ld, p, M.ld, false, n, nullptr, status);
}

// C = alpha A B + beta C for n x n blocks of a batch (blockIdx.z = batch element),
// 64 x 64 output tiles, 256 threads with 4 x 4 outputs each, k-steps of 16 through
// shared memory. C never aliases A or B.
template <typename T>
__global__ void __launch_bounds__(256) k_bgemm(int n, T alpha, BMat<T> A, BMat<T> B, T beta, BMat<T> C,
                                               const BcrItem *__restrict__ items) {
    __shared__ T As[16][64 + 1], Bs[16][64 + 1];
    const T *a = bmat_ptr(A, items, blockIdx.z);
    const T *b = bmat_ptr(B, items, blockIdx.z);
    T *c = bmat_ptr(C, items, blockIdx.z);
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < n; k0 += 16) {
        for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
            const int kk = idx & 15, rr = idx >> 4;  // A tile: rows r0.., cols k0..
            const int gr = r0 + rr, gk = k0 + kk;
            As[kk][rr] = (gr < n && gk < n) ? a[(size_t)gr * A.ld + gk] : T(0);
            const int cc = idx & 63, kb = idx >> 6;  // B tile: rows k0.., cols c0..
            const int gk2 = k0 + kb, gc = c0 + cc;
            Bs[kb][cc] = (gk2 < n && gc < n) ? b[(size_t)gk2 * B.ld + gc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gr = r0 + ty + 16 * i, gc = c0 + tx + 16 * j;
            if (gr < n && gc < n) {
                T *dst = c + (size_t)gr * C.ld + gc;
                *dst = alpha * acc[i][j] + (beta != T(0) ? beta * *dst : T(0));
            }
        }
}

// max|A| of each block of the batch (before inversion), for the growth check.
template <typename T>
__global__ void k_bamax(BMat<T> M, int n, const BcrItem *__restrict__ items, double *__restrict__ amax) {
    const T *p = bmat_ptr(M, items, blockIdx.x);
    double m = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x)
        m = fmax(m, fabs((double)p[(size_t)(idx / n) * M.ld + idx % n]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = fmax(r, red[i]);
        amax[blockIdx.x] = r;
    }
}

// In-place transpose of each n x n inverse (row-major -> the transposed layout of
// the BCR solve) with the growth check max|A| max|A^{-1}| and a finiteness check.
template <typename T>
__global__ void k_btranspose(BMat<T> M, int n, const BcrItem *__restrict__ items, const double *__restrict__ amax,
                             unsigned long long *__restrict__ growth, int *__restrict__ status) {
    T *p = bmat_ptr(M, items, blockIdx.x);
    double m = 0.0;
    bool bad = false;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx % n;
        if (j < i) continue;
        T *x = p + (size_t)i * M.ld + j, *y = p + (size_t)j * M.ld + i;
        const T a = *x, b = *y;
        *x = b;
        *y = a;
        m = fmax(m, fmax(fabs((double)a), fabs((double)b)));
        if (!isfinite((double)a) || !isfinite((double)b)) bad = true;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(growth, dkey(m * amax[blockIdx.x]));
    if (bad) atomicExch(status, 1);
}

}  // namespace fpsa
