// fpsa_sweep_noalloc: one LD transport sweep for callers that cannot allocate
// device memory (declaration and contract in include/fpsa.h).
//
// The context-based path keeps the sweep coefficients of every cell and
// ordinate in a cudaMalloc'ed buffer owned by the context. Some callers cannot
// allocate: code running inside another framework's memory pool or allocator
// lock, code that must not create allocations while a stream is being recorded
// into a CUDA graph, or processes whose device memory is fully reserved up front.
// For them this entry point runs the same two kernels (coefficients, then the
// affine-scan sweep) with that scratch placed in a fixed file-scope __device__
// array instead. The array is sized for FPSA_SWEEP_NOALLOC_MAX_CELL_ANGLES
// cell-angles and exists on every GPU that loads the library until the process
// exits.
#include <mutex>
#include <vector>

#include "fpsa_internal.h"
#include "kernels.cuh"

namespace {

constexpr int kNoallocMaxN = 256;
constexpr int kNoallocThreads = 256;
constexpr long long kMaxCellAngles = FPSA_SWEEP_NOALLOC_MAX_CELL_ANGLES;

// Scratch for the per-(cell, ordinate) sweep coefficients, coef[g][6][n].
static __device__ __align__(256) double g_noalloc_coef[6 * kMaxCellAngles];
// Ordinates and the one-instance geometry the sweep kernel reads.
static __device__ __align__(256) double g_noalloc_mu[kNoallocMaxN];
static __device__ __align__(256) int32_t g_noalloc_geom[2];  // {offset 0, K}

// Device addresses of the arrays above, looked up once per device with that
// device current (a host-side reference to a __device__ symbol is only a
// stand-in, never a usable device address).
struct DeviceSymbols {
    bool ready = false;
    double *coef = nullptr;
    double *mu = nullptr;
    int32_t *geom = nullptr;
};
constexpr int kMaxDevices = 64;
std::mutex g_symbols_mutex;
DeviceSymbols g_symbols[kMaxDevices];

int symbols_for_current_device(DeviceSymbols **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FPSA_ECUDA;
    std::lock_guard<std::mutex> lock(g_symbols_mutex);
    DeviceSymbols &s = g_symbols[dev];
    if (!s.ready) {
        if (cudaGetSymbolAddress((void **)&s.coef, g_noalloc_coef) != cudaSuccess) return FPSA_ECUDA;
        if (cudaGetSymbolAddress((void **)&s.mu, g_noalloc_mu) != cudaSuccess) return FPSA_ECUDA;
        if (cudaGetSymbolAddress((void **)&s.geom, g_noalloc_geom) != cudaSuccess) return FPSA_ECUDA;
        s.ready = true;
    }
    *out = &s;
    return FPSA_OK;
}

}  // namespace

extern "C" int fpsa_sweep_noalloc(int32_t n_ordinates, int32_t n_cells, const double *h, const double *sigma_t,
                                  const double *q, double *psi, void *stream) {
    const int N = n_ordinates, K = n_cells;
    if (N < 2 || N % 2 || K < 1 || !h || !sigma_t || !q || !psi) return FPSA_EINVAL;
    if (N > kNoallocMaxN || (long long)K * N > kMaxCellAngles) return FPSA_ENOTSUP;
    DeviceSymbols *sym = nullptr;
    int rc = symbols_for_current_device(&sym);
    if (rc != FPSA_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fpsa::Tables tab;
    fpsa::build_tables(N, 1, FPSA_LAPLACIAN_WFD, tab);  // only mu is used
    const int32_t geom[2] = {0, K};
    // Both copies are staged from pageable host memory before the calls return.
    if (cudaMemcpyAsync(sym->mu, tab.mu.data(), N * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FPSA_ECUDA;
    if (cudaMemcpyAsync(sym->geom, geom, sizeof(geom), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FPSA_ECUDA;
    const size_t tot = (size_t)K * N;
    // Every coefficient the sweep reads is rewritten here first, so nothing left
    // in the shared array by an earlier call is ever read.
    fpsa::k_sweep_coef<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(sym->mu, h, sigma_t, N, K, sym->coef);
    if (cudaGetLastError() != cudaSuccess) return FPSA_ECUDA;
    fpsa::k_sweep<double, kNoallocThreads><<<dim3(N, 1, 1), kNoallocThreads, 0, st>>>(
        q, psi, sym->coef, sym->mu, sym->geom, sym->geom + 1, N, K);
    if (cudaGetLastError() != cudaSuccess) return FPSA_ECUDA;
    return FPSA_OK;
}
