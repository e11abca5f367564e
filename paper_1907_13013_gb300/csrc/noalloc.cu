// fpsa_sweep_noalloc: one LD transport sweep for callers that cannot allocate
// device memory (declaration and contract in include/fpsa.h).
//
// The context-based path keeps the sweep coefficients of every cell and
// ordinate in a cudaMalloc'ed buffer owned by the context. Some callers cannot
// allocate: code running inside another framework's memory pool or under its
// allocator lock, or a process whose device memory is fully reserved up front.
// For them this entry point runs the coefficient kernel and an affine-scan sweep
// with that scratch placed in a fixed file-scope __device__ array instead. The
// array is sized for FPSA_SWEEP_NOALLOC_MAX_CELL_ANGLES cell-angles and exists on
// every GPU that loads the library until the process exits.
//
// Per call nothing is copied from host memory: the Gauss-Legendre ordinates of
// every even N up to the maximum are written into a second __device__ table once
// per device (the first call's set-up), and the slab's cell count reaches the
// device as a kernel argument.
#include <mutex>
#include <vector>

#include "fpsa_internal.h"
#include "kernels.cuh"

namespace {

constexpr int kNoallocMaxN = 256;
constexpr int kNoallocThreads = 256;
constexpr long long kMaxCellAngles = FPSA_SWEEP_NOALLOC_MAX_CELL_ANGLES;
// mu of order N (even) starts at (N/2 - 1)(N/2) in the ordinate table
constexpr int mu_offset(int N) { return (N / 2 - 1) * (N / 2); }
constexpr int kMuTable = mu_offset(kNoallocMaxN) + kNoallocMaxN;

// Scratch for the per-(cell, ordinate) sweep coefficients, coef[g][6][n].
static __device__ __align__(256) double g_noalloc_coef[6 * kMaxCellAngles];
// Ordinates of every even N <= kNoallocMaxN, ascending within each order.
static __device__ __align__(256) double g_noalloc_mu[kMuTable];
// One-instance geometry the sweep kernel reads: {offset 0, K}.
static __device__ __align__(256) int32_t g_noalloc_geom[2];

// Device addresses of the arrays above, looked up once per device with that
// device current (in host code the name of a __device__ array is only a stand-in,
// never a usable device address).
struct DeviceSymbols {
    bool ready = false;
    double *coef = nullptr;
    double *mu = nullptr;
    int32_t *geom = nullptr;
};
constexpr int kMaxDevices = 64;
std::mutex g_symbols_mutex;
DeviceSymbols g_symbols[kMaxDevices];

// First use on a device: the symbol addresses, then the ordinate table (one
// synchronous copy of host-built tables; later calls copy nothing).
int symbols_for_current_device(DeviceSymbols **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FPSA_ECUDA;
    std::lock_guard<std::mutex> lock(g_symbols_mutex);
    DeviceSymbols &s = g_symbols[dev];
    if (!s.ready) {
        DeviceSymbols t;
        if (cudaGetSymbolAddress((void **)&t.coef, g_noalloc_coef) != cudaSuccess) return FPSA_ECUDA;
        if (cudaGetSymbolAddress((void **)&t.mu, g_noalloc_mu) != cudaSuccess) return FPSA_ECUDA;
        if (cudaGetSymbolAddress((void **)&t.geom, g_noalloc_geom) != cudaSuccess) return FPSA_ECUDA;
        std::vector<double> mu(kMuTable, 0.0);
        for (int N = 2; N <= kNoallocMaxN; N += 2) {
            fpsa::Tables tab;
            fpsa::build_tables(N, 1, FPSA_LAPLACIAN_WFD, tab);  // only mu is used
            std::copy(tab.mu.begin(), tab.mu.end(), mu.begin() + mu_offset(N));
        }
        if (cudaMemcpy(t.mu, mu.data(), mu.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return FPSA_ECUDA;
        t.ready = true;
        s = t;
    }
    *out = &s;
    return FPSA_OK;
}

__global__ void k_noalloc_geometry(int32_t *geom, int K) {
    geom[0] = 0;
    geom[1] = K;
}

template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
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
    const double *mu = sym->mu + mu_offset(N);
    const size_t tot = (size_t)K * N;
    // Each launch's own status is checked (cudaLaunchKernelEx returns it), so an
    // error left pending by unrelated earlier work is neither reported nor cleared
    // here unless it has made the context unusable.
    if (launch(k_noalloc_geometry, dim3(1), dim3(1), st, sym->geom, K) != cudaSuccess) return FPSA_ECUDA;
    // Every coefficient the sweep reads is rewritten here first, so nothing left
    // in the shared array by an earlier call is ever read.
    if (launch(fpsa::k_sweep_coef<double>, dim3((unsigned)((tot + 255) / 256)), dim3(256), st, mu, h, sigma_t, N, K,
               sym->coef) != cudaSuccess)
        return FPSA_ECUDA;
    if (launch(fpsa::k_sweep<double, kNoallocThreads, false>, dim3(N, 1, 1), dim3(kNoallocThreads), st, q, psi,
               (const double *)sym->coef, mu, (const int32_t *)sym->geom, (const int32_t *)(sym->geom + 1), N, K,
               (const double *)nullptr, (const int32_t *)nullptr, (double *)nullptr) != cudaSuccess)
        return FPSA_ECUDA;
    return FPSA_OK;
}
