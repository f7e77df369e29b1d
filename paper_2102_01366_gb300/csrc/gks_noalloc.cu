// gks_noalloc.cu -- time-step reduction whose scratch lives in a fixed
// file-scope device array, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where device allocation is not allowed or not
// wanted -- inside a CUDA stream capture (cudaMalloc is illegal while a
// stream is being captured), in a real-time loop with a hard no-allocation
// rule, or under a framework whose allocator owns the whole device and hands
// out no scratch.  gks_timestep needs a gks_state and its caller-allocated
// workspace; gks_timestep_noalloc needs only the cell averages and radii.
//
// The per-block partial minima go to g_dt_partials, a static __device__
// array of GKS_NOALLOC_MAX_BLOCKS doubles (64 KiB) that every GPU loading the
// library keeps until the process exits.  Host code cannot use the symbol
// itself as a device pointer: the first call on each device (with that
// device current) resolves its address with cudaGetSymbolAddress and caches
// it per device.  Every call shares the array, so calls that overlap on the
// GPU (different streams, no ordering between them) race; each call
// overwrites every partial it later reads, so nothing needs clearing.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "gks_internal.h"
#include "gks_kernels.h"

namespace gks {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = GKS_NOALLOC_MAX_BLOCKS;
constexpr int NA_MAX_DEVICES = 64;

__device__ __align__(256) double g_dt_partials[NA_MAX_BLOCKS];

// the same local limit and reduction order as the workspace version
__global__ void __launch_bounds__(NA_THREADS) k_na_partials(const double* __restrict__ W,
                                                           const double* __restrict__ dr, int64_t nc,
                                                           HostPhys p, double* __restrict__ part) {
    __shared__ double smin[NA_THREADS];
    const int64_t c = (int64_t)blockIdx.x * NA_THREADS + threadIdx.x;
    double mn = INFINITY;
    if (c < nc) {
        double Wv[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) Wv[q] = W[q * nc + c];
        mn = local_dt(Wv, dr[c], p);
    }
    smin[threadIdx.x] = mn;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = smin[0];
}

__global__ void __launch_bounds__(NA_THREADS) k_na_finish(const double* __restrict__ part, int nblk,
                                                         double cfl, double* __restrict__ dt) {
    __shared__ double smin[NA_THREADS];
    double mn = INFINITY;
    for (int b = threadIdx.x; b < nblk; b += NA_THREADS) mn = fmin(mn, part[b]);
    smin[threadIdx.x] = mn;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *dt = cfl * smin[0];
}

std::mutex g_mu;
void* g_addr[NA_MAX_DEVICES] = {nullptr};

}  // namespace
}  // namespace gks

using namespace gks;

extern "C" gks_status gks_timestep_noalloc(const gks_params* p, const double* d_W, const double* d_dr,
                                           int64_t n_cell, double* d_dt, void* stream) {
    if (!p || !d_W || !d_dr || !d_dt) {
        set_error("gks_timestep_noalloc: NULL argument");
        return GKS_E_ARG;
    }
    if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || (p->viscous && !(p->mu > 0.0))) {
        set_error("gks_timestep_noalloc: needs gamma > 1, cfl > 0 and mu > 0 when viscous");
        return GKS_E_ARG;
    }
    const int64_t max_cells = (int64_t)NA_MAX_BLOCKS * NA_THREADS;
    if (n_cell <= 0 || n_cell > max_cells) {
        set_error("gks_timestep_noalloc: n_cell must be in [1, " + std::to_string(max_cells) +
                  "] (fixed scratch of " + std::to_string(NA_MAX_BLOCKS) + " block minima)");
        return GKS_E_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("gks_timestep_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return GKS_E_CUDA;
    }
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("gks_timestep_noalloc: device ordinal " + std::to_string(dev) + " beyond the " +
                  std::to_string(NA_MAX_DEVICES) + " devices it keeps scratch addresses for");
        return GKS_E_ARG;
    }
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_dt_partials);
            if (e != cudaSuccess || !addr) {
                set_error(std::string("gks_timestep_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return GKS_E_CUDA;
            }
            g_addr[dev] = addr;
        }
        part = static_cast<double*>(g_addr[dev]);
    }
    HostPhys hp{p->gamma, p->cfl, p->mu, p->eps_weno, p->tau_eps, p->tau_c,
                p->weno, p->order, p->smooth_flux, p->viscous};
    const int nblk = (int)((n_cell + NA_THREADS - 1) / NA_THREADS);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_na_partials<<<nblk, NA_THREADS, 0, s>>>(d_W, d_dr, n_cell, hp, part);
    k_na_finish<<<1, NA_THREADS, 0, s>>>(part, nblk, p->cfl, d_dt);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("gks_timestep_noalloc: launch: ") + cudaGetErrorString(e));
        return GKS_E_CUDA;
    }
    return GKS_OK;
}
