// gks_recon.cu -- reconstruction kernels (Sec. 4.1-4.3), sm_103a, FP64 and
// FP32-bulk instantiations.
//
//   k_slopes   reconstruction step 1: P1 slopes per cell (Sec. 4.3)
//   k_recon    reconstruction step 2: P2 by the 9x16 operator, smoothness
//              indicators, two-step beta_0, nonlinear weights, positivity
//              (Sec. 4.1-4.3); R written about the centroid in monomial form
//
// The first kernel of a step (block 0) also turns the per-case minima of
// the local time-step limits into each case's step (Sec. 5).
#include <cuda_runtime.h>

#include "gks_recon.cuh"

namespace gks {

// reconstruction step 1: P1 slopes b = M1 (Q_nb - Q_0), Sec. 4.3, the
// products in the operator precision TO
template <typename T, typename TO>
__global__ void __launch_bounds__(CELL_THREADS) k_slopes(DevMesh<T> m, const T* __restrict__ X,
                                                          T* __restrict__ slopes, FinArg<T> fin) {
    if (fin.dtmin && blockIdx.x == 0) finalize_cases(fin.dtmin, fin.case_t, fin.case_dt, fin.ncase, fin.cfl, fin.ctrl);
    const CellLane cl = cell_lane(m.nc);
    if (!cl.active) return;
    const int64_t nc = m.nc, c = cl.c;
    const int q = cl.q;
    T b[3];
    p1_slope<T, TO>(m, X, c, q, b);  // with the wall-constrained slopes of Sec. 4.4
    T* out = slopes + c * 15 + 3 * q;
    out[0] = b[0];
    out[1] = b[1];
    out[2] = b[2];
}

template <typename T, typename TO, bool WALL>
__global__ void __launch_bounds__(CELL_THREADS) k_recon(DevMesh<T> m, ReconConst<T> rc,
                                                         const T* __restrict__ X,
                                                         const T* __restrict__ slopes_in,
                                                         T* __restrict__ slopes_out,
                                                         T* __restrict__ poly,
                                                         int32_t* __restrict__ fallback,
                                                         FinArg<T> fin, int32_t* __restrict__ err) {
    __shared__ alignas(128) TO sT[TILE_ROWS][CELLS_PER_BLOCK];
    __shared__ alignas(8) unsigned long long bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();  // the barrier exists before anyone waits on it
    if (fin.dtmin && blockIdx.x == 0) finalize_cases(fin.dtmin, fin.case_t, fin.case_dt, fin.ncase, fin.cfl, fin.ctrl);
    recon_cells<T, TO, WALL>(m, rc, X, slopes_in, slopes_out, poly, fallback, err, blockIdx.x, threadIdx.x, sT, &bar,
                             0);
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
template <typename T>
static FinArg<T> fin_arg(const typename Launch<T>::Finalize* fin) {
    FinArg<T> a;
    a.dtmin = fin ? fin->dtmin : nullptr;
    a.case_t = fin ? fin->case_t : nullptr;
    a.case_dt = fin ? fin->case_dt : nullptr;
    a.ncase = fin ? fin->ncase : 0;
    a.cfl = fin ? fin->cfl : 0.0;
    a.ctrl = fin ? fin->ctrl : nullptr;
    return a;
}

template <typename T>
cudaError_t Launch<T>::slopes(const DevMesh<T>& m, const T* X, T* slopes, const Finalize* fin,
                              cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    if (m.M1d && sizeof(T) == 4)
        k_slopes<T, double><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, X, slopes, fin_arg<T>(fin));
    else
        k_slopes<T, T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, X, slopes, fin_arg<T>(fin));
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::recon(const DevMesh<T>& m, const HostPhys& p, const T* X, const T* slopes_in,
                             T* slopes, T* poly, int32_t* fallback, const Finalize* fin, int32_t* err,
                             cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    ReconConst<T> rc;
    rc.gm1 = (T)(p.gamma - 1.0);
    rc.eps = (T)p.eps_weno;
    rc.weno = p.weno;
    rc.order = p.order;
    // the wall-constrained instances only where the mesh has such cells
    auto go = [&](auto kernel) {
        kernel<<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, rc, X, slopes_in, slopes, poly, fallback, fin_arg<T>(fin),
                                                         err);
    };
    if (m.tiled && sizeof(T) == 4)
        m.wslot ? go(k_recon<T, double, true>) : go(k_recon<T, double, false>);
    else
        m.wslot ? go(k_recon<T, T, true>) : go(k_recon<T, T, false>);
    return cudaGetLastError();
}


#define GKS_RECON_INST(T)                                                                                  \
    template cudaError_t Launch<T>::slopes(const DevMesh<T>&, const T*, T*, const Launch<T>::Finalize*,     \
                                           cudaStream_t);                                                  \
    template cudaError_t Launch<T>::recon(const DevMesh<T>&, const HostPhys&, const T*, const T*, T*, T*,   \
                                          int32_t*, const Launch<T>::Finalize*, int32_t*, cudaStream_t);
GKS_RECON_INST(double)
GKS_RECON_INST(float)

// The bounded wait's failure path without a fault: an mbarrier that expects
// bytes no copy will deliver (nothing is in flight), polled `tries` times by
// the same try_wait as the reconstruction's tile wait; giving up sets
// ERR_TIMEOUT exactly as a stalled tile copy would.
__global__ void k_wait_probe(int32_t* __restrict__ err, int tries) {
    __shared__ alignas(8) unsigned long long bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);
    __syncthreads();
    bool ok = false;
    for (int i = 0; i < tries && !ok; ++i) ok = mbar_try_wait(&bar, 0);
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(err, ERR_TIMEOUT);
}

cudaError_t launch_wait_probe(int32_t* err, int tries, cudaStream_t s) {
    k_wait_probe<<<1, 64, 0, s>>>(err, tries);
    return cudaGetLastError();
}

}  // namespace gks
