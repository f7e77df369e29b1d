// gks_kernels.cu -- cell-update and bookkeeping kernels of one two-stage step
// (sm_103a, FP64 and FP32-bulk instantiations).  The reconstruction kernels
// are in gks_recon.cu, the face flux in gks_flux.cu.
//
//   k_update1  cell-ordered gather of the 4 face records (CSR, signed):
//              W*, grad W* and the saved stage-1 terms
//   k_update2  W^{n+1}, grad W^{n+1}; per-case minima of the next step's
//              local time-step limits (Sec. 5) and residual sums
//   k_dt_*     time-step rule of Sec. 5 (deterministic per-block minima)
//   k_pack / k_unpack_grad   public [component][cell] FP64 state <-> the
//              cell-major working state
//
// No atomics on data: every sum has a fixed order, so results are
// reproducible run to run (the per-case minima use atomicMin, which is
// exact).
#include <cuda_runtime.h>

#include <algorithm>

#include "gks_update.cuh"

namespace gks {


template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_update1(DevMesh<T> m, HostPhys p, DevState<T> st) {
    update1_cells<T>(m, p, st, blockIdx.x, threadIdx.x);
}

// the block's own slice of shared memory for a whole-block cell group
#define GKS_BLOCK_GROUP(name)                                        \
    __shared__ double name##_sv[CELLS_PER_BLOCK];                    \
    __shared__ int32_t name##_sc[CELLS_PER_BLOCK];                   \
    __shared__ double name##_red[CELL_THREADS / 32 * 6];             \
    const CellGroup name{(int64_t)blockIdx.x, (int)threadIdx.x, 0, name##_sv, name##_sc, name##_red}

template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_update2(DevMesh<T> m, HostPhys p, DevState<T> st) {
    GKS_BLOCK_GROUP(grp);
    update2_cells<T>(m, p, st, grp);
}

template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_dt_partials(DevMesh<T> m, HostPhys p,
                                                               const T* __restrict__ X,
                                                               double* __restrict__ part) {
    const CellLane cl = cell_lane(m.nc);
    T mn = T(INFINITY);
    T zero[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (cl.active && cl.q == 0) {
        T Wv[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) Wv[q] = X[cl.c * Stride<T>::xs + q];
        mn = local_dt(Wv, m.dr[cl.c], p);
    }
    GKS_BLOCK_GROUP(grp);
    block_reduce_part<T>(mn, zero, part + (int64_t)blockIdx.x * PART_N, grp);
}

template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_init_dtmin(DevMesh<T> m, HostPhys p, const T* __restrict__ X,
                                                              unsigned long long* __restrict__ dtmin) {
    const CellLane cl = cell_lane(m.nc);
    const bool lead = cl.active && cl.q == 0;
    double mn = INFINITY;
    if (lead) {
        T Wv[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) Wv[q] = X[cl.c * Stride<T>::xs + q];
        mn = (double)local_dt(Wv, m.dr[cl.c], p);
    }
    const int lc = (int)(cl.c - (int64_t)blockIdx.x * CELLS_PER_BLOCK);
    GKS_BLOCK_GROUP(grp);
    block_case_min(mn, m.cell_case[cl.c], lead && lc >= 0 && lc < CELLS_PER_BLOCK && mn < INFINITY, lc, dtmin, grp);
}

__global__ void k_set_control(double* ctrl, double* case_t, double* case_dt, unsigned long long* dtmin,
                              int32_t ncase, double dt_fixed, double t_end, int reset) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctrl[CTRL_DT_FIXED] = dt_fixed;
        ctrl[CTRL_T_END] = t_end;
    }
    if (reset)
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncase; k += gridDim.x * blockDim.x) {
            case_t[k] = 0.0;
            case_dt[k] = 0.0;
            dtmin[k] = (unsigned long long)__double_as_longlong(INFINITY);
        }
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}

// cperm (may be NULL): device cell -> the caller's cell of W, dW
template <typename T>
__global__ void k_pack(const double* __restrict__ W, const double* __restrict__ dW, T* __restrict__ X, int64_t nc,
                       const int32_t* __restrict__ cperm) {
    constexpr int XSR = Stride<T>::xs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc * XSR; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = i / XSR;
        const int64_t c = cperm ? (int64_t)cperm[d] : d;
        const int j = (int)(i - d * XSR);
        T v = T(0);
        if (j < 5) {
            v = (T)W[j * nc + c];
        } else if (j < 20) {
            v = (T)dW[(j - 5) * nc + c];
        } else if (sizeof(T) == 4 && j < XLO + 5) {
            const double w = W[(j - XLO) * nc + c];
            v = (T)(w - (double)(T)w);  // lo part of the FP32 pair
        }
        X[i] = v;
    }
}

template <typename T>
__global__ void k_unpack_grad(const T* __restrict__ X, double* __restrict__ dW, int64_t nc,
                              const int32_t* __restrict__ cperm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc * 15; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / nc, d = i - j * nc;
        dW[j * nc + (cperm ? (int64_t)cperm[d] : d)] = (double)X[d * Stride<T>::xs + 5 + j];
    }
}

// the averages of an FP64 working state [nc][XS] to W [5][nc]
__global__ void k_unpack_avg(const double* __restrict__ X, double* __restrict__ W, int64_t nc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc * 5; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i / nc, c = i - q * nc;
        W[q * nc + c] = X[c * Stride<double>::xs + q];
    }
}

cudaError_t launch_unpack_avg(const double* X, double* W, int64_t nc, cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((5 * nc + 255) / 256, 65535);
    k_unpack_avg<<<(unsigned)blocks, 256, 0, s>>>(X, W, nc);
    return cudaGetLastError();
}

// component-major [ncomp][nc] arrays between the device cell order and the
// caller's (cperm: device cell -> caller's cell)
__global__ void k_cells_perm(const double* __restrict__ in, double* __restrict__ out, int64_t nc, int ncomp,
                             const int32_t* __restrict__ cperm, int to_public) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc * ncomp; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / nc, d = i - k * nc, c = cperm[d];
        if (to_public)
            out[k * nc + c] = in[i];
        else
            out[i] = in[k * nc + c];
    }
}

// out row r = in row map[r], rows of `width` words of 4 bytes
__global__ void k_rows_gather(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t nrows, int width,
                              const int32_t* __restrict__ map) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows * width; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / width;
        out[i] = in[(int64_t)map[r] * width + (i - r * width)];
    }
}

template <typename T>
__global__ void k_rec_out(const T* __restrict__ rec, const int32_t* __restrict__ perm, double* __restrict__ out,
                          int64_t nf, int nr, DevMesh<T> m, const T* __restrict__ X, int addback, double gm1,
                          double dt) {
    constexpr int XSR = Stride<T>::xs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf * nr; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = i / nr;
        const int j = (int)(i - d * nr);
        // FP32 stage-1 records: device stride 50 (reference flux at 40..49)
        const int rs = (sizeof(T) == 4 && nr == 40) ? REC1_F32 : nr;
        const T* r = rec + d * rs;
        double v = (double)r[j];
        if (sizeof(T) == 4 && nr == 40 && j < 10) {
            // the reference flux (dt / 2) A F_n(W_m), twice in the S entries
            const double ref = (double)r[REC1_REF + j % 5] + (double)r[REC1_REF + 5 + j % 5];
            v += j < 5 ? ref : 2.0 * ref;
        }
        if (sizeof(T) == 4 && addback && j >= 10) {
            // the mean of the two averages (the interior one on a boundary
            // face) times sum_k w_k n = 3 w n
            const int k = (j - 10) % 15, q = k / 3, dir = k - 3 * q;
            const int L = m.flr[d], R = m.flr[m.nf + d];
            auto avg = [&](int c) { return (double)X[(int64_t)c * XSR + q] + (double)X[(int64_t)c * XSR + XLO + q]; };
            const double wm = (L >= 0 && R >= 0) ? 0.5 * (avg(L) + avg(R)) : avg(L >= 0 ? L : R);
            const T* geo = m.fgeo + d * FGEO;
            v += wm * 3.0 * (double)geo[3] * (double)geo[dir];
        }
        out[(int64_t)perm[d] * nr + j] = v;
    }
}

template <typename T>
__global__ void k_poly_out(const T* __restrict__ in, double* __restrict__ out, int64_t nc,
                           const int32_t* __restrict__ cperm) {
    constexpr int PS = Stride<T>::poly;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc * 50; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / 50;
        const int k = (int)(i - c * 50);
        const int64_t o = (cperm ? (int64_t)cperm[c] : c) * 50 + k;
        double v = (double)in[c * PS + k];
        if (sizeof(T) == 4 && k % 10 == 0) {
            // FP32 records hold R(centroid) minus the average: add the average back
            const int q = k / 10;
            v += (double)in[c * PS + PHI + q] + (double)in[c * PS + PLO + q];
        }
        out[o] = v;
    }
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
int update_blocks(int64_t nc) { return (int)cell_grid(nc); }

template <typename T>
cudaError_t Launch<T>::update1(const DevMesh<T>& m, const HostPhys& p, const DevState<T>& st, cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    k_update1<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, p, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::update2(const DevMesh<T>& m, const HostPhys& p, const DevState<T>& st,
                               cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    k_update2<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, p, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::dt_partials(const DevMesh<T>& m, const HostPhys& p, const T* X,
                                   double* part, cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    k_dt_partials<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, p, X, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::init_dtmin(const DevMesh<T>& m, const HostPhys& p, const T* X,
                                  unsigned long long* case_dtmin, cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    k_init_dtmin<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, p, X, case_dtmin);
    return cudaGetLastError();
}

static inline unsigned ew_grid(int64_t n) { return (unsigned)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192); }

template <typename T>
cudaError_t Launch<T>::pack(const double* W, const double* dW, T* X, int64_t nc, cudaStream_t s,
                            const int32_t* cperm) {
    if (nc == 0) return cudaSuccess;
    k_pack<T><<<ew_grid(nc * Stride<T>::xs), 256, 0, s>>>(W, dW, X, nc, cperm);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::unpack_grad(const T* X, double* dW, int64_t nc, cudaStream_t s, const int32_t* cperm) {
    if (nc == 0) return cudaSuccess;
    k_unpack_grad<T><<<ew_grid(nc * 15), 256, 0, s>>>(X, dW, nc, cperm);
    return cudaGetLastError();
}

cudaError_t launch_cells_perm(const double* in, double* out, int64_t nc, int ncomp, const int32_t* cperm,
                              int to_public, cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    k_cells_perm<<<ew_grid(nc * ncomp), 256, 0, s>>>(in, out, nc, ncomp, cperm, to_public);
    return cudaGetLastError();
}

cudaError_t launch_rows_gather(const void* in, void* out, int64_t nrows, int width_words, const int32_t* map,
                               cudaStream_t s) {
    if (nrows == 0) return cudaSuccess;
    k_rows_gather<<<ew_grid(nrows * width_words), 256, 0, s>>>(static_cast<const uint32_t*>(in),
                                                               static_cast<uint32_t*>(out), nrows, width_words, map);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::to_double(const T* in, double* out, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_convert<T, double><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::from_double(const double* in, T* out, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_convert<double, T><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::rec_to_double(const T* rec, const int32_t* perm, double* out, int64_t nf, int nr,
                                     const DevMesh<T>* m, const T* X, double gm1, double dt, cudaStream_t s) {
    if (nf == 0) return cudaSuccess;
    const int64_t n = nf * nr;
    const int addback = (m && X && nr == 40) ? 1 : 0;
    DevMesh<T> mv{};
    if (m) mv = *m;
    k_rec_out<T><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(rec, perm, out, nf, nr,
                                                                                            mv, X, addback, gm1, dt);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::poly_to_double(const T* in, double* out, int64_t nc, cudaStream_t s, const int32_t* cperm) {
    if (nc == 0) return cudaSuccess;
    const int64_t n = nc * 50;
    k_poly_out<T><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(in, out, nc, cperm);
    return cudaGetLastError();
}

cudaError_t launch_set_control(double* ctrl, double* case_t, double* case_dt, unsigned long long* case_dtmin,
                               int32_t ncase, double dt_fixed, double t_end, int reset_time, cudaStream_t s) {
    const int grid = reset_time ? (int)((ncase + 255) / 256 < 1024 ? (ncase + 255) / 256 : 1024) : 1;
    k_set_control<<<grid < 1 ? 1 : grid, 256, 0, s>>>(ctrl, case_t, case_dt, case_dtmin, ncase, dt_fixed,
                                                      t_end, reset_time);
    return cudaGetLastError();
}


#define GKS_CELLS_INST(T)                                                                                   \
    template cudaError_t Launch<T>::update1(const DevMesh<T>&, const HostPhys&, const DevState<T>&,         \
                                            cudaStream_t);                                                  \
    template cudaError_t Launch<T>::update2(const DevMesh<T>&, const HostPhys&, const DevState<T>&,         \
                                            cudaStream_t);                                                  \
    template cudaError_t Launch<T>::dt_partials(const DevMesh<T>&, const HostPhys&, const T*, double*,      \
                                                cudaStream_t);                                              \
    template cudaError_t Launch<T>::init_dtmin(const DevMesh<T>&, const HostPhys&, const T*,                \
                                               unsigned long long*, cudaStream_t);                          \
    template cudaError_t Launch<T>::pack(const double*, const double*, T*, int64_t, cudaStream_t,           \
                                         const int32_t*);                                                   \
    template cudaError_t Launch<T>::unpack_grad(const T*, double*, int64_t, cudaStream_t, const int32_t*);  \
    template cudaError_t Launch<T>::to_double(const T*, double*, int64_t, cudaStream_t);                    \
    template cudaError_t Launch<T>::from_double(const double*, T*, int64_t, cudaStream_t);                  \
    template cudaError_t Launch<T>::rec_to_double(const T*, const int32_t*, double*, int64_t, int,          \
                                                  const DevMesh<T>*, const T*, double, double, cudaStream_t); \
    template cudaError_t Launch<T>::poly_to_double(const T*, double*, int64_t, cudaStream_t, const int32_t*);
GKS_CELLS_INST(double)
GKS_CELLS_INST(float)

}  // namespace gks
