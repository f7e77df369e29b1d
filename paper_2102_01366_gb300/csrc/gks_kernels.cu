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

#include "gks_cells.cuh"
#include "gks_device.cuh"
#include "gks_kernels.h"

namespace gks {


// per-case minimum of the local limits of the cells of a block: the block's
// cells are contiguous and so are the cases, so its cases form runs; one
// thread scans the 24 values and issues one atomicMin per run (the minimum
// is exact, so the result does not depend on the order; the result of the
// atomic is not used, so it does not stall the thread)
__device__ void block_case_min(double v, int32_t cas, bool valid, int lc, unsigned long long* dtmin) {
    __shared__ double sv[CELLS_PER_BLOCK];
    __shared__ int32_t sc[CELLS_PER_BLOCK];
    if (threadIdx.x < CELLS_PER_BLOCK) sc[threadIdx.x] = -1;
    __syncthreads();
    if (valid) {
        sv[lc] = v;
        sc[lc] = cas;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // positive doubles order like their bit patterns
        auto commit = [&](int32_t k, double v) {
            atomicMin(dtmin + k, (unsigned long long)__double_as_longlong(v));
        };
        int32_t cur = -1;
        double mn = INFINITY;
        for (int i = 0; i < CELLS_PER_BLOCK; ++i) {
            if (sc[i] < 0) continue;
            if (sc[i] != cur) {
                if (cur >= 0 && mn < INFINITY) commit(cur, mn);
                cur = sc[i];
                mn = INFINITY;
            }
            mn = fmin(mn, sv[i]);
        }
        if (cur >= 0 && mn < INFINITY) commit(cur, mn);
    }
}

// --------------------------------------------------------------------------
// cell updates (5 lanes per cell)
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_update1(DevMesh<T> m, HostPhys p, DevState<T> st) {
    const CellLane cl = cell_lane(m.nc);
    if (!cl.active) return;
    const int64_t nc = m.nc, c = cl.c;
    if (!(st.case_dt[m.cell_case[c]] > 0.0)) return;  // finished case
    const int q = cl.q;
    CSum<T> fh, s1;
    fh.init();
    s1.init();
    T gs[3] = {T(0), T(0), T(0)}, g0[3] = {T(0), T(0), T(0)};
#pragma unroll
    constexpr int RS = sizeof(T) == 4 ? REC1_F32 : 40;
    for (int f = 0; f < 4; ++f) {
        const int e = m.cface[f * nc + c];
        const T s = (e & 1) ? T(-1) : T(1);
        const T* r = st.rec + (int64_t)(e >> 1) * RS;
        fh.add(s * r[q]);
        s1.add(s * r[5 + q]);
        if constexpr (sizeof(T) == 4) {
            // the reference flux (dt / 2) A F_n(W_m) of the face, hi + lo; the
            // S entry takes it twice (2 Fh - D / 3)
            fh.add(s * r[REC1_REF + q]);
            fh.add(s * r[REC1_REF + 5 + q]);
            s1.add(T(2) * s * r[REC1_REF + q]);
            s1.add(T(2) * s * r[REC1_REF + 5 + q]);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gs[i] += s * r[10 + 3 * q + i];
            g0[i] += s * r[25 + 3 * q + i];
        }
    }
    const double iv = m.inv_vol[c];
    constexpr int XSR = Stride<T>::xs;
    if constexpr (sizeof(T) == 4) {
        // FP32 records hold the interface states relative to the mean of the
        // face's two cell averages W_m (the interior cell's average on a
        // boundary face).  The cell needs sum_f s_f W_m A_f n_f back; as
        // sum_f s_f A_f n_f = 0 over a closed cell, that is
        // 1/2 sum_f s_f (W_nb - W_c) A_f n_f over its interior faces, formed
        // from the exact differences of the hi / lo pairs (A = 3 w).
        const T hc = st.X[c * XSR + q], lc = st.X[c * XSR + XLO + q];
        T ab[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const int nb = m.nbr[f * nc + c];
            if (nb < 0) continue;
            const int e = m.cface[f * nc + c];
            const T* geo = m.fgeo + (int64_t)(e >> 1) * FGEO;
            const T dw = (st.X[(int64_t)nb * XSR + q] - hc) + (st.X[(int64_t)nb * XSR + XLO + q] - lc);
            const T a = ((e & 1) ? T(-1.5) : T(1.5)) * geo[3] * dw;
#pragma unroll
            for (int i = 0; i < 3; ++i) ab[i] += a * geo[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gs[i] += ab[i];
            g0[i] += ab[i];
        }
    }
    T* xs = st.Xs + c * XSR;
    // W* = W^n - (1/|Omega|) sum s sum_k w Fh  (Eq. s2o4, first stage)
    const double wstar = st.Wd[q * nc + c] - fh.value() * iv;
    xs[q] = (T)wstar;
    if constexpr (sizeof(T) == 4) xs[XLO + q] = (T)(wstar - (double)(T)wstar);
    st.S[q * nc + c] = s1.value();
    const T ivr = (T)iv;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        xs[5 + 3 * q + i] = gs[i] * ivr;  // Eq. gauss-formula at t* (Eq. step-du)
        st.G[(3 * q + i) * nc + c] = g0[i];
    }
}

// deterministic block reduction of one min and five sums in precision R
// (warp shuffles, then the 4 warp results in a fixed order)
template <typename R>
__device__ __forceinline__ void block_reduce_part(R mn, const R* sums, double* out) {
    __shared__ R red[CELL_THREADS / 32][6];
    R v[6] = {mn, sums[0], sums[1], sums[2], sums[3], sums[4]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmin(v[0], __shfl_down_sync(0xffffffffu, v[0], o));
#pragma unroll
        for (int k = 1; k < 6; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        R r[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = red[0][k];
        for (int w = 1; w < CELL_THREADS / 32; ++w) {
            r[0] = fmin(r[0], red[w][0]);
#pragma unroll
            for (int k = 1; k < 6; ++k) r[k] += red[w][k];
        }
        out[PART_DTMIN] = (double)r[0];
#pragma unroll
        for (int q = 0; q < 5; ++q) out[PART_RES + q] = (double)r[1 + q];
    }
}

template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_update2(DevMesh<T> m, HostPhys p, DevState<T> st) {
    const CellLane cl = cell_lane(m.nc);
    const int64_t nc = m.nc, c = cl.c;
    const int q = cl.q;
    const int32_t cas = m.cell_case[c];
    const double dtd = st.case_dt[cas];
    const bool live = cl.active && dtd > 0.0;  // finished cases keep their state
    T mn = T(INFINITY);
    T res[5] = {T(0), T(0), T(0), T(0), T(0)};
    CSum<T> f2;
    f2.init();
    T dg[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int e = m.cface[f * nc + c];
        const T s = (e & 1) ? T(-1) : T(1);
        const T* r = st.rec + (int64_t)(e >> 1) * 20;
        f2.add(s * r[q]);
#pragma unroll
        for (int i = 0; i < 3; ++i) dg[i] += s * r[5 + 3 * q + i];
    }
    const double iv = m.inv_vol[c];
    // W^{n+1} |Omega| = W^n |Omega| - [dt F + dt^2/6 F_t](W^n) - [dt^2/3 F_t](W*)
    // (Eq. s2o4, second stage)
    const double inc = live ? ((st.S[q * nc + c] + (double)f2.hi) + (double)f2.lo) * iv : 0.0;
    const double wn = st.Wd[q * nc + c] - inc;
    const T Wq = (T)wn;
    if (live) {
        st.Wd[q * nc + c] = wn;
        T* x = st.X + c * Stride<T>::xs;
        x[q] = Wq;
        if constexpr (sizeof(T) == 4) x[XLO + q] = (T)(wn - (double)Wq);
        const T ivr = (T)iv;
#pragma unroll
        for (int i = 0; i < 3; ++i) x[5 + 3 * q + i] = (st.G[(3 * q + i) * nc + c] + dg[i]) * ivr;
        // squared rates of change (W^{n+1} - W^n) / dt for the residual
        const T ti = (T)inc / (T)dtd;
#pragma unroll
        for (int k = 0; k < 5; ++k) res[k] = k == q ? ti * ti : T(0);
    }
    // the cell's new state, gathered from its 5 lanes, for the positivity flag
    // and the next step's local time-step limit
    T Wn[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) Wn[k] = __shfl_sync(0xffffffffu, Wq, cl.base + k);
    const bool lead = cl.active && q == 0;
    if (lead) {
        const T pr = T(p.gamma - 1.0) * (Wn[4] - T(0.5) * (Wn[1] * Wn[1] + Wn[2] * Wn[2] + Wn[3] * Wn[3]) / Wn[0]);
        if (!(Wn[0] > T(0)) || !(pr > T(0))) atomicOr(st.err, ERR_STATE);
        else mn = local_dt(Wn, m.dr[c], p);
    }
    const int lc = (int)(c - (int64_t)blockIdx.x * CELLS_PER_BLOCK);
    block_case_min((double)mn, cas, lead && lc >= 0 && lc < CELLS_PER_BLOCK && mn < T(INFINITY), lc, st.case_dtmin);
    T mn_unused = T(INFINITY);
    block_reduce_part<T>(mn_unused, res, st.part + (int64_t)blockIdx.x * PART_N);
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
    block_reduce_part<T>(mn, zero, part + (int64_t)blockIdx.x * PART_N);
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
    block_case_min(mn, m.cell_case[cl.c], lead && lc >= 0 && lc < CELLS_PER_BLOCK && mn < INFINITY, lc, dtmin);
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
