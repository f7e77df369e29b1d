// gks_kernels.cu -- sm_103a kernels of one two-stage step of the compact
// gas-kinetic scheme on tetrahedra (FP64 and FP32-bulk instantiations).
//
//   k_slopes   reconstruction step 1: P1 slopes per cell (Sec. 4.3)
//   k_recon    reconstruction step 2: P2 by the 9x16 operator, smoothness
//              indicators, two-step beta_0, nonlinear weights, positivity
//              (Sec. 4.1-4.3); R written about the centroid in monomial form
//   k_flux     face-ordered: R of both cells at the 3 Gauss points, face
//              frame, kinetic solution (Sec. 2.2, 4.5), weighted face record
//              of the stage (Sec. 3 Eqs. linear-system, s2o4, step-du)
//   k_update1  cell-ordered gather of the 4 face records (CSR, signed):
//              W*, grad W* and the saved stage-1 terms
//   k_update2  W^{n+1}, grad W^{n+1}; per-block time-step minimum and
//              residual sums for the next step
//   k_dt_*     time-step rule of Sec. 5 (two-pass deterministic minimum)
//
// No atomics on data: every sum has a fixed order, so results are
// reproducible run to run.
#include <cuda_runtime.h>

#include "gks_device.cuh"
#include "gks_kernels.h"

namespace gks {

// ---- bulk copy global -> shared with an mbarrier (sm_90+ async proxy) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces the bytes the copy will deliver
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// bounded wait for phase `parity`: false if it gave up (each try_wait
// already suspends for a while, so the bound is far beyond any copy time)
constexpr int MBAR_TRIES = 1 << 16;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (int i = 0; i < MBAR_TRIES; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <typename T>
struct ReconConst {
    T gm1, eps;
    int weno, order;
};

// --------------------------------------------------------------------------
// cell kernels: 5 lanes per cell (one per conservative component), 6 cells
// per warp (lanes 30, 31 idle), CELLS_PER_BLOCK cells per 128-thread block
// --------------------------------------------------------------------------
// The step of every case from its minimum local limit (time-step rule of
// Sec. 5), with dt_fixed and t_end clipping; advances the case times and
// resets the minima for the next update.  One thread per case.
__device__ void finalize_cases(unsigned long long* __restrict__ dtmin, double* __restrict__ case_t,
                               double* __restrict__ case_dt, int32_t ncase, double cfl,
                               const double* __restrict__ ctrl) {
    const double dt_fixed = ctrl[CTRL_DT_FIXED], t_end = ctrl[CTRL_T_END];
    for (int k = threadIdx.x; k < ncase; k += blockDim.x) {
        const double mn = __longlong_as_double((long long)dtmin[k]);
        double dt = dt_fixed > 0.0 ? dt_fixed : (mn < INFINITY ? cfl * mn : 0.0);
        double t = case_t[k];
        if (t_end > 0.0) {
            const double rem = t_end - t;
            if (rem <= 1e-12 * t_end) {
                dt = 0.0;
                if (rem > 0.0) t = t_end;
            } else if (dt > rem) {
                dt = rem;
            }
        }
        if (!(dt > 0.0)) dt = 0.0;
        case_dt[k] = dt;
        case_t[k] = t + dt;
        dtmin[k] = (unsigned long long)__double_as_longlong(INFINITY);
    }
}

template <typename T>
struct FinArg {
    unsigned long long* dtmin;
    double* case_t;
    double* case_dt;
    int32_t ncase;
    double cfl;
    const double* ctrl;
};

// per-case minimum of the local limits of the cells of a block: the block's
// cells are contiguous and so are the cases, so its cases form runs; one
// thread scans the 24 values and issues one atomicMin per run (the minimum
// is exact, so the result does not depend on the order)
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
        // an update only when it can lower the current minimum: most blocks
        // then issue no atomic at all
        auto commit = [&](int32_t k, double v) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(v);
            if (b < *((volatile unsigned long long*)(dtmin + k))) atomicMin(dtmin + k, b);
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

struct CellLane {
    int64_t c;    // cell (clamped to a valid cell on idle lanes)
    int q;        // component
    int base;     // lane of component 0 of this cell
    bool active;  // lane carries a real (cell, component)
};

__device__ __forceinline__ CellLane cell_lane(int64_t nc) {
    CellLane L;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int cl = lane / 5;
    L.q = lane - 5 * cl;
    L.base = lane - L.q;
    const int64_t c = (int64_t)blockIdx.x * CELLS_PER_BLOCK + warp * 6 + cl;
    L.active = lane < 30 && c < nc;
    L.c = c < nc ? c : nc - 1;
    return L;
}

// reconstruction step 1: P1 slopes b = M1 (Q_nb - Q_0), Sec. 4.3
template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_slopes(DevMesh<T> m, const T* __restrict__ X,
                                                          T* __restrict__ slopes, FinArg<T> fin) {
    if (fin.dtmin && blockIdx.x == 0) finalize_cases(fin.dtmin, fin.case_t, fin.case_dt, fin.ncase, fin.cfl, fin.ctrl);
    const CellLane cl = cell_lane(m.nc);
    if (!cl.active) return;
    const int64_t nc = m.nc, c = cl.c;
    const int q = cl.q;
    const T Q0 = X[c * XS + q];
    T b0 = T(0), b1 = T(0), b2 = T(0);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int nb = m.nbr[f * nc + c];
        if (nb < 0) continue;
        const T dq = X[(int64_t)nb * XS + q] - Q0;
        b0 += m.M1[(0 * 4 + f) * nc + c] * dq;
        b1 += m.M1[(1 * 4 + f) * nc + c] * dq;
        b2 += m.M1[(2 * 4 + f) * nc + c] * dq;
    }
    T* out = slopes + c * 15 + 3 * q;
    out[0] = b0;
    out[1] = b1;
    out[2] = b2;
}

// P1 slope of cell x for component q (Sec. 4.3, reconstruction step 1):
// b = M1 (Q_nb - Q_x) over the existing neighbours
template <typename T>
__device__ __forceinline__ void p1_slope(const DevMesh<T>& m, const T* __restrict__ X, int64_t x, int q, T* b) {
    const int64_t nc = m.nc;
    const T Qx = X[x * XS + q];
    b[0] = b[1] = b[2] = T(0);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int nb = m.nbr[f * nc + x];
        if (nb < 0) continue;
        const T dq = X[(int64_t)nb * XS + q] - Qx;
        b[0] += m.M1[(0 * 4 + f) * nc + x] * dq;
        b[1] += m.M1[(1 * 4 + f) * nc + x] * dq;
        b[2] += m.M1[(2 * 4 + f) * nc + x] * dq;
    }
}

// reconstruction (Sec. 4.1-4.3): the cell's own P1 slopes and, for the
// two-step beta_0, its neighbours' P1 slopes (recomputed here, or read from
// a slopes pass); P2 = M2 d with the block's static data (M2, Gauss points,
// M1, moments) brought into shared memory by one bulk copy that overlaps the
// neighbour gathers;
// smoothness indicators, nonlinear weights, positivity at the cell's 12 face
// Gauss points (Sec. 4.2); R written about the centroid in monomial form
template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_recon(DevMesh<T> m, ReconConst<T> rc,
                                                         const T* __restrict__ X,
                                                         const T* __restrict__ slopes_in,
                                                         T* __restrict__ slopes_out,
                                                         T* __restrict__ poly,
                                                         int32_t* __restrict__ fallback,
                                                         FinArg<T> fin, int32_t* __restrict__ err) {
    __shared__ alignas(128) T sT[TILE_ROWS][CELLS_PER_BLOCK];
    __shared__ alignas(8) unsigned long long bar;
    constexpr unsigned TILE_BYTES = TILE_ROWS * CELLS_PER_BLOCK * sizeof(T);
    static_assert(TILE_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();  // the barrier exists before anyone waits on it
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, TILE_BYTES);
        bulk_load(&sT[0][0], m.tile + (int64_t)blockIdx.x * TILE_ROWS * CELLS_PER_BLOCK, TILE_BYTES, &bar);
    }
    if (fin.dtmin && blockIdx.x == 0) finalize_cases(fin.dtmin, fin.case_t, fin.case_dt, fin.ncase, fin.cfl, fin.ctrl);
    const int64_t nc = m.nc;
    const CellLane cl = cell_lane(nc);
    const int64_t c = cl.c;
    const int q = cl.q;
    const int lc = (int)(c - (int64_t)blockIdx.x * CELLS_PER_BLOCK) < CELLS_PER_BLOCK
                       ? (int)(c - (int64_t)blockIdx.x * CELLS_PER_BLOCK)
                       : CELLS_PER_BLOCK - 1;
    int nb[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) nb[f] = m.nbr[f * nc + c];
    const T Q0 = X[c * XS + q];

    // data vector [dQ_f (4); grad Q_{f,l} (12)] of this component
    T d[16];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const bool ok = nb[f] >= 0;
        const T* xn = X + (ok ? (int64_t)nb[f] : c) * XS;
        d[f] = ok ? xn[q] - Q0 : T(0);
#pragma unroll
        for (int l = 0; l < 3; ++l) d[4 + 3 * f + l] = ok ? xn[5 + 3 * q + l] : T(0);
    }
    // the tile has landed (all threads wait; a give-up is reported, and the
    // values computed from an incomplete tile are never trusted by the host)
    const bool tile_ok = mbar_wait(&bar, 0);
    if (!tile_ok && (threadIdx.x & 31) == 0) atomicOr(err, ERR_TIMEOUT);
    // P2 in the zero-mean basis of Eq. base: a = M2 d
    T a[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc += sT[TILE_M2 + k * 16 + j][lc] * d[j];
        a[k] = acc;
    }
    const T Mxx = sT[TILE_MOM + 0][lc], Mxy = sT[TILE_MOM + 1][lc], Mxz = sT[TILE_MOM + 2][lc];
    const T Myy = sT[TILE_MOM + 3][lc], Myz = sT[TILE_MOM + 4][lc], Mzz = sT[TILE_MOM + 5][lc];

    const T g22 = T(100.0 / 111.0), g12 = T(10.0 / 111.0), g02 = T(1.0 / 111.0);
    const T g11 = T(10.0 / 11.0), g01 = T(1.0 / 11.0);
    T R[9];
    T b[3] = {T(0), T(0), T(0)};
    if (rc.weno || rc.order == 2) {
        // own P1 slope from the neighbour differences already loaded
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (nb[f] < 0) continue;
            b[0] += sT[TILE_M1 + 0 * 4 + f][lc] * d[f];
            b[1] += sT[TILE_M1 + 1 * 4 + f][lc] * d[f];
            b[2] += sT[TILE_M1 + 2 * 4 + f][lc] * d[f];
        }
        if (slopes_out && cl.active) {
#pragma unroll
            for (int i = 0; i < 3; ++i) slopes_out[c * 15 + 3 * q + i] = b[i];
        }
    }
    if (!rc.weno) {
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = rc.order == 2 ? (k < 3 ? b[k] : T(0)) : a[k];
    } else {
        const T v23 = sT[TILE_V23][lc], v43 = sT[TILE_V43][lc];
        // smoothness indicators, Eq. smooth-indicator
        const T beta1 = v23 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        // two-step beta_0 from the neighbours' P1 slopes, Eq. p0-non-linear-weight
        T b0j[4];
        int nn = 0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (nb[f] < 0) continue;
            T bj[3];
            if (slopes_in) {
                const T* sj = slopes_in + (int64_t)nb[f] * 15 + 3 * q;
                bj[0] = sj[0];
                bj[1] = sj[1];
                bj[2] = sj[2];
            } else {
                p1_slope(m, X, nb[f], q, bj);
            }
            b0j[nn++] = v23 * (bj[0] * bj[0] + bj[1] * bj[1] + bj[2] * bj[2]);
        }
        T beta0 = T(0);
        if (nn > 0) {
            T sum = T(0);
            int npair = 0;
            for (int j = 0; j < nn; ++j)
                for (int k = 0; k < j; ++k) {
                    sum += d_abs(b0j[j] - b0j[k]);
                    ++npair;
                }
            const T s1 = npair ? pow43(sum / T(npair)) : T(0);
            T ws = T(0), acc = T(0);
            for (int j = 0; j < nn; ++j) {
                const T w1 = T(1) + s1 / (rc.eps + b0j[j]);
                ws += w1;
                acc += w1 * b0j[j];
            }
            beta0 = acc / ws;
        }
        if (rc.order == 2) {
            const T sigma = pow43(d_abs(beta1 - beta0));
            const T r0 = sigma / (rc.eps + beta0), r1 = sigma / (rc.eps + beta1);
            const T w0 = g01 * (T(1) + r0 * r0), w1 = g11 * (T(1) + r1 * r1);
            const T cl1 = (w1 / (w0 + w1)) / g11;
#pragma unroll
            for (int k = 0; k < 9; ++k) R[k] = k < 3 ? cl1 * b[k] : T(0);
        } else {
            // Hessian rows of P2 and the integrals of its derivatives
            const T H[3][3] = {{T(2) * a[3], a[4], a[5]}, {a[4], T(2) * a[6], a[7]}, {a[5], a[7], T(2) * a[8]}};
            T first = T(0);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const T h0 = H[l][0], h1 = H[l][1], h2 = H[l][2];
                const T hMh = h0 * (Mxx * h0 + Mxy * h1 + Mxz * h2) + h1 * (Mxy * h0 + Myy * h1 + Myz * h2) +
                              h2 * (Mxz * h0 + Myz * h1 + Mzz * h2);
                first += a[l] * a[l] + hMh;
            }
            const T second = H[0][0] * H[0][0] + a[4] * a[4] + a[5] * a[5] + H[1][1] * H[1][1] + a[7] * a[7] +
                             H[2][2] * H[2][2];
            const T beta2 = v23 * first + v43 * second;
            // global smoothness indicator and nonlinear weights, Eq. non-linear-weight
            const T sigma = pow43(T(0.5) * (d_abs(beta2 - beta1) + d_abs(beta2 - beta0)));
            const T r0 = sigma / (rc.eps + beta0), r1 = sigma / (rc.eps + beta1), r2 = sigma / (rc.eps + beta2);
            const T w0 = g02 * (T(1) + r0 * r0), w1 = g12 * (T(1) + r1 * r1), w2 = g22 * (T(1) + r2 * r2);
            const T iw = T(1) / (w0 + w1 + w2);
            const T c2 = (w2 * iw) / g22;
            const T cb = (w1 * iw) / g11 - c2 * g12 / g11;
#pragma unroll
            for (int k = 0; k < 9; ++k) R[k] = c2 * a[k] + (k < 3 ? cb * b[k] : T(0));
        }
    }
    // constant of the monomial form
    const T c0 = Q0 - (R[3] * Mxx + R[4] * Mxy + R[5] * Mxz + R[6] * Myy + R[7] * Myz + R[8] * Mzz);
    // positivity: the 5 lanes of the cell exchange their values at each point
    bool bad = false;
#pragma unroll 4
    for (int g = 0; g < 12; ++g) {
        const T gx = sT[TILE_G + g * 3 + 0][lc];
        const T gy = sT[TILE_G + g * 3 + 1][lc];
        const T gz = sT[TILE_G + g * 3 + 2][lc];
        const T v = c0 + R[0] * gx + R[1] * gy + R[2] * gz + R[3] * gx * gx + R[4] * gx * gy + R[5] * gx * gz +
                    R[6] * gy * gy + R[7] * gy * gz + R[8] * gz * gz;
        const T rho = __shfl_sync(0xffffffffu, v, cl.base + 0);
        const T m1 = __shfl_sync(0xffffffffu, v, cl.base + 1);
        const T m2 = __shfl_sync(0xffffffffu, v, cl.base + 2);
        const T m3 = __shfl_sync(0xffffffffu, v, cl.base + 3);
        const T en = __shfl_sync(0xffffffffu, v, cl.base + 4);
        const T pr = rc.gm1 * (en - T(0.5) * (m1 * m1 + m2 * m2 + m3 * m3) / rho);
        if (!(rho > T(0)) || !(pr > T(0))) bad = true;
    }
    if (!tile_ok) mbar_wait(&bar, 0);  // a late copy lands before the block exits
    if (!cl.active) return;
    T* out = poly + c * POLY_STRIDE + q * 10;
    out[0] = bad ? Q0 : c0;
#pragma unroll
    for (int k = 0; k < 9; ++k) out[1 + k] = bad ? T(0) : R[k];
    if (fallback && q == 0) fallback[c] = bad ? 1 : 0;
}

// --------------------------------------------------------------------------
// face flux
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void eval_poly(const T* __restrict__ P, const T* X, T* val, T (*g)[5]) {
    // the record is 16-byte aligned (POLY_STRIDE words): load it in vectors
    T c[POLY_STRIDE];
    if constexpr (sizeof(T) == 4) {
        const float4* p4 = reinterpret_cast<const float4*>(P);
#pragma unroll
        for (int i = 0; i < POLY_STRIDE / 4; ++i) {
            const float4 v = __ldg(p4 + i);
            c[4 * i] = v.x;
            c[4 * i + 1] = v.y;
            c[4 * i + 2] = v.z;
            c[4 * i + 3] = v.w;
        }
    } else {
        const double2* p2 = reinterpret_cast<const double2*>(P);
#pragma unroll
        for (int i = 0; i < POLY_STRIDE / 2; ++i) {
            const double2 v = __ldg(p2 + i);
            c[2 * i] = v.x;
            c[2 * i + 1] = v.y;
        }
    }
    const T x = X[0], y = X[1], z = X[2];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const T* cq = c + q * 10;
        val[q] = cq[0] + cq[1] * x + cq[2] * y + cq[3] * z + cq[4] * x * x + cq[5] * x * y + cq[6] * x * z +
                 cq[7] * y * y + cq[8] * y * z + cq[9] * z * z;
        g[0][q] = cq[1] + T(2) * cq[4] * x + cq[5] * y + cq[6] * z;
        g[1][q] = cq[2] + cq[5] * x + T(2) * cq[7] * y + cq[8] * z;
        g[2][q] = cq[3] + cq[6] * x + cq[8] * y + T(2) * cq[9] * z;
    }
}

// rows of the face frame: n, t1, t2 (Eq. rotate-matrix-3d; n1 = -1 uses the
// reflection diag(-1, -1, 1) of the velocity block)
template <typename T>
__device__ __forceinline__ void face_frame(const T* n, T (*Rm)[3]) {
    const T n1 = n[0], n2 = n[1], n3 = n[2];
    Rm[0][0] = n1;
    Rm[0][1] = n2;
    Rm[0][2] = n3;
    if (n1 == T(-1)) {
        Rm[1][0] = T(0); Rm[1][1] = T(-1); Rm[1][2] = T(0);
        Rm[2][0] = T(0); Rm[2][1] = T(0); Rm[2][2] = T(1);
        return;
    }
    const T r = T(1) / (T(1) + n1);
    Rm[1][0] = -n2;
    Rm[1][1] = n1 + n3 * n3 * r;
    Rm[1][2] = -n2 * n3 * r;
    Rm[2][0] = -n3;
    Rm[2][1] = -n2 * n3 * r;
    Rm[2][2] = T(1) - n3 * n3 * r;
}

template <typename T>
__device__ __forceinline__ void to_local(const T (*Rm)[3], const T* W, const T (*g)[5], T* Wt,
                                         T (*gt)[5]) {
    Wt[0] = W[0];
    Wt[4] = W[4];
#pragma unroll
    for (int j = 0; j < 3; ++j) Wt[1 + j] = Rm[j][0] * W[1] + Rm[j][1] * W[2] + Rm[j][2] * W[3];
    // directions first: h_j = sum_i R_ji g_i, then the momentum components
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T h[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) h[q] = Rm[j][0] * g[0][q] + Rm[j][1] * g[1][q] + Rm[j][2] * g[2][q];
        gt[j][0] = h[0];
        gt[j][4] = h[4];
#pragma unroll
        for (int k = 0; k < 3; ++k) gt[j][1 + k] = Rm[k][0] * h[1] + Rm[k][1] * h[2] + Rm[k][2] * h[3];
    }
}

// Slip-wall ghost (Sec. 4.4) of a state already in the face frame (x1 along
// the normal): the mirror image across the wall.  rho U1 changes sign; of the
// x1-derivatives all but that of rho U1 change sign; of the x2-, x3-derivatives
// only those of rho U1 do.
template <typename T>
__device__ __forceinline__ void slip_wall_ghost(T* Wt, T (*gt)[5]) {
    Wt[1] = -Wt[1];
    gt[0][0] = -gt[0][0];
    gt[0][2] = -gt[0][2];
    gt[0][3] = -gt[0][3];
    gt[0][4] = -gt[0][4];
    gt[1][1] = -gt[1][1];
    gt[2][1] = -gt[2][1];
}

// device encoding of a boundary face's missing side (flr): -1 - GKS_BC_*
constexpr int FLR_OPEN = -1, FLR_SLIP_WALL = -2, FLR_FIXED = -3;

// fixed boundary: the interior cell's fixed state (average and gradient)
// extended linearly to the point X (relative to the cell's centroid)
template <typename T>
__device__ __forceinline__ void fixed_ghost(const T* __restrict__ x0, const T* X, T* W, T (*g)[5]) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        T v = x0[q];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            g[i][q] = x0[5 + 3 * q + i];
            v += g[i][q] * X[i];
        }
        W[q] = v;
    }
}

template <typename T>
__device__ __forceinline__ void to_global(const T (*Rm)[3], T* v) {
    const T a = v[1], b = v[2], c = v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[1 + i] = Rm[0][i] * a + Rm[1][i] * b + Rm[2][i] * c;
}

// Face flux with 6 threads per face: 3 Gauss points x 2 sides.  The two sides
// of a Gauss point sit in different warps (warps 0-2 left, 3-5 right) so that
// no warp diverges on the side; the interface equilibrium, its slopes and the
// partial outputs are exchanged through shared memory:
//   phase 1  own side: state at the point, face frame, slopes, rho <psi>+-
//   phase 2  W^c, collision times; own kinetic part; rho <a_i psi>+-
//   phase 3  equilibrium slopes; left warps add the C2 (a^c.u) flux terms,
//            right warps the C1, C3 flux terms and the dW term
//   phase 4  left warps finish the flux entries, right warps the gradient
//            entries of the record; the 3 points of each face are summed.
constexpr int FP_GP = 3 * FLUX_FACES;  // Gauss points per block (96)

template <typename T, int NR>
struct FluxSmem {
    T w0[2][FP_GP][5];   // rho <psi>+- of each side
    T p[2][FP_GP];       // pressure of each side
    T dwc[2][FP_GP][15]; // rho <a_i psi>+- of each side
    T out[2][FP_GP][20]; // partial Fh, D, W0, dW of each side
    T red[FP_GP * NR];   // weighted record entries per Gauss point
};

template <typename T, int NR, int MINB>
__global__ void __launch_bounds__(2 * FP_GP, MINB) k_flux(DevMesh<T> m, Phys<T> ph,
                                                     const T* __restrict__ Wavg,
                                                     const T* __restrict__ poly,
                                                     T* __restrict__ rec,
                                                     const double* __restrict__ ctrl,
                                                     double dt_override) {
    __shared__ FluxSmem<T, NR> sm;
    const int side = threadIdx.x >= FP_GP ? 1 : 0;
    const int g = threadIdx.x - side * FP_GP;  // Gauss point within the block
    const int lf = g / 3;
    const int k = g - 3 * lf;
    const int64_t f0 = (int64_t)blockIdx.x * FLUX_FACES + lf;
    const bool active = f0 < m.nf;
    const int64_t f = active ? f0 : m.nf - 1;  // idle points compute a valid face, store nothing
    const int L = m.flr[f], Rc = m.flr[m.nf + f];
    // the face's case step; a finished case (dt = 0) computes with a dummy
    // step and its cells ignore the record
    const double dtc = ctrl ? ctrl[m.cell_case[L >= 0 ? L : Rc]] : dt_override;
    const T dt = dtc > 0.0 ? (T)dtc : T(1);
    const T* geo = m.fgeo + f * FGEO;
    const T n[3] = {geo[0], geo[1], geo[2]};
    const T w = geo[3];

    // ---- phase 1 ----
    const int mine = side == 0 ? L : Rc;
    const bool wall = mine == FLR_SLIP_WALL;
    T Ws[5], gs[3][5];
    if (mine >= 0 || wall) {
        // a wall side starts from the interior cell's value at the point
        const int src = mine >= 0 ? side : 1 - side;
        const int64_t cell = mine >= 0 ? mine : (side == 0 ? Rc : L);
        const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
        eval_poly(poly + cell * POLY_STRIDE, X, Ws, gs);
    } else if (mine == FLR_FIXED) {
        const int64_t in = side == 0 ? Rc : L;
        const int src = 1 - side;
        const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
        fixed_ghost(m.fixed + in * XS, X, Ws, gs);
    } else {
        // open boundary: the missing side is the interior cell's average with
        // zero gradient (zeroth-order extrapolation; the paper leaves outflow
        // boundaries open, and copying the interior Gauss-point state is not
        // stable)
        const int64_t in = side == 0 ? Rc : L;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            Ws[q] = Wavg[in * XS + q];
            gs[0][q] = gs[1][q] = gs[2][q] = T(0);
        }
    }
    T Rm[3][3];
    face_frame(n, Rm);
    T tW[5], tg[3][5];
    to_local(Rm, Ws, gs, tW, tg);
    if (wall) slip_wall_ghost(tW, tg);
    const Prim<T> S = to_prim(tW, ph.gm1);
    Tab<T> t;
    T a[3][5], A[5];
    kinetic_side(ph, S, tg, side == 0 ? +1 : -1, t, a, A);
    T mw0[5] = {T(0), T(0), T(0), T(0), T(0)};
    acc_psi<0, 0, 0>(t, S.rho, mw0);
#pragma unroll
    for (int q = 0; q < 5; ++q) sm.w0[side][g][q] = mw0[q];
    sm.p[side][g] = S.p;
    __syncthreads();

    // ---- phase 2 ----
    T Wc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Wc[q] = sm.w0[0][g][q] + sm.w0[1][g][q];
    const Prim<T> C = to_prim(Wc, ph.gm1);
    const TimeCoef<T> tc = time_coefs(ph, sm.p[0][g], sm.p[1][g], C.p, dt);
    const T tau = tc.tau;
    T Fh[5], D[5], W0[5], dWt[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Fh[q] = D[q] = W0[q] = dWt[q] = T(0);
    {
        T dwc[3][5];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int q = 0; q < 5; ++q) dwc[i][q] = T(0);
            acc_apsi<0, 0, 0>(t, a[i], S.rho, dwc[i]);
#pragma unroll
            for (int q = 0; q < 5; ++q) sm.dwc[side][g][5 * i + q] = dwc[i][q];
        }
    }
    if (!ph.smooth) {
        T mf0[5] = {0}, mf1[5] = {0}, mw1[5] = {0};
        acc_psi<1, 0, 0>(t, S.rho, mf0);
        acc_grad<1>(t, a, S.rho, mf1);
        acc_grad<0>(t, a, S.rho, mw1);
        axpy5(tc.k0, mf0, Fh);
        axpy5(-(tau * tc.k0 + tc.k1), mf1, Fh);
        axpy5(tc.dk0, mf0, D);
        axpy5(-(tau * tc.dk0 + tc.dk1), mf1, D);
        axpy5(T(1), mw0, W0);
        axpy5(-tau, mw1, W0);
        axpy5(tau - (tau + dt) * tc.E, mw1, dWt);
        if (ph.viscous) {
            T mf2[5] = {0}, mw2[5] = {0};
            acc_apsi<1, 0, 0>(t, A, S.rho, mf2);
            acc_apsi<0, 0, 0>(t, A, S.rho, mw2);
            axpy5(-tau * tc.k0, mf2, Fh);
            axpy5(-tau * tc.dk0, mf2, D);
            axpy5(-tau, mw2, W0);
            axpy5(tau * (T(1) - tc.E), mw2, dWt);
        }
    }
    __syncthreads();

    // ---- phase 3 ----
    {
        T dWc[3][5];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int q = 0; q < 5; ++q) dWc[i][q] = sm.dwc[0][g][5 * i + q] + sm.dwc[1][g][5 * i + q];
        make_tab(t, C, ph.K, 0);
        T ac[3][5], Ac[5];
        state_slopes(C, t, ph.K, dWc, ac, Ac);
        if (side == 0) {
            T mf1[5] = {T(0), T(0), T(0), T(0), T(0)};
            acc_grad<1>(t, ac, C.rho, mf1);
            if (ph.smooth) {
                axpy5(-tau * T(0.5) * dt, mf1, Fh);
            } else {
                axpy5(tc.q2, mf1, Fh);
                axpy5(tc.dq2, mf1, D);
            }
        } else {
            T mf0[5] = {0}, mf2[5] = {0}, mw1[5] = {0};
            acc_psi<1, 0, 0>(t, C.rho, mf0);
            acc_apsi<1, 0, 0>(t, Ac, C.rho, mf2);
            acc_grad<0>(t, ac, C.rho, mw1);  // rho <A^c psi> = -mw1 (Eq. co)
            if (ph.smooth) {
                const T hd = T(0.5) * dt;
                axpy5(hd, mf0, Fh);
                axpy5(T(0.5) * hd * hd - tau * hd, mf2, Fh);
                axpy5(T(0.25) * dt * dt, mf2, D);
#pragma unroll
                for (int q = 0; q < 5; ++q) W0[q] = Wc[q];  // tau terms cancel: <(a.u + A) psi> = 0
                axpy5(-dt, mw1, dWt);
            } else {
                axpy5(tc.q1, mf0, Fh);
                axpy5(tc.q3, mf2, Fh);
                axpy5(tc.dq1, mf0, D);
                axpy5(tc.dq3, mf2, D);
                const T C2 = (dt + tau) * tc.E - tau, C3 = dt - tau + tau * tc.E;
                axpy5(C2 - C3, mw1, dWt);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        sm.out[side][g][q] = Fh[q];
        sm.out[side][g][5 + q] = D[q];
        sm.out[side][g][10 + q] = W0[q];
        sm.out[side][g][15 + q] = dWt[q];
    }
    __syncthreads();

    // ---- phase 4: left warps the flux entries, right warps the gradient entries
    T* mine_rec = sm.red + g * NR;
    if (side == 0) {
        T Fs[5], Ds[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            Fs[q] = sm.out[0][g][q] + sm.out[1][g][q];
            Ds[q] = sm.out[0][g][5 + q] + sm.out[1][g][5 + q];
        }
        to_global(Rm, Fs);
        to_global(Rm, Ds);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (NR == 40) {
                // dt L + dt^2/6 L_t = 8/3 Fh - 1/3 F = 2 Fh - D / 3 (Eqs. linear-system, s2o4)
                mine_rec[q] = w * Fs[q];
                mine_rec[5 + q] = w * (T(2) * Fs[q] - Ds[q] * T(1.0 / 3.0));
            } else {
                mine_rec[q] = w * T(4.0 / 3.0) * Ds[q];  // dt^2/3 L_t(W*) = 4/3 (F* - 2 Fh*)
            }
        }
    } else {
        T Zs[5], Ys[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            Zs[q] = sm.out[0][g][10 + q] + sm.out[1][g][10 + q];
            Ys[q] = sm.out[0][g][15 + q] + sm.out[1][g][15 + q];
        }
        to_global(Rm, Zs);
        to_global(Rm, Ys);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (NR == 40) {
                const T ws = w * (Zs[q] + T(0.5) * Ys[q]);  // f* = f^n + dt/2 f_t^n
                const T w0 = w * Zs[q];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    mine_rec[10 + 3 * q + i] = ws * n[i];
                    mine_rec[25 + 3 * q + i] = w0 * n[i];
                }
            } else {
                const T dg = w * Ys[q];  // f^{n+1} = f^n + dt f_t^*
#pragma unroll
                for (int i = 0; i < 3; ++i) mine_rec[5 + 3 * q + i] = dg * n[i];
            }
        }
    }
    __syncthreads();
    // sum the three Gauss points of each face; coalesced record store
    const int64_t base = (int64_t)blockIdx.x * FLUX_FACES;
    for (int idx = threadIdx.x; idx < FLUX_FACES * NR; idx += 2 * FP_GP) {
        const int fl = idx / NR, j = idx - fl * NR;
        if (base + fl < m.nf) {
            const T* r = sm.red + fl * 3 * NR + j;
            rec[(base + fl) * NR + j] = (r[0] + r[NR]) + r[2 * NR];
        }
    }
}

// 3 threads per face, one Gauss point each (used for FP64, whose register
// footprint leaves no room for the lane-pair split)
template <typename T, int NR>
__global__ void __launch_bounds__(3 * FLUX_FACES) k_flux_single(DevMesh<T> m, Phys<T> ph,
                                                                 const T* __restrict__ Wavg,
                                                                 const T* __restrict__ poly,
                                                                 T* __restrict__ rec,
                                                                 const double* __restrict__ ctrl,
                                                                 double dt_override) {
    __shared__ T red[FLUX_FACES * 3 * NR];
    const int lf = threadIdx.x / 3;
    const int k = threadIdx.x - 3 * lf;
    const int64_t f = (int64_t)blockIdx.x * FLUX_FACES + lf;
    T* mine = red + (lf * 3 + k) * NR;
    if (f < m.nf) {
        const int L = m.flr[f], Rc = m.flr[m.nf + f];
        const double dtc = ctrl ? ctrl[m.cell_case[L >= 0 ? L : Rc]] : dt_override;
        const T dt = dtc > 0.0 ? (T)dtc : T(1);
        const T* geo = m.fgeo + f * FGEO;
        const T n[3] = {geo[0], geo[1], geo[2]};
        const T w = geo[3];
        T WL[5], gL[3][5], WR[5], gR[3][5];
        for (int side = 0; side < 2; ++side) {
            const int cell = side == 0 ? L : Rc;
            T* Wv = side == 0 ? WL : WR;
            T (*g)[5] = side == 0 ? gL : gR;
            if (cell >= 0 || cell == FLR_SLIP_WALL) {
                // a wall side starts from the interior cell's value at the point
                const int src = cell >= 0 ? side : 1 - side;
                const int64_t c = cell >= 0 ? cell : (side == 0 ? Rc : L);
                const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
                eval_poly(poly + c * POLY_STRIDE, X, Wv, g);
            } else if (cell == FLR_FIXED) {
                const int64_t in = side == 0 ? Rc : L;
                const int src = 1 - side;
                const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
                fixed_ghost(m.fixed + in * XS, X, Wv, g);
            } else {
                // open boundary: interior cell average, zero gradient
                const int64_t in = side == 0 ? Rc : L;
                for (int q = 0; q < 5; ++q) {
                    Wv[q] = Wavg[in * XS + q];
                    g[0][q] = g[1][q] = g[2][q] = T(0);
                }
            }
        }
        T Rm[3][3];
        face_frame(n, Rm);
        T tWL[5], tgL[3][5], tWR[5], tgR[3][5];
        to_local(Rm, WL, gL, tWL, tgL);
        to_local(Rm, WR, gR, tWR, tgR);
        if (L == FLR_SLIP_WALL) slip_wall_ghost(tWL, tgL);
        if (Rc == FLR_SLIP_WALL) slip_wall_ghost(tWR, tgR);
        T Fh[5], D[5], W0[5], dWt[5];
        gks_point(ph, tWL, tgL, tWR, tgR, dt, Fh, D, W0, dWt);
        to_global(Rm, Fh);
        to_global(Rm, D);
        to_global(Rm, W0);
        to_global(Rm, dWt);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (NR == 40) {
                mine[q] = w * Fh[q];
                mine[5 + q] = w * (T(2) * Fh[q] - D[q] * T(1.0 / 3.0));
                const T ws = w * (W0[q] + T(0.5) * dWt[q]);
                const T w0 = w * W0[q];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    mine[10 + 3 * q + i] = ws * n[i];
                    mine[25 + 3 * q + i] = w0 * n[i];
                }
            } else {
                mine[q] = w * T(4.0 / 3.0) * D[q];
                const T dg = w * dWt[q];
#pragma unroll
                for (int i = 0; i < 3; ++i) mine[5 + 3 * q + i] = dg * n[i];
            }
        }
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * FLUX_FACES;
    for (int idx = threadIdx.x; idx < FLUX_FACES * NR; idx += 3 * FLUX_FACES) {
        const int fl = idx / NR, j = idx - fl * NR;
        if (base + fl < m.nf) {
            const T* r = red + fl * 3 * NR + j;
            rec[(base + fl) * NR + j] = (r[0] + r[NR]) + r[2 * NR];
        }
    }
}

// --------------------------------------------------------------------------
// cell updates (5 lanes per cell)
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_update1(DevMesh<T> m, DevState<T> st) {
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
    for (int f = 0; f < 4; ++f) {
        const int e = m.cface[f * nc + c];
        const T s = (e & 1) ? T(-1) : T(1);
        const T* r = st.rec + (int64_t)(e >> 1) * 40;
        fh.add(s * r[q]);
        s1.add(s * r[5 + q]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gs[i] += s * r[10 + 3 * q + i];
            g0[i] += s * r[25 + 3 * q + i];
        }
    }
    const double iv = m.inv_vol[c];
    T* xs = st.Xs + c * XS;
    // W* = W^n - (1/|Omega|) sum s sum_k w Fh  (Eq. s2o4, first stage)
    xs[q] = (T)(st.Wd[q * nc + c] - fh.value() * iv);
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
        T* x = st.X + c * XS;
        x[q] = Wq;
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
        for (int q = 0; q < 5; ++q) Wv[q] = X[cl.c * XS + q];
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
        for (int q = 0; q < 5; ++q) Wv[q] = X[cl.c * XS + q];
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

template <typename T>
__global__ void k_pack(const double* __restrict__ W, const double* __restrict__ dW, T* __restrict__ X, int64_t nc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc * XS; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / XS;
        const int j = (int)(i - c * XS);
        X[i] = (T)(j < 5 ? W[j * nc + c] : dW[(j - 5) * nc + c]);
    }
}

template <typename T>
__global__ void k_unpack_grad(const T* __restrict__ X, double* __restrict__ dW, int64_t nc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc * 15; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / nc, c = i - j * nc;
        dW[i] = (double)X[c * XS + 5 + j];
    }
}

template <typename T>
__global__ void k_rec_out(const T* __restrict__ rec, const int32_t* __restrict__ perm, double* __restrict__ out,
                          int64_t nf, int nr) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf * nr; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = i / nr;
        out[(int64_t)perm[d] * nr + (i - d * nr)] = (double)rec[i];
    }
}

template <typename T>
__global__ void k_poly_out(const T* __restrict__ in, double* __restrict__ out, int64_t nc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc * 50; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[(i / 50) * POLY_STRIDE + i % 50];
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
static inline unsigned cell_grid(int64_t nc) { return (unsigned)((nc + CELLS_PER_BLOCK - 1) / CELLS_PER_BLOCK); }

int update_blocks(int64_t nc) { return (int)cell_grid(nc); }

template <typename T>
static Phys<T> make_phys(const HostPhys& p) {
    Phys<T> ph;
    ph.gamma = (T)p.gamma;
    ph.gm1 = (T)(p.gamma - 1.0);
    ph.K = (T)((5.0 - 3.0 * p.gamma) / (p.gamma - 1.0));
    ph.tau_eps = (T)p.tau_eps;
    ph.tau_c = (T)p.tau_c;
    ph.mu = (T)p.mu;
    ph.eps_w = (T)p.eps_weno;
    ph.viscous = p.viscous;
    ph.smooth = p.smooth;
    return ph;
}

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
    k_slopes<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, X, slopes, fin_arg<T>(fin));
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
    k_recon<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, rc, X, slopes_in, slopes, poly, fallback, fin_arg<T>(fin),
                                                        err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::flux(const DevMesh<T>& m, const HostPhys& p, const T* W, const T* poly, T* rec,
                            const double* ctrl, double dt_override, int stage, cudaStream_t s, int variant) {
    // ctrl is the per-case step array (NULL: dt_override everywhere)
    if (m.nf == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((m.nf + FLUX_FACES - 1) / FLUX_FACES);
    const Phys<T> ph = make_phys<T>(p);
    if constexpr (sizeof(T) == 4) {
        // FP32: the two sides of each Gauss point in separate warps; variant
        // 1 trades registers for occupancy (3 blocks per SM), variant 0 keeps
        // 2 blocks per SM without spills
        if (variant == 1) {
            if (stage == 1)
                k_flux<T, 40, 3><<<grid, 2 * FP_GP, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
            else
                k_flux<T, 20, 3><<<grid, 2 * FP_GP, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
        } else {
            if (stage == 1)
                k_flux<T, 40, 2><<<grid, 2 * FP_GP, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
            else
                k_flux<T, 20, 2><<<grid, 2 * FP_GP, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
        }
    } else {
        if (stage == 1)
            k_flux_single<T, 40><<<grid, 3 * FLUX_FACES, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
        else
            k_flux_single<T, 20><<<grid, 3 * FLUX_FACES, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::update1(const DevMesh<T>& m, const DevState<T>& st, cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    k_update1<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, st);
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
cudaError_t Launch<T>::pack(const double* W, const double* dW, T* X, int64_t nc, cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    k_pack<T><<<ew_grid(nc * XS), 256, 0, s>>>(W, dW, X, nc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::unpack_grad(const T* X, double* dW, int64_t nc, cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    k_unpack_grad<T><<<ew_grid(nc * 15), 256, 0, s>>>(X, dW, nc);
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
                                     cudaStream_t s) {
    if (nf == 0) return cudaSuccess;
    const int64_t n = nf * nr;
    k_rec_out<T><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(rec, perm, out, nf, nr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::poly_to_double(const T* in, double* out, int64_t nc, cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    const int64_t n = nc * 50;
    k_poly_out<T><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(in, out, nc);
    return cudaGetLastError();
}

cudaError_t launch_set_control(double* ctrl, double* case_t, double* case_dt, unsigned long long* case_dtmin,
                               int32_t ncase, double dt_fixed, double t_end, int reset_time, cudaStream_t s) {
    const int grid = reset_time ? (int)((ncase + 255) / 256 < 1024 ? (ncase + 255) / 256 : 1024) : 1;
    k_set_control<<<grid < 1 ? 1 : grid, 256, 0, s>>>(ctrl, case_t, case_dt, case_dtmin, ncase, dt_fixed,
                                                      t_end, reset_time);
    return cudaGetLastError();
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace gks
