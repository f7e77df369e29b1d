// gks_update.cuh -- the cell updates of one block of cells (Sec. 3) and the
// block reductions of the time-step rule (Sec. 5), shared by the
// standalone kernels and the persistent stage kernel.
#pragma once

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
__device__ inline void block_case_min(double v, int32_t cas, bool valid, int lc, unsigned long long* dtmin,
                               const CellGroup& grp) {
    double* sv = grp.sv;
    int32_t* sc = grp.sc;
    if (grp.tid < CELLS_PER_BLOCK) sc[grp.tid] = -1;
    grp.sync();
    if (valid) {
        sv[lc] = v;
        sc[lc] = cas;
    }
    grp.sync();
    if (grp.tid == 0) {
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
__device__ __forceinline__ void update1_cells(const DevMesh<T>& m, const HostPhys& p, const DevState<T>& st,
                                              int64_t vb, int tid) {
    const CellLane cl = cell_lane(m.nc, vb, tid);
    if (!cl.active) return;
    const int64_t nc = m.nc, c = cl.c;
    if (!(st.case_dt[m.cell_case[c]] > 0.0)) return;  // finished case
    const int q = cl.q;
    CSum<T> fh, s1;
    fh.init();
    s1.init();
    T gs[3] = {T(0), T(0), T(0)}, g0[3] = {T(0), T(0), T(0)};
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
__device__ __forceinline__ void block_reduce_part(R mn, const R* sums, double* out, const CellGroup& grp) {
    double (*red)[6] = reinterpret_cast<double (*)[6]>(grp.red);  // R values, held exactly
    R v[6] = {mn, sums[0], sums[1], sums[2], sums[3], sums[4]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmin(v[0], __shfl_down_sync(0xffffffffu, v[0], o));
#pragma unroll
        for (int k = 1; k < 6; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    const int warp = grp.tid >> 5;
    if ((grp.tid & 31) == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) red[warp][k] = (double)v[k];
    grp.sync();
    if (grp.tid == 0) {
        R r[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = (R)red[0][k];
        for (int w = 1; w < CELL_THREADS / 32; ++w) {
            r[0] = fmin(r[0], (R)red[w][0]);
#pragma unroll
            for (int k = 1; k < 6; ++k) r[k] += red[w][k];
        }
        out[PART_DTMIN] = (double)r[0];
#pragma unroll
        for (int q = 0; q < 5; ++q) out[PART_RES + q] = (double)r[1 + q];
    }
}

template <typename T>
__device__ __forceinline__ void update2_cells(const DevMesh<T>& m, const HostPhys& p, const DevState<T>& st,
                                              const CellGroup& grp) {
    const CellLane cl = cell_lane(m.nc, grp.vb, grp.tid);
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
    const int lc = (int)(c - grp.vb * CELLS_PER_BLOCK);
    block_case_min((double)mn, cas, lead && lc >= 0 && lc < CELLS_PER_BLOCK && mn < T(INFINITY), lc, st.case_dtmin,
                   grp);
    T mn_unused = T(INFINITY);
    block_reduce_part<T>(mn_unused, res, st.part + grp.vb * PART_N, grp);
}

}  // namespace gks
