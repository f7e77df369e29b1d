// gks_stage.cu -- one stage of the FP32-bulk step (reconstruction, face flux,
// cell update: Sec. 3-4) as a single persistent launch, sm_103a.
//
// One block of 384 threads per SM runs the stage's three phases over the
// whole (batched) mesh: the reconstruction as three groups of 128 threads
// on blocks of 24 cells, the face flux as two groups of 192 threads on
// blocks of 32 faces, the cell update as three groups of 128 threads, each
// group striding over its blocks; the phases are separated by grid-wide
// barriers.  It is the same per-block source as the standalone kernels (the
// numbers agree to FP32 rounding: the compiler may contract a few operations
// differently here); what it saves is the launches and the tails between
// the phases.  A grid barrier waits a bounded number of polls: if
// it gives up (not every block resident), the launch sets ERR_TIMEOUT and
// finishes; the host reports GKS_E_TIMEOUT.
#include <cuda_runtime.h>

#include "gks_flux.cuh"
#include "gks_recon.cuh"
#include "gks_update.cuh"

namespace gks {

constexpr int STAGE_THREADS = 384;  // 3 cell groups of 128 = 2 flux groups of 192
constexpr int CELL_GROUPS = STAGE_THREADS / CELL_THREADS, FLUX_GROUPS = STAGE_THREADS / (2 * FP_GP);
static_assert(CELL_GROUPS * CELL_THREADS == STAGE_THREADS && FLUX_GROUPS * 2 * FP_GP == STAGE_THREADS,
              "the stage block holds whole cell and flux groups");
// named barriers: flux side pairs 1-6, flux groups 7-8, cell groups 9-11
constexpr int BAR_FLUX_PAIRS = 1, BAR_FLUX_GROUP = 7, BAR_CELL_GROUP = 9;
// bounded grid-barrier wait: polls with a short sleep, about a second in all
constexpr int GRID_TRIES = 1 << 23;

// Bounded grid-wide barrier: the last block to arrive resets the count and
// advances the generation the others wait on.  Returns false (and sets
// ERR_TIMEOUT) if this block gave up waiting after `limit` polls.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, int32_t* err, int limit = GRID_TRIES) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = gen;
        const unsigned g0 = *vgen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(count, 1u) + 1u == gridDim.x) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            for (int tries = 0; *vgen == g0; ++tries) {
                if (tries >= limit) {
                    ok = 0;
                    atomicOr(err, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// The grid barrier's failure path without a fault: the count word starts
// far from the value the last arrival would make it equal to the grid size,
// so no block releases the others; each polls `limit` times, gives up, sets
// ERR_TIMEOUT and returns.  Nothing else is touched.
__global__ void k_grid_barrier_probe(unsigned* gbar, int32_t* err, int limit) {
    grid_barrier(gbar, gbar + 1, err, limit);
}

cudaError_t launch_grid_barrier_probe(unsigned* gbar, int32_t* err, int limit, cudaStream_t s) {
    // count = generation = 0x80808080: two arrivals bring the count to
    // 0x80808082, never to the grid size 2
    cudaError_t e = cudaMemsetAsync(gbar, 0x80, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_grid_barrier_probe<<<2, 32, 0, s>>>(gbar, err, limit);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemsetAsync(gbar, 0, 2 * sizeof(unsigned), s);
}

template <int NR>
constexpr size_t stage_smem_bytes() {
    const size_t recon = CELL_GROUPS * sizeof(Tile<float>) + CELL_GROUPS * sizeof(unsigned long long);
    const size_t flux = FLUX_GROUPS * sizeof(FluxSmem<float, NR>);
    const size_t upd = CELL_GROUPS * (2 * CELLS_PER_BLOCK + CELL_THREADS / 32 * 6) * sizeof(double);
    return recon > flux ? (recon > upd ? recon : upd) : (flux > upd ? flux : upd);
}

template <int STAGE, bool PRF>
__global__ void __launch_bounds__(STAGE_THREADS, 1)
    k_stage(DevMesh<float> m, Phys<float> ph, HostPhys hp, ReconConst<float> rc, DevState<float> st,
            FinArg<float> fin, unsigned* gbar) {
    constexpr int NR = STAGE == 1 ? 40 : 20;
    extern __shared__ __align__(128) unsigned char smem[];
    const float* X = STAGE == 1 ? st.X : st.Xs;
    const int64_t ncb = (m.nc + CELLS_PER_BLOCK - 1) / CELLS_PER_BLOCK;
    const int64_t nfb = (m.nf + FLUX_FACES - 1) / FLUX_FACES;
    if (STAGE == 1 && fin.dtmin && blockIdx.x == 0)
        finalize_cases(fin.dtmin, fin.case_t, fin.case_dt, fin.ncase, fin.cfl, fin.ctrl);

    // ---- reconstruction (Sec. 4.1-4.3)
    {
        const int grp = threadIdx.x / CELL_THREADS, tid = threadIdx.x % CELL_THREADS;
        Tile<float>* tiles = reinterpret_cast<Tile<float>*>(smem);
        unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + CELL_GROUPS * sizeof(Tile<float>));
        if (tid == 0) mbar_init(&bars[grp], 1);
        __syncthreads();
        unsigned parity = 0;
        for (int64_t vb = (int64_t)blockIdx.x * CELL_GROUPS + grp; vb < ncb; vb += (int64_t)gridDim.x * CELL_GROUPS) {
            recon_cells<float, float, true>(m, rc, X, nullptr, nullptr, st.poly, nullptr, st.err, vb, tid, tiles[grp],
                                      &bars[grp], parity);
            parity ^= 1u;
            group_barrier(BAR_CELL_GROUP + grp, CELL_THREADS);  // the tile is free for the next copy
        }
        if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&bars[grp])) : "memory");
    }
    grid_barrier(gbar, gbar + 1, st.err);

    // ---- face flux and records (Sec. 2.2, 3, 4.4, 4.5)
    {
        const int grp = threadIdx.x / (2 * FP_GP), tid = threadIdx.x % (2 * FP_GP);
        FluxSmem<float, NR>* fs = reinterpret_cast<FluxSmem<float, NR>*>(smem);
        for (int64_t fb = (int64_t)blockIdx.x * FLUX_GROUPS + grp; fb < nfb; fb += (int64_t)gridDim.x * FLUX_GROUPS) {
            flux_faces<float, NR, PRF>(m, ph, X, st.poly, st.rec, st.case_dt, 0.0, fb, tid, fs[grp],
                                       BAR_FLUX_PAIRS + 3 * grp, BAR_FLUX_GROUP + grp);
            group_barrier(BAR_FLUX_GROUP + grp, 2 * FP_GP);  // shared memory free for the next block
        }
    }
    grid_barrier(gbar, gbar + 1, st.err);

    // ---- cell update (Sec. 3, Eq. s2o4)
    {
        const int grp = threadIdx.x / CELL_THREADS, tid = threadIdx.x % CELL_THREADS;
        double* base = reinterpret_cast<double*>(smem) + grp * (2 * CELLS_PER_BLOCK + CELL_THREADS / 32 * 6);
        for (int64_t vb = (int64_t)blockIdx.x * CELL_GROUPS + grp; vb < ncb; vb += (int64_t)gridDim.x * CELL_GROUPS) {
            if (STAGE == 1) {
                update1_cells<float>(m, hp, st, vb, tid);
            } else {
                const CellGroup cg{vb, tid, BAR_CELL_GROUP + grp, base, reinterpret_cast<int32_t*>(base + CELLS_PER_BLOCK),
                                   base + 2 * CELLS_PER_BLOCK};
                update2_cells<float>(m, hp, st, cg);
            }
            group_barrier(BAR_CELL_GROUP + grp, CELL_THREADS);
        }
    }
}

template <int STAGE, bool PRF>
static cudaError_t launch_stage_kernel(const DevMesh<float>& m, const Phys<float>& ph, const HostPhys& hp,
                                       const ReconConst<float>& rc, const DevState<float>& st,
                                       const FinArg<float>& fin, unsigned* gbar, cudaStream_t s) {
    constexpr size_t smem = stage_smem_bytes<STAGE == 1 ? 40 : 20>();
    auto kern = k_stage<STAGE, PRF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, STAGE_THREADS, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // every block resident at once: one wave of the SMs
    const int64_t ncb = (m.nc + CELLS_PER_BLOCK - 1) / CELLS_PER_BLOCK;
    int64_t want = (ncb + CELL_GROUPS - 1) / CELL_GROUPS;
    const int64_t full = (int64_t)per_sm * nsm;
    const unsigned grid = (unsigned)(want < full ? (want < 1 ? 1 : want) : full);
    if ((e = cudaMemsetAsync(gbar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(STAGE_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, m, ph, hp, rc, st, fin, gbar);
}

cudaError_t launch_stage(const DevMesh<float>& m, const HostPhys& p, const DevState<float>& st, int stage,
                         const Launch<float>::Finalize* fin, unsigned* gbar, cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    Phys<float> ph;
    ph.gamma = (float)p.gamma;
    ph.gm1 = (float)(p.gamma - 1.0);
    ph.K = (float)((5.0 - 3.0 * p.gamma) / (p.gamma - 1.0));
    ph.tau_eps = (float)p.tau_eps;
    ph.tau_c = (float)p.tau_c;
    ph.mu = (float)p.mu;
    ph.eps_w = (float)p.eps_weno;
    ph.viscous = p.viscous;
    ph.smooth = p.smooth;
    ph.prf = (float)p.prf;
    ph.twall = (float)p.twall;
    for (int i = 0; i < 3; ++i) ph.uwall[i] = (float)p.uwall[i];
    ReconConst<float> rc;
    rc.gm1 = (float)(p.gamma - 1.0);
    rc.eps = (float)p.eps_weno;
    rc.weno = p.weno;
    rc.order = p.order;
    FinArg<float> fa{};
    if (fin) {
        fa.dtmin = fin->dtmin;
        fa.case_t = fin->case_t;
        fa.case_dt = fin->case_dt;
        fa.ncase = fin->ncase;
        fa.cfl = fin->cfl;
        fa.ctrl = fin->ctrl;
    }
    const bool prf = p.prf != 0.0;
    if (stage == 1)
        return prf ? launch_stage_kernel<1, true>(m, ph, p, rc, st, fa, gbar, s)
                   : launch_stage_kernel<1, false>(m, ph, p, rc, st, fa, gbar, s);
    return prf ? launch_stage_kernel<2, true>(m, ph, p, rc, st, fa, gbar, s)
               : launch_stage_kernel<2, false>(m, ph, p, rc, st, fa, gbar, s);
}

}  // namespace gks
