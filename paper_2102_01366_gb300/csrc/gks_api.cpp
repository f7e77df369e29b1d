// gks_api.cpp -- the extern "C" entry points of libgks (include/gks.h).
//
// Host objects: gks_mesh (connectivity, FP64 geometry and stencils) and
// gks_state (views into one caller-allocated device workspace, the stream,
// and the CUDA graph of one step).  Device storage is laid out once by
// layout_workspace(); nothing here allocates device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gks_internal.h"
#include "gks_kernels.h"

namespace gks {
namespace {
thread_local std::string g_err;
}
void set_error(const std::string& msg) { g_err = msg; }
}  // namespace gks

using namespace gks;

#define GKS_CHECK_CUDA(call)                                                        \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
            return GKS_E_CUDA;                                                      \
        }                                                                           \
    } while (0)

extern "C" const char* gks_last_error(void) { return g_err.c_str(); }

extern "C" void gks_params_default(gks_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->gamma = 1.4;
    p->cfl = 1.0;
    p->mu = 0.0;
    p->eps_weno = 1e-8;
    p->tau_eps = 0.01;
    p->tau_c = 1.0;
    p->prandtl = 1.0;
    p->wall_temperature = 1.0;
    p->weno = 1;
    p->order = 3;
    p->smooth_flux = 0;
    p->viscous = 0;
    p->precision = 0;
}

static gks_status check_params(const gks_params* p) {
    if (!p) { set_error("params is NULL"); return GKS_E_ARG; }
    if (!(p->gamma > 1.0 && p->gamma < 5.0 / 3.0 + 1e-12)) {
        set_error("gamma must lie in (1, 5/3]");
        return GKS_E_ARG;
    }
    if (!(p->cfl > 0.0) || !(p->eps_weno > 0.0) || !(p->tau_eps >= 0.0) || !(p->tau_c >= 0.0) ||
        !(p->mu >= 0.0) || !(p->prandtl > 0.0) || !(p->wall_temperature > 0.0)) {
        set_error("cfl, eps_weno, prandtl, wall_temperature must be positive; tau_eps, tau_c, mu non-negative");
        return GKS_E_ARG;
    }
    if ((p->weno != 0 && p->weno != 1) || (p->order != 2 && p->order != 3) ||
        (p->smooth_flux != 0 && p->smooth_flux != 1) || (p->viscous != 0 && p->viscous != 1) ||
        (p->precision < 0 || p->precision > 2) || (p->wall_constraint != 0 && p->wall_constraint != 1)) {
        set_error("weno, smooth_flux, viscous, wall_constraint must be 0 or 1; precision 0, 1 or 2; order 2 or 3");
        return GKS_E_ARG;
    }
    if (p->viscous && !(p->mu > 0.0)) {
        set_error("viscous flow needs mu > 0");
        return GKS_E_ARG;
    }
    if (!p->viscous && !(p->tau_eps > 0.0)) {
        set_error("inviscid flow needs tau_eps > 0 (numerical collision time)");
        return GKS_E_ARG;
    }
    return GKS_OK;
}

// ------------------------------------------------------------------ mesh --

extern "C" gks_status gks_mesh_create_cases(const double* xyz, int64_t n_vert, const int64_t* tet,
                                            const int8_t* shift, int64_t n_cell, const int32_t* tet_case,
                                            int32_t n_case, const double* period, gks_mesh** out) {
    if (!out) { set_error("gks_mesh_create: out is NULL"); return GKS_E_ARG; }
    *out = nullptr;
    if (!xyz || !tet || n_vert <= 0 || n_cell <= 0 || n_case < 1 || (n_case > 1 && !tet_case)) {
        set_error("gks_mesh_create: empty mesh, NULL arrays or bad case count");
        return GKS_E_ARG;
    }
    if (n_cell >= ((int64_t)1 << 30) || n_vert >= ((int64_t)1 << 40) || n_case > (1 << 24)) {
        set_error("gks_mesh_create: mesh too large (cells and faces are indexed by int32)");
        return GKS_E_ARG;
    }
    gks_mesh* m = new (std::nothrow) gks_mesh();
    if (!m) { set_error("out of memory"); return GKS_E_NOMEM; }
    try {
        m->nv = n_vert;
        m->nc = n_cell;
        m->ncase = n_case;
        m->period.assign((size_t)n_case * 3, 0.0);
        if (period) m->period.assign(period, period + (size_t)n_case * 3);
        for (double v : m->period)
            if (!(v >= 0.0)) {
                set_error("gks_mesh_create: negative period");
                delete m;
                return GKS_E_ARG;
            }
        m->cell_case.assign((size_t)n_cell, 0);
        if (tet_case) {
            for (int64_t c = 0; c < n_cell; ++c) {
                if (tet_case[c] < 0 || tet_case[c] >= n_case) {
                    set_error("gks_mesh_create: case id out of range");
                    delete m;
                    return GKS_E_ARG;
                }
                if (c > 0 && tet_case[c] < tet_case[c - 1]) {
                    set_error("gks_mesh_create: cells must be grouped by ascending case id");
                    delete m;
                    return GKS_E_ARG;
                }
                m->cell_case[c] = tet_case[c];
            }
        }
        m->xyz.assign(xyz, xyz + n_vert * 3);
        m->tet.assign(tet, tet + n_cell * 4);
        if (shift) m->shift.assign(shift, shift + n_cell * 12);
        else m->shift.assign((size_t)n_cell * 12, 0);
        for (int64_t i = 0; i < n_cell * 4; ++i)
            if (tet[i] < 0 || tet[i] >= n_vert) {
                set_error("gks_mesh_create: vertex id out of range");
                delete m;
                return GKS_E_MESH;
            }
        gks_status st = build_mesh(*m);
        if (st != GKS_OK) { delete m; return st; }
        if (m->nf >= ((int64_t)1 << 30)) {
            set_error("gks_mesh_create: too many faces");
            delete m;
            return GKS_E_ARG;
        }
    } catch (const std::bad_alloc&) {
        delete m;
        set_error("out of memory");
        return GKS_E_NOMEM;
    }
    *out = m;
    return GKS_OK;
}

extern "C" gks_status gks_mesh_create(const double* xyz, int64_t n_vert, const int64_t* tet,
                                      const int8_t* shift, int64_t n_cell, const double* period,
                                      gks_mesh** out) {
    return gks_mesh_create_cases(xyz, n_vert, tet, shift, n_cell, nullptr, 1, period, out);
}

extern "C" void gks_mesh_destroy(gks_mesh* mesh) { delete mesh; }

extern "C" gks_status gks_mesh_info(const gks_mesh* m, int64_t* n_cell, int64_t* n_face,
                                    int64_t* n_boundary_face) {
    if (!m) { set_error("mesh is NULL"); return GKS_E_ARG; }
    if (n_cell) *n_cell = m->nc;
    if (n_face) *n_face = m->nf;
    if (n_boundary_face) *n_boundary_face = m->nbf;
    return GKS_OK;
}

extern "C" gks_status gks_mesh_set_boundary(gks_mesh* m, const int8_t* kind) {
    if (!m || !kind) { set_error("gks_mesh_set_boundary: NULL argument"); return GKS_E_ARG; }
    std::vector<int8_t> bk((size_t)m->nf, 0);
    for (int64_t c = 0; c < m->nc; ++c)
        for (int f = 0; f < 4; ++f) {
            if (m->nbr[c * 4 + f] >= 0) continue;
            const int8_t k = kind[c * 4 + f];
            if (k != GKS_BC_OPEN && k != GKS_BC_SLIP_WALL && k != GKS_BC_FIXED && k != GKS_BC_NOSLIP_WALL &&
                k != GKS_BC_ISOTHERMAL_WALL && k != GKS_BC_MOVING_WALL) {
                set_error("gks_mesh_set_boundary: unknown kind " + std::to_string((int)k) + " at cell " +
                          std::to_string(c) + " face " + std::to_string(f));
                return GKS_E_ARG;
            }
            bk[(size_t)m->csr_face[c * 4 + f]] = k;
        }
    m->bkind.swap(bk);
    return GKS_OK;
}

extern "C" gks_status gks_mesh_cases(const gks_mesh* m, int32_t* n_case, int64_t* case_first_cell) {
    if (!m) { set_error("mesh is NULL"); return GKS_E_ARG; }
    if (n_case) *n_case = m->ncase;
    if (case_first_cell) {
        int64_t c = 0;
        for (int32_t k = 0; k < m->ncase; ++k) {
            while (c < m->nc && m->cell_case[c] < k) ++c;
            case_first_cell[k] = c;
        }
        case_first_cell[m->ncase] = m->nc;
    }
    return GKS_OK;
}

template <typename A>
static void copy_out(A* dst, const std::vector<A>& src) {
    if (dst) std::memcpy(dst, src.data(), sizeof(A) * src.size());
}

extern "C" gks_status gks_mesh_topology(const gks_mesh* m, int64_t* face_v, int64_t* face_lr,
                                        int64_t* nbr, int64_t* csr_face, int8_t* csr_sign) {
    if (!m) { set_error("mesh is NULL"); return GKS_E_ARG; }
    copy_out(face_v, m->face_v);
    copy_out(face_lr, m->face_lr);
    copy_out(nbr, m->nbr);
    copy_out(csr_face, m->csr_face);
    copy_out(csr_sign, m->csr_sign);
    return GKS_OK;
}

extern "C" gks_status gks_mesh_geometry(const gks_mesh* m, double* vol, double* cen, double* mom2,
                                        double* dr, double* farea, double* fnorm, double* gp_l,
                                        double* gp_r) {
    if (!m) { set_error("mesh is NULL"); return GKS_E_ARG; }
    copy_out(vol, m->vol);
    copy_out(cen, m->cen);
    copy_out(mom2, m->mom2);
    copy_out(dr, m->dr);
    copy_out(farea, m->farea);
    copy_out(fnorm, m->fnorm);
    copy_out(gp_l, m->gp_l);
    copy_out(gp_r, m->gp_r);
    return GKS_OK;
}

extern "C" gks_status gks_stencil_build(gks_mesh* m, int64_t* n_singular) {
    if (!m) { set_error("mesh is NULL"); return GKS_E_ARG; }
    try {
        gks_status st = build_stencils(*m);
        if (st != GKS_OK) return st;
    } catch (const std::bad_alloc&) {
        set_error("out of memory");
        return GKS_E_NOMEM;
    }
    if (n_singular) *n_singular = m->n_singular;
    return GKS_OK;
}

extern "C" gks_status gks_mesh_stencils(const gks_mesh* m, double* M1, double* M2) {
    if (!m) { set_error("mesh is NULL"); return GKS_E_ARG; }
    if (!m->has_stencils) { set_error("stencils not built"); return GKS_E_STENCIL; }
    copy_out(M1, m->M1);
    copy_out(M2, m->M2);
    return GKS_OK;
}

extern "C" gks_status gks_mesh_wall_stencils(const gks_mesh* m, double* W1, double* W2, int8_t* built,
                                             int64_t* n_built) {
    if (!m) { set_error("mesh is NULL"); return GKS_E_ARG; }
    int64_t n = 0;
    for (int64_t c = 0; c < m->nc; ++c) {
        double w1[15], w2[153];
        const bool ok = has_wall_face(*m, c) && cell_wall_stencil(*m, c, w2, w1);
        if (!ok) {
            std::memset(w1, 0, sizeof(w1));
            std::memset(w2, 0, sizeof(w2));
        }
        if (W1) std::memcpy(W1 + c * 15, w1, sizeof(w1));
        if (W2) std::memcpy(W2 + c * 153, w2, sizeof(w2));
        if (built) built[c] = ok ? 1 : 0;
        n += ok;
    }
    if (n_built) *n_built = n;
    return GKS_OK;
}

// ----------------------------------------------------------------- state --

namespace {

struct Layout {
    size_t total = 0;
    int64_t nwall = 0;  // slots of wall-constrained operators
    // mesh
    size_t nbr, cface, inv_vol, dr, M1, tile, flr, fgeo, fan, cell_case, perm;
    // state
    size_t Wd, X, Xs, X0, S, G, slopes, poly, rec, ctrl, case_t, case_dt, case_dtmin, part, err, stage, cperm, cinv,
        gbar, wslot, wop;
    size_t add(size_t bytes) {
        size_t off = total;
        total += (bytes + 255) & ~(size_t)255;
        return off;
    }
};

bool has_fixed(const gks_mesh& m) {
    for (int64_t f = 0; f < m.nf; ++f)
        if (m.bkind[f] == GKS_BC_FIXED) return true;
    return false;
}

// cells that take the Sec. 4.4 wall-constrained stencils (an upper bound:
// every cell with a non-slip adiabatic wall face) when the option is on
int64_t wall_cells(const gks_mesh& m, const gks_params& p) {
    if (!p.wall_constraint) return 0;
    int64_t n = 0;
    for (int64_t c = 0; c < m.nc; ++c) n += has_wall_face(m, c);
    return n;
}

Layout layout_workspace(int64_t nc, int64_t nf, int64_t ncase, bool fp32, bool fixed, bool ops64 = false,
                        int64_t nwall = 0) {
    Layout L;
    const size_t T = fp32 ? 4 : 8;
    // FP32 bulk with FP64 stencil operators: the reconstruction tile and the
    // step-1 operator stay FP64 (as in the FP64 path)
    const size_t TO = ops64 ? 8 : T;
    const size_t nblk = (size_t)update_blocks(nc);
    L.nbr = L.add(4 * 4 * nc);
    L.cface = L.add(4 * 4 * nc);
    L.inv_vol = L.add(8 * nc);
    L.dr = L.add(T * nc);
    L.M1 = L.add(TO * 12 * nc);
    L.tile = L.add(TO * TILE_ROWS * CELLS_PER_BLOCK * nblk);
    L.flr = L.add(4 * 2 * nf);
    L.fgeo = L.add(T * FGEO * nf);
    L.fan = fp32 ? L.add(4 * 6 * nf) : 0;  // FP32 bulk: face area vectors A n as FP32 hi / lo pairs
    L.cell_case = L.add(4 * nc);
    L.perm = L.add(4 * nf);
    L.Wd = L.add(8 * 5 * nc);
    const size_t xs = fp32 ? Stride<float>::xs : Stride<double>::xs;
    L.X = L.add(T * xs * nc);
    L.Xs = L.add(T * xs * nc);
    L.X0 = fixed ? L.add(T * xs * nc) : 0;  // state held by fixed boundary faces
    L.S = L.add(8 * 5 * nc);
    L.G = L.add(T * 15 * nc);
    L.slopes = L.add(T * 15 * nc);
    L.poly = L.add(T * (fp32 ? Stride<float>::poly : Stride<double>::poly) * nc);
    L.rec = L.add(T * (fp32 ? REC1_F32 : 40) * nf);
    L.ctrl = L.add(8 * CTRL_N);
    L.case_t = L.add(8 * ncase);
    L.case_dt = L.add(8 * ncase);
    L.case_dtmin = L.add(8 * ncase);
    L.part = L.add(8 * PART_N * nblk);
    L.err = L.add(4);
    L.gbar = L.add(2 * sizeof(unsigned));  // grid-barrier words of the one-launch stage
    // scratch: host-buffer staging, time-step partials, autotune snapshot,
    // re-ordering of the cells (FP64 averages, the working state and the
    // fixed state: 40 doubles a cell at most)
    L.stage = L.add(8 * (40 * nc + 3 * ncase + CTRL_N + 1));
    // FP32 bulk: device cell -> caller's cell (the cell ordering)
    L.cperm = fp32 ? L.add(4 * nc) : 0;
    L.cinv = fp32 ? L.add(4 * nc) : 0;
    // Sec. 4.4 wall-constrained momentum operators: slot of each (device)
    // cell, -1 for none, and per slot W2 [9][17] then W1 [3][5] in TO
    L.nwall = nwall;
    L.wslot = nwall ? L.add(4 * nc) : 0;
    L.wop = nwall ? L.add(TO * WOP_STRIDE * nwall) : 0;
    return L;
}

}  // namespace

struct gks_state {
    const gks_mesh* mesh = nullptr;
    gks_params params;
    HostPhys phys;
    bool fp32 = false;
    bool ops64 = false;  // precision 2: FP32 bulk with FP64 stencil operators
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char* ws = nullptr;
    Layout L;
    DevMesh<double> m64;
    DevMesh<float> m32;
    DevState<double> s64;
    DevState<float> s32;
    cudaGraphExec_t graph = nullptr;
    bool initialised = false;
    bool stage_valid = false;  // the stage buffer holds the last step's W*, grad W*
    bool fixed_pinned = false;  // gks_set_fixed_state was called: initialisations keep the fixed state
    int face_order = 0;    // 0: canonical face order, 1: grouped by left cell
    int flux_variant = 1;  // 1: 3 blocks/SM, 0: 2 blocks/SM (FP32 flux)
    int slopes_pass = 0;   // 1: reconstruction step 1 as its own pass
    int fused = 0;         // 1: each stage as one persistent launch (precision 1 only)
    // cell ordering of the device arrays (FP32 bulk): 0 the caller's, 1
    // reverse Cuthill-McKee, 2 Morton, each within each case; cperm maps a
    // device cell to the caller's cell, cinv back (empty: identity)
    int cell_order = 0;
    std::vector<int32_t> cperm, cinv;
    std::vector<int8_t> adj_rev;  // reverse face slots of the adjoint (built on first use)
    // device copy of cperm, or NULL for the caller's order
    const int32_t* dperm() const { return cperm.empty() ? nullptr : reinterpret_cast<const int32_t*>(ws + L.cperm); }
    const int32_t* dinv() const { return cinv.empty() ? nullptr : reinterpret_cast<const int32_t*>(ws + L.cinv); }
    int64_t pub(int64_t d) const { return cperm.empty() ? d : cperm[d]; }
    int64_t dev(int64_t c) const { return cinv.empty() ? c : cinv[c]; }
};

// ---------------------------------------------------------- orderings --

// Cell ordering within each case (the cases stay contiguous and in order).
// 1: reverse Cuthill-McKee on the face-neighbour graph, breadth first from a
// cell of least degree at the end of a few sweeps (a pseudo-peripheral
// cell), neighbours taken by increasing degree, the order reversed;
// 2: Morton (Z) order of the centroids, 10 bits per axis over the case's
// bounding box.  Returns device cell -> caller's cell.
static std::vector<int32_t> cell_permutation(const gks_mesh& g, int order) {
    const int64_t nc = g.nc;
    std::vector<int32_t> perm((size_t)nc);
    for (int64_t c = 0; c < nc; ++c) perm[c] = (int32_t)c;
    if (order == 0) return perm;
    int64_t c0 = 0;
    while (c0 < nc) {
        int64_t c1 = c0;
        while (c1 < nc && g.cell_case[c1] == g.cell_case[c0]) ++c1;
        const int64_t n = c1 - c0;
        if (order == 2) {
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int64_t c = c0; c < c1; ++c)
                for (int a = 0; a < 3; ++a) {
                    lo[a] = std::min(lo[a], g.cen[c * 3 + a]);
                    hi[a] = std::max(hi[a], g.cen[c * 3 + a]);
                }
            std::vector<std::pair<uint64_t, int32_t>> key((size_t)n);
            for (int64_t c = c0; c < c1; ++c) {
                uint64_t code = 0;
                uint32_t q[3];
                for (int a = 0; a < 3; ++a) {
                    const double t = hi[a] > lo[a] ? (g.cen[c * 3 + a] - lo[a]) / (hi[a] - lo[a]) : 0.0;
                    q[a] = (uint32_t)std::min(1023.0, std::max(0.0, std::floor(t * 1024.0)));
                }
                for (int b = 9; b >= 0; --b)
                    for (int a = 0; a < 3; ++a) code = (code << 1) | ((q[a] >> b) & 1u);
                key[c - c0] = {code, (int32_t)c};
            }
            std::stable_sort(key.begin(), key.end(),
                             [](const auto& x, const auto& y) { return x.first < y.first; });
            for (int64_t i = 0; i < n; ++i) perm[c0 + i] = key[i].second;
        } else {
            auto deg = [&](int64_t c) {
                int d = 0;
                for (int f = 0; f < 4; ++f) d += g.nbr[c * 4 + f] >= 0;
                return d;
            };
            std::vector<int64_t> level((size_t)n, -1), out;
            out.reserve((size_t)n);
            std::vector<char> seen((size_t)n, 0);
            // breadth-first order from `start` over the unvisited cells of the case;
            // returns the last cell reached (the far end of the sweep)
            auto sweep = [&](int64_t start, bool emit) {
                std::vector<int64_t> queue{start};
                std::vector<char> vis((size_t)n, 0);
                vis[start - c0] = 1;
                int64_t last = start;
                for (size_t h = 0; h < queue.size(); ++h) {
                    const int64_t c = queue[h];
                    last = c;
                    if (emit) {
                        out.push_back(c);
                        seen[c - c0] = 1;
                    }
                    int64_t nb[4];
                    int k = 0;
                    for (int f = 0; f < 4; ++f) {
                        const int64_t m = g.nbr[c * 4 + f];
                        if (m >= c0 && m < c1 && !vis[m - c0] && !(emit && seen[m - c0])) nb[k++] = m;
                    }
                    // by increasing degree, then id (a total order): insertion
                    // sort of the at most 4 candidates
                    auto before = [&](int64_t a, int64_t b) {
                        const int da = deg(a), db = deg(b);
                        return da != db ? da < db : a < b;
                    };
                    for (int i = 1; i < k; ++i)
                        for (int j = i; j > 0 && before(nb[j], nb[j - 1]); --j) std::swap(nb[j], nb[j - 1]);
                    for (int i = 0; i < k; ++i) {
                        if (vis[nb[i] - c0]) continue;
                        vis[nb[i] - c0] = 1;
                        queue.push_back(nb[i]);
                    }
                }
                return last;
            };
            for (int64_t s0 = c0; s0 < c1; ++s0) {
                if (seen[s0 - c0]) continue;
                // least-degree unvisited cell, then two sweeps to a far end
                int64_t start = s0;
                for (int64_t c = s0; c < c1; ++c)
                    if (!seen[c - c0] && deg(c) < deg(start)) start = c;
                int64_t far = start;
                for (int it = 0; it < 2; ++it) far = sweep(far, false);
                sweep(far, true);
            }
            for (int64_t i = 0; i < n; ++i) perm[c0 + i] = (int32_t)out[(size_t)(n - 1 - i)];
        }
        c0 = c1;
    }
    return perm;
}

template <typename T>
static T* at(gks_state* s, size_t off) {
    return reinterpret_cast<T*>(s->ws + off);
}

template <typename T>
static void make_views(gks_state* s, DevMesh<T>& m, DevState<T>& st) {
    const Layout& L = s->L;
    m.nc = s->mesh->nc;
    m.nf = s->mesh->nf;
    m.ncase = s->mesh->ncase;
    m.cell_case = at<int32_t>(s, L.cell_case);
    m.nbr = at<int32_t>(s, L.nbr);
    m.cface = at<int32_t>(s, L.cface);
    m.inv_vol = at<double>(s, L.inv_vol);
    m.dr = at<T>(s, L.dr);
    if (s->ops64) {
        m.M1 = nullptr;
        m.tile = nullptr;
        m.M1d = at<double>(s, L.M1);
        m.tiled = at<double>(s, L.tile);
    } else {
        m.M1 = at<T>(s, L.M1);
        m.tile = at<T>(s, L.tile);
        m.M1d = nullptr;
        m.tiled = nullptr;
    }
    m.flr = at<int32_t>(s, L.flr);
    m.fgeo = at<T>(s, L.fgeo);
    m.fan = L.fan ? at<float>(s, L.fan) : nullptr;
    m.fixed = L.X0 ? at<T>(s, L.X0) : nullptr;
    m.wslot = L.wslot ? at<int32_t>(s, L.wslot) : nullptr;
    m.wop = L.wslot && !s->ops64 ? at<T>(s, L.wop) : nullptr;
    m.wopd = L.wslot && s->ops64 ? at<double>(s, L.wop) : nullptr;
    m.xwalls = 0;
    for (int64_t f = 0; f < s->mesh->nf; ++f)
        if (s->mesh->bkind[f] == GKS_BC_ISOTHERMAL_WALL || s->mesh->bkind[f] == GKS_BC_MOVING_WALL) m.xwalls = 1;
    st.Wd = at<double>(s, L.Wd);
    st.X = at<T>(s, L.X);
    st.Xs = at<T>(s, L.Xs);
    st.S = at<double>(s, L.S);
    st.G = at<T>(s, L.G);
    st.slopes = at<T>(s, L.slopes);
    st.poly = at<T>(s, L.poly);
    st.rec = at<T>(s, L.rec);
    st.ctrl = at<double>(s, L.ctrl);
    st.case_t = at<double>(s, L.case_t);
    st.case_dt = at<double>(s, L.case_dt);
    st.case_dtmin = at<unsigned long long>(s, L.case_dtmin);
    st.part = at<double>(s, L.part);
    st.err = at<int32_t>(s, L.err);
}

// Device face order: canonical (0) or grouped by left cell (1).  perm maps a
// device face index to its canonical index; the cell-to-face list, the face
// arrays and the records use device indices.
static std::vector<int32_t> face_permutation(const gks_mesh& g, int order, const std::vector<int32_t>& cinv) {
    std::vector<int32_t> perm((size_t)g.nf);
    for (int64_t f = 0; f < g.nf; ++f) perm[f] = (int32_t)f;
    if (order == 1) {
        auto key = [&](int32_t f) {
            const int64_t l = g.face_lr[f * 2], r = g.face_lr[f * 2 + 1];
            const int64_t c = l >= 0 ? l : r;
            return std::make_pair(cinv.empty() ? c : (int64_t)cinv[c], (int64_t)f);
        };
        std::sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return key(a) < key(b); });
    }
    return perm;
}

template <typename T>
static gks_status upload_faces(gks_state* s) {
    const gks_mesh& g = *s->mesh;
    const int64_t nc = g.nc, nf = g.nf;
    const Layout& L = s->L;
    const std::vector<int32_t> perm = face_permutation(g, s->face_order, s->cinv);
    std::vector<int32_t> inv((size_t)nf);
    for (int64_t d = 0; d < nf; ++d) inv[perm[d]] = (int32_t)d;
    std::vector<int32_t> cface(4 * nc), flr(2 * nf);
    std::vector<T> fgeo(FGEO * nf, T(0));
    std::vector<float> fan(s->L.fan ? 6 * nf : 0, 0.0f);
    for (int64_t d = 0; d < nc; ++d) {
        const int64_t c = s->pub(d);
        for (int f = 0; f < 4; ++f) {
            const int64_t fi = g.csr_face[c * 4 + f];
            const bool left = g.csr_sign[c * 4 + f] > 0;
            cface[f * nc + d] = (int32_t)((int64_t)inv[fi] * 2 + (left ? 0 : 1));
        }
    }
    for (int64_t d = 0; d < nf; ++d) {
        const int64_t f = perm[d];
        // a boundary face's missing side carries its kind: -1 - GKS_BC_*
        const int32_t miss = -1 - (int32_t)g.bkind[f];
        flr[d] = g.face_lr[f * 2] >= 0 ? (int32_t)s->dev(g.face_lr[f * 2]) : miss;
        flr[nf + d] = g.face_lr[f * 2 + 1] >= 0 ? (int32_t)s->dev(g.face_lr[f * 2 + 1]) : miss;
        T* r = &fgeo[d * FGEO];
        for (int a = 0; a < 3; ++a) r[a] = (T)g.fnorm[f * 3 + a];
        r[3] = (T)(g.farea[f] / 3.0);
        for (int k = 0; k < 9; ++k) {
            r[4 + k] = (T)g.gp_l[f * 9 + k];
            r[13 + k] = (T)g.gp_r[f * 9 + k];
        }
        if (!fan.empty())
            for (int a = 0; a < 3; ++a) {
                const double v = g.farea[f] * g.fnorm[f * 3 + a];
                fan[d * 6 + 2 * a] = (float)v;
                fan[d * 6 + 2 * a + 1] = (float)(v - (double)(float)v);
            }
    }
    auto put = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
        return cudaMemcpyAsync(s->ws + off, src, bytes, cudaMemcpyHostToDevice, s->stream);
    };
    GKS_CHECK_CUDA(put(L.cface, cface.data(), 4 * cface.size()));
    GKS_CHECK_CUDA(put(L.flr, flr.data(), 4 * flr.size()));
    GKS_CHECK_CUDA(put(L.fgeo, fgeo.data(), sizeof(T) * fgeo.size()));
    if (!fan.empty()) GKS_CHECK_CUDA(put(L.fan, fan.data(), 4 * fan.size()));
    GKS_CHECK_CUDA(put(L.perm, perm.data(), 4 * perm.size()));
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));  // host vectors die here
    return GKS_OK;
}

// the reconstruction's static cell data in the operator precision TO
template <typename T, typename TO>
static gks_status upload_cells(gks_state* s) {
    const gks_mesh& g = *s->mesh;
    const int64_t nc = g.nc;
    const Layout& L = s->L;
    std::vector<int32_t> nbr(4 * nc);
    std::vector<double> inv_vol(nc);
    const int64_t nblk = update_blocks(nc);
    std::vector<T> dr(nc);
    std::vector<TO> M1(12 * nc);
    // per-block tile [blk][TILE_ROWS][CELLS_PER_BLOCK], zero past the last cell
    std::vector<TO> tile((size_t)nblk * TILE_ROWS * CELLS_PER_BLOCK, TO(0));
    // Sec. 4.4: with linear weights a boundary cell's third-order step is the
    // least-squares first-order fit to its P2 stencil
    const bool linear_boundary = !s->params.weno && s->params.order == 3;
    std::vector<int32_t> cell_case((size_t)nc);
    // Sec. 4.4 wall-constrained operators, slots in device-cell order
    std::vector<int32_t> wslot(L.wslot ? (size_t)nc : 0, -1);
    std::vector<TO> wop((size_t)L.nwall * WOP_STRIDE, TO(0));
    int64_t nwop = 0;
    // d: device cell; c: the caller's cell it holds
    for (int64_t d = 0; d < nc; ++d) {
        const int64_t c = s->pub(d);
        cell_case[d] = g.cell_case[c];
        TO* tc = &tile[(size_t)(d / CELLS_PER_BLOCK) * TILE_ROWS * CELLS_PER_BLOCK + d % CELLS_PER_BLOCK];
        auto put_row = [&](int row, double v) { tc[(size_t)row * CELLS_PER_BLOCK] = (TO)v; };
        for (int f = 0; f < 4; ++f) {
            nbr[f * nc + d] = g.nbr[c * 4 + f] >= 0 ? (int32_t)s->dev(g.nbr[c * 4 + f]) : -1;
            const int64_t fi = g.csr_face[c * 4 + f];
            const bool left = g.csr_sign[c * 4 + f] > 0;
            const double* gp = left ? &g.gp_l[fi * 9] : &g.gp_r[fi * 9];
            for (int k = 0; k < 9; ++k) put_row(TILE_G + f * 9 + k, gp[k]);
        }
        inv_vol[d] = 1.0 / g.vol[c];
        put_row(TILE_V23, std::pow(g.vol[c], 2.0 / 3.0));
        put_row(TILE_V43, std::pow(g.vol[c], 4.0 / 3.0));
        dr[d] = (T)g.dr[c];
        for (int q = 0; q < 6; ++q) put_row(TILE_MOM + q, g.mom2[c * 6 + q]);
        for (int k = 0; k < 12; ++k) {
            M1[k * nc + d] = (TO)g.M1[c * 12 + k];
            put_row(TILE_M1 + k, g.M1[c * 12 + k]);
        }
        if (L.wslot) {
            double w2[153], w1[15];
            if (has_wall_face(g, c) && cell_wall_stencil(g, c, w2, w1)) {
                wslot[d] = (int32_t)(nwop++);
                TO* o = &wop[(size_t)wslot[d] * WOP_STRIDE];
                for (int k = 0; k < 153; ++k) o[k] = (TO)w2[k];
                for (int k = 0; k < 15; ++k) o[WOP_W1 + k] = (TO)w1[k];
            }
        }
        const double* M2c = &g.M2[c * 144];
        double M2lin[144];
        if (linear_boundary && !g.singular[c] &&
            (g.nbr[c * 4] < 0 || g.nbr[c * 4 + 1] < 0 || g.nbr[c * 4 + 2] < 0 || g.nbr[c * 4 + 3] < 0) &&
            cell_linear_fit(g, c, M2lin))
            M2c = M2lin;
        for (int k = 0; k < 144; ++k) put_row(TILE_M2 + k, M2c[k]);
    }
    auto put = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
        return cudaMemcpyAsync(s->ws + off, src, bytes, cudaMemcpyHostToDevice, s->stream);
    };
    GKS_CHECK_CUDA(put(L.nbr, nbr.data(), 4 * nbr.size()));
    GKS_CHECK_CUDA(put(L.inv_vol, inv_vol.data(), 8 * inv_vol.size()));
    GKS_CHECK_CUDA(put(L.dr, dr.data(), sizeof(T) * dr.size()));
    GKS_CHECK_CUDA(put(L.M1, M1.data(), sizeof(TO) * M1.size()));
    GKS_CHECK_CUDA(put(L.tile, tile.data(), sizeof(TO) * tile.size()));
    GKS_CHECK_CUDA(put(L.cell_case, cell_case.data(), 4 * cell_case.size()));
    if (L.wslot) {
        GKS_CHECK_CUDA(put(L.wslot, wslot.data(), 4 * wslot.size()));
        if (nwop) GKS_CHECK_CUDA(put(L.wop, wop.data(), sizeof(TO) * WOP_STRIDE * nwop));
    }
    if (!s->cperm.empty()) {
        GKS_CHECK_CUDA(put(L.cperm, s->cperm.data(), 4 * s->cperm.size()));
        GKS_CHECK_CUDA(put(L.cinv, s->cinv.data(), 4 * s->cinv.size()));
    }
    GKS_CHECK_CUDA(cudaMemsetAsync(s->ws + L.ctrl, 0, 8 * CTRL_N, s->stream));
    GKS_CHECK_CUDA(cudaMemsetAsync(s->ws + L.err, 0, 4, s->stream));
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));  // host vectors die here
    return upload_faces<T>(s);
}

template <typename T>
static gks_status upload_mesh(gks_state* s) {
    return s->ops64 ? upload_cells<T, double>(s) : upload_cells<T, T>(s);
}

extern "C" size_t gks_workspace_bytes(const gks_mesh* mesh, const gks_params* params) {
    if (!mesh || check_params(params) != GKS_OK) return 0;
    return layout_workspace(mesh->nc, mesh->nf, mesh->ncase, params->precision != 0, has_fixed(*mesh),
                            params->precision == 2, wall_cells(*mesh, *params))
        .total;
}

extern "C" gks_status gks_state_create(const gks_mesh* mesh, const gks_params* params,
                                       void* d_workspace, size_t workspace_bytes, void* stream,
                                       gks_state** out) {
    if (!out) { set_error("gks_state_create: out is NULL"); return GKS_E_ARG; }
    *out = nullptr;
    if (!mesh) { set_error("gks_state_create: mesh is NULL"); return GKS_E_ARG; }
    gks_status ps = check_params(params);
    if (ps != GKS_OK) return ps;
    if (!mesh->has_stencils) { set_error("gks_state_create: stencils not built"); return GKS_E_STENCIL; }
    const bool fp32 = params->precision != 0;
    const bool ops64 = params->precision == 2;
    Layout L = layout_workspace(mesh->nc, mesh->nf, mesh->ncase, fp32, has_fixed(*mesh), ops64,
                                wall_cells(*mesh, *params));
    if (!d_workspace || workspace_bytes < L.total) {
        set_error("gks_state_create: workspace missing or smaller than gks_workspace_bytes()");
        return GKS_E_NOMEM;
    }
    if (((uintptr_t)d_workspace & 255) != 0) {
        set_error("gks_state_create: workspace must be 256-byte aligned");
        return GKS_E_ARG;
    }
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, d_workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        set_error("gks_state_create: workspace is not device memory");
        return GKS_E_ARG;
    }
    gks_state* s = new (std::nothrow) gks_state();
    if (!s) { set_error("out of memory"); return GKS_E_NOMEM; }
    s->mesh = mesh;
    s->params = *params;
    s->phys = HostPhys{params->gamma, params->cfl, params->mu, params->eps_weno, params->tau_eps,
                       params->tau_c, params->weno, params->order, params->smooth_flux, params->viscous,
                       params->viscous ? 1.0 / params->prandtl - 1.0 : 0.0, params->wall_temperature,
                       {params->wall_velocity[0], params->wall_velocity[1], params->wall_velocity[2]}};
    s->fp32 = fp32;
    s->ops64 = ops64;
    s->ws = static_cast<char*>(d_workspace);
    s->L = L;
    if (stream) {
        s->stream = static_cast<cudaStream_t>(stream);
    } else {
        // the legacy default stream cannot be captured into a graph
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            set_error(std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            delete s;
            return GKS_E_CUDA;
        }
        s->own_stream = true;
    }
    gks_status st;
    if (fp32) {
        make_views<float>(s, s->m32, s->s32);
        st = upload_mesh<float>(s);
    } else {
        make_views<double>(s, s->m64, s->s64);
        st = upload_mesh<double>(s);
    }
    if (st != GKS_OK) {
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return st;
    }
    *out = s;
    return GKS_OK;
}

extern "C" void gks_state_destroy(gks_state* s) {
    if (!s) return;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->own_stream) {
        cudaStreamSynchronize(s->stream);
        cudaStreamDestroy(s->stream);
    }
    delete s;
}

// the caller's legacy-stream work must finish before an internal stream reads
static void order_after_caller(gks_state* s) {
    if (s->own_stream) cudaStreamSynchronize(0);
}

template <typename T>
static gks_status init_impl(gks_state* s, DevMesh<T>& m, DevState<T>& st, const double* d_W,
                            const double* d_dW) {
    s->stage_valid = false;
    const int64_t nc = m.nc;
    if (s->dperm())
        GKS_CHECK_CUDA(launch_cells_perm(d_W, st.Wd, nc, 5, s->dperm(), 0, s->stream));
    else
        GKS_CHECK_CUDA(cudaMemcpyAsync(st.Wd, d_W, 8 * 5 * nc, cudaMemcpyDeviceToDevice, s->stream));
    GKS_CHECK_CUDA(Launch<T>::pack(d_W, d_dW, st.X, nc, s->stream, s->dperm()));
    if (m.fixed && !s->fixed_pinned)  // fixed boundaries hold the initial state
        GKS_CHECK_CUDA(cudaMemcpyAsync((void*)m.fixed, st.X, sizeof(T) * Stride<T>::xs * nc, cudaMemcpyDeviceToDevice,
                                       s->stream));
    GKS_CHECK_CUDA(launch_set_control(st.ctrl, st.case_t, st.case_dt, st.case_dtmin, m.ncase, 0.0, 0.0, 1, s->stream));
    GKS_CHECK_CUDA(cudaMemsetAsync(st.err, 0, 4, s->stream));
    GKS_CHECK_CUDA(Launch<T>::init_dtmin(m, s->phys, st.X, st.case_dtmin, s->stream));
    return GKS_OK;
}

extern "C" gks_status gks_set_fixed_state(gks_state* s, const double* d_W, const double* d_dW) {
    if (!s || !d_W || !d_dW) { set_error("gks_set_fixed_state: NULL argument"); return GKS_E_ARG; }
    if (!has_fixed(*s->mesh)) { set_error("gks_set_fixed_state: the mesh has no fixed boundary faces"); return GKS_E_ARG; }
    order_after_caller(s);
    const int64_t nc = s->mesh->nc;
    if (s->fp32)
        GKS_CHECK_CUDA(Launch<float>::pack(d_W, d_dW, const_cast<float*>(s->m32.fixed), nc, s->stream, s->dperm()));
    else
        GKS_CHECK_CUDA(Launch<double>::pack(d_W, d_dW, const_cast<double*>(s->m64.fixed), nc, s->stream));
    s->fixed_pinned = true;
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return GKS_OK;
}

extern "C" gks_status gks_init_state(gks_state* s, const double* d_W, const double* d_dW) {
    if (!s || !d_W || !d_dW) { set_error("gks_init_state: NULL argument"); return GKS_E_ARG; }
    order_after_caller(s);
    gks_status st = s->fp32 ? init_impl<float>(s, s->m32, s->s32, d_W, d_dW)
                            : init_impl<double>(s, s->m64, s->s64, d_W, d_dW);
    if (st != GKS_OK) return st;
    s->initialised = true;
    if (s->own_stream) GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return GKS_OK;
}

// reconstruction of one stage (Sec. 4.3): step 1 as its own pass when the
// variant asks for it and the scheme needs the slopes, else fused into step 2
template <typename T>
static cudaError_t enqueue_recon(gks_state* s, DevMesh<T>& m, DevState<T>& st, const T* X,
                                 const typename Launch<T>::Finalize* fin) {
    const HostPhys& p = s->phys;
    if (s->slopes_pass && p.weno) {
        cudaError_t e = Launch<T>::slopes(m, X, st.slopes, fin, s->stream);
        if (e != cudaSuccess) return e;
        return Launch<T>::recon(m, p, X, st.slopes, nullptr, st.poly, nullptr, nullptr, st.err, s->stream);
    }
    return Launch<T>::recon(m, p, X, nullptr, nullptr, st.poly, nullptr, fin, st.err, s->stream);
}

// one two-stage step (Sec. 3): enqueued on s->stream (captured into a graph).
// The first kernel's block 0 first turns the per-block time-step minima left
// by the previous update (or by gks_init_state) into this step's dt.
template <typename T>
static cudaError_t enqueue_step(gks_state* s, DevMesh<T>& m, DevState<T>& st) {
    const HostPhys& p = s->phys;
    cudaStream_t q = s->stream;
    const typename Launch<T>::Finalize fin{st.case_dtmin, st.case_t, st.case_dt, m.ncase, p.cfl, st.ctrl};
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
        if (s->fused) {
            unsigned* gbar = reinterpret_cast<unsigned*>(s->ws + s->L.gbar);
            if ((e = launch_stage(m, p, st, 1, &fin, gbar, q)) != cudaSuccess) return e;
            return launch_stage(m, p, st, 2, nullptr, gbar, q);
        }
    }
    for (int stage = 1; stage <= 2; ++stage) {
        // stage 1 from (W^n, grad W^n), stage 2 from (W*, grad W*)
        const T* X = stage == 1 ? st.X : st.Xs;
        if ((e = enqueue_recon(s, m, st, X, stage == 1 ? &fin : nullptr)) != cudaSuccess) return e;
        if ((e = Launch<T>::flux(m, p, X, st.poly, st.rec, st.case_dt, 0.0, stage, q, s->flux_variant)) != cudaSuccess)
            return e;
        if ((e = stage == 1 ? Launch<T>::update1(m, p, st, q) : Launch<T>::update2(m, p, st, q)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t set_control(gks_state* s, double dt_fixed, double t_end, int reset) {
    if (s->fp32)
        return launch_set_control(s->s32.ctrl, s->s32.case_t, s->s32.case_dt, s->s32.case_dtmin, s->mesh->ncase,
                                  dt_fixed, t_end, reset, s->stream);
    return launch_set_control(s->s64.ctrl, s->s64.case_t, s->s64.case_dt, s->s64.case_dtmin, s->mesh->ncase,
                              dt_fixed, t_end, reset, s->stream);
}

static gks_status build_graph(gks_state* s) {
    cudaGraph_t g = nullptr;
    GKS_CHECK_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = s->fp32 ? enqueue_step<float>(s, s->m32, s->s32) : enqueue_step<double>(s, s->m64, s->s64);
    cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        set_error(std::string("step capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return GKS_E_CUDA;
    }
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->graph = nullptr;
        set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        return GKS_E_CUDA;
    }
    return GKS_OK;
}

extern "C" gks_status gks_step(gks_state* s, int32_t nsteps, double dt_fixed, double t_end) {
    if (!s) { set_error("gks_step: state is NULL"); return GKS_E_ARG; }
    if (!s->initialised) { set_error("gks_step: state not initialised"); return GKS_E_STATE; }
    if (nsteps < 0) { set_error("gks_step: negative nsteps"); return GKS_E_ARG; }
    if (!std::isfinite(dt_fixed) || !std::isfinite(t_end)) { set_error("gks_step: non-finite dt/t_end"); return GKS_E_ARG; }
    if (!s->graph) {
        gks_status st = build_graph(s);
        if (st != GKS_OK) return st;
    }
    GKS_CHECK_CUDA(set_control(s, dt_fixed, t_end, 0));
    for (int32_t i = 0; i < nsteps; ++i) GKS_CHECK_CUDA(cudaGraphLaunch(s->graph, s->stream));
    if (nsteps > 0) s->stage_valid = true;
    return GKS_OK;
}

// kernel-by-kernel step with events between launches (profiling breakdown)
template <typename T>
static gks_status step_timed_impl(gks_state* s, DevMesh<T>& m, DevState<T>& st, int32_t nsteps,
                                  double* kernel_ms, int64_t* launches) {
    const HostPhys& p = s->phys;
    cudaStream_t q = s->stream;
    const int nev = 16;
    cudaEvent_t ev[nev];
    for (int i = 0; i < nev; ++i) GKS_CHECK_CUDA(cudaEventCreate(&ev[i]));
    double acc[GKS_NKERNELS] = {0};
    int64_t cnt[GKS_NKERNELS] = {0};
    gks_status status = GKS_OK;
    for (int32_t it = 0; it < nsteps && status == GKS_OK; ++it) {
        int kid[nev];
        int ne = 0;
        auto mark = [&](int k) {
            kid[ne] = k;
            return cudaEventRecord(ev[ne++], q);
        };
        cudaError_t e = cudaEventRecord(ev[ne], q);
        kid[ne++] = -1;
        const typename Launch<T>::Finalize fin{st.case_dtmin, st.case_t, st.case_dt, m.ncase, p.cfl, st.ctrl};
        const bool fused = sizeof(T) == 4 && s->fused;
        if constexpr (sizeof(T) == 4) {
            unsigned* gbar = reinterpret_cast<unsigned*>(s->ws + s->L.gbar);
            for (int stage = 1; stage <= 2 && fused && e == cudaSuccess; ++stage) {
                e = launch_stage(m, p, st, stage, stage == 1 ? &fin : nullptr, gbar, q);
                if (e == cudaSuccess) e = mark(stage == 1 ? GKS_K_STAGE1 : GKS_K_STAGE2);
            }
        }
        for (int stage = 1; stage <= 2 && !fused && e == cudaSuccess; ++stage) {
            const T* X = stage == 1 ? st.X : st.Xs;
            const typename Launch<T>::Finalize* f = stage == 1 ? &fin : nullptr;
            if (s->slopes_pass && p.weno) {
                if (e == cudaSuccess) e = Launch<T>::slopes(m, X, st.slopes, f, q);
                if (e == cudaSuccess) e = mark(GKS_K_SLOPES);
                if (e == cudaSuccess)
                    e = Launch<T>::recon(m, p, X, st.slopes, nullptr, st.poly, nullptr, nullptr, st.err, q);
            } else if (e == cudaSuccess) {
                e = Launch<T>::recon(m, p, X, nullptr, nullptr, st.poly, nullptr, f, st.err, q);
            }
            if (e == cudaSuccess) e = mark(GKS_K_RECON);
            if (e == cudaSuccess) e = Launch<T>::flux(m, p, X, st.poly, st.rec, st.case_dt, 0.0, stage, q, s->flux_variant);
            if (e == cudaSuccess) e = mark(stage == 1 ? GKS_K_FLUX1 : GKS_K_FLUX2);
            if (e == cudaSuccess) e = stage == 1 ? Launch<T>::update1(m, p, st, q) : Launch<T>::update2(m, p, st, q);
            if (e == cudaSuccess) e = mark(stage == 1 ? GKS_K_UPDATE1 : GKS_K_UPDATE2);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[ne - 1]);
        for (int i = 1; i < ne && e == cudaSuccess; ++i) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
            acc[kid[i]] += ms;
            cnt[kid[i]] += 1;
        }
        if (e != cudaSuccess) {
            set_error(std::string("gks_step_timed: ") + cudaGetErrorString(e));
            status = GKS_E_CUDA;
        }
    }
    for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
    if (status != GKS_OK) return status;
    for (int k = 0; k < GKS_NKERNELS; ++k) {
        if (kernel_ms) kernel_ms[k] += acc[k];
        if (launches) launches[k] += cnt[k];
    }
    return GKS_OK;
}

extern "C" gks_status gks_step_timed(gks_state* s, int32_t nsteps, double dt_fixed, double t_end,
                                     double* kernel_ms, int64_t* launches) {
    if (!s) { set_error("gks_step_timed: state is NULL"); return GKS_E_ARG; }
    if (!s->initialised) { set_error("gks_step_timed: state not initialised"); return GKS_E_STATE; }
    if (nsteps < 0) { set_error("gks_step_timed: negative nsteps"); return GKS_E_ARG; }
    GKS_CHECK_CUDA(set_control(s, dt_fixed, t_end, 0));
    gks_status st = s->fp32 ? step_timed_impl<float>(s, s->m32, s->s32, nsteps, kernel_ms, launches)
                            : step_timed_impl<double>(s, s->m64, s->s64, nsteps, kernel_ms, launches);
    if (st != GKS_OK) return st;
    if (nsteps > 0) s->stage_valid = true;
    return gks_sync(s);
}

extern "C" gks_status gks_sync(gks_state* s) {
    if (!s) { set_error("gks_sync: state is NULL"); return GKS_E_ARG; }
    int32_t err = 0;
    GKS_CHECK_CUDA(cudaMemcpyAsync(&err, s->fp32 ? s->s32.err : s->s64.err, 4, cudaMemcpyDeviceToHost, s->stream));
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    if (err & ERR_TIMEOUT) {
        set_error("a bounded device wait (reconstruction tile copy or grid barrier) gave up");
        return GKS_E_TIMEOUT;
    }
    if (err & ERR_STATE) {
        set_error("non-positive density or pressure in an updated cell average");
        return GKS_E_STATE;
    }
    return GKS_OK;
}

template <typename T>
static gks_status get_impl(gks_state* s, DevState<T>& st, int64_t nc, double* d_W, double* d_dW) {
    if (d_W) {
        if (s->dperm())
            GKS_CHECK_CUDA(launch_cells_perm(st.Wd, d_W, nc, 5, s->dperm(), 1, s->stream));
        else
            GKS_CHECK_CUDA(cudaMemcpyAsync(d_W, st.Wd, 8 * 5 * nc, cudaMemcpyDeviceToDevice, s->stream));
    }
    if (d_dW) GKS_CHECK_CUDA(Launch<T>::unpack_grad(st.X, d_dW, nc, s->stream, s->dperm()));
    return GKS_OK;
}

extern "C" gks_status gks_get_state(const gks_state* cs, double* d_W, double* d_dW) {
    gks_state* s = const_cast<gks_state*>(cs);
    if (!s) { set_error("gks_get_state: state is NULL"); return GKS_E_ARG; }
    gks_status st = s->fp32 ? get_impl<float>(s, s->s32, s->mesh->nc, d_W, d_dW)
                            : get_impl<double>(s, s->s64, s->mesh->nc, d_W, d_dW);
    if (st != GKS_OK) return st;
    if (s->own_stream) return gks_sync(s);
    return GKS_OK;
}

extern "C" gks_status gks_case_times(gks_state* s, double* t, double* dt_last) {
    if (!s) { set_error("gks_case_times: state is NULL"); return GKS_E_ARG; }
    const size_t n = (size_t)s->mesh->ncase;
    if (t)
        GKS_CHECK_CUDA(cudaMemcpyAsync(t, s->fp32 ? s->s32.case_t : s->s64.case_t, 8 * n, cudaMemcpyDeviceToHost,
                                       s->stream));
    if (dt_last)
        GKS_CHECK_CUDA(cudaMemcpyAsync(dt_last, s->fp32 ? s->s32.case_dt : s->s64.case_dt, 8 * n,
                                       cudaMemcpyDeviceToHost, s->stream));
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return GKS_OK;
}

extern "C" gks_status gks_get_time(gks_state* s, double* t, double* dt_last) {
    if (!s) { set_error("gks_get_time: state is NULL"); return GKS_E_ARG; }
    double c[2];
    GKS_CHECK_CUDA(cudaMemcpyAsync(&c[0], s->fp32 ? s->s32.case_t : s->s64.case_t, 8, cudaMemcpyDeviceToHost, s->stream));
    GKS_CHECK_CUDA(cudaMemcpyAsync(&c[1], s->fp32 ? s->s32.case_dt : s->s64.case_dt, 8, cudaMemcpyDeviceToHost, s->stream));
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    if (t) *t = c[0];
    if (dt_last) *dt_last = c[1];
    return GKS_OK;
}

template <typename T>
static gks_status step_host_impl(gks_state* s, DevMesh<T>& m, DevState<T>& st, const double* h_W,
                                 const double* h_dW, int32_t nsteps, double dt_fixed, double* h_W_out,
                                 double* h_dW_out) {
    const int64_t nc = m.nc;
    double* stage = at<double>(s, s->L.stage);
    if (s->dperm()) {
        // the caller's order in the staging buffer, then into device order
        GKS_CHECK_CUDA(cudaMemcpyAsync(stage + 15 * nc, h_W, 8 * 5 * nc, cudaMemcpyHostToDevice, s->stream));
        GKS_CHECK_CUDA(launch_cells_perm(stage + 15 * nc, st.Wd, nc, 5, s->dperm(), 0, s->stream));
        GKS_CHECK_CUDA(cudaMemcpyAsync(stage, h_dW, 8 * 15 * nc, cudaMemcpyHostToDevice, s->stream));
        GKS_CHECK_CUDA(Launch<T>::pack(stage + 15 * nc, stage, st.X, nc, s->stream, s->dperm()));
    } else {
        GKS_CHECK_CUDA(cudaMemcpyAsync(st.Wd, h_W, 8 * 5 * nc, cudaMemcpyHostToDevice, s->stream));
        GKS_CHECK_CUDA(cudaMemcpyAsync(stage, h_dW, 8 * 15 * nc, cudaMemcpyHostToDevice, s->stream));
        GKS_CHECK_CUDA(Launch<T>::pack(st.Wd, stage, st.X, nc, s->stream));
    }
    if (m.fixed && !s->fixed_pinned)
        GKS_CHECK_CUDA(cudaMemcpyAsync((void*)m.fixed, st.X, sizeof(T) * Stride<T>::xs * nc, cudaMemcpyDeviceToDevice,
                                       s->stream));
    GKS_CHECK_CUDA(set_control(s, 0.0, 0.0, 1));
    GKS_CHECK_CUDA(Launch<T>::init_dtmin(m, s->phys, st.X, st.case_dtmin, s->stream));
    s->initialised = true;
    gks_status r = gks_step(s, nsteps, dt_fixed, 0.0);
    if (r != GKS_OK) return r;
    if (s->dperm()) {
        GKS_CHECK_CUDA(launch_cells_perm(st.Wd, stage + 15 * nc, nc, 5, s->dperm(), 1, s->stream));
        GKS_CHECK_CUDA(cudaMemcpyAsync(h_W_out, stage + 15 * nc, 8 * 5 * nc, cudaMemcpyDeviceToHost, s->stream));
    } else {
        GKS_CHECK_CUDA(cudaMemcpyAsync(h_W_out, st.Wd, 8 * 5 * nc, cudaMemcpyDeviceToHost, s->stream));
    }
    GKS_CHECK_CUDA(Launch<T>::unpack_grad(st.X, stage, nc, s->stream, s->dperm()));
    GKS_CHECK_CUDA(cudaMemcpyAsync(h_dW_out, stage, 8 * 15 * nc, cudaMemcpyDeviceToHost, s->stream));
    return gks_sync(s);
}

extern "C" gks_status gks_step_host(gks_state* s, const double* h_W, const double* h_dW, int32_t nsteps,
                                    double dt_fixed, double* h_W_out, double* h_dW_out) {
    if (!s || !h_W || !h_dW || !h_W_out || !h_dW_out) {
        set_error("gks_step_host: NULL argument");
        return GKS_E_ARG;
    }
    return s->fp32 ? step_host_impl<float>(s, s->m32, s->s32, h_W, h_dW, nsteps, dt_fixed, h_W_out, h_dW_out)
                   : step_host_impl<double>(s, s->m64, s->s64, h_W, h_dW, nsteps, dt_fixed, h_W_out, h_dW_out);
}

template <typename T>
static gks_status timestep_impl(gks_state* s, DevMesh<T>& m, DevState<T>& st, double* dt) {
    const int nblk = update_blocks(m.nc);
    double* tmp = at<double>(s, s->L.stage);  // scratch for the partials
    GKS_CHECK_CUDA(Launch<T>::dt_partials(m, s->phys, st.X, tmp, s->stream));
    std::vector<double> part((size_t)nblk * PART_N);
    GKS_CHECK_CUDA(cudaMemcpyAsync(part.data(), tmp, 8 * part.size(), cudaMemcpyDeviceToHost, s->stream));
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    double mn = INFINITY;
    for (int b = 0; b < nblk; ++b) mn = std::fmin(mn, part[(size_t)b * PART_N + PART_DTMIN]);
    *dt = s->params.cfl * mn;
    return GKS_OK;
}

extern "C" gks_status gks_timestep(gks_state* s, double* dt) {
    if (!s || !dt) { set_error("gks_timestep: NULL argument"); return GKS_E_ARG; }
    if (!s->initialised) { set_error("gks_timestep: state not initialised"); return GKS_E_STATE; }
    return s->fp32 ? timestep_impl<float>(s, s->m32, s->s32, dt) : timestep_impl<double>(s, s->m64, s->s64, dt);
}

extern "C" gks_status gks_residual(gks_state* s, double* out_l2) {
    if (!s || !out_l2) { set_error("gks_residual: NULL argument"); return GKS_E_ARG; }
    const int nblk = update_blocks(s->mesh->nc);
    std::vector<double> part((size_t)nblk * PART_N);
    GKS_CHECK_CUDA(cudaMemcpyAsync(part.data(), s->fp32 ? s->s32.part : s->s64.part, 8 * part.size(),
                                   cudaMemcpyDeviceToHost, s->stream));
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    for (int q = 0; q < 5; ++q) {
        double acc = 0.0;
        for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * PART_N + PART_RES + q];
        out_l2[q] = std::sqrt(acc / (double)s->mesh->nc);
    }
    return GKS_OK;
}

// --------------------------------------------------------------- adjoint --

namespace {
struct AdjLayout {
    size_t poly1, src, lx, lpf, lp, ld, own, lXs, lX1, lbn, lds, lwo, rev, fallback, total = 0;
    size_t add(size_t bytes) {
        size_t off = total;
        total += (bytes + 255) & ~(size_t)255;
        return off;
    }
};

AdjLayout adj_layout(int64_t nc, int64_t nf) {
    AdjLayout L;
    L.poly1 = L.add(8 * POLY_STRIDE * nc);
    L.src = L.add(8 * 40 * nc);
    L.lx = L.add(8 * 120 * nf);
    L.lpf = L.add(8 * 100 * nf);
    L.lp = L.add(8 * 50 * nc);
    L.ld = L.add(8 * 80 * nc);
    L.own = L.add(8 * 5 * nc);
    L.lXs = L.add(8 * XS * nc);
    L.lX1 = L.add(8 * XS * nc);
    L.lbn = L.add(8 * 60 * nc);
    L.lds = L.add(8 * 20 * nc);
    L.lwo = L.add(8 * 5 * nf);
    L.rev = L.add(4 * nc);
    L.fallback = L.add(4 * 2 * nc);  // positivity-fallback flags of both stages
    return L;
}
}  // namespace

extern "C" size_t gks_adjoint_workspace_bytes(const gks_state* s) {
    if (!s) return 0;
    return adj_layout(s->mesh->nc, s->mesh->nf).total;
}

// d_Ws, d_dWs: the step's stage state from the caller (NULL: recomputed)
static gks_status adjoint_impl(gks_state* s, double dt, const double* d_W, const double* d_dW, const double* d_Ws,
                               const double* d_dWs, const double* d_lamW, const double* d_lamdW, double* d_lamW_out,
                               double* d_lamdW_out, void* d_scratch, size_t scratch_bytes) {
    if (!s || !d_W || !d_dW || !d_lamW || !d_lamdW || !d_lamW_out || !d_lamdW_out || !d_scratch) {
        set_error("gks_adjoint_step: NULL argument");
        return GKS_E_ARG;
    }
    if (!(dt > 0.0) || !std::isfinite(dt)) { set_error("gks_adjoint_step: dt must be positive"); return GKS_E_ARG; }
    const gks_mesh& g = *s->mesh;
    const AdjLayout A = adj_layout(g.nc, g.nf);
    if (scratch_bytes < A.total) {
        set_error("gks_adjoint_step: scratch smaller than gks_adjoint_workspace_bytes");
        return GKS_E_NOMEM;
    }
    if (s->fp32 || g.ncase != 1 || (has_fixed(g) && !s->fixed_pinned)) {
        set_error("gks_adjoint_step: needs an FP64 state on a single-case mesh, and on a mesh with "
                  "fixed-state faces a fixed state set by gks_set_fixed_state");
        return GKS_E_UNSUPPORTED;
    }
    if (s->L.wslot) {
        set_error("gks_adjoint_step: the wall-constrained reconstruction (wall_constraint = 1) has no adjoint");
        return GKS_E_UNSUPPORTED;
    }
    order_after_caller(s);
    DevMesh<double>& m = s->m64;
    DevState<double>& st = s->s64;
    const int64_t nc = g.nc;
    char* base = static_cast<char*>(d_scratch);
    // reverse face slots: rev[f][c] = the local face of neighbour n = nbr(c, f)
    // that is the same face
    std::vector<int8_t>& rev = s->adj_rev;
    if (rev.size() != (size_t)4 * nc) {
        rev.assign((size_t)4 * nc, 0);
        for (int64_t c = 0; c < nc; ++c)
            for (int f = 0; f < 4; ++f) {
                const int64_t n = g.nbr[c * 4 + f];
                if (n < 0) continue;
                const int64_t fi = g.csr_face[c * 4 + f];
                for (int r = 0; r < 4; ++r)
                    if (g.csr_face[n * 4 + r] == fi) rev[(size_t)f * nc + c] = (int8_t)r;
            }
    }
    GKS_CHECK_CUDA(cudaMemcpyAsync(base + A.rev, rev.data(), rev.size(), cudaMemcpyHostToDevice, s->stream));
    // forward recomputation of the step's two reconstructions with the frozen dt
    gks_status r = init_impl<double>(s, m, st, d_W, d_dW);
    if (r != GKS_OK) return r;
    s->initialised = true;
    const double dth = dt;
    GKS_CHECK_CUDA(cudaMemcpyAsync(st.case_dt, &dth, 8, cudaMemcpyHostToDevice, s->stream));
    int32_t* fb = reinterpret_cast<int32_t*>(base + A.fallback);
    double* poly1 = reinterpret_cast<double*>(base + A.poly1);
    GKS_CHECK_CUDA(Launch<double>::recon(m, s->phys, st.X, nullptr, nullptr, st.poly, fb, nullptr, st.err,
                                         s->stream));
    GKS_CHECK_CUDA(cudaMemcpyAsync(poly1, st.poly, 8 * POLY_STRIDE * nc, cudaMemcpyDeviceToDevice, s->stream));
    if (d_Ws) {
        // the caller's stage state in place of the stage-1 flux and update
        GKS_CHECK_CUDA(Launch<double>::pack(d_Ws, d_dWs, st.Xs, nc, s->stream));
    } else {
        GKS_CHECK_CUDA(Launch<double>::flux(m, s->phys, st.X, st.poly, st.rec, st.case_dt, 0.0, 1, s->stream,
                                            s->flux_variant));
        GKS_CHECK_CUDA(Launch<double>::update1(m, s->phys, st, s->stream));
    }
    GKS_CHECK_CUDA(Launch<double>::recon(m, s->phys, st.Xs, nullptr, nullptr, st.poly, fb + nc, nullptr, st.err,
                                         s->stream));
    AdjBuffers b;
    b.poly1 = poly1;
    b.poly2 = st.poly;
    b.src = reinterpret_cast<double*>(base + A.src);
    b.lx = reinterpret_cast<double*>(base + A.lx);
    b.lpf = reinterpret_cast<double*>(base + A.lpf);
    b.lp = reinterpret_cast<double*>(base + A.lp);
    b.ld = reinterpret_cast<double*>(base + A.ld);
    b.own = reinterpret_cast<double*>(base + A.own);
    b.lXs = reinterpret_cast<double*>(base + A.lXs);
    b.lX1 = reinterpret_cast<double*>(base + A.lX1);
    b.lbn = reinterpret_cast<double*>(base + A.lbn);
    b.lds = reinterpret_cast<double*>(base + A.lds);
    b.lwo = reinterpret_cast<double*>(base + A.lwo);
    b.rev = reinterpret_cast<const int8_t*>(base + A.rev);
    b.fallback = fb;
    GKS_CHECK_CUDA(adjoint_reverse(m, s->phys, dt, b, st.X, st.Xs, d_lamW, d_lamdW, d_lamW_out, d_lamdW_out,
                                   s->stream));
    return gks_sync(s);
}

extern "C" gks_status gks_adjoint_step(gks_state* s, double dt, const double* d_W, const double* d_dW,
                                       const double* d_lamW, const double* d_lamdW, double* d_lamW_out,
                                       double* d_lamdW_out, void* d_scratch, size_t scratch_bytes) {
    return adjoint_impl(s, dt, d_W, d_dW, nullptr, nullptr, d_lamW, d_lamdW, d_lamW_out, d_lamdW_out, d_scratch,
                        scratch_bytes);
}

extern "C" gks_status gks_adjoint_step_staged(gks_state* s, double dt, const double* d_W, const double* d_dW,
                                              const double* d_Ws, const double* d_dWs, const double* d_lamW,
                                              const double* d_lamdW, double* d_lamW_out, double* d_lamdW_out,
                                              void* d_scratch, size_t scratch_bytes) {
    if (!d_Ws || !d_dWs) { set_error("gks_adjoint_step_staged: NULL stage state"); return GKS_E_ARG; }
    return adjoint_impl(s, dt, d_W, d_dW, d_Ws, d_dWs, d_lamW, d_lamdW, d_lamW_out, d_lamdW_out, d_scratch,
                        scratch_bytes);
}

extern "C" gks_status gks_get_stage_state(gks_state* s, double* d_Ws, double* d_dWs) {
    if (!s || !d_Ws || !d_dWs) { set_error("gks_get_stage_state: NULL argument"); return GKS_E_ARG; }
    if (s->fp32) { set_error("gks_get_stage_state: FP64 states only"); return GKS_E_UNSUPPORTED; }
    if (!s->stage_valid) { set_error("gks_get_stage_state: no step since the initialisation"); return GKS_E_STATE; }
    GKS_CHECK_CUDA(launch_unpack_avg(s->s64.Xs, d_Ws, s->mesh->nc, s->stream));
    GKS_CHECK_CUDA(Launch<double>::unpack_grad(s->s64.Xs, d_dWs, s->mesh->nc, s->stream));
    return gks_sync(s);
}

// ----------------------------------------------------------- diagnostics --

template <typename T>
static gks_status debug_recon_impl(gks_state* s, DevMesh<T>& m, DevState<T>& st, double* d_poly,
                                   double* d_slopes, int32_t* d_fallback) {
    const HostPhys& p = s->phys;
    const bool need_b = p.weno || p.order == 2;
    const int64_t nc = m.nc;
    if (!need_b) GKS_CHECK_CUDA(cudaMemsetAsync(st.slopes, 0, sizeof(T) * 15 * nc, s->stream));
    // a reordered state writes per-cell outputs in device order to the
    // staging buffer first, then gathers them into the caller's order
    double* stage = at<double>(s, s->L.stage);
    int32_t* fb = (d_fallback && s->dinv()) ? reinterpret_cast<int32_t*>(stage) : d_fallback;
    GKS_CHECK_CUDA(Launch<T>::recon(m, p, st.X, nullptr, need_b ? st.slopes : nullptr, st.poly, fb,
                                    nullptr, st.err, s->stream));
    if (fb != d_fallback) GKS_CHECK_CUDA(launch_rows_gather(fb, d_fallback, nc, 1, s->dinv(), s->stream));
    if (d_poly) GKS_CHECK_CUDA(Launch<T>::poly_to_double(st.poly, d_poly, nc, s->stream, s->dperm()));
    if (d_slopes) {
        if (s->dinv()) {
            GKS_CHECK_CUDA(Launch<T>::to_double(st.slopes, stage + nc, 15 * nc, s->stream));
            GKS_CHECK_CUDA(launch_rows_gather(stage + nc, d_slopes, nc, 30, s->dinv(), s->stream));
        } else {
            GKS_CHECK_CUDA(Launch<T>::to_double(st.slopes, d_slopes, 15 * nc, s->stream));
        }
    }
    return GKS_OK;
}

extern "C" gks_status gks_debug_reconstruct(gks_state* s, double* d_poly, double* d_slopes,
                                            int32_t* d_fallback) {
    if (!s) { set_error("gks_debug_reconstruct: state is NULL"); return GKS_E_ARG; }
    if (!s->initialised) { set_error("state not initialised"); return GKS_E_STATE; }
    gks_status st = s->fp32 ? debug_recon_impl<float>(s, s->m32, s->s32, d_poly, d_slopes, d_fallback)
                            : debug_recon_impl<double>(s, s->m64, s->s64, d_poly, d_slopes, d_fallback);
    if (st != GKS_OK) return st;
    if (s->own_stream) return gks_sync(s);
    return GKS_OK;
}

template <typename T>
static gks_status debug_rec_impl(gks_state* s, DevMesh<T>& m, DevState<T>& st, double dt, int stage,
                                 double* d_rec) {
    gks_status r = debug_recon_impl<T>(s, m, st, nullptr, nullptr, nullptr);
    if (r != GKS_OK) return r;
    GKS_CHECK_CUDA(Launch<T>::flux(m, s->phys, st.X, st.poly, st.rec, nullptr, dt, stage, s->stream, s->flux_variant));
    GKS_CHECK_CUDA(Launch<T>::rec_to_double(st.rec, at<int32_t>(s, s->L.perm), d_rec, m.nf, stage == 1 ? 40 : 20,
                                            &m, st.X, s->phys.gamma - 1.0, dt, s->stream));
    return GKS_OK;
}

extern "C" gks_status gks_debug_face_records(gks_state* s, double dt, int32_t stage, double* d_rec) {
    if (!s || !d_rec) { set_error("gks_debug_face_records: NULL argument"); return GKS_E_ARG; }
    if (!s->initialised) { set_error("state not initialised"); return GKS_E_STATE; }
    if ((stage != 1 && stage != 2) || !(dt > 0.0)) { set_error("stage must be 1 or 2 and dt > 0"); return GKS_E_ARG; }
    gks_status st = s->fp32 ? debug_rec_impl<float>(s, s->m32, s->s32, dt, stage, d_rec)
                            : debug_rec_impl<double>(s, s->m64, s->s64, dt, stage, d_rec);
    if (st != GKS_OK) return st;
    if (s->own_stream) return gks_sync(s);
    return GKS_OK;
}

extern "C" gks_status gks_debug_wait_timeout(gks_state* s, int32_t tries) {
    if (!s) { set_error("gks_debug_wait_timeout: state is NULL"); return GKS_E_ARG; }
    if (tries < 0 || tries > (1 << 16)) { set_error("gks_debug_wait_timeout: tries must be in [0, 65536]"); return GKS_E_ARG; }
    int32_t* err = s->fp32 ? s->s32.err : s->s64.err;
    order_after_caller(s);
    GKS_CHECK_CUDA(launch_wait_probe(err, tries, s->stream));
    const gks_status st = gks_sync(s);
    GKS_CHECK_CUDA(cudaMemsetAsync(err, 0, 4, s->stream));  // the state stays usable
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return st;
}

extern "C" gks_status gks_debug_grid_barrier_timeout(gks_state* s, int32_t tries) {
    if (!s) { set_error("gks_debug_grid_barrier_timeout: state is NULL"); return GKS_E_ARG; }
    if (tries < 0 || tries > (1 << 16)) {
        set_error("gks_debug_grid_barrier_timeout: tries must be in [0, 65536]");
        return GKS_E_ARG;
    }
    int32_t* err = s->fp32 ? s->s32.err : s->s64.err;
    order_after_caller(s);
    GKS_CHECK_CUDA(launch_grid_barrier_probe(reinterpret_cast<unsigned*>(s->ws + s->L.gbar), err, tries, s->stream));
    const gks_status st = gks_sync(s);
    GKS_CHECK_CUDA(cudaMemsetAsync(err, 0, 4, s->stream));  // the state stays usable
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return st;
}

// ------------------------------------------------------------- variants --

extern "C" gks_status gks_state_set_variant(gks_state* s, int32_t face_order, int32_t flux_blocks,
                                            int32_t slopes_pass) {
    if (!s) { set_error("gks_state_set_variant: state is NULL"); return GKS_E_ARG; }
    if ((face_order != 0 && face_order != 1) || (flux_blocks != 2 && flux_blocks != 3) ||
        (slopes_pass != 0 && slopes_pass != 1)) {
        set_error("gks_state_set_variant: face_order and slopes_pass must be 0 or 1, flux_blocks 2 or 3");
        return GKS_E_ARG;
    }
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    s->flux_variant = flux_blocks == 3 ? 1 : 0;
    s->slopes_pass = slopes_pass;
    if (face_order != s->face_order) {
        s->face_order = face_order;
        gks_status st = s->fp32 ? upload_faces<float>(s) : upload_faces<double>(s);
        if (st != GKS_OK) return st;
    }
    return GKS_OK;
}

extern "C" gks_status gks_state_set_fused(gks_state* s, int32_t fused) {
    if (!s) { set_error("gks_state_set_fused: state is NULL"); return GKS_E_ARG; }
    if (fused != 0 && fused != 1) { set_error("gks_state_set_fused: fused must be 0 or 1"); return GKS_E_ARG; }
    if (fused && !(s->fp32 && !s->ops64)) {
        set_error("gks_state_set_fused: the one-launch stage exists for precision 1 only");
        return GKS_E_ARG;
    }
    if (fused != s->fused && s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    s->fused = fused;
    return GKS_OK;
}

extern "C" gks_status gks_state_get_fused(const gks_state* s, int32_t* fused) {
    if (!s || !fused) { set_error("gks_state_get_fused: NULL argument"); return GKS_E_ARG; }
    *fused = s->fused;
    return GKS_OK;
}

// Re-numbers the device cells (FP32 bulk): the mesh arrays are uploaded in
// the new order and the per-cell state (averages, working state, fixed
// state) is carried over by an exact gather, so the run continues unchanged.
template <typename T>
static gks_status reorder_impl(gks_state* s, DevMesh<T>& m, DevState<T>& st, int order) {
    const gks_mesh& g = *s->mesh;
    const int64_t nc = g.nc;
    std::vector<int32_t> np = cell_permutation(g, order);  // new device cell -> caller's cell
    std::vector<int32_t> map((size_t)nc);                  // new device cell -> old device cell
    for (int64_t d = 0; d < nc; ++d) map[d] = (int32_t)s->dev(np[d]);
    char* sb = s->ws + s->L.stage;
    const size_t wd_b = 8 * 5 * (size_t)nc, x_b = sizeof(T) * Stride<T>::xs * (size_t)nc;
    char* map_d = sb + wd_b + 2 * x_b;
    if (s->initialised) {
        GKS_CHECK_CUDA(cudaMemcpyAsync(sb, st.Wd, wd_b, cudaMemcpyDeviceToDevice, s->stream));
        GKS_CHECK_CUDA(cudaMemcpyAsync(sb + wd_b, st.X, x_b, cudaMemcpyDeviceToDevice, s->stream));
    }
    if (m.fixed) GKS_CHECK_CUDA(cudaMemcpyAsync(sb + wd_b + x_b, m.fixed, x_b, cudaMemcpyDeviceToDevice, s->stream));
    GKS_CHECK_CUDA(cudaMemcpyAsync(map_d, map.data(), 4 * (size_t)nc, cudaMemcpyHostToDevice, s->stream));
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));  // map dies with this call
    s->cell_order = order;
    if (order == 0) {
        s->cperm.clear();
        s->cinv.clear();
    } else {
        s->cperm = np;
        s->cinv.assign((size_t)nc, 0);
        for (int64_t d = 0; d < nc; ++d) s->cinv[np[d]] = (int32_t)d;
    }
    gks_status r = upload_mesh<T>(s);
    if (r != GKS_OK) return r;
    const int32_t* mp = reinterpret_cast<const int32_t*>(map_d);
    if (s->initialised) {
        for (int q = 0; q < 5; ++q)
            GKS_CHECK_CUDA(launch_rows_gather(sb + q * 8 * (size_t)nc, st.Wd + q * nc, nc, 2, mp, s->stream));
        GKS_CHECK_CUDA(launch_rows_gather(sb + wd_b, st.X, nc, (int)(sizeof(T) * Stride<T>::xs / 4), mp, s->stream));
    }
    if (m.fixed)
        GKS_CHECK_CUDA(launch_rows_gather(sb + wd_b + x_b, const_cast<T*>(m.fixed), nc,
                                          (int)(sizeof(T) * Stride<T>::xs / 4), mp, s->stream));
    GKS_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return GKS_OK;
}

extern "C" gks_status gks_state_set_cell_order(gks_state* s, int32_t order) {
    if (!s) { set_error("gks_state_set_cell_order: state is NULL"); return GKS_E_ARG; }
    if (order < 0 || order > 2) { set_error("gks_state_set_cell_order: order must be 0, 1 or 2"); return GKS_E_ARG; }
    if (order == s->cell_order) return GKS_OK;
    if (!s->fp32) {
        set_error("gks_state_set_cell_order: FP64 states keep the caller's cell order");
        return GKS_E_UNSUPPORTED;
    }
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    order_after_caller(s);
    return reorder_impl<float>(s, s->m32, s->s32, order);
}

extern "C" gks_status gks_state_get_cell_order(const gks_state* s, int32_t* order) {
    if (!s || !order) { set_error("gks_state_get_cell_order: NULL argument"); return GKS_E_ARG; }
    *order = s->cell_order;
    return GKS_OK;
}

template <typename T>
static gks_status snapshot(gks_state* s, DevState<T>& st, bool save) {
    const int64_t nc = s->mesh->nc, nk = s->mesh->ncase;
    char* base = s->ws + s->L.stage;
    struct Item { void* dev; size_t bytes; };
    const Item items[] = {{st.Wd, 8 * 5 * (size_t)nc},
                          {st.X, sizeof(T) * Stride<T>::xs * (size_t)nc},
                          {st.case_t, 8 * (size_t)nk},
                          {st.case_dt, 8 * (size_t)nk},
                          {st.case_dtmin, 8 * (size_t)nk},
                          {st.ctrl, 8 * (size_t)CTRL_N}};
    size_t off = 0;
    for (const Item& it : items) {
        void* dst = save ? (void*)(base + off) : it.dev;
        const void* src = save ? it.dev : (const void*)(base + off);
        GKS_CHECK_CUDA(cudaMemcpyAsync(dst, src, it.bytes, cudaMemcpyDeviceToDevice, s->stream));
        off += it.bytes;
    }
    return GKS_OK;
}

extern "C" gks_status gks_autotune(gks_state* s, int32_t steps, int32_t* face_order, int32_t* flux_blocks,
                                   int32_t* slopes_pass, double* ms_per_step) {
    if (!s || steps < 1) { set_error("gks_autotune: NULL state or steps < 1"); return GKS_E_ARG; }
    if (!s->initialised) { set_error("gks_autotune: state not initialised"); return GKS_E_STATE; }
    // variant v < 8: face order v & 1, slopes pass (v >> 1) & 1, flux blocks
    // 3 - (v >> 2); v = 8, 9: each stage as one launch, face order v & 1
    int orders[GKS_NVARIANTS], passes[GKS_NVARIANTS], blocks[GKS_NVARIANTS], fused[GKS_NVARIANTS];
    for (int v = 0; v < GKS_NVARIANTS; ++v) {
        orders[v] = v & 1;
        passes[v] = v < 8 ? (v >> 1) & 1 : 0;
        blocks[v] = v < 8 ? 3 - (v >> 2) : 3;
        fused[v] = v >= 8;
    }
    const bool can_fuse = s->fp32 && !s->ops64;
    const int nvar = s->fp32 ? 8 : 4;  // the FP64 flux has a single variant
    if (ms_per_step)
        for (int v = 0; v < GKS_NVARIANTS; ++v) ms_per_step[v] = NAN;
    gks_status r = s->fp32 ? snapshot<float>(s, s->s32, true) : snapshot<double>(s, s->s64, true);
    if (r != GKS_OK) return r;
    double best = INFINITY;
    int bi = 0;
    cudaEvent_t e0, e1;
    GKS_CHECK_CUDA(cudaEventCreate(&e0));
    GKS_CHECK_CUDA(cudaEventCreate(&e1));
    for (int v = 0; v < GKS_NVARIANTS && r == GKS_OK; ++v) {
        if (v >= nvar && !(fused[v] && can_fuse)) continue;
        r = gks_state_set_variant(s, orders[v], blocks[v], passes[v]);
        if (r == GKS_OK && s->fp32 && !s->ops64) r = gks_state_set_fused(s, fused[v]);
        if (r == GKS_OK) r = s->fp32 ? snapshot<float>(s, s->s32, false) : snapshot<double>(s, s->s64, false);
        if (r == GKS_OK) r = gks_step(s, 1, 0.0, 0.0);  // graph capture + warm-up
        if (r != GKS_OK) break;
        cudaEventRecord(e0, s->stream);
        r = gks_step(s, steps, 0.0, 0.0);
        cudaEventRecord(e1, s->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { set_error("gks_autotune: event"); r = GKS_E_CUDA; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / steps;
        if (ms_per_step) ms_per_step[v] = per;
        if (per < best) { best = per; bi = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != GKS_OK) return r;
    r = gks_state_set_variant(s, orders[bi], blocks[bi], passes[bi]);
    if (r == GKS_OK && can_fuse) r = gks_state_set_fused(s, fused[bi]);
    if (r == GKS_OK) r = s->fp32 ? snapshot<float>(s, s->s32, false) : snapshot<double>(s, s->s64, false);
    if (r != GKS_OK) return r;
    GKS_CHECK_CUDA(cudaMemsetAsync(s->fp32 ? (void*)s->s32.err : (void*)s->s64.err, 0, 4, s->stream));
    if (face_order) *face_order = orders[bi];
    if (flux_blocks) *flux_blocks = blocks[bi];
    if (slopes_pass) *slopes_pass = passes[bi];
    return gks_sync(s);
}

extern "C" gks_status gks_autotune_orders(gks_state* s, int32_t steps, int32_t* cell_order, int32_t* face_order,
                                          int32_t* flux_blocks, int32_t* slopes_pass, double* ms_per_order) {
    if (!s || steps < 1) { set_error("gks_autotune_orders: NULL state or steps < 1"); return GKS_E_ARG; }
    if (!s->initialised) { set_error("gks_autotune_orders: state not initialised"); return GKS_E_STATE; }
    const int norder = s->fp32 ? 3 : 1;
    double best = INFINITY;
    int bo = 0;
    int32_t bfo = 0, bfb = 3, bsp = 0, bfu = 0;
    for (int o = 0; o < norder; ++o) {
        gks_status r = gks_state_set_cell_order(s, o);
        if (r != GKS_OK) return r;
        int32_t fo = 0, fb = 3, sp = 0;
        double ms[GKS_NVARIANTS];
        r = gks_autotune(s, steps, &fo, &fb, &sp, ms);
        if (r != GKS_OK) return r;
        double m = INFINITY;
        for (int v = 0; v < GKS_NVARIANTS; ++v) m = std::fmin(m, ms[v]);  // fmin skips the untried (NaN)
        if (ms_per_order) ms_per_order[o] = m;
        if (m < best) {
            best = m;
            bo = o;
            bfo = fo;
            bfb = fb;
            bsp = sp;
            bfu = s->fused;
        }
    }
    gks_status r = gks_state_set_cell_order(s, bo);
    if (r == GKS_OK) r = gks_state_set_variant(s, bfo, bfb, bsp);
    if (r == GKS_OK && s->fp32 && !s->ops64) r = gks_state_set_fused(s, bfu);
    if (r != GKS_OK) return r;
    if (cell_order) *cell_order = bo;
    if (face_order) *face_order = bfo;
    if (flux_blocks) *flux_blocks = bfb;
    if (slopes_pass) *slopes_pass = bsp;
    return gks_sync(s);
}
