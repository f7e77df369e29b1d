// gks_mesh.cpp -- host mesh setup of libgks: face matching, canonical
// numbering and orientation, neighbours, and FP64 geometry.
//
// Paper: Sec. 2.1 (cells bounded by four triangular faces, face Gauss rule
// (xi, eta) = (1/6,1/6), (2/3,1/6), (1/6,2/3) with weights 1/3 of the
// reference area), Sec. 5 (inscribed-radius estimate 3|Omega| / sum |Gamma|).
//
// Faces are matched with hash tables keyed by the ascending vertex-id
// triple and the image shifts of the second and third vertex relative to the
// first, which identifies a face of a periodic mesh independently of which
// periodic copy a cell refers to.  The set-up runs on the host's hardware
// threads: the half-faces are split into partitions by key hash and each
// partition is matched by its own table, in ascending cell order; the faces
// are then put in key order by buckets of their first vertex id, each bucket
// sorted on its own.  Every loop writes disjoint entries, and the one sum
// (the inscribed-radius denominator) adds a cell's face areas in ascending
// face order as a serial loop over faces would, so the result does not
// depend on the number of threads.  The canonical numbering and orientation
// rules are fixed by the ABI so that connectivity is reproducible bit for
// bit: faces in ascending key order; the raw normal (x1 - x0) x (x2 - x0) of
// the face's vertices in ascending id order, flipped so that its first
// nonzero component is positive; "left" is the cell it points out of.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <system_error>
#include <thread>
#include <unordered_map>

#include "gks_internal.h"

namespace gks {
namespace {

struct FaceKey {
    int64_t v[3];
    int8_t img[6];  // shift of v[1], v[2] relative to v[0]
    bool operator==(const FaceKey& o) const {
        return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2] &&
               std::memcmp(img, o.img, 6) == 0;
    }
    bool operator<(const FaceKey& o) const {
        for (int i = 0; i < 3; ++i)
            if (v[i] != o.v[i]) return v[i] < o.v[i];
        for (int i = 0; i < 6; ++i)
            if (img[i] != o.img[i]) return img[i] < o.img[i];
        return false;
    }
};

struct FaceKeyHash {
    size_t operator()(const FaceKey& k) const {
        uint64_t h = 1469598103934665603ull;
        auto mix = [&](uint64_t x) {
            h ^= x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        };
        mix((uint64_t)k.v[0]);
        mix((uint64_t)k.v[1]);
        mix((uint64_t)k.v[2]);
        uint64_t s = 0;
        for (int i = 0; i < 6; ++i) s = (s << 8) | (uint8_t)k.img[i];
        mix(s);
        return (size_t)h;
    }
};

struct Side {
    int64_t cell;
    int local;        // local face index = local vertex opposite
    int8_t base[3];   // image shift of the face's first vertex in this cell
};

struct FaceEntry {
    FaceKey key;
    Side side[2];
    int count;
};

inline void vsub(const double* a, const double* b, double* c) {
    c[0] = a[0] - b[0];
    c[1] = a[1] - b[1];
    c[2] = a[2] - b[2];
}

struct HalfFace {
    FaceKey key;
    Side side;
};

int64_t host_threads(int64_t n) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    return std::min<int64_t>((int64_t)hw, std::max<int64_t>(1, n / 16384));
}

// fn(t, lo, hi) over nthr contiguous ranges of [0, n); range 0 on the calling
// thread, and any range whose thread cannot be started runs inline too
template <typename Fn>
void run_ranges(int64_t n, int64_t nthr, Fn fn) {
    const int64_t chunk = (n + nthr - 1) / nthr;
    std::vector<std::thread> pool;
    pool.reserve((size_t)nthr);
    for (int64_t t = 1; t < nthr; ++t) {
        const int64_t lo = std::min(n, t * chunk), hi = std::min(n, (t + 1) * chunk);
        try {
            pool.emplace_back(fn, t, lo, hi);
        } catch (const std::system_error&) {
            fn(t, lo, hi);
        }
    }
    fn((int64_t)0, (int64_t)0, std::min(n, chunk));
    for (auto& th : pool) th.join();
}

// The first failure of a parallel loop: the smallest index at which one was
// found, and its message (set_error is per thread, so workers only record).
struct FirstError {
    int64_t at = INT64_MAX;
    const char* msg = nullptr;
    void note(int64_t i, const char* m) {
        if (i < at) { at = i; msg = m; }
    }
};

gks_status report(const std::vector<FirstError>& errs) {
    const FirstError* best = nullptr;
    for (const FirstError& e : errs)
        if (e.msg && (!best || e.at < best->at)) best = &e;
    if (!best) return GKS_OK;
    set_error(best->msg);
    return GKS_E_MESH;
}

}  // namespace

gks_status build_mesh(gks_mesh& m) {
    const int64_t nc = m.nc;
    const int64_t nthr = host_threads(nc);
    std::vector<FirstError> errs((size_t)nthr);

    // ---- half-faces: cell c's local face f is the face opposite vertex f ---
    std::vector<HalfFace> half((size_t)nc * 4);
    run_ranges(nc, nthr, [&](int64_t t, int64_t lo, int64_t hi) {
        for (int64_t c = lo; c < hi; ++c) {
            for (int f = 0; f < 4; ++f) {
                int lv[3], k = 0;
                for (int v = 0; v < 4; ++v)
                    if (v != f) lv[k++] = v;
                std::sort(lv, lv + 3, [&](int a, int b) { return m.tet[c * 4 + a] < m.tet[c * 4 + b]; });
                HalfFace& h = half[(size_t)(c * 4 + f)];
                for (int i = 0; i < 3; ++i) h.key.v[i] = m.tet[c * 4 + lv[i]];
                if (h.key.v[0] == h.key.v[1] || h.key.v[1] == h.key.v[2])
                    errs[(size_t)t].note(c, "gks_mesh_create: a tetrahedron repeats a vertex id");
                h.side.cell = c;
                h.side.local = f;
                for (int a = 0; a < 3; ++a) {
                    int8_t b0 = m.shift[(c * 4 + lv[0]) * 3 + a];
                    h.side.base[a] = b0;
                    h.key.img[a] = (int8_t)(m.shift[(c * 4 + lv[1]) * 3 + a] - b0);
                    h.key.img[3 + a] = (int8_t)(m.shift[(c * 4 + lv[2]) * 3 + a] - b0);
                }
            }
        }
    });
    if (gks_status st = report(errs); st != GKS_OK) return st;

    // ---- match: partitions by key hash, half-faces ascending in each -------
    const int64_t nh = nc * 4;
    const int64_t nparts = nthr == 1 ? 1 : 8 * nthr;
    std::vector<int32_t> part((size_t)nh);
    std::vector<int64_t> cnt((size_t)(nthr * nparts), 0);
    run_ranges(nh, nthr, [&](int64_t t, int64_t lo, int64_t hi) {
        FaceKeyHash hf;
        for (int64_t i = lo; i < hi; ++i) {
            const int32_t p = (int32_t)(hf(half[(size_t)i].key) % (size_t)nparts);
            part[(size_t)i] = p;
            ++cnt[(size_t)(t * nparts + p)];
        }
    });
    // offsets partition-major, range-minor: each partition lists its
    // half-faces in ascending index order
    std::vector<int64_t> off((size_t)(nthr * nparts));
    std::vector<int64_t> part_first((size_t)nparts + 1, 0);
    {
        int64_t o = 0;
        for (int64_t p = 0; p < nparts; ++p) {
            part_first[(size_t)p] = o;
            for (int64_t t = 0; t < nthr; ++t) {
                off[(size_t)(t * nparts + p)] = o;
                o += cnt[(size_t)(t * nparts + p)];
            }
        }
        part_first[(size_t)nparts] = o;
    }
    std::vector<int64_t> order((size_t)nh);
    run_ranges(nh, nthr, [&](int64_t t, int64_t lo, int64_t hi) {
        int64_t* o = &off[(size_t)(t * nparts)];
        for (int64_t i = lo; i < hi; ++i) order[(size_t)(o[part[(size_t)i]]++)] = i;
    });
    part.clear();
    part.shrink_to_fit();
    std::vector<std::vector<FaceEntry>> pfaces((size_t)nparts);
    run_ranges(nparts, nthr, [&](int64_t t, int64_t lo, int64_t hi) {
        for (int64_t p = lo; p < hi; ++p) {
            const int64_t b = part_first[(size_t)p], e = part_first[(size_t)p + 1];
            std::unordered_map<FaceKey, int64_t, FaceKeyHash> index;
            index.reserve((size_t)(e - b));
            std::vector<FaceEntry>& faces = pfaces[(size_t)p];
            faces.reserve((size_t)((e - b) / 2 + 16));
            for (int64_t j = b; j < e; ++j) {
                const HalfFace& h = half[(size_t)order[(size_t)j]];
                auto it = index.find(h.key);
                if (it == index.end()) {
                    index.emplace(h.key, (int64_t)faces.size());
                    FaceEntry fe;
                    fe.key = h.key;
                    fe.side[0] = h.side;
                    fe.count = 1;
                    faces.push_back(fe);
                } else {
                    FaceEntry& fe = faces[(size_t)it->second];
                    if (fe.count >= 2)
                        errs[(size_t)t].note(order[(size_t)j] / 4,
                                             "gks_mesh_create: a face is shared by more than two cells");
                    else
                        fe.side[fe.count++] = h.side;
                }
            }
        }
    });
    half.clear();
    half.shrink_to_fit();
    order.clear();
    order.shrink_to_fit();
    if (gks_status st = report(errs); st != GKS_OK) return st;

    // ---- key order: buckets of the first vertex id, each sorted -----------
    int64_t nf = 0;
    for (const auto& pf : pfaces) nf += (int64_t)pf.size();
    // bucket = first vertex id / width: ascending buckets hold ascending keys
    const int64_t nv = std::max<int64_t>(1, m.nv);
    const int64_t width = std::max<int64_t>(1, (nv * 64 + nf) / (nf + 1));  // ~64 faces a bucket
    const int64_t nbuck = (nv + width - 1) / width;
    auto bucket_of = [&](const FaceEntry& fe) { return fe.key.v[0] / width; };
    std::vector<int64_t> bcnt((size_t)nbuck + 1, 0);
    for (const auto& pf : pfaces)
        for (const FaceEntry& fe : pf) ++bcnt[(size_t)bucket_of(fe) + 1];
    for (int64_t b = 0; b < nbuck; ++b) bcnt[(size_t)b + 1] += bcnt[(size_t)b];
    std::vector<FaceEntry> faces((size_t)nf);
    {
        std::vector<int64_t> fill(bcnt.begin(), bcnt.end() - 1);
        for (auto& pf : pfaces) {
            for (const FaceEntry& fe : pf) faces[(size_t)(fill[(size_t)bucket_of(fe)]++)] = fe;
            std::vector<FaceEntry>().swap(pf);
        }
    }
    run_ranges(nbuck, host_threads(nf), [&](int64_t, int64_t lo, int64_t hi) {
        for (int64_t b = lo; b < hi; ++b)
            std::sort(faces.begin() + bcnt[(size_t)b], faces.begin() + bcnt[(size_t)b + 1],
                      [](const FaceEntry& a, const FaceEntry& c) { return a.key < c.key; });
    });

    m.nf = nf;
    m.face_v.assign((size_t)nf * 3, 0);
    m.face_lr.assign((size_t)nf * 2, -1);
    m.bkind.assign((size_t)nf, 0);
    m.nbr.assign((size_t)nc * 4, -1);
    m.nbr_img.assign((size_t)nc * 12, 0);
    m.csr_face.assign((size_t)nc * 4, -1);
    m.csr_sign.assign((size_t)nc * 4, 0);
    m.farea.assign((size_t)nf, 0.0);
    m.fnorm.assign((size_t)nf * 3, 0.0);
    m.gp_l.assign((size_t)nf * 9, 0.0);
    m.gp_r.assign((size_t)nf * 9, 0.0);
    std::vector<double> gp_face((size_t)nf * 9);
    std::vector<int8_t> base_lr((size_t)nf * 6, 0);

    // Gauss points as barycentric weights of the ascending-id vertices
    static const double BARY[3][3] = {{2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0},
                                      {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0},
                                      {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0}};
    // ---- faces: geometry, orientation, neighbours (each face writes its own
    // entries and its cells' slots of its two local faces) -------------------
    const int64_t fthr = host_threads(nf);
    std::vector<FirstError> ferrs((size_t)fthr);
    std::vector<int64_t> nbf_part((size_t)fthr, 0);
    run_ranges(nf, fthr, [&](int64_t t, int64_t lo, int64_t hi) {
        FirstError& err = ferrs[(size_t)t];
        for (int64_t fi = lo; fi < hi; ++fi) {
            const FaceEntry& e = faces[(size_t)fi];
            const double* P = m.per(e.side[0].cell);
            if (e.count == 2 && m.cell_case[e.side[1].cell] != m.cell_case[e.side[0].cell]) {
                err.note(fi, "gks_mesh_create: cells of different cases share a face");
                return;
            }
            double x[3][3];
            for (int a = 0; a < 3; ++a) {
                x[0][a] = m.xyz[e.key.v[0] * 3 + a];
                x[1][a] = m.xyz[e.key.v[1] * 3 + a] + (double)e.key.img[a] * P[a];
                x[2][a] = m.xyz[e.key.v[2] * 3 + a] + (double)e.key.img[3 + a] * P[a];
            }
            double e1[3], e2[3], n[3];
            vsub(x[1], x[0], e1);
            vsub(x[2], x[0], e2);
            n[0] = e1[1] * e2[2] - e1[2] * e2[1];
            n[1] = e1[2] * e2[0] - e1[0] * e2[2];
            n[2] = e1[0] * e2[1] - e1[1] * e2[0];
            bool up = n[0] > 0.0 || (n[0] == 0.0 && (n[1] > 0.0 || (n[1] == 0.0 && n[2] > 0.0)));
            if (!up) {
                n[0] = -n[0];
                n[1] = -n[1];
                n[2] = -n[2];
            }
            double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            if (!(len > 0.0)) {
                err.note(fi, "gks_mesh_create: degenerate face");
                return;
            }
            for (int i = 0; i < 3; ++i) m.face_v[fi * 3 + i] = e.key.v[i];
            m.farea[fi] = 0.5 * len;
            for (int a = 0; a < 3; ++a) m.fnorm[fi * 3 + a] = n[a] / len;
            for (int k = 0; k < 3; ++k)
                for (int a = 0; a < 3; ++a)
                    gp_face[fi * 9 + k * 3 + a] =
                        BARY[k][0] * x[0][a] + BARY[k][1] * x[1][a] + BARY[k][2] * x[2][a];
            int local_lr[2] = {-1, -1};
            for (int s = 0; s < e.count; ++s) {
                const Side& sd = e.side[s];
                const int64_t c = sd.cell;
                const int64_t o = m.tet[c * 4 + sd.local];
                double d[3];
                for (int a = 0; a < 3; ++a) {
                    double xo = m.xyz[o * 3 + a] +
                                (double)(m.shift[(c * 4 + sd.local) * 3 + a] - sd.base[a]) * P[a];
                    d[a] = xo - x[0][a];
                }
                double side = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
                if (side == 0.0) {
                    err.note(fi, "gks_mesh_create: flat tetrahedron");
                    return;
                }
                int lr = side < 0.0 ? 0 : 1;  // the normal leaves the left cell
                if (m.face_lr[fi * 2 + lr] != -1) {
                    err.note(fi, "gks_mesh_create: two cells on the same side of a face");
                    return;
                }
                m.face_lr[fi * 2 + lr] = c;
                local_lr[lr] = sd.local;
                for (int a = 0; a < 3; ++a) base_lr[fi * 6 + lr * 3 + a] = sd.base[a];
                m.csr_face[c * 4 + sd.local] = fi;
                m.csr_sign[c * 4 + sd.local] = (int8_t)(lr == 0 ? 1 : -1);
            }
            if (e.count == 2) {
                int64_t cl = m.face_lr[fi * 2], cr = m.face_lr[fi * 2 + 1];
                m.nbr[cl * 4 + local_lr[0]] = cr;
                m.nbr[cr * 4 + local_lr[1]] = cl;
                for (int a = 0; a < 3; ++a) {
                    int d = base_lr[fi * 6 + a] - base_lr[fi * 6 + 3 + a];
                    m.nbr_img[(cl * 4 + local_lr[0]) * 3 + a] = d;
                    m.nbr_img[(cr * 4 + local_lr[1]) * 3 + a] = -d;
                }
            } else {
                ++nbf_part[(size_t)t];
            }
        }
    });
    if (gks_status st = report(ferrs); st != GKS_OK) return st;
    m.nbf = 0;
    for (int64_t v : nbf_part) m.nbf += v;
    std::vector<FaceEntry>().swap(faces);

    // ---- cell geometry -------------------------------------------------
    m.vol.assign((size_t)nc, 0.0);
    m.cen.assign((size_t)nc * 3, 0.0);
    m.mom2.assign((size_t)nc * 6, 0.0);
    m.dr.assign((size_t)nc, 0.0);
    std::fill(errs.begin(), errs.end(), FirstError());
    run_ranges(nc, nthr, [&](int64_t t, int64_t lo, int64_t hi) {
        for (int64_t c = lo; c < hi; ++c) {
            const double* P = m.per(c);
            double x[4][3];
            for (int v = 0; v < 4; ++v) {
                int64_t id = m.tet[c * 4 + v];
                for (int a = 0; a < 3; ++a)
                    x[v][a] = m.xyz[id * 3 + a] + (double)m.shift[(c * 4 + v) * 3 + a] * P[a];
            }
            double a1[3], a2[3], a3[3];
            vsub(x[1], x[0], a1);
            vsub(x[2], x[0], a2);
            vsub(x[3], x[0], a3);
            double det = a1[0] * (a2[1] * a3[2] - a2[2] * a3[1]) - a1[1] * (a2[0] * a3[2] - a2[2] * a3[0]) +
                         a1[2] * (a2[0] * a3[1] - a2[1] * a3[0]);
            if (!(det > 0.0)) {
                errs[(size_t)t].note(c, "gks_mesh_create: tetrahedron with non-positive volume");
                return;
            }
            m.vol[c] = det / 6.0;
            double ce[3];
            for (int a = 0; a < 3; ++a) ce[a] = 0.25 * ((x[0][a] + x[1][a]) + (x[2][a] + x[3][a]));
            for (int a = 0; a < 3; ++a) m.cen[c * 3 + a] = ce[a];
            // covariance of the uniform measure on a simplex with centred
            // vertices y_v: (1/20) sum_v y_v y_v^T
            double S[6] = {0, 0, 0, 0, 0, 0};
            for (int v = 0; v < 4; ++v) {
                double y0 = x[v][0] - ce[0], y1 = x[v][1] - ce[1], y2 = x[v][2] - ce[2];
                S[0] += y0 * y0;
                S[1] += y0 * y1;
                S[2] += y0 * y2;
                S[3] += y1 * y1;
                S[4] += y1 * y2;
                S[5] += y2 * y2;
            }
            for (int q = 0; q < 6; ++q) m.mom2[c * 6 + q] = S[q] / 20.0;
        }
    });
    if (gks_status st = report(errs); st != GKS_OK) return st;
    // Gauss points relative to each side's centroid
    run_ranges(nf, fthr, [&](int64_t, int64_t lo, int64_t hi) {
        for (int64_t fi = lo; fi < hi; ++fi) {
            for (int lr = 0; lr < 2; ++lr) {
                int64_t c = m.face_lr[fi * 2 + lr];
                if (c < 0) continue;
                const double* P = m.per(c);
                double* out = lr == 0 ? &m.gp_l[fi * 9] : &m.gp_r[fi * 9];
                for (int k = 0; k < 3; ++k)
                    for (int a = 0; a < 3; ++a)
                        out[k * 3 + a] = gp_face[fi * 9 + k * 3 + a] +
                                         (double)base_lr[fi * 6 + lr * 3 + a] * P[a] - m.cen[c * 3 + a];
            }
        }
    });
    // dr = 3 |Omega| / sum of the cell's face areas, summed in ascending face
    // order (a face that joins a cell to its own periodic image counts twice)
    run_ranges(nc, nthr, [&](int64_t, int64_t lo, int64_t hi) {
        for (int64_t c = lo; c < hi; ++c) {
            int64_t fs[4];
            for (int f = 0; f < 4; ++f) fs[f] = m.csr_face[c * 4 + f];
            std::sort(fs, fs + 4);
            double sum = 0.0;
            for (int f = 0; f < 4; ++f) sum += m.farea[fs[f]];
            m.dr[c] = 3.0 * m.vol[c] / sum;
        }
    });
    return GKS_OK;
}

}  // namespace gks
