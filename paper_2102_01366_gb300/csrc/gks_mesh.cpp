// gks_mesh.cpp -- host mesh setup of libgks: face matching, canonical
// numbering and orientation, neighbours, and FP64 geometry.
//
// Paper: Sec. 2.1 (cells bounded by four triangular faces, face Gauss rule
// (xi, eta) = (1/6,1/6), (2/3,1/6), (1/6,2/3) with weights 1/3 of the
// reference area), Sec. 5 (inscribed-radius estimate 3|Omega| / sum |Gamma|).
//
// Faces are matched with a hash table keyed by the ascending vertex-id
// triple and the image shifts of the second and third vertex relative to the
// first, which identifies a face of a periodic mesh independently of which
// periodic copy a cell refers to.  The canonical numbering and orientation
// rules are fixed by the ABI so that connectivity is reproducible bit for
// bit: faces in ascending key order; the raw normal (x1 - x0) x (x2 - x0) of
// the face's vertices in ascending id order, flipped so that its first
// nonzero component is positive; "left" is the cell it points out of.
#include <algorithm>
#include <cmath>
#include <cstring>
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

}  // namespace

gks_status build_mesh(gks_mesh& m) {
    const int64_t nc = m.nc;
    // ---- match faces -------------------------------------------------
    std::unordered_map<FaceKey, int64_t, FaceKeyHash> index;
    index.reserve((size_t)(nc * 3));
    std::vector<FaceEntry> faces;
    faces.reserve((size_t)(nc * 2 + 16));
    for (int64_t c = 0; c < nc; ++c) {
        for (int f = 0; f < 4; ++f) {
            int lv[3], k = 0;
            for (int v = 0; v < 4; ++v)
                if (v != f) lv[k++] = v;
            std::sort(lv, lv + 3, [&](int a, int b) { return m.tet[c * 4 + a] < m.tet[c * 4 + b]; });
            FaceKey key;
            for (int i = 0; i < 3; ++i) key.v[i] = m.tet[c * 4 + lv[i]];
            if (key.v[0] == key.v[1] || key.v[1] == key.v[2]) {
                set_error("gks_mesh_create: a tetrahedron repeats a vertex id");
                return GKS_E_MESH;
            }
            Side s;
            s.cell = c;
            s.local = f;
            for (int a = 0; a < 3; ++a) {
                int8_t b0 = m.shift[(c * 4 + lv[0]) * 3 + a];
                s.base[a] = b0;
                key.img[a] = (int8_t)(m.shift[(c * 4 + lv[1]) * 3 + a] - b0);
                key.img[3 + a] = (int8_t)(m.shift[(c * 4 + lv[2]) * 3 + a] - b0);
            }
            auto it = index.find(key);
            if (it == index.end()) {
                index.emplace(key, (int64_t)faces.size());
                FaceEntry e;
                e.key = key;
                e.side[0] = s;
                e.count = 1;
                faces.push_back(e);
            } else {
                FaceEntry& e = faces[(size_t)it->second];
                if (e.count >= 2) {
                    set_error("gks_mesh_create: a face is shared by more than two cells");
                    return GKS_E_MESH;
                }
                e.side[e.count++] = s;
            }
        }
    }
    index.clear();
    std::sort(faces.begin(), faces.end(),
              [](const FaceEntry& a, const FaceEntry& b) { return a.key < b.key; });
    const int64_t nf = (int64_t)faces.size();
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
    m.nbf = 0;

    // Gauss points as barycentric weights of the ascending-id vertices
    static const double BARY[3][3] = {{2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0},
                                      {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0},
                                      {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0}};
    for (int64_t fi = 0; fi < nf; ++fi) {
        const FaceEntry& e = faces[(size_t)fi];
        const double* P = m.per(e.side[0].cell);
        if (e.count == 2 && m.cell_case[e.side[1].cell] != m.cell_case[e.side[0].cell]) {
            set_error("gks_mesh_create: cells of different cases share a face");
            return GKS_E_MESH;
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
            set_error("gks_mesh_create: degenerate face");
            return GKS_E_MESH;
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
                set_error("gks_mesh_create: flat tetrahedron");
                return GKS_E_MESH;
            }
            int lr = side < 0.0 ? 0 : 1;  // the normal leaves the left cell
            if (m.face_lr[fi * 2 + lr] != -1) {
                set_error("gks_mesh_create: two cells on the same side of a face");
                return GKS_E_MESH;
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
            ++m.nbf;
        }
    }

    // ---- cell geometry -------------------------------------------------
    m.vol.assign((size_t)nc, 0.0);
    m.cen.assign((size_t)nc * 3, 0.0);
    m.mom2.assign((size_t)nc * 6, 0.0);
    m.dr.assign((size_t)nc, 0.0);
    for (int64_t c = 0; c < nc; ++c) {
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
            set_error("gks_mesh_create: tetrahedron with non-positive volume");
            return GKS_E_MESH;
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
    for (int64_t fi = 0; fi < nf; ++fi) {
        for (int lr = 0; lr < 2; ++lr) {
            int64_t c = m.face_lr[fi * 2 + lr];
            if (c < 0) continue;
            const double* P = m.per(c);
            double* out = lr == 0 ? &m.gp_l[fi * 9] : &m.gp_r[fi * 9];
            for (int k = 0; k < 3; ++k)
                for (int a = 0; a < 3; ++a)
                    out[k * 3 + a] = gp_face[fi * 9 + k * 3 + a] +
                                     (double)base_lr[fi * 6 + lr * 3 + a] * P[a] - m.cen[c * 3 + a];
            m.dr[c] += m.farea[fi];
        }
    }
    for (int64_t c = 0; c < nc; ++c) m.dr[c] = 3.0 * m.vol[c] / m.dr[c];
    return GKS_OK;
}

}  // namespace gks
