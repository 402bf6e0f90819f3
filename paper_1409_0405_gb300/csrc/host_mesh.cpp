// Host mesh processing: element geometry at solution and flux points, face
// connectivity, periodic face matching and flux-point pairing.
//
// Element maps: tets are affine in the barycentric coordinates; prisms use
// the linear-triangle x linear-zeta map and hexes the trilinear map, neither
// affine once nodes are jittered; quadratically curved elements the
// Lagrange map of their degree-2 space through their quadratic nodes.  With A = dx/dxi (columns a_d), S = J dxi/dx = adj(A) has rows
// a_1 x a_2, a_2 x a_0, a_0 x a_1; a physical flux F becomes F~_d =
// sum_m S[d][m] F_m, and at a face the scaled physical normal is S^T n^.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "fr_internal.h"

namespace fr {
namespace {

using Vec3 = std::array<double, 3>;

// shape functions N[nv] and derivatives dN[nv][3] at reference point x
void shape(int etype, const double *x, double *N, double (*dN)[3]) {
    const double xi = x[0], eta = x[1], zeta = x[2];
    if (etype == FR_ETYPE_TET) {
        N[0] = -0.5 * (1 + xi + eta + zeta);
        N[1] = 0.5 * (1 + xi);
        N[2] = 0.5 * (1 + eta);
        N[3] = 0.5 * (1 + zeta);
        const double d[4][3] = {{-0.5, -0.5, -0.5}, {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}};
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < 3; ++k) dN[a][k] = d[a][k];
        return;
    }
    if (etype == FR_ETYPE_HEX) {
        // N_a = (1 + s0 xi)(1 + s1 eta)(1 + s2 zeta) / 8, s the vertex signs
        const int sg[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                              {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
        for (int a = 0; a < 8; ++a) {
            const double f0 = 1 + sg[a][0] * xi, f1 = 1 + sg[a][1] * eta, f2 = 1 + sg[a][2] * zeta;
            N[a] = 0.125 * f0 * f1 * f2;
            dN[a][0] = 0.125 * sg[a][0] * f1 * f2;
            dN[a][1] = 0.125 * f0 * sg[a][1] * f2;
            dN[a][2] = 0.125 * f0 * f1 * sg[a][2];
        }
        return;
    }
    const double tau[3] = {-0.5 * (xi + eta), 0.5 * (1 + xi), 0.5 * (1 + eta)};
    const double dtau[3][2] = {{-0.5, -0.5}, {0.5, 0.0}, {0.0, 0.5}};
    const double lo = 0.5 * (1 - zeta), hi = 0.5 * (1 + zeta);
    for (int a = 0; a < 3; ++a) {
        N[a] = tau[a] * lo;
        N[a + 3] = tau[a] * hi;
        for (int k = 0; k < 2; ++k) {
            dN[a][k] = dtau[a][k] * lo;
            dN[a + 3][k] = dtau[a][k] * hi;
        }
        dN[a][2] = -0.5 * tau[a];
        dN[a + 3][2] = 0.5 * tau[a];
    }
}

// Quadratically curved elements: the Lagrange basis of the element's
// degree-2 space (tet P2, prism P2(triangle) x P2(zeta), hex Q2) through its
// quadratic nodes, N_a(x) = sum_m mono_m(x) C[m][a] with C the inverse of
// the monomial Vandermonde matrix at the nodes (solved once per type).
constexpr int kMaxQ = 27;
struct QuadShape {
    int nq = 0;
    std::vector<std::array<int, 3>> ex;
    std::vector<double> C;  // nq x nq, row m = monomial, column a = node
};

const double kTri6[6][2] = {{-1, -1}, {1, -1}, {-1, 1}, {0, -1}, {0, 0}, {-1, 0}};

void quad_nodes(int etype, std::vector<std::array<double, 3>> &nodes) {
    nodes.clear();
    if (etype == FR_ETYPE_TET) {
        const double t[10][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}, {0, -1, -1},
                                 {-1, 0, -1},  {-1, -1, 0}, {0, 0, -1},  {0, -1, 0},  {-1, 0, 0}};
        for (auto &p : t) nodes.push_back({p[0], p[1], p[2]});
    } else if (etype == FR_ETYPE_PRI) {
        for (int c = -1; c <= 1; ++c)
            for (auto &p : kTri6) nodes.push_back({p[0], p[1], (double)c});
    } else {
        for (int c = -1; c <= 1; ++c)
            for (int b = -1; b <= 1; ++b)
                for (int a = -1; a <= 1; ++a) nodes.push_back({(double)a, (double)b, (double)c});
    }
}

bool build_quad_shape(int etype, QuadShape &q) {
    std::vector<std::array<double, 3>> nodes;
    quad_nodes(etype, nodes);
    q.nq = (int)nodes.size();
    q.ex.clear();
    for (int c = 0; c <= 2; ++c)
        for (int b = 0; b <= 2; ++b)
            for (int a = 0; a <= 2; ++a) {
                const bool in = etype == FR_ETYPE_TET ? a + b + c <= 2 : etype == FR_ETYPE_PRI ? a + b <= 2 : true;
                if (in) q.ex.push_back({a, b, c});
            }
    const int n = q.nq;
    if ((int)q.ex.size() != n) return false;
    // [V | I] -> [I | V^-1] by Gauss-Jordan with partial pivoting
    std::vector<double> M((size_t)n * 2 * n, 0.0);
    for (int r = 0; r < n; ++r) {
        for (int m = 0; m < n; ++m) {
            double v = 1.0;
            for (int d = 0; d < 3; ++d)
                for (int k = 0; k < q.ex[m][d]; ++k) v *= nodes[r][d];
            M[(size_t)r * 2 * n + m] = v;
        }
        M[(size_t)r * 2 * n + n + r] = 1.0;
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(M[(size_t)r * 2 * n + col]) > std::fabs(M[(size_t)piv * 2 * n + col])) piv = r;
        if (std::fabs(M[(size_t)piv * 2 * n + col]) < 1e-12) return false;
        if (piv != col)
            for (int k = 0; k < 2 * n; ++k) std::swap(M[(size_t)piv * 2 * n + k], M[(size_t)col * 2 * n + k]);
        const double inv = 1.0 / M[(size_t)col * 2 * n + col];
        for (int k = 0; k < 2 * n; ++k) M[(size_t)col * 2 * n + k] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = M[(size_t)r * 2 * n + col];
            if (f != 0.0)
                for (int k = 0; k < 2 * n; ++k) M[(size_t)r * 2 * n + k] -= f * M[(size_t)col * 2 * n + k];
        }
    }
    // V^-1 maps node values to monomial coefficients: C[m][a] = (V^-1)[m][a]
    q.C.assign((size_t)n * n, 0.0);
    for (int m = 0; m < n; ++m)
        for (int a = 0; a < n; ++a) q.C[(size_t)m * n + a] = M[(size_t)m * 2 * n + n + a];
    return true;
}

void quad_shape(const QuadShape &q, const double *x, double *N, double (*dN)[3]) {
    const int n = q.nq;
    double mono[kMaxQ], dmono[kMaxQ][3];
    for (int m = 0; m < n; ++m) {
        const auto &e = q.ex[m];
        double pw[3][3];  // pw[d][k] = x_d^k
        for (int d = 0; d < 3; ++d) {
            pw[d][0] = 1.0;
            pw[d][1] = x[d];
            pw[d][2] = x[d] * x[d];
        }
        mono[m] = pw[0][e[0]] * pw[1][e[1]] * pw[2][e[2]];
        for (int d = 0; d < 3; ++d) {
            if (e[d] == 0) {
                dmono[m][d] = 0.0;
                continue;
            }
            double v = (double)e[d] * pw[d][e[d] - 1];
            for (int k = 0; k < 3; ++k)
                if (k != d) v *= pw[k][e[k]];
            dmono[m][d] = v;
        }
    }
    for (int a = 0; a < n; ++a) {
        double s = 0.0, g[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < n; ++m) {
            const double c = q.C[(size_t)m * n + a];
            s += mono[m] * c;
            for (int d = 0; d < 3; ++d) g[d] += dmono[m][d] * c;
        }
        N[a] = s;
        for (int d = 0; d < 3; ++d) dN[a][d] = g[d];
    }
}

struct PointGeo {
    Vec3 x;
    double S[9];
    double J;
};

// geometry at a reference point: straight map of the vertices (q null) or
// the quadratic map of the nodes (q set); X holds the vertices or nodes
PointGeo point_geo(int etype, const double (*X)[3], const double *ref, const QuadShape *q = nullptr) {
    const int nv = q ? q->nq : etype == FR_ETYPE_TET ? 4 : etype == FR_ETYPE_HEX ? 8 : 6;
    double N[kMaxQ], dN[kMaxQ][3];
    if (q)
        quad_shape(*q, ref, N, dN);
    else
        shape(etype, ref, N, dN);
    PointGeo g{};
    double A[3][3] = {{0}};  // A[k][d] = dx_k / dxi_d
    for (int a = 0; a < nv; ++a)
        for (int k = 0; k < 3; ++k) {
            g.x[k] += N[a] * X[a][k];
            for (int d = 0; d < 3; ++d) A[k][d] += dN[a][d] * X[a][k];
        }
    Vec3 col[3];
    for (int d = 0; d < 3; ++d) col[d] = {A[0][d], A[1][d], A[2][d]};
    auto cross = [](const Vec3 &a, const Vec3 &b) {
        return Vec3{a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    };
    Vec3 r0 = cross(col[1], col[2]), r1 = cross(col[2], col[0]), r2 = cross(col[0], col[1]);
    for (int m = 0; m < 3; ++m) {
        g.S[0 * 3 + m] = r0[m];
        g.S[1 * 3 + m] = r1[m];
        g.S[2 * 3 + m] = r2[m];
    }
    g.J = col[0][0] * r0[0] + col[0][1] * r0[1] + col[0][2] * r0[2];
    return g;
}

struct FaceRec {
    int t, lf;
    int64_t e;
};

struct KeyHash {
    size_t operator()(const std::array<int64_t, 4> &k) const {
        uint64_t h = 1469598103934665603ull;
        for (int i = 0; i < 4; ++i) {
            h ^= (uint64_t)k[i] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        }
        return (size_t)h;
    }
};

struct CellHash {
    size_t operator()(const std::array<int64_t, 3> &k) const {
        return (size_t)((uint64_t)k[0] * 73856093ull ^ (uint64_t)k[1] * 19349663ull ^
                        (uint64_t)k[2] * 83492791ull);
    }
};

}  // namespace

int build_geometry(const fr_mesh *m, const RefOps ops[NT], TypeGeo geo[NT], std::string &err) {
    const int64_t *conn[NT] = {m->tet, m->pri, m->hex};
    const int64_t ne[NT] = {m->n_tet, m->n_pri, m->n_hex};
    const double *qnodes[NT] = {m->tet_nodes, m->pri_nodes, m->hex_nodes};
    const int nvs[NT] = {4, 6, 8};
    if (m->geom_order < 0 || m->geom_order > 2) {
        err = "geom_order must be 1 (straight) or 2 (quadratic)";
        return FR_ERR_MESH;
    }
    const bool curved = m->geom_order == 2;
    for (int t = 0; t < NT; ++t) {
        TypeGeo &G = geo[t];
        G = TypeGeo();
        G.ne = ne[t];
        if (ne[t] == 0) continue;
        QuadShape qs;
        if (curved) {
            if (!qnodes[t]) {
                err = "geom_order 2 needs the quadratic node coordinates of every element type present";
                return FR_ERR_MESH;
            }
            if (!build_quad_shape(t, qs)) {
                err = "quadratic shape functions: singular node set";
                return FR_ERR_MESH;
            }
        }
        const RefOps &o = ops[t];
        G.nu = o.nu;
        G.nf = o.nf;
        G.xu.resize((size_t)ne[t] * o.nu * 3);
        G.S.resize((size_t)ne[t] * o.nu * 9);
        G.J.resize((size_t)ne[t] * o.nu);
        G.xf.resize((size_t)ne[t] * o.nf * 3);
        G.fn.resize((size_t)ne[t] * o.nf * 3);
        G.fmag.resize((size_t)ne[t] * o.nf);
        const QuadShape *qp = curved ? &qs : nullptr;
        for (int64_t e = 0; e < ne[t]; ++e) {
            double X[kMaxQ][3];
            for (int a = 0; a < nvs[t]; ++a) {
                int64_t v = conn[t][e * nvs[t] + a];
                if (v < 0 || v >= m->n_nodes) {
                    err = "node id out of range";
                    return FR_ERR_MESH;
                }
                if (!curved)
                    for (int k = 0; k < 3; ++k) X[a][k] = m->xyz[3 * v + k];
            }
            if (curved) {
                const int nq = qs.nq;
                for (int a = 0; a < nq; ++a)
                    for (int k = 0; k < 3; ++k) X[a][k] = qnodes[t][((size_t)e * nq + a) * 3 + k];
            }
            for (int j = 0; j < o.nu; ++j) {
                PointGeo g = point_geo(t, X, &o.upts[3 * j], qp);
                if (!(g.J > 0.0)) {
                    err = "non-positive Jacobian at a solution point";
                    return FR_ERR_MESH;
                }
                size_t ij = (size_t)e * o.nu + j;
                for (int k = 0; k < 3; ++k) G.xu[3 * ij + k] = g.x[k];
                for (int k = 0; k < 9; ++k) G.S[9 * ij + k] = g.S[k];
                G.J[ij] = g.J;
            }
            for (int f = 0; f < o.nf; ++f) {
                PointGeo g = point_geo(t, X, &o.fpts[3 * f], qp);
                const double *nh = &o.fnorm[3 * f];
                double sn[3];
                for (int mm = 0; mm < 3; ++mm)
                    sn[mm] = nh[0] * g.S[0 * 3 + mm] + nh[1] * g.S[1 * 3 + mm] + nh[2] * g.S[2 * 3 + mm];
                double mag = std::sqrt(sn[0] * sn[0] + sn[1] * sn[1] + sn[2] * sn[2]);
                if (!(mag > 0.0)) {
                    err = "degenerate face";
                    return FR_ERR_MESH;
                }
                size_t fj = (size_t)e * o.nf + f;
                for (int k = 0; k < 3; ++k) {
                    G.xf[3 * fj + k] = g.x[k];
                    G.fn[3 * fj + k] = sn[k] / mag;
                }
                G.fmag[fj] = mag;
            }
        }
    }
    return FR_OK;
}

int build_faces(const fr_mesh *m, const RefOps ops[NT], const TypeGeo geo[NT], Faces &F,
                std::string &err) {
    F = Faces();
    const int64_t *conn[NT] = {m->tet, m->pri, m->hex};
    const int64_t ne[NT] = {m->n_tet, m->n_pri, m->n_hex};
    const int nvs[NT] = {4, 6, 8};

    // bounding box -> matching tolerance
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t v = 0; v < m->n_nodes; ++v)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], m->xyz[3 * v + k]);
            hi[k] = std::max(hi[k], m->xyz[3 * v + k]);
        }
    double diag = 0;
    for (int k = 0; k < 3; ++k) diag += (hi[k] - lo[k]) * (hi[k] - lo[k]);
    diag = std::sqrt(diag);
    const double tol = 1e-7 * diag;

    // ---- interior faces by shared vertex sets
    std::unordered_map<std::array<int64_t, 4>, std::vector<FaceRec>, KeyHash> map;
    size_t nfaces_total = 0;
    for (int t = 0; t < NT; ++t) nfaces_total += (size_t)ne[t] * ops[t].nfaces * (ne[t] > 0);
    map.reserve(nfaces_total);
    for (int t = 0; t < NT; ++t) {
        if (ne[t] == 0) continue;
        for (int64_t e = 0; e < ne[t]; ++e)
            for (int lf = 0; lf < ops[t].nfaces; ++lf) {
                const auto &fv = ops[t].face_verts[lf];
                std::array<int64_t, 4> key = {-1, -1, -1, -1};
                for (size_t a = 0; a < fv.size(); ++a) key[a] = conn[t][e * nvs[t] + fv[a]];
                std::sort(key.begin(), key.begin() + fv.size());
                map[key].push_back({t, lf, e});
            }
    }
    struct Pair {
        FaceRec a, b;
        Vec3 shift;
    };
    std::vector<Pair> pairs;
    std::vector<FaceRec> free_faces;
    for (auto &kv : map) {
        if (kv.second.size() == 2) {
            FaceRec a = kv.second[0], b = kv.second[1];
            pairs.push_back({a, b, {0, 0, 0}});
        } else if (kv.second.size() == 1) {
            free_faces.push_back(kv.second[0]);
        } else {
            err = "a face is shared by more than two elements";
            return FR_ERR_MESH;
        }
    }
    auto rec_less = [](const FaceRec &x, const FaceRec &y) {
        if (x.t != y.t) return x.t < y.t;
        if (x.e != y.e) return x.e < y.e;
        return x.lf < y.lf;
    };
    std::sort(free_faces.begin(), free_faces.end(), rec_less);
    // deterministic order of interior pairs: by the smaller side
    for (auto &p : pairs)
        if (rec_less(p.b, p.a)) std::swap(p.a, p.b);
    std::sort(pairs.begin(), pairs.end(), [&](const Pair &x, const Pair &y) { return rec_less(x.a, y.a); });

    // ---- boundary faces
    std::vector<char> used(free_faces.size(), 0);
    auto find_free = [&](int t, int64_t e, int lf) -> int64_t {
        FaceRec key{t, lf, e};
        auto it = std::lower_bound(free_faces.begin(), free_faces.end(), key, rec_less);
        if (it != free_faces.end() && it->t == t && it->e == e && it->lf == lf)
            return it - free_faces.begin();
        return -1;
    };
    struct BRec {
        FaceRec r;
        int tag;
    };
    std::vector<BRec> bfaces;
    for (int64_t i = 0; i < m->n_bface; ++i) {
        const int64_t *b = &m->bface[4 * i];
        int t = (int)b[0];
        if (t < 0 || t >= NT || ne[t] == 0 || b[1] < 0 || b[1] >= ne[t] || b[2] < 0 || b[2] >= ops[t].nfaces ||
            (b[3] != FR_BC_WALL && b[3] != FR_BC_FARFIELD)) {
            err = "invalid boundary face record";
            return FR_ERR_MESH;
        }
        int64_t idx = find_free(t, b[1], (int)b[2]);
        if (idx < 0 || used[idx]) {
            err = "boundary face is not a free face";
            return FR_ERR_MESH;
        }
        used[idx] = 1;
        bfaces.push_back({free_faces[idx], (int)b[3]});
    }

    // ---- periodic matching of the remaining free faces by centroid
    std::vector<int64_t> rem;
    for (size_t i = 0; i < free_faces.size(); ++i)
        if (!used[i]) rem.push_back((int64_t)i);
    if (!rem.empty()) {
        bool anyper = m->period[0] > 0 || m->period[1] > 0 || m->period[2] > 0;
        if (!anyper) {
            err = "unmatched faces and no periodic axis";
            return FR_ERR_MESH;
        }
        const double cell = 1e-5 * diag;
        std::vector<Vec3> cen(rem.size());
        std::unordered_map<std::array<int64_t, 3>, std::vector<int64_t>, CellHash> grid;
        for (size_t i = 0; i < rem.size(); ++i) {
            const FaceRec &r = free_faces[rem[i]];
            const auto &fv = ops[r.t].face_verts[r.lf];
            Vec3 c = {0, 0, 0};
            for (int a : fv) {
                int64_t v = conn[r.t][r.e * nvs[r.t] + a];
                for (int k = 0; k < 3; ++k) c[k] += m->xyz[3 * v + k] / fv.size();
            }
            cen[i] = c;
            std::array<int64_t, 3> q = {(int64_t)std::floor(c[0] / cell), (int64_t)std::floor(c[1] / cell),
                                        (int64_t)std::floor(c[2] / cell)};
            grid[q].push_back((int64_t)i);
        }
        std::vector<Vec3> shifts;
        for (int sx = -1; sx <= 1; ++sx)
            for (int sy = -1; sy <= 1; ++sy)
                for (int sz = -1; sz <= 1; ++sz) {
                    int s[3] = {sx, sy, sz};
                    bool ok = true, nz = false;
                    for (int k = 0; k < 3; ++k) {
                        if (s[k] != 0 && !(m->period[k] > 0)) ok = false;
                        if (s[k] != 0) nz = true;
                    }
                    if (ok && nz) shifts.push_back({s[0] * m->period[0], s[1] * m->period[1], s[2] * m->period[2]});
                }
        std::vector<int64_t> partner(rem.size(), -1);
        for (size_t i = 0; i < rem.size(); ++i) {
            if (partner[i] >= 0) continue;
            bool found = false;
            for (const Vec3 &s : shifts) {
                Vec3 c = {cen[i][0] + s[0], cen[i][1] + s[1], cen[i][2] + s[2]};
                int64_t q0 = (int64_t)std::floor(c[0] / cell), q1 = (int64_t)std::floor(c[1] / cell),
                        q2 = (int64_t)std::floor(c[2] / cell);
                for (int d0 = -1; d0 <= 1 && !found; ++d0)
                    for (int d1 = -1; d1 <= 1 && !found; ++d1)
                        for (int d2 = -1; d2 <= 1 && !found; ++d2) {
                            auto it = grid.find({q0 + d0, q1 + d1, q2 + d2});
                            if (it == grid.end()) continue;
                            for (int64_t j : it->second) {
                                if ((size_t)j == i || partner[j] >= 0) continue;
                                double dd = 0;
                                for (int k = 0; k < 3; ++k) dd += (cen[j][k] - c[k]) * (cen[j][k] - c[k]);
                                if (std::sqrt(dd) < tol) {
                                    partner[i] = j;
                                    partner[j] = (int64_t)i;
                                    pairs.push_back({free_faces[rem[i]], free_faces[rem[j]], s});
                                    found = true;
                                    break;
                                }
                            }
                        }
                if (found) break;
            }
            if (!found) {
                err = "a free face has no periodic partner (non-conforming mesh?)";
                return FR_ERR_MESH;
            }
        }
    }

    // ---- flux-point pairing by physical position
    struct PP {
        int ta, fa, tb, fb;
        int64_t ea, eb;
        Vec3 n;
        double ma, mb;
    };
    std::vector<PP> pp;
    for (const Pair &P : pairs) {
        const auto &ia = ops[P.a.t].face_fpts[P.a.lf];
        const auto &ib = ops[P.b.t].face_fpts[P.b.lf];
        if (ia.size() != ib.size()) {
            err = "non-conforming face pair (triangle against quad)";
            return FR_ERR_MESH;
        }
        const TypeGeo &Ga = geo[P.a.t], &Gb = geo[P.b.t];
        std::vector<char> taken(ib.size(), 0);
        for (size_t k = 0; k < ia.size(); ++k) {
            size_t fa = (size_t)P.a.e * Ga.nf + ia[k];
            Vec3 xa = {Ga.xf[3 * fa] + P.shift[0], Ga.xf[3 * fa + 1] + P.shift[1], Ga.xf[3 * fa + 2] + P.shift[2]};
            double best = 1e300;
            size_t bi = 0;
            for (size_t q = 0; q < ib.size(); ++q) {
                size_t fb = (size_t)P.b.e * Gb.nf + ib[q];
                double dd = 0;
                for (int c = 0; c < 3; ++c) dd += (Gb.xf[3 * fb + c] - xa[c]) * (Gb.xf[3 * fb + c] - xa[c]);
                if (dd < best) {
                    best = dd;
                    bi = q;
                }
            }
            if (std::sqrt(best) > tol || taken[bi]) {
                err = "flux points of a face pair do not coincide";
                return FR_ERR_MESH;
            }
            taken[bi] = 1;
            size_t fb = (size_t)P.b.e * Gb.nf + ib[bi];
            PP r;
            r.ta = P.a.t;
            r.fa = ia[k];
            r.ea = P.a.e;
            r.tb = P.b.t;
            r.fb = ib[bi];
            r.eb = P.b.e;
            r.n = {Ga.fn[3 * fa], Ga.fn[3 * fa + 1], Ga.fn[3 * fa + 2]};
            r.ma = Ga.fmag[fa];
            r.mb = Gb.fmag[fb];
            pp.push_back(r);
        }
    }
    // order pairs so consecutive threads read consecutive side-a elements
    std::sort(pp.begin(), pp.end(), [](const PP &x, const PP &y) {
        if (x.ta != y.ta) return x.ta < y.ta;
        if (x.fa != y.fa) return x.fa < y.fa;
        return x.ea < y.ea;
    });
    size_t np = pp.size();
    F.ta.resize(np);
    F.fa.resize(np);
    F.ea.resize(np);
    F.tb.resize(np);
    F.fb.resize(np);
    F.eb.resize(np);
    F.n.resize(3 * np);
    F.maga.resize(np);
    F.magb.resize(np);
    for (size_t k = 0; k < np; ++k) {
        F.ta[k] = pp[k].ta;
        F.fa[k] = pp[k].fa;
        F.ea[k] = (int)pp[k].ea;
        F.tb[k] = pp[k].tb;
        F.fb[k] = pp[k].fb;
        F.eb[k] = (int)pp[k].eb;
        for (int c = 0; c < 3; ++c) F.n[3 * k + c] = pp[k].n[c];
        F.maga[k] = pp[k].ma;
        F.magb[k] = pp[k].mb;
    }

    struct BP {
        int t, f, tag;
        int64_t e;
    };
    std::vector<BP> bp;
    for (const BRec &b : bfaces)
        for (int f : ops[b.r.t].face_fpts[b.r.lf]) bp.push_back({b.r.t, f, b.tag, b.r.e});
    std::sort(bp.begin(), bp.end(), [](const BP &x, const BP &y) {
        if (x.t != y.t) return x.t < y.t;
        if (x.f != y.f) return x.f < y.f;
        return x.e < y.e;
    });
    for (const BP &b : bp) {
        const TypeGeo &G = geo[b.t];
        size_t fj = (size_t)b.e * G.nf + b.f;
        F.bt.push_back(b.t);
        F.bf.push_back(b.f);
        F.be.push_back((int)b.e);
        F.btag.push_back(b.tag);
        for (int c = 0; c < 3; ++c) F.bn.push_back(G.fn[3 * fj + c]);
        F.bmag.push_back(G.fmag[fj]);
    }

    // every flux point covered exactly once
    for (int t = 0; t < NT; ++t) {
        if (ne[t] == 0) continue;
        std::vector<unsigned char> cov((size_t)ne[t] * ops[t].nf, 0);
        for (size_t k = 0; k < np; ++k) {
            if (F.ta[k] == t) cov[(size_t)F.ea[k] * ops[t].nf + F.fa[k]]++;
            if (F.tb[k] == t) cov[(size_t)F.eb[k] * ops[t].nf + F.fb[k]]++;
        }
        for (size_t k = 0; k < F.bt.size(); ++k)
            if (F.bt[k] == t) cov[(size_t)F.be[k] * ops[t].nf + F.bf[k]]++;
        for (unsigned char c : cov)
            if (c != 1) {
                err = "flux points not covered exactly once";
                return FR_ERR_MESH;
            }
    }
    return FR_OK;
}

}  // namespace fr
