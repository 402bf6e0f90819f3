// Host construction of the FR points and operator matrices.
//
// Basis: the orthogonal collapsed-coordinate (Dubiner) polynomials of the
// element space (tet: P_p; prism: P_p(triangle) x P_p(zeta); hex: Q_p, the
// Legendre tensor products P_i(xi) P_j(eta) P_k(zeta), i, j, k <= p), whose
// dimensions are Table 2's solution-point counts:
//   tet  psi_ijk = P_i(a) ((1-b)/2)^i P_j^(2i+1,0)(b) ((1-c)/2)^(i+j)
//                  P_k^(2i+2j+2,0)(c),
//        a = 2(1+xi)/(-eta-zeta) - 1, b = 2(1+eta)/(1-zeta) - 1, c = zeta;
//   tri  psi_ij = P_i(a) ((1-b)/2)^i P_j^(2i+1,0)(b),
//        a = 2(1+xi)/(1-eta) - 1, b = eta;
//   prism: tri x Legendre P_k(zeta);  quad faces: Legendre x Legendre.
// They are polynomials in the reference coordinates; their derivatives are
// taken exactly with forward-mode dual numbers (every evaluation point lies
// off the collapsed edge), and each is normalised by its quadrature norm.
// Integrals use collapsed (Duffy) Gauss-Legendre rules exact for the degrees
// involved.  Everything is computed in double-double arithmetic and rounded
// to double once, so the operators are correctly rounded: small operator
// errors would otherwise show up as spurious jumps between neighbouring
// elements, amplified by 1/h in thin wall layers.
//
// Operators (the paper casts each as a constant matrix A in C <- c1 A B + c2 C,
// Sec. 2.1 Eq. 1; it writes out only M0, Table 2):
//   M0  Lagrange interpolation from solution to flux points.
//   D   reference gradient of the solution-point interpolant.
//   M3  the correction recovering nodal DG (Sec. 3.4): column f is, at the
//       solution points, the g_f of the element space with
//       int g_f v = int_F l_f v dS for all v of the space (l_f the face
//       Lagrange polynomial of flux point f, dS the reference face measure).
//   W   integrals of the solution-point Lagrange polynomials.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "dd.h"
#include "fr_internal.h"

namespace fr {
namespace {

using R = DD;
using Vec3 = std::array<R, 3>;

const int TET_V[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
const int PRI_V[6][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}};
const std::vector<std::vector<int>> TET_FACES = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
const std::vector<std::vector<int>> PRI_FACES = {
    {0, 1, 2}, {3, 4, 5}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};
const int HEX_V[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                         {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
const std::vector<std::vector<int>> HEX_FACES = {{0, 1, 2, 3}, {0, 1, 5, 4}, {1, 2, 6, 5},
                                                 {2, 3, 7, 6}, {3, 0, 4, 7}, {4, 5, 6, 7}};

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes/weights in double-double (Newton on P_n)
void gl_dd(int n, std::vector<R> &x, std::vector<R> &w) {
    x.assign(n, R(0.0));
    w.assign(n, R(0.0));
    const double pi = 3.14159265358979323846;
    auto eval = [n](const R &z, R &pn, R &dpn) {
        R p0(1.0), p1 = z;
        for (int k = 2; k <= n; ++k) {
            R p2 = (R(2.0 * k - 1.0) * z * p1 - R(k - 1.0) * p0) / R((double)k);
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) {
            p0 = R(1.0);
            p1 = z;
        }
        pn = p1;
        dpn = R((double)n) * (z * p1 - p0) / (z * z - R(1.0));
    };
    for (int i = 0; i < n; ++i) {
        R z(-std::cos(pi * (i + 0.75) / (n + 0.5)));
        for (int it = 0; it < 60; ++it) {
            R pn, dpn;
            eval(z, pn, dpn);
            R dz = pn / dpn;
            z -= dz;
            if (std::fabs(dz.hi) < 1e-32) break;
        }
        R pn, dpn;
        eval(z, pn, dpn);
        x[i] = z;
        w[i] = R(2.0) / ((R(1.0) - z * z) * dpn * dpn);
    }
}

// ---------------------------------------------------------------------------
struct Mat {
    int r = 0, c = 0;
    std::vector<R> a;
    Mat() {}
    Mat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_, R(0.0)) {}
    R &operator()(int i, int j) { return a[(size_t)i * c + j]; }
    const R &operator()(int i, int j) const { return a[(size_t)i * c + j]; }
};

Mat matmul(const Mat &A, const Mat &B) {
    Mat C(A.r, B.c);
    for (int i = 0; i < A.r; ++i)
        for (int k = 0; k < A.c; ++k) {
            const R aik = A(i, k);
            if (aik.hi == 0.0) continue;
            for (int j = 0; j < B.c; ++j) C(i, j) += aik * B(k, j);
        }
    return C;
}

// Solve A X = B by LU with partial pivoting (double-double).
bool solve(const Mat &A, const Mat &B, Mat &X) {
    const int n = A.r;
    Mat LU = A;
    std::vector<int> piv(n);
    for (int i = 0; i < n; ++i) piv[i] = i;
    for (int k = 0; k < n; ++k) {
        int pr = k;
        for (int i = k + 1; i < n; ++i)
            if (dd_abs(LU(i, k)) > dd_abs(LU(pr, k))) pr = i;
        if (LU(pr, k).hi == 0.0) return false;
        if (pr != k) {
            for (int j = 0; j < n; ++j) std::swap(LU(k, j), LU(pr, j));
            std::swap(piv[k], piv[pr]);
        }
        for (int i = k + 1; i < n; ++i) {
            LU(i, k) /= LU(k, k);
            const R l = LU(i, k);
            for (int j = k + 1; j < n; ++j) LU(i, j) -= l * LU(k, j);
        }
    }
    X = Mat(n, B.c);
    for (int col = 0; col < B.c; ++col) {
        std::vector<R> y(n);
        for (int i = 0; i < n; ++i) {
            R s = B(piv[i], col);
            for (int j = 0; j < i; ++j) s -= LU(i, j) * y[j];
            y[i] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            R s = y[i];
            for (int j = i + 1; j < n; ++j) s -= LU(i, j) * X(j, col);
            X(i, col) = s / LU(i, i);
        }
    }
    return true;
}

Mat identity(int n) {
    Mat I(n, n);
    for (int i = 0; i < n; ++i) I(i, i) = R(1.0);
    return I;
}

// Blyth-Pozrikidis barycentric coordinates of multi-index I from the 1-D
// nodes v on [0, 1]: lambda_a = (1 + d v_{I_a} - sum_{b != a} v_{I_b}) / (d+1)
template <int NB>
std::array<R, NB> bp_bary(const std::array<int, NB> &I, const std::vector<R> &v) {
    const int d = NB - 1;
    R tot(0.0);
    for (int a = 0; a < NB; ++a) tot += v[I[a]];
    std::array<R, NB> lam;
    for (int a = 0; a < NB; ++a) lam[a] = (R(1.0) + R((double)d) * v[I[a]] - (tot - v[I[a]])) / R(d + 1.0);
    return lam;
}

std::vector<R> gl01(int n) {
    std::vector<R> x, w;
    gl_dd(n, x, w);
    for (auto &xi : x) xi = R(0.5) * (xi + R(1.0));
    return x;
}

std::vector<std::array<R, 3>> tri_set(int p) {
    std::vector<R> v = gl01(p + 1);
    std::vector<std::array<R, 3>> out;
    for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= p - j; ++i) out.push_back(bp_bary<3>({p - i - j, i, j}, v));
    return out;
}

// forward-mode dual number with three partial derivatives
struct Dual {
    R v, d[3];
};
inline Dual dc(const R &c) { return {c, {R(0.0), R(0.0), R(0.0)}}; }
inline Dual operator+(const Dual &a, const Dual &b) {
    return {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}};
}
inline Dual operator-(const Dual &a, const Dual &b) {
    return {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}};
}
inline Dual operator*(const Dual &a, const Dual &b) {
    return {a.v * b.v,
            {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1], a.d[2] * b.v + a.v * b.d[2]}};
}
inline Dual operator/(const Dual &a, const Dual &b) {
    const R q = a.v / b.v;
    return {q, {(a.d[0] - q * b.d[0]) / b.v, (a.d[1] - q * b.d[1]) / b.v, (a.d[2] - q * b.d[2]) / b.v}};
}
inline Dual scale(const R &c, const Dual &a) { return {c * a.v, {c * a.d[0], c * a.d[1], c * a.d[2]}}; }
Dual dpow(const Dual &a, int n) {
    Dual r = dc(R(1.0));
    for (int i = 0; i < n; ++i) r = r * a;
    return r;
}

// Jacobi polynomial P_n^(al, 0)(x) (unnormalised three-term recurrence)
Dual jacobi(int n, double al, const Dual &x) {
    const double be = 0.0;
    Dual p0 = dc(R(1.0));
    if (n == 0) return p0;
    Dual p1 = scale(R(0.5 * (al + be + 2.0)), x) + dc(R(0.5 * (al - be)));
    for (int k = 2; k <= n; ++k) {
        const double s = 2.0 * k + al + be;
        const R A(2.0 * k * (k + al + be) * (s - 2.0));
        const R B((s - 1.0) * s * (s - 2.0));
        const R Cc((s - 1.0) * (al * al - be * be));
        const R Dd(2.0 * (k + al - 1.0) * (k + be - 1.0) * s);
        Dual p2 = scale(R(1.0) / A, (scale(B, x) + dc(Cc)) * p1 - scale(Dd, p0));
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

struct Basis {
    int etype, p;
    std::vector<std::array<int, 3>> ex;
    std::vector<R> scl;  // 1 / quadrature norm of each function
    explicit Basis(int et, int p_) : etype(et), p(p_) {
        for (int c = 0; c <= p; ++c)
            for (int b = 0; b <= p; ++b)
                for (int a = 0; a <= p; ++a) {
                    bool in = (etype == FR_ETYPE_TET) ? (a + b + c <= p)
                              : (etype == FR_ETYPE_HEX) ? true
                                                        : (a + b <= p);
                    if (in) ex.push_back({a, b, c});
                }
        scl.assign(ex.size(), R(1.0));
    }
    int size() const { return (int)ex.size(); }
    Dual raw(int m, const Vec3 &x) const {
        const Dual one = dc(R(1.0));
        Dual xi{x[0], {R(1.0), R(0.0), R(0.0)}}, eta{x[1], {R(0.0), R(1.0), R(0.0)}},
            zeta{x[2], {R(0.0), R(0.0), R(1.0)}};
        const int i = ex[m][0], j = ex[m][1], k = ex[m][2];
        const Dual half = dc(R(0.5)), two = dc(R(2.0));
        if (etype == FR_ETYPE_TET) {
            Dual a = (two * (one + xi)) / (dc(R(0.0)) - eta - zeta) - one;
            Dual b = (two * (one + eta)) / (one - zeta) - one;
            Dual c = zeta;
            return jacobi(i, 0, a) * dpow(half * (one - b), i) * jacobi(j, 2 * i + 1, b) *
                   dpow(half * (one - c), i + j) * jacobi(k, 2 * i + 2 * j + 2, c);
        }
        if (etype == FR_ETYPE_HEX) return jacobi(i, 0, xi) * jacobi(j, 0, eta) * jacobi(k, 0, zeta);
        Dual a = (two * (one + xi)) / (one - eta) - one;
        Dual b = eta;
        return jacobi(i, 0, a) * dpow(half * (one - b), i) * jacobi(j, 2 * i + 1, b) * jacobi(k, 0, zeta);
    }
    // values (and optionally the three derivatives, [d][m]) at x
    void eval(const Vec3 &x, R *phi, R *dphi) const {
        const int n = size();
        for (int m = 0; m < n; ++m) {
            Dual r = raw(m, x);
            phi[m] = scl[m] * r.v;
            if (dphi)
                for (int d = 0; d < 3; ++d) dphi[d * n + m] = scl[m] * r.d[d];
        }
    }
};

struct FaceBasis {
    bool tri;
    int p;
    std::vector<std::array<int, 2>> ex;
    FaceBasis(bool t, int p_) : tri(t), p(p_) {
        for (int b = 0; b <= p; ++b)
            for (int a = 0; a <= p; ++a)
                if (!tri || a + b <= p) ex.push_back({a, b});
    }
    void eval(const R &r, const R &s, R *psi) const {
        const Dual one = dc(R(1.0)), two = dc(R(2.0)), half = dc(R(0.5));
        Dual Rr{r, {R(1.0), R(0.0), R(0.0)}}, S{s, {R(0.0), R(1.0), R(0.0)}};
        for (size_t m = 0; m < ex.size(); ++m) {
            const int i = ex[m][0], j = ex[m][1];
            if (tri) {
                Dual a = (two * (one + Rr)) / (one - S) - one;
                psi[m] = (jacobi(i, 0, a) * dpow(half * (one - S), i) * jacobi(j, 2 * i + 1, S)).v;
            } else {
                psi[m] = (jacobi(i, 0, Rr) * jacobi(j, 0, S)).v;
            }
        }
    }
};

// Collapsed Gauss rules (points in the parameter domain, weights summing
// to its measure).
void rule_unit_tri(int n, std::vector<std::array<R, 2>> &pts, std::vector<R> &wts) {
    std::vector<R> x, w;
    gl_dd(n, x, w);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            R u = R(0.5) * (x[a] + R(1.0)), v = R(0.5) * (x[b] + R(1.0));
            R wu = R(0.5) * w[a], wv = R(0.5) * w[b];
            pts.push_back({u, v * (R(1.0) - u)});
            wts.push_back(wu * wv * (R(1.0) - u));
        }
}

void rule_volume(int etype, int n, std::vector<Vec3> &pts, std::vector<R> &wts) {
    std::vector<R> x, w;
    gl_dd(n, x, w);
    if (etype == FR_ETYPE_TET) {
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b)
                for (int c = 0; c < n; ++c) {
                    R u = R(0.5) * (x[a] + R(1.0)), v = R(0.5) * (x[b] + R(1.0)), t = R(0.5) * (x[c] + R(1.0));
                    R px = u, py = v * (R(1.0) - u), pz = t * (R(1.0) - u) * (R(1.0) - v);
                    pts.push_back({R(2.0) * px - R(1.0), R(2.0) * py - R(1.0), R(2.0) * pz - R(1.0)});
                    wts.push_back(w[a] * w[b] * w[c] * (R(1.0) - u) * (R(1.0) - u) * (R(1.0) - v));
                }
    } else if (etype == FR_ETYPE_HEX) {
        for (int c = 0; c < n; ++c)
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) {
                    pts.push_back({x[a], x[b], x[c]});
                    wts.push_back(w[a] * w[b] * w[c]);
                }
    } else {
        std::vector<std::array<R, 2>> tp;
        std::vector<R> tw;
        rule_unit_tri(n, tp, tw);
        for (int c = 0; c < n; ++c)
            for (size_t q = 0; q < tp.size(); ++q) {
                pts.push_back({R(2.0) * tp[q][0] - R(1.0), R(2.0) * tp[q][1] - R(1.0), x[c]});
                wts.push_back(R(4.0) * tw[q] * w[c]);
            }
    }
}

Vec3 vsub(const Vec3 &a, const Vec3 &b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
Vec3 vcross(const Vec3 &a, const Vec3 &b) {
    return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}

std::vector<double> to_d(const std::vector<R> &v) {
    std::vector<double> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = v[i].to_double();
    return o;
}

}  // namespace

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    std::vector<R> xd, wd;
    gl_dd(n, xd, wd);
    x = to_d(xd);
    w = to_d(wd);
}

int nupts_of(int etype, int p) {
    if (etype == FR_ETYPE_TET) return (p + 1) * (p + 2) * (p + 3) / 6;
    if (etype == FR_ETYPE_HEX) return (p + 1) * (p + 1) * (p + 1);
    return (p + 1) * (p + 1) * (p + 2) / 2;
}

int nfpts_of(int etype, int p) {
    if (etype == FR_ETYPE_TET) return 4 * (p + 1) * (p + 2) / 2;
    if (etype == FR_ETYPE_HEX) return 6 * (p + 1) * (p + 1);
    return 2 * (p + 1) * (p + 2) / 2 + 3 * (p + 1) * (p + 1);
}

namespace {
int build_ref_ops_uncached(int etype, int p, RefOps &o, std::string &err);
}

// Operators depend only on (etype, p): built once per process and reused.
int build_ref_ops(int etype, int p, RefOps &o, std::string &err) {
    if (etype < FR_ETYPE_TET || etype > FR_ETYPE_HEX || p < 1 || p > 4) {
        err = "build_ref_ops: etype must be 0/1/2 and order 1..4";
        return FR_ERR_ARG;
    }
    static std::mutex mtx;
    static std::map<std::pair<int, int>, RefOps> cache;
    {
        std::lock_guard<std::mutex> lock(mtx);
        auto it = cache.find({etype, p});
        if (it != cache.end()) {
            o = it->second;
            return FR_OK;
        }
    }
    int rc = build_ref_ops_uncached(etype, p, o, err);
    if (rc == FR_OK) {
        std::lock_guard<std::mutex> lock(mtx);
        cache[{etype, p}] = o;
    }
    return rc;
}

namespace {
int build_ref_ops_uncached(int etype, int p, RefOps &o, std::string &err) {
    o = RefOps();
    o.etype = etype;
    o.p = p;
    const bool tet = etype == FR_ETYPE_TET, hex = etype == FR_ETYPE_HEX;
    const int nverts = tet ? 4 : hex ? 8 : 6;
    std::vector<Vec3> V(nverts);
    for (int i = 0; i < nverts; ++i)
        for (int k = 0; k < 3; ++k) V[i][k] = R((double)(tet ? TET_V[i][k] : hex ? HEX_V[i][k] : PRI_V[i][k]));
    o.face_verts = tet ? TET_FACES : hex ? HEX_FACES : PRI_FACES;
    o.nfaces = (int)o.face_verts.size();

    // ---- solution points
    std::vector<Vec3> up;
    std::vector<R> glx, glw;
    gl_dd(p + 1, glx, glw);
    if (tet) {
        std::vector<R> v = gl01(p + 1);
        for (int k = 0; k <= p; ++k)
            for (int j = 0; j <= p - k; ++j)
                for (int i = 0; i <= p - k - j; ++i) {
                    auto lam = bp_bary<4>({p - i - j - k, i, j, k}, v);
                    Vec3 x = {R(0.0), R(0.0), R(0.0)};
                    for (int a = 0; a < 4; ++a)
                        for (int c = 0; c < 3; ++c) x[c] += lam[a] * V[a][c];
                    up.push_back(x);
                }
    } else if (hex) {
        for (int c = 0; c <= p; ++c)
            for (int b = 0; b <= p; ++b)
                for (int a = 0; a <= p; ++a) up.push_back({glx[a], glx[b], glx[c]});
    } else {
        auto tri = tri_set(p);
        for (int c = 0; c <= p; ++c)
            for (auto &lam : tri) {
                R xi(0.0), eta(0.0);
                for (int a = 0; a < 3; ++a) {
                    xi += lam[a] * V[a][0];
                    eta += lam[a] * V[a][1];
                }
                up.push_back({xi, eta, glx[c]});
            }
    }
    const int nu = (int)up.size();

    // ---- flux points, face parameters, normals, areas
    std::vector<Vec3> fp;
    std::vector<std::array<R, 2>> fparam;
    std::vector<Vec3> face_n(o.nfaces);
    std::vector<R> face_area(o.nfaces);
    o.face_fpts.assign(o.nfaces, {});
    Vec3 cen_e = {R(0.0), R(0.0), R(0.0)};
    for (auto &v : V)
        for (int c = 0; c < 3; ++c) cen_e[c] += v[c] / R((double)nverts);
    for (int fi = 0; fi < o.nfaces; ++fi) {
        const auto &fv = o.face_verts[fi];
        const bool tri = fv.size() == 3;
        Vec3 A = V[fv[0]], B = V[fv[1]], C = V[fv[2]];
        Vec3 Dq = tri ? C : V[fv[3]];
        Vec3 cr = vcross(vsub(B, A), vsub(Dq, A));
        R nn = dd_sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        face_area[fi] = tri ? R(0.5) * nn : nn;
        Vec3 n = {cr[0] / nn, cr[1] / nn, cr[2] / nn};
        Vec3 cen_f = {R(0.0), R(0.0), R(0.0)};
        for (int vi : fv)
            for (int c = 0; c < 3; ++c) cen_f[c] += V[vi][c] / R((double)fv.size());
        R s(0.0);
        for (int c = 0; c < 3; ++c) s += (cen_f[c] - cen_e[c]) * n[c];
        if (s.hi < 0)
            for (int c = 0; c < 3; ++c) n[c] = -n[c];
        face_n[fi] = n;
        if (tri) {
            for (auto &lam : tri_set(p)) {
                Vec3 x;
                for (int c = 0; c < 3; ++c) x[c] = lam[0] * A[c] + lam[1] * B[c] + lam[2] * C[c];
                o.face_fpts[fi].push_back((int)fp.size());
                fp.push_back(x);
                fparam.push_back({R(2.0) * lam[1] - R(1.0), R(2.0) * lam[2] - R(1.0)});
            }
        } else {
            Vec3 Dv = V[fv[3]];
            for (int b = 0; b <= p; ++b)
                for (int a = 0; a <= p; ++a) {
                    const R s_ = glx[a], t_ = glx[b];
                    const R one(1.0), q(0.25);
                    Vec3 x;
                    for (int c = 0; c < 3; ++c)
                        x[c] = q * (A[c] * (one - s_) * (one - t_) + B[c] * (one + s_) * (one - t_) +
                                    C[c] * (one + s_) * (one + t_) + Dv[c] * (one - s_) * (one + t_));
                    o.face_fpts[fi].push_back((int)fp.size());
                    fp.push_back(x);
                    fparam.push_back({s_, t_});
                }
        }
    }
    const int nf = (int)fp.size();
    if (nu != nupts_of(etype, p) || nf != nfpts_of(etype, p)) {
        err = "build_ref_ops: point count mismatch";
        return FR_ERR_ARG;
    }
    o.nu = nu;
    o.nf = nf;
    o.upts.resize(3 * nu);
    o.fpts.resize(3 * nf);
    o.fface.resize(nf);
    o.fnorm.resize(3 * nf);
    for (int j = 0; j < nu; ++j)
        for (int c = 0; c < 3; ++c) o.upts[3 * j + c] = up[j][c].to_double();
    for (int fi = 0; fi < o.nfaces; ++fi)
        for (int f : o.face_fpts[fi]) {
            o.fface[f] = fi;
            for (int c = 0; c < 3; ++c) {
                o.fpts[3 * f + c] = fp[f][c].to_double();
                o.fnorm[3 * f + c] = face_n[fi][c].to_double();
            }
        }

    // ---- basis, normalised by its quadrature norms
    Basis B(etype, p);
    if (B.size() != nu) {
        err = "build_ref_ops: basis size mismatch";
        return FR_ERR_ARG;
    }
    std::vector<Vec3> qp;
    std::vector<R> qw;
    rule_volume(etype, p + 3, qp, qw);
    std::vector<R> phi(nu), dphi(3 * nu);
    {
        std::vector<R> nrm(nu, R(0.0));
        for (size_t q = 0; q < qp.size(); ++q) {
            B.eval(qp[q], phi.data(), nullptr);
            for (int m = 0; m < nu; ++m) nrm[m] += qw[q] * phi[m] * phi[m];
        }
        for (int m = 0; m < nu; ++m) B.scl[m] = R(1.0) / dd_sqrt(nrm[m]);
    }

    // ---- Vandermonde, interpolation, derivatives
    Mat Vm(nu, nu), Vd[3] = {Mat(nu, nu), Mat(nu, nu), Mat(nu, nu)};
    for (int j = 0; j < nu; ++j) {
        B.eval(up[j], phi.data(), dphi.data());
        for (int m = 0; m < nu; ++m) {
            Vm(j, m) = phi[m];
            for (int d = 0; d < 3; ++d) Vd[d](j, m) = dphi[d * nu + m];
        }
    }
    Mat Vinv;
    if (!solve(Vm, identity(nu), Vinv)) {
        err = "build_ref_ops: singular Vandermonde";
        return FR_ERR_ARG;
    }
    Mat Vf(nf, nu);
    for (int f = 0; f < nf; ++f) {
        B.eval(fp[f], phi.data(), nullptr);
        for (int m = 0; m < nu; ++m) Vf(f, m) = phi[m];
    }
    Mat M0 = matmul(Vf, Vinv);
    Mat Dm[3] = {matmul(Vd[0], Vinv), matmul(Vd[1], Vinv), matmul(Vd[2], Vinv)};

    // ---- mass matrix (the identity up to rounding) and basis integrals
    Mat Mass(nu, nu);
    std::vector<R> intphi(nu, R(0.0));
    for (size_t q = 0; q < qp.size(); ++q) {
        B.eval(qp[q], phi.data(), nullptr);
        for (int m = 0; m < nu; ++m) {
            intphi[m] += qw[q] * phi[m];
            const R wp = qw[q] * phi[m];
            for (int n2 = 0; n2 < nu; ++n2) Mass(m, n2) += wp * phi[n2];
        }
    }

    // ---- face moments  Bf[m][f] = int_F phi_m l_f dS, and the face
    // weights FWr[f] = int_F l_f dS (l_f the face Lagrange function)
    Mat Bf(nu, nf);
    std::vector<R> FWr(nf, R(0.0));
    for (int fi = 0; fi < o.nfaces; ++fi) {
        const auto &fv = o.face_verts[fi];
        const bool tri = fv.size() == 3;
        const auto &idx = o.face_fpts[fi];
        const int nk = (int)idx.size();
        FaceBasis FB(tri, p);
        if ((int)FB.ex.size() != nk) {
            err = "build_ref_ops: face basis size mismatch";
            return FR_ERR_ARG;
        }
        Mat W(nk, nk);
        std::vector<R> psi(nk);
        for (int k = 0; k < nk; ++k) {
            FB.eval(fparam[idx[k]][0], fparam[idx[k]][1], psi.data());
            for (int q = 0; q < nk; ++q) W(k, q) = psi[q];
        }
        Mat Winv;
        if (!solve(W, identity(nk), Winv)) {
            err = "build_ref_ops: singular face Vandermonde";
            return FR_ERR_ARG;
        }
        std::vector<std::array<R, 2>> rp;
        std::vector<R> rw;
        const int nq = p + 3;
        if (tri) {
            std::vector<std::array<R, 2>> tp;
            std::vector<R> tw;
            rule_unit_tri(nq, tp, tw);
            for (size_t q = 0; q < tp.size(); ++q) {
                rp.push_back({R(2.0) * tp[q][0] - R(1.0), R(2.0) * tp[q][1] - R(1.0)});
                rw.push_back(R(4.0) * tw[q]);
            }
        } else {
            std::vector<R> x, w;
            gl_dd(nq, x, w);
            for (int a = 0; a < nq; ++a)
                for (int b = 0; b < nq; ++b) {
                    rp.push_back({x[a], x[b]});
                    rw.push_back(w[a] * w[b]);
                }
        }
        const R scale = face_area[fi] / R(tri ? 2.0 : 4.0);
        const Vec3 A = V[fv[0]], Bv = V[fv[1]], C = V[fv[2]];
        const Vec3 Dv = tri ? C : V[fv[3]];
        const R one(1.0), q4(0.25), half(0.5);
        for (size_t q = 0; q < rp.size(); ++q) {
            const R r = rp[q][0], s = rp[q][1];
            Vec3 x;
            if (tri) {
                R l1 = half * (r + one), l2 = half * (s + one), l0 = one - l1 - l2;
                for (int c = 0; c < 3; ++c) x[c] = l0 * A[c] + l1 * Bv[c] + l2 * C[c];
            } else {
                for (int c = 0; c < 3; ++c)
                    x[c] = q4 * (A[c] * (one - r) * (one - s) + Bv[c] * (one + r) * (one - s) +
                                 C[c] * (one + r) * (one + s) + Dv[c] * (one - r) * (one + s));
            }
            FB.eval(r, s, psi.data());
            std::vector<R> ell(nk, R(0.0));
            for (int k = 0; k < nk; ++k)
                for (int qq = 0; qq < nk; ++qq) ell[k] += psi[qq] * Winv(qq, k);
            B.eval(x, phi.data(), nullptr);
            const R wq = rw[q] * scale;
            for (int k = 0; k < nk; ++k) FWr[idx[k]] += wq * ell[k];
            for (int m = 0; m < nu; ++m) {
                const R wp = wq * phi[m];
                for (int k = 0; k < nk; ++k) Bf(m, idx[k]) += wp * ell[k];
            }
        }
    }
    Mat Cc;
    if (!solve(Mass, Bf, Cc)) {
        err = "build_ref_ops: singular mass matrix";
        return FR_ERR_ARG;
    }
    Mat M3 = matmul(Vm, Cc);

    // ---- store (rounded once to double)
    o.M0 = to_d(M0.a);
    o.M3 = to_d(M3.a);
    o.D.assign((size_t)3 * nu * nu, 0.0);
    for (int j = 0; j < nu; ++j)
        for (int d = 0; d < 3; ++d)
            for (int i = 0; i < nu; ++i) o.D[((size_t)(j * 3 + d)) * nu + i] = Dm[d](j, i).to_double();
    o.FW.assign(nf, 0.0);
    for (int f = 0; f < nf; ++f) o.FW[f] = FWr[f].to_double();
    o.W.assign(nu, 0.0);
    for (int j = 0; j < nu; ++j) {
        R s(0.0);
        for (int m = 0; m < nu; ++m) s += intphi[m] * Vinv(m, j);
        o.W[j] = s.to_double();
    }

    // corrected-gradient operator [D | n^ (x) M3], rows (j, d)
    const int kg = nu + nf;
    o.AGRAD.assign((size_t)3 * nu * kg, 0.0);
    for (int j = 0; j < nu; ++j)
        for (int d = 0; d < 3; ++d) {
            double *row = &o.AGRAD[((size_t)(j * 3 + d)) * kg];
            for (int i = 0; i < nu; ++i) row[i] = Dm[d](j, i).to_double();
            for (int f = 0; f < nf; ++f) row[nu + f] = (face_n[o.fface[f]][d] * M3(j, f)).to_double();
        }
    // divergence-plus-correction operator [M1 - M3 M2 | M3]; the product
    // M3 M2 (M2 = n^ (x) M0) is formed in double-double before rounding
    const int kd = 3 * nu + nf;
    o.ADIV.assign((size_t)nu * kd, 0.0);
    for (int j = 0; j < nu; ++j) {
        double *row = &o.ADIV[(size_t)j * kd];
        for (int i = 0; i < nu; ++i)
            for (int d = 0; d < 3; ++d) {
                R s = Dm[d](j, i);
                for (int f = 0; f < nf; ++f) s -= M3(j, f) * face_n[o.fface[f]][d] * M0(f, i);
                row[i * 3 + d] = s.to_double();
            }
        for (int f = 0; f < nf; ++f) row[3 * nu + f] = M3(j, f).to_double();
    }
    // Entries that vanish in exact arithmetic (the prism's triangle x line
    // structure zeroes most of its operators) come out of the double-double
    // construction as residue of order 1e-32 next to O(1) entries; they are
    // set to exact zeros, which the operator kernels may then skip.
    for (std::vector<double> *m : {&o.M0, &o.D, &o.M3, &o.AGRAD, &o.ADIV}) {
        double mx = 0.0;
        for (double v : *m) mx = std::max(mx, std::fabs(v));
        for (double &v : *m)
            if (std::fabs(v) < 1e-20 * mx) v = 0.0;
    }
    return FR_OK;
}
}  // namespace

// Transfer between orders (restriction p_from > p_to, prolongation p_from <
// p_to) as the L2 projection onto the target space in the reference element.
// The Dubiner polynomials of order max(p_from, p_to) are mutually orthogonal
// and each space is spanned by a subset of them (tet: i+j+k <= p; prism:
// i+j <= p and k <= p; hex: i, j, k <= p), so the projection keeps the modal coefficients the
// target space shares with the source and drops the rest:
//   R = V_to[:, shared] (V_from^-1)[shared, :],
// V the Vandermondes of each space's modes at its own solution points.
int build_transfer(int etype, int p_from, int p_to, std::vector<double> &out, std::string &err) {
    RefOps from, to;
    int rc = build_ref_ops(etype, p_from, from, err);
    if (rc) return rc;
    if ((rc = build_ref_ops(etype, p_to, to, err))) return rc;
    const int pm = std::max(p_from, p_to);
    Basis B(etype, pm);
    auto in_space = [etype](const std::array<int, 3> &e, int p) {
        if (etype == FR_ETYPE_HEX) return e[0] <= p && e[1] <= p && e[2] <= p;
        return etype == FR_ETYPE_TET ? (e[0] + e[1] + e[2] <= p) : (e[0] + e[1] <= p && e[2] <= p);
    };
    std::vector<int> mf, mt;  // modes of each space (indices into B)
    for (int m = 0; m < B.size(); ++m) {
        if (in_space(B.ex[m], p_from)) mf.push_back(m);
        if (in_space(B.ex[m], p_to)) mt.push_back(m);
    }
    const int nf = from.nu, nt = to.nu;
    if ((int)mf.size() != nf || (int)mt.size() != nt) {
        err = "build_transfer: basis size mismatch";
        return FR_ERR_ARG;
    }
    std::vector<R> phi(B.size());
    Mat Vf(nf, nf);
    for (int j = 0; j < nf; ++j) {
        const Vec3 x = {R(from.upts[3 * j]), R(from.upts[3 * j + 1]), R(from.upts[3 * j + 2])};
        B.eval(x, phi.data(), nullptr);
        for (int a = 0; a < nf; ++a) Vf(j, a) = phi[mf[a]];
    }
    Mat Vfi;
    if (!solve(Vf, identity(nf), Vfi)) {
        err = "build_transfer: singular Vandermonde";
        return FR_ERR_ARG;
    }
    out.assign((size_t)nt * nf, 0.0);
    for (int i = 0; i < nt; ++i) {
        const Vec3 x = {R(to.upts[3 * i]), R(to.upts[3 * i + 1]), R(to.upts[3 * i + 2])};
        B.eval(x, phi.data(), nullptr);
        for (int j = 0; j < nf; ++j) {
            DD s(0.0);
            for (int a = 0; a < nf; ++a)
                if (in_space(B.ex[mf[a]], p_to)) s += phi[mf[a]] * Vfi(a, j);
            out[(size_t)i * nf + j] = s.to_double();
        }
    }
    return FR_OK;
}

}  // namespace fr
