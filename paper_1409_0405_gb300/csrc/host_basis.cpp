// Host construction of the FR points and operator matrices.
//
// Basis: the orthogonal collapsed-coordinate (Dubiner) polynomials of the
// element space (tet: P_p; prism: P_p(triangle) x P_p(zeta)), whose
// dimensions are Table 2's solution-point counts:
//   tet  psi_ijk = P_i(a) ((1-b)/2)^i P_j^(2i+1,0)(b) ((1-c)/2)^(i+j)
//                  P_k^(2i+2j+2,0)(c),
//        a = 2(1+xi)/(-eta-zeta) - 1, b = 2(1+eta)/(1-zeta) - 1, c = zeta;
//   tri  psi_ij = P_i(a) ((1-b)/2)^i P_j^(2i+1,0)(b),
//        a = 2(1+xi)/(1-eta) - 1, b = eta;
//   prism: tri x Legendre P_k(zeta);  quad faces: Legendre x Legendre.
// They are polynomials in the reference coordinates; their derivatives are
// taken exactly with forward-mode dual numbers (every evaluation point lies
// off the collapsed edge), and each is normalised by its quadrature norm, so
// the mass matrix is the identity up to rounding and every Vandermonde is
// well conditioned.  Integrals use collapsed (Duffy) Gauss-Legendre rules
// exact for the degrees involved.
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
#include <array>
#include <cmath>
#include <string>
#include <vector>

#include "fr_internal.h"

namespace fr {
namespace {

const double TET_V[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
const double PRI_V[6][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1},
                            {-1, -1, 1},  {1, -1, 1},  {-1, 1, 1}};
const std::vector<std::vector<int>> TET_FACES = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
const std::vector<std::vector<int>> PRI_FACES = {
    {0, 1, 2}, {3, 4, 5}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};

using Vec3 = std::array<double, 3>;

struct Mat {
    int r = 0, c = 0;
    std::vector<double> a;
    Mat() {}
    Mat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_, 0.0) {}
    double &operator()(int i, int j) { return a[(size_t)i * c + j]; }
    double operator()(int i, int j) const { return a[(size_t)i * c + j]; }
};

Mat matmul(const Mat &A, const Mat &B) {
    Mat C(A.r, B.c);
    for (int i = 0; i < A.r; ++i)
        for (int k = 0; k < A.c; ++k) {
            double aik = A(i, k);
            if (aik == 0.0) continue;
            for (int j = 0; j < B.c; ++j) C(i, j) += aik * B(k, j);
        }
    return C;
}

// Solve A X = B by LU with partial pivoting plus one step of iterative
// refinement.  Returns false if A is singular.
bool solve(const Mat &A, const Mat &B, Mat &X) {
    int n = A.r;
    Mat LU = A;
    std::vector<int> piv(n);
    for (int i = 0; i < n; ++i) piv[i] = i;
    for (int k = 0; k < n; ++k) {
        int pr = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(LU(i, k)) > std::fabs(LU(pr, k))) pr = i;
        if (LU(pr, k) == 0.0) return false;
        if (pr != k) {
            for (int j = 0; j < n; ++j) std::swap(LU(k, j), LU(pr, j));
            std::swap(piv[k], piv[pr]);
        }
        for (int i = k + 1; i < n; ++i) {
            LU(i, k) /= LU(k, k);
            double l = LU(i, k);
            for (int j = k + 1; j < n; ++j) LU(i, j) -= l * LU(k, j);
        }
    }
    auto lu_solve = [&](const Mat &rhs, Mat &out) {
        out = Mat(n, rhs.c);
        for (int col = 0; col < rhs.c; ++col) {
            std::vector<double> y(n);
            for (int i = 0; i < n; ++i) {
                double s = rhs(piv[i], col);
                for (int j = 0; j < i; ++j) s -= LU(i, j) * y[j];
                y[i] = s;
            }
            for (int i = n - 1; i >= 0; --i) {
                double s = y[i];
                for (int j = i + 1; j < n; ++j) s -= LU(i, j) * out(j, col);
                out(i, col) = s / LU(i, i);
            }
        }
    };
    lu_solve(B, X);
    // one refinement step: X += A^{-1} (B - A X)
    Mat AX = matmul(A, X);
    Mat res(n, B.c);
    for (size_t i = 0; i < res.a.size(); ++i) res.a[i] = B.a[i] - AX.a[i];
    Mat dX;
    lu_solve(res, dX);
    for (size_t i = 0; i < X.a.size(); ++i) X.a[i] += dX.a[i];
    return true;
}

Mat identity(int n) {
    Mat I(n, n);
    for (int i = 0; i < n; ++i) I(i, i) = 1.0;
    return I;
}

// Blyth-Pozrikidis barycentric coordinates of multi-index I from the 1-D
// nodes v on [0, 1]: lambda_a = (1 + d v_{I_a} - sum_{b != a} v_{I_b}) / (d+1)
template <int NB>
std::array<double, NB> bp_bary(const std::array<int, NB> &I, const std::vector<double> &v) {
    const int d = NB - 1;
    double tot = 0.0;
    for (int a = 0; a < NB; ++a) tot += v[I[a]];
    std::array<double, NB> lam;
    for (int a = 0; a < NB; ++a) lam[a] = (1.0 + d * v[I[a]] - (tot - v[I[a]])) / (d + 1);
    return lam;
}

std::vector<double> gl01(int n) {
    std::vector<double> x, w;
    gauss_legendre(n, x, w);
    for (auto &xi : x) xi = 0.5 * (xi + 1.0);
    return x;
}

std::vector<std::array<double, 3>> tri_set(int p) {
    std::vector<double> v = gl01(p + 1);
    std::vector<std::array<double, 3>> out;
    for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= p - j; ++i) out.push_back(bp_bary<3>({p - i - j, i, j}, v));
    return out;
}

// forward-mode dual number with three partial derivatives
struct Dual {
    double v, d[3];
};
inline Dual dc(double c) { return {c, {0, 0, 0}}; }
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}}; }
inline Dual operator*(Dual a, Dual b) {
    return {a.v * b.v, {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1], a.d[2] * b.v + a.v * b.d[2]}};
}
inline Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return {q, {(a.d[0] - q * b.d[0]) / b.v, (a.d[1] - q * b.d[1]) / b.v, (a.d[2] - q * b.d[2]) / b.v}};
}
inline Dual operator*(double c, Dual a) { return {c * a.v, {c * a.d[0], c * a.d[1], c * a.d[2]}}; }
inline Dual operator+(double c, Dual a) { return {c + a.v, {a.d[0], a.d[1], a.d[2]}}; }
inline Dual operator-(double c, Dual a) { return {c - a.v, {-a.d[0], -a.d[1], -a.d[2]}}; }
Dual dpow(Dual a, int n) {
    Dual r = dc(1.0);
    for (int i = 0; i < n; ++i) r = r * a;
    return r;
}

// Jacobi polynomial P_n^(al, 0)(x) (unnormalised three-term recurrence)
Dual jacobi(int n, double al, Dual x) {
    const double be = 0.0;
    Dual p0 = dc(1.0);
    if (n == 0) return p0;
    Dual p1 = 0.5 * ((al + be + 2.0) * x) + dc(0.5 * (al - be));
    for (int k = 2; k <= n; ++k) {
        const double s = 2.0 * k + al + be;
        const double A = 2.0 * k * (k + al + be) * (s - 2.0);
        const double B = (s - 1.0) * s * (s - 2.0);
        const double Cc = (s - 1.0) * (al * al - be * be);
        const double Dd = 2.0 * (k + al - 1.0) * (k + be - 1.0) * s;
        Dual p2 = (1.0 / A) * ((B * x + dc(Cc)) * p1 - Dd * p0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

struct Basis {
    int etype, p;
    std::vector<std::array<int, 3>> ex;
    std::vector<double> scale;  // 1 / quadrature norm of each function
    explicit Basis(int et, int p_) : etype(et), p(p_) {
        for (int c = 0; c <= p; ++c)
            for (int b = 0; b <= p; ++b)
                for (int a = 0; a <= p; ++a) {
                    bool in = (etype == FR_ETYPE_TET) ? (a + b + c <= p) : (a + b <= p);
                    if (in) ex.push_back({a, b, c});
                }
        scale.assign(ex.size(), 1.0);
    }
    int size() const { return (int)ex.size(); }
    Dual raw(int m, const Vec3 &x) const {
        Dual xi{x[0], {1, 0, 0}}, eta{x[1], {0, 1, 0}}, zeta{x[2], {0, 0, 1}};
        const int i = ex[m][0], j = ex[m][1], k = ex[m][2];
        if (etype == FR_ETYPE_TET) {
            Dual a = (2.0 * (1.0 + xi)) / (dc(0.0) - eta - zeta) - dc(1.0);
            Dual b = (2.0 * (1.0 + eta)) / (1.0 - zeta) - dc(1.0);
            Dual c = zeta;
            return jacobi(i, 0, a) * dpow(0.5 * (1.0 - b), i) * jacobi(j, 2 * i + 1, b) *
                   dpow(0.5 * (1.0 - c), i + j) * jacobi(k, 2 * i + 2 * j + 2, c);
        }
        Dual a = (2.0 * (1.0 + xi)) / (1.0 - eta) - dc(1.0);
        Dual b = eta;
        return jacobi(i, 0, a) * dpow(0.5 * (1.0 - b), i) * jacobi(j, 2 * i + 1, b) * jacobi(k, 0, zeta);
    }
    // values (and optionally the three derivatives) of every basis function at x
    void eval(const Vec3 &x, double *phi, double *dphi /* size 3 x n or null */) const {
        const int n = size();
        for (int m = 0; m < n; ++m) {
            Dual r = raw(m, x);
            phi[m] = scale[m] * r.v;
            if (dphi)
                for (int d = 0; d < 3; ++d) dphi[d * n + m] = scale[m] * r.d[d];
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
    void eval(double r, double s, double *psi) const {
        Dual R{r, {1, 0, 0}}, S{s, {0, 1, 0}};
        for (size_t m = 0; m < ex.size(); ++m) {
            const int i = ex[m][0], j = ex[m][1];
            if (tri) {
                Dual a = (2.0 * (1.0 + R)) / (1.0 - S) - dc(1.0);
                psi[m] = (jacobi(i, 0, a) * dpow(0.5 * (1.0 - S), i) * jacobi(j, 2 * i + 1, S)).v;
            } else {
                psi[m] = (jacobi(i, 0, R) * jacobi(j, 0, S)).v;
            }
        }
    }
};

// Collapsed Gauss rules.  Each returns points in the relevant parameter
// domain and weights summing to its measure.
void rule_unit_tri(int n, std::vector<std::array<double, 2>> &pts, std::vector<double> &wts) {
    std::vector<double> x, w;
    gauss_legendre(n, x, w);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double u = 0.5 * (x[a] + 1), v = 0.5 * (x[b] + 1);
            double wu = 0.5 * w[a], wv = 0.5 * w[b];
            pts.push_back({u, v * (1 - u)});
            wts.push_back(wu * wv * (1 - u));
        }
}

void rule_volume(int etype, int n, std::vector<Vec3> &pts, std::vector<double> &wts) {
    std::vector<double> x, w;
    gauss_legendre(n, x, w);
    if (etype == FR_ETYPE_TET) {
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b)
                for (int c = 0; c < n; ++c) {
                    double u = 0.5 * (x[a] + 1), v = 0.5 * (x[b] + 1), t = 0.5 * (x[c] + 1);
                    double px = u, py = v * (1 - u), pz = t * (1 - u) * (1 - v);
                    pts.push_back({2 * px - 1, 2 * py - 1, 2 * pz - 1});
                    wts.push_back(8.0 * 0.125 * w[a] * w[b] * w[c] * (1 - u) * (1 - u) * (1 - v));
                }
    } else {
        std::vector<std::array<double, 2>> tp;
        std::vector<double> tw;
        rule_unit_tri(n, tp, tw);
        for (int c = 0; c < n; ++c)
            for (size_t q = 0; q < tp.size(); ++q) {
                pts.push_back({2 * tp[q][0] - 1, 2 * tp[q][1] - 1, x[c]});
                wts.push_back(4.0 * tw[q] * w[c]);
            }
    }
}

Vec3 vsub(const Vec3 &a, const Vec3 &b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
Vec3 vcross(const Vec3 &a, const Vec3 &b) {
    return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
double vnorm(const Vec3 &a) { return std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

}  // namespace

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = -std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) {
                p0 = 1.0;
                p1 = z;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged root for the weight
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

int nupts_of(int etype, int p) {
    return etype == FR_ETYPE_TET ? (p + 1) * (p + 2) * (p + 3) / 6 : (p + 1) * (p + 1) * (p + 2) / 2;
}

int nfpts_of(int etype, int p) {
    return etype == FR_ETYPE_TET ? 4 * (p + 1) * (p + 2) / 2
                                 : 2 * (p + 1) * (p + 2) / 2 + 3 * (p + 1) * (p + 1);
}

int build_ref_ops(int etype, int p, RefOps &o, std::string &err) {
    if ((etype != FR_ETYPE_TET && etype != FR_ETYPE_PRI) || p < 1 || p > 4) {
        err = "build_ref_ops: etype must be 0/1 and order 1..4";
        return FR_ERR_ARG;
    }
    o = RefOps();
    o.etype = etype;
    o.p = p;
    const bool tet = etype == FR_ETYPE_TET;
    const int nverts = tet ? 4 : 6;
    std::vector<Vec3> V(nverts);
    for (int i = 0; i < nverts; ++i)
        for (int k = 0; k < 3; ++k) V[i][k] = tet ? TET_V[i][k] : PRI_V[i][k];
    o.face_verts = tet ? TET_FACES : PRI_FACES;
    o.nfaces = (int)o.face_verts.size();

    // ---- solution points
    std::vector<Vec3> up;
    std::vector<double> glx, glw;
    gauss_legendre(p + 1, glx, glw);
    if (tet) {
        std::vector<double> v = gl01(p + 1);
        for (int k = 0; k <= p; ++k)
            for (int j = 0; j <= p - k; ++j)
                for (int i = 0; i <= p - k - j; ++i) {
                    auto lam = bp_bary<4>({p - i - j - k, i, j, k}, v);
                    Vec3 x = {0, 0, 0};
                    for (int a = 0; a < 4; ++a)
                        for (int c = 0; c < 3; ++c) x[c] += lam[a] * V[a][c];
                    up.push_back(x);
                }
    } else {
        auto tri = tri_set(p);
        for (int c = 0; c <= p; ++c)
            for (auto &lam : tri) {
                double xi = 0, eta = 0;
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
    std::vector<std::array<double, 2>> fparam;
    std::vector<Vec3> face_n(o.nfaces);
    std::vector<double> face_area(o.nfaces);
    o.face_fpts.assign(o.nfaces, {});
    Vec3 cen_e = {0, 0, 0};
    for (auto &v : V)
        for (int c = 0; c < 3; ++c) cen_e[c] += v[c] / nverts;
    for (int fi = 0; fi < o.nfaces; ++fi) {
        const auto &fv = o.face_verts[fi];
        const bool tri = fv.size() == 3;
        Vec3 A = V[fv[0]], B = V[fv[1]], C = V[fv[2]];
        Vec3 Dq = tri ? C : V[fv[3]];
        Vec3 cr = vcross(vsub(B, A), vsub(Dq, A));
        double nn = vnorm(cr);
        face_area[fi] = tri ? 0.5 * nn : nn;
        Vec3 n = {cr[0] / nn, cr[1] / nn, cr[2] / nn};
        Vec3 cen_f = {0, 0, 0};
        for (int vi : fv)
            for (int c = 0; c < 3; ++c) cen_f[c] += V[vi][c] / fv.size();
        double s = 0;
        for (int c = 0; c < 3; ++c) s += (cen_f[c] - cen_e[c]) * n[c];
        if (s < 0)
            for (int c = 0; c < 3; ++c) n[c] = -n[c];
        face_n[fi] = n;
        if (tri) {
            for (auto &lam : tri_set(p)) {
                Vec3 x;
                for (int c = 0; c < 3; ++c) x[c] = lam[0] * A[c] + lam[1] * B[c] + lam[2] * C[c];
                o.face_fpts[fi].push_back((int)fp.size());
                fp.push_back(x);
                fparam.push_back({2 * lam[1] - 1, 2 * lam[2] - 1});
            }
        } else {
            Vec3 Dv = V[fv[3]];
            for (int b = 0; b <= p; ++b)
                for (int a = 0; a <= p; ++a) {
                    double s_ = glx[a], t_ = glx[b];
                    Vec3 x;
                    for (int c = 0; c < 3; ++c)
                        x[c] = 0.25 * (A[c] * (1 - s_) * (1 - t_) + B[c] * (1 + s_) * (1 - t_) +
                                       C[c] * (1 + s_) * (1 + t_) + Dv[c] * (1 - s_) * (1 + t_));
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
        for (int c = 0; c < 3; ++c) o.upts[3 * j + c] = up[j][c];
    for (int fi = 0; fi < o.nfaces; ++fi)
        for (int f : o.face_fpts[fi]) {
            o.fface[f] = fi;
            for (int c = 0; c < 3; ++c) {
                o.fpts[3 * f + c] = fp[f][c];
                o.fnorm[3 * f + c] = face_n[fi][c];
            }
        }

    // ---- basis, normalised by its quadrature norms
    Basis B(etype, p);
    if (B.size() != nu) {
        err = "build_ref_ops: basis size mismatch";
        return FR_ERR_ARG;
    }
    std::vector<Vec3> qp;
    std::vector<double> qw;
    rule_volume(etype, p + 3, qp, qw);
    {
        std::vector<double> nrm(nu, 0.0), v(nu);
        for (size_t q = 0; q < qp.size(); ++q) {
            B.eval(qp[q], v.data(), nullptr);
            for (int m = 0; m < nu; ++m) nrm[m] += qw[q] * v[m] * v[m];
        }
        for (int m = 0; m < nu; ++m) B.scale[m] = 1.0 / std::sqrt(nrm[m]);
    }

    // ---- Vandermonde, interpolation, derivatives
    Mat Vm(nu, nu), Vd[3] = {Mat(nu, nu), Mat(nu, nu), Mat(nu, nu)};
    std::vector<double> phi(nu), dphi(3 * nu);
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
    std::vector<double> intphi(nu, 0.0);
    for (size_t q = 0; q < qp.size(); ++q) {
        B.eval(qp[q], phi.data(), nullptr);
        for (int m = 0; m < nu; ++m) {
            intphi[m] += qw[q] * phi[m];
            for (int n2 = 0; n2 < nu; ++n2) Mass(m, n2) += qw[q] * phi[m] * phi[n2];
        }
    }

    // ---- face moments  Bf[m][f] = int_F phi_m l_f dS
    Mat Bf(nu, nf);
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
        std::vector<double> psi(nk);
        for (int k = 0; k < nk; ++k) {
            FB.eval(fparam[idx[k]][0], fparam[idx[k]][1], psi.data());
            for (int q = 0; q < nk; ++q) W(k, q) = psi[q];
        }
        Mat Winv;
        if (!solve(W, identity(nk), Winv)) {
            err = "build_ref_ops: singular face Vandermonde";
            return FR_ERR_ARG;
        }
        // face quadrature in the parameter domain
        std::vector<std::array<double, 2>> rp;
        std::vector<double> rw;
        const int nq = p + 3;
        if (tri) {
            std::vector<std::array<double, 2>> tp;
            std::vector<double> tw;
            rule_unit_tri(nq, tp, tw);
            for (size_t q = 0; q < tp.size(); ++q) {
                rp.push_back({2 * tp[q][0] - 1, 2 * tp[q][1] - 1});
                rw.push_back(4.0 * tw[q]);
            }
        } else {
            std::vector<double> x, w;
            gauss_legendre(nq, x, w);
            for (int a = 0; a < nq; ++a)
                for (int b = 0; b < nq; ++b) {
                    rp.push_back({x[a], x[b]});
                    rw.push_back(w[a] * w[b]);
                }
        }
        const double scale = face_area[fi] / (tri ? 2.0 : 4.0);
        Vec3 A = V[fv[0]], Bv = V[fv[1]], C = V[fv[2]];
        Vec3 Dv = tri ? C : V[fv[3]];
        for (size_t q = 0; q < rp.size(); ++q) {
            double r = rp[q][0], s = rp[q][1];
            Vec3 x;
            if (tri) {
                double l1 = 0.5 * (r + 1), l2 = 0.5 * (s + 1), l0 = 1 - l1 - l2;
                for (int c = 0; c < 3; ++c) x[c] = l0 * A[c] + l1 * Bv[c] + l2 * C[c];
            } else {
                for (int c = 0; c < 3; ++c)
                    x[c] = 0.25 * (A[c] * (1 - r) * (1 - s) + Bv[c] * (1 + r) * (1 - s) +
                                   C[c] * (1 + r) * (1 + s) + Dv[c] * (1 - r) * (1 + s));
            }
            FB.eval(r, s, psi.data());
            std::vector<double> ell(nk, 0.0);
            for (int k = 0; k < nk; ++k)
                for (int qq = 0; qq < nk; ++qq) ell[k] += psi[qq] * Winv(qq, k);
            B.eval(x, phi.data(), nullptr);
            double wq = rw[q] * scale;
            for (int m = 0; m < nu; ++m)
                for (int k = 0; k < nk; ++k) Bf(m, idx[k]) += wq * phi[m] * ell[k];
        }
    }
    Mat Cc;
    if (!solve(Mass, Bf, Cc)) {
        err = "build_ref_ops: singular mass matrix";
        return FR_ERR_ARG;
    }
    Mat M3 = matmul(Vm, Cc);

    // ---- store
    o.M0 = M0.a;
    o.M3 = M3.a;
    o.D.assign((size_t)3 * nu * nu, 0.0);
    for (int j = 0; j < nu; ++j)
        for (int d = 0; d < 3; ++d)
            for (int i = 0; i < nu; ++i) o.D[((size_t)(j * 3 + d)) * nu + i] = Dm[d](j, i);
    o.W.assign(nu, 0.0);
    for (int j = 0; j < nu; ++j)
        for (int m = 0; m < nu; ++m) o.W[j] += intphi[m] * Vinv(m, j);

    // corrected-gradient operator [D | n^ (x) M3], rows (j, d)
    const int kg = nu + nf;
    o.AGRAD.assign((size_t)3 * nu * kg, 0.0);
    for (int j = 0; j < nu; ++j)
        for (int d = 0; d < 3; ++d) {
            double *row = &o.AGRAD[((size_t)(j * 3 + d)) * kg];
            for (int i = 0; i < nu; ++i) row[i] = Dm[d](j, i);
            for (int f = 0; f < nf; ++f) row[nu + f] = o.fnorm[3 * f + d] * M3(j, f);
        }
    // divergence-plus-correction operator [M1 - M3 M2 | M3]
    const int kd = 3 * nu + nf;
    o.ADIV.assign((size_t)nu * kd, 0.0);
    for (int j = 0; j < nu; ++j) {
        double *row = &o.ADIV[(size_t)j * kd];
        for (int i = 0; i < nu; ++i)
            for (int d = 0; d < 3; ++d) {
                double s = Dm[d](j, i);
                for (int f = 0; f < nf; ++f) s -= M3(j, f) * o.fnorm[3 * f + d] * M0(f, i);
                row[i * 3 + d] = s;
            }
        for (int f = 0; f < nf; ++f) row[3 * nu + f] = M3(j, f);
    }
    return FR_OK;
}

}  // namespace fr
