"""Points and operator matrices of the FR scheme for one element type and
order, built exactly: monomial bases, rational monomial integrals and
Vandermonde solves in 60-digit decimal arithmetic, rounded to float64 once
at the end.

Readings (the paper names no point sets and writes out only M0, Table 2):
  * Spaces: tet P_p; prism P_p(triangle) x P_p(zeta); hex Q_p (degree <= p
    in each coordinate).  Their dimensions are Table 2's solution-point
    counts.
  * Reference tet vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1);
    reference prism = triangle {(-1,-1),(1,-1),(-1,1)} x [-1,1]; reference
    hex = [-1,1]^3, vertices 0..3 the bottom face counter-clockwise from
    (-1,-1,-1), vertex a+4 above vertex a.
  * Solution points: a symmetric, constructive, interior set built from the
    p+1 Gauss-Legendre nodes v_0 < ... < v_p mapped to [0,1] (the
    Blyth-Pozrikidis barycentric construction).  For a simplex with d+1
    vertices and a multi-index I (sum I_a = p), the barycentric coordinates
    are  lambda_a = (1 + d v_{I_a} - sum_{b != a} v_{I_b}) / (d+1).
    Tet: d = 3, I = (p-i-j-k, i, j, k), ordered k, j, i from slowest to
    fastest.  Prism: the triangle set (d = 2, I = (p-i-j, i, j), ordered j, i)
    times the Gauss-Legendre points in zeta, zeta index slowest.  Hex: the
    (p+1)^3 Gauss-Legendre tensor points, zeta slowest, xi fastest.
  * Flux points.  Triangle faces (A, B, C): the same triangle set,
    lambda_0 A + lambda_1 B + lambda_2 C; quad faces (A, B, C, D): Gauss-
    Legendre x Gauss-Legendre in the bilinear parameters (s along A->B, t
    along A->D).  Both sets are invariant under the face's symmetries, so
    the points of two neighbours coincide.  Element flux points are the
    faces' points concatenated in local-face order.
  * M0: Lagrange interpolation from solution to flux points (Table 2).
  * D_d: the reference derivative d/dxi_d of the solution-point Lagrange
    interpolant, evaluated at the solution points.
  * M3: the correction that recovers nodal DG (Sec. 3.4): for flux point f
    on face F, column f of M3 holds at the solution points the polynomial
    g_f of the element space with  int_elem g_f v = int_F l_f v dS
    for every v of the space, where l_f is the Lagrange polynomial of the
    face's trace space at the face's flux points and dS the reference face
    measure.
  * w: w_j = integral over the reference element of the j-th Lagrange
    polynomial.
"""
from __future__ import annotations

import math
from decimal import Decimal, localcontext
from fractions import Fraction
from functools import lru_cache

import numpy as np

PREC = 60

TET_VERTS = ((-1, -1, -1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1))
PRI_VERTS = ((-1, -1, -1), (1, -1, -1), (-1, 1, -1),
             (-1, -1, 1), (1, -1, 1), (-1, 1, 1))
TET_FACES = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
PRI_FACES = ((0, 1, 2), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5))
HEX_VERTS = ((-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1),
             (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1))
HEX_FACES = ((0, 1, 2, 3), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7),
             (4, 5, 6, 7))

ETYPES = ("tet", "pri", "hex")


def _dec(x):
    if isinstance(x, Decimal):
        return x
    if isinstance(x, Fraction):
        return Decimal(x.numerator) / Decimal(x.denominator)
    return Decimal(x)


# --------------------------------------------------------------------------
# Gauss-Legendre nodes (roots of P_n), Newton iteration in decimal
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def gauss_legendre(n):
    with localcontext() as c:
        c.prec = PREC
        eps = Decimal(10) ** (-(PREC - 5))
        nodes = []
        for i in range(n):
            x = Decimal(repr(-math.cos(math.pi * (i + 0.75) / (n + 0.5))))
            for _ in range(200):
                p0, p1 = Decimal(1), x
                for k in range(2, n + 1):
                    p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
                if n == 0:
                    break
                dp = n * (x * p1 - p0) / (x * x - 1)
                dx = p1 / dp
                x -= dx
                if abs(dx) < eps:
                    break
            nodes.append(+x)
        return tuple(sorted(nodes))


# --------------------------------------------------------------------------
# monomial spaces and exact integrals
# --------------------------------------------------------------------------
def exponents(etype, p):
    if etype == "tet":
        return [(a, b, c) for c in range(p + 1) for b in range(p + 1 - c)
                for a in range(p + 1 - b - c)]
    if etype == "hex":
        return [(a, b, c) for c in range(p + 1) for b in range(p + 1)
                for a in range(p + 1)]
    return [(a, b, c) for c in range(p + 1) for b in range(p + 1)
            for a in range(p + 1 - b)]


def face_exponents(kind, p):
    if kind == "tri":
        return [(a, b) for b in range(p + 1) for a in range(p + 1 - b)]
    return [(a, b) for b in range(p + 1) for a in range(p + 1)]


def _shifted(a):
    """(2x-1)^a = sum_i coef_i x^i, exact."""
    return [(i, Fraction(math.comb(a, i) * 2 ** i * (-1) ** (a - i)))
            for i in range(a + 1)]


@lru_cache(maxsize=None)
def int_tri(a, b):
    """Exact integral of xi^a eta^b over {xi, eta >= -1, xi + eta <= 0}."""
    s = Fraction(0)
    for i, ci in _shifted(a):
        for j, cj in _shifted(b):
            s += ci * cj * Fraction(math.factorial(i) * math.factorial(j),
                                    math.factorial(i + j + 2))
    return 4 * s


@lru_cache(maxsize=None)
def int_line(c):
    return Fraction(2, c + 1) if c % 2 == 0 else Fraction(0)


@lru_cache(maxsize=None)
def int_tet(a, b, c):
    """Exact integral of xi^a eta^b zeta^c over the reference tet."""
    s = Fraction(0)
    for i, ci in _shifted(a):
        for j, cj in _shifted(b):
            for k, ck in _shifted(c):
                s += ci * cj * ck * Fraction(
                    math.factorial(i) * math.factorial(j) * math.factorial(k),
                    math.factorial(i + j + k + 3))
    return 8 * s


def int_elem(etype, e):
    if etype == "tet":
        return int_tet(*e)
    if etype == "hex":
        return int_line(e[0]) * int_line(e[1]) * int_line(e[2])
    return int_tri(e[0], e[1]) * int_line(e[2])


def int_face_param(kind, e):
    """Integral of r^a s^b over the face parameter domain (reference
    triangle for 'tri', [-1,1]^2 for 'quad')."""
    if kind == "tri":
        return int_tri(*e)
    return int_line(e[0]) * int_line(e[1])


def _mono(e, x):
    r = Decimal(1)
    for ei, xi in zip(e, x):
        if ei:
            r *= xi ** ei
    return r


def _dmono(e, x, d):
    if e[d] == 0:
        return Decimal(0)
    r = Decimal(e[d])
    for k, (ei, xi) in enumerate(zip(e, x)):
        pw = ei - 1 if k == d else ei
        if pw:
            r *= xi ** pw
    return r


# --------------------------------------------------------------------------
# dense decimal linear algebra
# --------------------------------------------------------------------------
def _solve(A, B):
    """Solve A X = B (lists of lists of Decimal) by Gauss-Jordan elimination
    with partial pivoting."""
    n = len(A)
    m = len(B[0])
    M = [list(A[i]) + list(B[i]) for i in range(n)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(M[r][col]))
        if M[piv][col] == 0:
            raise ValueError("singular matrix")
        M[col], M[piv] = M[piv], M[col]
        inv = 1 / M[col][col]
        rowc = [v * inv for v in M[col]]
        M[col] = rowc
        for r in range(n):
            if r != col:
                f = M[r][col]
                if f != 0:
                    rr = M[r]
                    M[r] = [a - f * b for a, b in zip(rr, rowc)]
    return [row[n:n + m] for row in M]


def _matmul(A, B):
    Bt = list(zip(*B))
    return [[sum((a * b for a, b in zip(row, col)), Decimal(0)) for col in Bt]
            for row in A]


def _eye(n):
    return [[Decimal(1) if i == j else Decimal(0) for j in range(n)]
            for i in range(n)]


# --------------------------------------------------------------------------
# points
# --------------------------------------------------------------------------
def nupts(etype, p):
    if etype == "tet":
        return (p + 1) * (p + 2) * (p + 3) // 6
    if etype == "hex":
        return (p + 1) ** 3
    return (p + 1) ** 2 * (p + 2) // 2


def nfpts(etype, p):
    if etype == "tet":
        return 4 * (p + 1) * (p + 2) // 2
    if etype == "hex":
        return 6 * (p + 1) ** 2
    return 2 * (p + 1) * (p + 2) // 2 + 3 * (p + 1) ** 2


def _bp_bary(I, v):
    """Blyth-Pozrikidis barycentric coordinates of multi-index I from the
    1-D nodes v on [0, 1]."""
    d = len(I) - 1
    tot = sum(v[i] for i in I)
    return [(1 + d * v[I[a]] - (tot - v[I[a]])) / (d + 1) for a in range(d + 1)]


def _gl01(n):
    return [(x + 1) / 2 for x in gauss_legendre(n)]


def tri_bary(p):
    """Barycentric coordinates of the triangle point set, order j, i."""
    v = _gl01(p + 1)
    return [_bp_bary((p - i - j, i, j), v) for j in range(p + 1)
            for i in range(p + 1 - j)]


def upts_exact(etype, p):
    pts = []
    if etype == "tet":
        v = _gl01(p + 1)
        X = [[Decimal(c) for c in x] for x in TET_VERTS]
        for k in range(p + 1):
            for j in range(p + 1 - k):
                for i in range(p + 1 - k - j):
                    lam = _bp_bary((p - i - j - k, i, j, k), v)
                    pts.append(tuple(sum(lam[a] * X[a][c] for a in range(4))
                                     for c in range(3)))
    elif etype == "hex":
        gl = gauss_legendre(p + 1)
        for c in range(p + 1):
            for b in range(p + 1):
                for a in range(p + 1):
                    pts.append((gl[a], gl[b], gl[c]))
    else:
        gl = gauss_legendre(p + 1)
        X = [[Decimal(c) for c in x] for x in PRI_VERTS[:3]]
        tri = [tuple(sum(lam[a] * X[a][c] for a in range(3)) for c in range(2))
               for lam in tri_bary(p)]
        for c in range(p + 1):
            for (x, y) in tri:
                pts.append((x, y, gl[c]))
    return pts


def faces(etype):
    return {"tet": (TET_VERTS, TET_FACES), "pri": (PRI_VERTS, PRI_FACES),
            "hex": (HEX_VERTS, HEX_FACES)}[etype]


def _face_geometry(verts, fv):
    """Outward unit reference normal and reference area of a face."""
    A = [Decimal(v) for v in verts[fv[0]]]
    B = [Decimal(v) for v in verts[fv[1]]]
    C = [Decimal(v) for v in verts[fv[2] if len(fv) == 3 else fv[3]]]
    u = [b - a for a, b in zip(A, B)]
    v = [c - a for a, c in zip(A, C)]
    cr = [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
          u[0] * v[1] - u[1] * v[0]]
    nrm = sum(x * x for x in cr).sqrt()
    area = nrm / 2 if len(fv) == 3 else nrm
    n = [x / nrm for x in cr]
    cen_e = [sum(Decimal(v[k]) for v in verts) / len(verts) for k in range(3)]
    cen_f = [sum(Decimal(verts[i][k]) for i in fv) / len(fv) for k in range(3)]
    if sum((cf - ce) * nk for cf, ce, nk in zip(cen_f, cen_e, n)) < 0:
        n = [-x for x in n]
    return n, area


def fpts_exact(etype, p):
    """Flux points: list of (xyz_ref, face index, face-parameter coords)."""
    verts, flist = faces(etype)
    out = []
    gl = gauss_legendre(p + 1)
    for fi, fv in enumerate(flist):
        V = [[Decimal(c) for c in verts[i]] for i in fv]
        if len(fv) == 3:
            for (m0, m1, m2) in tri_bary(p):
                x = tuple(m0 * V[0][k] + m1 * V[1][k] + m2 * V[2][k]
                          for k in range(3))
                out.append((x, fi, (2 * m1 - 1, 2 * m2 - 1)))
        else:
            for b in range(p + 1):
                for a in range(p + 1):
                    s, t = gl[a], gl[b]
                    w = ((1 - s) * (1 - t) / 4, (1 + s) * (1 - t) / 4,
                         (1 + s) * (1 + t) / 4, (1 - s) * (1 + t) / 4)
                    x = tuple(sum(w[n] * V[n][k] for n in range(4))
                              for k in range(3))
                    out.append((x, fi, (s, t)))
    return out


# --------------------------------------------------------------------------
# operators
# --------------------------------------------------------------------------
class Operators:
    """float64 operators of one (etype, p).

    upts (Nu,3), fpts (Nf,3) reference coordinates; fface (Nf,) face index of
    each flux point; fnorm (Nf,3) outward unit reference normal at each flux
    point; nfaces; M0 (Nf,Nu); D (3,Nu,Nu) with D[d] @ u = d u / d xi_d at
    the solution points; M3 (Nu,Nf); w (Nu,); fw (Nf,) the integral of each
    flux point's face Lagrange polynomial over its face.
    """


@lru_cache(maxsize=None)
def operators(etype, p):
    with localcontext() as c:
        c.prec = PREC
        ex = exponents(etype, p)
        up = upts_exact(etype, p)
        fp = fpts_exact(etype, p)
        nu, nf = len(up), len(fp)
        assert nu == len(ex) == nupts(etype, p) and nf == nfpts(etype, p)
        verts, flist = faces(etype)
        fgeo = [_face_geometry(verts, fv) for fv in flist]

        V = [[_mono(e, x) for e in ex] for x in up]
        Vinv = _solve(V, _eye(nu))
        Vf = [[_mono(e, x) for e in ex] for (x, _, _) in fp]
        M0 = _matmul(Vf, Vinv)
        Dm = []
        for d in range(3):
            Vd = [[_dmono(e, x, d) for e in ex] for x in up]
            Dm.append(_matmul(Vd, Vinv))

        # DG lift: Mass C = B,  B[m][f] = int_F phi_m l_f dS
        Ielem = {}
        for e1 in ex:
            for e2 in ex:
                s = (e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2])
                if s not in Ielem:
                    Ielem[s] = _dec(int_elem(etype, s))
        Mass = [[Ielem[(a[0] + b[0], a[1] + b[1], a[2] + b[2])] for b in ex]
                for a in ex]
        B = [[Decimal(0)] * nf for _ in range(nu)]
        fw = [Decimal(0)] * nf
        for fi, fv in enumerate(flist):
            kind = "tri" if len(fv) == 3 else "quad"
            idx = [k for k, (_, ff, _) in enumerate(fp) if ff == fi]
            fex = face_exponents(kind, p)
            assert len(fex) == len(idx)
            area = fgeo[fi][1]
            pdom = Decimal(2) if kind == "tri" else Decimal(4)
            scale = area / pdom
            W = [[_mono(e, fp[k][2]) for e in fex] for k in idx]
            Winv = _solve(W, _eye(len(idx)))
            G = [[_dec(int_face_param(kind, (a[0] + b[0], a[1] + b[1]))) * scale
                  for b in fex] for a in fex]
            MF = _matmul(_matmul(list(map(list, zip(*Winv))), G), Winv)
            for kk, k in enumerate(idx):
                fw[k] = sum(MF[kk], Decimal(0))
            for m in range(nu):
                vals = [_mono(ex[m], fp[k][0]) for k in idx]
                for kk, k in enumerate(idx):
                    B[m][k] = sum((vals[q] * MF[q][kk] for q in range(len(idx))),
                                  Decimal(0))
        Cc = _solve(Mass, B)
        M3 = _matmul(V, Cc)
        Iw = [_dec(int_elem(etype, e)) for e in ex]
        w = [sum((Iw[m] * Vinv[m][j] for m in range(nu)), Decimal(0))
             for j in range(nu)]

        op = Operators()
        op.etype, op.p, op.nu, op.nf = etype, p, nu, nf
        f64 = lambda M: np.array([[float(v) for v in row] for row in M])
        op.upts = f64(up)
        op.fpts = f64([x for (x, _, _) in fp])
        op.fface = np.array([ff for (_, ff, _) in fp], dtype=np.int64)
        op.nfaces = len(flist)
        op.face_normal = f64([g[0] for g in fgeo])
        op.face_area = np.array([float(g[1]) for g in fgeo])
        op.fnorm = op.face_normal[op.fface]
        op.M0 = f64(M0)
        op.D = np.stack([f64(Dm[d]) for d in range(3)])
        op.M3 = f64(M3)
        op.w = np.array([float(v) for v in w])
        op.fw = np.array([float(v) for v in fw])
        op.face_kind = ["tri" if len(fv) == 3 else "quad" for fv in flist]
        op.face_verts = flist
        op.ref_verts = np.array(verts, dtype=np.float64)
        return op
