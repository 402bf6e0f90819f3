"""Independent quadrature and polynomial helpers for the tests.

Collapsed (Duffy) Gauss-Legendre rules built from numpy's leggauss; they
share nothing with the oracle's exact rational integrals or with the CUDA
path's quadrature.
"""
import numpy as np
from numpy.polynomial.legendre import leggauss

TET_V = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)
PRI_V = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1],
                  [-1, -1, 1], [1, -1, 1], [-1, 1, 1]], float)
TET_F = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
PRI_F = ((0, 1, 2), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5))
HEX_V = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                  [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float)
HEX_F = ((0, 1, 2, 3), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7), (4, 5, 6, 7))


def ref_verts_faces(etype):
    return {"tet": (TET_V, TET_F), "pri": (PRI_V, PRI_F), "hex": (HEX_V, HEX_F)}[etype]


def gl01(n):
    x, w = leggauss(n)
    return (x + 1) / 2, w / 2


def unit_triangle_rule(n=12):
    """Points (m,2) and weights on the unit triangle {x,y>=0, x+y<=1}."""
    u, wu = gl01(n)
    pts, wts = [], []
    for a in range(n):
        for b in range(n):
            x = u[a]
            y = u[b] * (1 - x)
            pts.append((x, y))
            wts.append(wu[a] * wu[b] * (1 - x))
    return np.array(pts), np.array(wts)


def unit_tet_rule(n=12):
    u, wu = gl01(n)
    pts, wts = [], []
    for a in range(n):
        for b in range(n):
            for c in range(n):
                x = u[a]
                y = u[b] * (1 - x)
                z = u[c] * (1 - x) * (1 - u[b])
                pts.append((x, y, z))
                wts.append(wu[a] * wu[b] * wu[c] * (1 - x) ** 2 * (1 - u[b]))
    return np.array(pts), np.array(wts)


def ref_rule(etype, n=12):
    """Quadrature over the reference element (points in reference coords)."""
    if etype == "tet":
        p, w = unit_tet_rule(n)
        return -1 + 2 * p, 8 * w
    if etype == "hex":
        x, wx = leggauss(n)
        pts = np.array([(a, b, c) for c in x for b in x for a in x])
        wts = np.array([wa * wb * wc for wc in wx for wb in wx for wa in wx])
        return pts, wts
    tp, tw = unit_triangle_rule(n)
    z, wz = leggauss(n)
    pts = np.array([(-1 + 2 * x, -1 + 2 * y, zz) for zz in z for (x, y) in tp])
    wts = np.array([4 * a * b for b in wz for a in tw])
    return pts, wts


def face_rule(verts, n=12):
    """Quadrature over a planar reference face with the given 3 or 4
    vertices (reference coords); weights include the face's area element."""
    V = np.asarray(verts, float)
    if len(V) == 3:
        tp, tw = unit_triangle_rule(n)
        pts = V[0] + np.outer(tp[:, 0], V[1] - V[0]) + np.outer(tp[:, 1], V[2] - V[0])
        area2 = np.linalg.norm(np.cross(V[1] - V[0], V[2] - V[0]))
        return pts, tw * area2
    u, wu = gl01(n)
    pts, wts = [], []
    for a in range(n):
        for b in range(n):
            s, t = u[a], u[b]
            x = V[0] * (1 - s) * (1 - t) + V[1] * s * (1 - t) + V[2] * s * t + V[3] * (1 - s) * t
            pts.append(x)
            wts.append(wu[a] * wu[b])
    area = np.linalg.norm(np.cross(V[1] - V[0], V[3] - V[0]))
    return np.array(pts), np.array(wts) * area


def space_exponents(etype, p):
    if etype == "tet":
        return [(a, b, c) for a in range(p + 1) for b in range(p + 1)
                for c in range(p + 1) if a + b + c <= p]
    if etype == "hex":
        return [(a, b, c) for a in range(p + 1) for b in range(p + 1) for c in range(p + 1)]
    return [(a, b, c) for a in range(p + 1) for b in range(p + 1)
            for c in range(p + 1) if a + b <= p]


def eval_poly(coef, ex, x):
    x = np.asarray(x, float)
    out = np.zeros(len(x))
    for c, (a, b, d) in zip(coef, ex):
        out += c * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** d
    return out


def eval_grad(coef, ex, x):
    x = np.asarray(x, float)
    g = np.zeros((len(x), 3))
    for c, (a, b, d) in zip(coef, ex):
        if a:
            g[:, 0] += c * a * x[:, 0] ** (a - 1) * x[:, 1] ** b * x[:, 2] ** d
        if b:
            g[:, 1] += c * b * x[:, 0] ** a * x[:, 1] ** (b - 1) * x[:, 2] ** d
        if d:
            g[:, 2] += c * d * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** (d - 1)
    return g


def fit_poly(values, ex, x):
    """Monomial coefficients of the element-space polynomial through values
    at points x (float64 least squares)."""
    V = np.array([[xi ** a * yi ** b * zi ** d for (a, b, d) in ex] for (xi, yi, zi) in x])
    return np.linalg.solve(V, values)
