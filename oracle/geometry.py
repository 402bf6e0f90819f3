"""Element maps and metric terms.

Readings: tets are affine, x = sum_a lambda_a(xi) X_a with the barycentric
lambda of the reference tet.  Prisms use the linear-triangle x linear-zeta
map x = sum_a tau_a(xi, eta) [(1-zeta)/2 X_a + (1+zeta)/2 X_{a+3}],
which is not affine once nodes are jittered.  Hexes use the trilinear map
x = sum_a N_a(xi) X_a, N_a = (1 + s_a0 xi)(1 + s_a1 eta)(1 + s_a2 zeta)/8
with s_a the signs of reference vertex a.  Quadratically curved elements
(10-node tets, 18-node prisms, 27-node hexes; node positions in
QUAD_NODES) use the Lagrange basis of the degree-2 space of the element
(P2; P2(triangle) x P2(zeta); Q2) through those nodes, x = sum_a N_a X_a,
with N found by solving the monomial Vandermonde system.  Writing A = dx/dxi (columns
a_d = dx/dxi_d), the transformed-flux matrix is S = J dxi/dx = adj(A),
whose rows are a_1 x a_2, a_2 x a_0, a_0 x a_1.  A flux F in physical space
becomes F~_d = sum_m S[d][m] F_m in reference space; at a face with
reference outward normal n^ the physical normal scaled by dS/dS^ is S^T n^.
"""
from __future__ import annotations

import numpy as np


_TRI6 = ((-1, -1), (1, -1), (-1, 1), (0, -1), (0, 0), (-1, 0))
QUAD_NODES = {
    "tet": ((-1, -1, -1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1),
            (0, -1, -1), (-1, 0, -1), (-1, -1, 0), (0, 0, -1), (0, -1, 0), (-1, 0, 0)),
    "pri": tuple((a, b, c) for c in (-1, 0, 1) for (a, b) in _TRI6),
    "hex": tuple((a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)),
}


def _quad_exponents(etype):
    if etype == "tet":
        return [(a, b, c) for c in range(3) for b in range(3) for a in range(3) if a + b + c <= 2]
    if etype == "pri":
        return [(a, b, c) for c in range(3) for b in range(3) for a in range(3) if a + b <= 2]
    return [(a, b, c) for c in range(3) for b in range(3) for a in range(3)]


def _quad_shape(etype, ref):
    ex = _quad_exponents(etype)
    nodes = np.array(QUAD_NODES[etype], dtype=np.float64)
    V = np.array([[x ** a * y ** b * z ** c for (a, b, c) in ex] for (x, y, z) in nodes])
    C = np.linalg.inv(V)                       # N_a(x) = sum_m mono_m(x) C[m, a]
    mono = np.stack([ref[:, 0] ** a * ref[:, 1] ** b * ref[:, 2] ** c for (a, b, c) in ex], axis=1)
    dmono = np.zeros(mono.shape + (3,))
    for m, (a, b, c) in enumerate(ex):
        e = (a, b, c)
        for d in range(3):
            if e[d] == 0:
                continue
            f = float(e[d])
            pw = list(e)
            pw[d] -= 1
            dmono[:, m, d] = f * ref[:, 0] ** pw[0] * ref[:, 1] ** pw[1] * ref[:, 2] ** pw[2]
    return mono @ C, np.einsum("pmd,ma->pad", dmono, C)


def shape(etype, ref, nv=None):
    """Shape functions N (npts, nv) and derivatives dN (npts, nv, 3) at
    reference points ref (npts, 3); nv = the quadratic node count selects the
    curved element's basis."""
    if nv is not None and nv == len(QUAD_NODES[etype]):
        return _quad_shape(etype, np.asarray(ref, dtype=np.float64))
    xi, eta, zeta = ref[:, 0], ref[:, 1], ref[:, 2]
    npt = len(ref)
    if etype == "tet":
        N = np.stack([-(1 + xi + eta + zeta) / 2, (1 + xi) / 2, (1 + eta) / 2,
                      (1 + zeta) / 2], axis=1)
        dN = np.zeros((npt, 4, 3))
        dN[:, 0, :] = -0.5
        dN[:, 1, 0] = 0.5
        dN[:, 2, 1] = 0.5
        dN[:, 3, 2] = 0.5
        return N, dN
    if etype == "hex":
        sg = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                       [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)
        f = [1.0 + sg[None, :, k] * ref[:, k:k + 1] for k in range(3)]    # (npt, 8)
        N = f[0] * f[1] * f[2] / 8.0
        dN = np.stack([sg[None, :, 0] * f[1] * f[2], f[0] * sg[None, :, 1] * f[2],
                       f[0] * f[1] * sg[None, :, 2]], axis=-1) / 8.0
        return N, dN
    tau = np.stack([-(xi + eta) / 2, (1 + xi) / 2, (1 + eta) / 2], axis=1)
    dtau = np.array([[-0.5, -0.5], [0.5, 0.0], [0.0, 0.5]])   # d tau_a / d(xi, eta)
    lo, hi = (1 - zeta) / 2, (1 + zeta) / 2
    N = np.concatenate([tau * lo[:, None], tau * hi[:, None]], axis=1)
    dN = np.zeros((npt, 6, 3))
    for a in range(3):
        for d in range(2):
            dN[:, a, d] = dtau[a, d] * lo
            dN[:, a + 3, d] = dtau[a, d] * hi
        dN[:, a, 2] = -tau[:, a] / 2
        dN[:, a + 3, 2] = tau[:, a] / 2
    return N, dN


def map_points(etype, X, ref):
    """Physical coordinates (ne, npts, 3) of reference points for element
    vertex coordinates X (ne, nv, 3)."""
    N, _ = shape(etype, ref, X.shape[1])
    return np.einsum("pv,evk->epk", N, X)


def jacobian(etype, X, ref):
    """A[e, p, k, d] = d x_k / d xi_d."""
    _, dN = shape(etype, ref, X.shape[1])
    return np.einsum("pvd,evk->epkd", dN, X)


def metric(etype, X, ref):
    """J (ne, npts) and S (ne, npts, 3, 3) with S[..., d, m] = J dxi_d/dx_m."""
    A = jacobian(etype, X, ref)
    a0, a1, a2 = A[..., 0], A[..., 1], A[..., 2]
    S = np.stack([np.cross(a1, a2), np.cross(a2, a0), np.cross(a0, a1)], axis=-2)
    J = np.einsum("...k,...k->...", a0, np.cross(a1, a2))
    return J, S


def face_normals(etype, X, ref, nhat):
    """Physical unit outward normals n (ne, npts, 3) and magnitudes
    |S^T n^| (ne, npts) at reference face points ref with reference outward
    unit normals nhat (npts, 3)."""
    _, S = metric(etype, X, ref)
    sn = np.einsum("epdm,pd->epm", S, nhat)
    mag = np.linalg.norm(sn, axis=-1)
    return sn / mag[..., None], mag
