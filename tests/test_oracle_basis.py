"""Pins of the oracle's points and operators (CPU only).

Every check compares against something the oracle does not compute itself:
the paper's Table 2, polynomial exactness evaluated by direct monomial
evaluation, and integrals from an independent collapsed Gauss rule.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import basis
from tests import _quad as Q

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = [(t, p) for t in ("tet", "pri", "hex") for p in (1, 2, 3, 4)]


def _table2():
    rows = {}
    with open(os.path.join(HERE, "golden", "table2_m0_dims.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t, p, nu, nf = line.split()
            rows[(t, int(p))] = (int(nu), int(nf))
    return rows


@pytest.mark.parametrize("etype,p", CASES)
def test_table2_dimensions(etype, p):
    """Table 2 prints dim M0 as Nupts x Nfpts for tet, prism and hex at p=1..4."""
    nu, nf = _table2()[(etype, p)]
    op = basis.operators(etype, p)
    assert op.M0.shape == (nf, nu)
    assert op.upts.shape == (nu, 3) and op.fpts.shape == (nf, 3)


def _inside(etype, x, tol=1e-12):
    if etype == "tet":
        return (np.all(x >= -1 - tol, axis=1) & (x.sum(1) <= -1 + tol))
    if etype == "hex":
        return np.all(np.abs(x) <= 1 + tol, axis=1)
    return ((x[:, 0] >= -1 - tol) & (x[:, 1] >= -1 - tol) &
            (x[:, 0] + x[:, 1] <= tol) & (np.abs(x[:, 2]) <= 1 + tol))


@pytest.mark.parametrize("etype,p", CASES)
def test_points_interior_and_distinct(etype, p):
    op = basis.operators(etype, p)
    assert np.all(_inside(etype, op.upts, tol=-1e-9))          # strictly inside
    assert np.all(_inside(etype, op.fpts))
    d = np.linalg.norm(op.upts[:, None] - op.upts[None], axis=-1)
    assert np.min(d + np.eye(len(d)) * 9) > 1e-3


@pytest.mark.parametrize("etype,p", CASES)
def test_face_point_sets_symmetric(etype, p):
    """Each face's flux-point set is invariant under the face's vertex
    symmetries, so two neighbours' points coincide whatever their local
    orientation."""
    op = basis.operators(etype, p)
    V, F = Q.ref_verts_faces(etype)
    for fi, fv in enumerate(F):
        pts = op.fpts[op.fface == fi]
        verts = V[list(fv)]
        if len(fv) == 3:
            # barycentric coords w.r.t. the face vertices, then permute
            A = np.stack([verts[1] - verts[0], verts[2] - verts[0]], axis=1)
            lam12 = np.linalg.lstsq(A, (pts - verts[0]).T, rcond=None)[0].T
            bary = np.c_[1 - lam12.sum(1), lam12]
            for perm in itertools.permutations(range(3)):
                img = bary[:, perm] @ verts
                d = np.linalg.norm(img[:, None] - pts[None], axis=-1).min(1)
                assert d.max() < 1e-12
        else:
            # the 8 symmetries of the square in bilinear parameters
            e1, e2 = verts[1] - verts[0], verts[3] - verts[0]
            st = np.linalg.lstsq(np.stack([e1, e2], 1), (pts - verts[0]).T, rcond=None)[0].T
            st = 2 * st - 1
            for sw in (False, True):
                for s1 in (1, -1):
                    for s2 in (1, -1):
                        q = st[:, ::-1] if sw else st
                        q = q * np.array([s1, s2])
                        img = verts[0] + np.outer((q[:, 0] + 1) / 2, e1) + np.outer((q[:, 1] + 1) / 2, e2)
                        d = np.linalg.norm(img[:, None] - pts[None], axis=-1).min(1)
                        assert d.max() < 1e-12


@pytest.mark.parametrize("etype,p", CASES)
def test_interpolation_and_derivatives_exact(etype, p):
    """M0 and D_d are exact on every polynomial of the element space."""
    op = basis.operators(etype, p)
    ex = Q.space_exponents(etype, p)
    rng = np.random.default_rng(1)
    for _ in range(3):
        c = rng.normal(size=len(ex))
        u = Q.eval_poly(c, ex, op.upts)
        np.testing.assert_allclose(op.M0 @ u, Q.eval_poly(c, ex, op.fpts), atol=1e-12, rtol=0)
        g = Q.eval_grad(c, ex, op.upts)
        for d in range(3):
            np.testing.assert_allclose(op.D[d] @ u, g[:, d], atol=1e-11, rtol=0)


@pytest.mark.parametrize("etype,p", CASES)
def test_weights_integrate_space_exactly(etype, p):
    op = basis.operators(etype, p)
    ex = Q.space_exponents(etype, p)
    qp, qw = Q.ref_rule(etype)
    rng = np.random.default_rng(2)
    c = rng.normal(size=len(ex))
    exact = qw @ Q.eval_poly(c, ex, qp)
    assert abs(op.w @ Q.eval_poly(c, ex, op.upts) - exact) < 1e-12
    assert abs(op.w.sum() - {"tet": 4.0 / 3.0, "pri": 4.0, "hex": 8.0}[etype]) < 1e-13


@pytest.mark.parametrize("etype,p", CASES)
def test_face_weights(etype, p):
    """fw integrates the face trace space exactly (checked on the trace of
    random element polynomials)."""
    op = basis.operators(etype, p)
    ex = Q.space_exponents(etype, p)
    V, F = Q.ref_verts_faces(etype)
    rng = np.random.default_rng(3)
    c = rng.normal(size=len(ex))
    for fi, fv in enumerate(F):
        sel = op.fface == fi
        qp, qw = Q.face_rule(V[list(fv)])
        exact = qw @ Q.eval_poly(c, ex, qp)
        assert abs(op.fw[sel] @ Q.eval_poly(c, ex, op.fpts[sel]) - exact) < 1e-12


@pytest.mark.parametrize("etype,p", CASES)
def test_lift_galerkin_identity(etype, p):
    """The DG correction: for face data Delta equal to the trace of a face
    polynomial q_F, g = M3 Delta satisfies  int v g = sum_F int_F q_F v
    for every v of the element space (brute force on one element)."""
    op = basis.operators(etype, p)
    ex = Q.space_exponents(etype, p)
    V, F = Q.ref_verts_faces(etype)
    rng = np.random.default_rng(4)
    qcoef = [rng.normal(size=len(ex)) for _ in F]
    delta = np.zeros(op.nf)
    for fi in range(len(F)):
        sel = op.fface == fi
        delta[sel] = Q.eval_poly(qcoef[fi], ex, op.fpts[sel])
    g_upts = op.M3 @ delta
    gc = Q.fit_poly(g_upts, ex, op.upts)
    vp, vw = Q.ref_rule(etype)
    for _ in range(4):
        vc = rng.normal(size=len(ex))
        lhs = vw @ (Q.eval_poly(vc, ex, vp) * Q.eval_poly(gc, ex, vp))
        rhs = 0.0
        for fi, fv in enumerate(F):
            fp, fw = Q.face_rule(V[list(fv)])
            rhs += fw @ (Q.eval_poly(qcoef[fi], ex, fp) * Q.eval_poly(vc, ex, fp))
        assert abs(lhs - rhs) < 1e-10 * (1 + abs(rhs))


def test_gauss_legendre_nodes():
    """Nodes agree with numpy's Golub-Welsch based leggauss."""
    from numpy.polynomial.legendre import leggauss
    for n in range(1, 7):
        np.testing.assert_allclose([float(x) for x in basis.gauss_legendre(n)],
                                   leggauss(n)[0], atol=1e-14)
