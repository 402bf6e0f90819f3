"""Pins of the oracle's learned-closure pieces (CPU only): the restriction
reproduces the low-order space and is the L2 projection (independent
quadrature), GELU against its closed form, the MLP backward pass against
central finite differences, Adam against its update formula written out for
one scalar, and the BF16 rounding on known bit patterns."""
import math

import numpy as np
import pytest

from oracle import basis, closure
from tests import _quad as Q


@pytest.mark.parametrize("etype", ["tet", "pri"])
def test_restriction_is_the_l2_projection(etype):
    R = closure.restriction(etype, 4, 2)
    hi, lo = basis.operators(etype, 4), basis.operators(etype, 2)
    ex_lo = Q.space_exponents(etype, 2)
    ex_hi = Q.space_exponents(etype, 4)
    rng = np.random.default_rng(5)
    # p=2 polynomials are reproduced exactly
    c = rng.normal(size=len(ex_lo))
    np.testing.assert_allclose(R @ Q.eval_poly(c, ex_lo, hi.upts), Q.eval_poly(c, ex_lo, lo.upts), atol=1e-12)
    # the residual of a p=4 polynomial is orthogonal to the p=2 space
    ch = rng.normal(size=len(ex_hi))
    proj = Q.fit_poly(R @ Q.eval_poly(ch, ex_hi, hi.upts), ex_lo, lo.upts)
    qp, qw = Q.ref_rule(etype)
    res = Q.eval_poly(ch, ex_hi, qp) - Q.eval_poly(proj, ex_lo, qp)
    for k in range(len(ex_lo)):
        e = np.zeros(len(ex_lo))
        e[k] = 1.0
        assert abs(qw @ (res * Q.eval_poly(e, ex_lo, qp))) < 1e-11


def test_gelu_closed_form():
    x = np.linspace(-4, 4, 17)
    exp = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in x])
    np.testing.assert_allclose(closure.gelu(x), exp, rtol=1e-15, atol=1e-16)
    h = 1e-6
    np.testing.assert_allclose(closure.gelu_grad(x), (closure.gelu(x + h) - closure.gelu(x - h)) / (2 * h),
                               atol=1e-8)


@pytest.mark.parametrize("q", [False, True])
def test_mlp_backward_matches_finite_differences(q):
    rng = np.random.default_rng(6)
    nin, nh, nout, B = 7, 6, 3, 5
    params = closure.init_params(nin, nh, nout, seed=1)
    params[1] = rng.normal(size=nh) * 0.1
    X = rng.normal(size=(B, nin))
    T = rng.normal(size=(B, nout))

    def loss(flat):
        y, _ = closure.forward(closure.unpack(flat, nin, nh, nout), X, q=False)
        return closure.mse(y, T)[0]

    y, cache = closure.forward(params, X)
    _, dy = closure.mse(y, T)
    g = closure.pack(closure.backward(params, cache, dy))
    flat = closure.pack(params)
    h = 1e-6
    fd = np.array([(loss(flat + h * np.eye(flat.size)[i]) - loss(flat - h * np.eye(flat.size)[i])) / (2 * h)
                   for i in range(flat.size)])
    np.testing.assert_allclose(g, fd, atol=1e-8, rtol=1e-6)
    if q:  # the quantised forward pass stays close to the exact one
        yq, _ = closure.forward(params, X, q=True)
        assert np.max(np.abs(yq - y)) < 2e-2 * (1 + np.max(np.abs(y)))


def test_adam_single_scalar():
    p, g = [np.array([0.5])], [np.array([0.2])]
    m, v = [np.zeros(1)], [np.zeros(1)]
    p1, m1, v1 = closure.adam(p, g, m, v, step=1, lr=1e-3)
    # step 1: m = 0.1 g, v = 0.001 g^2, bias-corrected to g and g^2
    np.testing.assert_allclose(m1[0], [0.02])
    np.testing.assert_allclose(v1[0], [0.001 * 0.04])
    np.testing.assert_allclose(p1[0], [0.5 - 1e-3 * 0.2 / (0.2 + 1e-8)])


def test_bf16_rounding():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert closure.bf16(1.0 + 2.0 ** -8) == 1.0
    assert closure.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert closure.bf16(-2.5) == -2.5
    assert closure.bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7


def _proj_ref(etype, ch, ex_hi, ex_lo, pts_lo):
    """L2 projection onto the p_lo space on the reference element, by the
    normal equations in the monomial basis under the independent collapsed
    Gauss rule, evaluated at pts_lo."""
    qp, qw = Q.ref_rule(etype)
    Ml = np.stack([Q.eval_poly(np.eye(len(ex_lo))[k], ex_lo, qp) for k in range(len(ex_lo))])
    G = (Ml * qw) @ Ml.T
    b = (Ml * qw) @ Q.eval_poly(ch, ex_hi, qp)
    return Q.eval_poly(np.linalg.solve(G, b), ex_lo, pts_lo)


def test_restrict_state_projects_each_element_and_variable():
    """restrict_state on a mixed mesh, public layout [elem][var][upt]: every
    (element, variable) carries its own random polynomial of the p=4 space
    (reference coordinates); the result must be that polynomial's L2
    projection onto the p=2 space at the p=2 points, which is the polynomial
    itself when it already lies in the p=2 space.  A swapped variable/point
    axis or a transposed restriction matrix fails it."""
    import synth
    from oracle.solver import Solver
    mesh = synth.vortex_box(n=2)
    hi, lo = Solver(mesh, 4), Solver(mesh, 2)
    rng = np.random.default_rng(11)
    uh, expect = {}, {}
    for t in hi.types:
        ex_hi, ex_lo = Q.space_exponents(t, 4), Q.space_exponents(t, 2)
        ph, pl = basis.operators(t, 4).upts, basis.operators(t, 2).upts
        ne = hi.m.ne[t]
        uh[t] = np.empty((ne, 5, len(ph)))
        expect[t] = np.empty((ne, 5, len(pl)))
        for e in range(ne):
            for v in range(5):
                if (e + v) % 2:     # inside the p=2 space: reproduced exactly
                    cl = rng.normal(size=len(ex_lo))
                    uh[t][e, v] = Q.eval_poly(cl, ex_lo, ph)
                    expect[t][e, v] = Q.eval_poly(cl, ex_lo, pl)
                else:
                    ch = rng.normal(size=len(ex_hi))
                    uh[t][e, v] = Q.eval_poly(ch, ex_hi, ph)
                    expect[t][e, v] = _proj_ref(t, ch, ex_hi, ex_lo, pl)
    got = lo.split(closure.restrict_state(hi, lo, hi.join(uh)))
    for t in lo.types:
        np.testing.assert_allclose(got[t], expect[t], atol=1e-11)


def test_features_of_a_linear_field_by_hand():
    """features() on a field linear in x, whose corrected gradient is exact
    on every element without a boundary face (no interface jumps): each
    such element's row must be [u(x_j) - u_ref for v, j (variable-major)]
    followed by [b_v[m] for m, v, j (direction-major)], assembled by hand."""
    import synth
    from oracle.solver import Solver
    c = np.linspace(-2.0, 2.0, 5)
    mesh = synth.layered_box((c, c, c), 2, 2, (False, False, False), jitter=0.05, seed=8)
    sol = Solver(mesh, 2, viscous=True, mu=0.01, p_inf=1.0 / 1.4)
    rng = np.random.default_rng(12)
    uref = np.array([1.0, 0.3, -0.2, 0.1, 2.0])
    a = uref + 0.05 * rng.normal(size=5)
    b = 0.02 * rng.normal(size=(5, 3))
    xyz = sol.upts_xyz_points()
    u = sol.state_from_points(a[None, :] + xyz @ b.T)
    feats = closure.features(sol, u, uref)
    tname = {0: "tet", 1: "pri"}
    on_bnd = {(tname[int(r[0])], int(r[1])) for r in mesh["bface"]}
    checked = 0
    for t in sol.types:
        X = sol.m.upts_x[t]                                     # (ne, nu, 3)
        nu = X.shape[1]
        for e in range(sol.m.ne[t]):
            if (t, e) in on_bnd:
                continue
            du = (a[None, :] + X[e] @ b.T - uref[None, :]).T    # (5, nu)
            gr = np.broadcast_to(b.T[:, :, None], (3, 5, nu))   # (m, v, j)
            hand = np.concatenate([du.reshape(-1), gr.reshape(-1)])
            np.testing.assert_allclose(feats[t][e], hand, atol=1e-11)
            checked += 1
    assert checked >= 40
