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
