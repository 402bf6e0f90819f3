"""Learned-closure pieces of the oracle (TEST INFRASTRUCTURE ONLY): the
restriction between orders, the per-element features of a p=2 state, and
a plain FP64 multilayer perceptron with its backward pass and Adam.

Readings (the closure is not in the paper; the workload asks for a p=2
solve plus a per-element MLP trained on restricted p=4 right-hand sides):
  * restriction p_hi -> p_lo: the L2 projection in the reference element
    (on the affine elements of the Taylor-Green mesh this equals the
    physical, J-weighted projection), as a matrix on solution-point values;
  * features of an element: its p=2 solution-point values u - u_inf
    (5 x nu, variable-major) followed by the corrected physical gradient
    (3 x 5 x nu, direction-major), i.e. the element's degrees of freedom in
    the nodal basis (any basis of the same space carries the same
    information);
  * target: R(RHS_4(u_4)) - RHS_2(R u_4) at the p=2 solution points
    (5 x nu, variable-major), scaled by one constant out_scale;
  * network: in -> 128 -> 128 -> out, GELU (erf form) after the two hidden
    layers, MSE loss, Adam (beta 0.9 / 0.999, eps 1e-8);
  * BF16 points (optional, to mirror the CUDA kernels): the GEMM inputs
    (features, weights, hidden activations) rounded to bfloat16
    (round-to-nearest-even from float32); biases, accumulations and the
    backward pass in full precision.
"""
from __future__ import annotations

import math
from decimal import Decimal, localcontext

import numpy as np
from scipy.special import erf

from . import basis


# ---------------------------------------------------------------------------
# restriction between orders (exact, decimal)
# ---------------------------------------------------------------------------
def restriction(etype, p_hi, p_lo):
    """Matrix R (nu_lo x nu_hi): nodal values of the p_hi interpolant ->
    nodal values of its L2 projection onto the p_lo space.  With monomial
    bases phi (p_lo) and psi (p_hi):  R = V_lo G_ll^-1 G_lh V_hi^-1, where
    G_ll = int phi phi^T, G_lh = int phi psi^T exactly and V the monomial
    Vandermondes at the solution points."""
    with localcontext() as c:
        c.prec = basis.PREC
        el = basis.exponents(etype, p_lo)
        eh = basis.exponents(etype, p_hi)
        ul = basis.upts_exact(etype, p_lo)
        uh = basis.upts_exact(etype, p_hi)
        Vl = [[basis._mono(e, x) for e in el] for x in ul]
        Vh = [[basis._mono(e, x) for e in eh] for x in uh]
        Vh_inv = basis._solve(Vh, basis._eye(len(eh)))

        def gram(ea, eb):
            return [[basis._dec(basis.int_elem(etype, (a[0] + b[0], a[1] + b[1], a[2] + b[2])))
                     for b in eb] for a in ea]

        Gll = gram(el, el)
        Glh = gram(el, eh)
        X = basis._solve(Gll, basis._matmul(Glh, Vh_inv))
        R = basis._matmul(Vl, X)
        return np.array([[float(v) for v in row] for row in R])


# ---------------------------------------------------------------------------
# features and the restricted state
# ---------------------------------------------------------------------------
def restrict_state(sol_hi, sol_lo, u_hi):
    """Apply the restriction element by element (public layouts)."""
    a = sol_hi.split(np.asarray(u_hi, dtype=np.float64))
    out = {}
    for t in sol_lo.types:
        R = restriction(t, sol_hi.p, sol_lo.p)
        out[t] = a[t] @ R.T
    return sol_lo.join(out)


def features(sol_lo, u_lo, u_ref):
    """Per type: (ne, 20 nu) features [u - u_ref (5 x nu), grad (3 x 5 x nu)]."""
    u = sol_lo.split(np.asarray(u_lo, dtype=np.float64))
    g = sol_lo.gradient(u_lo)                     # (ne, V, nu, m)
    out = {}
    for t in sol_lo.types:
        du = u[t] - np.asarray(u_ref)[None, :, None]
        gm = g[t].transpose(0, 3, 1, 2)            # (ne, m, V, nu)
        out[t] = np.concatenate([du.reshape(len(du), -1), gm.reshape(len(gm), -1)], axis=1)
    return out


# ---------------------------------------------------------------------------
# the MLP
# ---------------------------------------------------------------------------
def bf16(x):
    """Round to bfloat16 (nearest even) through float32, returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def init_params(nin, nh, nout, seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = [(nh, nin), (nh,), (nh, nh), (nh,), (nout, nh), (nout,)]
    out = []
    for s in shapes:
        if len(s) == 2:
            lim = 1.0 / math.sqrt(s[1])
            out.append(rng.uniform(-lim, lim, size=s))
        else:
            out.append(np.zeros(s))
    return out


def pack(params):
    return np.concatenate([p.reshape(-1) for p in params])


def unpack(flat, nin, nh, nout):
    shapes = [(nh, nin), (nh,), (nh, nh), (nh,), (nout, nh), (nout,)]
    out, off = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(np.asarray(flat[off:off + n], dtype=np.float64).reshape(s))
        off += n
    return out


def forward(params, X, q=False):
    """Returns y and the cache of the backward pass; q: BF16 GEMM inputs."""
    W1, b1, W2, b2, W3, b3 = params
    r = bf16 if q else (lambda a: np.asarray(a, dtype=np.float64))
    x0 = r(X)
    z1 = x0 @ r(W1).T + b1
    h1 = r(gelu(z1))
    z2 = h1 @ r(W2).T + b2
    h2 = r(gelu(z2))
    y = h2 @ r(W3).T + b3
    return y, (x0, z1, h1, z2, h2)


def backward(params, cache, dy, q=False):
    """Gradients of the loss w.r.t. (W1, b1, W2, b2, W3, b3) given dL/dy."""
    W1, b1, W2, b2, W3, b3 = params
    r = bf16 if q else (lambda a: np.asarray(a, dtype=np.float64))
    x0, z1, h1, z2, h2 = cache
    dW3 = dy.T @ h2
    db3 = dy.sum(0)
    dz2 = (dy @ r(W3)) * gelu_grad(z2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(0)
    dz1 = (dz2 @ r(W2)) * gelu_grad(z1)
    dW1 = dz1.T @ x0
    db1 = dz1.sum(0)
    return [dW1, db1, dW2, db2, dW3, db3]


def mse(y, t):
    """Mean squared error and its gradient dL/dy."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(params, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new params, m, v."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = b1 * mm + (1 - b1) * g
        vv = b2 * vv + (1 - b2) * g * g
        mh = mm / (1 - b1 ** step)
        vh = vv / (1 - b2 ** step)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v
