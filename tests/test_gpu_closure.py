"""GPU tests of the learned closure against the oracle (tests/ only):

* the network's forward pass layer by layer, its backward pass and Adam
  against oracle/closure.py, with the BF16 rounding decisions taken on the
  same FP32 values on both sides (the oracle receives the kernel's
  pre-activations, so a rounding tie cannot flip between them);
* the order transfer, the features and the training samples (target =
  P RHS_4(u_4) - RHS_2(P u_4)) against the oracle's restriction, gradient and
  right-hand sides;
* the closure inside the RHS and the RK4 step;
* training on the GPU lowers the RHS error on a held-out state.
"""
import math

import numpy as np
import pytest

import synth
from oracle import closure as OC
from oracle.solver import Solver
from tests import _cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GAMMA, MACH = 1.4, 0.1
TGV = dict(gamma=GAMMA, mu=1.0 / 1600.0, prandtl=0.72, viscous=True, rho_inf=1.0,
           vel_inf=(0.0, 0.0, 0.0), p_inf=1.0 / (GAMMA * MACH * MACH))


def _fr():
    _cases.library()
    from paper_1409_0405_gb300 import fr
    return fr


def _uref():
    p = TGV["p_inf"]
    return np.array([1.0, 0.0, 0.0, 0.0, p / (GAMMA - 1.0)])


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


# ---------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------
NIN, NH, NOUT, NS = 45, 72, 13, 333   # ragged against the 64 x 64 tiles


def _net_case(seed=4):
    rng = np.random.default_rng(seed)
    flat = synth.mlp_init(NIN, NH, NOUT, seed=seed)
    flat = flat.astype(np.float32).astype(np.float64)
    params = OC.unpack(flat, NIN, NH, NOUT)
    for k in (1, 3, 5):   # non-zero biases
        params[k][:] = (rng.normal(size=params[k].shape) * 0.1).astype(np.float32)
    flat = OC.pack(params)
    X = rng.normal(size=(NS, NIN)).astype(np.float32).astype(np.float64)
    T = rng.normal(size=(NS, NOUT)).astype(np.float32).astype(np.float64)
    return params, flat, X, T


def _gemm_bound(a, b):
    """FP32 accumulation bound of a @ b.T: K * 2^-23 * sum |a_k b_k|."""
    return a.shape[1] * 2.0 ** -23 * (np.abs(a) @ np.abs(b).T) + 1e-30


def _ws_views(ws, n, nin=NIN, nh=NH, nout=NOUT):
    """The workspace layout of include/fr.h: a status word (4 floats), then
    feature-major arrays of npad = n rounded up to 4 columns: X [nin], Z1,
    H1, Z2, H2, dZ2, dZ1 [nh], y, dL/dy [nout]; returned per sample (n x
    rows), padding columns dropped."""
    npad = (n + 3) // 4 * 4
    off = 4 + nin * npad
    out = []
    for rows in (nh,) * 6 + (nout,) * 2:
        out.append(ws[off:off + rows * npad].reshape(rows, npad)[:, :n].T)
        off += rows * npad
    return tuple(out)


def _ws_status(ws_t):
    """The status int of the workspace (non-zero: a tensor-core wait gave up)."""
    return int(ws_t[:1].view(torch.int32).item())


def test_mlp_forward_layers_match_oracle():
    fr = _fr()
    params, flat, X, _ = _net_case()
    W1, b1, W2, b2, W3, b3 = params
    q = OC.bf16
    P, Xd = _dev(flat, torch.float32), _dev(X, torch.float32)
    Y = torch.empty(NS, NOUT, dtype=torch.float32, device="cuda")
    ws = torch.zeros(fr.mlp_workspace(NIN, NH, NOUT, NS), dtype=torch.float32, device="cuda")
    fr.mlp_forward(NIN, NH, NOUT, NS, Xd.data_ptr(), P.data_ptr(), Y.data_ptr(), ws.data_ptr())
    Z1, H1, Z2, H2, *_ = _ws_views(_host(ws), NS)
    Yg = _host(Y)
    assert _ws_status(ws) == 0
    # layer 1 from the inputs
    z1 = q(X) @ q(W1).T + b1
    assert np.all(np.abs(Z1 - z1) <= _gemm_bound(q(X), q(W1)) + 1.2e-7 * (np.abs(b1) + np.abs(z1)))
    np.testing.assert_allclose(H1, OC.gelu(Z1), rtol=2e-6, atol=5e-7)
    # layers 2 and 3 from the kernel's own activations
    z2 = q(H1) @ q(W2).T + b2
    assert np.all(np.abs(Z2 - z2) <= _gemm_bound(q(H1), q(W2)) + 1.2e-7 * (np.abs(b2) + np.abs(z2)))
    np.testing.assert_allclose(H2, OC.gelu(Z2), rtol=2e-6, atol=5e-7)
    y = q(H2) @ q(W3).T + b3
    assert np.all(np.abs(Yg - y) <= _gemm_bound(q(H2), q(W3)) + 1.2e-7 * (np.abs(b3) + np.abs(y)))
    # end to end, against the oracle's own forward pass (a BF16 tie may round
    # differently from an FP64 pre-activation: one unit in 2^8 of one input)
    yo, _ = OC.forward(params, X, q=True)
    assert np.max(np.abs(Yg - yo)) < 1e-2 * np.max(np.abs(yo))
    # and the unquantised network is close (BF16 keeps 8 bits)
    yf, _ = OC.forward(params, X, q=False)
    assert np.max(np.abs(Yg - yf)) < 5e-2 * np.max(np.abs(yf))


def test_mlp_grad_matches_oracle_backward():
    fr = _fr()
    params, flat, X, T = _net_case(seed=5)
    q = OC.bf16
    P, Xd, Td = _dev(flat, torch.float32), _dev(X, torch.float32), _dev(T, torch.float32)
    G = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ws = torch.zeros(fr.mlp_workspace(NIN, NH, NOUT, NS), dtype=torch.float32, device="cuda")
    fr.mlp_grad(NIN, NH, NOUT, NS, Xd.data_ptr(), Td.data_ptr(), P.data_ptr(), G.data_ptr(), loss.data_ptr(),
                ws.data_ptr())
    Z1, H1, Z2, H2, _, _, Y, dY = _ws_views(_host(ws), NS)
    # the loss and dL/dy of the kernel's own outputs
    L, dy = OC.mse(Y, T)
    assert abs(_host(loss)[0] - L) <= 1e-5 * L
    np.testing.assert_allclose(dY, dy, rtol=1e-6, atol=1e-12)
    # the oracle's backward pass on the kernel's cached activations
    cache = (q(X), Z1, q(H1), Z2, q(H2))
    go = OC.backward(params, cache, dy, q=True)
    gg = OC.unpack(_host(G), NIN, NH, NOUT)
    # W3, b3 use dL/dy as computed (FP32 sums); the earlier layers take dL/dz
    # through the tensor cores as bf16 hi + lo, which carries at most 2^-18
    # (3.8e-6) relative error per entry: a few units in 1e-5 of the largest
    # gradient after the sums over samples
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), gg, go):
        scale = np.max(np.abs(b))
        tol = 2e-5 if name in ("W3", "b3") else 1e-4
        assert np.max(np.abs(a - b)) <= tol * scale, (name, np.max(np.abs(a - b)) / scale)
    assert _ws_status(ws) == 0


def test_mlp_grad_split_k_large_batch():
    """The weight gradients over 20,000 samples run split-K; they must equal
    the single-slice sums up to FP32 reordering."""
    fr = _fr()
    rng = np.random.default_rng(8)
    n = 20000
    params = OC.unpack(synth.mlp_init(NIN, NH, NOUT, seed=8).astype(np.float32).astype(np.float64), NIN, NH, NOUT)
    flat = OC.pack(params)
    X = rng.normal(size=(n, NIN)).astype(np.float32).astype(np.float64)
    T = rng.normal(size=(n, NOUT)).astype(np.float32).astype(np.float64)
    P, Xd, Td = _dev(flat, torch.float32), _dev(X, torch.float32), _dev(T, torch.float32)
    G = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ws = torch.zeros(fr.mlp_workspace(NIN, NH, NOUT, n), dtype=torch.float32, device="cuda")
    fr.mlp_grad(NIN, NH, NOUT, n, Xd.data_ptr(), Td.data_ptr(), P.data_ptr(), G.data_ptr(), loss.data_ptr(),
                ws.data_ptr())
    wsh = _host(ws)
    Z1, H1, Z2, H2, _, _, Y, _ = _ws_views(wsh, n)
    _, dy = OC.mse(Y, T)
    go = OC.backward(params, (OC.bf16(X), Z1, OC.bf16(H1), Z2, OC.bf16(H2)), dy, q=True)
    gg = OC.unpack(_host(G), NIN, NH, NOUT)
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), gg, go):
        tol = 5e-5 if name in ("W3", "b3") else 2e-4
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b)), name


def test_mlp_adam_matches_oracle():
    fr = _fr()
    rng = np.random.default_rng(6)
    n = 1000
    p = rng.normal(size=n).astype(np.float32).astype(np.float64)
    m = np.zeros(n)
    v = np.zeros(n)
    P, M, V = _dev(p, torch.float32), _dev(m, torch.float32), _dev(v, torch.float32)
    for step in (1, 2, 3):
        g = rng.normal(size=n).astype(np.float32).astype(np.float64)
        fr.mlp_adam(n, P.data_ptr(), _dev(g, torch.float32).data_ptr(), M.data_ptr(), V.data_ptr(), step, 1e-3)
        torch.cuda.synchronize()
        [p], [m], [v] = OC.adam([p], [g], [m], [v], step, lr=1e-3)
    np.testing.assert_allclose(_host(M), m, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(_host(V), v, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(_host(P), p, rtol=0, atol=2e-6)


def test_mlp_rejects_bad_arguments():
    fr = _fr()
    with pytest.raises(fr.FRError):
        fr.mlp_forward(0, 4, 4, 10, 1, 1, 1, 1)
    with pytest.raises(fr.FRError):
        fr.mlp_adam(10, 1, 1, 1, 1, 0, 1e-3)


# ---------------------------------------------------------------------------
# transfer, features, samples
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tgv4():
    """Oracle solvers and library contexts at p=4 and p=2 on a 4^3 TGV mesh."""
    mesh = synth.tgv_box(n=4, jitter=0.05, seed=3)
    s4, c4 = _cases.make_pair(mesh, 4, **TGV)
    s2, c2 = _cases.make_pair(mesh, 2, **TGV)
    xyz = s4.upts_xyz_points()
    # a blend of two physical periodic states stays physical
    q = 0.97 * synth.taylor_green(xyz, GAMMA, MACH) + 0.03 * synth.taylor_green(2.0 * xyz + 0.3, GAMMA, MACH)
    return s4, c4, s2, c2, s4.state_from_points(q)


def test_transfer_state_matches_oracle(tgv4):
    s4, c4, s2, c2, u4 = tgv4
    ud = _dev(u4)
    out = torch.zeros(c2.ndof, dtype=torch.float64, device="cuda")
    c2.transfer_from(c4, ud.data_ptr(), out.data_ptr())
    ref = OC.restrict_state(s4, s2, u4)
    np.testing.assert_allclose(_host(out), ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


@pytest.mark.parametrize("etype", [0, 1])
def test_features_match_oracle(tgv4, etype):
    s4, c4, s2, c2, u4 = tgv4
    u2 = OC.restrict_state(s4, s2, u4)
    ne, nu = c2.ne(etype), c2.nu(etype)
    X = torch.zeros(ne, 20 * nu, dtype=torch.float32, device="cuda")
    c2.closure_features(_dev(u2).data_ptr(), etype, X.data_ptr())
    ref = OC.features(s2, u2, _uref())["tet" if etype == 0 else "pri"]
    np.testing.assert_allclose(_host(X), ref, rtol=1e-7, atol=1e-10 * np.max(np.abs(ref)))


@pytest.mark.parametrize("etype", [0, 1])
@pytest.mark.parametrize("given_lo", [False, True])
def test_samples_match_oracle(tgv4, etype, given_lo):
    """Target P RHS_4(u_4) - RHS_2(u_2) with u_2 = P u_4 (given_lo False) or
    an independent p=2 state (True), per-variable scales, per-variable sums
    of squares and the features of u_2."""
    s4, c4, s2, c2, u4 = tgv4
    key = "tet" if etype == 0 else "pri"
    r4 = s4.rhs(u4)
    u2 = OC.restrict_state(s4, s2, u4)
    if given_lo:
        xyz = s2.upts_xyz_points()
        u2 = s2.state_from_points(0.9 * synth.taylor_green(xyz, GAMMA, MACH)
                                  + 0.1 * synth.taylor_green(xyz + 0.2, GAMMA, MACH))
    ne, nu = c2.ne(etype), c2.nu(etype)
    target = s2.split(OC.restrict_state(s4, s2, r4) - s2.rhs(u2))[key]        # (ne, 5, nu)
    X = torch.zeros(ne, 20 * nu, dtype=torch.float32, device="cuda")
    T = torch.zeros(ne, 5 * nu, dtype=torch.float32, device="cuda")
    ss = torch.zeros(5, dtype=torch.float64, device="cuda")
    scale = np.array([0.37, 1.5, 2.0, 0.25, 40.0])
    u2d = _dev(u2)
    c2.closure_sample(c4, _dev(u4).data_ptr(), etype, 1.0 / scale, X.data_ptr(), T.data_ptr(), ss.data_ptr(),
                      u_lo_ptr=u2d.data_ptr() if given_lo else None)
    got = _host(T).reshape(ne, 5, nu) * scale[None, :, None]
    # the target is a difference of two RHS of size |r4|: FP64 parity of
    # each (1e-12 of its scale) plus the FP32 rounding of the stored value
    tol = 1e-11 * np.max(np.abs(r4)) + 1e-7 * np.abs(target)
    assert np.all(np.abs(got - target) <= tol)
    np.testing.assert_allclose(_host(ss), np.sum(target ** 2, axis=(0, 2)), rtol=1e-6)
    ref = OC.features(s2, u2, _uref())[key]
    np.testing.assert_allclose(_host(X), ref, rtol=1e-7, atol=1e-10 * np.max(np.abs(ref)))


# ---------------------------------------------------------------------------
# the closure inside the RHS and the RK step
# ---------------------------------------------------------------------------
def _attach_random(c2, scale, nh=32, seed=11):
    nets = {}
    for et in (0, 1):
        nu = c2.nu(et)
        flat = synth.mlp_init(20 * nu, nh, 5 * nu, seed=seed + et)
        flat = flat + 0.05 * np.random.default_rng(seed + et).normal(size=flat.size)
        P = _dev(flat, torch.float32)
        c2.closure_set(et, P.data_ptr(), nh, scale)
        nets[et] = (flat.astype(np.float32).astype(np.float64), P)
    return nets


def test_closure_in_rhs(tgv4):
    fr = _fr()
    s4, c4, s2, c2, u4 = tgv4
    u2 = OC.restrict_state(s4, s2, u4)
    ud = _dev(u2)
    r_off = torch.zeros_like(ud)
    r_on = torch.zeros_like(ud)
    c2.rhs(ud.data_ptr(), r_off.data_ptr())
    scale, nh = np.array([0.5, 0.25, 0.25, 0.75, 2.0]), 32
    nets = _attach_random(c2, scale, nh)
    try:
        c2.rhs(ud.data_ptr(), r_on.data_ptr())
    finally:
        for et in (0, 1):
            c2.closure_set(et, None)
    diff = s2.split(_host(r_on) - _host(r_off))
    rmax = float(np.max(np.abs(_host(r_off))))
    oracle_rhs = s2.split(s2.rhs(u2))
    feats = OC.features(s2, u2, _uref())
    for et, key in ((0, "tet"), (1, "pri")):
        ne, nu = c2.ne(et), c2.nu(et)
        flat, P = nets[et]
        # the same network on the library's features, through fr_mlp_forward
        X = torch.zeros(ne, 20 * nu, dtype=torch.float32, device="cuda")
        c2.closure_features(ud.data_ptr(), et, X.data_ptr())
        Y = torch.zeros(ne, 5 * nu, dtype=torch.float32, device="cuda")
        ws = torch.zeros(fr.mlp_workspace(20 * nu, nh, 5 * nu, ne), dtype=torch.float32, device="cuda")
        fr.mlp_forward(20 * nu, nh, 5 * nu, ne, X.data_ptr(), P.data_ptr(), Y.data_ptr(), ws.data_ptr())
        sc = np.repeat(scale, nu)[None, :]
        corr = sc * _host(Y)
        got = diff[key].reshape(ne, -1)
        assert np.max(np.abs(got - corr)) <= 1e-13 * rmax + 1e-7 * np.max(np.abs(corr))
        # and the oracle: its RHS plus its network on its features
        yo, _ = OC.forward(OC.unpack(flat, 20 * nu, nh, 5 * nu), feats[key], q=True)
        full = _host(r_on)
        r_on_t = s2.split(full)[key].reshape(ne, -1)
        ref = oracle_rhs[key].reshape(ne, -1) + sc * yo
        assert np.max(np.abs(r_on_t - ref)) <= 1e-12 * rmax + 1e-2 * np.max(np.abs(sc * yo))


def test_closure_in_rk_step(tgv4):
    s4, c4, s2, c2, u4 = tgv4
    u2 = OC.restrict_state(s4, s2, u4)
    dt = 1e-3
    _attach_random(c2, 0.5)
    try:
        # manual RK4 through fr_rhs with the closure on
        u = _dev(u2)

        def R(x):
            r = torch.zeros_like(x)
            c2.rhs(x.data_ptr(), r.data_ptr())
            return r

        k1 = R(u)
        k2 = R(u + 0.5 * dt * k1)
        k3 = R(u + 0.5 * dt * k2)
        k4 = R(u + dt * k3)
        ref = _host(u + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4))
        c2.set_state(u2)
        c2.step(dt, 1)
        got = c2.get_state()
    finally:
        for et in (0, 1):
            c2.closure_set(et, None)
    inc = np.max(np.abs(ref - u2))
    assert np.max(np.abs(got - ref)) <= 1e-10 * inc + 1e-14 * np.max(np.abs(u2))


def test_closure_set_errors(tgv4):
    fr = _fr()
    s4, c4, s2, c2, u4 = tgv4
    with pytest.raises(fr.FRError):
        c2.closure_set(2, None)
    mesh = synth.tgv_box(n=2)
    euler = fr.Context(mesh, 2, **dict(TGV, viscous=False, mu=0.0))
    P = torch.zeros(fr.mlp_nparams(200, 8, 50), dtype=torch.float32, device="cuda")
    with pytest.raises(fr.FRError) as e:
        euler.closure_set(0, P.data_ptr(), 8, 1.0)
    assert e.value.code == fr.FR_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# what training gains
# ---------------------------------------------------------------------------
def test_trained_closure_reduces_rhs_error():
    """TGV (Re 1600, Ma 0.1) on an 8^3 periodic mesh: states along a p=4
    run; networks trained on the earlier ones; on the last (held out), the
    closed p=2 RHS is closer to the projected p=4 RHS than the plain one."""
    _fr()
    from paper_1409_0405_gb300 import closure
    from paper_1409_0405_gb300 import fr
    mesh = synth.tgv_box(n=8)
    c4 = fr.Context(mesh, 4, **TGV)
    c2 = fr.Context(mesh, 2, **TGV)
    s4 = Solver(mesh, 4, gamma=GAMMA, mu=TGV["mu"], viscous=True, vel_inf=(0, 0, 0), p_inf=TGV["p_inf"])
    u0 = s4.state_from_points(synth.taylor_green(s4.upts_xyz_points(), GAMMA, MACH))
    dt = s4.dt_cfl(u0, 0.1)
    c4.set_state(u0)
    states = []
    for k in range(9):
        states.append(_dev(c4.get_state()))
        c4.step(dt, 100)
    train, held = states[:-1], states[-1:]
    cl = closure.Closure(c2, seed=1)
    log = cl.fit(c4, train, iters=1500, lr=1e-3, log_every=500)
    err = cl.error(c4, held)
    print("losses", log, "held-out relative error", err)
    for et in (0, 1):
        assert log[et][-1] < 0.2 * log[et][0]
        assert err[et][0] < 0.5, (et, err[et])


# ---------------------------------------------------------------------------
# p-sequenced restart: prolongation through the same transfer
# ---------------------------------------------------------------------------
def test_prolongation_restart_matches_oracle(tgv4):
    """A p=2 state prolonged to p=4 (fr_transfer_state, lower to higher
    order) equals the oracle's L2 projection (exact for the p=2 polynomial),
    projects back unchanged, and the p=4 solver runs from it (an RHS that
    matches the oracle's on the prolonged state)."""
    s4, c4, s2, c2, u4 = tgv4
    u2 = OC.restrict_state(s4, s2, u4)
    a2 = s2.split(u2)
    ref = s4.join({t: a2[t] @ OC.restriction(t, 2, 4).T for t in s4.types})
    up = torch.zeros(c4.ndof, dtype=torch.float64, device="cuda")
    c4.transfer_from(c2, _dev(u2).data_ptr(), up.data_ptr())
    got = _host(up)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))
    back = torch.zeros(c2.ndof, dtype=torch.float64, device="cuda")
    c2.transfer_from(c4, up.data_ptr(), back.data_ptr())
    np.testing.assert_allclose(_host(back), u2, rtol=0, atol=1e-13 * np.max(np.abs(u2)))
    r = torch.zeros_like(up)
    c4.rhs(up.data_ptr(), r.data_ptr())
    err = _cases.per_quantity_rel_err(s4, s4.rhs(got), _host(r))
    assert np.all(err < 1e-12), err
