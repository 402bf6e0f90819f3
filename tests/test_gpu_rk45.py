"""RK45[2R+] on the GPU (fr_step_rk45, fr_rk45_error, fr_rk45_get_error,
fr_step_rk45_adaptive) against the oracle's RK4(3)5[2R+]C (GPU).

States must match the oracle to 1e-12 per conserved quantity, as for RK4.
The error register is a difference of two solutions, E = dt sum_i
(b_i - bhat_i) k_i, whose terms cancel to O(dt^4): its absolute deviation
is bounded by the RHS parity instead, |dE| <= 1e-12 dt sum_i |b_i - bhat_i|
max|k|, and the error norm, whose weights are >= atol, moves by at most
that bound over atol.
"""
import numpy as np
import pytest

import synth
from oracle import solver as osv
from tests._cases import bl_params, library, make_pair, per_quantity_rel_err, state

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    library()


def _e_bound(sol, u, dt):
    return TOL * dt * sum(abs(x) for x in osv.RK45_2R_E) * float(np.max(np.abs(sol.rhs(u))))


def _fixed_steps(sol, ctx, u, dt, n, atol=1e-6, rtol=1e-6):
    ctx.set_state(u)
    ctx.step_rk45(dt, n)
    got, e_got = ctx.get_state(), ctx.rk45_get_error()
    nrm_got = ctx.rk45_error(atol, rtol)
    ref = u
    for _ in range(n):
        ref, e_ref = sol.rk45_step(ref, dt)
    err = per_quantity_rel_err(sol, ref, got)
    assert np.all(err <= TOL), err
    bound = _e_bound(sol, ref, dt)
    assert np.max(np.abs(e_got - e_ref)) <= bound, (np.max(np.abs(e_got - e_ref)), bound)
    nrm_ref = osv.rk45_error_norm(ref, e_ref, atol, rtol)
    assert abs(nrm_got - nrm_ref) <= bound / atol, (nrm_got, nrm_ref)
    return u, ref


def test_vortex_rk45_fixed_steps():
    """The vortex workload (Euler, p = 2): 20 RK45[2R+] steps at CFL 0.1;
    the periodic totals do not drift."""
    sol, ctx = make_pair(synth.vortex_box(), 2)
    u = state(sol, "vortex")
    _fixed_steps(sol, ctx, u, sol.dt_cfl(u, 0.1), 20)
    np.testing.assert_allclose(ctx.reduce()[:5], sol.integrals(u), rtol=1e-12, atol=1e-9)


def test_boundary_layer_rk45_fixed_steps():
    """A small boundary-layer box (Navier-Stokes, p = 3, wall and far field):
    3 RK45[2R+] steps."""
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = make_pair(m, 3, **bl_params(mu=0.01))
    u = state(sol, "bl")
    _fixed_steps(sol, ctx, u, 0.2 * sol.dt_cfl(u, 0.1), 3)


def test_hex_prism_rk45_fixed_steps():
    """Hexahedra beside prism pairs (Navier-Stokes, p = 2): 4 steps."""
    m = synth.hex_box(n=4, n_hex_cols=2)
    sol, ctx = make_pair(m, 2, viscous=True, mu=0.02)
    u = state(sol, "smooth", seed=4)
    _fixed_steps(sol, ctx, u, sol.dt_cfl(u, 0.1), 4)


def test_vortex_rk45_adaptive_matches_the_oracle_controller():
    """Error-controlled steps over a fixed span, from a first step far
    above the tolerance's size: the same accepted/rejected sequence, the
    same next step size and the same final state as the oracle's driver."""
    sol, ctx = make_pair(synth.vortex_box(), 2)
    u = state(sol, "vortex")
    dt0 = sol.dt_cfl(u, 0.1)
    span, atol, rtol = 12 * dt0, 1e-7, 1e-7
    ctx.set_state(u)
    dt_got, acc, rej = ctx.step_rk45_adaptive(span, 8 * dt0, atol, rtol)
    ref, dt_ref, acc_ref, rej_ref = sol.rk45_adaptive(u, span, 8 * dt0, atol, rtol)
    assert (acc, rej) == (acc_ref, rej_ref)
    assert rej >= 1
    np.testing.assert_allclose(dt_got, dt_ref, rtol=1e-6)
    err = per_quantity_rel_err(sol, ref, ctx.get_state())
    assert np.all(err <= TOL), err


@pytest.mark.parametrize("prec", ["FR_FP32", "FR_BF16X3", "FR_TF32X3"])
def test_reduced_precision_rk45_state_error(prec):
    """20 RK45[2R+] steps of the vortex with the RHS in reduced precision
    (FP64 registers): the state increment against the FP64 oracle's, at the
    tolerance of the RK4 tests in the same precisions."""
    from paper_1409_0405_gb300 import fr
    sol, ctx = make_pair(synth.vortex_box(), 2, precision=getattr(fr, prec))
    u0 = state(sol, "vortex")
    dt = sol.dt_cfl(u0, 0.1)
    ctx.set_state(u0)
    ctx.step_rk45(dt, 20)
    got = ctx.get_state()
    ref = u0
    for _ in range(20):
        ref, _ = sol.rk45_step(ref, dt)
    err = per_quantity_rel_err(sol, ref - u0, got - u0)
    print(prec, "20-step increment error:", err)
    assert np.all(err <= (1e-4 if prec != "FR_BF16X3" else 2e-3)), err
    ctx.reduce()   # raises on a tensor-core wait that gave up


def test_rk45_queries_before_a_step_are_rejected():
    """The error norm and register exist only after an RK45 step."""
    from paper_1409_0405_gb300 import fr
    sol, ctx = make_pair(synth.vortex_box(), 1)
    ctx.set_state(state(sol, "vortex"))
    with pytest.raises(fr.FRError) as ei:
        ctx.rk45_error(1e-6, 1e-6)
    assert ei.value.code == fr.FR_ERR_ARG
    with pytest.raises(fr.FRError):
        ctx.rk45_get_error()
    ctx.step_rk45(1e-4, 0)                    # no step: nothing allocated, no error
    with pytest.raises(fr.FRError):
        ctx.step_rk45_adaptive(1.0, 1e-3, 0.0, 0.0)   # atol + rtol must be positive
