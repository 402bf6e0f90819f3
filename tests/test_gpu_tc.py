"""GPU tests of the tensor-core modes FR_BF16X3 and FR_TF32X3: the operator
applications on tcgen05 (split BF16 / split TF32 with FP32 accumulation)
against the FP64 oracle and against the FR_FP32 mode, over both element
types, orders 1-4, Euler and Navier-Stokes, ragged column tiles, the RK
update and the full-size boundary-layer RHS."""
import numpy as np
import pytest

import synth
from tests import _cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# split BF16 keeps ~16 bits of each operand, split TF32 ~22; with the
# operators' cancellation the RHS error is a few 1e-5 (BF16X3) and a few
# 1e-6 (TF32X3, about the FP32 mode's) of its scale (measured); a layout or
# epilogue mistake gives O(1)
TOLS = {"bf16x3": 5e-4, "tf32x3": 5e-5}
TC_RHS_TOL = TOLS["bf16x3"]
MODES = ["bf16x3", "tf32x3"]


def _prec(fr, mode):
    return {"bf16x3": fr.FR_BF16X3, "tf32x3": fr.FR_TF32X3}[mode]


def _fr():
    _cases.library()
    from paper_1409_0405_gb300 import fr
    return fr


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("viscous", [False, True])
def test_tc_rhs_matches_oracle(p, viscous, mode):
    fr = _fr()
    mesh = synth.vortex_box(n=4, jitter=0.05, seed=0)
    prm = dict(viscous=viscous, mu=0.01 if viscous else 0.0, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0)
    sol, ctx = _cases.make_pair(mesh, p, precision=_prec(fr, mode), **prm)
    _, c32 = _cases.make_pair(mesh, p, precision=fr.FR_FP32, **prm)
    u = _cases.state(sol, "vortex")
    ref = sol.rhs(u)
    got = _cases.gpu_rhs(ctx, u)
    err = _cases.per_quantity_rel_err(sol, ref, got)
    e32 = _cases.per_quantity_rel_err(sol, ref, _cases.gpu_rhs(c32, u))
    print(p, viscous, mode, err, "fp32", e32)
    assert np.all(err < TOLS[mode]), err
    ctx.reduce(check=False)   # raises FR_ERR_TIMEOUT if a bounded wait of a kernel gave up


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("etypes", ["tet", "pri"])
def test_tc_single_type_ragged(etypes, mode):
    """One element type only, element counts that leave a ragged last tile."""
    fr = _fr()
    coords = [np.linspace(-5, 5, 4), np.linspace(-5, 5, 3), np.linspace(-5, 5, 4)]
    mesh = synth.layered_box(coords, 2, 3 if etypes == "pri" else 0, (True, True, True), jitter=0.05, seed=4)
    prm = dict(viscous=True, mu=0.01, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0)
    sol, ctx = _cases.make_pair(mesh, 3, precision=_prec(fr, mode), **prm)
    u = _cases.state(sol, "vortex")
    err = _cases.per_quantity_rel_err(sol, sol.rhs(u), _cases.gpu_rhs(ctx, u))
    assert np.all(err < TOLS[mode]), err


def test_tc_rk_step_matches_fp32_mode():
    """The RK update: one RK4 step in the tensor-core modes and FR_FP32
    against the oracle's step."""
    fr = _fr()
    mesh = synth.vortex_box(n=4, jitter=0.05, seed=0)
    prm = dict(viscous=True, mu=0.01, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0)
    sol, c16 = _cases.make_pair(mesh, 4, precision=fr.FR_BF16X3, **prm)
    _, ctf = _cases.make_pair(mesh, 4, precision=fr.FR_TF32X3, **prm)
    _, c32 = _cases.make_pair(mesh, 4, precision=fr.FR_FP32, **prm)
    u = _cases.state(sol, "vortex")
    dt = sol.dt_cfl(u, 0.1)
    ref = sol.rk4_step(u, dt)
    out = {}
    for name, c in (("bf16x3", c16), ("tf32x3", ctf), ("fp32", c32)):
        c.set_state(u)
        c.step(dt, 1)
        out[name] = c.get_state()
    inc = ref - u
    for name, got in out.items():
        err = _cases.per_quantity_rel_err(sol, inc, got - u)
        print(name, err)
        assert np.all(err < 5e-3), (name, err)


@pytest.mark.parametrize("mode", MODES)
def test_tc_full_size_boundary_layer(mode):
    """The benchmark workload (42.4 M DOF, p=4 NS with walls and far field):
    the tensor-core RHS against the FR_FP64 RHS of the library (which
    matches the FP64 oracle to 1e-12 at this size), per conserved quantity
    (mass, momentum vector, energy: max |d| / max |ref| each)."""
    fr = _fr()
    mesh = synth.boundary_layer_box()
    prm = _cases.bl_params()
    c64 = fr.Context(mesh, 4, **prm)
    c16 = fr.Context(mesh, 4, precision=_prec(fr, mode), **prm)
    xyz = c64.upts_points()
    q = synth.perturbed_freestream(xyz, seed=2, wall_delta=_cases.BL_DELTA)
    counts = [(c64.info["n_tet"], c64.info["nu_tet"]), (c64.info["n_pri"], c64.info["nu_pri"])]
    out, off = [], 0
    for ne, nu in counts:
        out.append(q[off:off + ne * nu].reshape(ne, nu, 5).transpose(0, 2, 1).reshape(-1))
        off += ne * nu
    u = torch.from_numpy(np.concatenate(out)).cuda()
    r64, r16 = torch.empty_like(u), torch.empty_like(u)
    c64.rhs(u.data_ptr(), r64.data_ptr())
    c16.rhs(u.data_ptr(), r16.data_ptr())
    torch.cuda.synchronize()
    a, b = r64.cpu().numpy(), r16.cpu().numpy()
    num, den, off = np.zeros(3), np.zeros(3), 0
    for ne, nu in counts:
        ra = a[off:off + ne * 5 * nu].reshape(ne, 5, nu)
        rb = b[off:off + ne * 5 * nu].reshape(ne, 5, nu)
        for k, sl in enumerate((slice(0, 1), slice(1, 4), slice(4, 5))):
            num[k] = max(num[k], float(np.max(np.linalg.norm(rb[:, sl] - ra[:, sl], axis=1))))
            den[k] = max(den[k], float(np.max(np.linalg.norm(ra[:, sl], axis=1))))
        off += ne * 5 * nu
    d = num / den
    print("full-size", mode, "rel err per quantity", d)
    assert np.all(d < TOLS[mode]), d
    c16.reduce(check=False)


@pytest.mark.parametrize("mode", MODES)
def test_tc_bounded_wait_timeout_is_reported(mode):
    """Failure detection without a GPU fault: the operator kernel launched
    with its state loads withheld lets every bounded wait run out (~2 s),
    takes its abort path and reports FR_ERR_TIMEOUT through the context
    status; the self-test checks that and clears it, and the same context
    then evaluates a correct RHS."""
    fr = _fr()
    mesh = synth.vortex_box(n=4, jitter=0.05, seed=0)
    prm = dict(viscous=True, mu=0.01, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0)
    sol, ctx = _cases.make_pair(mesh, 2, precision=_prec(fr, mode), **prm)
    u = _cases.state(sol, "vortex")
    ctx.set_state(u)
    ctx.selftest_wait_timeout()
    ref = sol.rhs(u)
    err = _cases.per_quantity_rel_err(sol, ref, _cases.gpu_rhs(ctx, u))
    assert np.all(err < TOLS[mode]), err
    ctx.reduce()  # the status is clear again
