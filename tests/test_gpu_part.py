"""Partitioned meshes on the GPU (fr_part_*): the partitions of one mesh on
one device, exchanging cut-face flux-point states and gradients through
device-local halo buffers every RHS (GPU).

Every cut interface pair is computed by both partitions with the global
pair data, so in FP64 the partitioned RHS and RK4 states equal the
unpartitioned context's bit for bit; both are also checked against the
oracle at 1e-12 per conserved quantity.  Reductions differ only in their
summation order.
"""
import numpy as np
import pytest

import synth
from tests._cases import bl_params, library, make_pair, per_quantity_rel_err, state

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    library()


def _rhs(obj, u):
    import torch
    ut = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    rt = torch.full_like(ut, float("nan"))
    obj.rhs(ut.data_ptr(), rt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rt.cpu().numpy()


CASES = {
    "vortex_euler_p2": (lambda: synth.vortex_box(), 2, {}, "vortex"),
    "bl_ns_p3": (lambda: synth.boundary_layer_box(nx=8, nz=3, n_prism_layers=4, n_tet_layers=3), 3,
                 bl_params(mu=0.01), "bl"),
    "hexprism_ns_p2": (lambda: synth.hex_box(n=4, n_hex_cols=2), 2, dict(viscous=True, mu=0.02), "smooth"),
    "curved_ns_p3": (lambda: synth.curve_mesh(synth.vortex_box(n=3), amp=0.15), 3, dict(viscous=True, mu=0.02),
                     "smooth"),
}


@pytest.mark.parametrize("nparts", [2, 3, 4])
@pytest.mark.parametrize("case", sorted(CASES))
def test_partitioned_rhs_equals_unpartitioned_and_oracle(case, nparts):
    from paper_1409_0405_gb300 import fr
    mk, p, prm, kind = CASES[case]
    mesh = mk()
    sol, ctx = make_pair(mesh, p, **prm)
    u = state(sol, kind, seed=3)
    one = _rhs(ctx, u)
    pc = fr.PartContext(mesh, p, nparts, **prm)
    assert np.all(pc.info[:, :3].sum(axis=1) > 0) and np.all(pc.info[:, 3] > 0)
    got = _rhs(pc, u)
    assert np.array_equal(got, one), np.max(np.abs(got - one))
    err = per_quantity_rel_err(sol, sol.rhs(u), got)
    assert np.all(err <= TOL), err


@pytest.mark.parametrize("nparts", [2, 4])
def test_partitioned_rk4_steps_and_reductions(nparts):
    """3 RK4 steps of the Navier-Stokes boundary-layer box (wall, far field,
    periodic z): bitwise equal to the unpartitioned context, 1e-12 from the
    oracle; the summed reductions agree to rounding."""
    from paper_1409_0405_gb300 import fr
    mk, p, prm, kind = CASES["bl_ns_p3"]
    mesh = mk()
    sol, ctx = make_pair(mesh, p, **prm)
    u = state(sol, kind)
    dt = 0.2 * sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 3)
    pc = fr.PartContext(mesh, p, nparts, **prm)
    pc.set_state(u)
    assert np.array_equal(pc.get_state(), u)
    pc.step(dt, 3)
    got = pc.get_state()
    assert np.array_equal(got, ctx.get_state())
    ref = u
    for _ in range(3):
        ref = sol.rk4_step(ref, dt)
    err = per_quantity_rel_err(sol, ref, got)
    assert np.all(err <= TOL), err
    np.testing.assert_allclose(pc.reduce()[:6], ctx.reduce()[:6], rtol=1e-13)
    assert pc.launches() > 0


def test_explicit_partition_array_and_single_partition():
    """A caller-given partition (alternate element stripes, many cut faces)
    and the one-partition mesh (no halo) both reproduce the context."""
    from paper_1409_0405_gb300 import fr
    mk, p, prm, kind = CASES["vortex_euler_p2"]
    mesh = mk()
    sol, ctx = make_pair(mesh, p, **prm)
    u = state(sol, kind)
    one = _rhs(ctx, u)
    n = len(mesh["tet"]) + len(mesh["pri"])
    stripes = (np.arange(n) % 3).astype(np.int32)
    assert np.array_equal(_rhs(fr.PartContext(mesh, p, 3, part=stripes, **prm), u), one)
    single = fr.PartContext(mesh, p, 1, **prm)
    assert single.info[0, 3] == 0
    assert np.array_equal(_rhs(single, u), one)
    with pytest.raises(fr.FRError):
        fr.PartContext(mesh, p, 2, part=np.zeros(n, dtype=np.int32), **prm)   # an empty partition


@pytest.mark.parametrize("prec", ["FR_FP32", "FR_BF16X3", "FR_TF32X3"])
def test_partitioned_reduced_precision(prec):
    """The reduced-precision modes partitioned in 3: every point-wise and
    face value is computed from the same operands, so the RHS equals the
    unpartitioned one up to the operator kernels' column placement (equal
    in practice; bounded at the mode's own rounding here)."""
    from paper_1409_0405_gb300 import fr
    mk, p, prm, kind = CASES["bl_ns_p3"]
    mesh = mk()
    prm = dict(prm, precision=getattr(fr, prec))
    sol, ctx = make_pair(mesh, p, **prm)
    u = state(sol, kind)
    one = _rhs(ctx, u)
    pc = fr.PartContext(mesh, p, 3, **prm)
    got = _rhs(pc, u)
    print(prec, "bitwise equal:", bool(np.array_equal(got, one)))
    err = per_quantity_rel_err(sol, one, got)
    assert np.all(err <= 1e-6), err
    dt = 0.2 * sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    pc.set_state(u)
    ctx.step(dt, 2)
    pc.step(dt, 2)
    e2 = per_quantity_rel_err(sol, ctx.get_state() - u, pc.get_state() - u)
    assert np.all(e2 <= 1e-5), e2
    pc.reduce()
