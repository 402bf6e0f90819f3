"""The batched engine against the per-problem launch sequence (bit for bit)
and against the FP64 oracle, in both of its schedules: one persistent
cooperative launch per RK stage (phases separated by grid barriers with
bounded waits), and one grouped launch per operator class; both replayed
from a CUDA graph.  The barrier's bounded wait is exercised by withholding
one CTA (a reported timeout, no fault)."""
import numpy as np
import pytest

import synth
from tests._cases import library, per_quantity_rel_err
from oracle.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    library()


def _problems():
    # uneven sizes, mixes and orders (tets only, prisms only, mixed)
    return [(synth.vortex_box(n=3, n_prism_layers=1, seed=11), 1),
            (synth.vortex_box(n=4, n_prism_layers=0, seed=12), 3),
            (synth.vortex_box(n=2, n_prism_layers=2, seed=13), 4),
            (synth.vortex_box(n=5, n_prism_layers=3, seed=14), 2)]


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_per_problem(precision):
    from paper_1409_0405_gb300 import fr
    probs = _problems()
    b = fr.Batch([m for m, _ in probs], [p for _, p in probs], precision=precision)
    u0 = [c.upts_points() for c in b.problems]
    states = [np.ascontiguousarray(synth.isentropic_vortex(x)[:, :].reshape(-1, 5)) for x in u0]
    pub = []
    for c, q in zip(b.problems, states):
        blocks, off = [], 0
        for ne, nu in ((c.info["n_tet"], c.info["nu_tet"]), (c.info["n_pri"], c.info["nu_pri"])):
            if ne:
                blocks.append(q[off:off + ne * nu].reshape(ne, nu, 5).transpose(0, 2, 1).reshape(-1))
                off += ne * nu
        pub.append(np.concatenate(blocks))
    dts = [0.01, 0.02, 0.005, 0.01]

    def run(batched, nsteps=3):
        for c, u in zip(b.problems, pub):
            c.set_state(u)
        b.step(dts, nsteps, batched=batched)
        return [c.get_state() for c in b.problems]

    ref = run(False)
    got = run(True)                                   # one persistent launch per stage
    for r, g in zip(ref, got):
        np.testing.assert_array_equal(g, r)
    info = b.info()
    assert info["launches_batched"] == 4              # one per RK stage
    assert info["grid_stage"] > 0
    got_g = run(2)                                    # grouped launches per class
    for r, g in zip(ref, got_g):
        np.testing.assert_array_equal(g, r)
    info = b.info()
    assert info["launches_batched"] == info["launches_grouped"] == 4 * 4   # Euler: M0, flux, common flux, div
    # per problem and stage (Euler): per type M0, flux, div (FP32: and the
    # separate RK update), + 1 face kernel
    per_type = 3 + (precision == fr.FR_FP32)
    per = sum(4 * (per_type * ((c.info["n_tet"] > 0) + (c.info["n_pri"] > 0)) + 1) for c in b.problems)
    assert info["launches_per_problem"] == per > info["launches_grouped"]
    b.tune()
    for mode in (True, 2):
        got2 = run(mode)
        for r, g in zip(ref, got2):
            np.testing.assert_array_equal(g, r)
    b.check()
    b.close()


def test_batched_problem_against_oracle():
    from paper_1409_0405_gb300 import fr
    probs = _problems()
    b = fr.Batch([m for m, _ in probs], [p for _, p in probs], precision=fr.FR_FP32)
    i = 3
    mesh, p = probs[i]
    sol = Solver(mesh, p)
    u = sol.state_from_points(synth.isentropic_vortex(sol.upts_xyz_points()))
    dt = 0.1 * sol.dt_cfl(u, 1.0)
    # problem i carries the vortex; the others a uniform state at rest
    for j, c in enumerate(b.problems):
        c.set_state(u if j == i else _uniform_pub(c))
    dts = [dt] * len(probs)
    b.step(dts, 5, batched=True)
    got = b.problems[i].get_state()
    ref = u
    for _ in range(5):
        ref = sol.rk4_step(ref, dt)
    err = per_quantity_rel_err(sol, ref - u, got - u)
    assert np.all(err <= 1e-4), err
    b.close()


def _uniform_pub(c):
    out = []
    for ne, nu in ((c.info["n_tet"], c.info["nu_tet"]), (c.info["n_pri"], c.info["nu_pri"])):
        if ne:
            blk = np.zeros((ne, 5, nu))
            blk[:, 0] = 1.0
            blk[:, 4] = 2.5
            out.append(blk.reshape(-1))
    return np.concatenate(out)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_navier_stokes_equals_per_problem(precision):
    """Navier-Stokes batches (common solution, gradient, M0 on gradients in
    the grouped launches): bit-identical to each problem's own launches."""
    from paper_1409_0405_gb300 import fr
    probs = [(synth.vortex_box(n=3, n_prism_layers=1, seed=31), 2), (synth.hex_box(n=3, n_hex_cols=2, seed=32), 3),
             (synth.vortex_box(n=4, n_prism_layers=2, seed=33), 1)]
    prm = dict(viscous=True, mu=0.02, precision=precision, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0, rho_inf=1.0)
    states = []
    for batched in (False, True, 2):
        b = fr.Batch([m for m, _ in probs], [p for _, p in probs], **prm)
        for c in b.problems:
            q = synth.isentropic_vortex(c.upts_points())
            out, off = [], 0
            for ne, nu in c.counts():
                if ne:
                    out.append(q[off:off + ne * nu].reshape(ne, nu, 5).transpose(0, 2, 1).reshape(-1))
                    off += ne * nu
            c.set_state(np.concatenate(out))
        b.step([2e-3] * len(probs), 3, batched=batched)
        states.append([c.get_state() for c in b.problems])
        if batched is True:
            assert b.info()["launches_batched"] == 4
        b.check()
        b.close()
    for other in states[1:]:
        for a, g in zip(states[0], other):
            np.testing.assert_array_equal(g, a)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_navier_stokes_against_oracle(precision):
    """A Navier-Stokes batch in the persistent schedule against the FP64
    oracle: after 3 RK4 steps every problem's state matches the oracle's to
    1e-12 per quantity in FP64 (its change over the steps to 1e-10), and
    the change to 1e-4 with FP32 storage."""
    from paper_1409_0405_gb300 import fr
    probs = [(synth.vortex_box(n=3, n_prism_layers=1, seed=41), 2), (synth.vortex_box(n=2, n_prism_layers=2, seed=42), 3),
             (synth.vortex_box(n=3, n_prism_layers=0, seed=43), 1)]
    prm = dict(viscous=True, mu=0.02, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0, rho_inf=1.0)
    b = fr.Batch([m for m, _ in probs], [p for _, p in probs], precision=precision, **prm)
    sols, u0 = [], []
    for (mesh, p), c in zip(probs, b.problems):
        sol = Solver(mesh, p, **prm)
        u = sol.state_from_points(synth.isentropic_vortex(sol.upts_xyz_points()))
        c.set_state(u)
        sols.append(sol)
        u0.append(u)
    dt, nsteps = 2e-3, 3
    b.step([dt] * len(probs), nsteps, batched=True)
    assert b.info()["launches_batched"] == 4
    b.check()
    for sol, u, c in zip(sols, u0, b.problems):
        got = c.get_state()
        ref = u
        for _ in range(nsteps):
            ref = sol.rk4_step(ref, dt)
        inc = per_quantity_rel_err(sol, ref - u, got - u)
        if precision == 0:
            err = per_quantity_rel_err(sol, ref, got)
            assert np.all(err <= 1e-12), err
            assert np.all(inc <= 1e-10), inc
        else:
            assert np.all(inc <= 1e-4), inc
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_stage_barrier_timeout_is_reported_and_recovered(precision):
    """Failure detection of the persistent stage kernel: one CTA is withheld
    from the grid barriers, every other CTA's bounded wait (~2 s) runs out,
    the timeout is reported through fr_batch_check and cleared, and the
    batch then steps bit-identically to the per-problem launches."""
    from paper_1409_0405_gb300 import fr
    probs = _problems()
    b = fr.Batch([m for m, _ in probs], [p for _, p in probs], precision=precision)
    pub = [_uniform_pub(c) + 0.0 for c in b.problems]
    for c, u in zip(b.problems, pub):
        c.set_state(u)
    b.selftest_wait_timeout()
    b.check()                                          # the status was cleared
    q = [synth.isentropic_vortex(c.upts_points()) for c in b.problems]
    pub = []
    for c, x in zip(b.problems, q):
        out, off = [], 0
        for ne, nu in c.counts():
            if ne:
                out.append(x[off:off + ne * nu].reshape(ne, nu, 5).transpose(0, 2, 1).reshape(-1))
                off += ne * nu
        pub.append(np.concatenate(out))
    dts = [0.01, 0.02, 0.005, 0.01]
    res = []
    for batched in (False, True):
        for c, u in zip(b.problems, pub):
            c.set_state(u)
        b.step(dts, 2, batched=batched)
        res.append([c.get_state() for c in b.problems])
    for a, g in zip(*res):
        np.testing.assert_array_equal(g, a)
    b.check()
    b.close()
