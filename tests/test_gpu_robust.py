"""Failure paths of the library that need no GPU fault (GPU).

Allocation failures are injected on the host: fr_debug_fail_alloc makes the
k-th device allocation fail as if the device were out of memory.  For every
k up to the number of allocations a creation makes, fr_create,
fr_batch_create and fr_part_create must return FR_ERR_NOMEM and free
everything they had taken (the library's live-allocation count returns to
its value before the call).
"""
import gc

import numpy as np
import pytest

import synth
from tests._cases import library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    library()
    yield
    from paper_1409_0405_gb300 import fr
    fr.debug_fail_alloc(0)


def _makers():
    from paper_1409_0405_gb300 import fr
    mesh = synth.vortex_box(n=2)
    ns = dict(viscous=True, mu=0.01)
    return {
        "context_fp64_ns": lambda: fr.Context(mesh, 2, **ns),
        "context_bf16x3_euler": lambda: fr.Context(mesh, 1, precision=fr.FR_BF16X3),
        "batch_fp32": lambda: fr.Batch([mesh, synth.hex_box(n=2)], [1, 2], precision=fr.FR_FP32),
        "partitioned_ns": lambda: fr.PartContext(mesh, 2, 3, **ns),
    }


@pytest.mark.parametrize("what", ["context_fp64_ns", "context_bf16x3_euler", "batch_fp32", "partitioned_ns"])
def test_every_allocation_failure_is_reported_and_leaks_nothing(what):
    from paper_1409_0405_gb300 import fr
    make = _makers()[what]
    fr.debug_fail_alloc(0)
    # objects of earlier tests that only the cycle collector frees would
    # otherwise release their allocations in the middle of the count
    gc.collect()
    live0 = fr.debug_alloc_stats()[1]
    obj = make()
    n, live = fr.debug_alloc_stats()
    assert n >= 5 and live > live0
    obj.close()
    del obj
    assert fr.debug_alloc_stats()[1] == live0
    for k in range(1, n + 1):
        fr.debug_fail_alloc(k)
        with pytest.raises(fr.FRError) as ei:
            make()
        assert ei.value.code == fr.FR_ERR_NOMEM, (k, str(ei.value))
        del ei
        gc.collect()
        assert fr.debug_alloc_stats()[1] == live0, k
    fr.debug_fail_alloc(0)
    obj = make()       # the library is still usable
    obj.close()


def test_step_reports_a_blown_up_state_on_the_next_call():
    """The state check that ends every stepping call: a time step far above
    the stability limit blows the vortex up; fr_check then reports
    FR_ERR_NONFINITE, the next fr_step refuses to run, and fr_set_state
    clears the condition."""
    from paper_1409_0405_gb300 import fr
    from tests._cases import make_pair, state
    sol, ctx = make_pair(synth.vortex_box(), 2)
    u = state(sol, "vortex")
    dt = sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 3)
    ctx.check()                                  # a healthy run passes
    ctx.step(400 * dt, 40)                       # unstable: overflows to inf / NaN
    with pytest.raises(fr.FRError) as ei:
        ctx.check()
    assert ei.value.code == fr.FR_ERR_NONFINITE
    with pytest.raises(fr.FRError) as ei:
        ctx.step(dt, 1)
    assert ei.value.code == fr.FR_ERR_NONFINITE
    with pytest.raises(fr.FRError) as ei:
        ctx.step_rk45(dt, 1)
    assert ei.value.code == fr.FR_ERR_NONFINITE
    ctx.set_state(u)
    ctx.step(dt, 2)
    ctx.check()
    np.testing.assert_allclose(ctx.reduce()[:5], sol.integrals(u), rtol=1e-12, atol=1e-9)


def test_step_reports_a_planted_nonphysical_point():
    """A host-built state with one negative density: the first step call
    runs, its state check sets the flag, and once that call has completed
    on the device the next call refuses (the flag is read without a
    synchronisation, so the test waits for the device first)."""
    import torch
    from paper_1409_0405_gb300 import fr
    from tests._cases import make_pair, state
    sol, ctx = make_pair(synth.vortex_box(), 1)
    u = state(sol, "vortex")
    bad = u.copy()
    bad[0] = -1.0
    ctx.set_state(bad)
    ctx.step(1e-4, 1)
    torch.cuda.synchronize()
    with pytest.raises(fr.FRError) as ei:
        ctx.step(1e-4, 1)
    assert ei.value.code == fr.FR_ERR_NONFINITE


def test_state_copies_through_mapped_pinned_buffers():
    """fr_set_state / fr_get_state read and write a mapped page-locked host
    buffer in place (the layout kernel accesses it over the CPU-GPU link)
    and copy any other host buffer through device memory: both give the
    same state bit for bit, on tets + prisms and on a hex mesh, and a step
    from either is the same."""
    import torch
    from paper_1409_0405_gb300 import fr
    for mesh, p in ((synth.vortex_box(n=3, n_prism_layers=1), 3), (synth.hex_box(n=2, n_hex_cols=1), 2)):
        ctx = fr.Context(mesh, p, viscous=True, mu=0.01)
        rng = np.random.default_rng(5)
        u = np.empty(ctx.ndof)
        off = 0
        for ne, nu in ctx.counts():
            blk = np.tile(np.array([1.0, 0.3, -0.2, 0.1, 3.0])[None, :, None], (ne, 1, nu))
            u[off:off + blk.size] = (blk * (1.0 + 0.01 * rng.normal(size=blk.shape))).reshape(-1)
            off += blk.size
        pin_in = torch.from_numpy(u.copy()).pin_memory()
        pin_out = torch.zeros(ctx.ndof, dtype=torch.float64).pin_memory()
        ctx.set_state(pin_in.numpy())
        got_pinned = ctx.get_state(out=pin_out.numpy()).copy()
        assert np.array_equal(got_pinned, u)
        ctx.set_state(u)
        assert np.array_equal(ctx.get_state(), u)
        ctx.step(1e-3, 1)
        after_pageable = ctx.get_state()
        ctx.set_state(pin_in.numpy())
        ctx.step(1e-3, 1)
        after_pinned = ctx.get_state(out=pin_out.numpy()).copy()
        assert np.array_equal(after_pinned, after_pageable)
        ctx.close()
