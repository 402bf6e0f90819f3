"""Partitioned meshes on the CPU (no GPU): the weighted partitioner, the
exchange plan, and the plan's pack -> exchange -> unpack path across two
gloo ranks.

Sec. 5.2 weights a mixed mesh hex : pri : tet = 3 : 2 : 1; Sec. 2.5 has
the ranks of a partitioned mesh exchange interface data.  The plan comes
from the library's host code (fr_partition, fr_part_plan: the same code the
GPU partitions use); the values exchanged are the oracle's flux-point
states u_f = M0 u, so a rank's halo must hold exactly the oracle's values
at the remote sides of its cut interface pairs, which the oracle's own face
matching (independent of the library's) identifies.
"""
import os
import socket

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ETYPES = ("tet", "pri", "hex")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from tests._cases import library
    library()


def _bl():
    return synth.boundary_layer_box(nx=8, nz=3, n_prism_layers=4, n_tet_layers=3)


def _split(mesh, part):
    out, off = {}, 0
    for t in ETYPES:
        n = len(mesh.get(t, ()))
        out[t] = np.asarray(part[off:off + n])
        off += n
    return out


@pytest.mark.parametrize("nparts", [2, 3, 4, 5])
def test_partition_balances_the_paper_weights(nparts):
    """Every partition non-empty; the weighted load (tet 1, prism 2, hex 3)
    of each within two element weights of the ideal share; deterministic."""
    from paper_1409_0405_gb300 import fr
    m = _bl()
    part = fr.partition(m, nparts)
    assert np.array_equal(part, fr.partition(m, nparts))
    ps = _split(m, part)
    load = np.zeros(nparts)
    for t, w in zip(ETYPES, (1.0, 2.0, 3.0)):
        np.add.at(load, ps[t], w)
    assert part.min() == 0 and part.max() == nparts - 1
    ideal = load.sum() / nparts
    # recursive bisection rounds at every level: allow 2 prism weights per level
    assert np.max(np.abs(load - ideal)) <= 2 * 2.0 * np.ceil(np.log2(nparts)), (load, ideal)


def test_partition_respects_custom_weights_and_rejects_bad_input():
    from paper_1409_0405_gb300 import fr
    m = _bl()
    part = fr.partition(m, 2, weights=(1.0, 10.0, 3.0))
    ps = _split(m, part)
    load = np.zeros(2)
    np.add.at(load, ps["tet"], 1.0)
    np.add.at(load, ps["pri"], 10.0)
    assert abs(load[0] - load[1]) <= 10.0
    with pytest.raises(fr.FRError):
        fr.partition(m, 2, weights=(1.0, 0.0, 3.0))
    with pytest.raises(fr.FRError):
        fr.partition(m, len(m["tet"]) + len(m["pri"]) + 1)


def _cut_pairs(sol, part):
    """Oracle's interface flux-point pairs (global flux ids) whose sides lie
    in different partitions, as (type, element, flux point) per side."""
    m = sol.m
    ps = {t: v for t, v in _split({t: m.conn[t] for t in m.types}, part).items()}

    def side(g):
        for t in m.types:
            n = m.ne[t] * m.ops[t].nf
            if m.foff[t] <= g < m.foff[t] + n:
                e, f = divmod(g - m.foff[t], m.ops[t].nf)
                return t, int(e), int(f)
        raise AssertionError(g)

    out = []
    for ga, gb in zip(m.pa, m.pb):
        a, b = side(int(ga)), side(int(gb))
        if ps[a[0]][a[1]] != ps[b[0]][b[1]]:
            out.append((a, b))
    return out, ps


@pytest.mark.parametrize("nparts", [2, 3])
def test_plan_matches_the_oracles_cut_faces(nparts):
    """The plan's halo slots of every rank are exactly the remote sides of
    the oracle's cut flux-point pairs, each once; send and receive counts
    are symmetric."""
    from oracle.solver import Solver
    from paper_1409_0405_gb300 import fr
    m = _bl()
    sol = Solver(m, 2)
    part = fr.partition(m, nparts)
    cut, ps = _cut_pairs(sol, part)
    tid = {t: k for k, t in enumerate(ETYPES)}
    counts = {}
    for r in range(nparts):
        c, send, halo = fr.part_plan(m, 2, part, r)
        counts[r] = c
        expect = set()
        for a, b in cut:
            for mine, other in ((a, b), (b, a)):
                if ps[mine[0]][mine[1]] == r:
                    expect.add((tid[other[0]], other[1], other[2]))
        got = [tuple(int(x) for x in row) for row in halo]
        assert len(got) == len(set(got)) == len(expect)
        assert set(got) == expect
        # every sent point is one of this rank's own flux points
        for t, e, f in send:
            assert 0 <= e < int(np.sum(ps[ETYPES[t]] == r))
    for r in range(nparts):
        for q in range(nparts):
            assert counts[r][q] == counts[q][r]
        assert counts[r][r] == 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle.solver import Solver
    from paper_1409_0405_gb300 import fr
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = _bl()
        sol = Solver(m, 2)
        u = sol.split(sol.state_from_points(synth.random_smooth_state(sol.upts_xyz_points(), seed=9)))
        uf = {t: u[t] @ sol.m.ops[t].M0.T for t in sol.types}          # (ne, V, nf)
        part = fr.partition(m, world)
        ps = _split(m, part)
        mine = {t: np.nonzero(ps[t] == rank)[0] for t in sol.types}     # local -> global
        counts, send, halo = fr.part_plan(m, 2, part, rank)
        # pack: this rank's own flux points, grouped by destination
        vals = np.array([uf[ETYPES[t]][mine[ETYPES[t]][e], :, f] for t, e, f in send]).reshape(-1, 5)
        recv = np.zeros((int(counts.sum()), 5))
        off = 0
        reqs = []
        for q in range(world):
            n = int(counts[q])
            if q == rank or n == 0:
                continue
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(vals[off:off + n])), dst=q))
            off += n
        off = 0
        for q in range(world):
            n = int(counts[q])
            if q == rank or n == 0:
                continue
            buf = torch.zeros((n, 5), dtype=torch.float64)
            dist.recv(buf, src=q)
            recv[off:off + n] = buf.numpy()          # unpack: the halo is the receive buffer
            off += n
        for r_ in reqs:
            r_.wait()
        expect = np.array([uf[ETYPES[t]][e, :, f] for t, e, f in halo]).reshape(-1, 5)
        out.put((rank, int(counts.sum()), float(np.max(np.abs(recv - expect))) if len(expect) else 0.0))
    finally:
        dist.destroy_process_group()


def test_two_rank_halo_exchange_over_gloo():
    """Two CPU ranks pack their cut-face flux-point states by the plan,
    exchange them point to point, and find in their halo slots exactly the
    oracle's values of the remote sides (bitwise: the values are copied)."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, n, err in res:
        assert n > 0
        assert err == 0.0, (rank, err)


@pytest.mark.parametrize("nparts", [2, 3, 4, 8])
def test_partition_avoids_a_handful_of_elements_of_a_type(nparts):
    """Sec. 5.2: no partition should hold only a few (fewer than about a
    thousand) elements of a type, unless it holds none.  On the full
    boundary-layer workload (57,600 prisms + 118,800 tets) the partitioner
    meets that rule at 2..8 partitions within 2% of the weighted balance."""
    from paper_1409_0405_gb300 import fr
    m = synth.boundary_layer_box()
    part = fr.partition(m, nparts)
    ps = _split(m, part)
    load = np.zeros(nparts)
    for t, w in zip(ETYPES, (1.0, 2.0, 3.0)):
        cnt = np.bincount(ps[t], minlength=nparts) if len(ps[t]) else np.zeros(nparts, int)
        assert np.all((cnt == 0) | (cnt >= 1000)), (t, cnt)
        np.add.at(load, ps[t], w)
    assert load.max() / load.mean() - 1.0 < 0.02, load
