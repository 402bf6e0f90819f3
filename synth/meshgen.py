"""Structured-then-split mixed hexahedron/prism/tetrahedron meshes with
seeded node jitter.

Every mesh is a logically structured box of hexahedral cells.  The cells of
the first ``n_prism_layers`` layers along ``layer_axis`` are each split into
two triangular prisms extruded along that axis, except those of the first
``n_hex_cols`` cell columns along the first base axis, which stay
hexahedra (they meet the prisms on vertical quad faces); the remaining cells
are each split into six Kuhn (Freudenthal) tetrahedra along the cell's
min-to-max diagonal (a mesh with hexahedra has no tetrahedral layers, since
a hexahedron's quad face cannot meet two tetrahedra conformingly).  The prism base quads are cut along the same min-to-max diagonal,
so every face is conforming, including the prism/tet transition and all
periodic wraps.  This stands in for the paper's mixed cylinder mesh
(prisms in the near-wall layer, tets in the far field; Sec. 3.3), which is
not available.

Vertex order conventions (the only conventions the mesh format carries):

* tet: vertices 0..3 map to reference vertices (-1,-1,-1), (1,-1,-1),
  (-1,1,-1), (-1,-1,1); local faces are the vertex triples in ``TET_FACES``.
* prism: vertices 0..2 form the bottom triangle (reference zeta=-1),
  vertices 3..5 the top triangle (zeta=+1), vertex a+3 above vertex a;
  local faces are the vertex lists in ``PRI_FACES`` (two triangles, then
  three quads).
* hex: vertices 0..3 the bottom face (reference zeta=-1) counter-clockwise
  from reference vertex (-1,-1,-1), vertex a+4 above vertex a; local faces
  are the vertex quadruples in ``HEX_FACES``.

Every element is emitted with positive orientation.

Returned meshes are dicts with
``xyz`` (n_nodes, 3) float64, ``tet`` (n_tet, 4) int64, ``pri`` (n_pri, 6)
int64, ``hex`` (n_hex, 8) int64, ``bface`` (n_bface, 4) int64 rows (etype, elem, local face, bc tag)
and ``period`` (3,) float64 (0 = axis not periodic).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

ETYPE_TET = 0
ETYPE_PRI = 1
ETYPE_HEX = 2
BC_WALL = 1        # no-slip isothermal wall
BC_FARFIELD = 2    # Riemann-invariant far field

TET_FACES = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
PRI_FACES = ((0, 1, 2), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5))
HEX_FACES = ((0, 1, 2, 3), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7),
             (4, 5, 6, 7))

# (a0, a1, a2) axis orders that are even permutations of (x, y, z), keyed by
# the layer axis a2; a base triangle counter-clockwise in (a0, a1) extruded
# along +a2 is then positively oriented.
_AXES = {2: (0, 1, 2), 1: (2, 0, 1), 0: (1, 2, 0)}


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def layered_box(coords, layer_axis, n_prism_layers, periodic, bcs=None,
                jitter=0.0, seed=0, n_hex_cols=0):
    """Build a mixed prism/tet box mesh.

    coords: three increasing 1-D arrays, the node coordinates along x, y, z.
    layer_axis: axis (0, 1, 2) of the prism extrusion; layers are counted
        from the low end of this axis.
    n_prism_layers: number of cell layers (from the low end) split into prisms.
    periodic: three bools.  A periodic axis has period coords[-1]-coords[0]
        and its last node plane is the translate of its first.
    bcs: dict {(axis, side): tag} for each non-periodic side (side 0 = low,
        1 = high).  Missing sides default to BC_FARFIELD.
    jitter: node jitter as a fraction of the local cell size per component;
        nodes on non-periodic boundaries are not moved, and periodic images
        move identically.
    seed: PCG64 seed of the jitter.
    n_hex_cols: the cells of the prism layers whose index along the first
        base axis is below this stay hexahedra (needs n_prism_layers equal
        to the number of cell layers).
    """
    bcs = dict(bcs or {})
    axes = _AXES[layer_axis]
    ax_coords = [np.asarray(coords[a], dtype=np.float64) for a in axes]
    ncell = [len(c) - 1 for c in ax_coords]
    nnode = [n + 1 for n in ncell]
    per = [bool(periodic[a]) for a in axes]
    if n_hex_cols > 0 and n_prism_layers < ncell[2]:
        raise ValueError("hexahedra need every cell layer in the prism/hex part")

    # node grid in (a0, a1, a2) order, id = (i2 * nn1 + i1) * nn0 + i0
    g0, g1, g2 = np.meshgrid(*ax_coords, indexing="ij")
    grid = np.stack([g0, g1, g2], axis=-1)          # (nn0, nn1, nn2, 3) in axis order

    if jitter > 0.0:
        rng = _rng(seed)
        amp = []
        for k in range(3):
            c = ax_coords[k]
            h = np.diff(c)
            left = np.concatenate([[h[-1] if per[k] else h[0]], h])
            right = np.concatenate([h, [h[0] if per[k] else h[-1]]])
            amp.append(jitter * np.minimum(left, right))
        jit = rng.uniform(-1.0, 1.0, size=grid.shape)
        for k in range(3):
            shape = [1, 1, 1]
            shape[k] = nnode[k]
            jit[..., k] *= amp[k].reshape(shape)
        for k in range(3):
            sl_last = [slice(None)] * 3
            sl_first = [slice(None)] * 3
            sl_last[k] = -1
            sl_first[k] = 0
            if per[k]:
                jit[tuple(sl_last)] = jit[tuple(sl_first)]
        for k in range(3):
            if not per[k]:
                for idx in (0, -1):
                    sl = [slice(None)] * 3
                    sl[k] = idx
                    jit[tuple(sl)] = 0.0
        grid = grid + jit

    # back to physical (x, y, z) component order
    xyz_axis = grid.reshape(-1, 3, order="F")       # id order: i0 fastest
    xyz = np.empty_like(xyz_axis)
    for k, a in enumerate(axes):
        xyz[:, a] = xyz_axis[:, k]

    def nid(i0, i1, i2):
        return (i2 * nnode[1] + i1) * nnode[0] + i0

    c0, c1, c2 = np.meshgrid(np.arange(ncell[0]), np.arange(ncell[1]),
                             np.arange(ncell[2]), indexing="ij")
    c0 = c0.ravel(order="F")
    c1 = c1.ravel(order="F")
    c2 = c2.ravel(order="F")
    is_hex_cell = (c2 < n_prism_layers) & (c0 < n_hex_cols)
    is_pri_cell = (c2 < n_prism_layers) & ~is_hex_cell

    hc0, hc1, hc2 = c0[is_hex_cell], c1[is_hex_cell], c2[is_hex_cell]
    hverts, hgidx = [], []
    for (d0, d1, d2) in ((0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                         (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)):
        hverts.append(nid(hc0 + d0, hc1 + d1, hc2 + d2))
        hgidx.append(np.stack([hc0 + d0, hc1 + d1, hc2 + d2], axis=-1))
    hexa = np.stack(hverts, axis=-1).reshape(-1, 8)
    hex_g = np.stack(hgidx, axis=1).reshape(-1, 8, 3)

    pri_list, pri_gidx = [], []
    tet_list, tet_gidx = [], []
    # prisms: base triangles cut along the (0,0)-(1,1) diagonal
    tris = (((0, 0), (1, 0), (1, 1)), ((0, 0), (1, 1), (0, 1)))
    pc0, pc1, pc2 = c0[is_pri_cell], c1[is_pri_cell], c2[is_pri_cell]
    for tri in tris:
        verts, gidx = [], []
        for d2 in (0, 1):
            for (d0, d1) in tri:
                verts.append(nid(pc0 + d0, pc1 + d1, pc2 + d2))
                gidx.append(np.stack([pc0 + d0, pc1 + d1, pc2 + d2], axis=-1))
        pri_list.append(np.stack(verts, axis=-1))
        pri_gidx.append(np.stack(gidx, axis=1))
    # Kuhn tets: monotone lattice paths from (0,0,0) to (1,1,1)
    is_tet_cell = c2 >= n_prism_layers
    tc0, tc1, tc2 = c0[is_tet_cell], c1[is_tet_cell], c2[is_tet_cell]
    for perm in itertools.permutations(range(3)):
        path = [np.zeros(3, dtype=np.int64)]
        for k in perm:
            nxt = path[-1].copy()
            nxt[k] += 1
            path.append(nxt)
        e1, e2, e3 = path[1] - path[0], path[2] - path[0], path[3] - path[0]
        if np.linalg.det(np.stack([e1, e2, e3]).astype(float)) < 0.0:
            path = [path[0], path[2], path[1], path[3]]
        verts, gidx = [], []
        for d in path:
            verts.append(nid(tc0 + d[0], tc1 + d[1], tc2 + d[2]))
            gidx.append(np.stack([tc0 + d[0], tc1 + d[1], tc2 + d[2]], axis=-1))
        tet_list.append(np.stack(verts, axis=-1))
        tet_gidx.append(np.stack(gidx, axis=1))

    # interleave the pieces of each cell so that element order follows cells
    pri = (np.stack(pri_list, axis=1).reshape(-1, 6) if pri_list
           else np.zeros((0, 6), np.int64))
    pri_g = (np.stack(pri_gidx, axis=1).reshape(-1, 6, 3) if pri_gidx
             else np.zeros((0, 6, 3), np.int64))
    tet = (np.stack(tet_list, axis=1).reshape(-1, 4) if tet_list
           else np.zeros((0, 4), np.int64))
    tet_g = (np.stack(tet_gidx, axis=1).reshape(-1, 4, 3) if tet_gidx
             else np.zeros((0, 4, 3), np.int64))

    # boundary faces on non-periodic sides
    bface = []
    for etype, conn_g, faces in ((ETYPE_TET, tet_g, TET_FACES),
                                 (ETYPE_PRI, pri_g, PRI_FACES),
                                 (ETYPE_HEX, hex_g, HEX_FACES)):
        if len(conn_g) == 0:
            continue
        for lf, fv in enumerate(faces):
            fg = conn_g[:, list(fv), :]          # (ne, nfv, 3) grid indices
            for k in range(3):
                if per[k]:
                    continue
                for side, target in ((0, 0), (1, ncell[k])):
                    on = np.all(fg[:, :, k] == target, axis=1)
                    if np.any(on):
                        tag = bcs.get((axes[k], side), BC_FARFIELD)
                        el = np.nonzero(on)[0]
                        bface.append(np.stack([np.full_like(el, etype), el,
                                               np.full_like(el, lf),
                                               np.full_like(el, tag)], axis=-1))
    bface = (np.concatenate(bface).astype(np.int64) if bface
             else np.zeros((0, 4), np.int64))

    period = np.zeros(3)
    for k, a in enumerate(axes):
        if per[k]:
            period[a] = ax_coords[k][-1] - ax_coords[k][0]
    return {"xyz": np.ascontiguousarray(xyz), "tet": tet.astype(np.int64),
            "pri": pri.astype(np.int64), "hex": hexa.astype(np.int64), "bface": bface,
            "period": period}


def vortex_box(n=4, jitter=0.05, seed=0, n_prism_layers=None, lo=-5.0, hi=5.0):
    """Periodic cube [lo,hi]^3 of n^3 cells: lower half prisms, upper half
    Kuhn tets (the isentropic-vortex workload; 4^3 cells, seed 0 gives 64
    prisms and 192 tets)."""
    c = np.linspace(lo, hi, n + 1)
    npl = n // 2 if n_prism_layers is None else n_prism_layers
    return layered_box((c, c, c), 2, npl, (True, True, True), jitter=jitter,
                       seed=seed)


def boundary_layer_box(nx=75, nz=12, n_prism_layers=32, n_tet_layers=22,
                       h0=0.03208, ratio=1.1, lx=20.0, ly=20.0, lz=math.pi,
                       jitter=0.05, seed=1, all_hex=False):
    """Box [0,lx]x[0,ly]x[0,lz]: geometrically stretched prism layers on a
    no-slip wall at y=0 under uniform Kuhn-tet layers up to y=ly; far field
    at x=0, x=lx, y=ly; periodic in z.  The defaults give 57,600 prisms and
    118,800 tets.  all_hex: the same layers, every cell a hexahedron
    (nx=75, nz=29 gives 117,450 hexahedra)."""
    yb = h0 * (ratio ** np.arange(n_prism_layers + 1) - 1.0) / (ratio - 1.0)
    yt = np.linspace(yb[-1], ly, n_tet_layers + 1)[1:]
    y = np.concatenate([yb, yt])
    x = np.linspace(0.0, lx, nx + 1)
    z = np.linspace(0.0, lz, nz + 1)
    bcs = {(1, 0): BC_WALL, (1, 1): BC_FARFIELD, (0, 0): BC_FARFIELD,
           (0, 1): BC_FARFIELD}
    if all_hex:
        return layered_box((x, y, z), 1, len(y) - 1, (False, False, True), bcs=bcs,
                           jitter=jitter, seed=seed, n_hex_cols=nz)
    return layered_box((x, y, z), 1, n_prism_layers, (False, False, True),
                       bcs=bcs, jitter=jitter, seed=seed)


def wall_channel(nx=3, ny=3, nz=2, n_prism_layers=2, lx=2.0, ly=1.5, lz=1.0,
                 jitter=0.05, seed=4, n_hex_cols=0):
    """Box [0,lx]x[0,ly]x[0,lz] periodic in x and z with a no-slip wall at
    y=0 and far field at y=ly; the lowest n_prism_layers cell layers are
    prisms (extruded along y), the rest Kuhn tets; with n_hex_cols > 0
    (and n_prism_layers = ny) the first n_hex_cols cell columns along the
    first base axis (z) are hexahedra."""
    x = np.linspace(0.0, lx, nx + 1)
    y = np.linspace(0.0, ly, ny + 1)
    z = np.linspace(0.0, lz, nz + 1)
    bcs = {(1, 0): BC_WALL, (1, 1): BC_FARFIELD}
    return layered_box((x, y, z), 1, n_prism_layers, (True, False, True),
                       bcs=bcs, jitter=jitter, seed=seed, n_hex_cols=n_hex_cols)


def tgv_box(n=24, jitter=0.0, seed=0):
    """Periodic cube [0,2pi]^3 of n^3 cells, lower half prisms, upper half tets."""
    c = np.linspace(0.0, 2.0 * math.pi, n + 1)
    return layered_box((c, c, c), 2, n // 2, (True, True, True), jitter=jitter,
                       seed=seed)


def hex_box(n=4, n_hex_cols=None, jitter=0.05, seed=0, lo=-5.0, hi=5.0):
    """Periodic cube [lo,hi]^3 of n^3 cells extruded along z: the first
    n_hex_cols columns along x hexahedra (all of them by default), the rest
    prism pairs."""
    c = np.linspace(lo, hi, n + 1)
    nh = n if n_hex_cols is None else n_hex_cols
    return layered_box((c, c, c), 2, n, (True, True, True), jitter=jitter,
                       seed=seed, n_hex_cols=nh)


# Quadratic (curved) element node positions in reference coordinates: the
# vertices, then (tet) the midpoints of edges (0,1), (0,2), (0,3), (1,2),
# (1,3), (2,3); (prism) three zeta levels -1, 0, 1 of the six triangle nodes
# (vertices 0, 1, 2, then midpoints of (0,1), (1,2), (2,0)); (hex) the
# 3 x 3 x 3 grid of {-1, 0, 1}, xi fastest.
_TRI6 = ((-1, -1), (1, -1), (-1, 1), (0, -1), (0, 0), (-1, 0))
QUAD_NODES = {
    "tet": ((-1, -1, -1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1),
            (0, -1, -1), (-1, 0, -1), (-1, -1, 0), (0, 0, -1), (0, -1, 0), (-1, 0, 0)),
    "pri": tuple((a, b, c) for c in (-1, 0, 1) for (a, b) in _TRI6),
    "hex": tuple((a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)),
}


def _linear_weights(etype, r):
    """Weights of the element's vertices at reference point r for its
    straight-sided (vertex) map."""
    xi, eta, zeta = r
    if etype == "tet":
        return np.array([-(1 + xi + eta + zeta) / 2, (1 + xi) / 2, (1 + eta) / 2, (1 + zeta) / 2])
    if etype == "pri":
        tau = np.array([-(xi + eta) / 2, (1 + xi) / 2, (1 + eta) / 2])
        return np.concatenate([tau * (1 - zeta) / 2, tau * (1 + zeta) / 2])
    sg = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                   [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)
    return np.prod(1.0 + sg * np.array([xi, eta, zeta]), axis=1) / 8.0


def curve_mesh(mesh, amp=0.1):
    """Quadratically curved version of a mesh: each element's quadratic
    nodes (QUAD_NODES) placed on the straight element and moved by the
    smooth map x -> x + d(x), d_i = amp (L_i / 2 pi) prod_k sin(2 pi (x_k -
    lo_k) / L_k), with L_k the period of a periodic axis (d is periodic, so
    periodic images still match) and the bounding-box extent of another (d
    vanishes on those boundary planes, which stay planar).  Vertex ids are
    kept for the topology.  Adds 'geom_order' = 2 and '<type>_nodes'
    (n, nq, 3) arrays."""
    xyz = np.asarray(mesh["xyz"], dtype=np.float64)
    lo, hi = xyz.min(0), xyz.max(0)
    per = np.asarray(mesh.get("period", np.zeros(3)), dtype=np.float64)
    L = np.where(per > 0, per, hi - lo)

    def phi(x):
        sk = np.sin(2.0 * math.pi * (x - lo) / L)
        return x + amp * (L / (2.0 * math.pi)) * np.prod(sk, axis=-1, keepdims=True)

    out = dict(mesh)
    out["geom_order"] = 2
    for t, nv in (("tet", 4), ("pri", 6), ("hex", 8)):
        conn = np.asarray(mesh.get(t, np.zeros((0, nv))), dtype=np.int64).reshape(-1, nv)
        W = np.array([_linear_weights(t, r) for r in QUAD_NODES[t]])        # (nq, nv)
        X = np.einsum("qv,evk->eqk", W, xyz[conn])
        out[t + "_nodes"] = phi(X)
    return out


def mesh_counts(mesh):
    return len(mesh["tet"]), len(mesh["pri"])


def batch_problem_params(i, seed=3, n_lo=1000, n_hi=80000):
    """Draw (n_elements, prism:tet ratio, order) of batched problem i:
    n log-uniform in [n_lo, n_hi], ratio = n_pri/n_tet uniform in [0, 1],
    order uniform in {1, 2, 3, 4}."""
    rng = _rng([seed, i])
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    r = float(rng.uniform(0.0, 1.0))
    p = int(rng.integers(1, 5))
    return n, r, p


def batch_problem_mesh(i, seed=3):
    """A periodic vortex box m x m x nz whose element count and prism:tet
    ratio approximate batch_problem_params(i): a layer of m^2 cells gives
    2 m^2 prisms or 6 m^2 tets, nz = kp + kt layers with kp/kt chosen so that
    2 kp / (6 kt) ~ r."""
    n, r, p = batch_problem_params(i, seed)
    # elements = m^2 (2 kp + 6 kt); pick kt, kp from the ratio, then m
    best = None
    for nz in range(2, 41):
        for kp in range(0, nz):
            kt = nz - kp
            rr = 2.0 * kp / (6.0 * kt)
            per_layer = 2 * kp + 6 * kt
            m = max(2, int(round(math.sqrt(n / per_layer))))
            ne = m * m * per_layer
            score = abs(math.log(ne / n)) + 2.0 * abs(rr - r)
            if best is None or score < best[0]:
                best = (score, m, kp, kt)
    _, m, kp, kt = best
    nz = kp + kt
    L = 10.0
    cxy = np.linspace(-L / 2, L / 2, m + 1)
    cz = np.linspace(-L / 2, L / 2, nz + 1)
    mesh = layered_box((cxy, cxy, cz), 2, kp, (True, True, True), jitter=0.05,
                       seed=1000 + i)
    return mesh, p
