"""Mesh bookkeeping of the oracle: geometry at solution and flux points,
face connectivity, periodic face matching and flux-point pairing.

Readings: faces of two elements that share their vertex set are neighbours;
faces listed as boundary faces carry a boundary tag; every other face must
be the periodic translate (by a combination of the mesh's period vectors) of
another such face, else the mesh is rejected.  Flux points of two matched
faces are paired by physical position (after the periodic shift).
Everything is indexed by a global flux-point id: tets first, element-major,
then prisms, then hexes.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.spatial import cKDTree

from . import basis, geometry

ETYPES = ("tet", "pri", "hex")


class MeshError(ValueError):
    pass


class Mesh:
    def __init__(self, m, p):
        self.p = p
        xyz = np.asarray(m["xyz"], dtype=np.float64)
        conn = {"tet": np.asarray(m["tet"], dtype=np.int64).reshape(-1, 4),
                "pri": np.asarray(m["pri"], dtype=np.int64).reshape(-1, 6),
                "hex": np.asarray(m.get("hex", np.zeros((0, 8))), dtype=np.int64).reshape(-1, 8)}
        self.period = np.asarray(m.get("period", np.zeros(3)), dtype=np.float64)
        bface = np.asarray(m.get("bface", np.zeros((0, 4))), dtype=np.int64).reshape(-1, 4)
        self.types = [t for t in ETYPES if len(conn[t]) > 0]
        self.ops = {t: basis.operators(t, p) for t in self.types}
        self.ne = {t: len(conn[t]) for t in self.types}
        self.conn = conn
        self.xyz = xyz
        bbox = xyz.max(0) - xyz.min(0)
        self.tol = 1e-7 * float(np.linalg.norm(bbox))

        # geometry
        self.X, self.upts_x, self.J, self.S = {}, {}, {}, {}
        self.fpts_x, self.fn, self.fmag = {}, {}, {}
        # quadratically curved elements: per-element node coordinates
        curved = int(m.get("geom_order", 1)) == 2
        for t in self.types:
            op = self.ops[t]
            if curved:
                X = np.asarray(m[t + "_nodes"], dtype=np.float64).reshape(
                    self.ne[t], len(geometry.QUAD_NODES[t]), 3)
            else:
                X = xyz[conn[t]]
            self.X[t] = X
            self.upts_x[t] = geometry.map_points(t, X, op.upts)
            J, S = geometry.metric(t, X, op.upts)
            if np.any(J <= 0.0):
                raise MeshError(f"non-positive Jacobian in a {t} element")
            self.J[t], self.S[t] = J, S
            self.fpts_x[t] = geometry.map_points(t, X, op.fpts)
            n, mag = geometry.face_normals(t, X, op.fpts, op.fnorm)
            self.fn[t], self.fmag[t] = n, mag

        # global flux-point numbering
        self.foff = {}
        off = 0
        for t in self.types:
            self.foff[t] = off
            off += self.ne[t] * self.ops[t].nf
        self.nfpts_total = off

        self._connect(bface)

    # ------------------------------------------------------------------
    def gid(self, t, e, f):
        return self.foff[t] + e * self.ops[t].nf + f

    def _face_fpts(self, t, lf):
        return np.nonzero(self.ops[t].fface == lf)[0]

    def _connect(self, bface):
        # all element faces
        recs = []          # (t, e, lf)
        keys = {}
        for t in self.types:
            op = self.ops[t]
            for lf, fv in enumerate(op.face_verts):
                vids = np.sort(self.conn[t][:, list(fv)], axis=1)
                for e in range(self.ne[t]):
                    k = tuple(vids[e])
                    keys.setdefault(k, []).append((t, e, lf))
                    recs.append((t, e, lf))
        pairs = []         # ((t,e,lf), (t,e,lf), shift)
        single = set()
        for k, lst in keys.items():
            if len(lst) == 2:
                pairs.append((lst[0], lst[1], np.zeros(3)))
            elif len(lst) == 1:
                single.add(lst[0])
            else:
                raise MeshError("a face is shared by more than two elements")

        self.bfaces = []   # ((t,e,lf), tag)
        for et, e, lf, tag in bface:
            t = ETYPES[int(et)]
            r = (t, int(e), int(lf))
            if r not in single:
                raise MeshError("boundary face is not a free face")
            single.discard(r)
            self.bfaces.append((r, int(tag)))

        # periodic matching of the remaining free faces by centroid
        free = sorted(single, key=lambda r: (ETYPES.index(r[0]), r[1], r[2]))
        if free:
            if not np.any(self.period > 0):
                raise MeshError("unmatched faces and no periodicity")
            cen = np.array([self.xyz[self.conn[t][e, list(self.ops[t].face_verts[lf])]].mean(0)
                            for (t, e, lf) in free])
            tree = cKDTree(cen)
            axes = [a for a in range(3) if self.period[a] > 0]
            shifts = []
            for ks in itertools.product((-1, 0, 1), repeat=len(axes)):
                if any(ks):
                    s = np.zeros(3)
                    for a, k in zip(axes, ks):
                        s[a] = k * self.period[a]
                    shifts.append(s)
            matched = {}
            for i, r in enumerate(free):
                if i in matched:
                    continue
                for s in shifts:
                    d, j = tree.query(cen[i] + s)
                    if d < self.tol and j != i and j not in matched:
                        matched[i] = j
                        matched[j] = i
                        pairs.append((r, free[j], s))
                        break
                else:
                    raise MeshError("a free face has no periodic partner")

        # pair flux points face by face
        A_t, A_e, A_f, B_t, B_e, B_f = [], [], [], [], [], []
        for (ra, rb, s) in pairs:
            (ta, ea, lfa), (tb, eb, lfb) = ra, rb
            ia = self._face_fpts(ta, lfa)
            ib = self._face_fpts(tb, lfb)
            if len(ia) != len(ib):
                raise MeshError("non-conforming face pair")
            xa = self.fpts_x[ta][ea, ia] + s
            xb = self.fpts_x[tb][eb, ib]
            dist = np.linalg.norm(xa[:, None, :] - xb[None, :, :], axis=-1)
            j = np.argmin(dist, axis=1)
            if dist[np.arange(len(ia)), j].max() > self.tol or len(set(j)) != len(j):
                raise MeshError("flux points of a face pair do not coincide")
            A_t += [ta] * len(ia)
            A_e += [ea] * len(ia)
            A_f += list(ia)
            B_t += [tb] * len(ia)
            B_e += [eb] * len(ia)
            B_f += list(ib[j])
        self.pa = np.array([self.gid(t, e, f) for t, e, f in zip(A_t, A_e, A_f)], dtype=np.int64)
        self.pb = np.array([self.gid(t, e, f) for t, e, f in zip(B_t, B_e, B_f)], dtype=np.int64)

        bt, bg = [], []
        for (t, e, lf), tag in self.bfaces:
            for f in self._face_fpts(t, lf):
                bg.append(self.gid(t, e, f))
                bt.append(tag)
        self.bg = np.array(bg, dtype=np.int64)
        self.btag = np.array(bt, dtype=np.int64)

        cover = np.zeros(self.nfpts_total, dtype=np.int64)
        np.add.at(cover, self.pa, 1)
        np.add.at(cover, self.pb, 1)
        np.add.at(cover, self.bg, 1)
        if not np.all(cover == 1):
            raise MeshError("flux points not covered exactly once")

        # per-flux-point geometry in global numbering
        self.gn = np.concatenate([self.fn[t].reshape(-1, 3) for t in self.types])
        self.gmag = np.concatenate([self.fmag[t].reshape(-1) for t in self.types])

    # ------------------------------------------------------------------
    def to_global(self, arrs):
        """per-type (ne, k, nf) arrays -> (nfpts_total, k)."""
        return np.concatenate([arrs[t].transpose(0, 2, 1).reshape(-1, arrs[t].shape[1])
                               for t in self.types])

    def from_global(self, g):
        out = {}
        for t in self.types:
            nf = self.ops[t].nf
            blk = g[self.foff[t]:self.foff[t] + self.ne[t] * nf]
            out[t] = blk.reshape(self.ne[t], nf, -1).transpose(0, 2, 1)
        return out
