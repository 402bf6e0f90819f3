// Mesh partitioning for the partitioned engine (host only).
//
// Sec. 5.2 partitions a mixed mesh with per-type weights
// hex : pri : tet = 3 : 2 : 1 (the relative cost of an element), and warns
// against partitions holding only a handful (fewer than about a thousand)
// elements of a type.  The paper hands the weighted graph to METIS or
// SCOTCH; here the partition is a weighted recursive coordinate bisection
// of the element centroids (no graph library in this build): split along
// the longest extent of the current set at the weighted median, giving each
// side a share of the weight proportional to its number of partitions.
// The paper's other rule, no partition with only a few elements of a type,
// is honoured where the mesh allows: a split that would leave a side with
// more than none but fewer than kMinPerType elements of a type per partition
// it will hold is moved to the nearest position (within 5% of the side's
// weight) where every type is either absent or at that minimum.
//
// Sec. 2.5: ranks exchange the interface data of their partitions; the
// exchange does not depend on the backend.  The plan built here is that
// exchange: for every pair of partitions (Q, P) sharing faces, the flux
// points of Q that P needs (Q's "send list" to P) in the order of the
// global interface pairs, landing in a contiguous range of P's halo slots
// (source partitions in increasing order).  Every cut interface pair is
// kept by both partitions with its global data (side a's normal, both
// magnitudes, the LDG switch), its remote side renamed (HALO, 0, slot), so
// a partition computes the same common values as the unpartitioned mesh.
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "fr_part.h"

namespace fr {
namespace {

constexpr int64_t kMinPerType = 1000;  // elements of a type per partition (Sec. 5.2)

struct Item {
    int t;
    int64_t e;
    double w;
    double x[3];
};

void rcb(std::vector<Item> &it, size_t b, size_t e, int nparts, int base, std::vector<std::vector<int32_t>> &out) {
    if (nparts <= 1 || e - b <= 1) {
        for (size_t i = b; i < e; ++i) out[it[i].t][it[i].e] = base;
        return;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    double wtot = 0.0;
    for (size_t i = b; i < e; ++i) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], it[i].x[k]);
            hi[k] = std::max(hi[k], it[i].x[k]);
        }
        wtot += it[i].w;
    }
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (hi[k] - lo[k] > hi[ax] - lo[ax]) ax = k;
    std::sort(it.begin() + b, it.begin() + e, [ax](const Item &p, const Item &q) {
        if (p.x[ax] != q.x[ax]) return p.x[ax] < q.x[ax];
        if (p.t != q.t) return p.t < q.t;
        return p.e < q.e;
    });
    const int nl = nparts / 2;
    const double target = wtot * nl / nparts;
    // first split index whose prefix weight reaches the target, or the one
    // before it if that lands closer; every side keeps at least one element
    double acc = 0.0;
    size_t m = b;
    while (m < e && acc + it[m].w < target) acc += it[m++].w;
    if (m < e && std::fabs(acc + it[m].w - target) < std::fabs(acc - target)) ++m;
    m = std::max(m, b + 1);
    m = std::min(m, e - 1);
    // per-type counts: the split is acceptable when every type is absent
    // from a side or present at kMinPerType per partition of that side
    int64_t tot[NT] = {0, 0, 0};
    for (size_t i = b; i < e; ++i) ++tot[it[i].t];
    auto ok = [&](const int64_t left[NT]) {
        for (int t = 0; t < NT; ++t) {
            const int64_t r = tot[t] - left[t];
            if ((left[t] > 0 && left[t] < kMinPerType * nl) || (r > 0 && r < kMinPerType * (nparts - nl)))
                return false;
        }
        return true;
    };
    int64_t left[NT] = {0, 0, 0};
    for (size_t i = b; i < m; ++i) ++left[it[i].t];
    if (!ok(left)) {
        int64_t cnt[NT] = {0, 0, 0};
        double w = 0.0, best = 0.05 * target;
        size_t mbest = 0;
        for (size_t i = b; i + 1 < e; ++i) {
            ++cnt[it[i].t];
            w += it[i].w;
            if (std::fabs(w - target) <= best && ok(cnt)) {
                best = std::fabs(w - target);
                mbest = i + 1;
            }
        }
        if (mbest) m = mbest;
    }
    rcb(it, b, m, nl, base, out);
    rcb(it, m, e, nparts - nl, base + nl, out);
}

}  // namespace

int partition_rcb(const fr_mesh *mesh, int nparts, const double w[NT], std::vector<int32_t> &part,
                  std::string &err) {
    const int64_t *conn[NT] = {mesh->tet, mesh->pri, mesh->hex};
    const int64_t ne[NT] = {mesh->n_tet, mesh->n_pri, mesh->n_hex};
    const int nvs[NT] = {4, 6, 8};
    std::vector<Item> it;
    for (int t = 0; t < NT; ++t)
        for (int64_t e = 0; e < ne[t]; ++e) {
            Item q{t, e, w[t], {0, 0, 0}};
            for (int a = 0; a < nvs[t]; ++a) {
                const int64_t v = conn[t][e * nvs[t] + a];
                if (v < 0 || v >= mesh->n_nodes) {
                    err = "element node id out of range";
                    return FR_ERR_MESH;
                }
                for (int k = 0; k < 3; ++k) q.x[k] += mesh->xyz[3 * v + k] / nvs[t];
            }
            it.push_back(q);
        }
    if ((int64_t)it.size() < nparts) {
        err = "fewer elements than partitions";
        return FR_ERR_ARG;
    }
    std::vector<std::vector<int32_t>> out(NT);
    for (int t = 0; t < NT; ++t) out[t].assign((size_t)ne[t], -1);
    rcb(it, 0, it.size(), nparts, 0, out);
    part.clear();
    for (int t = 0; t < NT; ++t) part.insert(part.end(), out[t].begin(), out[t].end());
    return FR_OK;
}

int build_part_plan(const HostSetup &h, int nparts, const int32_t *part, PartPlan &pl, std::string &err) {
    pl = PartPlan();
    pl.nparts = nparts;
    const int64_t ne[NT] = {h.geo[0].ne, h.geo[1].ne, h.geo[2].ne};
    // local numbering: a partition's elements of a type in increasing global order
    std::vector<int32_t> pof[NT];
    std::vector<int64_t> loc[NT];
    for (int t = 0; t < NT; ++t) pl.elems[t].assign(nparts, {});
    int64_t off = 0;
    for (int t = 0; t < NT; ++t) {
        pof[t].resize((size_t)ne[t]);
        loc[t].resize((size_t)ne[t]);
        for (int64_t e = 0; e < ne[t]; ++e) {
            const int32_t P = part[off + e];
            if (P < 0 || P >= nparts) {
                err = "partition index out of range";
                return FR_ERR_ARG;
            }
            pof[t][e] = P;
            loc[t][e] = (int64_t)pl.elems[t][P].size();
            pl.elems[t][P].push_back(e);
        }
        off += ne[t];
    }
    for (int P = 0; P < nparts; ++P) {
        int64_t n = 0;
        for (int t = 0; t < NT; ++t) n += (int64_t)pl.elems[t][P].size();
        if (n == 0) {
            err = "a partition has no elements";
            return FR_ERR_ARG;
        }
    }
    pl.local.assign(nparts, {});
    // geometry of each partition's elements
    for (int P = 0; P < nparts; ++P)
        for (int t = 0; t < NT; ++t) {
            const TypeGeo &G = h.geo[t];
            TypeGeo &L = pl.local[P].geo[t];
            const auto &el = pl.elems[t][P];
            L.ne = (int64_t)el.size();
            L.nu = G.nu;
            L.nf = G.nf;
            if (!L.ne) continue;
            auto take = [&](const std::vector<double> &src, std::vector<double> &dst, size_t per) {
                dst.resize(el.size() * per);
                for (size_t i = 0; i < el.size(); ++i)
                    std::copy(src.begin() + (size_t)el[i] * per, src.begin() + ((size_t)el[i] + 1) * per,
                              dst.begin() + i * per);
            };
            take(G.xu, L.xu, (size_t)G.nu * 3);
            take(G.S, L.S, (size_t)G.nu * 9);
            take(G.J, L.J, (size_t)G.nu);
            take(G.xf, L.xf, (size_t)G.nf * 3);
            take(G.fn, L.fn, (size_t)G.nf * 3);
            take(G.fmag, L.fmag, (size_t)G.nf);
        }
    // cut pairs per (destination, source), in global pair order
    const Faces &F = h.faces;
    const size_t npairs = F.ta.size();
    std::vector<std::vector<std::vector<int64_t>>> cut(nparts, std::vector<std::vector<int64_t>>(nparts));
    for (size_t k = 0; k < npairs; ++k) {
        const int Pa = pof[F.ta[k]][F.ea[k]], Pb = pof[F.tb[k]][F.eb[k]];
        if (Pa == Pb) continue;
        cut[Pa][Pb].push_back((int64_t)k);  // Pa receives side b from Pb
        cut[Pb][Pa].push_back((int64_t)k);  // Pb receives side a from Pa
    }
    // halo offsets: per destination, sources in increasing order
    std::vector<std::vector<int64_t>> hoff(nparts, std::vector<int64_t>(nparts, 0));
    for (int P = 0; P < nparts; ++P) {
        int64_t o = 0;
        for (int Q = 0; Q < nparts; ++Q) {
            hoff[P][Q] = o;
            o += (int64_t)cut[P][Q].size();
        }
        pl.local[P].nhalo = o;
    }
    // segments (source Q -> destination P): Q's own flux points
    for (int P = 0; P < nparts; ++P)
        for (int Q = 0; Q < nparts; ++Q) {
            if (cut[P][Q].empty()) continue;
            PartPlan::Seg sg;
            sg.src = Q;
            sg.dst = P;
            sg.off = hoff[P][Q];
            for (int64_t k : cut[P][Q]) {
                // the side of pair k that lies in Q
                const bool a_in_q = pof[F.ta[k]][F.ea[k]] == Q;
                const int t = a_in_q ? F.ta[k] : F.tb[k];
                const int f = a_in_q ? F.fa[k] : F.fb[k];
                const int64_t e = a_in_q ? F.ea[k] : F.eb[k];
                sg.t.push_back(t);
                sg.f.push_back(f);
                sg.e.push_back((int)loc[t][e]);
                sg.ge.push_back(e);
            }
            pl.segs.push_back(std::move(sg));
        }
    // each partition's pairs (global order) and boundary points
    std::vector<std::vector<int64_t>> pos(nparts, std::vector<int64_t>(nparts, 0));
    for (size_t k = 0; k < npairs; ++k) {
        const int Pa = pof[F.ta[k]][F.ea[k]], Pb = pof[F.tb[k]][F.eb[k]];
        for (int side = 0; side < 2; ++side) {
            const int P = side ? Pb : Pa;
            if (side && Pa == Pb) break;
            Faces &L = pl.local[P].faces;
            int ta = F.ta[k], fa = F.fa[k], tb = F.tb[k], fb = F.fb[k];
            int ea = (int)loc[ta][F.ea[k]], eb = (int)loc[tb][F.eb[k]];
            if (Pa != Pb) {
                const int Q = side ? Pa : Pb;  // the other partition
                const int slot = (int)(hoff[P][Q] + pos[P][Q]++);
                if (side) {
                    ta = HALO;
                    fa = 0;
                    ea = slot;
                } else {
                    tb = HALO;
                    fb = 0;
                    eb = slot;
                }
            }
            L.ta.push_back(ta);
            L.fa.push_back(fa);
            L.ea.push_back(ea);
            L.tb.push_back(tb);
            L.fb.push_back(fb);
            L.eb.push_back(eb);
            for (int c = 0; c < 3; ++c) L.n.push_back(F.n[3 * k + c]);
            L.maga.push_back(F.maga[k]);
            L.magb.push_back(F.magb[k]);
        }
    }
    for (size_t k = 0; k < F.bt.size(); ++k) {
        const int t = F.bt[k];
        const int P = pof[t][F.be[k]];
        Faces &L = pl.local[P].faces;
        L.bt.push_back(t);
        L.bf.push_back(F.bf[k]);
        L.be.push_back((int)loc[t][F.be[k]]);
        L.btag.push_back(F.btag[k]);
        for (int c = 0; c < 3; ++c) L.bn.push_back(F.bn[3 * k + c]);
        L.bmag.push_back(F.bmag[k]);
    }
    return FR_OK;
}

}  // namespace fr
