// Partitioned meshes (internal): the weighted partitioner and the exchange
// plan (host_part.cpp), shared by the partitioned engine (fr_part.cu) and
// the host-only plan query of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fr_internal.h"
#include "fr_kernels.h"

namespace fr {

struct PartPlan {
    int nparts = 0;
    // elems[t][P]: global ids of partition P's elements of type t, increasing
    // (its local numbering)
    std::vector<std::vector<int64_t>> elems[NT];
    // per partition: its elements' geometry, its interface pairs (cut pairs
    // with the remote side (HALO, 0, slot)) and boundary points, in the
    // global order, and its number of halo slots
    struct Local {
        TypeGeo geo[NT];
        Faces faces;
        int64_t nhalo = 0;
    };
    std::vector<Local> local;
    // exchange segment: source partition src sends the flux points
    // (t[i], f[i], local element e[i]) to partition dst, where they fill
    // halo slots off .. off + n - 1 in order; ge[i] is the global element
    struct Seg {
        int src = 0, dst = 0;
        int64_t off = 0;
        std::vector<int> t, f, e;
        std::vector<int64_t> ge;
    };
    std::vector<Seg> segs;
};

// weighted recursive coordinate bisection of the element centroids;
// part receives the partition of every element in public order (tets,
// prisms, hexes)
int partition_rcb(const fr_mesh *mesh, int nparts, const double w[NT], std::vector<int32_t> &part, std::string &err);
int build_part_plan(const HostSetup &h, int nparts, const int32_t *part, PartPlan &pl, std::string &err);

}  // namespace fr
