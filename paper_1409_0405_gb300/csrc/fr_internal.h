// Internal declarations shared by the host set-up code and the CUDA launch
// code of the FR engine.  Not part of the public ABI (see include/fr.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fr.h"

#ifndef FR_NT_DEFINED
#define FR_NT_DEFINED
namespace fr {
constexpr int NT = FR_NTYPES;  // element types: tet, prism, hex
}
#endif

namespace fr {

constexpr int NV = FR_NVARS;

// Host-side points and operators of one element type at one order.
struct RefOps {
    int etype = 0, p = 0, nu = 0, nf = 0, nfaces = 0;
    std::vector<double> upts;    // nu x 3 reference solution points
    std::vector<double> fpts;    // nf x 3 reference flux points
    std::vector<int> fface;      // nf, local face of each flux point
    std::vector<double> fnorm;   // nf x 3 outward unit reference normals
    std::vector<double> M0;      // nf x nu
    std::vector<double> D;       // (3 nu) x nu, rows (j, d)
    std::vector<double> M3;      // nu x nf
    std::vector<double> W;       // nu quadrature weights
    std::vector<double> FW;      // nf face weights: integral of each flux point's face Lagrange function
    std::vector<double> AGRAD;   // (3 nu) x (nu + nf)
    std::vector<double> ADIV;    // nu x (3 nu + nf): [M1 - M3 M2 | M3]
    std::vector<std::vector<int>> face_fpts;   // flux points of each face
    std::vector<std::vector<int>> face_verts;  // vertex ids of each face
};

int nupts_of(int etype, int p);
int nfpts_of(int etype, int p);
// Builds every operator of (etype, p).  Returns FR_OK or FR_ERR_ARG.
int build_ref_ops(int etype, int p, RefOps &out, std::string &err);

// Geometry of all elements of one type.
struct TypeGeo {
    int64_t ne = 0;
    int nu = 0, nf = 0;
    std::vector<double> xu;    // ne x nu x 3 physical solution points
    std::vector<double> S;     // ne x nu x 9, S[d][m] = J dxi_d/dx_m
    std::vector<double> J;     // ne x nu
    std::vector<double> xf;    // ne x nf x 3 physical flux points
    std::vector<double> fn;    // ne x nf x 3 physical unit outward normals
    std::vector<double> fmag;  // ne x nf, |S^T n^|
};

// Interface flux-point pairs and boundary flux points.
struct Faces {
    // pair k couples (ta, fa, ea) with (tb, fb, eb); n is side a's outward
    // unit normal; maga/magb are each side's |S^T n^|.
    std::vector<int> ta, fa, ea, tb, fb, eb;
    std::vector<double> n, maga, magb;
    // boundary point k: (bt, bf, be), tag, outward unit normal, magnitude
    std::vector<int> bt, bf, be, btag;
    std::vector<double> bn, bmag;
};

int build_geometry(const fr_mesh *mesh, const RefOps ops[NT], TypeGeo geo[NT],
                   std::string &err);
int build_faces(const fr_mesh *mesh, const RefOps ops[NT], const TypeGeo geo[NT],
                Faces &faces, std::string &err);

// host set-up of a mesh: operators of the types present, geometry, faces
struct HostSetup {
    RefOps ops[NT];
    TypeGeo geo[NT];
    Faces faces;
};

// L2 projection between the spaces of orders p_from and p_to on one
// reference element, as a matrix (nu_to x nu_from, row-major) on
// solution-point values.
int build_transfer(int etype, int p_from, int p_to, std::vector<double> &R, std::string &err);

// Gauss-Legendre nodes and weights on [-1, 1], ascending.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);

}  // namespace fr
