// refelem.h -- host-side reference element of libfem (quadrature, Lagrange
// basis and the constant factors Q of the element product V = X Q).
#pragma once
#include <vector>

namespace fem {

struct RefElem {
    int d = 0, p = 0, qdeg = 0, nq = 0, np = 0, ns = 0, nsym = 0;
    std::vector<double> xq;    // nq x d
    std::vector<double> wq;    // nq, sum = 1/d!
    std::vector<double> phi;   // nq x np
    std::vector<double> grad;  // nq x np x d (the paper's J_q)
    std::vector<double> QM;    // (nq) x nsym              (Section 4.1, Phi (.) Phi, symmetric rows)
    std::vector<double> QK;    // (nq*ns) x nsym           (Section 4.2, [J_q (x) J_q], symmetric)
    std::vector<double> QT;    // (nq*d) x np^2            (Section 5.2 tensor o_2 u)
};

// Boundary facets of an element type (Section 5: B_ik = int g_N'(u_h) phi_i
// phi_k dS over the boundary): face f is the face opposite local vertex f;
// its nodes are the element's local nodes whose barycentric multi-index is
// 0 at vertex f (in ascending local order).  Quadrature on the reference
// facet: Gauss-Legendre with p+1 points on [0, 1] (weights summing to 1)
// for the edges of triangles, the library's triangle rule of degree 2p
// (weights summing to 1/2) for the faces of tetrahedra; the facet's measure
// factor is then the edge length, resp. twice the face's area.
struct FacetTab {
    int d = 0, p = 0, nfaces = 0, nf = 0, nq = 0;   // faces, nodes per face, points
    std::vector<int> fnode;     // nfaces x nf element-local node indices
    std::vector<double> w;      // nq
    std::vector<double> phi;    // nfaces x nq x nf: the face nodes' basis values at the face points
};
bool build_facets(int d, int p, FacetTab& out);
const FacetTab* facets_for_type(int type);

// Builds the tables for (d, p) with the rule of degree qdeg (0 = 2p; only
// 2p is supported).  Returns false on unsupported input or if the rule
// solver does not reach 1e-14 moment residuals.
bool build_refelem(int d, int p, int qdeg, RefElem& out);

// Cached, thread-safe access by element type index 0..5 ((d-2)*3 + p-1).
const RefElem* refelem_for_type(int type);

}  // namespace fem
