// Host side of the far-field acceleration of the dense sum (the fast
// summation of K v inside GMRES, Sec. 2.5): the octree over the tube nodes'
// integer grid indices and the interaction lists of the target blocks.
// Plain C++ (no CUDA): every decision is integer arithmetic, so the tree and
// the lists are a pure function of the node indices and the parameters.
#pragma once

#include <stdint.h>

#include <vector>

namespace ctr {
namespace tree {

// Octree: a cell is the tight integer box [lo, hi) of its nodes; a cell of
// more than `leaf` nodes is split at mid = lo + (hi - lo) / 2 in every axis
// with hi - lo >= 2 into octants, taken in the order x-bit + 2 y-bit + 4 z-bit
// (empty ones dropped).  The leaves in depth-first order give the tree
// positions: perm[p] is the node at position p; a leaf lists its nodes by
// increasing index.  Cluster c covers the positions [begin[c], end[c]).
struct Octree {
    std::vector<int32_t> perm;
    std::vector<int32_t> begin, end;
    std::vector<int32_t> lo, hi;            // 3 per cluster
    std::vector<int32_t> child_ptr, child;  // children of c: child[child_ptr[c] .. child_ptr[c+1])
    int32_t n_clusters() const { return (int32_t)begin.size(); }
};

void build_octree(const int32_t* ijk, int64_t M, int leaf, Octree& t);

// theta as the integer tq of theta = tq / 1024, tq = floor(1024 theta + 1/2).
int theta_q(double theta);

// Separation of two node sets whose integer boxes, widened by g grid units,
// have doubled centres cB, cC and doubled squared half-diagonals R2B, R2C:
// theta |cB - cC| > rB + rC, decided exactly:
//   A = tq^2 D2 - 2^20 (R2B + R2C) > 0  and  A^2 > 2^42 R2B R2C.
bool separated(const int64_t cB[3], int64_t R2B, const int64_t cC[3], int64_t R2C, int tq);

// Doubled centre and squared doubled half-diagonal of [lo, hi) widened by g.
void widened(const int32_t lo[3], const int32_t hi[3], int g, int64_t c2[3], int64_t* R2);

// Interaction lists of the target blocks [I*BS, (I+1)*BS) of tree positions.
// From the root: a cluster that is well separated from the block and holds
// none of the block's excluded (correction) nodes is approximated when it
// has more than min_far nodes and summed directly otherwise; any other
// cluster is summed directly if it is a leaf and opened otherwise.  Direct
// position ranges are merged when adjacent.
struct Lists {
    int BS = 0;
    std::vector<int64_t> near_ptr;    // nb + 1
    std::vector<int32_t> near_rng;    // 2 per range: [begin, end) positions
    std::vector<int64_t> far_ptr;     // nb + 1
    std::vector<int32_t> far_cl;      // cluster ids
};

// excl_ptr / excl: for each node (original index) its excluded source nodes.
void interaction_lists(const Octree& t, const int32_t* ijk, const int32_t* excl_ptr, const int32_t* excl,
                       int BS, int tq, int64_t min_far, int g, Lists& L);

}  // namespace tree
}  // namespace ctr
