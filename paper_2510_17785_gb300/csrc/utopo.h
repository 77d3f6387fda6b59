// Topology of an unstructured quadrilateral (d = 2) / hexahedral (d = 3)
// mesh on the host: entities, boundary, the global DoF numbering of the
// degree-q space, vertex patches and their colours.
//
// A cell is its 2^d vertex ids in lexicographic corner order (corner c at
// the reference point whose k-th coordinate is bit k of c); cells are
// multilinear images of [0,1]^d.  The boundary of the domain is the union of
// the facets (edges in 2D, faces in 3D) that belong to one cell only.
//
// DoF numbering of the degree-q space (the paper works with its library's
// numbering and fixes none; this is the one the library exports):
//   vertices by id; then edges sorted by (smaller id, larger id), q - 1 nodes
//   each, numbered from the end with the smaller vertex id; then (3D) faces
//   sorted by their sorted vertex ids, (q - 1)^2 nodes in the frame of the
//   face's smallest-id corner (first axis toward the smaller-id of its two
//   face neighbours, first axis fastest); then cells by id, (q - 1)^d nodes in
//   the cell's reference frame, x fastest.
//
// Patches (Section 2.1): one per interior vertex, in increasing vertex id:
// the cells containing the vertex.  Colours: two patches conflict when they
// share a cell; vertices are taken in decreasing priority
// (splitmix64(id ^ seed), id) and each gets the smallest colour that no
// conflicting, already coloured patch has.  Patches of one colour share no
// cell, so their interiors are disjoint.
#pragma once
#include <stdint.h>

#include <array>
#include <map>
#include <string>
#include <vector>

namespace pmg {

struct UTopo {
  int dim = 0;
  int64_t nv = 0, nc = 0;
  std::vector<int64_t> cells;                      // nc x 2^d
  std::vector<std::array<int64_t, 2>> edges;       // sorted keys
  std::vector<std::array<int64_t, 4>> faces;       // sorted keys (3D)
  std::map<std::array<int64_t, 2>, int64_t> edge_id;
  std::map<std::array<int64_t, 4>, int64_t> face_id;
  std::vector<std::vector<int64_t>> vertex_cells;  // cells containing each vertex, increasing
  std::vector<uint8_t> vertex_on_boundary;
  std::vector<uint8_t> edge_on_boundary, face_on_boundary;
};

// Builds the topology; vob (n_v flags) may be NULL (derived from the
// facets).  Returns "" or an error message (bad vertex ids, a facet shared by
// more than two cells, ...).
std::string utopo_build(int dim, int64_t nv, int64_t nc, const int64_t* cells, const uint8_t* vob, UTopo* t);

int64_t utopo_ndofs(const UTopo& t, int q);
// [nc][(q+1)^d] global DoF ids of every cell's nodes (local order lexicographic, x fastest)
std::vector<int32_t> utopo_cell_dofs(const UTopo& t, int q);
// 1 on the DoFs of boundary facets (with their edges and vertices)
std::vector<uint8_t> utopo_boundary_dofs(const UTopo& t, int q);
// interior vertices (patches), increasing id
std::vector<int64_t> utopo_patch_vertices(const UTopo& t);
// colour of every patch (same order as utopo_patch_vertices)
std::vector<uint8_t> utopo_colours(const UTopo& t, const std::vector<int64_t>& pverts, uint64_t seed, int* ncolours);

}  // namespace pmg
